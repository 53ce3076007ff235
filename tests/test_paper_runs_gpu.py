"""The paper's 3D3V production set-ups (Sec. 5, Table 1) on the CUDA path.

All four runs of Table 1, TSI-0.1, TSI-0.3, WBI-0.04 and WBI-0.2 (the suffix
is dt), are run over the windows the paper fits its growth rates on
(0 <= t <= 2 for the two-stream, 0 <= t <= 1.6 for Weibel), from the growing
finite-grid eigenmodes of Eqs. two-stream-initial-fields and
weibel-initial-fields/particles.  The least-squares slope of the log mode
amplitude |f_k| / N_g must match the closed-form finite-grid rates
Gamma_TS = 9.109138040e-2 and Gamma_W = 5.103647904e-1 (the paper's own fits
are off by 7.95e-4 and 1.45e-3 for the two-stream, 1.07e-3 and 1.93e-3 for
Weibel), and the total energy must be conserved to the nonlinear tolerance
(Thm. energy; the paper reports <= 6.2e-12 over much longer runs).  The
two-stream fits also reproduce the rates the paper prints, 0.09101901 for
TSI-0.1 and 0.09095955 for TSI-0.3, to the printed digits.  The Weibel fits
land closer to Gamma_W than the paper's printed 0.510911239 and 0.511347526;
the paper does not state its loading in enough detail (positions of the 25
pairs in a cell) to reproduce those numbers.
"""
import math
import os

import numpy as np
import pytest

import pic_inputs
from tests._common import make_gpu

pytestmark = pytest.mark.gpu


def _golden(name):
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.txt")
    for line in open(path):
        if line.startswith(name + " "):
            return float(line.split()[1])
    raise KeyError(name)


def _spectral_deriv(f, axis, L):
    n = f.shape[axis]
    k = 2 * np.pi * np.fft.fftfreq(n, d=L / n)
    k[n // 2] = 0.0
    shape = [1, 1, 1]
    shape[axis] = n
    return np.real(np.fft.ifftn(1j * k.reshape(shape) * np.fft.fftn(f)))


def _fit(ts, amps):
    return np.polyfit(np.asarray(ts), np.log(np.asarray(amps)), 1)[0]


@pytest.mark.parametrize("dt,golden", [(0.1, "tsi01_fitted_rate"), (0.3, "tsi03_fitted_rate")])
def test_tsi_3d_growth_rate_and_energy(dt, golden):
    from oracle import closed_form as cf
    G = cf.two_stream_rate(0.25, 0.9, math.pi / 4)
    assert G == pytest.approx(9.109138040e-2, abs=1e-11)
    cfg = pic_inputs.two_stream_3d(eigen_rate=G, eigen_chi=cf.chi(0.25, math.pi / 4), dt=dt)
    s = make_gpu(cfg)
    s.start()
    n, L = 32, 8 * math.pi
    ts, amps, dE = [0.0], [], 0.0

    def mode():
        f = s.fields()
        phi = f["phi"].reshape(n, n, n)  # (z, y, x)
        Ex = -_spectral_deriv(phi, 2, L) - f["U"][: n ** 3].reshape(n, n, n)
        return abs(np.fft.fftn(Ex)[0, 0, 1]) / n ** 3

    amps.append(mode())
    for st in range(1, int(math.floor(2.0 / dt + 1e-9)) + 1):  # the fit window 0 <= t <= 2
        r = s.step(cfg["tol"])
        assert r["status"] == 0
        dE = max(dE, abs(r["rel_dE"]))
        ts.append(st * cfg["dt"])
        amps.append(mode())
    rate = _fit(ts, amps)
    print(f"TSI-{dt} 3D: fitted rate {rate:.8f} vs Gamma_TS {G:.8f} (rel {rate / G - 1:+.2e}), "
          f"paper {_golden(golden):.8f}, max |dE/E| {dE:.2e}, stats {s.stats()}")
    assert rate == pytest.approx(G, rel=3e-3)
    # the same fit reproduces the rate the paper prints (8 digits)
    assert rate == pytest.approx(_golden(golden), abs=2e-8)
    assert dE < 1e-11


@pytest.mark.parametrize("dt,golden", [(0.04, "wbi004_fitted_rate"), (0.2, "wbi02_fitted_rate")])
def test_wbi_3d_growth_rate_and_energy(dt, golden):
    from oracle import closed_form as cf
    G = cf.weibel_rate(1.0, 0.9, math.pi / 16)
    assert G == pytest.approx(5.103647904e-1, abs=1e-10)
    cfg = pic_inputs.weibel_3d(eigen_rate=G, eigen_chi=cf.chi(1.0, math.pi / 16), dt=dt)
    s = make_gpu(cfg, inner_tol_scale=0.1)  # Table 1: WBI inner tolerances 10x tighter
    s.start()
    n, L = 32, 2 * math.pi
    ts, amps, dE = [0.0], [], 0.0

    def mode():
        f = s.fields()
        A = f["A"].reshape(3, n, n, n)
        Bz = _spectral_deriv(A[1], 2, L) - _spectral_deriv(A[0], 1, L)
        return abs(np.fft.fftn(Bz)[0, 1, 0]) / n ** 3

    amps.append(mode())
    for st in range(1, int(math.floor(1.6 / dt + 1e-9)) + 1):  # the fit window 0 <= t <= 1.6
        r = s.step(cfg["tol"])
        assert r["status"] == 0
        dE = max(dE, abs(r["rel_dE"]))
        ts.append(st * cfg["dt"])
        amps.append(mode())
    rate = _fit(ts, amps)
    print(f"WBI-{dt} 3D: fitted rate {rate:.8f} vs Gamma_W {G:.8f} (rel {rate / G - 1:+.2e}), "
          f"paper {_golden(golden):.9f}, max |dE/E| {dE:.2e}, stats {s.stats()}")
    assert rate == pytest.approx(G, rel=3e-3)
    assert dE < 1e-11


def test_tsi01_through_the_first_saturation():
    """Sec. 5.1: TSI-0.1 from its eigenmode to t = 43.5, past the first
    large maximum of |E_x(k_x)| / N_g, which the paper prints as 0.25296 near
    t = 42.6.  The maximum's time and amplitude (within two units of the last
    printed digit) and energy conservation at the solver tolerance are
    checked; the particle-averaged inner iteration count of each step's final
    evaluation (the paper's run mean 3.267, maximum 6) and the outer counts
    are reported.  The shortened form of the full T = 60 run below."""
    from oracle import closed_form as cf
    G = cf.two_stream_rate(0.25, 0.9, math.pi / 4)
    cfg = pic_inputs.two_stream_3d(eigen_rate=G, eigen_chi=cf.chi(0.25, math.pi / 4))
    s = make_gpu(cfg)
    s.start()
    n, L = 32, 8 * math.pi

    def mode():
        f = s.fields()
        phi = f["phi"].reshape(n, n, n)
        Ex = -_spectral_deriv(phi, 2, L) - f["U"][: n ** 3].reshape(n, n, n)
        return abs(np.fft.fftn(Ex)[0, 0, 1]) / n ** 3

    ts, amps, outer, inner, inner_max, dE = [0.0], [mode()], [], [], 0, 0.0
    for st in range(1, 436):
        r = s.step(cfg["tol"])
        assert r["status"] == 0
        dE = max(dE, abs(r["rel_dE"]))
        outer.append(r["outer_iters"])
        inner.append(r["inner_mean"])
        inner_max = max(inner_max, r["inner_max"])
        ts.append(st * 0.1)
        amps.append(mode())
    amps = np.array(amps)
    i_max = int(np.argmax(amps))
    print(f"TSI-0.1 to t = 43.5: first maximum {amps[i_max]:.5f} at t = {ts[i_max]:.1f} "
          f"(paper 0.25296 near 42.6); inner iterations mean {np.mean(inner):.4f} max {inner_max}; "
          f"outer iterations mean {np.mean(outer):.3f} max {max(outer)}; max |dE/E| {dE:.2e}")
    assert abs(ts[i_max] - 42.6) <= 0.05
    assert abs(amps[i_max] - 0.25296) <= 2e-5
    assert dE < 1e-11
    s.close()


@pytest.mark.skipif(os.environ.get("PIC_LONG_RUNS") != "1",
                    reason="two 600-step 3D runs (about 3 minutes); set PIC_LONG_RUNS=1")
def test_tsi_nyquist_projection_on_off():
    """Sec. 5.3: TSI-0.1 to T = 60 with and without the Nyquist projector.
    The charge-weighted transverse RMS velocity (Eq. transverse-rms-results)
    stays near roundoff with projection (paper: 2.28724e-12; measured here
    2.78e-8) and grows to order one without it (paper: 0.366930; measured
    0.519).  The projected value grows from rounding noise that differs
    between transverse lines; the deposit's summation order is not its
    source (the deterministic deposit gives the same order of magnitude), so
    it is bounded, not matched."""
    from oracle import closed_form as cf
    G = cf.two_stream_rate(0.25, 0.9, math.pi / 4)
    out = {}
    for proj in (1, 0):
        cfg = pic_inputs.two_stream_3d(eigen_rate=G, eigen_chi=cf.chi(0.25, math.pi / 4))
        s = make_gpu(cfg, project_nyquist=proj)
        s.start()
        dE = 0.0
        for _ in range(600):
            r = s.step(cfg["tol"])
            assert r["status"] == 0
            dE = max(dE, abs(r["rel_dE"]))
        u = s.velocities()
        gam = np.sqrt(1.0 + np.sum(u * u, axis=0))
        v = u / gam
        wq = np.abs(cfg["w"])
        vperp = math.sqrt(np.sum(wq * (v[1] ** 2 + v[2] ** 2)) / np.sum(wq))
        vpar = math.sqrt(np.sum(wq * v[0] ** 2) / np.sum(wq))
        out[proj] = (vperp, vpar, dE)
        print(f"TSI-0.1 T=60 projection={proj}: v_perp_rms {vperp:.6e}, v_par_rms {vpar:.6f}, "
              f"max |dE/E| {dE:.2e}")
        s.close()
    assert out[1][0] < 1e-6
    assert out[0][0] > 0.1
    assert out[0][0] > 1e5 * out[1][0]
    assert out[1][2] < 1e-10 and out[0][2] < 1e-10


def test_tsi_nyquist_projection_contrast_to_t30():
    """Sec. 5.3: TSI-0.1 to t = 30 with and without the Nyquist projector
    (the first half of the T = 60 study above, run by default).  Without the
    projector the transverse Nyquist modes grow from rounding and the
    charge-weighted transverse RMS velocity (Eq. transverse-rms-results) has
    reached about 1.5e-7 by t = 30; with it, about 3e-12.  The contrast is
    what the test checks: more than four orders of magnitude, each run
    conserving energy to the nonlinear tolerance."""
    from oracle import closed_form as cf
    G = cf.two_stream_rate(0.25, 0.9, math.pi / 4)
    out = {}
    for proj in (1, 0):
        cfg = pic_inputs.two_stream_3d(eigen_rate=G, eigen_chi=cf.chi(0.25, math.pi / 4))
        s = make_gpu(cfg, project_nyquist=proj)
        s.start()
        dE = 0.0
        for _ in range(300):
            r = s.step(cfg["tol"])
            assert r["status"] == 0
            dE = max(dE, abs(r["rel_dE"]))
        u = s.velocities()
        v = u / np.sqrt(1.0 + np.sum(u * u, axis=0))
        wq = np.abs(cfg["w"])
        vperp = math.sqrt(np.sum(wq * (v[1] ** 2 + v[2] ** 2)) / np.sum(wq))
        out[proj] = (vperp, dE)
        print(f"TSI-0.1 t=30 projection={proj}: v_perp_rms {vperp:.3e}, max |dE/E| {dE:.1e}")
        s.close()
    assert out[1][0] < 1e-9
    assert out[0][0] > 1e-8
    assert out[0][0] > 1e4 * out[1][0]
    assert out[1][1] < 1e-10 and out[0][1] < 1e-10


@pytest.mark.skipif(os.environ.get("PIC_LONG_RUNS") != "1",
                    reason="two 600-step 3D runs (several minutes); set PIC_LONG_RUNS=1")
def test_tsi_shape_degree_comparison():
    """Sec. 5.3: TSI-0.1 to T = 60 with linear (r = 1) and quadratic (r = 2)
    shapes, projection on, the same convergence-triggered refinement policy
    (up to 2 levels: particle steps dt/2 and dt/4).  The paper finds that
    only the degree-one run needs refinement (first at t = 53.9); both
    conserve energy to the solver tolerance."""
    from oracle import closed_form as cf
    G = cf.two_stream_rate(0.25, 0.9, math.pi / 4)
    out = {}
    for order in (2, 1):
        cfg = pic_inputs.two_stream_3d(eigen_rate=G, eigen_chi=cf.chi(0.25, math.pi / 4))
        s = make_gpu(cfg, order=order, refine_max=2)
        s.start()
        dE, first, total = 0.0, None, 0
        for st in range(1, 601):
            r = s.step(cfg["tol"])
            assert r["status"] == 0, (order, st, r)
            dE = max(dE, abs(r["rel_dE"]))
            if r["refined"] and first is None:
                first = st * cfg["dt"]
            total += r["refined"]
        out[order] = (first, total, dE, s.stats())
        print(f"TSI-0.1 T=60 order={order}: first refinement at t={first}, refined particle "
              f"solves {total}, max |dE/E| {dE:.2e}")
        s.close()
    assert out[2][1] == 0  # quadratic shapes never need refinement
    assert out[2][2] < 1e-10 and out[1][2] < 1e-10


@pytest.mark.skipif(os.environ.get("PIC_LONG_RUNS") != "1",
                    reason="600- and 200-step 3D runs (about 3 minutes); set PIC_LONG_RUNS=1")
@pytest.mark.parametrize("dt,key", [(0.1, "tsi01"), (0.3, "tsi03")])
def test_tsi_full_run_matches_printed_diagnostics(dt, key):
    """Sec. 5.1 and Sec. 5.3: TSI-0.1 and TSI-0.3 to T = 60, against what the
    paper prints for these runs: the first large maximum of |E_x(k_x)| / N_g
    (0.25296 and 0.25141 near t = 42.6), the amplitude at T = 60 (0.0405932,
    0.0400176), the |q|-weighted longitudinal RMS velocity at T = 60
    (0.836845, 0.836425), each within two units of its last printed digit,
    and the energy error (printed <= 3.53e-12, 6.17e-12).  The mean (max)
    outer iterations per step are reported beside the printed 6.360 (11) and
    7.555 (10) and not bounded: they depend on solver details the paper does
    not pin down, while the fixed points, and with them every diagnostic
    above, do not."""
    from oracle import closed_form as cf
    printed = {"tsi01": dict(tmax=42.6, amax=0.25296, a60=0.0405932, vpar=0.836845,
                             outer=6.360, outer_max=11),
               "tsi03": dict(tmax=42.6, amax=0.25141, a60=0.0400176, vpar=0.836425,
                             outer=7.555, outer_max=10)}[key]
    G = cf.two_stream_rate(0.25, 0.9, math.pi / 4)
    cfg = pic_inputs.two_stream_3d(eigen_rate=G, eigen_chi=cf.chi(0.25, math.pi / 4), dt=dt)
    s = make_gpu(cfg)
    s.start()
    n, L = 32, 8 * math.pi

    def mode():
        f = s.fields()
        phi = f["phi"].reshape(n, n, n)
        Ex = -_spectral_deriv(phi, 2, L) - f["U"][: n ** 3].reshape(n, n, n)
        return abs(np.fft.fftn(Ex)[0, 0, 1]) / n ** 3

    nsteps = int(math.floor(60.0 / dt + 1e-9))
    ts, amps, outer, dE = [0.0], [mode()], [], 0.0
    for st in range(1, nsteps + 1):
        r = s.step(cfg["tol"])
        assert r["status"] == 0
        dE = max(dE, abs(r["rel_dE"]))
        outer.append(r["outer_iters"])
        ts.append(st * dt)
        amps.append(mode())
    amps = np.array(amps)
    i_max = int(np.argmax(amps))
    u = s.velocities()
    v = u / np.sqrt(1.0 + np.sum(u * u, axis=0))
    wq = np.abs(cfg["w"])
    vpar = math.sqrt(np.sum(wq * v[0] ** 2) / np.sum(wq))
    print(f"{key} T=60: first maximum {amps[i_max]:.5f} at t={ts[i_max]:.1f} "
          f"(paper {printed['amax']} near {printed['tmax']}), amplitude at T=60 {amps[-1]:.7f} "
          f"(paper {printed['a60']}), v_par,rms {vpar:.6f} (paper {printed['vpar']}), "
          f"outer iterations mean {np.mean(outer):.3f} max {max(outer)} "
          f"(paper {printed['outer']} ({printed['outer_max']})), max |dE/E| {dE:.2e}")
    assert abs(ts[i_max] - printed["tmax"]) <= 0.5 * dt
    assert abs(amps[i_max] - printed["amax"]) <= 2e-5
    assert abs(amps[-1] - printed["a60"]) <= 2e-7
    assert abs(vpar - printed["vpar"]) <= 2e-6
    assert dE < 1e-11


def test_wbi02_residuals_to_t20():
    """Sec. 5.2: WBI-0.2 to t = 20 (100 steps, the first fifth of the run
    below), with every step's Gauss and Lorenz RMS residuals, |dE/E|, the
    chain-rule residual R_A and the work residual within ten times the
    maxima the paper prints for the whole run (5.12e-13, 3.95e-14, 4.13e-13,
    5.57e-16, 1.31e-13), and the final-evaluation inner counts reported beside
    the paper's run mean 5.038 (maximum 8)."""
    from oracle import closed_form as cf
    G = cf.weibel_rate(1.0, 0.9, math.pi / 16)
    cfg = pic_inputs.weibel_3d(eigen_rate=G, eigen_chi=cf.chi(1.0, math.pi / 16), dt=0.2)
    s = make_gpu(cfg, inner_tol_scale=0.1)  # Table 1: WBI inner tolerances 10x tighter
    s.start()
    printed = dict(gauss=5.12e-13, lorenz=3.95e-14, dE=4.13e-13, chain=5.57e-16, work=1.31e-13)
    mx = dict(gauss=0.0, lorenz=0.0, dE=0.0, chain=0.0, work=0.0)
    inner, inner_max, outer = [], 0, []
    for _ in range(100):
        r = s.step(cfg["tol"])
        assert r["status"] == 0
        mx["gauss"] = max(mx["gauss"], r["gauss_rms"])
        mx["lorenz"] = max(mx["lorenz"], r["lorenz_rms"])
        mx["dE"] = max(mx["dE"], abs(r["rel_dE"]))
        mx["chain"] = max(mx["chain"], r["chain_rms"])
        mx["work"] = max(mx["work"], abs(r["work_residual"]))
        inner.append(r["inner_mean"])
        inner_max = max(inner_max, r["inner_max"])
        outer.append(r["outer_iters"])
    print("WBI-0.2 to t = 20: " + ", ".join(f"max {k} {v:.2e}" for k, v in mx.items())
          + f"; inner mean {np.mean(inner):.3f} max {inner_max}; outer mean {np.mean(outer):.3f}")
    for k, v in mx.items():
        assert v <= 10 * printed[k], k
    s.close()


@pytest.mark.skipif(os.environ.get("PIC_LONG_RUNS") != "1",
                    reason="2500- and 500-step 3D runs (WBI-0.04 alone about 30 minutes); "
                           "set PIC_LONG_RUNS=1")
@pytest.mark.parametrize("dt,key", [(0.04, "wbi004"), (0.2, "wbi02")])
def test_wbi_full_run_residuals(dt, key):
    """Sec. 5.2: WBI-0.04 and WBI-0.2 to T = 100.  The paper prints the
    maxima over the run of the Gauss RMS residual (1.22e-12, 5.12e-13), the
    Lorenz RMS residual (1.40e-13, 3.95e-14), |dE/E| (3.74e-14, 4.13e-13),
    the chain-rule RMS residual R_A (6.68e-16, 5.57e-16) and the work
    residual (1.44e-14, 1.31e-13).  The loading of the 25 pairs per cell is
    not stated in full, so the runs are not identical; each maximum must stay
    within ten times the printed one (the theorems behind them hold at the
    solver tolerance for any loading)."""
    from oracle import closed_form as cf
    printed = {"wbi004": dict(gauss=1.22e-12, lorenz=1.40e-13, dE=3.74e-14, chain=6.68e-16,
                              work=1.44e-14),
               "wbi02": dict(gauss=5.12e-13, lorenz=3.95e-14, dE=4.13e-13, chain=5.57e-16,
                             work=1.31e-13)}[key]
    G = cf.weibel_rate(1.0, 0.9, math.pi / 16)
    cfg = pic_inputs.weibel_3d(eigen_rate=G, eigen_chi=cf.chi(1.0, math.pi / 16), dt=dt)
    s = make_gpu(cfg, inner_tol_scale=0.1)  # Table 1: WBI inner tolerances 10x tighter
    s.start()
    mx = dict(gauss=0.0, lorenz=0.0, dE=0.0, chain=0.0, work=0.0)
    outer = []
    for _ in range(int(math.floor(100.0 / dt + 1e-9))):
        r = s.step(cfg["tol"])
        assert r["status"] == 0
        mx["gauss"] = max(mx["gauss"], r["gauss_rms"])
        mx["lorenz"] = max(mx["lorenz"], r["lorenz_rms"])
        mx["dE"] = max(mx["dE"], abs(r["rel_dE"]))
        mx["chain"] = max(mx["chain"], r["chain_rms"])
        mx["work"] = max(mx["work"], abs(r["work_residual"]))
        outer.append(r["outer_iters"])
    print(f"{key} T=100: " + ", ".join(f"max {k} {v:.2e} (paper {printed[k]:.2e})"
                                       for k, v in mx.items())
          + f"; outer iterations mean {np.mean(outer):.3f} max {max(outer)}")
    for k, v in mx.items():
        assert v <= 10 * printed[k], k


@pytest.mark.skipif(os.environ.get("PIC_LONG_RUNS") != "1",
                    reason="a 600-step 3D run with the deterministic deposit (about 3 minutes); "
                           "set PIC_LONG_RUNS=1")
def test_tsi_projected_transverse_velocity_with_deterministic_deposit():
    """Sec. 5.3: TSI-0.1 to T = 60 with the projector and the deterministic
    deposit.  The loading is the same in every transverse line, so the
    transverse modes are seeded only by rounding; the atomic deposit sums
    each node's contributions in a different order on every line, the
    deterministic one in the same order.  The transverse RMS velocity is
    reported beside the paper's 2.29e-12; it is bounded as in the projection
    study."""
    from oracle import closed_form as cf
    G = cf.two_stream_rate(0.25, 0.9, math.pi / 4)
    cfg = pic_inputs.two_stream_3d(eigen_rate=G, eigen_chi=cf.chi(0.25, math.pi / 4))
    s = make_gpu(cfg, deterministic_deposit=1)
    s.start()
    dE = 0.0
    for _ in range(600):
        r = s.step(cfg["tol"])
        assert r["status"] == 0
        dE = max(dE, abs(r["rel_dE"]))
    u = s.velocities()
    v = u / np.sqrt(1.0 + np.sum(u * u, axis=0))
    wq = np.abs(cfg["w"])
    vperp = math.sqrt(np.sum(wq * (v[1] ** 2 + v[2] ** 2)) / np.sum(wq))
    vpar = math.sqrt(np.sum(wq * v[0] ** 2) / np.sum(wq))
    print(f"TSI-0.1 T=60, deterministic deposit: v_perp,rms {vperp:.3e} (paper 2.29e-12), "
          f"v_par,rms {vpar:.6f} (paper 0.836845), max |dE/E| {dE:.2e}")
    assert vperp < 1e-6
    assert abs(vpar - 0.836845) <= 2e-6
    assert dE < 1e-11


def _stored_form_quiet_pairs(cfg, pairs=10):
    """The quiet start of two_stream_3d in stored form: node index and offset
    of every particle, the offsets of a sub-cell slot bit-identical in every
    cell (the same sub-cell positions the generator uses)."""
    k = np.arange(pairs)
    sub = np.stack([(k + 0.5) / pairs, (k * 0.6180339887498949 + 0.25) % 1.0,
                    (k * 0.7548776662466927 + 0.5) % 1.0])
    n = cfg["n"]
    ncell = n[0] * n[1] * n[2]
    ci = np.stack(np.unravel_index(np.repeat(np.arange(ncell), pairs), (n[2], n[1], n[0]))[::-1])
    kk = np.tile(k, ncell)
    cell = np.zeros(ci.shape, np.int32)
    off = np.zeros(ci.shape)
    for l in range(3):
        s_ = sub[l][kk]
        up = s_ >= 0.5
        cell[l] = (ci[l] + up) % n[l]
        off[l] = np.where(up, s_ - 1.0, s_)
    return np.concatenate([cell, cell], axis=1), np.concatenate([off, off], axis=1)


def test_tsi01_transverse_symmetry_is_exact_without_rounding_seeds():
    """Sec. 5.3: the projected TSI-0.1 run keeps its transverse symmetry to the
    rounding level when nothing breaks it between transverse lines: the
    particles loaded in stored form with bit-identical offsets in every cell
    (absolute coordinates round differently per cell) and the deterministic
    deposit (the atomic one sums each node in a different order).  Then
    v_perp,rms stays near 1e-17 through t = 20 (and 1.5e-16 at T = 60, below
    the paper's 2.29e-12), where the default loading and deposit have
    already grown it to 3e-14."""
    from oracle import closed_form as cf
    G = cf.two_stream_rate(0.25, 0.9, math.pi / 4)
    cfg = pic_inputs.two_stream_3d(eigen_rate=G, eigen_chi=cf.chi(0.25, math.pi / 4))
    import paper_2609_36383_b300 as pic
    s = pic.Simulation(3, cfg["n"], cfg["L"], cfg["x0"], cfg["species"], cfg["dt"],
                       rho_bg=cfg["rho_bg"], deterministic_deposit=1)
    cell, off = _stored_form_quiet_pairs(cfg)
    s.set_particles_local(cell, off, cfg["u"], cfg["w"], cfg["sp"])
    s.set_potentials(cfg["A"], cfg["U"])
    s.start()
    dE = 0.0
    for _ in range(200):
        r = s.step(cfg["tol"])
        assert r["status"] == 0
        dE = max(dE, abs(r["rel_dE"]))
    u = s.velocities()
    v = u / np.sqrt(1.0 + np.sum(u * u, axis=0))
    wq = np.abs(cfg["w"])
    vperp = math.sqrt(np.sum(wq * (v[1] ** 2 + v[2] ** 2)) / np.sum(wq))
    print(f"TSI-0.1 t = 20, bit-identical offsets and deterministic deposit: v_perp,rms {vperp:.2e}"
          f", max |dE/E| {dE:.1e}")
    assert vperp < 1e-15
    assert dE < 1e-11
    s.close()
