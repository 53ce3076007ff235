"""GPU parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (FP64 path):
- set-up and one map evaluation from identical state and trial current, with
  an inner tolerance of 1e-14 so that both sides converge the inner Picard
  iteration to roundoff: 1e-12 relative (the oracle uses 8 Gauss-Legendre
  points per knot-split piece, the kernels the minimal exact count, so both
  compute the exact orbit integrals and differ only by rounding);
- whole free-running steps at nonlinear tolerance 1e-12: both sides stop
  anywhere inside the tolerance ball of the same fixed point, so states agree
  to a few times the tolerance (1e-9 relative bound, stated in the test).
The mixed path (FP32 push/gather/deposit) is bounded per quantity against the
FP64 oracle; the bounds are FP32 rounding times the measured sensitivity.
"""
import math

import numpy as np
import pytest

import pic_inputs
from tests._common import (gross_scales, make_gpu, make_oracle, periodic_diff, rel_err,
                           scaled_err, small_1d, small_2d)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2609_36383_b300 import build
    build.build()
    import oracle
    oracle.build()


def _ragged_2d():
    cfg = small_2d(n=16, ppc=8, T=0.02, u_drift=0.6, dt=0.2, seed=5)
    # 37 extra particles make N ragged against the block size; a few sit
    # exactly on knots (offset -1/2) and move in both directions
    rng = np.random.default_rng(9)
    k = 37
    dx = cfg["L"][0] / cfg["n"][0]
    xe = cfg["x0"][0] + (rng.integers(0, 16, (2, k)) - 0.5) * dx
    ue = rng.standard_normal((3, k)) * 0.4
    cfg["x"] = np.concatenate([cfg["x"], xe], axis=1)
    cfg["u"] = np.concatenate([cfg["u"], ue], axis=1)
    cfg["w"] = np.concatenate([cfg["w"], np.full(k, cfg["w"][0])])
    cfg["w"] *= (4 * math.pi ** 2) / cfg["w"].sum()
    cfg["sp"] = np.zeros(cfg["w"].shape[0], np.int32)
    return cfg


def _fast_2d():
    # displacements above one cell per step: several knot crossings per dimension
    return small_2d(n=32, ppc=4, T=0.05, u_drift=0.9, dt=0.5, seed=7)


def _two_species_2d():
    cfg = pic_inputs.weibel_2d_ions(n=16, ppc_beam=2, ppc_ion=4, u_drift=0.9, T=0.05,
                                    mass_ratio=100.0, dt=0.1, seed=11, kmax=3)
    return cfg


def _thermal_3d():
    return pic_inputs.thermal_box(dim=3, n=8, ppc=2, T=0.05, u_drift=0.3, dt=0.2, seed=4)


def _rect_2d():
    # a rectangular mesh (32 x 8 nodes, rectangular cells): rows and columns of
    # the 2D field step differ in length
    return pic_inputs.thermal_box(dim=2, n=(32, 8), ppc=6, T=0.05, u_drift=0.4, dt=0.2, seed=6)


CASES = {
    "1d_two_stream": small_1d,
    "3d_thermal": _thermal_3d,
    "2d_weibel": small_2d,
    "2d_ragged_knots": _ragged_2d,
    "2d_fast_multicross": _fast_2d,
    "2d_two_species": _two_species_2d,
    "2d_rect_32x8": _rect_2d,
}


@pytest.fixture(params=sorted(CASES))
def case(request):
    return request.param, CASES[request.param]()


def _field_close(a, b, tol, cfg):
    """Potentials relative to their own maximum; deposited charge and current
    relative to their gross (one-sign) magnitude."""
    g = gross_scales(cfg)
    for k in ("phi", "psi", "A", "U", "rho", "J"):
        err = scaled_err(a[k], b[k], g.get(k, 0.0))
        assert err <= tol, (k, err)


def test_start_parity(case):
    name, cfg = case
    o = make_oracle(cfg)
    ro = o.start()
    s = make_gpu(cfg)
    rs = s.start()
    _field_close(s.fields(), o.fields(), 1e-12, cfg)
    xs, Ps, ws, _ = s.particles()
    xo, Po, wo, _ = o.particles()
    assert np.abs(periodic_diff(xs, xo, cfg["L"])).max() < 1e-12
    assert rel_err(Ps, Po) < 1e-12
    assert np.array_equal(ws, wo)
    for k in ("K", "W", "E_tot"):
        assert rs[k] == pytest.approx(ro[k], rel=1e-12, abs=1e-18), k
    assert rs["gauss_rms"] < 1e-12 and rs["lorenz_rms"] < 1e-12


def test_velocities_round_trip(case):
    """pic_get_velocities returns u = (P - q A_h(x)) / m: right after start it
    recovers the loaded proper velocities (P was formed as m u + q A_h(x))."""
    name, cfg = case
    s = make_gpu(cfg)
    s.start()
    u = s.velocities()
    scale = max(np.abs(cfg["u"]).max(), 1e-30)
    assert np.abs(u - cfg["u"]).max() <= 1e-13 * scale


def test_single_map_evaluation_parity(case):
    """H(j), vbar, P^{n+1} and inner counts of one evaluation (Sec. 4.5)."""
    name, cfg = case
    o = make_oracle(cfg)
    o.start()
    s = make_gpu(cfg)
    s.start()
    rng = np.random.default_rng(2)
    J = o.fields()["J"]
    j = J + 0.05 * np.abs(J).max() * o.project(rng.standard_normal(J.shape[0]), 3)
    st_o, Ho, vo, Po, io = o.eval_map(j, 1e-14)
    st_s, Hs, vs, Ps, is_ = s.eval_map(j, 1e-14)
    assert st_o == 0 and st_s == 0
    assert scaled_err(Hs, Ho, gross_scales(cfg)["H"]) < 1e-12
    assert rel_err(vs, vo) < 1e-12
    assert rel_err(Ps, Po) < 1e-12
    assert np.all(np.abs(is_ - io) <= 1)
    assert abs(is_.mean() - io.mean()) < 0.05 * io.mean()


def test_free_running_steps_parity_and_energy(case):
    name, cfg = case
    o = make_oracle(cfg)
    o.start()
    s = make_gpu(cfg)
    s.start()
    for _ in range(3):
        ro = o.step(1e-12)
        rs = s.step(1e-12)
        assert ro["status"] == 0 and rs["status"] == 0
        assert abs(rs["rel_dE"]) < 1e-11
        assert rs["chain_rms"] < 1e-14
        assert abs(rs["work_residual"]) < 1e-14 * max(1.0, rs["K"])
        assert rs["gauss_rms"] < 1e-11 and rs["lorenz_rms"] < 1e-11
        assert rs["res_scaled_rms"] <= 1.0 and rs["res_scaled_max"] <= 1.0
    xs, Ps, _, _ = s.particles()
    xo, Po, _, _ = o.particles()
    assert np.abs(periodic_diff(xs, xo, cfg["L"])).max() < 1e-9 * max(cfg["L"])
    assert rel_err(Ps, Po) < 1e-9
    _field_close(s.fields(), o.fields(), 1e-9, cfg)


def test_cell_sort_does_not_change_results():
    """Counting-sorting the particles by cell (every step vs never) changes only
    the summation order of the deposit: results agree at roundoff."""
    cfg = _ragged_2d()
    a = make_gpu(cfg, sort_every=1)
    b = make_gpu(cfg, sort_every=0)
    a.start()
    b.start()
    for _ in range(3):
        ra = a.step(1e-12)
        rb = b.step(1e-12)
        assert ra["status"] == 0 and rb["status"] == 0
        assert ra["E_tot"] == pytest.approx(rb["E_tot"], rel=1e-13)
    xa, Pa, wa, sa = a.particles()
    xb, Pb, wb, sb = b.particles()
    assert np.abs(periodic_diff(xa, xb, cfg["L"])).max() < 1e-9 * max(cfg["L"])
    assert rel_err(Pa, Pb) < 1e-9
    assert np.array_equal(wa, wb) and np.array_equal(sa, sb)
    _field_close(a.fields(), b.fields(), 1e-9, cfg)


def test_inner_warm_start_option():
    """Option inner_warm_start (later evaluations of a step start the inner
    iteration from the previous evaluation's orbit velocity), used with an
    inner tolerance ten times tighter: the steps still converge to the same
    fixed point as the cold-started oracle, with fewer inner iterations."""
    cfg = small_2d()
    o = make_oracle(cfg)
    o.start()
    s = make_gpu(cfg, inner_warm_start=1, inner_tol_scale=0.1)
    s.start()
    c = make_gpu(cfg)
    c.start()
    for _ in range(3):
        ro = o.step(1e-12)
        rs = s.step(1e-12)
        rc = c.step(1e-12)
        assert ro["status"] == 0 and rs["status"] == 0 and rc["status"] == 0
        assert abs(rs["rel_dE"]) < 1e-11
    assert s.stats()["inner_iters"] < c.stats()["inner_iters"]
    xs, Ps, _, _ = s.particles()
    xo, Po, _, _ = o.particles()
    assert np.abs(periodic_diff(xs, xo, cfg["L"])).max() < 1e-9 * max(cfg["L"])
    assert rel_err(Ps, Po) < 1e-9


def test_failed_step_leaves_state_unchanged():
    cfg = small_2d()
    s = make_gpu(cfg)
    s.start()
    xa, Pa, _, _ = s.particles()
    fa = s.fields()
    r = s.step(0.0)  # the inner test cannot pass with zero tolerance
    assert r["status"] == -4
    xb, Pb, _, _ = s.particles()
    fb = s.fields()
    assert np.array_equal(xa, xb) and np.array_equal(Pa, Pb)
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k
    r = s.step(1e-12)  # and the context keeps working
    assert r["status"] == 0


def test_outer_failure_leaves_state_unchanged():
    cfg = small_2d()
    s = make_gpu(cfg, outer_max=1, inner_tol_scale=1e18)
    s.start()
    xa, Pa, _, _ = s.particles()
    fa = s.fields()
    r = s.step(1e-28)
    assert r["status"] == -5
    xb, Pb, _, _ = s.particles()
    fb = s.fields()
    assert np.array_equal(xa, xb) and np.array_equal(Pa, Pb)
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k


def test_empty_particle_set_vacuum_fields():
    """No particles: the CN field step alone conserves the field energy."""
    cfg = small_2d()
    for k in ("x", "u"):
        cfg[k] = cfg[k][:, :0]
    cfg["w"] = cfg["w"][:0]
    cfg["sp"] = cfg["sp"][:0]
    cfg["rho_bg"] = 0.0
    rng = np.random.default_rng(4)
    cfg["U"] = 1e-3 * rng.standard_normal((3, 256))
    o = make_oracle(cfg)
    o.start()
    s = make_gpu(cfg)
    rs0 = s.start()
    for _ in range(2):
        ro = o.step(1e-12)
        rs = s.step(1e-12)
        assert rs["status"] == 0 and ro["status"] == 0
    assert abs(rs["rel_dE"]) < 1e-13
    _field_close(s.fields(), o.fields(), 1e-12, cfg)
    assert rs0["W"] > 0


def test_two_stream_growth_and_energy_gpu():
    """Same physics pin as the oracle's: Gamma_TS and energy conservation."""
    from oracle import closed_form as cf
    u0, L, n = 0.6, 4 * math.pi, 64
    G = cf.two_stream_rate(0.5, u0 / math.sqrt(1 + u0 * u0), L / n)
    cfg = pic_inputs.two_stream_1d(eigen_rate=G, eigen_chi=cf.chi(0.5, L / n))
    s = make_gpu(cfg)
    s.start()
    k = 2 * np.pi * np.fft.fftfreq(n, d=L / n)
    k[n // 2] = 0.0
    ts, amps, dE = [], [], 0.0
    for st in range(1, 61):
        r = s.step(cfg["tol"])
        assert r["status"] == 0
        dE = max(dE, abs(r["rel_dE"]))
        f = s.fields()
        Ex = np.real(np.fft.ifft(-1j * k * np.fft.fft(f["phi"]))) - f["U"][:n]
        ts.append(st * cfg["dt"])
        amps.append(abs(np.fft.fft(Ex)[1]) / n)
    rate = np.polyfit(np.array(ts), np.log(np.array(amps)), 1)[0]
    assert rate == pytest.approx(G, rel=2e-3)
    assert dE < 1e-12


def test_full_size_weibel_sampled_parity():
    """128^2 mesh, 64 particles/cell (1,048,576 particles), in the launch
    configuration the benchmark times: the oracle recomputes the inner solves
    of 512 sampled particles one by one at the same trial current, and the
    total current sum_g H_g dV = sum_i q_i vbar_i holds at full size."""
    cfg = pic_inputs.weibel_2d()
    o = make_oracle(cfg)
    o.start()
    s = make_gpu(cfg)
    s.start()
    J = o.fields()["J"]
    st_s, Hs, vs, Ps, its = s.eval_map(J, 1e-13)
    assert st_s == 0
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(cfg["w"].shape[0], 512, replace=False))
    st_o, vo, Po, io = o.eval_particles(J, 1e-13, idx)
    assert st_o == 0
    assert rel_err(vs[:, idx], vo) < 1e-11
    assert rel_err(Ps[:, idx], Po) < 1e-11
    assert np.all(np.abs(its[idx] - io) <= 1)
    dV = (2 * math.pi / 128) ** 2
    q = -cfg["w"]
    tot_particles = (q[None, :] * vs).sum(axis=1)
    tot_mesh = Hs.reshape(3, -1).sum(axis=1) * dV
    assert np.allclose(tot_mesh, tot_particles, rtol=1e-10, atol=1e-12 * np.abs(q).sum())


def test_mixed_precision_bounded_against_fp64_oracle():
    cfg = small_2d()
    o = make_oracle(cfg)
    o.start()
    s = make_gpu(cfg, precision=1)
    s.start()
    J = o.fields()["J"]
    st_o, Ho, vo, Po, io = o.eval_map(J, 1e-14)
    st_s, Hs, vs, Ps, is_ = s.eval_map(J, 1e-14)
    assert st_o == 0 and st_s == 0
    # FP32 push/gather/deposit: ~1e-7 relative per quantity (6e-8 rounding,
    # a few operations deep), H additionally sums ~600 particles per node
    assert rel_err(vs, vo) < 2e-6
    assert rel_err(Ps, Po) < 2e-6
    assert scaled_err(Hs, Ho, gross_scales(cfg)["H"]) < 2e-6
    for _ in range(3):
        r = s.step(1e-10)
        assert r["status"] == 0
        assert abs(r["rel_dE"]) < 1e-6


def test_full_size_mixed_sampled_parity():
    """The FP32-mixed map at full size (128^2 mesh, 1,048,576 particles) in the
    launch configuration the benchmark times: 512-particle chunks whose inputs
    are staged in shared memory, and deposits from the records the solve pass
    writes.  Sampled orbit velocities and momenta against the oracle's FP64
    inner solves at the same trial current, the deposited current against the
    FP64 GPU path (itself checked against the oracle above), at the FP32
    bounds of the small mixed case.  333 particles are left out, so the last
    chunk of each launch is ragged."""
    cfg = pic_inputs.weibel_2d()
    keep = cfg["w"].shape[0] - 333
    for k in ("x", "u"):
        cfg[k] = cfg[k][:, :keep]
    cfg["w"] = cfg["w"][:keep]
    cfg["sp"] = cfg["sp"][:keep]
    o = make_oracle(cfg)
    o.start()
    J = o.fields()["J"]
    s64 = make_gpu(cfg)
    s64.start()
    st64, H64, _, _, _ = s64.eval_map(J, 1e-14)
    s64.close()
    s32 = make_gpu(cfg, precision=1)
    s32.start()
    st32, H32, v32, P32, _ = s32.eval_map(J, 1e-14)
    s32.close()
    assert st64 == 0 and st32 == 0
    rng = np.random.default_rng(1)
    idx = np.sort(rng.choice(cfg["w"].shape[0], 512, replace=False))
    st_o, vo, Po, _ = o.eval_particles(J, 1e-14, idx)
    assert st_o == 0
    assert rel_err(v32[:, idx], vo) < 2e-6
    assert rel_err(P32[:, idx], Po) < 2e-6
    assert scaled_err(H32, H64, gross_scales(cfg)["H"]) < 2e-6
