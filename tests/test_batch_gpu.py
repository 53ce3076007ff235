"""Batched ensembles of 1D3V problems (pic_batch_*) on the CUDA path.

Every instance of a batch must compute what a single-problem context (and the
FP64 oracle) computes for the same data: the same step of Algorithm 1 with the
same options.  The two differ only in the summation order of reductions and
deposits, so after free-running steps at nonlinear tolerance 1e-12 their
states agree to a few times the tolerance (1e-9 relative bound, as for the
single-problem parity tests).  The ensemble mixes mesh sizes, particle counts
that are ragged against the 128-particle block, beam speeds, an instance with
no particles and (in the failure test) instances that succeed next to one
that fails.
"""
import math

import numpy as np
import pytest

import pic_inputs
from tests._common import gross_scales, make_gpu, make_oracle, periodic_diff, rel_err, scaled_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2609_36383_b300 import build
    build.build()
    import oracle
    oracle.build()


def _vacuum_wave(nx=16, amp=1e-3):
    """No particles; a transverse vacuum wave A_y = a cos(k x) in the box of
    the ensemble (L = 4 pi), neutral background."""
    L = 4 * math.pi
    x0 = -0.5 * L
    xg = x0 + np.arange(nx) * (L / nx)
    A = np.zeros((3, nx))
    A[1] = amp * np.cos(0.5 * (xg - x0))
    return dict(name="vacuum_wave", dim=1, n=[nx], L=[L], x0=[x0], species=[(-1.0, 1.0)],
                rho_bg=0.0, dt=0.1, tol=1e-12, steps=10, x=np.zeros((1, 0)), u=np.zeros((3, 0)),
                w=np.zeros(0), sp=np.zeros(0, np.int32), A=A.reshape(-1), U=None)


def _ensemble(B=5, seed=1, with_vacuum=False):
    cfgs = pic_inputs.two_stream_ensemble(B=B, seed=seed, nx_choices=(8, 16, 32, 64),
                                          ppc_range=(4, 20), u_range=(0.2, 0.95), tol=1e-12)
    if with_vacuum:
        v = _vacuum_wave()
        v["rho_bg"] = cfgs[0]["rho_bg"]  # shared option; no particles, so rho stays rho_bg
        cfgs.insert(2, v)
    return cfgs


def _make_batch(cfgs, precision=0, **kw):
    import paper_2609_36383_b300 as P
    return P.batch_from_configs(cfgs, precision=precision, **kw)


def _assert_state_close(xa, Pa, fa, xb, Pb, fb, cfg, tol):
    if xa.size:
        assert np.abs(periodic_diff(xa, xb, cfg["L"])).max() < tol * cfg["L"][0]
        assert rel_err(Pa, Pb) < tol
    g = gross_scales(cfg) if cfg["w"].size else {}
    for k in ("phi", "psi", "A", "U", "rho", "J"):
        err = scaled_err(fa[k], fb[k], g.get(k, 0.0))
        assert err <= tol, (k, err)


def test_batch_steps_match_single_contexts():
    cfgs = _ensemble(with_vacuum=True)
    bt = _make_batch(cfgs)
    rb0 = bt.start()
    singles = [make_gpu(c) for c in cfgs]
    rs0 = [s.start() for s in singles]
    for b in range(len(cfgs)):
        assert rb0[b]["E_tot"] == rs0[b]["E_tot"]
    for _ in range(3):
        rb = bt.step(1e-12)
        rs = [s.step(1e-12) for s in singles]
        for b, c in enumerate(cfgs):
            assert rb[b]["status"] == 0 and rs[b]["status"] == 0, (b, rb[b], rs[b])
            assert abs(rb[b]["rel_dE"]) < 1e-11, (b, rb[b])
            assert rb[b]["E_tot"] == pytest.approx(rs[b]["E_tot"], rel=1e-11), b
            assert rb[b]["res_scaled_rms"] <= 1.0 and rb[b]["res_scaled_max"] <= 1.0
            if not c["w"].size:
                # the background charge alone is not neutral: the k = 0 modes
                # of Gauss's law and of psi (which the uniform charge drives)
                # depart from the constraints, identically in both
                assert rb[b]["gauss_rms"] == pytest.approx(rs[b]["gauss_rms"], rel=1e-12)
                assert rb[b]["lorenz_rms"] == pytest.approx(rs[b]["lorenz_rms"], rel=1e-12)
            else:
                assert rb[b]["gauss_rms"] < 1e-11 and rb[b]["lorenz_rms"] < 1e-11
                assert rb[b]["chain_rms"] < 1e-14
                assert abs(rb[b]["work_residual"]) < 1e-14 * max(1.0, rb[b]["K"])
                assert rb[b]["inner_mean"] == pytest.approx(rs[b]["inner_mean"], rel=0.05)
            # the same decisions of Algorithm 1 in almost every step
            assert abs(rb[b]["map_evals"] - rs[b]["map_evals"]) <= 2
    for b, c in enumerate(cfgs):
        xb, Pb, wb, sb = bt.particles(b)
        xs, Ps, ws, ss = singles[b].particles()
        assert np.array_equal(wb, ws) and np.array_equal(sb, ss)
        _assert_state_close(xb, Pb, bt.fields(b), xs, Ps, singles[b].fields(), c, 1e-9)
    st = bt.stats()
    assert st["pushes"] > 0 and st["inner_iters"] > 0 and st["map_launches"] > 0


def test_batch_matches_oracle():
    cfgs = _ensemble(B=3, seed=4)
    bt = _make_batch(cfgs)
    bt.start()
    orcs = [make_oracle(c) for c in cfgs]
    for o in orcs:
        o.start()
    for _ in range(2):
        rb = bt.step(1e-12)
        ro = [o.step(1e-12) for o in orcs]
        for b in range(len(cfgs)):
            assert rb[b]["status"] == 0 and ro[b]["status"] == 0
            assert rb[b]["E_tot"] == pytest.approx(ro[b]["E_tot"], rel=1e-11)
    for b, c in enumerate(cfgs):
        xb, Pb, _, _ = bt.particles(b)
        xo, Po, _, _ = orcs[b].particles()
        _assert_state_close(xb, Pb, bt.fields(b), xo, Po, orcs[b].fields(), c, 1e-9)


def test_batch_vacuum_wave_conserves_energy():
    """An instance without particles: the CN update of a vacuum wave conserves
    the field energy exactly in exact arithmetic (Thm. energy)."""
    cfgs = _ensemble(B=2, seed=2, with_vacuum=True)
    bt = _make_batch(cfgs)
    r0 = bt.start()
    W0 = r0[2]["W"]
    assert W0 > 0.0
    for _ in range(5):
        r = bt.step(1e-12)
        assert all(x["status"] == 0 for x in r)
    assert r[2]["W"] == pytest.approx(W0, rel=1e-13)
    assert r[2]["K"] == 0.0


def test_batch_failure_keeps_state_and_spares_other_instances():
    """With an inner iteration cap of 1, the instances at rest converge (their
    orbit velocity does not move) while the drifting two-stream instances fail
    (PIC_EINNER); the failed ones keep their accepted state, as pic_step does,
    and the others commit."""
    rest = pic_inputs.two_stream_1d(nx=16, ppc_beam=4, u0=0.0, pert=0.0, tol=1e-12)
    cfgs = [rest, pic_inputs.two_stream_1d(nx=16, ppc_beam=4, u0=0.6, tol=1e-12), dict(rest)]
    bt = _make_batch(cfgs, inner_max=1)
    bt.start()
    before = [bt.particles(b) for b in range(3)]
    f_before = bt.fields(1)
    r = bt.step(1e-12)
    assert r[0]["status"] == 0 and r[2]["status"] == 0
    assert r[1]["status"] == -4  # PIC_EINNER
    x1, P1, _, _ = bt.particles(1)
    assert np.array_equal(x1, before[1][0]) and np.array_equal(P1, before[1][1])
    f1 = bt.fields(1)
    for k in f1:
        assert np.array_equal(f1[k], f_before[k]), k


def test_batch_sort_does_not_change_results():
    cfgs = _ensemble(B=4, seed=5)
    a = _make_batch(cfgs, sort_every=1)
    b = _make_batch(cfgs, sort_every=0)
    a.start()
    b.start()
    for _ in range(3):
        ra = a.step(1e-12)
        rb = b.step(1e-12)
        for k in range(len(cfgs)):
            assert ra[k]["status"] == 0 and rb[k]["status"] == 0
            assert ra[k]["E_tot"] == pytest.approx(rb[k]["E_tot"], rel=1e-12)
    for k, c in enumerate(cfgs):
        xa, Pa, wa, sa = a.particles(k)
        xb, Pb, wb, sb = b.particles(k)
        assert np.array_equal(wa, wb) and np.array_equal(sa, sb)
        _assert_state_close(xa, Pa, a.fields(k), xb, Pb, b.fields(k), c, 1e-9)


def test_batch_mixed_precision_bounds():
    """FP32 push/gather/deposit with FP64 field solve and sums, against the
    FP64 batch: the mixed tolerance floor (1e-5) bounds the nonlinear error."""
    cfgs = _ensemble(B=4, seed=6)
    m = _make_batch(cfgs, precision=1, sort_every=4)
    d = _make_batch(cfgs)
    m.start()
    d.start()
    for _ in range(3):
        rm = m.step(1e-10)
        rd = d.step(1e-12)
        for k in range(len(cfgs)):
            assert rm[k]["status"] == 0 and rd[k]["status"] == 0
            assert abs(rm[k]["rel_dE"]) < 1e-5
            assert rm[k]["E_tot"] == pytest.approx(rd[k]["E_tot"], rel=1e-5)
    for k, c in enumerate(cfgs):
        xm, Pm, _, _ = m.particles(k)
        xd, Pd, _, _ = d.particles(k)
        assert np.abs(periodic_diff(xm, xd, c["L"])).max() < 1e-5 * c["L"][0]
        assert rel_err(Pm, Pd) < 1e-4


def test_batch_rejects_bad_arguments():
    import paper_2609_36383_b300 as P
    with pytest.raises(P.PicError):
        P.Batch([12], [1.0], [0.0], [0], [(-1.0, 1.0)], 0.1)  # not a power of two
    with pytest.raises(P.PicError):
        P.Batch([2048], [1.0], [0.0], [0], [(-1.0, 1.0)], 0.1)  # above 1024 nodes
    with pytest.raises(P.PicError):
        P.Batch([16], [1.0], [0.0], [0], [(-1.0, 1.0)], 0.1, anderson_m=9)
    bt = P.Batch([16, 16], [1.0, 1.0], [0.0, 0.0], [0, 0], [(-1.0, 1.0)], 0.1)
    with pytest.raises(P.PicError):
        bt.start()  # instances not staged


@pytest.mark.parametrize("precision,tol,bound", [(0, 1e-12, 1e-9), (1, 1e-10, 2e-5)],
                         ids=["fp64", "mixed"])
def test_batch_production_sizes_match_single_contexts(precision, tol, bound):
    """Instances at the ensemble workload's extremes: 512 cells with 256
    particles per cell at u = 0.95 (131,072 particles, the largest mesh and
    per-instance particle count the workload draws, the fastest beams), 256
    cells with 128 per cell, and 32 cells with 16 per cell at u = 0.2, through
    the shared-memory spectral solve and the persistent batch map, against
    single-problem contexts with the same data, FP64 and FP32-mixed."""
    cfgs = [pic_inputs.two_stream_1d(nx=512, ppc_beam=128, u0=0.95, tol=tol, seed=7),
            pic_inputs.two_stream_1d(nx=256, ppc_beam=64, u0=0.6, tol=tol, seed=8),
            pic_inputs.two_stream_1d(nx=32, ppc_beam=8, u0=0.2, tol=tol, seed=9)]
    bt = _make_batch(cfgs, precision=precision)
    bt.start()
    singles = [make_gpu(c, precision=precision) for c in cfgs]
    for s in singles:
        s.start()
    for st in range(3):
        rb = bt.step(tol)
        rs = [s.step(tol) for s in singles]
        for b in range(len(cfgs)):
            assert rb[b]["status"] == 0 and rs[b]["status"] == 0, (b, rb[b], rs[b])
            assert rb[b]["E_tot"] == pytest.approx(rs[b]["E_tot"], rel=bound), b
            if precision == 0:
                assert abs(rb[b]["rel_dE"]) < 1e-11, (b, rb[b])
                assert abs(rb[b]["map_evals"] - rs[b]["map_evals"]) <= 2
    for b, c in enumerate(cfgs):
        xb, Pb, _, _ = bt.particles(b)
        xs, Ps, _, _ = singles[b].particles()
        if precision == 0:
            _assert_state_close(xb, Pb, bt.fields(b), xs, Ps, singles[b].fields(), c, bound)
        else:
            # FP32 rounding differs between the two: particles, and the
            # deposited rho and J against their gross (one-sign) scales; the
            # potentials follow from these (psi, a small difference of
            # large terms, is not a meaningful relative measure here)
            assert np.abs(periodic_diff(xb, xs, c["L"])).max() < bound * c["L"][0]
            assert rel_err(Pb, Ps) < bound
            g = gross_scales(c)
            fb, fs = bt.fields(b), singles[b].fields()
            for k in ("rho", "J"):
                assert scaled_err(fb[k], fs[k], g[k]) <= bound, k
    for s in singles:
        s.close()
