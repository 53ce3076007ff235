"""GPU parity of the degree-one particle shapes and of convergence-triggered
particle refinement (Sec. 5.3) with the FP64 oracle.

Degree-one shapes change only the particle-mesh weights and the knots the
orbit is split at, so the tolerances of the degree-two parity tests apply
(1e-12 for start and one map evaluation at inner tolerance 1e-14, 1e-9 after
free-running steps at tolerance 1e-12).

Refinement is decided per particle by whether its full-step Picard iteration
converges within the inner limit.  A particle whose count sits exactly at the
limit can take the other branch on the two sides (rounding moves its last
residual across the tolerance), and a refined and an unrefined orbit differ by
the time-discretisation error, not by rounding.  So the map evaluation is
compared particle by particle where both sides took the same number of
iterations (at 1e-12), and the number of refined particles must agree to a
few; the energy theorem (Thm. energy) must hold with refinement active.
"""
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


def _thermal_3d():
    return pic_inputs.thermal_box(dim=3, n=8, ppc=2, T=0.05, u_drift=0.3, dt=0.2, seed=4)


CASES = {"1d_two_stream": small_1d, "2d_weibel": small_2d, "3d_thermal": _thermal_3d}


@pytest.fixture(params=sorted(CASES))
def case(request):
    return request.param, CASES[request.param]()


def _field_close(a, b, tol, cfg):
    g = gross_scales(cfg)
    for k in ("phi", "psi", "A", "U", "rho", "J"):
        err = scaled_err(a[k], b[k], g.get(k, 0.0))
        assert err <= tol, (k, err)


def test_degree_one_start_and_map_evaluation_parity(case):
    name, cfg = case
    o = make_oracle(cfg, order=1)
    ro = o.start()
    s = make_gpu(cfg, order=1)
    rs = s.start()
    _field_close(s.fields(), o.fields(), 1e-12, cfg)
    for k in ("K", "W", "E_tot"):
        assert rs[k] == pytest.approx(ro[k], rel=1e-12, abs=1e-18), k
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


def test_degree_one_free_running_steps(case):
    name, cfg = case
    o = make_oracle(cfg, order=1)
    o.start()
    s = make_gpu(cfg, order=1)
    s.start()
    for _ in range(3):
        ro = o.step(1e-12)
        rs = s.step(1e-12)
        assert ro["status"] == 0 and rs["status"] == 0
        assert abs(rs["rel_dE"]) < 1e-11
        assert rs["chain_rms"] < 1e-14
        assert abs(rs["work_residual"]) < 1e-14 * max(1.0, rs["K"])
    xs, Ps, _, _ = s.particles()
    xo, Po, _, _ = o.particles()
    assert np.abs(periodic_diff(xs, xo, cfg["L"])).max() < 1e-9 * max(cfg["L"])
    assert rel_err(Ps, Po) < 1e-9
    _field_close(s.fields(), o.fields(), 1e-9, cfg)


REFINE = {  # order: (dt, inner limit, refinement depth) where full steps fail for some
    2: (0.5, 5, 2),
    1: (0.3, 5, 3),
}


def _refine_cfg(dt):
    return pic_inputs.thermal_box(dim=1, n=16, ppc=8, T=0.05, u_drift=0.6, dt=dt, seed=4)


@pytest.mark.parametrize("order", [2, 1])
def test_refinement_map_evaluation_parity(order):
    dt, im, R = REFINE[order]
    cfg = _refine_cfg(dt)
    o = make_oracle(cfg, order=order, inner_max=im, refine_max=R)
    s = make_gpu(cfg, order=order, inner_max=im, refine_max=R)
    o.start()
    s.start()
    # advance both to a state where refinement is active, with the oracle's
    # accepted state copied into the GPU context
    for _ in range(2):
        assert o.step(1e-12)["status"] == 0
    x, P, w, sp = o.particles()
    f = o.fields()
    s.set_state(x, P, w, sp, f, 1.0)
    st_o, Ho, vo, Po, io = o.eval_map(f["J"], 1e-12)
    st_s, Hs, vs, Ps, is_ = s.eval_map(f["J"], 1e-12)
    assert st_o == 0 and st_s == 0
    ref_o = o.refined()
    # refined particles report the iterations of all their substeps, more than
    # the inner limit of one full-step solve
    ref_s = int(np.sum(is_ > im))
    assert ref_o > 0 and abs(ref_s - int(np.sum(io > im))) <= 3
    same = is_ == io
    assert same.mean() > 0.9
    assert rel_err(vs[:, same], vo[:, same]) < 1e-12
    assert rel_err(Ps[:, same], Po[:, same]) < 1e-12
    if same.all():
        assert scaled_err(Hs, Ho, gross_scales(cfg)["H"]) < 1e-12


@pytest.mark.parametrize("order", [2, 1])
def test_refinement_steps_conserve_energy(order):
    dt, im, R = REFINE[order]
    cfg = _refine_cfg(dt)
    base = make_gpu(cfg, order=order, inner_max=im)
    base.start()
    assert any(base.step(1e-12)["status"] == -4 for _ in range(3))  # fails without refinement
    s = make_gpu(cfg, order=order, inner_max=im, refine_max=R)
    s.start()
    refined = 0
    for _ in range(3):
        r = s.step(1e-12)
        assert r["status"] == 0
        refined += r["refined"]
        assert abs(r["rel_dE"]) < 1e-12
        assert r["chain_rms"] < 1e-15
        assert abs(r["work_residual"]) < 1e-15
    assert refined > 0 and s.stats()["refined"] > 0


def test_refinement_in_a_batch():
    """A batch with refinement enabled matches single contexts with it."""
    import paper_2609_36383_b300 as P
    dt, im, R = REFINE[2]
    cfgs = [_refine_cfg(dt), pic_inputs.thermal_box(dim=1, n=32, ppc=4, T=0.05, u_drift=0.5,
                                                     dt=dt, seed=7)]
    bt = P.batch_from_configs(cfgs, inner_max=im, refine_max=R, sort_every=0)
    bt.start()
    singles = [make_gpu(c, inner_max=im, refine_max=R, sort_every=0) for c in cfgs]
    for sm in singles:
        sm.start()
    for _ in range(2):
        rb = bt.step(1e-12)
        rs = [sm.step(1e-12) for sm in singles]
        for b in range(2):
            assert rb[b]["status"] == 0 and rs[b]["status"] == 0
            assert abs(rb[b]["rel_dE"]) < 1e-12
            assert abs(rb[b]["refined"] - rs[b]["refined"]) <= 2
    assert bt.stats()["refined"] > 0
