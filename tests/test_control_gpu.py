"""Algorithm 1 decided on the device against the same decisions taken on the
host (Sec. 4.5; option host_control).

Both paths take the same decisions in the same order from the same sums; the
device path merges the residual and Gram sums in another (fixed) order, so
values agree to rounding and the decisions agree except at a threshold.  On
the cases below every step's counters (outer iterations, map evaluations,
inner iterations of the final evaluation) must be identical and the energies
and states equal to rounding, in FP64 and FP32-mixed, 1D to 3D, and also
when the outer solver fails (inner limit 1: the step must fail on both paths
with the state unchanged).
"""
import numpy as np
import pytest

import paper_2609_36383_b300 as pic
import pic_inputs
from tests._common import make_gpu, small_1d, small_2d

pytestmark = pytest.mark.gpu


def _thermal_3d():
    return pic_inputs.thermal_box(dim=3, n=8, ppc=2, T=0.05, u_drift=0.3, seed=2)


@pytest.mark.parametrize("make_cfg,precision,steps", [
    (small_1d, pic.PIC_FP64, 6), (small_2d, pic.PIC_FP64, 4), (_thermal_3d, pic.PIC_FP64, 3),
    (small_2d, pic.PIC_MIXED, 4)], ids=["1d", "2d", "3d", "2d_mixed"])
def test_device_and_host_control_agree(make_cfg, precision, steps):
    cfg = make_cfg()
    tol = 1e-12 if precision == pic.PIC_FP64 else 1e-5
    sims = [make_gpu(cfg, precision=precision, host_control=h) for h in (0, 1)]
    for s in sims:
        s.start()
    for st in range(steps):
        rd, rh = [s.step(tol) for s in sims]
        assert rd["status"] == 0 and rh["status"] == 0
        for k in ("outer_iters", "map_evals", "inner_max"):
            assert rd[k] == rh[k], (st, k, rd[k], rh[k])
        assert rd["inner_mean"] == pytest.approx(rh["inner_mean"], rel=1e-12)
        for k in ("K", "W", "E_tot"):
            assert rd[k] == pytest.approx(rh[k], rel=1e-11 if precision == pic.PIC_FP64 else 1e-6)
        assert abs(rd["rel_dE"]) < (1e-11 if precision == pic.PIC_FP64 else 1e-5)
    xd, Pd, _, _ = sims[0].particles()
    xh, Ph, _, _ = sims[1].particles()
    scale = np.abs(Ph).max()
    assert np.abs(Pd - Ph).max() <= (1e-10 if precision == pic.PIC_FP64 else 1e-5) * scale
    sd, sh = sims[0].stats(), sims[1].stats()
    assert sd["map_launches"] == sh["map_launches"]
    assert sd["pushes"] == sh["pushes"] and sd["inner_iters"] == sh["inner_iters"]
    assert sd["map_ms"] > 0.0
    for s in sims:
        s.close()


def test_device_control_failure_keeps_the_state():
    """Inner limit 1: the first evaluation fails its inner solves; both paths
    return PIC_EINNER with the accepted state unchanged (compared as
    checkpoint images)."""
    cfg = small_2d()
    for h in (0, 1):
        s = make_gpu(cfg, inner_max=1, host_control=h)
        s.start()
        before = s.checkpoint()
        r = s.step(1e-12)
        assert r["status"] == pic.PIC_EINNER
        assert s.checkpoint() == before
        s.close()


def test_device_control_outer_limit():
    """Outer limit 2 at an outer tolerance no iterate can meet (the inner
    solves pass at 1e-10): PIC_EOUTER on both paths after the same
    evaluations, the state unchanged."""
    cfg = small_2d()
    res = []
    for h in (0, 1):
        s = make_gpu(cfg, outer_max=2, inner_tol_scale=1e18, host_control=h)
        s.start()
        before = s.checkpoint()
        r = s.step(1e-28)
        res.append(r)
        assert r["status"] == pic.PIC_EOUTER
        assert s.checkpoint() == before
        s.close()
    assert res[0]["map_evals"] == res[1]["map_evals"]
    assert res[0]["outer_iters"] == res[1]["outer_iters"]
