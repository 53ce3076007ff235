"""The FP32 stage of an FP64 context (option fp32_first) on the CUDA path.

Each step first iterates with the particle map in FP32 arithmetic (FP64
particle state) to the FP32 floor of the tolerance, then continues in FP64
from that current to the FP64 tolerance and verifies.  The committed step is
an FP64 step: it passes the same outer tests and verification as the plain
FP64 path, so the two runs stay within the outer tolerance of each other,
the energy theorem (Sec. 4.3) holds at the FP64 tolerance, and the FP64 map
evaluations are fewer.
"""
import numpy as np
import pytest

import paper_2609_36383_b300 as pic
from tests._common import make_gpu, small_1d, small_2d

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("make_cfg,tol", [(small_1d, 1e-12), (small_2d, 1e-10)], ids=["1d", "2d"])
def test_fp32_first_reaches_the_fp64_fixed_point(make_cfg, tol):
    cfg = make_cfg()
    a = make_gpu(cfg)
    b = make_gpu(cfg, fp32_first=1)
    a.start()
    b.start()
    fp64_a = fp64_b = 0
    for st in range(4):
        ra, rb = a.step(tol), b.step(tol)
        assert ra["status"] == 0 and rb["status"] == 0, rb
        assert rb["fp32_evals"] > 0 and ra["fp32_evals"] == 0
        assert rb["res_scaled_rms"] <= 1.0 and rb["res_scaled_max"] <= 1.0
        assert abs(rb["rel_dE"]) < 1e-11 and rb["chain_rms"] < 1e-13
        fp64_a += ra["map_evals"]
        fp64_b += rb["map_evals"] - rb["fp32_evals"]
        print(f"step {st}: FP64 {ra['map_evals']} evaluations; FP32 stage {rb['fp32_evals']} "
              f"+ FP64 {rb['map_evals'] - rb['fp32_evals']}")
    assert fp64_b < fp64_a
    Ja, Jb = a.fields()["J"], b.fields()["J"]
    assert np.abs(Jb - Ja).max() <= 1e-7 * np.abs(Ja).max()
    _, Pa, _, _ = a.particles()
    _, Pb, _, _ = b.particles()
    assert np.abs(Pb - Pa).max() <= 1e-9 * np.abs(Pa).max()
    a.close()
    b.close()


def test_fp32_first_is_refused_outside_its_scope():
    for kw in (dict(precision=pic.PIC_MIXED), dict(order=1), dict(refine_max=1),
               dict(nonlinear_solver=pic.PIC_SOLVER_NEWTON_KRYLOV), dict(host_control=1)):
        with pytest.raises(pic.PicError):
            make_gpu(small_1d(), fp32_first=1, **kw)
