"""The knot-jump regularity diagnostic (pic_knot_jumps, Sec. 5.3) on the CUDA
path.

  * Parity with the oracle (orc_knot_jumps, pinned by closed forms in
    tests/test_oracle_pins_shapes.py) on random fields, for linear and
    quadratic shapes in 1D, 2D and 3D.  Degree one: the jumps are O(1) and
    agree to 1e-12.  Degree two: they are O(eps) differences of O(1) values,
    so each side's rounding (and the GPU's FFT round trip of phi and U)
    enters relative to eps; the bound is 1e-6.
  * The contrast the paper draws (Sec. 5.3): after 40 steps of the 1D
    two-stream instability the degree-one jumps are O(1) while the
    degree-two ones are O(eps) times the fields' curvature, many orders of
    magnitude smaller.
"""
import math

import numpy as np
import pytest

import paper_2609_36383_b300 as pic
import pic_inputs
from tests._common import make_gpu, small_1d

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2609_36383_b300 import build
    build.build()
    import oracle
    oracle.build()


GRIDS = {1: [32], 2: [16, 8], 3: [8, 8, 4]}


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("dim", [1, 2, 3])
def test_knot_jumps_match_the_oracle(dim, order):
    import oracle
    n = GRIDS[dim]
    L = [2 * math.pi * (1 + 0.5 * l) for l in range(dim)]
    x0 = [-0.5 * v for v in L]
    Ng = int(np.prod(n))
    rng = np.random.default_rng(10 * dim + order)
    f = dict(phi=rng.standard_normal(Ng), psi=np.zeros(Ng), A=rng.standard_normal(3 * Ng),
             U=rng.standard_normal(3 * Ng), rho=np.zeros(Ng), J=np.zeros(3 * Ng))
    empty = (np.zeros((dim, 0)), np.zeros((3, 0)), np.zeros(0), np.zeros(0, np.int32))
    s = pic.Simulation(dim, n, L, x0, [(-1.0, 1.0)], 0.1, order=order)
    s.set_state(*empty, f, 1.0)
    o = oracle.Oracle(dim, n, L, x0, [(-1.0, 1.0)], dt=0.1, order=order)
    o.set_state(*empty, f)
    Eg, Gg = s.knot_jumps(1e-8)
    Eo, Go = o.knot_jumps(1e-8)
    print(f"dim {dim} r {order}: E jump GPU {Eg:.10e} oracle {Eo:.10e}; "
          f"grad A jump GPU {Gg:.10e} oracle {Go:.10e}")
    rel = 1e-12 if order == 1 else 1e-6
    assert Eg == pytest.approx(Eo, rel=rel)
    assert Gg == pytest.approx(Go, rel=rel)
    assert Eo > 0 and Go > 0


def test_degree_one_jumps_are_order_one_and_degree_two_jumps_order_eps():
    res = {}
    for order in (1, 2):
        cfg = small_1d()
        s = make_gpu(cfg, order=order, refine_max=2)
        s.start()
        for _ in range(40):
            assert s.step(1e-12)["status"] == 0
        res[order] = s.knot_jumps(1e-8)
    print(f"two-stream, 40 steps: r = 1 jumps E {res[1][0]:.3e}, grad A {res[1][1]:.3e}; "
          f"r = 2 jumps E {res[2][0]:.3e}, grad A {res[2][1]:.3e}")
    assert res[1][0] > 1e4 * res[2][0]
    assert res[2][0] < 1e-6
