"""The deterministic orbit deposit (option deterministic_deposit) on the CUDA
path: it computes the same current as the atomic deposit (to the rounding of
two summation orders, bounded against the gross current as in the parity
tests), and it is reproducible bit for bit from run to run, which the atomic
deposit does not promise."""
import numpy as np
import pytest

import pic_inputs
from tests._common import gross_scales, make_gpu, make_oracle, small_1d, small_2d

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


@pytest.mark.parametrize("name", sorted(CASES))
def test_deterministic_deposit_matches_the_atomic_deposit(name):
    cfg = CASES[name]()
    o = make_oracle(cfg)
    o.start()
    j = o.fields()["J"]
    a = make_gpu(cfg)
    a.start()
    b = make_gpu(cfg, deterministic_deposit=1)
    b.start()
    gs = gross_scales(cfg)
    # pic_start's point deposits
    fa, fb = a.fields(), b.fields()
    assert np.abs(fa["rho"] - fb["rho"]).max() <= 1e-13 * gs["rho"]
    assert np.abs(fa["J"] - fb["J"]).max() <= 1e-13 * gs["J"]
    # one map evaluation
    st1, Ha, _, _, _ = a.eval_map(j, 1e-14)
    st2, Hb, _, _, _ = b.eval_map(j, 1e-14)
    assert st1 == 0 and st2 == 0
    err = np.abs(Ha - Hb).max() / gs["J"]
    print(f"{name}: max |H_det - H_atomic| = {err:.2e} of the gross current")
    assert err <= 1e-12


@pytest.mark.parametrize("name", sorted(CASES))
def test_deterministic_deposit_is_reproducible_bit_for_bit(name):
    cfg = CASES[name]()
    runs = []
    for _ in range(2):
        s = make_gpu(cfg, deterministic_deposit=1)
        s.start()
        j = s.fields()["J"]
        _, H, _, _, _ = s.eval_map(j, 1e-14)
        reps = [s.step(cfg["tol"]) for _ in range(2)]
        assert all(r["status"] == 0 for r in reps)
        x, P, _, _ = s.particles()
        runs.append((H, x, P, s.fields()["A"], [r["E_tot"] for r in reps]))
    for u, v in zip(runs[0], runs[1]):
        assert np.array_equal(np.asarray(u), np.asarray(v))


def test_deterministic_deposit_rejected_where_unsupported():
    import paper_2609_36383_b300 as P
    cfg = small_2d()
    for kw in (dict(precision=P.PIC_MIXED), dict(refine_max=1)):
        with pytest.raises(RuntimeError):
            make_gpu(cfg, deterministic_deposit=1, **kw)
