"""The sort-interval autotuner (pic_tune_sort) on the CUDA path: it measures
every candidate, leaves the state as it found it (up to the round trip of
positions through physical coordinates), keeps the statistics clean, and the
context then steps as a fresh context with the chosen interval does."""
import numpy as np
import pytest

from tests._common import make_gpu, periodic_diff, small_2d

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2609_36383_b300 import build
    build.build()


def test_tune_sort_restores_the_state_and_picks_a_candidate():
    cfg = small_2d()
    tol = 1e-12
    s = make_gpu(cfg, sort_every=0)
    s.start()
    assert s.step(tol)["status"] == 0
    x0, P0, _, _ = s.particles()
    f0 = s.fields()
    st0 = s.stats()
    cand = (0, 1, 3)
    best, ms = s.tune_sort(tol, 4, cand)
    print(f"candidates {cand}: ms/step {np.round(ms, 3)}, chose {best}")
    assert best in cand
    assert np.all(ms > 0) and np.all(np.isfinite(ms))
    assert s.stats() == st0
    x1, P1, _, _ = s.particles()
    f1 = s.fields()
    assert np.abs(periodic_diff(x1, x0, cfg["L"])).max() <= 1e-13 * max(cfg["L"])
    assert np.abs(P1 - P0).max() <= 1e-15 * np.abs(P0).max()
    for k in ("phi", "psi", "A", "U", "rho", "J"):
        assert np.abs(f1[k] - f0[k]).max() <= 1e-12 * max(np.abs(f0[k]).max(), 1e-300), k
    # the next step matches a fresh context set up with the chosen interval
    ref = make_gpu(cfg, sort_every=best)
    ref.start()
    assert ref.step(tol)["status"] == 0
    r1 = s.step(tol)
    r2 = ref.step(tol)
    assert r1["status"] == 0 and r2["status"] == 0
    _, Pa, _, _ = s.particles()
    _, Pb, _, _ = ref.particles()
    assert np.abs(Pa - Pb).max() <= 1e-9 * np.abs(Pb).max()
    assert abs(r1["E_tot"] - r2["E_tot"]) <= 1e-11 * abs(r2["E_tot"])


def test_tune_sort_rejects_bad_arguments():
    cfg = small_2d()
    s = make_gpu(cfg)
    s.start()
    with pytest.raises(RuntimeError):
        s.tune_sort(1e-12, 2, (-1, 2))
