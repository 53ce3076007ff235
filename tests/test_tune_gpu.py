"""The sort-interval autotuner (pic_tune_sort) on the CUDA path: it measures
every candidate, leaves the state exactly as it found it (the checkpoint
image after the call equals the one before, but for the sort interval),
keeps the statistics clean, and the context then steps as a fresh context
with the chosen interval does."""
import numpy as np
import pytest

import paper_2609_36383_b300 as pic
from tests._common import make_gpu, small_2d

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
    img0 = s.checkpoint()
    st0 = s.stats()
    cand = (0, 1, 3)
    best, ms = s.tune_sort(tol, 4, cand)
    print(f"candidates {cand}: ms/step {np.round(ms, 3)}, chose {best}")
    assert best in cand
    assert np.all(ms > 0) and np.all(np.isfinite(ms))
    assert s.stats() == st0
    img1 = s.checkpoint()
    assert img1[256:] == img0[256:]  # every state byte
    h0, h1 = pic.inspect_checkpoint(img0), pic.inspect_checkpoint(img1)
    assert h1.pop("sort_every") == best and h0.pop("sort_every") == 0
    assert h0 == h1
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
