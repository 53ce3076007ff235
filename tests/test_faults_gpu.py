"""Failure detection on the CUDA path, with the failures made on the host.

Sec. 4.5 and Algorithm 1 define the failures of a step: an inner particle
solve that hits its iteration limit, turns non-finite or superluminal, and an
outer solve that runs out of iterations or finds no accepted direction.  A
failed step leaves the accepted state unchanged.  Here each failure is
provoked through the public calls only (a NaN momentum loaded into one
particle, an inner iteration limit of 1), and the state before and after the
failed step is compared as checkpoint images, byte for byte (NaNs included).

Why these inputs are safe to run: a non-finite velocity reaches the orbit
walk, whose piece loop is bounded by its piece limit, and every node index
the kernels form is reduced modulo the (power-of-two) mesh size, so a NaN
changes values, never addresses; the inner loop then flags the particle as
non-finite and the step returns PIC_EINNER.
"""
import numpy as np
import pytest

import paper_2609_36383_b300 as pic
from tests._common import make_gpu, small_1d, small_2d

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2609_36383_b300 import build
    build.build()


@pytest.mark.parametrize("precision", [pic.PIC_FP64, pic.PIC_MIXED])
def test_nan_momentum_fails_the_step_and_keeps_the_state(precision):
    cfg = small_2d()
    s = make_gpu(cfg, precision=precision)
    s.start()
    assert s.step(1e-12)["status"] == 0
    x, P, w, sp = s.particles()
    f = s.fields()
    P = P.copy()
    P[1, 17] = np.nan  # one particle's canonical momentum
    E0 = pic.inspect_checkpoint(s.checkpoint())["E0"]
    s.set_state(x, P, w, sp, f, E0=E0)
    before = s.checkpoint()
    r = s.step(1e-12)
    assert r["status"] == pic.PIC_EINNER
    assert s.checkpoint() == before
    # a valid state loaded again steps normally
    P[1, 17] = 0.0
    s.set_state(x, P, w, sp, f, E0=E0)
    assert s.step(1e-12)["status"] == 0


def test_nan_velocity_at_load_fails_the_first_step():
    cfg = small_1d()
    cfg["u"] = cfg["u"].copy()
    cfg["u"][0, 5] = np.nan
    s = make_gpu(cfg)
    s.start()
    before = s.checkpoint()
    r = s.step(1e-12)
    assert r["status"] == pic.PIC_EINNER
    assert s.checkpoint() == before


@pytest.mark.parametrize("name,make", [("1d", small_1d), ("2d", small_2d)])
def test_inner_iteration_limit_of_one_fails_and_keeps_the_state(name, make):
    cfg = make()
    s = make_gpu(cfg, inner_max=1)
    s.start()
    before = s.checkpoint()
    r = s.step(1e-12)
    assert r["status"] == pic.PIC_EINNER
    assert s.checkpoint() == before


def test_outer_iteration_limit_fails_and_keeps_the_state():
    cfg = small_2d()
    s = make_gpu(cfg, outer_max=2, inner_tol_scale=1e18)
    s.start()
    before = s.checkpoint()
    r = s.step(1e-28)  # the inner solves pass at 1e-10; the outer test cannot
    assert r["status"] == pic.PIC_EOUTER and 1 <= r["outer_iters"] <= 2
    assert s.checkpoint() == before


@pytest.mark.parametrize("bad_index", [-1, 2])
def test_device_species_out_of_range_is_refused(bad_index):
    """A species index outside [0, nspecies) in a DEVICE array is refused by
    the loading kernel (which stores 0 in its place, so no kernel ever
    indexes the species tables with it): PIC_EARG, and the context is left
    empty and unstarted, so a step before a valid load and pic_start is
    refused with PIC_ESTATE."""
    import torch
    cfg = small_2d()
    assert len(cfg["species"]) == 1
    s = make_gpu(cfg)
    s.start()
    dev = lambda a, t=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=t,
                                                     device="cuda")
    sp = np.zeros(cfg["w"].shape[0], np.int32)
    sp[len(sp) // 3] = bad_index
    with pytest.raises(pic.PicError) as ei:
        s.set_particles(dev(cfg["x"]), dev(cfg["u"]), dev(cfg["w"]), dev(sp, torch.int32),
                        on_device=True)
    assert ei.value.code == pic.PIC_EARG
    assert s.num_particles() == 0
    with pytest.raises(pic.PicError) as ei:
        s.step(1e-12)
    assert ei.value.code == pic.PIC_ESTATE
    # a valid load afterwards works as usual
    s.set_particles(cfg["x"], cfg["u"], cfg["w"], cfg["sp"])
    s.set_potentials(cfg["A"], cfg["U"])
    s.start()
    assert s.step(1e-12)["status"] == 0
    s.close()
