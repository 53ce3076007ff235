"""Particles loaded in the stored form (pic_set_particles_local: nearest node
plus offset, Sec. 2.4) on the CUDA path.

- The same particles given as absolute positions and as (node, offset) pairs
  computed the way the library computes them load the same state: the
  exported positions agree bit for bit, and one step gives the same report.
- An index or offset out of range is refused with PIC_EARG, from host arrays
  before any copy and from device arrays by the loading kernel (which stores
  node 0, offset 0 in its place, so no kernel indexes the mesh with it); the
  context is then empty and unstarted.
"""
import numpy as np
import pytest

import paper_2609_36383_b300 as pic
from tests._common import make_gpu, small_2d

pytestmark = pytest.mark.gpu


def _stored_form(cfg):
    """(node, offset) of every particle, with the arithmetic of the loader."""
    d = cfg["dim"]
    x = np.asarray(cfg["x"], np.float64).reshape(d, -1)
    cell = np.zeros(x.shape, np.int32)
    off = np.zeros(x.shape)
    for l in range(d):
        dx = cfg["L"][l] / cfg["n"][l]
        u = (x[l] - cfg["x0"][l]) * (1.0 / dx)
        nn = float(cfg["n"][l])
        u = u - nn * np.floor(u / nn)
        c = np.floor(u + 0.5)
        off[l] = u - c
        c[c >= cfg["n"][l]] -= cfg["n"][l]
        cell[l] = c.astype(np.int32)
    return cell, off


def test_local_load_matches_absolute_positions():
    cfg = small_2d()
    a = make_gpu(cfg)
    b = pic.Simulation(cfg["dim"], cfg["n"], cfg["L"], cfg["x0"], cfg["species"], cfg["dt"],
                       rho_bg=cfg["rho_bg"])
    cell, off = _stored_form(cfg)
    b.set_particles_local(cell, off, cfg["u"], cfg["w"], cfg["sp"])
    b.set_potentials(cfg["A"], cfg["U"])
    ra0, rb0 = a.start(), b.start()
    xa, Pa, _, _ = a.particles()
    xb, Pb, _, _ = b.particles()
    assert np.array_equal(xa, xb) and np.array_equal(Pa, Pb)
    ra, rb = a.step(1e-12), b.step(1e-12)
    assert ra["status"] == 0 and rb["status"] == 0
    for k in ("K", "W", "E_tot"):
        assert rb0[k] == pytest.approx(ra0[k], rel=1e-13)
        assert rb[k] == pytest.approx(ra[k], rel=1e-12)
    a.close()
    b.close()


@pytest.mark.parametrize("where", ["host", "device"])
@pytest.mark.parametrize("bad", ["cell_high", "cell_negative", "offset_half", "offset_nan"])
def test_local_load_refuses_out_of_range(where, bad):
    import torch
    cfg = small_2d()
    cell, off = _stored_form(cfg)
    i = cell.shape[1] // 2
    if bad == "cell_high":
        cell[1, i] = cfg["n"][1]
    elif bad == "cell_negative":
        cell[0, i] = -1
    elif bad == "offset_half":
        off[0, i] = 0.5
    else:
        off[1, i] = np.nan
    s = pic.Simulation(cfg["dim"], cfg["n"], cfg["L"], cfg["x0"], cfg["species"], cfg["dt"],
                       rho_bg=cfg["rho_bg"])
    args = [cell, off, np.asarray(cfg["u"], np.float64), np.asarray(cfg["w"], np.float64)]
    if where == "device":
        args = [torch.as_tensor(np.ascontiguousarray(a), device="cuda") for a in args]
    with pytest.raises(pic.PicError) as ei:
        s.set_particles_local(*args, on_device=(where == "device"))
    assert ei.value.code == pic.PIC_EARG
    assert s.num_particles() == 0
    # a valid load afterwards works as usual
    s.set_particles(cfg["x"], cfg["u"], cfg["w"], cfg["sp"])
    s.set_potentials(cfg["A"], cfg["U"])
    s.start()
    assert s.step(1e-12)["status"] == 0
    s.close()
