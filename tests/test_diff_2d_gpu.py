"""The drift gradient of the differentiation workload on the CUDA path.

Workload: 2D3V two-stream on 256^2 cells (box of side 4 pi), 100 particles
per cell (6,553,600), beams u_x = +-0.8 with Maxwell-Juettner T = 1e-3,
dt = 0.05.  The quantity is the field energy W after 50 steps and the
parameter the beam drift: each beam's x proper velocity moves with it,
u_x -> u_x + h s (s = +1 for the forward beam, -1 for the backward one).
The forward sensitivity carried through every step (pic_tangent_begin with
du = (s, 0, 0); implicit differentiation of each step's fixed point, GMRES on
FP64 dual-number Jacobian-vector products) must equal the central difference
(W(+h) - W(-h)) / 2h at h = 1e-6 of two runs of the same GPU path, and the
tangent of the total energy must stay at its initial value (the energy
theorem holds for every initial condition).  The steps converge to 1e-12,
so the difference quotient's solver noise (about 1e-12 of W over 2h) stays
far below the bound.  About two minutes on a B300.
"""
import numpy as np
import pytest

import paper_2609_36383_b300 as pic
import pic_inputs
from tests._common import make_gpu

pytestmark = pytest.mark.gpu

STEPS, TOL, H = 50, 1e-12, 1e-6


def _run(cfg, du=None, h=0.0):
    c = dict(cfg)
    if h:
        c["u"] = cfg["u"].copy()
        c["u"][0] += h * cfg["beam"]
    s = make_gpu(c)
    r0 = s.start()
    if du is not None:
        s.tangent_begin(du=du)
    for st in range(STEPS):
        r = s.step(TOL)
        assert r["status"] == 0, (st, r)
    out = dict(W=r["W"], E0=r0["E_tot"], dE=r["rel_dE"])
    if du is not None:
        t = s.tangent()
        out.update(dW=t["dW"], dK=t["dK"])
        s.tangent_end()
    s.close()
    return out


def test_drift_gradient_of_field_energy_after_50_steps():
    cfg = pic_inputs.two_stream_2d()
    du = np.zeros((3, cfg["w"].shape[0]))
    du[0] = cfg["beam"]
    tan = _run(cfg, du=du)
    wp = _run(cfg, h=H)["W"]
    wm = _run(cfg, h=-H)["W"]
    fd = (wp - wm) / (2 * H)
    rel = abs(tan["dW"] - fd) / abs(fd)
    print(f"d W(50 steps) / d drift: tangent {tan['dW']:.10e}, central difference (h = {H}) "
          f"{fd:.10e}, relative difference {rel:.2e}; W = {tan['W']:.6e}, "
          f"|dE/E| {abs(tan['dE']):.1e}, dK + dW = {tan['dK'] + tan['dW']:.3e}")
    assert rel < 1e-4
    assert abs(tan["dE"]) < 1e-11
