"""torch.autograd wrappers of the library's derivatives.

* ``map_eval(sim, j, tol)``: H(j) = P J_orb(j) of Sec. 4.5 as a function of
  the trial current; its forward-mode derivative (``torch.autograd.forward_ad``
  dual tensors) is ``pic_eval_map_jvp``, its reverse mode (``backward``)
  ``pic_eval_map_vjp``.
* ``energies_after(theta, make, seed, steps, tol)``: (W, K) after ``steps``
  implicit steps of the started simulation ``make(theta)`` as a function of
  one scalar parameter theta of the initial condition; ``seed(theta)`` gives
  d(u, A, U)/d theta.  The forward pass carries the step tangent
  (``pic_tangent_begin`` / ``pic_get_tangent``), so both the forward- and
  the reverse-mode derivative of this scalar-input function are exact
  products with d(W, K)/d theta.

Argument marshalling only: every derivative is computed by the library.
"""
from __future__ import annotations

import numpy as np
import torch


class _MapEval(torch.autograd.Function):
    @staticmethod
    def forward(j, sim, tol):
        rc, H, _, _, _ = sim.eval_map(j.detach().cpu().numpy().astype(np.float64), tol)
        if rc:
            raise RuntimeError(f"map evaluation failed with status {rc}")
        return torch.from_numpy(H).to(j.device)

    @staticmethod
    def setup_context(ctx, inputs, output):
        j, sim, tol = inputs
        ctx.sim, ctx.tol = sim, tol
        ctx.j = j.detach().cpu().numpy().astype(np.float64)

    @staticmethod
    def jvp(ctx, dj, _dsim, _dtol):
        rc, _, dH = ctx.sim.eval_map_jvp(ctx.j, dj.detach().cpu().numpy().astype(np.float64),
                                         ctx.tol)
        if rc:
            raise RuntimeError(f"map evaluation failed with status {rc}")
        return torch.from_numpy(dH).to(dj.device)

    @staticmethod
    def backward(ctx, gH):
        rc, _, jbar = ctx.sim.eval_map_vjp(ctx.j, gH.detach().cpu().numpy().astype(np.float64),
                                           ctx.tol)
        if rc:
            raise RuntimeError(f"map evaluation failed with status {rc}")
        return torch.from_numpy(jbar).to(gH.device), None, None


def map_eval(sim, j: torch.Tensor, tol: float) -> torch.Tensor:
    """H(j) (float64, 3 * Ng) with forward-mode derivative H'(j) dj."""
    return _MapEval.apply(j, sim, tol)


class _EnergiesAfter(torch.autograd.Function):
    @staticmethod
    def forward(theta, make, seed, steps, tol):
        if steps < 1:
            raise ValueError("energies_after needs at least one step")
        th = float(theta)
        sim = make(th)
        sim.tangent_begin(**seed(th))
        for _ in range(steps):
            r = sim.step(tol)
            if r["status"]:
                raise RuntimeError(f"step failed with status {r['status']}")
        t = sim.tangent()
        out = torch.tensor([r["W"], r["K"]], dtype=torch.float64)
        jac = torch.tensor([t["dW"], t["dK"]], dtype=torch.float64)
        return out, jac

    @staticmethod
    def setup_context(ctx, inputs, output):
        ctx.jac = output[1].detach()
        ctx.mark_non_differentiable(output[1])

    @staticmethod
    def backward(ctx, g_out, _g_jac):
        return (g_out * ctx.jac).sum(), None, None, None, None

    @staticmethod
    def jvp(ctx, dtheta, _dmake, _dseed, _dsteps, _dtol):
        return ctx.jac * dtheta, None


def energies_after(theta: torch.Tensor, make, seed, steps: int, tol: float) -> torch.Tensor:
    """(W, K) after ``steps`` steps, differentiable in the scalar ``theta``.

    make(theta) -> a started Simulation (FP64, quadratic shapes);
    seed(theta) -> dict(du=..., dA=..., dU=...) of d/d theta of the initial
    condition (any may be omitted)."""
    out, _ = _EnergiesAfter.apply(theta, make, seed, steps, tol)
    return out
