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

* ``state_after(sim, tol, steps, x, P, f)``: the state after ``steps``
  implicit steps from the state (x, P, f) (positions, canonical momenta and
  the potentials packed as [phi, psi, A, U, rho]), as tensors; its reverse
  mode is a sweep of ``pic_step_vjp`` over the checkpoint images the forward
  pass keeps, so one backward pass gives the gradient with respect to every
  particle and every mesh value.

Argument marshalling only: every derivative is computed by the library.
Tensors on the GPU go to the library as device pointers (no host copy);
tensors on the host (and simulations without device calls) go through the
host-array calls.
"""
from __future__ import annotations

import numpy as np
import torch


def _on_device(sim, t: torch.Tensor) -> bool:
    return t.is_cuda and hasattr(sim, "eval_map_device")


def _host(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy().astype(np.float64)


def _check(rc):
    if rc:
        raise RuntimeError(f"map evaluation failed with status {rc}")


class _MapEval(torch.autograd.Function):
    @staticmethod
    def forward(j, sim, tol):
        if _on_device(sim, j):
            rc, H = sim.eval_map_device(j, tol)
            _check(rc)
            return H
        rc, H, _, _, _ = sim.eval_map(_host(j), tol)
        _check(rc)
        return torch.from_numpy(H).to(j.device)

    @staticmethod
    def setup_context(ctx, inputs, output):
        j, sim, tol = inputs
        ctx.sim, ctx.tol = sim, tol
        ctx.dev = _on_device(sim, j)
        ctx.j = j.detach().clone() if ctx.dev else _host(j)

    @staticmethod
    def jvp(ctx, dj, _dsim, _dtol):
        if ctx.dev:
            rc, _, dH = ctx.sim.eval_map_jvp_device(ctx.j, dj, ctx.tol)
            _check(rc)
            return dH
        rc, _, dH = ctx.sim.eval_map_jvp(ctx.j, _host(dj), ctx.tol)
        _check(rc)
        return torch.from_numpy(dH).to(dj.device)

    @staticmethod
    def backward(ctx, gH):
        if ctx.dev:
            rc, _, jbar = ctx.sim.eval_map_vjp_device(ctx.j, gH, ctx.tol)
            _check(rc)
            return jbar, None, None
        rc, _, jbar = ctx.sim.eval_map_vjp(ctx.j, _host(gH), ctx.tol)
        _check(rc)
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


FIELD_PARTS = (("phi", 1), ("psi", 1), ("A", 3), ("U", 3), ("rho", 1))


def pack_fields(f: dict, Ng: int) -> np.ndarray:
    """{phi, psi, A, U, rho} -> one array of 9 Ng values (that order)."""
    return np.concatenate([np.asarray(f[k], np.float64).reshape(nc * Ng) for k, nc in FIELD_PARTS])


def unpack_fields(a: np.ndarray, Ng: int) -> dict:
    out, off = {}, 0
    for k, nc in FIELD_PARTS:
        out[k] = np.array(a[off:off + nc * Ng], np.float64)
        off += nc * Ng
    return out


class _StateAfter(torch.autograd.Function):
    @staticmethod
    def forward(x, P, f, sim, tol, steps):
        if steps < 1:
            raise ValueError("state_after needs at least one step")
        if x.is_cuda and hasattr(sim, "particles_device"):
            return _state_after_device(x, P, f, sim, tol, steps)
        _, _, w, sp = sim.particles()
        seed = sim.fields()["J"]
        E0 = sim.checkpoint_header()["E0"]
        fields = unpack_fields(f.detach().cpu().numpy(), sim.Ng)
        fields["J"] = seed
        sim.set_state(x.detach().cpu().numpy(), P.detach().cpu().numpy(), w, sp, fields, E0)
        images = []
        for _ in range(steps):
            images.append(sim.checkpoint())
            r = sim.step(tol)
            if r["status"]:
                raise RuntimeError(f"step failed with status {r['status']}")
        x1, P1, _, _ = sim.particles()
        f1 = pack_fields(sim.fields(), sim.Ng)
        sim._autograd_images = images  # kept for the backward sweep
        dev = x.device
        return (torch.from_numpy(x1).to(dev), torch.from_numpy(P1).to(dev),
                torch.from_numpy(f1).to(dev))

    @staticmethod
    def setup_context(ctx, inputs, output):
        _, _, _, sim, tol, steps = inputs
        ctx.sim, ctx.tol = sim, tol
        ctx.images = sim._autograd_images
        del sim._autograd_images

    @staticmethod
    def backward(ctx, gx, gP, gf):
        sim = ctx.sim
        final = sim.checkpoint()
        if gx.is_cuda and hasattr(sim, "step_vjp_device"):
            for img in reversed(ctx.images):
                sim.restore(img)
                gx, gP, gf = sim.step_vjp_device(ctx.tol, gx, gP, gf)
            sim.restore(final)
            return gx, gP, gf, None, None, None
        g = {"x": gx.detach().cpu().numpy(), "P": gP.detach().cpu().numpy(),
             "fields": unpack_fields(gf.detach().cpu().numpy(), sim.Ng)}
        for img in reversed(ctx.images):
            sim.restore(img)
            g = sim.step_vjp(ctx.tol, g["x"], g["P"], g["fields"])
        sim.restore(final)
        dev = gx.device
        return (torch.from_numpy(g["x"]).to(dev), torch.from_numpy(g["P"]).to(dev),
                torch.from_numpy(pack_fields(g["fields"], sim.Ng)).to(dev), None, None, None)


def _state_after_device(x, P, f, sim, tol, steps):
    """The forward pass of state_after on device tensors: the state goes in
    and comes out through the library's device-pointer calls."""
    _, _, w, sp = sim.particles_device()
    J = sim.fields_device()["J"]
    E0 = sim.checkpoint_header()["E0"]
    Ng = sim.Ng
    fc = f.detach().to(torch.float64).contiguous()
    fields, off = {}, 0
    for k, nc in FIELD_PARTS:
        fields[k] = fc[off:off + nc * Ng]
        off += nc * Ng
    fields["J"] = J
    torch.cuda.current_stream().synchronize()
    sim.set_state(x.detach().contiguous(), P.detach().contiguous(), w, sp, fields, E0,
                  on_device=True)
    images = []
    for _ in range(steps):
        images.append(sim.checkpoint())
        r = sim.step(tol)
        if r["status"]:
            raise RuntimeError(f"step failed with status {r['status']}")
    x1, P1, _, _ = sim.particles_device()
    f1 = sim.fields_device()
    sim._autograd_images = images  # kept for the backward sweep
    return x1, P1, torch.cat([f1[k].reshape(-1) for k, _ in FIELD_PARTS])


def state_after(sim, tol: float, steps: int, x: torch.Tensor, P: torch.Tensor, f: torch.Tensor):
    """(x, P, f) after ``steps`` steps of the started FP64 simulation ``sim``
    from the state (x, P, f); differentiable in all three (reverse mode).

    x: dim x N positions, P: 3 x N canonical momenta (load order), f: the
    9 Ng potentials [phi, psi, A, U, rho] as ``pack_fields`` packs
    ``sim.fields()``.  Weights, species and the reference energy are the
    simulation's own; the simulation is left in the final state."""
    return _StateAfter.apply(x, P, f, sim, tol, steps)
