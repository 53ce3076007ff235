"""The torch.autograd wrappers (paper_2609_36383_b300.autograd) marshal the
library's derivatives correctly: checked on the CPU against a stand-in
simulation whose map is affine and whose energies are closed forms, so that
torch's own forward and reverse modes have exact answers."""
import numpy as np
import pytest
import torch
import torch.autograd.forward_ad as fwAD

from paper_2609_36383_b300 import autograd as pa


class _AffineMap:
    """H(j) = M j + c, with the JVP M dj."""

    def __init__(self, n=12, seed=0):
        rng = np.random.default_rng(seed)
        self.M = rng.standard_normal((n, n))
        self.c = rng.standard_normal(n)

    def eval_map(self, j, tol):
        return 0, self.M @ j + self.c, None, None, None

    def eval_map_jvp(self, j, dj, tol):
        return 0, self.M @ j + self.c, self.M @ dj

    def eval_map_vjp(self, j, ybar, tol):
        return 0, self.M @ j + self.c, self.M.T @ ybar


class _Run:
    """W(theta) = theta^3, K(theta) = sin(theta) after any number of steps,
    with their derivatives as the tangent."""

    def __init__(self, theta):
        self.theta = theta
        self.seeded = False

    def tangent_begin(self, **seed):
        assert set(seed) == {"du"}
        self.seeded = True

    def step(self, tol):
        return dict(status=0, W=self.theta ** 3, K=np.sin(self.theta))

    def tangent(self):
        assert self.seeded
        return dict(dW=3 * self.theta ** 2, dK=np.cos(self.theta))


def test_map_eval_forward_mode_is_the_jvp_and_reverse_mode_the_vjp():
    sim = _AffineMap()
    j = torch.randn(12, dtype=torch.float64)
    dj = torch.randn(12, dtype=torch.float64)
    with fwAD.dual_level():
        H, dH = fwAD.unpack_dual(pa.map_eval(sim, fwAD.make_dual(j, dj), 1e-12))
    assert torch.allclose(H, torch.from_numpy(sim.M @ j.numpy() + sim.c), atol=1e-13)
    assert torch.allclose(dH, torch.from_numpy(sim.M @ dj.numpy()), atol=1e-13)
    jr = j.clone().requires_grad_(True)
    w = torch.randn(12, dtype=torch.float64)
    (w * pa.map_eval(sim, jr, 1e-12)).sum().backward()
    assert torch.allclose(jr.grad, torch.from_numpy(sim.M.T @ w.numpy()), atol=1e-13)


def test_energies_after_reverse_and_forward_modes():
    theta = torch.tensor(0.7, dtype=torch.float64, requires_grad=True)
    out = pa.energies_after(theta, _Run, lambda th: dict(du=np.zeros(3)), 5, 1e-12)
    assert torch.allclose(out, torch.tensor([0.7 ** 3, np.sin(0.7)], dtype=torch.float64))
    (2.0 * out[0] + 3.0 * out[1]).backward()
    assert abs(theta.grad.item() - (2 * 3 * 0.7 ** 2 + 3 * np.cos(0.7))) < 1e-14
    with fwAD.dual_level():
        th = fwAD.make_dual(torch.tensor(0.7, dtype=torch.float64),
                            torch.tensor(2.0, dtype=torch.float64))
        _, t = fwAD.unpack_dual(pa.energies_after(th, _Run, lambda x: dict(du=np.zeros(3)), 5,
                                                  1e-12))
    assert torch.allclose(t, torch.tensor([2 * 3 * 0.7 ** 2, 2 * np.cos(0.7)],
                                          dtype=torch.float64))
    with pytest.raises(ValueError):
        pa.energies_after(theta, _Run, lambda th: dict(du=np.zeros(3)), 0, 1e-12)


class _LinearSteps:
    """A stand-in simulation whose step is S' = M S on the flattened state
    (x, P, f), with pic_step_vjp's counterpart S_bar = M^T S_bar'."""

    def __init__(self, dim=1, N=5, Ng=4, seed=3):
        rng = np.random.default_rng(seed)
        self.dim, self.N, self.Ng = dim, N, Ng
        self.sizes = (dim * N, 3 * N, 9 * Ng)
        n = sum(self.sizes)
        self.M = np.eye(n) + 0.1 * rng.standard_normal((n, n))
        self.S = rng.standard_normal(n)

    def _split(self, S):
        a, b, _ = self.sizes
        return (S[:a].reshape(self.dim, self.N), S[a:a + b].reshape(3, self.N),
                pa.unpack_fields(S[a + b:], self.Ng))

    def _join(self, x, P, f):
        return np.concatenate([np.ravel(x), np.ravel(P), pa.pack_fields(f, self.Ng)])

    def particles(self):
        x, P, _ = self._split(self.S)
        return x, P, np.ones(self.N), np.zeros(self.N, np.int32)

    def fields(self):
        f = self._split(self.S)[2]
        f["J"] = np.zeros(3 * self.Ng)
        return f

    def checkpoint_header(self):
        return {"E0": 1.0}

    def set_state(self, x, P, w, sp, fields, E0):
        self.S = self._join(x, P, fields)

    def checkpoint(self):
        return self.S.tobytes()

    def restore(self, img):
        self.S = np.frombuffer(img).copy()

    def step(self, tol):
        self.S = self.M @ self.S
        return {"status": 0}

    def step_vjp(self, tol, xb, Pb, fb):
        x, P, f = self._split(self.M.T @ self._join(xb, Pb, fb))
        return {"x": x, "P": P, "fields": f, "gmres_iters": 0}


def test_state_after_reverse_mode_chains_the_step_adjoint():
    sim = _LinearSteps()
    rng = np.random.default_rng(8)
    x0, P0, _, _ = sim.particles()
    f0 = pa.pack_fields(sim.fields(), sim.Ng)
    S0 = np.concatenate([x0.ravel(), P0.ravel(), f0])
    x = torch.tensor(x0, requires_grad=True)
    P = torch.tensor(P0, requires_grad=True)
    f = torch.tensor(f0, requires_grad=True)
    steps = 3
    x3, P3, f3 = pa.state_after(sim, 1e-12, steps, x, P, f)
    M3 = np.linalg.matrix_power(sim.M, steps)
    S3 = M3 @ S0
    assert np.allclose(np.concatenate([x3.detach().numpy().ravel(), P3.detach().numpy().ravel(),
                                       f3.detach().numpy()]), S3, rtol=1e-13, atol=1e-13)
    c = [torch.from_numpy(rng.standard_normal(t.shape)) for t in (x3, P3, f3)]
    loss = sum((ci * t).sum() for ci, t in zip(c, (x3, P3, f3)))
    loss.backward()
    g = M3.T @ np.concatenate([ci.numpy().ravel() for ci in c])
    got = np.concatenate([x.grad.numpy().ravel(), P.grad.numpy().ravel(), f.grad.numpy()])
    assert np.allclose(got, g, rtol=1e-12, atol=1e-12)
    # the simulation is left in the final state
    assert np.allclose(sim.S, S3, rtol=1e-13, atol=1e-13)
