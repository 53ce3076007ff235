"""The forward sensitivity of the step (pic_tangent_*) on the CUDA path.

The tangent is the derivative of the exact fixed point of every step
(implicit differentiation of j = H(j; S)), carried over many steps.  It is
checked against what does not depend on it:
  * d(W after 50 steps)/d(u0) for the 1D two-stream (u0 = the beams' drift)
    against central differences with h = 1e-6 of the GPU path and of the FP64
    oracle (the oracle's own gradient);
  * the energy theorem: E_tot = K + W is conserved by every converged step
    for every initial condition, so its tangent dK + dW is constant;
  * the tangent state (dx, dP, dA, dU) after steps against central
    differences of the state, in 2D and 3D, with potentials in the seed and
    with a sort between steps (the tangents travel with their particles).

Tolerances: the steps converge to tol = 1e-12 (relative); a difference
quotient with step h divides that error by h, so central differences agree
with the exact derivative to about 1e-12 / h = 1e-6 relative, more where the
quantity's net value is a small part of its gross terms; the bounds are 2e-4
(energies over 50 unstable steps) and 2e-5 (state after two steps).
"""
import numpy as np
import pytest

import pic_inputs
from tests._common import make_gpu, make_oracle, periodic_diff, small_2d

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2609_36383_b300 import build
    build.build()
    import oracle
    oracle.build()


U0 = 0.6
STEPS = 50


def _two_stream(u0):
    return pic_inputs.two_stream_1d(nx=64, ppc_beam=32, u0=u0)


def _du(u0, delta=1e-6):
    """d u / d u0 of the input generator (it is linear in u0)."""
    return (_two_stream(u0 + delta)["u"] - _two_stream(u0 - delta)["u"]) / (2 * delta)


def _run_W(make, u0, tol):
    cfg = _two_stream(u0)
    s = make(cfg)
    s.start()
    for _ in range(STEPS):
        r = s.step(tol)
        assert r["status"] == 0
    return r["W"]


@pytest.fixture(scope="module")
def tangent_run():
    cfg = _two_stream(U0)
    tol = cfg["tol"]
    s = make_gpu(cfg)
    r0 = s.start()
    s.tangent_begin(du=_du(U0))
    t0 = s.tangent()
    dE = [t0["dK"] + t0["dW"]]
    iters = []
    for _ in range(STEPS):
        r = s.step(tol)
        assert r["status"] == 0
        t = s.tangent()
        dE.append(t["dK"] + t["dW"])
        iters.append(t["gmres_iters"])
    return dict(tol=tol, W=r["W"], K0=r0["K"], t=t, dE=np.array(dE), iters=iters,
                t0=t0)


def test_tangent_of_50_step_field_energy_matches_central_differences(tangent_run):
    tr = tangent_run
    h = 1e-6
    tol = tr["tol"]
    fd_gpu = (_run_W(make_gpu, U0 + h, tol) - _run_W(make_gpu, U0 - h, tol)) / (2 * h)
    fd_orc = (_run_W(make_oracle, U0 + h, tol) - _run_W(make_oracle, U0 - h, tol)) / (2 * h)
    dW = tr["t"]["dW"]
    print(f"dW50/du0: tangent {dW:.10e}, GPU central difference {fd_gpu:.10e}, "
          f"oracle central difference {fd_orc:.10e}; GMRES iterations per step "
          f"{np.mean(tr['iters']):.1f} (max {max(tr['iters'])})")
    assert abs(dW) > 0
    assert abs(dW - fd_gpu) < 2e-4 * abs(dW)
    assert abs(dW - fd_orc) < 2e-4 * abs(dW)


def test_tangent_of_total_energy_is_conserved(tangent_run):
    """E_tot(n) = E_tot(0) for every u0, so dK + dW stays at its step-0 value."""
    dE = tangent_run["dE"]
    t0 = tangent_run["t0"]
    scale = abs(t0["dK"]) + abs(t0["dW"])
    print(f"dE_tot/du0 at step 0: {dE[0]:.12e}; max drift over {STEPS} steps "
          f"{np.abs(dE - dE[0]).max() / scale:.2e} of |dK| + |dW|")
    assert np.abs(dE - dE[0]).max() < 1e-9 * scale


def _state(s):
    x, P, _, _ = s.particles()
    f = s.fields()
    return x, P, f["A"], f["U"]


def _cases():
    c2 = small_2d()
    c3 = pic_inputs.thermal_box(dim=3, n=8, ppc=2, T=0.05, u_drift=0.3, dt=0.2, seed=4)
    return {"2d_weibel": c2, "3d_thermal": c3}


@pytest.mark.parametrize("name", ["2d_weibel", "3d_thermal"])
def test_tangent_state_matches_central_differences(name):
    cfg = _cases()[name]
    rng = np.random.default_rng(7)
    N = cfg["u"].shape[1]
    Ng = int(np.prod(cfg["n"]))
    du = rng.standard_normal((3, N)) * np.abs(cfg["u"]).max()
    dA = pic_inputs.random_fields(rng, Ng, scale=1e-2)
    dU = pic_inputs.random_fields(rng, Ng, scale=1e-2)
    tol, nsteps, h = 1e-12, 2, 1e-6

    A0 = np.zeros((3, Ng)) if cfg["A"] is None else cfg["A"]
    U0 = np.zeros((3, Ng)) if cfg["U"] is None else cfg["U"]

    def run(eps, tangent=False):
        c = dict(cfg)
        c["u"] = cfg["u"] + eps * du
        c["A"] = A0 + eps * dA
        c["U"] = U0 + eps * dU
        s = make_gpu(c, sort_every=1)
        s.start()
        if tangent:
            s.tangent_begin(du=du, dA=dA, dU=dU)
        for _ in range(nsteps):
            assert s.step(tol)["status"] == 0
        return s

    s = run(0.0, tangent=True)
    t = s.tangent()
    xp, Pp, Ap, Up = _state(run(h))
    xm, Pm, Am, Um = _state(run(-h))
    fd_x = periodic_diff(xp, xm, cfg["L"]) / (2 * h)
    fd = {"dx": fd_x, "dP": (Pp - Pm) / (2 * h), "dA": (Ap - Am) / (2 * h),
          "dU": (Up - Um) / (2 * h)}
    for k, v in fd.items():
        err = np.abs(t[k] - v).max() / np.abs(v).max()
        print(f"{name} {k}: max |tangent - central difference| = {err:.2e} of max |.|")
        assert err < 2e-5, k


def test_tangent_end_and_restart_release_it():
    cfg = small_2d()
    s = make_gpu(cfg)
    s.start()
    s.tangent_begin(du=np.zeros((3, cfg["u"].shape[1])))
    assert s.step(1e-12)["status"] == 0
    t = s.tangent()
    assert np.abs(t["dP"]).max() == 0 and t["dW"] == 0 and t["gmres_iters"] == 0
    s.tangent_end()
    with pytest.raises(RuntimeError):
        s.tangent()


def test_autograd_wrappers_use_the_library_derivatives(tangent_run):
    """torch.autograd: reverse mode of energies_after and both modes of
    map_eval reproduce the library's tangent, JVP and VJP."""
    import torch
    import torch.autograd.forward_ad as fwAD
    from paper_2609_36383_b300 import autograd as pa

    def make(u0):
        s = make_gpu(_two_stream(u0))
        s.start()
        return s

    theta = torch.tensor(U0, dtype=torch.float64, requires_grad=True)
    out = pa.energies_after(theta, make, lambda u0: dict(du=_du(u0)), STEPS, tangent_run["tol"])
    out[0].backward()
    assert abs(theta.grad.item() - tangent_run["t"]["dW"]) <= 1e-12 * abs(tangent_run["t"]["dW"])
    # two runs differ in the summation order of the deposit atomics only
    assert abs(out[0].item() - tangent_run["W"]) <= 1e-10 * abs(tangent_run["W"])
    # forward mode through one map evaluation
    cfg = small_2d()
    s = make_gpu(cfg)
    s.start()
    j = torch.from_numpy(s.fields()["J"].copy())
    dj = torch.from_numpy(np.random.default_rng(1).standard_normal(j.shape[0]) * 1e-3)
    with fwAD.dual_level():
        H, dH = fwAD.unpack_dual(pa.map_eval(s, fwAD.make_dual(j, dj), 1e-14))
    st, H_ref, dH_ref = s.eval_map_jvp(j.numpy(), dj.numpy(), 1e-14)
    assert st == 0
    assert np.abs(H.numpy() - H_ref).max() <= 1e-12 * np.abs(H_ref).max()
    assert np.abs(dH.numpy() - dH_ref).max() <= 1e-12 * np.abs(dH_ref).max()
    # reverse mode through one map evaluation
    jr = j.clone().requires_grad_(True)
    yb = torch.from_numpy(np.random.default_rng(2).standard_normal(j.shape[0]))
    (yb * pa.map_eval(s, jr, 1e-14)).sum().backward()
    st, _, jbar_ref = s.eval_map_vjp(j.numpy(), yb.numpy(), 1e-14)
    assert st == 0
    assert np.abs(jr.grad.numpy() - jbar_ref).max() <= 1e-12 * np.abs(jbar_ref).max()
