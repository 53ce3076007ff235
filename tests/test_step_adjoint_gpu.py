"""The adjoint of a step (pic_step_vjp) on the CUDA path.

  * One step, 1D/2D/3D: for a random linear functional L = <c, S'> of the
    state after the step (positions, momenta and all five potentials) and a
    random direction dS of the state before it, <Sbar, dS> from the adjoint
    equals the central difference (L(S + h dS) - L(S - h dS)) / 2h, h = 1e-6.
    The steps converge to tol = 1e-12, so the difference quotient carries
    about 1e-12 / h = 1e-6 of the state's size as noise; the bound is 1e-5 of
    the sum of the magnitudes of its terms.
  * Twenty steps of the 1D two-stream instability, reverse sweep over saved
    checkpoint images (Simulation.run_adjoint): the gradient with respect to
    every initial momentum, dotted with the momentum change m du of a drift
    change du, equals the forward sensitivity (pic_tangent_*) of the same
    functional in the same direction.  Both are exact derivatives of the
    discrete step up to the solves' tolerances, so the bound is 1e-8 of the
    functional's gross size.
  * The same functional and directions against central differences of the
    FP64 oracle's step (an implementation that shares no code with the CUDA
    path), with the same bound.
  * The state is unchanged by the call; unsupported contexts are refused.
"""
import numpy as np
import pytest

import paper_2609_36383_b300 as pic
import pic_inputs
from tests._common import make_gpu, make_oracle, periodic_diff, small_1d, small_2d

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2609_36383_b300 import build
    build.build()


def _thermal_3d():
    return pic_inputs.thermal_box(dim=3, n=8, ppc=2, T=0.05, u_drift=0.3, dt=0.2, seed=4)


CASES = {"1d_two_stream": small_1d, "2d_weibel": small_2d, "3d_thermal": _thermal_3d}
TOL = 1e-12
FIELDS = ("phi", "psi", "A", "U", "rho")


def _read(s):
    x, P, _, _ = s.particles()
    return x, P, s.fields()


def _scale(a):
    m = np.abs(a).max()
    return m if m > 0 else 1.0


@pytest.mark.parametrize("name", sorted(CASES))
def test_step_adjoint_matches_central_differences(name):
    cfg = CASES[name]()
    rng = np.random.default_rng(11)
    s = make_gpu(cfg)
    s.start()
    assert s.step(TOL)["status"] == 0  # a generic state: every potential nonzero
    x0, P0, w, sp = s.particles()
    f0 = s.fields()
    E0 = pic.inspect_checkpoint(s.checkpoint())["E0"]
    dxc = np.asarray(cfg["L"][:cfg["dim"]], float) / np.asarray(cfg["n"][:cfg["dim"]], float)
    dx = rng.standard_normal(x0.shape) * dxc[:, None]
    dP = rng.standard_normal(P0.shape) * _scale(P0)
    df = {k: rng.standard_normal(f0[k].shape) * _scale(f0[k]) for k in FIELDS}
    cx = rng.standard_normal(x0.shape)
    cP = rng.standard_normal(P0.shape)
    cf = {k: rng.standard_normal(f0[k].shape) for k in FIELDS}

    def load(eps):
        f = dict(f0)
        for k in FIELDS:
            f[k] = f0[k] + eps * df[k]
        s.set_state(x0 + eps * dx, P0 + eps * dP, w, sp, f, E0)

    load(0.0)
    img = s.checkpoint()
    g = s.step_vjp(TOL, cx, cP, cf)
    assert s.checkpoint() == img  # the state is unchanged
    lhs_terms = [np.sum(g["x"] * dx), np.sum(g["P"] * dP)] + \
                [np.sum(g["fields"][k] * df[k]) for k in FIELDS]
    h = 1e-6
    out = {}
    for sgn in (1, -1):
        load(sgn * h)
        assert s.step(TOL)["status"] == 0
        out[sgn] = _read(s)
    (xp, Pp, fp), (xm, Pm, fm) = out[1], out[-1]
    fd_terms = [np.sum(cx * periodic_diff(xp, xm, cfg["L"])) / (2 * h),
                np.sum(cP * (Pp - Pm)) / (2 * h)] + \
               [np.sum(cf[k] * (fp[k] - fm[k])) / (2 * h) for k in FIELDS]
    gross = sum(abs(t) for t in fd_terms) + sum(abs(t) for t in lhs_terms)
    lhs, fd = sum(lhs_terms), sum(fd_terms)
    print(f"{name}: <Sbar, dS> {lhs:.10e}, central difference {fd:.10e}, "
          f"|diff| / gross {abs(lhs - fd) / gross:.2e}, GMRES applications {g['gmres_iters']}; "
          f"terms adjoint {np.array(lhs_terms)}, FD {np.array(fd_terms)}")
    assert abs(lhs - fd) <= 1e-5 * gross


@pytest.mark.parametrize("name", sorted(CASES))
def test_step_adjoint_matches_oracle_central_differences(name):
    import oracle
    oracle.build()
    cfg = CASES[name]()
    rng = np.random.default_rng(13)
    s = make_gpu(cfg)
    s.start()
    assert s.step(TOL)["status"] == 0
    x0, P0, w, sp = s.particles()
    f0 = s.fields()
    E0 = pic.inspect_checkpoint(s.checkpoint())["E0"]
    dxc = np.asarray(cfg["L"][:cfg["dim"]], float) / np.asarray(cfg["n"][:cfg["dim"]], float)
    dx = rng.standard_normal(x0.shape) * dxc[:, None]
    dP = rng.standard_normal(P0.shape) * _scale(P0)
    df = {k: rng.standard_normal(f0[k].shape) * _scale(f0[k]) for k in FIELDS}
    cx = rng.standard_normal(x0.shape)
    cP = rng.standard_normal(P0.shape)
    cf = {k: rng.standard_normal(f0[k].shape) for k in FIELDS}
    s.set_state(x0, P0, w, sp, f0, E0)
    g = s.step_vjp(TOL, cx, cP, cf)
    lhs = np.sum(g["x"] * dx) + np.sum(g["P"] * dP) + \
        sum(np.sum(g["fields"][k] * df[k]) for k in FIELDS)
    o = make_oracle(cfg)
    h = 1e-6
    out = {}
    for sgn in (1, -1):
        f = {k: f0[k] + sgn * h * df[k] for k in FIELDS}
        f["J"] = f0["J"]
        o.set_state(x0 + sgn * h * dx, P0 + sgn * h * dP, w, sp, f)
        assert o.step(TOL)["status"] == 0
        xo, Po, _, _ = o.particles()
        out[sgn] = (xo, Po, o.fields())
    (xp, Pp, fp), (xm, Pm, fm) = out[1], out[-1]
    terms = [np.sum(cx * periodic_diff(xp, xm, cfg["L"])) / (2 * h),
             np.sum(cP * (Pp - Pm)) / (2 * h)] + \
            [np.sum(cf[k] * (fp[k] - fm[k])) / (2 * h) for k in FIELDS]
    fd, gross = sum(terms), sum(abs(t) for t in terms)
    print(f"{name}: GPU adjoint {lhs:.10e}, oracle central difference {fd:.10e}, "
          f"|diff| / gross {abs(lhs - fd) / gross:.2e}")
    assert abs(lhs - fd) <= 1e-5 * gross


def test_twenty_step_reverse_sweep_matches_the_forward_sensitivity():
    u0, steps = 0.6, 20
    mk = lambda u: pic_inputs.two_stream_1d(nx=64, ppc_beam=32, u0=u)
    cfg = mk(u0)
    du = (mk(u0 + 1e-6)["u"] - mk(u0 - 1e-6)["u"]) / 2e-6
    N, Ng = cfg["u"].shape[1], int(np.prod(cfg["n"]))
    rng = np.random.default_rng(5)
    cx = rng.standard_normal((cfg["dim"], N))
    cP = rng.standard_normal((3, N))
    cA = rng.standard_normal(3 * Ng)
    cU = rng.standard_normal(3 * Ng)
    # forward: the tangent of the final state in the direction du
    s = make_gpu(cfg)
    s.start()
    s.tangent_begin(du=du)
    for _ in range(steps):
        assert s.step(TOL)["status"] == 0
    t = s.tangent()
    fwd_terms = [np.sum(cx * t["dx"]), np.sum(cP * t["dP"]), np.sum(cA * t["dA"]),
                 np.sum(cU * t["dU"])]
    # reverse: one sweep gives the gradient with respect to every momentum
    s2 = make_gpu(cfg)
    s2.start()
    g = s2.run_adjoint(TOL, steps, cx, cP, {"A": cA, "U": cU})
    ms = np.array([m for _, m in cfg["species"]])
    m_p = cfg["w"] * ms[cfg["sp"]]
    adj = np.sum(g["P"] * (m_p * du))
    fwd = sum(fwd_terms)
    gross = sum(abs(v) for v in fwd_terms)
    print(f"d<c, S_20>/du0: adjoint {adj:.12e}, forward {fwd:.12e}, |diff| / gross "
          f"{abs(adj - fwd) / gross:.2e}; GMRES applications per step {g['gmres_iters']}")
    assert abs(adj - fwd) <= 1e-8 * gross
    # the sweep leaves the context in the final state, which steps on
    assert s2.step(TOL)["status"] == 0


def test_step_vjp_refuses_unsupported_contexts():
    cfg = small_2d()
    s = make_gpu(cfg, precision=pic.PIC_MIXED)
    s.start()
    with pytest.raises(pic.PicError) as ei:
        s.step_vjp(TOL)
    assert ei.value.code == pic.PIC_EARG
    t = make_gpu(cfg)
    with pytest.raises(pic.PicError) as ei:
        t.step_vjp(TOL)
    assert ei.value.code == pic.PIC_ESTATE


def test_state_after_autograd_gradient_matches_central_differences():
    """torch.autograd through two steps (paper_2609_36383_b300.autograd.state_after):
    the reverse-mode gradient of <c, S_2> with respect to every position,
    momentum and potential of S_0, dotted with a random direction, equals
    the central difference of the forward pass."""
    import torch
    from paper_2609_36383_b300 import autograd as pa
    cfg = small_2d()
    s = make_gpu(cfg)
    s.start()
    assert s.step(TOL)["status"] == 0
    x0, P0, _, _ = s.particles()
    f0 = pa.pack_fields(s.fields(), s.Ng)
    base = s.checkpoint()
    rng = np.random.default_rng(21)
    dxc = np.asarray(cfg["L"][:2], float) / np.asarray(cfg["n"][:2], float)
    d = [rng.standard_normal(x0.shape) * dxc[:, None],
         rng.standard_normal(P0.shape) * _scale(P0),
         rng.standard_normal(f0.shape) * _scale(f0)]
    c = [rng.standard_normal(x0.shape), rng.standard_normal(P0.shape),
         rng.standard_normal(f0.shape)]
    x, P, f = (torch.tensor(a, requires_grad=True) for a in (x0, P0, f0))
    out = pa.state_after(s, TOL, 2, x, P, f)
    loss = sum((torch.from_numpy(ci) * t).sum() for ci, t in zip(c, out))
    loss.backward()
    lhs = sum(np.sum(g.grad.numpy() * di) for g, di in zip((x, P, f), d))
    h = 1e-6
    res = {}
    for sg in (1, -1):
        s.restore(base)
        with torch.no_grad():
            res[sg] = [t.numpy() for t in pa.state_after(
                s, TOL, 2, *(torch.from_numpy(a + sg * h * di) for a, di in zip((x0, P0, f0), d)))]
    terms = [np.sum(c[0] * periodic_diff(res[1][0], res[-1][0], cfg["L"])) / (2 * h)] + \
            [np.sum(ci * (res[1][k] - res[-1][k])) / (2 * h) for k, ci in ((1, c[1]), (2, c[2]))]
    fd = sum(terms)
    gross = sum(abs(t) for t in terms)
    print(f"autograd <grad, d> {lhs:.10e}, central difference {fd:.10e}, "
          f"|diff| / gross {abs(lhs - fd) / gross:.2e}")
    assert abs(lhs - fd) <= 1e-5 * gross


def test_step_vjp_with_device_buffers_matches_host_buffers():
    """on_device = 1: the cotangents in and out as CUDA device pointers give
    the host call's results (to the atomic scatters' summation order)."""
    import ctypes as C
    import torch
    cfg = small_2d()
    s = make_gpu(cfg)
    s.start()
    assert s.step(TOL)["status"] == 0
    N, Ng, d = s.num_particles(), s.Ng, s.dim
    rng = np.random.default_rng(3)
    cx = rng.standard_normal((d, N))
    cP = rng.standard_normal((3, N))
    cf = {k: rng.standard_normal(v.shape) for k, v in s.fields().items() if k != "J"}
    ref = s.step_vjp(TOL, cx, cP, cf)
    dev = torch.device("cuda")
    t_in = [torch.from_numpy(np.ascontiguousarray(a)).to(dev)
            for a in (cx, cP, s._pack_fields(cf))]
    t_out = [torch.zeros(d * N, dtype=torch.float64, device=dev),
             torch.zeros(3 * N, dtype=torch.float64, device=dev),
             torch.zeros(9 * Ng, dtype=torch.float64, device=dev)]
    its = C.c_int(0)
    torch.cuda.synchronize()
    rc = pic.lib().pic_step_vjp(s.handle, TOL, *[C.c_void_p(t.data_ptr()) for t in t_in],
                                *[C.c_void_p(t.data_ptr()) for t in t_out], C.byref(its), 1)
    assert rc == 0
    torch.cuda.synchronize()
    got = [t.cpu().numpy() for t in t_out]
    want = [ref["x"].ravel(), ref["P"].ravel(), s._pack_fields(ref["fields"])]
    for g, w in zip(got, want):
        assert np.abs(g - w).max() <= 1e-10 * np.abs(w).max()


@pytest.mark.parametrize("project", [1, 0])
def test_vacuum_step_adjoint_is_the_transpose_of_the_field_step(project):
    """No particles: the step is the CN field update alone, linear in the
    state, so <ybar, step(dS)> = <step^T ybar, dS> to rounding for any dS
    (checked through the linear map itself, step(S + dS) - step(S)), with
    and without the Nyquist projector."""
    cfg = small_2d()
    n, Ng = cfg["n"], int(np.prod(cfg["n"]))
    rng = np.random.default_rng(30 + project)
    s = pic.Simulation(2, n, cfg["L"], cfg["x0"], cfg["species"], cfg["dt"],
                       project_nyquist=project)
    empty = (np.zeros((2, 0)), np.zeros((3, 0)), np.zeros(0), np.zeros(0, np.int32))
    f0 = {k: rng.standard_normal(m * Ng) for k, m in
          (("phi", 1), ("psi", 1), ("A", 3), ("U", 3), ("rho", 1))}
    f0["J"] = np.zeros(3 * Ng)
    d = {k: rng.standard_normal(v.shape) for k, v in f0.items() if k != "J"}
    yb = {k: rng.standard_normal(v.shape) for k, v in f0.items() if k != "J"}

    def step_from(f):
        s.set_state(*empty, f, 1.0)
        assert s.step(1e-12)["status"] == 0
        return s.fields()

    base = step_from(f0)
    moved = step_from({**f0, **{k: f0[k] + d[k] for k in d}})
    lhs = sum(np.sum(yb[k] * (moved[k] - base[k])) for k in yb)
    s.set_state(*empty, f0, 1.0)
    g = s.step_vjp(1e-12, fbar=yb)["fields"]
    rhs = sum(np.sum(g[k] * d[k]) for k in d)
    gross = sum(np.sum(np.abs(yb[k] * (moved[k] - base[k]))) for k in yb)
    print(f"project {project}: <ybar, step dS> {lhs:.14e}, <step^T ybar, dS> {rhs:.14e}")
    assert abs(lhs - rhs) <= 1e-12 * gross


def test_autograd_wrappers_on_device_tensors_match_host_tensors():
    """The torch.autograd wrappers with CUDA tensors (device pointers into the
    library, no host copy of the tensors) give what they give with host
    tensors: state_after's gradient through two steps, and map_eval's value,
    forward- and reverse-mode derivatives."""
    import torch
    import torch.autograd.forward_ad as fwAD
    from paper_2609_36383_b300 import autograd as pa
    cfg = small_2d()
    s = make_gpu(cfg)
    s.start()
    assert s.step(TOL)["status"] == 0
    x0, P0, _, _ = s.particles()
    f0 = pa.pack_fields(s.fields(), s.Ng)
    base = s.checkpoint()
    rng = np.random.default_rng(5)
    c = [rng.standard_normal(x0.shape), rng.standard_normal(P0.shape),
         rng.standard_normal(f0.shape)]
    grads = {}
    for dev in ("cpu", "cuda"):
        s.restore(base)
        x, P, f = (torch.tensor(a, device=dev, requires_grad=True) for a in (x0, P0, f0))
        out = pa.state_after(s, TOL, 2, x, P, f)
        assert all(t.device.type == dev for t in out)
        loss = sum((torch.tensor(ci, device=dev) * t).sum() for ci, t in zip(c, out))
        loss.backward()
        grads[dev] = [g.grad.detach().cpu().numpy() for g in (x, P, f)]
    for a, b in zip(grads["cpu"], grads["cuda"]):
        assert np.abs(a - b).max() <= 1e-9 * max(np.abs(a).max(), 1e-300)
    s.restore(base)
    j0 = s.fields()["J"]
    dj = rng.standard_normal(j0.shape) * np.abs(j0).max()
    ybar = rng.standard_normal(j0.shape)
    res = {}
    for dev in ("cpu", "cuda"):
        j = torch.tensor(j0, device=dev, requires_grad=True)
        with fwAD.dual_level():
            jd = fwAD.make_dual(j.detach(), torch.tensor(dj, device=dev))
            H, dH = fwAD.unpack_dual(pa.map_eval(s, jd, TOL))
        Hr = pa.map_eval(s, j, TOL)
        (Hr * torch.tensor(ybar, device=dev)).sum().backward()
        res[dev] = [t.detach().cpu().numpy() for t in (H, dH, j.grad)]
    for a, b in zip(res["cpu"], res["cuda"]):
        assert np.abs(a - b).max() <= 1e-10 * max(np.abs(a).max(), 1e-300)
