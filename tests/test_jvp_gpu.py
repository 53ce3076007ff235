"""The tangent of one map evaluation (pic_eval_map_jvp) and its adjoint
(pic_eval_map_vjp) on the CUDA path.

dH = H'(j) dj is checked against central finite differences of the map
itself (on the GPU and in the FP64 oracle), for linearity, and by using it:
a Newton-Krylov solve (GMRES(20) with the JVP) of the outer fixed point
j = H(j) of one step must reach the step's fixed point, which the paper's
Picard/Anderson iteration (pic_step) also reaches.

The adjoint is checked by the dot-product identity <ybar, H'(j) dj> =
<H'(j)^T ybar, dj> against the JVP, and against central differences of the
scalar <ybar, H(j)>.

Tolerances: the map is evaluated with the inner tolerance 1e-14; central
differences with step h carry a truncation error O(h^2 H''') and a rounding
error O(1e-14 / h), so with h = 1e-4 (relative) they agree with the exact
tangent to about 1e-7 of its size; the bound is 2e-6.
"""
import numpy as np
import pytest

import paper_2609_36383_b300 as pic
import pic_inputs
from tests._common import gross_scales, make_gpu, make_oracle, small_1d, small_2d

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2609_36383_b300 import build
    build.build()
    import oracle
    oracle.build()


def _thermal_3d():
    return pic_inputs.thermal_box(dim=3, n=8, ppc=2, T=0.05, u_drift=0.3, dt=0.2, seed=4)


CASES = {"1d_two_stream": small_1d, "2d_weibel": small_2d, "3d_thermal": _thermal_3d}


def _trial(o, gross, seed=2):
    """A trial current near the accepted one and a projected direction.  The
    size is that of the net current, but at least 1e-3 of the gross
    (one-sign) current: the symmetric two-stream's net current is at
    rounding level."""
    rng = np.random.default_rng(seed)
    J = o.fields()["J"]
    s = max(np.abs(J).max(), 1e-3 * gross)
    j = J + 0.05 * s * o.project(rng.standard_normal(J.shape[0]), 3)
    dj = s * o.project(rng.standard_normal(J.shape[0]), 3)
    return j, dj


@pytest.mark.parametrize("name", sorted(CASES))
def test_jvp_matches_central_differences(name):
    cfg = CASES[name]()
    o = make_oracle(cfg)
    o.start()
    s = make_gpu(cfg)
    s.start()
    gross = gross_scales(cfg)["J"]
    j, dj = _trial(o, gross)
    st, H, dH = s.eval_map_jvp(j, dj, 1e-14)
    assert st == 0
    scale = np.abs(dH).max()
    assert scale > 0
    # step: 1e-4 of the larger of the trial current and the gross current, so
    # that rounding in the deposit (about 1e-16 of the gross current) stays
    # far below the difference it is divided into
    h = 1e-4 * max(np.abs(j).max(), gross) / np.abs(dj).max()
    # the GPU map itself
    _, Hp, _, _, _ = s.eval_map(j + h * dj, 1e-14)
    _, Hm, _, _, _ = s.eval_map(j - h * dj, 1e-14)
    fd = (Hp - Hm) / (2 * h)
    assert np.abs(dH - fd).max() < 2e-6 * scale
    # the FP64 oracle's map (its gradient by central differences)
    _, Hp, _, _, _ = o.eval_map(j + h * dj, 1e-14)
    _, Hm, _, _, _ = o.eval_map(j - h * dj, 1e-14)
    fdo = (Hp - Hm) / (2 * h)
    assert np.abs(dH - fdo).max() < 2e-6 * scale
    # the value is the map's value
    _, H0, _, _, _ = s.eval_map(j, 1e-14)
    assert np.abs(H - H0).max() < 1e-12 * np.abs(H0).max()


@pytest.mark.parametrize("name", sorted(CASES))
def test_vjp_is_the_transpose_of_the_jvp(name):
    """<ybar, H'(j) dj> = <H'(j)^T ybar, dj> for random ybar and dj; both
    products are exact derivatives of the converged inner fixed point up to
    the inner tolerance 1e-14, so they agree to about 1e-12 of the gross
    magnitudes of the two sums."""
    cfg = CASES[name]()
    o = make_oracle(cfg)
    o.start()
    s = make_gpu(cfg)
    s.start()
    gross = gross_scales(cfg)["J"]
    j, dj = _trial(o, gross)
    ybar = np.random.default_rng(5).standard_normal(j.shape[0])
    st, H1, dH = s.eval_map_jvp(j, dj, 1e-14)
    assert st == 0
    st, H2, jbar = s.eval_map_vjp(j, ybar, 1e-14)
    assert st == 0
    # the two evaluations deposit in different orders: their rounding is
    # bounded by the gross (one-sign) deposit magnitude, which the
    # counter-streaming beams' net current can lie far below
    assert np.abs(H1 - H2).max() <= 1e-12 * max(np.abs(H1).max(), gross)
    lhs, rhs = ybar @ dH, jbar @ dj
    gross_sum = max(np.abs(ybar * dH).sum(), np.abs(jbar * dj).sum())
    print(f"{name}: <ybar, J dj> = {lhs:.12e}, <J^T ybar, dj> = {rhs:.12e}, "
          f"difference {abs(lhs - rhs) / gross_sum:.2e} of the gross sum")
    assert abs(lhs - rhs) <= 1e-10 * gross_sum
    # the scalar <ybar, H(j)> by central differences along dj
    h = 1e-4 * max(np.abs(j).max(), gross) / np.abs(dj).max()
    _, Hp, _, _, _ = s.eval_map(j + h * dj, 1e-14)
    _, Hm, _, _, _ = s.eval_map(j - h * dj, 1e-14)
    fd = ybar @ (Hp - Hm) / (2 * h)
    assert abs(fd - rhs) <= 2e-6 * gross_sum


def test_jvp_is_linear_in_the_direction():
    cfg = small_2d()
    o = make_oracle(cfg)
    o.start()
    s = make_gpu(cfg)
    s.start()
    gross = gross_scales(cfg)["J"]
    j, d1 = _trial(o, gross, seed=3)
    _, d2 = _trial(o, gross, seed=4)
    _, _, a = s.eval_map_jvp(j, d1, 1e-14)
    _, _, b = s.eval_map_jvp(j, d2, 1e-14)
    _, _, c = s.eval_map_jvp(j, 2.0 * d1 - 0.5 * d2, 1e-14)
    scale = max(np.abs(a).max(), np.abs(b).max())
    assert np.abs(c - (2.0 * a - 0.5 * b)).max() < 1e-9 * scale


def _scaled_rms(r, H, j, tol, ratio=0.01):
    rms = lambda v: np.sqrt(np.mean(v * v))
    return rms(r) / (tol * ratio + 0.5 * tol * (rms(H) + rms(j)))


def _gmres(matvec, b, m=20, rtol=1e-4, max_restarts=5):
    """Restarted GMRES(m) for A x = b from x = 0; returns x and the matvecs used."""
    n = b.shape[0]
    x = np.zeros(n)
    used = 0
    bnorm = np.linalg.norm(b)
    for _ in range(max_restarts):
        r = b - matvec(x) if used else b.copy()
        beta = np.linalg.norm(r)
        if beta <= rtol * bnorm:
            break
        V = np.zeros((m + 1, n))
        Hh = np.zeros((m + 1, m))
        V[0] = r / beta
        k_end = m
        for k in range(m):
            w = matvec(V[k])
            used += 1
            for i in range(k + 1):
                Hh[i, k] = w @ V[i]
                w = w - Hh[i, k] * V[i]
            Hh[k + 1, k] = np.linalg.norm(w)
            e1 = np.zeros(k + 2)
            e1[0] = beta
            y, *_ = np.linalg.lstsq(Hh[:k + 2, :k + 1], e1, rcond=None)
            res = np.linalg.norm(Hh[:k + 2, :k + 1] @ y - e1)
            if Hh[k + 1, k] == 0 or res <= rtol * bnorm:
                k_end = k + 1
                break
            V[k + 1] = w / Hh[k + 1, k]
        x = x + V[:k_end].T @ y
        used += 1
        if np.linalg.norm(b - matvec(x)) <= rtol * bnorm:
            break
    return x, used


def test_newton_krylov_outer_solve_reaches_the_step_fixed_point():
    """One step's outer problem F(j) = H(j) - j = 0 solved by Newton with
    GMRES(20) on J_F v = H'(j) v - v (the JVP), against Algorithm 1's
    Picard/Anderson iteration (pic_step): both reach the same fixed point;
    the numbers of map evaluations are reported."""
    cfg = small_2d()
    tol = 1e-10
    ref = make_gpu(cfg)
    ref.start()
    nk = make_gpu(cfg)
    nk.start()
    j = nk.fields()["J"].copy()
    r = ref.step(tol)
    assert r["status"] == 0
    J_ref = ref.fields()["J"]
    evals = 0
    for newton in range(12):
        st, H, _ = nk.eval_map_jvp(j, np.zeros_like(j), tol)
        evals += 1
        assert st == 0
        F = H - j
        if _scaled_rms(F, H, j, tol) <= 1.0:
            break

        def matvec(v):
            st, _, dH = nk.eval_map_jvp(j, v, tol)
            assert st == 0
            return dH - v

        dx, used = _gmres(matvec, -F)
        evals += used
        j = j + dx
    assert _scaled_rms(F, H, j, tol) <= 1.0
    err = np.abs(j - J_ref).max() / np.abs(J_ref).max()
    print(f"Newton-Krylov: {newton} Newton steps, {evals} map evaluations (with tangents); "
          f"Picard/Anderson: {r['map_evals']} map evaluations; |j - J| = {err:.2e}")
    assert err < 1e-7


@pytest.mark.parametrize("make_cfg,tol", [(small_1d, 1e-12), (small_2d, 1e-10)], ids=["1d", "2d"])
def test_newton_krylov_option_matches_algorithm_1(make_cfg, tol):
    """The library's Newton-Krylov outer solver (nonlinear_solver =
    PIC_SOLVER_NEWTON_KRYLOV) against Algorithm 1's Anderson iteration over
    three steps from the same state: every step passes the same outer tests
    and verification, so the committed states agree to the outer tolerance
    and the energy theorem holds on both; the evaluation counts are
    reported (plain map evaluations and Jacobian-vector products)."""
    cfg = make_cfg()
    a = make_gpu(cfg)
    n = make_gpu(cfg, nonlinear_solver=pic.PIC_SOLVER_NEWTON_KRYLOV)
    a.start()
    n.start()
    for st in range(3):
        ra, rn = a.step(tol), n.step(tol)
        assert ra["status"] == 0 and rn["status"] == 0, rn
        assert rn["jvp_evals"] > 0 and ra["jvp_evals"] == 0
        assert rn["res_scaled_rms"] <= 1.0 and rn["res_scaled_max"] <= 1.0
        assert abs(rn["rel_dE"]) < 1e-11 and rn["chain_rms"] < 1e-13
        print(f"step {st}: Anderson {ra['outer_iters']} iterations / {ra['map_evals']} evaluations;"
              f" Newton-Krylov {rn['outer_iters']} iterations / {rn['map_evals']} evaluations + "
              f"{rn['jvp_evals']} JVPs")
    Ja, Jn = a.fields()["J"], n.fields()["J"]
    assert np.abs(Jn - Ja).max() <= 1e-8 * np.abs(Ja).max()
    xa, Pa, _, _ = a.particles()
    xn, Pn, _, _ = n.particles()
    assert np.abs(Pn - Pa).max() <= 1e-9 * np.abs(Pa).max()
    a.close()
    n.close()


def test_newton_krylov_option_is_refused_where_the_tangent_is_not_built():
    for kw in (dict(precision=pic.PIC_MIXED), dict(order=1), dict(refine_max=1),
               dict(inner_warm_start=1)):
        with pytest.raises(pic.PicError):
            make_gpu(small_1d(), nonlinear_solver=pic.PIC_SOLVER_NEWTON_KRYLOV, **kw)
