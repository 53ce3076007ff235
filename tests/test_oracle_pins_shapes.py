"""Pins of the oracle's degree-one particle shapes and of its
convergence-triggered particle refinement (Sec. 5.3), against what the
mathematics fixes: exact integrals (sympy), the partition of unity, linear
reproduction, the exact discrete chain rule (Lemma exact-chain-rule) and the
total-energy theorem (Thm. energy), which holds for any shape degree and, with
orbit-averaged currents, for particles that take several substeps of the field
step.  None compares the oracle with itself.
"""
import math

import numpy as np
import pytest

import pic_inputs


def _oracle(orc, dim=2, n=16, dt=0.3, **kw):
    L = 2 * math.pi
    return orc.Oracle(dim, [n] * dim, [L] * dim, [-math.pi] * dim, [(-1.0, 1.0)], dt=dt,
                      rho_bg=1.0, **kw)


def test_linear_bspline_values_partition_and_derivative(orc):
    assert orc.S1(0.0) == 1.0 and orc.S1(0.5) == 0.5 and orc.S1(-0.25) == 0.75
    assert orc.S1(1.0) == 0.0 and orc.S1(-1.3) == 0.0
    rng = np.random.default_rng(1)
    for u in rng.uniform(-5, 5, 50):
        g = np.arange(math.floor(u) - 3, math.floor(u) + 4)
        assert sum(orc.S1(u - k) for k in g) == pytest.approx(1.0, abs=1e-15)
        assert sum(orc.dS1(u - k) for k in g) == pytest.approx(0.0, abs=1e-15)
    h = 1e-7
    for xi in (-0.7, -0.2, 0.3, 0.9):
        fd = (orc.S1(xi + h) - orc.S1(xi - h)) / (2 * h)
        assert orc.dS1(xi) == pytest.approx(fd, abs=1e-8)


def test_orbit_average_degree_one_matches_exact_sympy_integral(orc):
    """Sbar_g = int_0^1 S_1(u0 + s delta - g) ds computed exactly by sympy, for
    orbits that cross several of the integer knots of S_1 (reading R15)."""
    import sympy as sp
    s = sp.symbols("s", real=True)

    def S1sym(xi):
        return sp.Max(1 - sp.Abs(xi), 0)

    n, L = 16, 16.0  # dx = 1
    o = orc.Oracle(1, [n], [L], [0.0], [(-1.0, 1.0)], dt=1.0, order=1)
    for u0, dl in [(sp.Rational(37, 10), sp.Rational(23, 10)),
                   (sp.Rational(81, 10), sp.Rational(-17, 10)),
                   (sp.Rational(5, 1), sp.Rational(3, 4)),
                   (sp.Rational(9, 2), sp.Rational(-1, 2))]:
        for g in range(int(u0) - 4, int(u0) + 5):
            ex = sp.integrate(S1sym(u0 + s * dl - g), (s, 0, 1))
            G = np.zeros((3, n))
            G[0, g % n] = 1.0
            od = o.orbit_data(np.array([float(u0)]), np.array([float(dl), 0, 0]), G,
                              np.zeros((3, n)), np.zeros((3, n)), None)
            assert od["gphi"][0] == pytest.approx(float(ex), abs=2e-15)


def test_degree_one_chain_rule_partition_and_linear_reproduction(orc):
    """Lemma exact-chain-rule holds for any shape degree: R_A = 0 on random
    orbits and mesh data; Sbar sums to one; linear B-splines reproduce linear
    data (the gather of a linear field is its value at the orbit midpoint, D of
    a linear A its gradient)."""
    rng = np.random.default_rng(21)
    for dt in (0.3, 1.0):
        o = _oracle(orc, dt=dt, order=1)
        Ng = o.Ng
        for _ in range(30):
            An = rng.standard_normal((3, Ng))
            Ap = rng.standard_normal((3, Ng))
            Uh = (Ap - An) / dt
            x = rng.uniform(-math.pi, math.pi, 2)
            vbar = rng.standard_normal(3) * 0.6
            od = o.orbit_data(x, vbar, None, An, Ap, Uh)
            RA = od["Aplus"] - od["Aminus"] - dt * (od["Ubar"] + od["D"] @ vbar)
            assert np.abs(RA).max() < 1e-13
            assert od["Sbar_sum"] == pytest.approx(1.0, abs=1e-14)
    o = _oracle(orc, n=32, dt=0.5, order=1)
    dx = 2 * math.pi / 32
    xs = -math.pi + np.arange(32) * dx
    Y, X = np.meshgrid(xs, xs, indexing="ij")
    G = np.stack([0.2 + 0.3 * X - 0.1 * Y, -0.4 * X, 0.7 * Y]).reshape(3, -1)
    x = np.array([0.11, -0.23])
    vbar = np.array([0.9, -0.7, 0.2])
    od = o.orbit_data(x, vbar, G, G, G, G)
    mid = x + 0.5 * 0.5 * vbar[:2]
    expect = np.array([0.2 + 0.3 * mid[0] - 0.1 * mid[1], -0.4 * mid[0], 0.7 * mid[1]])
    assert np.allclose(od["gphi"], expect, atol=1e-13)
    assert np.allclose(od["D"][:, :2], np.array([[0.3, -0.1], [-0.4, 0], [0, 0.7]]), atol=1e-12)


def test_degree_one_whole_step_conserves_energy(orc):
    """Thm. energy with linear shapes: total energy to the nonlinear tolerance,
    R_A and R_work at roundoff."""
    cfg = pic_inputs.weibel_2d(n=16, ppc_beam=4, u_drift=0.5, T=0.01, dt=0.2, tol=1e-12,
                               steps=3, seed=12, noise=1e-3, kmax=3)
    from tests._common import make_oracle
    o = make_oracle(cfg, order=1)
    o.start()
    for _ in range(3):
        r = o.step(1e-12)
        assert r["status"] == 0
        assert abs(r["rel_dE"]) < 1e-11
        assert r["chain_rms"] < 1e-15
        assert abs(r["work_residual"]) < 1e-15
        assert r["gauss_rms"] < 1e-12 and r["lorenz_rms"] < 1e-12


def _refine_case(dt):
    # 1D thermal beams with a small inner limit: some particles need more
    # Picard iterations over the full step than the limit allows, but fewer
    # over substeps
    return pic_inputs.thermal_box(dim=1, n=16, ppc=8, T=0.05, u_drift=0.6, dt=dt, seed=4)


@pytest.mark.parametrize("order,dt,inner_max,levels", [(2, 0.5, 5, 2), (1, 0.3, 5, 3)])
def test_refinement_triggers_and_conserves_energy(orc, order, dt, inner_max, levels):
    """Convergence-triggered refinement (reading R16): particles whose full-step
    solve fails are retried with substeps, the step succeeds, and the energy
    theorem still holds exactly: the orbit-averaged current (each substep's
    current weighted by its share of the step) matches the substeps' particle
    work, and each substep satisfies the chain rule with the time-linear A."""
    from tests._common import make_oracle
    cfg = _refine_case(dt)
    ref = make_oracle(cfg, inner_max=inner_max, refine_max=0, order=order)
    ref.start()
    assert any(ref.step(1e-12)["status"] == -4 for _ in range(3))  # fails without refinement
    o = make_oracle(cfg, inner_max=inner_max, refine_max=levels, order=order)
    o.start()
    q = np.array([cfg["species"][s][0] for s in cfg["sp"]]) * cfg["w"]
    dV = cfg["L"][0] / cfg["n"][0]
    refined = checked = 0
    for _ in range(3):
        # total-current identity of the orbit-averaged deposit: sum_g H_g dV =
        # sum_i q_i vbar_i, with vbar the substep-averaged orbit velocity
        st, H, vb, Pn, it = o.eval_map(o.fields()["J"], 1e-12)
        if st == 0 and o.refined() > 0:
            tot = H.reshape(3, -1).sum(axis=1) * dV
            assert np.allclose(tot, (q * vb).sum(axis=1), atol=1e-14 * np.abs(q).sum())
            checked += 1
        r = o.step(1e-12)
        assert r["status"] == 0
        refined += o.refined()
        assert abs(r["rel_dE"]) < 1e-12
        assert r["chain_rms"] < 1e-15
        assert abs(r["work_residual"]) < 1e-15
    assert refined > 0 and checked > 0


def test_refinement_inactive_changes_nothing(orc):
    """With every full-step solve converging, enabling refinement changes no
    bit of the result."""
    from tests._common import make_oracle
    cfg = pic_inputs.thermal_box(dim=1, n=16, ppc=8, T=0.05, u_drift=0.6, dt=0.2, seed=4)
    a = make_oracle(cfg, refine_max=0)
    b = make_oracle(cfg, refine_max=3)
    a.start()
    b.start()
    for _ in range(2):
        ra = a.step(1e-12)
        rb = b.step(1e-12)
        assert ra["status"] == 0 and rb["status"] == 0 and b.refined() == 0
        assert ra["E_tot"] == rb["E_tot"]
    xa, Pa, _, _ = a.particles()
    xb, Pb, _, _ = b.particles()
    assert np.array_equal(xa, xb) and np.array_equal(Pa, Pb)


# ---- knot-jump regularity diagnostic (Sec. 5.3) ---------------------------
# The interpolant F_h = sum_g F_g S_r(x - x_g) has knots where S_r changes
# polynomial piece: the nodes for r = 1, the cell midpoints for r = 2.  With
# the probe at +-eps node units about a knot, closed forms follow from the
# piecewise structure:
#  * r = 1: F_h is linear between nodes, so d F_h / dx jumps at node i by the
#    second difference (F_{i+1} - 2 F_i + F_{i-1}) / dx;
#  * r = 2: d F_h / dx is continuous and piecewise linear, with slope
#    D_i = (F_{i+1} - 2 F_i + F_{i-1}) / dx^2 on the cell of node i, so the
#    two-sided difference across the knot between nodes i and i + 1 is
#    eps dx (D_i + D_{i+1});
#  * a separable field F_{ij} = f_i g_j probed along x on a line y = y* half a
#    cell from the y-knots (y_j for r = 2, y_{j+1/2} for r = 1) has
#    E = -(f_h'(x) g_h(y*), f_h(x) g_h'(y*)): the x-component jumps by the
#    slope jump of f times g_h(y*), and the y-component changes by
#    f_h(x+) - f_h(x-) = eps (f_{i+1} - f_{i-1}) (r = 1) or
#    2 eps (f_{i+1} - f_i) (r = 2, to O(eps^2)) times g_h'(y*), with
#    g_h(y_{j+1/2}) = (g_j + g_{j+1}) / 2 and g_h' = (g_{j+1} - g_j) / dx
#    (r = 1), g_h(y_j) = (g_{j-1} + 6 g_j + g_{j+1}) / 8 and
#    g_h'(y_j) = (g_{j+1} - g_{j-1}) / (2 dx) (r = 2, from S_2 and S_2' at
#    0 and +-1).

def _second_diff(f):
    return np.roll(f, -1) - 2 * f + np.roll(f, 1)


def _jumps_1d(o, phi=None, A=None, eps=1e-8):
    Ng = o.Ng
    z1, z3 = np.zeros(Ng), np.zeros(3 * Ng)
    o.set_state(np.zeros((o.dim, 0)), np.zeros((3, 0)), np.zeros(0), np.zeros(0, np.int32),
                dict(phi=z1 if phi is None else phi, psi=z1, A=z3 if A is None else A, U=z3,
                     rho=z1, J=z3))
    return o.knot_jumps(eps)


@pytest.mark.parametrize("order", [1, 2])
def test_knot_jump_closed_forms_in_1d(orc, order):
    n, L, eps = 32, 4 * math.pi, 1e-8
    dx = L / n
    o = orc.Oracle(1, [n], [L], [0.0], [(-1.0, 1.0)], dt=0.1, order=order)
    rng = np.random.default_rng(40 + order)
    phi = rng.standard_normal(n)
    A = rng.standard_normal(3 * n)
    Ej, Gj = _jumps_1d(o, phi=phi)
    Ej0, Gj_A = _jumps_1d(o, A=A)
    assert Gj == 0.0 and Ej0 == 0.0
    Ac = A.reshape(3, n)
    if order == 1:
        want_E = np.abs(_second_diff(phi)).max() / dx
        want_G = np.sqrt((_second_diff(Ac.T.T) ** 2).sum(axis=0)).max() / dx
        assert Ej == pytest.approx(want_E, rel=1e-12)
        assert Gj_A == pytest.approx(want_G, rel=1e-12)
    else:
        D = _second_diff(phi) / dx ** 2
        want_E = (eps * dx * np.abs(D + np.roll(D, -1))).max()
        DA = np.stack([_second_diff(a) for a in Ac]) / dx ** 2
        want_G = (eps * dx * np.sqrt(((DA + np.roll(DA, -1, axis=1)) ** 2).sum(axis=0))).max()
        assert Ej == pytest.approx(want_E, rel=1e-6)
        assert Gj_A == pytest.approx(want_G, rel=1e-6)


@pytest.mark.parametrize("order", [1, 2])
def test_knot_jump_separable_field_in_2d(orc, order):
    n, L, eps = 16, 2 * math.pi, 1e-8
    dx = L / n
    o = orc.Oracle(2, [n, n], [L, L], [-math.pi, -math.pi], [(-1.0, 1.0)], dt=0.1, order=order)
    rng = np.random.default_rng(7 + order)
    f, g = rng.standard_normal(n), rng.standard_normal(n)
    phi = np.outer(g, f).ravel()  # phi[i + n j] = f_i g_j (x fastest)

    def along(v, w):
        """max jump probing along the axis of v, the transverse factor w."""
        if order == 1:
            a = _second_diff(v) / dx                      # slope jump at node i
            dv = eps * (np.roll(v, -1) - np.roll(v, 1))   # v_h(x+) - v_h(x-)
            wh = (w + np.roll(w, -1)) / 2
            wp = (np.roll(w, -1) - w) / dx
        else:
            D = _second_diff(v) / dx ** 2
            a = eps * dx * (D + np.roll(D, -1))           # across the knot i + 1/2
            dv = 2 * eps * (np.roll(v, -1) - v)
            wh = (np.roll(w, 1) + 6 * w + np.roll(w, -1)) / 8
            wp = (np.roll(w, -1) - np.roll(w, 1)) / (2 * dx)
        return np.sqrt(np.outer(a, wh) ** 2 + np.outer(dv, wp) ** 2).max()

    Ej, _ = _jumps_1d(o, phi=phi)
    want = max(along(f, g), along(g, f))
    assert Ej == pytest.approx(want, rel=1e-12 if order == 1 else 1e-6)
