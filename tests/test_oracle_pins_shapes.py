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
