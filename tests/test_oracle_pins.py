"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these tests compares the oracle with itself: each checks a printed
constant, a closed form, an exact identity the paper proves, an independent
exact integral (sympy), a finite-difference derivative or a library routine of
a different implementation (numpy.fft).  The oracle is the reference for the
CUDA path, so each pin below is chosen so that a dropped term, a wrong sign or
index, or a transposed operand in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import pic_inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.txt")


def golden():
    out = {}
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        name, val, _cite = line.split()
        out[name] = float(val)
    return out


# ---------------------------------------------------------------- Sec. 5 constants
def test_closed_form_constants_match_paper():
    from oracle import closed_form as cf
    g = golden()
    assert cf.gamma_of_velocity(0.9) == pytest.approx(g["gamma0"], abs=1e-10)
    assert cf.chi(0.25, math.pi / 4) ** 2 == pytest.approx(g["chi2_sq"], abs=1e-10)
    assert cf.chi(1.0, math.pi / 16) ** 2 == pytest.approx(g["chi2_sq"], abs=1e-10)
    assert cf.two_stream_rate(0.25, 0.9, math.pi / 4) == pytest.approx(g["gamma_ts"], abs=1e-11)
    A, C = cf.weibel_coeffs(1.0, 0.9, math.pi / 16)
    assert A == pytest.approx(g["weibel_A"], abs=1e-10)
    assert C == pytest.approx(g["weibel_C"], abs=1e-10)
    assert cf.weibel_rate(1.0, 0.9, math.pi / 16) == pytest.approx(g["gamma_w"], abs=1e-10)


def test_two_stream_rate_solves_dispersion_relation():
    """omega = i Gamma_TS is a root of Eq. rel-ts-cont (checked by substitution)."""
    from oracle import closed_form as cf
    k, v0, dx = 0.5, 0.6 / math.sqrt(1.36), math.pi / 16
    G = cf.two_stream_rate(k, v0, dx)
    g0 = cf.gamma_of_velocity(v0)
    w2 = cf.omega_ph2(k, dx)
    om = 1j * G
    res = 1 - w2 / (2 * g0 ** 3) * (1 / (om - k * v0) ** 2 + 1 / (om + k * v0) ** 2)
    assert abs(res) < 1e-12
    assert G == pytest.approx(0.2147689, abs=1e-7)


# ---------------------------------------------------------------- shape (Sec. 4.5)
def test_quadratic_bspline_values_and_partition(orc):
    assert orc.S2(0.0) == 0.75
    assert orc.S2(1.0) == 0.125 and orc.S2(-1.0) == 0.125
    assert orc.S2(0.5) == 0.5 and orc.S2(1.5) == 0.0 and orc.S2(2.0) == 0.0
    rng = np.random.default_rng(1)
    for u in rng.uniform(-3, 3, 50):
        s = sum(orc.S2(u - g) for g in range(-6, 7))
        d = sum(orc.dS2(u - g) for g in range(-6, 7))
        m1 = sum(g * orc.S2(u - g) for g in range(-6, 7))  # linear reproduction
        assert s == pytest.approx(1.0, abs=1e-15)
        assert d == pytest.approx(0.0, abs=1e-14)
        assert m1 == pytest.approx(u, abs=1e-14)
    h = 1e-6
    for xi in rng.uniform(-1.6, 1.6, 50):
        fd = (orc.S2(xi + h) - orc.S2(xi - h)) / (2 * h)
        assert orc.dS2(xi) == pytest.approx(fd, abs=1e-8)
    for kn in (-1.5, -0.5, 0.5, 1.5):  # C1 at the knots (R1)
        assert abs(orc.dS2(kn + 1e-12) - orc.dS2(kn - 1e-12)) < 1e-10


def test_gauss_legendre_exact_degree(orc):
    for n in (1, 2, 3, 4, 8):
        t, w = orc.gauss_legendre(n)
        for k in range(2 * n):
            assert np.dot(w, t ** k) == pytest.approx(1.0 / (k + 1), rel=1e-14, abs=1e-15)
        assert abs(np.dot(w, t ** (2 * n)) - 1.0 / (2 * n + 1)) > 1e-12


# ---------------------------------------------------------------- DFT
def test_dft_against_numpy_and_closed_forms(orc):
    rng = np.random.default_rng(2)
    for shape in [(16,), (8, 12), (4, 6, 5)]:
        f = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
        assert np.allclose(orc.dft(f), np.fft.fftn(f), atol=1e-11)
        assert np.allclose(orc.dft(orc.dft(f), inverse=True), f, atol=1e-13)
    N = 32
    x = np.arange(N)
    F = orc.dft(np.cos(2 * np.pi * 3 * x / N))
    expect = np.zeros(N, complex)
    expect[3] = expect[N - 3] = N / 2
    assert np.allclose(F, expect, atol=1e-12)


# ---------------------------------------------------------------- HC map (Sec. 3.2)
def _cmat(B):
    """C(B) v = v x B, Eq. cross-matrix."""
    return np.array([[0, B[2], -B[1]], [-B[2], 0, B[0]], [B[1], -B[0], 0]])


def test_hc_map_norm_cayley_and_centred_gamma(orc):
    rng = np.random.default_rng(3)
    for _ in range(200):
        um = rng.standard_normal(3) * rng.uniform(0.01, 5)
        B = rng.standard_normal(3) * rng.uniform(0.0, 4)
        a = rng.uniform(-1, 1)  # q dt / 2m
        up, g = orc.hc_map(um, B, a)
        assert np.linalg.norm(up) == pytest.approx(np.linalg.norm(um), rel=1e-13)
        # Cayley form, Eq. hc-cayley-B (u = p / m kappa, so the scale cancels)
        Cb = _cmat(B) * a / g
        Q = np.linalg.solve(np.eye(3) - Cb, np.eye(3) + Cb)
        assert np.allclose(Q @ um, up, rtol=1e-12, atol=1e-13)
        # HC gamma equals the centred factor, Eq. Gamma-centered-overview
        assert g == pytest.approx(math.sqrt(1 + np.sum(((up + um) / 2) ** 2)), rel=1e-13)
        # u(+) - u(-) = (u+ + u-) x (a B / g), Eq. hc-centered-rotation-overview
        assert np.allclose(up - um, np.cross(up + um, a * B / g), rtol=1e-11, atol=1e-13)
    up, g = orc.hc_map(np.array([0.3, -0.2, 0.1]), np.zeros(3), 0.7)
    assert np.array_equal(up, np.array([0.3, -0.2, 0.1]))


def test_hc_map_unit_jacobian_fd(orc):
    """Volume preservation of the full nonlinear HC map (Sec. 3.2, Higuera-Cary)."""
    rng = np.random.default_rng(4)
    h = 1e-6
    for _ in range(20):
        um = rng.standard_normal(3)
        B = rng.standard_normal(3) * 2
        a = 0.4
        J = np.zeros((3, 3))
        for c in range(3):
            e = np.zeros(3); e[c] = h
            J[:, c] = (orc.hc_map(um + e, B, a)[0] - orc.hc_map(um - e, B, a)[0]) / (2 * h)
        assert np.linalg.det(J) == pytest.approx(1.0, abs=1e-8)


# ---------------------------------------------------------------- push (Sec. 3.4, 4.1-4.2)
def _rand_push_data(rng, kappa=1.0):
    return dict(Pn=rng.standard_normal(3) * 0.5, Am=rng.standard_normal(3) * 0.1,
                Ap=rng.standard_normal(3) * 0.1, gphi=rng.standard_normal(3) * 0.3,
                D=rng.standard_normal((3, 3)) * 0.5, vbar=rng.standard_normal(3) * 0.2,
                q=-rng.uniform(0.5, 2), m=rng.uniform(0.5, 2), kappa=kappa, dt=rng.uniform(0.02, 0.3))


def _gamma(p, m, kappa):
    return math.sqrt(1 + np.dot(p, p) / (m * m * kappa * kappa))


def test_push_single_particle_energy_and_mechanical_form(orc):
    """Eq. single-particle-work and the mechanical split, Eq. mechanical-split.

    With Ubar defined through the chain rule (Eq. A-chain-rule),
    Ebar = -gphi - Ubar, the canonical step must satisfy p- = p^n + q dt/2 Ebar,
    p^{n+1} = p+ + q dt/2 Ebar, |p+| = |p-|, and the kinetic-energy change
    q dt Ebar . vnew exactly."""
    rng = np.random.default_rng(5)
    for _ in range(200):
        d = _rand_push_data(rng)
        o = orc.push(**d)
        q, m, k, dt = d["q"], d["m"], d["kappa"], d["dt"]
        pn = d["Pn"] - q * d["Am"]
        pnp1 = o["Pnp1"] - q * d["Ap"]
        Ubar = (d["Ap"] - d["Am"]) / dt - d["D"] @ d["vbar"]
        Ebar = -d["gphi"] - Ubar
        assert np.allclose(o["pminus"], pn + 0.5 * q * dt * Ebar, atol=1e-13)
        assert np.allclose(pnp1, o["pplus"] + 0.5 * q * dt * Ebar, atol=1e-13)
        assert np.linalg.norm(o["pplus"]) == pytest.approx(np.linalg.norm(o["pminus"]), rel=1e-13)
        K = lambda p: m * k * k * (_gamma(p, m, k) - 1)
        assert K(pnp1) - K(pn) == pytest.approx(q * dt * np.dot(Ebar, o["vnew"]), abs=1e-13)
        # Eq. hc-magnetic-increment with K = D^T - D and Gamma = gamma_HC
        Km = d["D"].T - d["D"]
        _, g = orc.hc_map(o["pminus"] / (m * k),
                          np.array([Km[1, 2], -Km[0, 2], Km[0, 1]]), q * dt / (2 * m))
        assert np.allclose(o["pplus"] - o["pminus"],
                           q * dt * Km @ ((o["pplus"] + o["pminus"]) / (2 * m * g)), atol=1e-13)


def test_secant_velocity_identity(orc):
    """Eq. rel-sec: K(pa) - K(pb) = Vdg(pa, pb) . (pa - pb), via the orbit velocity."""
    rng = np.random.default_rng(6)
    for _ in range(100):
        # with D = 0, Ap = Am = 0 and gphi = 0 the push is the identity and
        # vnew = Vdg(Pn, Pn) = v(Pn): compare with the definition of v(p)
        m, kappa = rng.uniform(0.5, 2), rng.uniform(0.5, 3)
        Pn = rng.standard_normal(3)
        z = np.zeros(3)
        o = orc.push(Pn, z, z, z, np.zeros((3, 3)), z, -1.0, m, kappa, 0.1)
        assert np.allclose(o["vnew"], Pn / (m * _gamma(Pn, m, kappa)), rtol=1e-14)


def test_push_nonrelativistic_limit(orc):
    """As kappa -> inf the step tends to the implicit-midpoint GM push of Part I:
    p^{n+1} - p^n = q dt (Ebar + K (p^n + p^{n+1}) / 2m), defect O(1/kappa^2)."""
    rng = np.random.default_rng(7)
    d = _rand_push_data(rng)
    defects = []
    for kappa in (10.0, 100.0, 1000.0):
        d["kappa"] = kappa
        o = orc.push(**d)
        q, m, dt = d["q"], d["m"], d["dt"]
        pn = d["Pn"] - q * d["Am"]
        pnp1 = o["Pnp1"] - q * d["Ap"]
        Ebar = -d["gphi"] - ((d["Ap"] - d["Am"]) / dt - d["D"] @ d["vbar"])
        Km = d["D"].T - d["D"]
        res = pnp1 - pn - q * dt * (Ebar + Km @ ((pn + pnp1) / (2 * m)))
        vres = o["vnew"] - (pn + pnp1) / (2 * m)
        defects.append(max(np.abs(res).max(), np.abs(vres).max()))
    assert defects[0] / defects[1] == pytest.approx(100.0, rel=0.05)
    assert defects[1] / defects[2] == pytest.approx(100.0, rel=0.05)


def test_push_reduces_to_mechanical_hc_in_linear_fields(orc):
    """Static linear potentials A = B x x / 2, phi = -E . x on a mesh: the orbit
    data give D = grad A, B_eff = B, gphi = -E, and the GM-HC step equals the
    mechanical kick-rotate-kick of Eq. hc-leapfrog-template with E and B."""
    n = 48
    L = 12.0
    o = orc.Oracle(3, [n, n, n], [L, L, L], [-L / 2] * 3, [(-1.0, 1.0)], dt=0.1, gl_points=8)
    xs = -L / 2 + np.arange(n) * L / n
    Z, Y, X = np.meshgrid(xs, xs, xs, indexing="ij")
    Bv = np.array([0.3, -0.5, 0.8])
    Ev = np.array([0.2, 0.1, -0.4])
    A = np.stack([0.5 * (Bv[1] * Z - Bv[2] * Y), 0.5 * (Bv[2] * X - Bv[0] * Z),
                  0.5 * (Bv[0] * Y - Bv[1] * X)]).reshape(3, -1)
    gphi_mesh = np.tile(-Ev[:, None], (1, n ** 3))
    x = np.array([0.13, -0.21, 0.07])
    vbar = np.array([0.35, -0.2, 0.4])
    od = o.orbit_data(x, vbar, gphi_mesh, A, A, None)
    assert np.allclose(od["D"], np.array([[0, -Bv[2], Bv[1]], [Bv[2], 0, -Bv[0]],
                                          [-Bv[1], Bv[0], 0]]) * 0.5, atol=1e-13)
    q, m, kap, dt = -1.0, 1.0, 1.0, 0.1
    pn = np.array([0.4, 0.1, -0.3])
    Pn = pn + q * od["Aminus"]
    r = orc.push(Pn, od["Aminus"], od["Aplus"], od["gphi"], od["D"], vbar, q, m, kap, dt)
    pm = pn + 0.5 * q * dt * Ev
    up, _ = orc.hc_map(pm / (m * kap), Bv, q * dt / (2 * m))
    pnp1 = m * kap * up + 0.5 * q * dt * Ev
    assert np.allclose(r["Pnp1"] - q * od["Aplus"], pnp1, atol=1e-13)


def test_frozen_orbit_map_unit_jacobian(orc):
    """Theorem fixed-volume: det d(x',P')/d(x,P) = 1 for the frozen-orbit map.
    A^n_h and A^{n+1}_h are mesh interpolants of smooth fields; gphi, D and
    vbar are frozen; x' = x + dt vbar."""
    n, L = 32, 2 * math.pi
    o = orc.Oracle(2, [n, n], [L, L], [0, 0], [(-1.0, 1.0)], dt=0.2)
    xs = np.arange(n) * L / n
    Y, X = np.meshgrid(xs, xs, indexing="ij")
    An = np.stack([0.3 * np.sin(Y), 0.4 * np.cos(X + 0.3), 0.2 * np.sin(X + Y)]).reshape(3, -1)
    Ap = np.stack([0.35 * np.sin(Y + 0.1), 0.4 * np.cos(X), 0.25 * np.sin(X - Y)]).reshape(3, -1)
    rng = np.random.default_rng(8)
    gphi = rng.standard_normal(3) * 0.2
    D = rng.standard_normal((3, 3)) * 0.4
    vbar = np.array([0.3, -0.25, 0.1])
    q, m, kap, dt = -1.0, 1.0, 1.0, 0.2

    def fmap(z):
        x, P = z[:2], z[2:]
        od = o.orbit_data(x, vbar, None, An, Ap, None)
        r = orc.push(P, od["Aminus"], od["Aplus"], gphi, D, vbar, q, m, kap, dt)
        return np.concatenate([x + dt * vbar[:2], r["Pnp1"]])

    z0 = np.array([1.1, 2.3, 0.2, -0.4, 0.3])
    h = 1e-6
    J = np.zeros((5, 5))
    for c in range(5):
        e = np.zeros(5); e[c] = h
        J[:, c] = (fmap(z0 + e) - fmap(z0 - e)) / (2 * h)
    assert np.linalg.det(J) == pytest.approx(1.0, abs=1e-7)


# ---------------------------------------------------------------- orbit quadrature (Sec. 2.4-2.5)
def _oracle2d(orc, n=16, project=1, dt=0.3):
    L = 2 * math.pi
    return orc.Oracle(2, [n, n], [L, L], [-math.pi, -math.pi], [(-1.0, 1.0)], dt=dt,
                      project=project, rho_bg=1.0)


def test_orbit_chain_rule_and_partition_of_unity(orc):
    """Lemma exact-chain-rule (R_A = 0) and sum_g Sbar_g = 1 for random orbits
    that cross several knots in both dimensions, and random mesh data."""
    rng = np.random.default_rng(9)
    for dt in (0.3, 1.0):
        o = _oracle2d(orc, dt=dt)
        Ng = o.Ng
        for _ in range(40):
            An = rng.standard_normal((3, Ng))
            Ap = rng.standard_normal((3, Ng))
            Uh = (Ap - An) / dt  # Eq. cn-A
            x = rng.uniform(-math.pi, math.pi, 2)
            vbar = rng.standard_normal(3) * 0.6
            od = o.orbit_data(x, vbar, None, An, Ap, Uh)
            RA = od["Aplus"] - od["Aminus"] - dt * (od["Ubar"] + od["D"] @ vbar)
            assert np.abs(RA).max() < 1e-13
            assert od["Sbar_sum"] == pytest.approx(1.0, abs=1e-14)
            assert np.all(od["D"][:, 2] == 0.0)  # ignorable z (reading R4)


def test_orbit_gather_linear_reproduction(orc):
    """Quadratic B-splines reproduce linear data: the orbit gather of a linear
    mesh field equals its value at the orbit midpoint, and D of a linear A is
    its exact gradient (away from the periodic wrap)."""
    o = _oracle2d(orc, n=32, dt=0.5)
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


def test_orbit_average_matches_exact_sympy_integral(orc):
    """Sbar_g = int_0^1 S_2(u0 + s delta - g) ds computed exactly by sympy."""
    import sympy as sp
    s = sp.symbols("s", real=True)

    def S2sym(xi):
        a = sp.Abs(xi)
        return sp.Rational(1, 2) * (sp.Max(sp.Rational(3, 2) - a, 0) ** 2
                                    - 3 * sp.Max(sp.Rational(1, 2) - a, 0) ** 2)

    n, L = 16, 16.0  # dx = 1
    o = orc.Oracle(1, [n], [L], [0.0], [(-1.0, 1.0)], dt=1.0)
    for u0, dl in [(sp.Rational(37, 10), sp.Rational(23, 10)), (sp.Rational(81, 10), sp.Rational(-17, 10)),
                   (sp.Rational(5, 1) + sp.Rational(1, 2), sp.Rational(3, 4))]:
        for g in range(int(u0) - 4, int(u0) + 5):
            ex = sp.integrate(S2sym(u0 + s * dl - g), (s, 0, 1))
            G = np.zeros((3, n)); G[0, g % n] = 1.0
            od = o.orbit_data(np.array([float(u0)]), np.array([float(dl), 0, 0]), G,
                              np.zeros((3, n)), np.zeros((3, n)), None)
            assert od["gphi"][0] == pytest.approx(float(ex), abs=2e-15)


def test_deposit_gather_adjointness(orc):
    """Eq. scatter-gather-work: sum_i q_i vbar_i . Gbar_i = sum_g J_g . G_g dV."""
    rng = np.random.default_rng(10)
    o = _oracle2d(orc, n=16, dt=0.4)
    npart = 64
    x = rng.uniform(-math.pi, math.pi, (2, npart))
    w = rng.uniform(0.5, 1.5, npart)
    o.set_particles(x, np.zeros((3, npart)), w)
    vbar = rng.standard_normal((3, npart)) * 0.5
    J = o.deposit(vbar.reshape(-1))
    G = rng.standard_normal((3, o.Ng))
    lhs = 0.0
    xs, _, _, _ = o.particles()
    for i in range(npart):
        od = o.orbit_data(xs[:, i], vbar[:, i], G, np.zeros_like(G), np.zeros_like(G), None)
        lhs += -w[i] * np.dot(vbar[:, i], od["gphi"])
    dV = (2 * math.pi / 16) ** 2
    rhs = np.sum(J.reshape(3, -1) * G) * dV
    assert lhs == pytest.approx(rhs, rel=1e-13)


# ---------------------------------------------------------------- projector and fields (Sec. 2.3, 4.5)
def test_projector_idempotent_selfadjoint_and_nyquist_example(orc):
    rng = np.random.default_rng(11)
    o = _oracle2d(orc, n=12)
    f = rng.standard_normal(3 * o.Ng)
    g = rng.standard_normal(3 * o.Ng)
    Pf = o.project(f, 3)
    assert np.allclose(o.project(Pf, 3), Pf, atol=1e-13)
    assert np.dot(Pf, g) == pytest.approx(np.dot(f, o.project(g, 3)), rel=1e-12)
    # Sec. 4.5 example: A_x = a (-1)^{j_y} has zero mesh curl but a nonzero orbit K
    jy = np.repeat(np.arange(12), 12)
    A = np.zeros((3, o.Ng)); A[0] = 0.1 * (-1.0) ** jy
    x = np.array([0.37, -1.11]); vbar = np.array([0.2, 0.3, 0.0])
    od = o.orbit_data(x, vbar, None, A, A, None)
    K = od["D"].T - od["D"]
    assert abs(K[0, 1]) > 1e-3
    zero = np.zeros(o.Ng)
    B_mesh_energy = o.field_energy(zero, A.reshape(-1), np.zeros(3 * o.Ng))
    assert B_mesh_energy < 1e-28  # represented curl vanishes
    PA = o.project(A.reshape(-1), 3)
    assert np.abs(PA).max() < 1e-15
    od2 = o.orbit_data(x, vbar, None, PA.reshape(3, -1), PA.reshape(3, -1), None)
    assert np.abs(od2["D"]).max() < 1e-15


def _started_2d(orc, n=16, npart=256, seed=12, dt=0.1):
    rng = np.random.default_rng(seed)
    o = _oracle2d(orc, n=n, dt=dt)
    x = rng.uniform(-math.pi, math.pi, (2, npart))
    u = rng.standard_normal((3, npart)) * 0.3
    w = np.full(npart, 4 * math.pi ** 2 / npart)
    o.set_particles(x, u, w)
    A = rng.standard_normal((3, o.Ng)) * 1e-2
    U = rng.standard_normal((3, o.Ng)) * 1e-2
    o.set_potentials(A, U)
    o.start()
    return o, rng


def test_cn_field_energy_balance_and_constraints(orc):
    """Eq. field-work-balance: W^{n+1} - W^n = -dt <J, E^{1/2}> for a prescribed
    projected current, with Gauss and Lorenz residuals staying at roundoff."""
    o, rng = _started_2d(orc)
    f0 = o.fields()
    g0, l0 = o.constraint_rms(f0["phi"], f0["psi"], f0["A"], f0["U"], f0["rho"])
    assert g0 < 1e-12 and l0 < 1e-13
    J = o.project(rng.standard_normal(3 * o.Ng) * 0.1, 3)
    out = o.field_solve(J)
    W0 = o.field_energy(f0["phi"], f0["A"], f0["U"])
    W1 = o.field_energy(out["phi_np1"], out["A_np1"], out["U_np1"])
    Eh = -out["gradphi_half"] - out["U_half"]
    dV = (2 * math.pi / 16) ** 2
    work = np.sum(J * Eh) * dV
    assert (W1 - W0) == pytest.approx(-0.1 * work, rel=1e-11, abs=1e-16)
    g1, l1 = o.constraint_rms(out["phi_np1"], out["psi_np1"], out["A_np1"], out["U_np1"],
                              out["rho_np1"])
    assert g1 < 1e-12 and l1 < 1e-13
    # continuity in real space, Eq. cn-continuity, with the spectral divergence
    Jh = [np.fft.fft2(J.reshape(3, 16, 16)[a]) for a in range(2)]
    k = 2 * np.pi * np.fft.fftfreq(16, d=2 * math.pi / 16)
    k[8] = 0.0
    div = np.real(np.fft.ifft2(1j * (k[None, :] * Jh[0] + k[:, None] * Jh[1]))).reshape(-1)
    assert np.allclose(out["rho_np1"], f0["rho"] - 0.1 * div, atol=1e-13)


def test_cn_solve_matches_closed_form_mode(orc):
    """A single vacuum mode (no source): the CN map of (A, U) is the Cayley
    rotation of the harmonic oscillator with frequency kappa |k|, so the
    discrete energy |U|^2 + kappa^2 k^2 |A|^2 is conserved exactly and the
    phase advance is 2 atan(dt w / 2)."""
    n, L = 16, 2 * math.pi
    o = orc.Oracle(1, [n], [L], [0.0], [(-1.0, 1.0)], dt=0.3)
    o.set_particles(np.zeros((1, 0)), np.zeros((3, 0)), np.zeros(0))
    xs = np.arange(n) * L / n
    A = np.zeros((3, n)); A[1] = np.cos(3 * xs)
    o.set_potentials(A, None)
    o.start()
    out = o.field_solve(np.zeros(3 * n))
    wdt = 3.0 * 0.3
    th = 2 * math.atan(wdt / 2)
    Ay = out["A_np1"].reshape(3, n)[1]
    assert np.allclose(Ay, math.cos(th) * np.cos(3 * xs), atol=1e-14)


# ---------------------------------------------------------------- whole step (Algorithm 1, Thm. energy)
def test_whole_step_conserves_energy_small_2d(orc):
    o, _ = _started_2d(orc, n=16, npart=512, dt=0.2)
    for _ in range(3):
        r = o.step(1e-12)
        assert r["status"] == 0
        assert abs(r["rel_dE"]) < 1e-11
        assert r["chain_rms"] < 1e-15
        assert abs(r["work_residual"]) < 1e-15
        assert r["gauss_rms"] < 1e-12 and r["lorenz_rms"] < 1e-12
        assert r["res_scaled_rms"] <= 1 and r["res_scaled_max"] <= 1


def test_failed_step_leaves_state_unchanged(orc):
    """Algorithm 1: a failed step returns a flag and leaves the accepted state
    unchanged, both for an inner failure (tolerance 0 cannot be met) and for an
    outer failure (outer limit 1 with a tolerance the outer test cannot meet)."""
    import oracle as O
    for tol, kw, expect in ((0.0, dict(), O.ORC_EINNER),
                            (1e-28, dict(outer_max=1, inner_tol_scale=1e18), O.ORC_EOUTER)):
        o3 = O.Oracle(2, [16, 16], [2 * math.pi] * 2, [-math.pi] * 2, [(-1.0, 1.0)], dt=0.1,
                      rho_bg=1.0, **kw)
        rng = np.random.default_rng(12)
        x = rng.uniform(-math.pi, math.pi, (2, 128))
        u = rng.standard_normal((3, 128)) * 0.3
        o3.set_particles(x, u, np.full(128, 4 * math.pi ** 2 / 128))
        o3.start()
        xa, Pa, _, _ = o3.particles()
        fa = o3.fields()
        r = o3.step(tol)
        assert r["status"] == expect
        xc, Pc, _, _ = o3.particles()
        fc = o3.fields()
        assert np.array_equal(xa, xc) and np.array_equal(Pa, Pc)
        for k in fa:
            assert np.array_equal(fa[k], fc[k])


def test_set_state_continues_a_run_exactly(orc):
    """The oracle's full-state restore (test support for derivative checks):
    a context given another's accepted state (canonical momenta and every
    mesh array) takes the same next step, to the last bit."""
    import oracle as O
    def make():
        o = O.Oracle(2, [16, 16], [2 * math.pi] * 2, [-math.pi] * 2, [(-1.0, 1.0)], dt=0.1,
                     rho_bg=1.0)
        rng = np.random.default_rng(12)
        x = rng.uniform(-math.pi, math.pi, (2, 128))
        u = rng.standard_normal((3, 128)) * 0.3
        o.set_particles(x, u, np.full(128, 4 * math.pi ** 2 / 128))
        o.start()
        return o
    a = make()
    assert a.step(1e-12)["status"] == 0
    x, P, w, sp = a.particles()
    b = O.Oracle(2, [16, 16], [2 * math.pi] * 2, [-math.pi] * 2, [(-1.0, 1.0)], dt=0.1,
                 rho_bg=1.0)
    b.set_state(x, P, w, sp, a.fields())
    ra, rb = a.step(1e-12), b.step(1e-12)
    assert ra["status"] == 0 and rb["status"] == 0
    for u, v in zip(a.particles(), b.particles()):
        assert np.array_equal(u, v)
    fa, fb = a.fields(), b.fields()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k


def test_two_stream_growth_rate_and_energy(orc):
    """1D3V two-stream with u = +-0.6, k = 0.5, dx = pi/16, seeded with the
    growing finite-grid eigenvector (Sec. 5.1): the k = 0.5 mode of E_x grows
    at Gamma_TS of Eq. gamma-ts with the finite-grid plasma frequency
    (0.2147689), and the relative total-energy change stays at the nonlinear
    tolerance level (Thm. energy)."""
    from oracle import closed_form as cf
    u0 = 0.6
    L, n = 4 * math.pi, 64
    G = cf.two_stream_rate(0.5, u0 / math.sqrt(1 + u0 * u0), L / n)
    cfg = pic_inputs.two_stream_1d(eigen_rate=G, eigen_chi=cf.chi(0.5, L / n))
    o = orc.Oracle(1, cfg["n"], cfg["L"], cfg["x0"], cfg["species"], dt=cfg["dt"],
                   rho_bg=cfg["rho_bg"])
    o.set_particles(cfg["x"], cfg["u"], cfg["w"], cfg["sp"])
    o.start()
    k = 2 * np.pi * np.fft.fftfreq(n, d=L / n)
    k[n // 2] = 0.0
    ts, amps, dE = [], [], 0.0
    for s in range(1, 61):
        r = o.step(cfg["tol"])
        assert r["status"] == 0
        assert r["inner_max"] <= 8 and r["outer_iters"] <= 20
        dE = max(dE, abs(r["rel_dE"]))
        f = o.fields()
        Ex = np.real(np.fft.ifft(-1j * k * np.fft.fft(f["phi"]))) - f["U"][:n]
        ts.append(s * cfg["dt"])
        amps.append(abs(np.fft.fft(Ex)[1]) / n)
    rate = np.polyfit(np.array(ts), np.log(np.array(amps)), 1)[0]
    assert rate == pytest.approx(G, rel=2e-3)
    assert dE < 1e-12
