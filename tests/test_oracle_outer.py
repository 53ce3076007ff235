"""Pins of the oracle's outer solve (Sec. 4.5, Algorithm 1, Eqs.
mixed-nonlinear-tests and anderson-type-two-update) on stand-in maps.

orc_step runs the same outer-solve code on the particle map; here it is fed
affine maps H(j) = M j + b, for which the mathematics fixes what it must do:

- the scaled tests of Eq. mixed-nonlinear-tests against values worked out by
  hand on a two-node vector (a dropped 1/2, an RMS over nodes instead of
  components, or a per-component instead of per-node norm all change them);
- damped Picard j + beta r before the iteration where Anderson becomes
  eligible (iterations counted from 1, so m_A = 2 leaves one Picard step);
- type-II Anderson with an untruncated history is GMRES in disguise (Walker
  and Ni, SIAM J. Numer. Anal. 49 (2011) 1715): the averaged iterate
  xbar_k = j_k - dJ gamma minimises |r| over the affine hull of the iterates
  so far, which is j_0 + K_k(A, r_0) with A = M - I, and the next iterate is
  xbar_k + beta r(xbar_k).  So the iterates are checked against a GMRES
  written here with numpy (least squares on an orthonormal Krylov basis), and
  the solve must converge once the Krylov space is the whole space;
- with a history window of m columns, xbar_k minimises |r| over the affine
  hull of the last m + 1 iterates;
- backtracking halves alpha until the scaled RMS residual decreases.
"""
import numpy as np
import pytest


def _affine(seed, n3, lo, hi):
    """Symmetric M with eigenvalues in [lo, hi] and a random b."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n3, n3)))
    lam = np.linspace(lo, hi, n3)
    M = (Q * lam) @ Q.T
    return M, rng.standard_normal(n3)


# tolerances: tau_a = tol * ratio dominates the denominators of the scaled
# tests, so acceptance and convergence follow the plain residual.  tau_a =
# 1e-9 of the O(1) initial residual: the Gram (normal-equation) solve of the
# Anderson update squares the condition number of the residual differences,
# so a step that is exact in exact arithmetic leaves about 1e-12 behind.
_PLAIN = dict(tol=1e-20, tol_abs_ratio=1e11)  # tau_a = 1e-9, tau_r = 1e-20


def test_scaled_tests_worked_by_hand(orc):
    # two nodes, component-major (x of both nodes, then y, then z)
    # node 0: r = (3, 0, 4), H = (6, 8, 0), j = 0;  node 1: r = 0, H = (0, 0, 2), j = (2, 0, 0)
    r = np.array([3.0, 0.0, 0.0, 0.0, 4.0, 0.0])
    H = np.array([6.0, 0.0, 8.0, 0.0, 0.0, 2.0])
    j = np.array([0.0, 2.0, 0.0, 0.0, 0.0, 0.0])
    # RMS over the 6 components: |r| 2.0412414523193151 (= sqrt(25/6)),
    # |H| 4.1633319989322652 (sqrt(104/6)), |j| 0.81649658092772603 (sqrt(4/6));
    # tau_r = 0.1, tau_a = 0.01: denominator 0.01 + 0.05 (4.16333 + 0.81650)
    # = 0.25899142899, scaled RMS 2.04124145232 / 0.25899142899 = 7.8815019488
    # node 0: |r_g| = 5, |H_g| = 10, |j_g| = 0: 5 / (0.01 + 0.05 * 10) = 9.8039215686
    # node 1: |r_g| = 0
    srms, smax = orc.scaled_tests(r, H, j, 0.1, 0.01)
    assert srms == pytest.approx(7.8815019488, rel=1e-10)
    assert smax == pytest.approx(9.8039215686, rel=1e-10)


def _gmres_iterate(M, b, j0, k):
    """argmin |M x + b - x| over x in j0 + K_k(M - I, r0), r0 = M j0 + b - j0."""
    A = M - np.eye(len(b))
    r0 = A @ j0 + b
    V = np.zeros((len(b), k))
    v = r0 / np.linalg.norm(r0)
    for i in range(k):  # Arnoldi with twice-repeated Gram-Schmidt
        V[:, i] = v
        w = A @ v
        for _ in range(2):
            w -= V[:, :i + 1] @ (V[:, :i + 1].T @ w)
        v = w / np.linalg.norm(w)
    y, *_ = np.linalg.lstsq(A @ V, -r0, rcond=None)
    return j0 + V @ y


def test_picard_before_anderson_becomes_eligible(orc):
    M, b = _affine(1, 6, -0.5, 0.9)
    st, _, rep, tr = orc.outer_affine(M, b, np.zeros(6), trace_cap=40, anderson_m=8,
                                      lambda_=0.0, **_PLAIN)
    assert st == 0
    beta = 0.5
    # iterations are counted from 1 and m_A = 2: the first is damped Picard
    # with alpha = 1, every later one Anderson
    assert tr["kind"][0] == 0 and tr["alpha"][0] == 1.0
    r = M @ tr["j"][0] + b - tr["j"][0]
    np.testing.assert_allclose(tr["j"][1], tr["j"][0] + beta * r, rtol=0, atol=1e-14)
    assert (tr["kind"][1:-1] == 1).all()
    # with m_A = 3 the first two are damped Picard
    st, _, rep, tr = orc.outer_affine(M, b, np.zeros(6), trace_cap=40, anderson_m=8,
                                      anderson_start=3, lambda_=0.0, **_PLAIN)
    assert st == 0
    assert (tr["kind"][:2] == 0).all() and (tr["kind"][2:-1] == 1).all()


def test_anderson_untruncated_is_gmres(orc):
    """Iterates against GMRES (Walker and Ni 2011); convergence once the Krylov
    space is the whole 6-dimensional space: the Anderson step of 0-based
    iteration 6 has six columns, so xbar_6 is the solution, j_7 = xbar_6 +
    beta r(xbar_6) too, and the tests pass at 0-based iteration 7
    (outer_iters = dim + 2)."""
    n3 = 6
    M, b = _affine(2, n3, -0.5, 0.9)
    j0 = np.zeros(n3)
    st, j, rep, tr = orc.outer_affine(M, b, j0, trace_cap=40, anderson_m=8, lambda_=0.0,
                                      **_PLAIN)
    assert st == 0
    xs = np.linalg.solve(np.eye(n3) - M, b)
    assert np.abs(j - xs).max() <= 1e-9 * np.abs(xs).max()
    assert rep["outer_iters"] <= n3 + 2
    beta = 0.5
    Bmat = (1 - beta) * np.eye(n3) + beta * M  # j_{k+1} = Bmat xbar_k + beta b when alpha = 1
    checked = 0
    for k in range(1, tr["kind"].size):
        if tr["kind"][k] != 1 or tr["alpha"][k] != 1.0 or k >= n3:
            continue
        xbar = np.linalg.solve(Bmat, tr["j"][k + 1] - beta * b)
        xg = _gmres_iterate(M, b, j0, k)
        assert np.abs(xbar - xg).max() <= 1e-11 * np.abs(xs).max(), k
        checked += 1
    assert checked >= n3 - 2


def test_anderson_regularisation_is_a_small_perturbation(orc):
    """lambda = 1e-12 (the paper's value) moves the solution by rounding only."""
    M, b = _affine(3, 6, -0.5, 0.9)
    st0, j0, _, _ = orc.outer_affine(M, b, np.zeros(6), anderson_m=8, lambda_=0.0, **_PLAIN)
    st1, j1, _, _ = orc.outer_affine(M, b, np.zeros(6), anderson_m=8, lambda_=1e-12, **_PLAIN)
    assert st0 == 0 and st1 == 0
    xs = np.linalg.solve(np.eye(6) - M, b)
    assert np.abs(j1 - j0).max() <= 1e-9 * np.abs(xs).max()


def test_truncated_history_window(orc):
    """With m = 2 history columns, xbar_k minimises |r| over the affine hull
    of the last three iterates j_{k-2}, j_{k-1}, j_k (the oldest column is
    dropped when the window is full)."""
    n3, m, beta = 9, 2, 0.5
    M, b = _affine(4, n3, -0.3, 0.95)
    # convergence with a window of 2 is slow here; 20 iterations show the window
    st, j, rep, tr = orc.outer_affine(M, b, np.zeros(n3), trace_cap=80, anderson_m=m,
                                      lambda_=0.0, outer_max=20, **_PLAIN)
    assert st == orc.ORC_EOUTER and rep["outer_iters"] == 20
    Bmat = (1 - beta) * np.eye(n3) + beta * M
    A = M - np.eye(n3)
    checked = 0
    for k in range(m + 2, tr["kind"].size - 1):
        if tr["kind"][k] != 1 or tr["alpha"][k] != 1.0 or tr["mh"][k - 1] < m:
            continue
        xbar = np.linalg.solve(Bmat, tr["j"][k + 1] - beta * b)
        J = tr["j"][k - m:k + 1]  # the last m + 1 iterates
        D = (J[:-1] - J[-1]).T    # hull directions
        y, *_ = np.linalg.lstsq(A @ D, -(A @ J[-1] + b), rcond=None)
        x_ref = J[-1] + D @ y
        scale = max(np.abs(xbar).max(), 1.0)
        assert np.abs(xbar - x_ref).max() <= 1e-10 * scale, k
        checked += 1
    assert checked >= 3


def test_backtracking_halves_alpha_until_the_residual_decreases(orc):
    """H(j) = -3 j + b: the damped Picard step j + beta r (beta = 1/2) maps
    r to (1 - 2 alpha) r, so alpha = 1 leaves |r| unchanged and is refused
    (a decrease by 1 - 1e-4 alpha is required); alpha = 1/2 lands on the
    fixed point.  Evaluations: the first, two trials, the verification."""
    M = -3.0 * np.eye(3)
    b = np.array([1.0, -2.0, 0.5])
    st, j, rep, tr = orc.outer_affine(M, b, np.zeros(3), trace_cap=10, anderson_start=50,
                                      **_PLAIN)
    assert st == 0
    assert tr["kind"][0] == 0 and tr["alpha"][0] == 0.5
    assert rep["outer_iters"] == 2 and rep["map_evals"] == 4
    np.testing.assert_allclose(j, b / 4.0, rtol=0, atol=1e-15)


def test_no_accepted_direction_fails(orc):
    """H(j) = -1e6 j + b: no alpha down to 1/64 reduces the residual of the
    damped Picard step (factor 1 - alpha (1 + 1e6) / 2), so the outer solve
    reports failure (ORC_EOUTER) after trying every step length."""
    M = -1e6 * np.eye(3)
    b = np.array([1.0, 1.0, 1.0])
    st, j, rep, tr = orc.outer_affine(M, b, np.zeros(3), trace_cap=10, anderson_start=50,
                                      **_PLAIN)
    assert st == orc.ORC_EOUTER
    assert rep["map_evals"] == 1 + 7
