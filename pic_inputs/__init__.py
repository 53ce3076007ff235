"""Seeded synthetic inputs for the relativistic two-stream and Weibel workloads.

This module is the only code that both the CUDA path and the oracle use.  It
draws particle positions, proper velocities, weights and seed potentials; it
contains none of the method's arithmetic (no shapes, no deposits, no field
solve, no push).  Every draw comes from ``numpy.random.default_rng(seed)``
(PCG64).

Conventions: positions are absolute coordinates, shaped (dim, N); velocities are
proper velocities u = gamma v (so p = m u), shaped (3, N); weights w are such
that a particle's charge and mass are w times its species' per-unit values;
mesh arrays are flattened with x fastest, vector arrays shaped (3, Ng).

Recipes (sizes of the paper's two test problems, Sec. 5, with the 1D/2D
workload sizes used here):
- ``two_stream_1d``: 1D3V cold relativistic two-stream; L = 2 pi / k with
  k = 0.5, 64 cells, two beams u_x = +-0.6, 32 particles/cell/beam on a quiet
  start (evenly spaced, the second beam offset by half a spacing), weights
  (rho0 L / N)(1 + 1e-3 cos k x), fixed neutralising background.
- ``weibel_2d``: 2D3V Weibel/filamentation; [-pi, pi]^2, counter-streaming
  beams u_z = +-u_d with an isotropic Maxwell-Juettner spread of temperature T
  (rest-frame sample by inverse transform of the tabulated CDF, then boosted
  with Zenitani's flipping method, Zenitani 2015), uniform random positions in
  each cell, random-phase A_z seed noise of amplitude 1e-4 over 1 <= |k| <= 8.
- ``weibel_2d_ions``: the large case with a mobile ion species of mass ratio
  100 at rest (same temperature in energy units) and no background.
- ``two_stream_ensemble``: many independent ``two_stream_1d`` instances with
  drawn mesh sizes, particles per cell and beam velocities.
- ``two_stream_2d``: 2D3V two-stream for the differentiation workload; box of
  side 4 pi, 256^2 cells, beams u_x = +-0.8 with Maxwell-Juettner T = 1e-3,
  100 particles/cell (6,553,600), density seed 1e-3 cos k x, dt = 0.05.
"""
from __future__ import annotations

import math

import numpy as np


def _mj_speed_samples(rng, theta: float, n: int) -> np.ndarray:
    """|u| samples of the rest-frame Maxwell-Juettner density u^2 exp(-gamma/theta)."""
    if theta <= 0.0 or n == 0:
        return np.zeros(n)
    gmax = 1.0 + 60.0 * theta
    umax = math.sqrt(gmax * gmax - 1.0)
    grid = np.linspace(0.0, umax, 40001)
    dens = grid ** 2 * np.exp(-(np.sqrt(1.0 + grid ** 2) - 1.0) / theta)
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (dens[1:] + dens[:-1]) * np.diff(grid))])
    cdf /= cdf[-1]
    return np.interp(rng.random(n), cdf, grid)


def _isotropic(rng, speed: np.ndarray) -> np.ndarray:
    n = speed.shape[0]
    cz = 2.0 * rng.random(n) - 1.0
    ph = 2.0 * math.pi * rng.random(n)
    sz = np.sqrt(np.maximum(0.0, 1.0 - cz * cz))
    return np.stack([speed * sz * np.cos(ph), speed * sz * np.sin(ph), speed * cz])


def drifting_mj(rng, theta: float, u_drift: float, axis: int, n: int) -> np.ndarray:
    """Proper velocities of a Maxwell-Juettner beam drifting with proper speed u_drift."""
    u = _isotropic(rng, _mj_speed_samples(rng, theta, n))
    if u_drift == 0.0:
        return u
    gd = math.sqrt(1.0 + u_drift * u_drift)
    bd = u_drift / gd
    gam = np.sqrt(1.0 + np.sum(u * u, axis=0))
    flip = -bd * u[axis] > rng.random(n) * gam
    u[axis] = np.where(flip, -u[axis], u[axis])
    u[axis] = gd * (u[axis] + bd * gam)
    return u


def _seed_noise_2d(rng, n, L, x0, amp, kmax, comp):
    nx, ny = n
    xs = x0[0] + np.arange(nx) * L[0] / nx
    ys = x0[1] + np.arange(ny) * L[1] / ny
    X, Y = np.meshgrid(xs, ys)  # shape (ny, nx): x fastest when flattened
    A = np.zeros((3, ny * nx))
    f = np.zeros((ny, nx))
    for kx in range(-kmax, kmax + 1):
        for ky in range(0, kmax + 1):
            if ky == 0 and kx <= 0:
                continue
            kk = math.hypot(kx, ky)
            if kk < 1.0 or kk > kmax:
                continue
            ph = 2.0 * math.pi * rng.random()
            f += (amp / kk) * np.cos(2 * math.pi * kx * (X - x0[0]) / L[0]
                                     + 2 * math.pi * ky * (Y - x0[1]) / L[1] + ph)
    A[comp] = f.reshape(-1)
    return A


def two_stream_1d(nx=64, ppc_beam=32, u0=0.6, k=0.5, pert=1e-3, dt=0.1, tol=1e-12,
                  steps=200, seed=0, eigen_rate=None, eigen_chi=None):
    """Quiet-start two-stream beams.

    Without ``eigen_rate`` the seed is the density modulation
    w ~ 1 + pert cos(k x) on both beams.  With ``eigen_rate`` (the growth rate
    Gamma of the cold relativistic two-stream branch) and ``eigen_chi`` (the
    shape factor chi_2(k)), the beams instead carry the growing cold-fluid
    eigenvector of Sec. 5.1 (velocities and relative weights driven by the
    gathered field chi E), scaled so that the relative density perturbation of
    each beam has amplitude ``pert``.  Both numbers are inputs: this module
    does not compute them.
    """
    L = 2.0 * math.pi / k
    x0 = -0.5 * L
    nb = nx * ppc_beam
    s = L / nb
    xa = x0 + (np.arange(nb) + 0.5) * s
    xb = x0 + (np.arange(nb) + 1.0) * s
    x = np.concatenate([xa, xb])
    N = x.shape[0]
    g0 = math.sqrt(1.0 + u0 * u0)
    v0 = u0 / g0
    vel = np.concatenate([np.full(nb, v0), np.full(nb, -v0)])
    if eigen_rate is None:
        w = (1.0 * L / N) * (1.0 + pert * np.cos(k * (x - x0)))
    else:
        om = 1j * eigen_rate
        qm = -1.0
        ph = np.exp(1j * k * (x - x0))
        dv = 1j * qm * eigen_chi / (g0 ** 3 * (om - k * vel))       # per unit field amplitude
        dn = k * dv / (om - k * vel)
        scale = pert / np.abs(dn).max()
        vel = vel + np.real(scale * dv * ph)
        w = (1.0 * L / N) * (1.0 + np.real(scale * dn * ph))
    u = np.zeros((3, N))
    u[0] = vel / np.sqrt(1.0 - vel * vel)
    perm = np.random.default_rng(seed).permutation(N)
    return dict(name=f"two_stream_1d_{nx}c_{2 * ppc_beam}ppc", dim=1, n=[nx], L=[L], x0=[x0],
                species=[(-1.0, 1.0)], rho_bg=1.0, dt=dt, tol=tol, steps=steps,
                x=x[perm][None, :].copy(), u=u[:, perm].copy(), w=w[perm].copy(),
                sp=np.zeros(N, np.int32), A=None, U=None)


def weibel_2d(n=128, ppc_beam=32, u_drift=0.5, T=0.01, dt=0.05, tol=1e-10, steps=500, seed=0,
              noise=1e-4, kmax=8):
    rng = np.random.default_rng(seed)
    L = [2.0 * math.pi, 2.0 * math.pi]
    x0 = [-math.pi, -math.pi]
    ncell = n * n
    nb = ncell * ppc_beam
    dx = L[0] / n
    cells = np.repeat(np.arange(ncell), ppc_beam)
    xs = []
    us = []
    for sgn in (1.0, -1.0):
        cx = cells % n
        cy = cells // n
        px = x0[0] + (cx + rng.random(nb)) * dx
        py = x0[1] + (cy + rng.random(nb)) * dx
        xs.append(np.stack([px, py]))
        us.append(drifting_mj(rng, T, sgn * u_drift, 2, nb))
    x = np.concatenate(xs, axis=1)
    u = np.concatenate(us, axis=1)
    N = x.shape[1]
    w = np.full(N, 1.0 * L[0] * L[1] / N)
    A = _seed_noise_2d(rng, (n, n), L, x0, noise, kmax, comp=2)
    return dict(name=f"weibel_2d_{n}x{n}_{2 * ppc_beam}ppc", dim=2, n=[n, n], L=L, x0=x0,
                species=[(-1.0, 1.0)], rho_bg=1.0, dt=dt, tol=tol, steps=steps,
                x=x, u=u, w=w, sp=np.zeros(N, np.int32), A=A, U=None)


def weibel_2d_ions(n=512, ppc_beam=64, ppc_ion=128, u_drift=0.9, T=0.05, mass_ratio=100.0,
                   dt=0.02, tol=1e-10, steps=2000, seed=0, noise=1e-4, kmax=8):
    e = weibel_2d(n=n, ppc_beam=ppc_beam, u_drift=u_drift, T=T, dt=dt, tol=tol, steps=steps,
                  seed=seed, noise=noise, kmax=kmax)
    rng = np.random.default_rng(seed + 1)
    ncell = n * n
    dx = e["L"][0] / n
    cells = np.repeat(np.arange(ncell), ppc_ion)
    ni = cells.shape[0]
    xi = np.stack([e["x0"][0] + (cells % n + rng.random(ni)) * dx,
                   e["x0"][1] + (cells // n + rng.random(ni)) * dx])
    ui = drifting_mj(rng, T / mass_ratio, 0.0, 2, ni)
    area = e["L"][0] * e["L"][1]
    ne = e["w"].shape[0]
    we = np.full(ne, area / ne)
    wi = np.full(ni, area / ni)
    return dict(name=f"weibel_2d_ions_{n}x{n}", dim=2, n=[n, n], L=e["L"], x0=e["x0"],
                species=[(-1.0, 1.0), (1.0, mass_ratio)], rho_bg=0.0, dt=dt, tol=tol,
                steps=steps, x=np.concatenate([e["x"], xi], axis=1),
                u=np.concatenate([e["u"], ui], axis=1), w=np.concatenate([we, wi]),
                sp=np.concatenate([np.zeros(ne, np.int32), np.ones(ni, np.int32)]),
                A=e["A"], U=None)


def two_stream_2d(n=256, ppc_beam=50, u_drift=0.8, T=1e-3, k=0.5, pert=1e-3, dt=0.05,
                  tol=1e-10, steps=50, seed=0):
    """2D3V relativistic two-stream (the differentiation workload): a square
    box of side 2 pi / k (k = 0.5: L = 4 pi), n^2 cells, counter-streaming
    electron beams u_x = +-u_drift with a Maxwell-Juettner spread of
    temperature T, ppc_beam particles per cell per beam at uniform random
    positions, weights (rho0 L^2 / N)(1 + pert cos k x), a fixed
    neutralising background.  Each particle's beam sign (+1 or -1) is
    returned as `beam`, so that a drift derivative can be seeded."""
    rng = np.random.default_rng(seed)
    Lx = 2.0 * math.pi / k
    L = [Lx, Lx]
    x0 = [-0.5 * Lx, -0.5 * Lx]
    ncell = n * n
    nb = ncell * ppc_beam
    dx = Lx / n
    cells = np.repeat(np.arange(ncell), ppc_beam)
    xs, us, beam = [], [], []
    for sgn in (1.0, -1.0):
        px = x0[0] + (cells % n + rng.random(nb)) * dx
        py = x0[1] + (cells // n + rng.random(nb)) * dx
        xs.append(np.stack([px, py]))
        us.append(drifting_mj(rng, T, sgn * u_drift, 0, nb))
        beam.append(np.full(nb, sgn))
    x = np.concatenate(xs, axis=1)
    u = np.concatenate(us, axis=1)
    N = x.shape[1]
    w = (Lx * Lx / N) * (1.0 + pert * np.cos(k * (x[0] - x0[0])))
    return dict(name=f"two_stream_2d_{n}x{n}_{2 * ppc_beam}ppc", dim=2, n=[n, n], L=L, x0=x0,
                species=[(-1.0, 1.0)], rho_bg=1.0, dt=dt, tol=tol, steps=steps,
                x=x, u=u, w=w, sp=np.zeros(N, np.int32), A=None, U=None,
                beam=np.concatenate(beam))


def thermal_box(dim=3, n=8, ppc=2, T=0.05, u_drift=0.3, dt=0.1, tol=1e-12, seed=0,
                L=2.0 * math.pi, noise=1e-3):
    """Counter-streaming Maxwell-Juettner beams along z in a periodic box of
    any dimension (used for parity checks in 1D-3D): uniform random positions
    per cell, `ppc` particles per cell split between the beams, a random
    vector-potential seed of amplitude `noise` on every node.  `n` is the
    node count of every axis, or a sequence of one count per axis (a box of
    side L on every axis, so the cells are not square then)."""
    rng = np.random.default_rng(seed)
    ns = [int(v) for v in n] if hasattr(n, "__len__") else [n] * dim
    assert len(ns) == dim
    Ls = [L] * dim
    x0 = [-0.5 * L] * dim
    ncell = int(np.prod(ns))
    cells = np.repeat(np.arange(ncell), ppc)
    N = cells.shape[0]
    idx = np.stack(np.unravel_index(cells, ns[::-1])[::-1])  # x fastest
    x = np.stack([x0[l] + (idx[l] + rng.random(N)) * Ls[l] / ns[l] for l in range(dim)])
    half = N // 2
    u = np.concatenate([drifting_mj(rng, T, u_drift, 2, half),
                        drifting_mj(rng, T, -u_drift, 2, N - half)], axis=1)
    perm = rng.permutation(N)
    u = u[:, perm]
    w = np.full(N, float(np.prod(Ls)) / N)
    A = noise * rng.standard_normal((3, ncell))
    return dict(name=f"thermal_box_{dim}d_{'x'.join(map(str, ns))}_{ppc}ppc", dim=dim, n=ns,
                L=Ls, x0=x0,
                species=[(-1.0, 1.0)], rho_bg=1.0, dt=dt, tol=tol, steps=4,
                x=x, u=u, w=w, sp=np.zeros(N, np.int32), A=A, U=None)


def _quiet_pairs_3d(n, L, x0, pairs):
    """Pair positions: the same `pairs` sub-cell offsets in every cell (a
    Weyl sequence in y and z, evenly spaced in x), so that deposits are
    uniform across cells and no transverse mode is seeded by the loading."""
    k = np.arange(pairs)
    sub = np.stack([(k + 0.5) / pairs, (k * 0.6180339887498949 + 0.25) % 1.0,
                    (k * 0.7548776662466927 + 0.5) % 1.0])
    ncell = n[0] * n[1] * n[2]
    cells = np.repeat(np.arange(ncell), pairs)
    ci = np.stack(np.unravel_index(cells, (n[2], n[1], n[0]))[::-1])
    return np.stack([x0[l] + (ci[l] + np.tile(sub[l], ncell)) * L[l] / n[l] for l in range(3)])


def two_stream_3d(n=32, pairs=10, v0=0.9, alpha=5e-3, dt=0.1, tol=1e-11, steps=600, *,
                  eigen_rate, eigen_chi):
    """3D3V cold relativistic two-stream of Sec. 5.1 (TSI, Table 1): [-4 pi, 4 pi]^3,
    pairs of electrons at +-v0 along x in every cell, seeded with the growing
    cold-fluid eigenvector whose grid density is alpha rho0 cos(k x) and
    E_x = (sigma1 alpha rho0 / k) sin(k x), k = 1/4; the particle responses use
    the gathered field chi_2(k) E_x.  eigen_rate (Gamma_TS) and eigen_chi are
    inputs, not computed here."""
    L = [8.0 * math.pi] * 3
    x0 = [-4.0 * math.pi] * 3
    ns = [n, n, n]
    k = 2.0 * math.pi / L[0]
    xp = _quiet_pairs_3d(ns, L, x0, pairs)
    m = xp.shape[1]
    g0 = 1.0 / math.sqrt(1.0 - v0 * v0)
    om = 1j * eigen_rate
    Ehat = -1j * alpha / k  # E_x = Re(Ehat e^{ikx}) = (alpha / k) sin(kx), sigma1 = rho0 = 1
    ph = np.exp(1j * k * xp[0])
    xs, us, ws = [], [], []
    for sgn in (1.0, -1.0):
        vs = sgn * v0
        dv = 1j * (-1.0) * eigen_chi * Ehat / (g0 ** 3 * (om - k * vs))
        dn = k * dv / (om - k * vs)
        vx = vs + np.real(dv * ph)
        u = np.zeros((3, m))
        u[0] = vx / np.sqrt(1.0 - vx * vx)
        xs.append(xp)
        us.append(u)
        ws.append(1.0 + np.real(dn * ph))
    N = 2 * m
    w = np.concatenate(ws) * (float(np.prod(L)) / N)
    return dict(name=f"two_stream_3d_{n}cubed_{pairs}pairs", dim=3, n=ns, L=L, x0=x0,
                species=[(-1.0, 1.0)], rho_bg=1.0, dt=dt, tol=tol, steps=steps,
                x=np.concatenate(xs, axis=1), u=np.concatenate(us, axis=1), w=w,
                sp=np.zeros(N, np.int32), A=None, U=None)


def weibel_3d(n=32, pairs=25, v0=0.9, B0=1e-4, dt=0.04, tol=1e-11, steps=2500, *,
              eigen_rate, eigen_chi):
    """3D3V cold relativistic Weibel/filamentation of Sec. 5.2 (WBI, Table 1):
    [-pi, pi]^3, pairs of electrons at +-v0 along x, seeded with the growing
    eigenmode of Eqs. weibel-initial-fields and weibel-initial-particles
    (k_y = 1): A_x = (B0/k) cos(k y), U_x = Gamma_W A_x, and per beam
    v_x = s v0 + chi B0 cos(k y) / (k g0^3), v_y = s chi v0 B0 sin(k y) / (g0 Gamma_W),
    w = 1 - s chi v0 k B0 cos(k y) / (g0 Gamma_W^2).  eigen_rate (Gamma_W) and
    eigen_chi are inputs, not computed here."""
    L = [2.0 * math.pi] * 3
    x0 = [-math.pi] * 3
    ns = [n, n, n]
    k = 2.0 * math.pi / L[1]
    xp = _quiet_pairs_3d(ns, L, x0, pairs)
    m = xp.shape[1]
    g0 = 1.0 / math.sqrt(1.0 - v0 * v0)
    G = eigen_rate
    y = xp[1]
    xs, us, ws = [], [], []
    for sgn in (1.0, -1.0):
        vx = sgn * v0 + eigen_chi * B0 * np.cos(k * y) / (k * g0 ** 3)
        vy = sgn * eigen_chi * v0 * B0 * np.sin(k * y) / (g0 * G)
        gam = 1.0 / np.sqrt(1.0 - vx * vx - vy * vy)
        u = np.zeros((3, m))
        u[0] = gam * vx
        u[1] = gam * vy
        xs.append(xp)
        us.append(u)
        ws.append(1.0 - sgn * eigen_chi * v0 * k * B0 * np.cos(k * y) / (g0 * G * G))
    N = 2 * m
    w = np.concatenate(ws) * (float(np.prod(L)) / N)
    ys = x0[1] + np.arange(n) * L[1] / n
    Ax = np.broadcast_to((B0 / k) * np.cos(k * ys)[None, :, None], (n, n, n)).reshape(-1)
    A = np.zeros((3, n ** 3))
    U = np.zeros((3, n ** 3))
    A[0] = Ax
    U[0] = G * Ax
    return dict(name=f"weibel_3d_{n}cubed_{pairs}pairs", dim=3, n=ns, L=L, x0=x0,
                species=[(-1.0, 1.0)], rho_bg=1.0, dt=dt, tol=tol, steps=steps,
                x=np.concatenate(xs, axis=1), u=np.concatenate(us, axis=1), w=w,
                sp=np.zeros(N, np.int32), A=A, U=U)


def two_stream_ensemble(B=256, seed=0, nx_choices=(32, 64, 128, 256, 512), ppc_range=(16, 256),
                        u_range=(0.2, 0.95), dt=0.1, tol=1e-10, steps=1000, pert=1e-3):
    """An ensemble of B independent 1D3V two-stream instances on L = 4 pi
    (k = 0.5): per instance a mesh size drawn uniformly from ``nx_choices``, an
    even particle count per cell drawn uniformly from ``ppc_range`` (half per
    beam), a beam proper velocity u drawn uniformly from ``u_range``, and its
    own storage-order seed.  Each instance is ``two_stream_1d`` with those
    values."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(B):
        nx = int(rng.choice(nx_choices))
        ppc = int(rng.integers(ppc_range[0] // 2, ppc_range[1] // 2 + 1)) * 2
        u0 = float(rng.uniform(*u_range))
        out.append(two_stream_1d(nx=nx, ppc_beam=ppc // 2, u0=u0, k=0.5, pert=pert, dt=dt,
                                 tol=tol, steps=steps, seed=seed * 100003 + b))
    return out


def random_fields(rng, Ng, scale=1e-2):
    """Smooth-free random mesh data for unit-level parity checks."""
    return scale * rng.standard_normal((3, Ng))
