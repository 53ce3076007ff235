"""Shared test set-up: builds the same seeded problem for the CUDA path and the
oracle.  Imports both sides but adds no arithmetic of its own."""
import math

import numpy as np

import pic_inputs


def small_2d(n=16, ppc=8, T=0.01, u_drift=0.5, dt=0.1, seed=3, noise=1e-3):
    return pic_inputs.weibel_2d(n=n, ppc_beam=ppc // 2, u_drift=u_drift, T=T, dt=dt, tol=1e-12,
                                steps=4, seed=seed, noise=noise, kmax=3)


def small_1d(nx=64, ppc_beam=32):
    return pic_inputs.two_stream_1d(nx=nx, ppc_beam=ppc_beam)


def make_oracle(cfg, **kw):
    import oracle
    o = oracle.Oracle(cfg["dim"], cfg["n"], cfg["L"], cfg["x0"], cfg["species"], dt=cfg["dt"],
                      rho_bg=cfg["rho_bg"], **kw)
    o.set_particles(cfg["x"], cfg["u"], cfg["w"], cfg["sp"])
    o.set_potentials(cfg["A"], cfg["U"])
    return o


def make_gpu(cfg, precision=0, **kw):
    import paper_2609_36383_b300 as P
    sim = P.Simulation(cfg["dim"], cfg["n"], cfg["L"], cfg["x0"], cfg["species"], cfg["dt"],
                       precision=precision, rho_bg=cfg["rho_bg"], **kw)
    sim.set_particles(cfg["x"], cfg["u"], cfg["w"], cfg["sp"])
    sim.set_potentials(cfg["A"], cfg["U"])
    return sim


def rel_err(a, b):
    a = np.asarray(a, float); b = np.asarray(b, float)
    den = max(np.abs(b).max(), 1e-300)
    return np.abs(a - b).max() / den


def periodic_diff(xa, xb, L):
    d = np.asarray(xa) - np.asarray(xb)
    L = np.asarray(L, float).reshape(-1, 1)
    return d - L * np.round(d / L)


def gross_scales(cfg):
    """Gross magnitudes of the deposited mesh quantities: rounding in a sum is
    bounded by eps * sum |terms|, so deposit parity is measured against the
    one-sign density sum_i |q_i| / V (+ |rho_bg|) and the matching current
    sum_i |q_i| |v_i|_inf / V, not against the (cancelling) net values."""
    q = np.array([cfg["species"][s][0] for s in cfg["sp"]]) * cfg["w"]
    V = float(np.prod(cfg["L"]))
    u = np.asarray(cfg["u"])
    v = u / np.sqrt(1.0 + np.sum(u * u, axis=0))
    rho = np.abs(q).sum() / V + abs(cfg["rho_bg"])
    J = (np.abs(q) * np.abs(v).max(axis=0)).sum() / V if q.size else 0.0
    return dict(rho=rho, J=J, H=J)


def scaled_err(a, b, floor=0.0):
    """max |a - b| / max(max |b|, floor)"""
    a = np.asarray(a, float); b = np.asarray(b, float)
    den = max(np.abs(b).max() if b.size else 0.0, floor, 1e-300)
    return np.abs(a - b).max() / den if a.size else 0.0
