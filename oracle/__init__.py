"""Plain FP64 CPU oracle of the GM-HC-CN implicit PIC step (arxiv 2609.36383).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library ``paper_2609_36383_b300`` and neither imports the other;
the only module both sides use is ``pic_inputs`` (seeded input generation,
which holds none of the method's arithmetic).

The arithmetic lives in ``pic_oracle.c`` (see its header for the sections of
the paper it follows).  This module compiles it with gcc and wraps it with
ctypes and numpy.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pic_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

ORC_OK, ORC_EARG, ORC_EINNER, ORC_EOUTER = 0, -1, -4, -5


def build(force: bool = False) -> str:
    """Compile pic_oracle.c into liboracle.so (gcc, -O2, OpenMP)."""
    src_m = os.path.getmtime(_SRC)
    hdr_m = os.path.getmtime(os.path.join(_HERE, "pic_oracle.h"))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(src_m, hdr_m):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared",
               "-Wall", "-Wno-unused-function", _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class _Params(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("n", C.c_int * 3), ("L", C.c_double * 3), ("x0", C.c_double * 3),
        ("dt", C.c_double), ("kappa", C.c_double), ("sigma1", C.c_double), ("sigma2", C.c_double),
        ("rho_bg", C.c_double),
        ("project", C.c_int), ("gl_points", C.c_int), ("inner_max", C.c_int), ("outer_max", C.c_int),
        ("anderson_m", C.c_int), ("anderson_start", C.c_int), ("backtrack_levels", C.c_int),
        ("beta", C.c_double), ("lambda_", C.c_double), ("decrease_coef", C.c_double),
        ("growth_limit", C.c_double), ("tol_abs_ratio", C.c_double), ("inner_tol_scale", C.c_double),
        ("nspecies", C.c_int), ("q", C.c_double * 4), ("m", C.c_double * 4),
        ("order", C.c_int), ("refine_max", C.c_int), ("growth_scaled", C.c_int),
    ]


class OuterTrace(C.Structure):
    _fields_ = [("cap", C.c_int), ("j", C.POINTER(C.c_double)), ("srms", C.POINTER(C.c_double)),
                ("smax", C.POINTER(C.c_double)), ("kind", C.POINTER(C.c_int)),
                ("alpha", C.POINTER(C.c_double)), ("mh", C.POINTER(C.c_int)), ("n", C.c_int)]


class Report(C.Structure):
    _fields_ = [
        ("W", C.c_double), ("K", C.c_double), ("E_tot", C.c_double), ("rel_dE", C.c_double),
        ("gauss_rms", C.c_double), ("lorenz_rms", C.c_double), ("work_residual", C.c_double),
        ("chain_rms", C.c_double), ("res_scaled_rms", C.c_double), ("res_scaled_max", C.c_double),
        ("outer_iters", C.c_int), ("map_evals", C.c_int), ("inner_max", C.c_int),
        ("inner_mean", C.c_double), ("status", C.c_int),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.POINTER(_Params)]
        L.orc_free.argtypes = [C.c_void_p]
        L.orc_set_particles.argtypes = [C.c_void_p, C.c_long, _I, _D, _D, C.c_int, _D]
        L.orc_set_potentials.argtypes = [C.c_void_p, _D, _D]
        L.orc_start.argtypes = [C.c_void_p, C.POINTER(Report)]
        L.orc_step.argtypes = [C.c_void_p, C.c_double, C.POINTER(Report)]
        L.orc_eval_map.argtypes = [C.c_void_p, _D, C.c_double, _D, _D, _D, _I]
        L.orc_num_particles.restype = C.c_long
        L.orc_num_particles.argtypes = [C.c_void_p]
        L.orc_last_refined.restype = C.c_long
        L.orc_last_refined.argtypes = [C.c_void_p]
        L.orc_S1.restype = C.c_double
        L.orc_S1.argtypes = [C.c_double]
        L.orc_dS1.restype = C.c_double
        L.orc_dS1.argtypes = [C.c_double]
        L.orc_get_particles.argtypes = [C.c_void_p, _D, _D, _D, _I]
        L.orc_get_fields.argtypes = [C.c_void_p, _D, _D, _D, _D, _D, _D]
        L.orc_set_fields.argtypes = [C.c_void_p, _D, _D, _D, _D, _D, _D]
        L.orc_knot_jumps.argtypes = [C.c_void_p, C.c_double, _D, _D]
        L.orc_set_state.argtypes = [C.c_void_p, C.c_long, C.POINTER(C.c_int), _D, _D, _D, _D, _D,
                                    _D, _D, _D, _D]
        L.orc_S2.restype = C.c_double
        L.orc_S2.argtypes = [C.c_double]
        L.orc_dS2.restype = C.c_double
        L.orc_dS2.argtypes = [C.c_double]
        L.orc_gauss_legendre.argtypes = [C.c_int, _D, _D]
        L.orc_dft.argtypes = [C.c_int, _I, _D, _D, _D, _D, C.c_int]
        L.orc_hc_map.argtypes = [_D, _D, C.c_double, _D, _D]
        L.orc_push.argtypes = [_D, _D, _D, _D, _D, _D, C.c_double, C.c_double, C.c_double,
                               C.c_double, _D, _D, _D, _D]
        L.orc_orbit_data.argtypes = [C.c_void_p, _D, _D, _D, _D, _D, _D, _D, _D, _D, _D, _D, _D]
        L.orc_field_solve.argtypes = [C.c_void_p, _D, _D, _D, _D, _D, _D, _D, _D]
        L.orc_field_energy.restype = C.c_double
        L.orc_field_energy.argtypes = [C.c_void_p, _D, _D, _D]
        L.orc_constraint_rms.argtypes = [C.c_void_p, _D, _D, _D, _D, _D, _D, _D]
        L.orc_project.argtypes = [C.c_void_p, _D, C.c_int]
        L.orc_deposit.argtypes = [C.c_void_p, _D, _D]
        L.orc_eval_particles.argtypes = [C.c_void_p, _D, C.c_double, C.c_long,
                                         C.POINTER(C.c_long), _D, _D, _I]
        L.orc_scaled_tests.argtypes = [C.c_long, _D, _D, _D, C.c_double, C.c_double, _D, _D]
        L.orc_outer_affine.argtypes = [C.POINTER(_Params), C.c_long, _D, _D, _D, C.c_double,
                                       C.POINTER(OuterTrace), C.POINTER(Report)]
    return _lib


def _p(a):
    """Pointer to a contiguous float64 numpy array (or NULL)."""
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def _pi(a):
    if a is None:
        return None
    assert a.dtype == np.int32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_I)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# paper defaults (Sec. 5 parameter paragraph and Table 1)
DEFAULTS = dict(dt=0.1, kappa=1.0, sigma1=1.0, sigma2=1.0, rho_bg=0.0, project=1, gl_points=8,
                inner_max=64, outer_max=80, anderson_m=4, anderson_start=2, backtrack_levels=7,
                beta=0.5, lambda_=1e-12, decrease_coef=1e-4, growth_limit=1.2,
                tol_abs_ratio=0.01, inner_tol_scale=1.0, order=2, refine_max=0,
                growth_scaled=0)


def S2(xi: float) -> float:
    return lib().orc_S2(float(xi))


def dS2(xi: float) -> float:
    return lib().orc_dS2(float(xi))


def S1(xi: float) -> float:
    return lib().orc_S1(float(xi))


def dS1(xi: float) -> float:
    return lib().orc_dS1(float(xi))


def gauss_legendre(n: int):
    t = np.zeros(n)
    w = np.zeros(n)
    lib().orc_gauss_legendre(n, _p(t), _p(w))
    return t, w


def dft(f, inverse=False):
    """Direct DFT of a real or complex array shaped (n_z.., n_y, n_x) with x fastest."""
    f = np.asarray(f)
    dim = f.ndim
    n = (C.c_int * 3)(*([*f.shape[::-1]] + [1] * (3 - dim)))
    re = _f64(f.real)
    im = _f64(f.imag) if np.iscomplexobj(f) else np.zeros_like(re)
    ore = np.zeros_like(re)
    oim = np.zeros_like(re)
    lib().orc_dft(dim, n, _p(re), _p(im), _p(ore), _p(oim), 1 if inverse else 0)
    return ore + 1j * oim


def hc_map(um, B, qdt_2m):
    um = _f64(um); B = _f64(B)
    up = np.zeros(3)
    g = C.c_double(0.0)
    lib().orc_hc_map(_p(um), _p(B), float(qdt_2m), _p(up), C.byref(g))
    return up, g.value


def push(Pn, Am, Ap, gphi, D, vbar, q, m, kappa, dt):
    args = [_f64(a) for a in (Pn, Am, Ap, gphi, np.asarray(D).reshape(9), vbar)]
    outs = [np.zeros(3) for _ in range(4)]
    lib().orc_push(*[_p(a) for a in args], float(q), float(m), float(kappa), float(dt),
                   *[_p(o) for o in outs])
    return dict(pminus=outs[0], pplus=outs[1], Pnp1=outs[2], vnew=outs[3])


def scaled_tests(r, H, j, tau_r, tau_a):
    """Eq. mixed-nonlinear-tests on mesh vectors of 3 components per node,
    component-major (3 x Ng): (scaled RMS, scaled maximum-node residual)."""
    r, H, j = _f64(r).reshape(-1), _f64(H).reshape(-1), _f64(j).reshape(-1)
    srms, smax = C.c_double(), C.c_double()
    lib().orc_scaled_tests(r.size // 3, _p(r), _p(H), _p(j), float(tau_r), float(tau_a),
                           C.byref(srms), C.byref(smax))
    return srms.value, smax.value


def outer_affine(M, b, j0, tol, trace_cap=0, **opts):
    """The outer solve of Algorithm 1 (the code orc_step runs) on the affine
    map H(j) = M j + b over 3 Ng components.  Returns (status, last iterate,
    report, trace); trace holds per outer iteration the iterate its tests ran
    at, its scaled residuals, the accepted direction kind (0 Picard, 1
    Anderson, 2 Picard after a rejected Anderson direction, -1 none), the
    accepted step length and the history size after the update."""
    M = _f64(M)
    b = _f64(b).reshape(-1)
    j = _f64(j0).reshape(-1).copy()
    N3 = b.size
    assert N3 % 3 == 0 and M.shape == (N3, N3)
    prm = _Params()
    for k, v in {**DEFAULTS, **opts}.items():
        if hasattr(prm, k):
            setattr(prm, k, v)
    tr = OuterTrace()
    cap = int(trace_cap)
    buf = dict(j=np.zeros((max(cap, 1), N3)), srms=np.zeros(max(cap, 1)),
               smax=np.zeros(max(cap, 1)), kind=np.zeros(max(cap, 1), np.int32),
               alpha=np.zeros(max(cap, 1)), mh=np.zeros(max(cap, 1), np.int32))
    tr.cap = cap
    for k in ("j", "srms", "smax", "alpha"):
        setattr(tr, k, buf[k].ctypes.data_as(_D))
    for k in ("kind", "mh"):
        setattr(tr, k, buf[k].ctypes.data_as(_I))
    rep = Report()
    st = lib().orc_outer_affine(C.byref(prm), N3 // 3, _p(M), _p(b), _p(j), float(tol),
                                C.byref(tr), C.byref(rep))
    n = tr.n
    trace = {k: v[:n] for k, v in buf.items()}
    return st, j, rep.as_dict(), trace


class Oracle:
    """One oracle simulation context (FP64, CPU)."""

    def __init__(self, dim, n, L, x0, species, **kw):
        prm = dict(DEFAULTS)
        prm.update(kw)
        P = _Params()
        P.dim = dim
        n3 = list(n) + [1] * (3 - len(n))
        L3 = list(L) + [1.0] * (3 - len(L))
        x3 = list(x0) + [0.0] * (3 - len(x0))
        for a in range(3):
            P.n[a] = int(n3[a]); P.L[a] = float(L3[a]); P.x0[a] = float(x3[a])
        for k, v in prm.items():
            setattr(P, k, v)
        P.nspecies = len(species)
        for s, (q, m) in enumerate(species):
            P.q[s] = q; P.m[s] = m
        self.dim = dim
        self.n = [int(v) for v in n3[:dim]]
        self.Ng = int(np.prod(self.n))
        self.prm = prm
        self._h = lib().orc_create(C.byref(P))
        if not self._h:
            raise ValueError("orc_create rejected the parameters")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_free(h)
            self._h = None

    # -- set-up -----------------------------------------------------------
    def set_particles(self, x, u_or_P, w, species=None, canonical=False):
        x = _f64(x); u = _f64(u_or_P); w = _f64(w)
        npart = w.shape[0]
        sp = np.zeros(npart, np.int32) if species is None else np.ascontiguousarray(species, np.int32)
        st = lib().orc_set_particles(self._h, npart, _pi(sp), _p(x), _p(u), int(canonical), _p(w))
        if st:
            raise ValueError(f"orc_set_particles: {st}")

    def set_potentials(self, A=None, U=None):
        A = None if A is None else _f64(A)
        U = None if U is None else _f64(U)
        lib().orc_set_potentials(self._h, _p(A), _p(U))

    def start(self) -> dict:
        r = Report()
        lib().orc_start(self._h, C.byref(r))
        return r.as_dict()

    # -- stepping -----------------------------------------------------------
    def step(self, tol) -> dict:
        r = Report()
        lib().orc_step(self._h, float(tol), C.byref(r))
        return r.as_dict()

    def eval_map(self, j, tol):
        npart = self.num_particles()
        j = _f64(j)
        H = np.zeros(3 * self.Ng)
        vb = np.zeros(3 * npart)
        Pn = np.zeros(3 * npart)
        it = np.zeros(npart, np.int32)
        st = lib().orc_eval_map(self._h, _p(j), float(tol), _p(H), _p(vb), _p(Pn), _pi(it))
        return st, H, vb.reshape(3, npart), Pn.reshape(3, npart), it

    def eval_particles(self, j, tol, idx):
        """Inner solves of the particles ``idx`` at trial current j (no deposit)."""
        idx = np.ascontiguousarray(idx, np.int64)
        k = idx.shape[0]
        vb = np.zeros(3 * k); Pn = np.zeros(3 * k); it = np.zeros(k, np.int32)
        st = lib().orc_eval_particles(self._h, _p(_f64(j)), float(tol), k,
                                      idx.ctypes.data_as(C.POINTER(C.c_long)), _p(vb), _p(Pn),
                                      _pi(it))
        return st, vb.reshape(3, k), Pn.reshape(3, k), it

    # -- state access -------------------------------------------------------
    def num_particles(self) -> int:
        return int(lib().orc_num_particles(self._h))

    def refined(self) -> int:
        """Particles that needed substeps in the last map evaluation."""
        return int(lib().orc_last_refined(self._h))

    def particles(self):
        npart = self.num_particles()
        x = np.zeros(self.dim * npart); P = np.zeros(3 * npart); w = np.zeros(npart)
        sp = np.zeros(npart, np.int32)
        lib().orc_get_particles(self._h, _p(x), _p(P), _p(w), _pi(sp))
        return x.reshape(self.dim, npart), P.reshape(3, npart), w, sp

    def fields(self) -> dict:
        N = self.Ng
        out = dict(phi=np.zeros(N), psi=np.zeros(N), A=np.zeros(3 * N), U=np.zeros(3 * N),
                   rho=np.zeros(N), J=np.zeros(3 * N))
        lib().orc_get_fields(self._h, *[_p(out[k]) for k in ("phi", "psi", "A", "U", "rho", "J")])
        return out

    def set_fields(self, phi=None, psi=None, A=None, U=None, rho=None, J=None):
        vals = [None if v is None else _f64(v) for v in (phi, psi, A, U, rho, J)]
        lib().orc_set_fields(self._h, *[_p(v) for v in vals])

    def knot_jumps(self, eps=1e-8):
        """(E_shape jump, grad A jump) maxima over the interpolant's knots (Sec. 5.3)."""
        Ej, Gj = C.c_double(0.0), C.c_double(0.0)
        lib().orc_knot_jumps(self._h, float(eps), C.byref(Ej), C.byref(Gj))
        return Ej.value, Gj.value

    def set_state(self, x, P, w, species, fields):
        """A full accepted state (canonical momenta, every mesh array); the
        context is started and steps on from it."""
        x = _f64(x); P = _f64(P); w = _f64(w)
        sp = np.ascontiguousarray(species, np.int32)
        f = {k: _f64(fields[k]) for k in ("phi", "psi", "A", "U", "rho", "J")}
        st = lib().orc_set_state(self._h, w.shape[0], _pi(sp), _p(x), _p(P), _p(w),
                                 *[_p(f[k]) for k in ("phi", "psi", "A", "U", "rho", "J")])
        if st:
            raise ValueError(f"orc_set_state: {st}")

    # -- unit-level pieces ------------------------------------------------
    def field_solve(self, j):
        N = self.Ng
        out = dict(gradphi_half=np.zeros(3 * N), A_np1=np.zeros(3 * N), U_half=np.zeros(3 * N),
                   phi_np1=np.zeros(N), psi_np1=np.zeros(N), U_np1=np.zeros(3 * N),
                   rho_np1=np.zeros(N))
        lib().orc_field_solve(self._h, _p(_f64(j)), *[_p(out[k]) for k in (
            "gradphi_half", "A_np1", "U_half", "phi_np1", "psi_np1", "U_np1", "rho_np1")])
        return out

    def field_energy(self, phi, A, U) -> float:
        return lib().orc_field_energy(self._h, _p(_f64(phi)), _p(_f64(A)), _p(_f64(U)))

    def constraint_rms(self, phi, psi, A, U, rho):
        g = C.c_double(); l = C.c_double()
        lib().orc_constraint_rms(self._h, *[_p(_f64(v)) for v in (phi, psi, A, U, rho)],
                                 C.byref(g), C.byref(l))
        return g.value, l.value

    def project(self, f, ncomp):
        f = _f64(f).copy()
        lib().orc_project(self._h, _p(f), int(ncomp))
        return f

    def deposit(self, vbar):
        J = np.zeros(3 * self.Ng)
        st = lib().orc_deposit(self._h, _p(_f64(vbar)), _p(J))
        if st:
            raise ValueError("orbit wider than the oracle's node window")
        return J

    def orbit_data(self, x, vbar, gradphi, An, Anp1, Uhalf):
        out = dict(gphi=np.zeros(3), Ubar=np.zeros(3), D=np.zeros(9), Aplus=np.zeros(3),
                   Aminus=np.zeros(3))
        ssum = C.c_double()
        st = lib().orc_orbit_data(self._h, _p(_f64(x)), _p(_f64(vbar)),
                                  _p(None if gradphi is None else _f64(gradphi)),
                                  _p(_f64(An)), _p(_f64(Anp1)),
                                  _p(None if Uhalf is None else _f64(Uhalf)),
                                  *[_p(out[k]) for k in ("gphi", "Ubar", "D", "Aplus", "Aminus")],
                                  C.byref(ssum))
        if st:
            raise ValueError("orbit wider than the oracle's node window")
        out["D"] = out["D"].reshape(3, 3)
        out["Sbar_sum"] = ssum.value
        return out
