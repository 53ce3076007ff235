"""B300 (sm_103a) implementation of the GM-HC-CN implicit PIC step (arxiv 2609.36383).

Thin ctypes binding over the C ABI declared in ``include/pic.h`` and built into
``libpic.so`` by ``build.py``.  This module only marshals arguments: every step
of the method runs in the library's CUDA kernels.  Host arrays are numpy
arrays (``on_device = 0``); device arrays are torch CUDA tensors
(``on_device = 1``), whose ``data_ptr`` is handed to the library.  Importing
the module does not need a GPU; creating a :class:`Simulation` does, and it
fails loudly when the library or the GPU is missing (there is no CPU path).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpic.so")

PIC_OK, PIC_EARG, PIC_ENOMEM, PIC_ECUDA, PIC_EINNER, PIC_EOUTER, PIC_ESTATE = 0, -1, -2, -3, -4, -5, -6
PIC_ETOOBIG = -7
NOALLOC_MAX_PARTICLES = 16384 * 256
PIC_FP64, PIC_MIXED = 0, 1
PIC_SOLVER_ANDERSON, PIC_SOLVER_NEWTON_KRYLOV = 0, 1

# every symbol include/pic.h declares (checked by the CPU test suite)
EXPORTS = ("pic_default_options", "pic_init", "pic_set_particles", "pic_set_particles_local",
           "pic_set_potentials",
           "pic_start", "pic_step", "pic_eval_map", "pic_eval_map_jvp", "pic_eval_map_vjp", "pic_step_vjp", "pic_tune_sort",
           "pic_tangent_begin", "pic_tangent_end", "pic_get_tangent", "pic_num_particles", "pic_get_particles",
           "pic_get_velocities", "pic_get_potentials", "pic_set_state", "pic_checkpoint_bytes",
           "pic_checkpoint_save", "pic_checkpoint_inspect", "pic_checkpoint_load",
           "pic_get_stats", "pic_reset_stats",
           "pic_fma_throughput", "pic_kinetic_energy_noalloc", "pic_knot_jumps", "pic_last_error", "pic_free",
           "pic_batch_init", "pic_batch_set_instance", "pic_batch_start", "pic_batch_step",
           "pic_batch_num_particles", "pic_batch_get_particles", "pic_batch_get_potentials",
           "pic_batch_get_stats", "pic_batch_reset_stats", "pic_batch_last_error", "pic_batch_free")


class Grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("L", C.c_double * 3), ("x0", C.c_double * 3)]


class Species(C.Structure):
    _fields_ = [("q", C.c_double), ("m", C.c_double)]


class Options(C.Structure):
    _fields_ = [
        ("kappa", C.c_double), ("sigma1", C.c_double), ("sigma2", C.c_double), ("rho_bg", C.c_double),
        ("project_nyquist", C.c_int), ("gl_points", C.c_int), ("inner_max", C.c_int),
        ("outer_max", C.c_int), ("anderson_m", C.c_int), ("anderson_start", C.c_int),
        ("backtrack_levels", C.c_int), ("beta", C.c_double), ("lambda_", C.c_double),
        ("decrease_coef", C.c_double), ("growth_limit", C.c_double), ("tol_abs_ratio", C.c_double),
        ("inner_tol_scale", C.c_double), ("precision", C.c_int), ("mixed_tol_floor", C.c_double),
        ("sort_every", C.c_int), ("cuda_stream", C.c_void_p), ("inner_warm_start", C.c_int),
        ("order", C.c_int), ("refine_max", C.c_int), ("deterministic_deposit", C.c_int),
        ("growth_scaled", C.c_int), ("host_control", C.c_int), ("nonlinear_solver", C.c_int),
        ("fp32_first", C.c_int),
    ]


class CheckpointHeader(C.Structure):
    """pic_checkpoint_header: the 256-byte head of a checkpoint image."""
    _fields_ = [
        ("magic", C.c_char * 8), ("version", C.c_uint32), ("header_bytes", C.c_uint32),
        ("total_bytes", C.c_uint64), ("checksum", C.c_uint64), ("dim", C.c_int32),
        ("n", C.c_int32 * 3), ("precision", C.c_int32), ("nspecies", C.c_int32),
        ("sort_every", C.c_int32), ("reserved0", C.c_int32), ("L", C.c_double * 3),
        ("x0", C.c_double * 3), ("q", C.c_double * 4), ("m", C.c_double * 4), ("dt", C.c_double),
        ("E0", C.c_double), ("np", C.c_int64), ("steps_done", C.c_int64),
        ("reserved", C.c_uint8 * 48),
    ]

    def as_dict(self) -> dict:
        d = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            if k.startswith("reserved"):
                continue
            d[k] = list(v) if hasattr(v, "__len__") and not isinstance(v, bytes) else v
        return d


assert C.sizeof(CheckpointHeader) == 256


class Stats(C.Structure):
    _fields_ = [("launches", C.c_int64), ("map_launches", C.c_int64), ("map_ms", C.c_double),
                ("pushes", C.c_int64), ("inner_iters", C.c_int64), ("pieces", C.c_int64),
                ("refined", C.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class Report(C.Structure):
    _fields_ = [
        ("W", C.c_double), ("K", C.c_double), ("E_tot", C.c_double), ("rel_dE", C.c_double),
        ("gauss_rms", C.c_double), ("lorenz_rms", C.c_double), ("work_residual", C.c_double),
        ("chain_rms", C.c_double), ("res_scaled_rms", C.c_double), ("res_scaled_max", C.c_double),
        ("outer_iters", C.c_int), ("map_evals", C.c_int), ("inner_max", C.c_int),
        ("inner_mean", C.c_double), ("status", C.c_int), ("refined", C.c_int),
        ("jvp_evals", C.c_int), ("fp32_evals", C.c_int),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_VP = C.c_void_p


def lib():
    """Load libpic.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2609_36383_b300/build.py")
        L = C.CDLL(LIB_PATH)
        L.pic_default_options.argtypes = [C.POINTER(Options)]
        L.pic_init.argtypes = [C.POINTER(_VP), C.POINTER(Grid), C.POINTER(Species), C.c_int,
                               C.c_double, C.POINTER(Options)]
        L.pic_set_particles.argtypes = [_VP, C.c_int64, _VP, _VP, _VP, C.c_int, _VP, C.c_int]
        L.pic_set_particles_local.argtypes = [_VP, C.c_int64, _VP, _VP, _VP, _VP, C.c_int, _VP,
                                              C.c_int]
        L.pic_set_potentials.argtypes = [_VP, _VP, _VP, C.c_int]
        L.pic_start.argtypes = [_VP, C.POINTER(Report)]
        L.pic_step.argtypes = [_VP, C.c_double, C.POINTER(Report)]
        L.pic_eval_map.argtypes = [_VP, _VP, C.c_double, _VP, _VP, _VP, _VP, C.c_int]
        L.pic_eval_map_jvp.argtypes = [_VP, _VP, _VP, C.c_double, _VP, _VP, C.c_int]
        L.pic_eval_map_vjp.argtypes = [_VP, _VP, _VP, C.c_double, _VP, _VP, C.c_int]
        L.pic_step_vjp.argtypes = [_VP, C.c_double, _VP, _VP, _VP, _VP, _VP, _VP,
                                   C.POINTER(C.c_int), C.c_int]
        L.pic_tune_sort.argtypes = [_VP, C.c_double, C.c_int, _VP, C.c_int, C.POINTER(C.c_int),
                                    _VP]
        L.pic_tangent_begin.argtypes = [_VP, _VP, _VP, _VP, C.c_int]
        L.pic_tangent_end.argtypes = [_VP]
        L.pic_get_tangent.argtypes = [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, C.c_int]
        L.pic_num_particles.restype = C.c_int64
        L.pic_num_particles.argtypes = [_VP]
        L.pic_get_particles.argtypes = [_VP, _VP, _VP, _VP, _VP, C.c_int]
        L.pic_get_potentials.argtypes = [_VP, _VP, _VP, _VP, _VP, _VP, _VP, C.c_int]
        L.pic_get_velocities.argtypes = [_VP, _VP, C.c_int]
        L.pic_set_state.argtypes = [_VP, C.c_int64, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP,
                                    _VP, C.c_double, C.c_int]
        L.pic_checkpoint_bytes.argtypes = [_VP, C.POINTER(C.c_uint64)]
        L.pic_checkpoint_save.argtypes = [_VP, _VP, C.c_uint64]
        L.pic_checkpoint_inspect.argtypes = [_VP, C.c_uint64, C.POINTER(CheckpointHeader),
                                             C.c_char_p, C.c_int]
        L.pic_checkpoint_load.argtypes = [_VP, _VP, C.c_uint64]
        L.pic_knot_jumps.argtypes = [_VP, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.pic_get_stats.argtypes = [_VP, C.POINTER(Stats)]
        L.pic_reset_stats.argtypes = [_VP]
        L.pic_fma_throughput.argtypes = [C.c_int, C.POINTER(C.c_double)]
        L.pic_kinetic_energy_noalloc.argtypes = [C.POINTER(Grid), C.POINTER(Species), C.c_int,
                                                 C.c_double, C.c_int64, _VP, _VP, _VP, _VP, _VP,
                                                 C.POINTER(C.c_double), _VP]
        L.pic_last_error.restype = C.c_char_p
        L.pic_last_error.argtypes = [_VP]
        L.pic_free.argtypes = [_VP]
        L.pic_batch_init.argtypes = [C.POINTER(_VP), C.c_int, _VP, _VP, _VP, _VP,
                                     C.POINTER(Species), C.c_int, C.c_double, C.POINTER(Options)]
        L.pic_batch_set_instance.argtypes = [_VP, C.c_int, _VP, _VP, _VP, _VP, _VP, _VP]
        L.pic_batch_start.argtypes = [_VP, _VP]
        L.pic_batch_step.argtypes = [_VP, C.c_double, _VP]
        L.pic_batch_num_particles.restype = C.c_int64
        L.pic_batch_num_particles.argtypes = [_VP, C.c_int]
        L.pic_batch_get_particles.argtypes = [_VP, C.c_int, _VP, _VP, _VP, _VP]
        L.pic_batch_get_potentials.argtypes = [_VP, C.c_int, _VP, _VP, _VP, _VP, _VP, _VP]
        L.pic_batch_get_stats.argtypes = [_VP, C.POINTER(Stats)]
        L.pic_batch_reset_stats.argtypes = [_VP]
        L.pic_batch_last_error.restype = C.c_char_p
        L.pic_batch_last_error.argtypes = [_VP]
        L.pic_batch_free.argtypes = [_VP]
        _lib = L
    return _lib


def default_options() -> Options:
    o = Options()
    lib().pic_default_options(C.byref(o))
    return o


def inspect_checkpoint(image) -> dict:
    """Validate a checkpoint image (bytes, or a path to a file holding one) on
    the host and return its header; raises PicError(PIC_EARG) with the reason
    when the image is damaged or not an image.  Needs no GPU."""
    if isinstance(image, (str, os.PathLike)):
        with open(image, "rb") as f:
            image = f.read()
    buf = np.frombuffer(image, np.uint8)
    h = CheckpointHeader()
    why = C.create_string_buffer(256)
    rc = lib().pic_checkpoint_inspect(C.c_void_p(buf.ctypes.data), buf.size, C.byref(h), why, 256)
    if rc:
        raise PicError(rc, why.value.decode())
    return h.as_dict()


class PicError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"pic error {code}: {msg}")
        self.code = code


def _ptr(a, on_device):
    """Raw pointer of a numpy array (host) or torch tensor (device); None -> NULL."""
    if a is None:
        return None
    if on_device:
        return C.c_void_p(a.data_ptr())
    assert a.flags["C_CONTIGUOUS"]
    return C.c_void_p(a.ctypes.data)


class Simulation:
    """One simulation context of the C ABI (one GPU, one stream)."""

    def __init__(self, dim, n, L, x0, species, dt, precision=PIC_FP64, stream=None, **opts):
        g = Grid()
        g.dim = dim
        n3 = list(n) + [1] * (3 - len(n))
        L3 = list(L) + [1.0] * (3 - len(L))
        x3 = list(x0) + [0.0] * (3 - len(x0))
        for a in range(3):
            g.n[a] = int(n3[a]); g.L[a] = float(L3[a]); g.x0[a] = float(x3[a])
        sp = (Species * len(species))(*[Species(float(q), float(m)) for q, m in species])
        o = default_options()
        o.precision = precision
        for k, v in opts.items():
            setattr(o, "lambda_" if k == "lambda" else k, v)
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream().cuda_stream
            except Exception:
                stream = None
        o.cuda_stream = stream or None
        h = C.c_void_p()
        rc = lib().pic_init(C.byref(h), C.byref(g), sp, len(species), float(dt), C.byref(o))
        if rc:
            raise PicError(rc, "pic_init rejected the arguments or could not allocate")
        self._h = h
        self.dim = dim
        self.n = [int(v) for v in n3[:dim]]
        self.Ng = int(np.prod(self.n))

    def close(self):
        if getattr(self, "_h", None):
            lib().pic_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, allow=()):
        if rc and rc not in allow:
            raise PicError(rc, lib().pic_last_error(self._h).decode())
        return rc

    # -- set-up -------------------------------------------------------------
    def set_particles(self, x, u_or_P, w, species=None, canonical=False, on_device=False):
        if not on_device:
            x = np.ascontiguousarray(x, np.float64); u_or_P = np.ascontiguousarray(u_or_P, np.float64)
            w = np.ascontiguousarray(w, np.float64)
            species = None if species is None else np.ascontiguousarray(species, np.int32)
        n = int(w.shape[0])
        self._check(lib().pic_set_particles(self._h, n, _ptr(species, on_device), _ptr(x, on_device),
                                            _ptr(u_or_P, on_device), int(canonical),
                                            _ptr(w, on_device), int(on_device)))

    def set_particles_local(self, cell, offset, u_or_P, w, species=None, canonical=False,
                            on_device=False):
        """Particles in the stored form: node index per dimension (dim x N int32)
        and offset from it in node units in [-1/2, 1/2) (dim x N)."""
        if not on_device:
            cell = np.ascontiguousarray(cell, np.int32)
            offset = np.ascontiguousarray(offset, np.float64)
            u_or_P = np.ascontiguousarray(u_or_P, np.float64)
            w = np.ascontiguousarray(w, np.float64)
            species = None if species is None else np.ascontiguousarray(species, np.int32)
        n = int(w.shape[0])
        self._check(lib().pic_set_particles_local(
            self._h, n, _ptr(species, on_device), _ptr(cell, on_device), _ptr(offset, on_device),
            _ptr(u_or_P, on_device), int(canonical), _ptr(w, on_device), int(on_device)))

    def set_potentials(self, A=None, U=None, on_device=False):
        if not on_device:
            A = None if A is None else np.ascontiguousarray(A, np.float64)
            U = None if U is None else np.ascontiguousarray(U, np.float64)
        self._check(lib().pic_set_potentials(self._h, _ptr(A, on_device), _ptr(U, on_device),
                                             int(on_device)))

    def start(self) -> dict:
        r = Report()
        self._check(lib().pic_start(self._h, C.byref(r)))
        return r.as_dict()

    def step(self, tol, raise_on_fail=False) -> dict:
        r = Report()
        rc = lib().pic_step(self._h, float(tol), C.byref(r))
        if raise_on_fail or rc not in (PIC_OK, PIC_EINNER, PIC_EOUTER):
            self._check(rc)
        d = r.as_dict()
        d["status"] = rc
        return d

    def eval_map(self, j, tol):
        """H(j), orbit velocities, candidate P^{n+1} and inner counts (host arrays)."""
        npart = self.num_particles()
        j = np.ascontiguousarray(j, np.float64)
        H = np.zeros(3 * self.Ng)
        vb = np.zeros(3 * npart); Pn = np.zeros(3 * npart); it = np.zeros(npart, np.int32)
        rc = lib().pic_eval_map(self._h, _ptr(j, 0), float(tol), _ptr(H, 0), _ptr(vb, 0),
                                _ptr(Pn, 0), _ptr(it, 0), 0)
        self._check(rc, allow=(PIC_EINNER,))
        return rc, H, vb.reshape(3, npart), Pn.reshape(3, npart), it

    def eval_map_jvp(self, j, dj, tol):
        """H(j) and the directional derivative H'(j) dj (host arrays)."""
        j = np.ascontiguousarray(j, np.float64)
        dj = np.ascontiguousarray(dj, np.float64)
        H = np.zeros(3 * self.Ng)
        dH = np.zeros(3 * self.Ng)
        rc = lib().pic_eval_map_jvp(self._h, _ptr(j, 0), _ptr(dj, 0), float(tol), _ptr(H, 0),
                                    _ptr(dH, 0), 0)
        self._check(rc, allow=(PIC_EINNER,))
        return rc, H, dH

    def eval_map_vjp(self, j, ybar, tol):
        """H(j) and the adjoint product H'(j)^T ybar (host arrays)."""
        j = np.ascontiguousarray(j, np.float64)
        ybar = np.ascontiguousarray(ybar, np.float64)
        H = np.zeros(3 * self.Ng)
        jbar = np.zeros(3 * self.Ng)
        rc = lib().pic_eval_map_vjp(self._h, _ptr(j, 0), _ptr(ybar, 0), float(tol), _ptr(H, 0),
                                    _ptr(jbar, 0), 0)
        self._check(rc, allow=(PIC_EINNER,))
        return rc, H, jbar

    # -- the same calls on device tensors (torch, float64, on this GPU) -------
    @staticmethod
    def _dev_in(t, n):
        import torch
        t = t.detach().to(torch.float64).contiguous().reshape(-1)
        assert t.is_cuda and t.numel() == n
        torch.cuda.current_stream().synchronize()  # torch's writes land before the library reads
        return t

    def eval_map_device(self, j, tol):
        """H(j) for a device tensor j (3 Ng), as a device tensor."""
        import torch
        j = self._dev_in(j, 3 * self.Ng)
        H = torch.empty_like(j)
        rc = lib().pic_eval_map(self._h, _ptr(j, 1), float(tol), _ptr(H, 1), None, None, None, 1)
        self._check(rc, allow=(PIC_EINNER,))
        return rc, H

    def eval_map_jvp_device(self, j, dj, tol):
        """H(j) and H'(j) dj for device tensors, as device tensors."""
        import torch
        j, dj = self._dev_in(j, 3 * self.Ng), self._dev_in(dj, 3 * self.Ng)
        H, dH = torch.empty_like(j), torch.empty_like(j)
        rc = lib().pic_eval_map_jvp(self._h, _ptr(j, 1), _ptr(dj, 1), float(tol), _ptr(H, 1),
                                    _ptr(dH, 1), 1)
        self._check(rc, allow=(PIC_EINNER,))
        return rc, H, dH

    def eval_map_vjp_device(self, j, ybar, tol):
        """H(j) and H'(j)^T ybar for device tensors, as device tensors."""
        import torch
        j, ybar = self._dev_in(j, 3 * self.Ng), self._dev_in(ybar, 3 * self.Ng)
        H, jbar = torch.empty_like(j), torch.empty_like(j)
        rc = lib().pic_eval_map_vjp(self._h, _ptr(j, 1), _ptr(ybar, 1), float(tol), _ptr(H, 1),
                                    _ptr(jbar, 1), 1)
        self._check(rc, allow=(PIC_EINNER,))
        return rc, H, jbar

    def particles_device(self):
        """x (dim, N), P (3, N), w (N), species (N) as device tensors, load order."""
        import torch
        n = self.num_particles()
        dev = dict(dtype=torch.float64, device="cuda")
        x = torch.empty(self.dim * max(n, 1), **dev)
        P = torch.empty(3 * max(n, 1), **dev)
        w = torch.empty(max(n, 1), **dev)
        sp = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
        self._check(lib().pic_get_particles(self._h, _ptr(x, 1), _ptr(P, 1), _ptr(w, 1),
                                            _ptr(sp, 1), 1))
        return x[:self.dim * n].reshape(self.dim, n), P[:3 * n].reshape(3, n), w[:n], sp[:n]

    def fields_device(self) -> dict:
        """The potentials, rho and the accepted current as device tensors."""
        import torch
        N = self.Ng
        dev = dict(dtype=torch.float64, device="cuda")
        out = dict(phi=torch.empty(N, **dev), psi=torch.empty(N, **dev),
                   A=torch.empty(3 * N, **dev), U=torch.empty(3 * N, **dev),
                   rho=torch.empty(N, **dev), J=torch.empty(3 * N, **dev))
        self._check(lib().pic_get_potentials(self._h, *[_ptr(out[k], 1) for k in
                                                        ("phi", "psi", "A", "U", "rho", "J")], 1))
        return out

    def step_vjp_device(self, tol, xbar, Pbar, fbar):
        """pic_step_vjp on device tensors: xbar (dim x N), Pbar (3 x N) in load
        order and fbar (9 Ng, [phi, psi, A, U, rho]); returns the cotangents
        before the step as device tensors of the same shapes."""
        import torch
        n = self.num_particles()
        x1 = self._dev_in(xbar, self.dim * n)
        P1 = self._dev_in(Pbar, 3 * n)
        f1 = self._dev_in(fbar, 9 * self.Ng)
        x0, P0, f0 = torch.empty_like(x1), torch.empty_like(P1), torch.empty_like(f1)
        its = C.c_int(0)
        self._check(lib().pic_step_vjp(self._h, float(tol), _ptr(x1, 1), _ptr(P1, 1), _ptr(f1, 1),
                                       _ptr(x0, 1), _ptr(P0, 1), _ptr(f0, 1), C.byref(its), 1))
        return x0.reshape(self.dim, n), P0.reshape(3, n), f0

    def tune_sort(self, tol, steps, candidates=(0, 1, 2, 5, 10, 20)):
        """Measure each candidate sort interval over `steps` steps from the
        current state, restore the state and keep the fastest; returns
        (best interval, ms per step of every candidate)."""
        cand = np.ascontiguousarray(candidates, np.int32)
        ms = np.zeros(cand.shape[0])
        best = C.c_int(-1)
        self._check(lib().pic_tune_sort(self._h, float(tol), int(steps), _ptr(cand, 0),
                                        int(cand.shape[0]), C.byref(best), _ptr(ms, 0)))
        return best.value, ms

    def tangent_begin(self, du=None, dA=None, dU=None):
        """Seed the forward sensitivity at the started state: du (3, N) in load
        order, dA and dU (3 * Ng); None = zero.  Every later step advances it."""
        arrs = [None if a is None else np.ascontiguousarray(a, np.float64).ravel()
                for a in (du, dA, dU)]
        self._check(lib().pic_tangent_begin(self._h, *[_ptr(a, 0) for a in arrs], 0))

    def tangent_end(self):
        self._check(lib().pic_tangent_end(self._h))

    def tangent(self) -> dict:
        """The tangent of the accepted state: dx (dim, N), dP (3, N) in load
        order, dA, dU (3 * Ng), dK, dW and the last step's GMRES iterations."""
        n = self.num_particles()
        dx = np.zeros(self.dim * n); dP = np.zeros(3 * n)
        dA = np.zeros(3 * self.Ng); dU = np.zeros(3 * self.Ng)
        dK = C.c_double(); dW = C.c_double(); it = C.c_int()
        self._check(lib().pic_get_tangent(self._h, _ptr(dx, 0), _ptr(dP, 0), _ptr(dA, 0),
                                          _ptr(dU, 0), C.byref(dK), C.byref(dW), C.byref(it),
                                          0))
        return dict(dx=dx.reshape(self.dim, n), dP=dP.reshape(3, n), dA=dA, dU=dU,
                    dK=dK.value, dW=dW.value, gmres_iters=it.value)

    # -- state access ---------------------------------------------------------
    def num_particles(self) -> int:
        return int(lib().pic_num_particles(self._h))

    def particles(self):
        npart = self.num_particles()
        x = np.zeros(self.dim * npart); P = np.zeros(3 * npart); w = np.zeros(npart)
        sp = np.zeros(npart, np.int32)
        self._check(lib().pic_get_particles(self._h, _ptr(x, 0), _ptr(P, 0), _ptr(w, 0),
                                            _ptr(sp, 0), 0))
        return x.reshape(self.dim, npart), P.reshape(3, npart), w, sp

    def velocities(self):
        """Proper velocities u = p / m of the particles, shape (3, N), load order."""
        u = np.zeros(3 * self.num_particles())
        self._check(lib().pic_get_velocities(self._h, _ptr(u, 0), 0))
        return u.reshape(3, -1)

    def fields(self) -> dict:
        N = self.Ng
        out = dict(phi=np.zeros(N), psi=np.zeros(N), A=np.zeros(3 * N), U=np.zeros(3 * N),
                   rho=np.zeros(N), J=np.zeros(3 * N))
        self._check(lib().pic_get_potentials(self._h, *[_ptr(out[k], 0) for k in
                                                        ("phi", "psi", "A", "U", "rho", "J")], 0))
        return out

    def set_state(self, x, P, w, species, fields, E0, on_device=False):
        if not on_device:
            x = np.ascontiguousarray(x, np.float64); P = np.ascontiguousarray(P, np.float64)
            w = np.ascontiguousarray(w, np.float64)
            species = None if species is None else np.ascontiguousarray(species, np.int32)
            fields = {k: np.ascontiguousarray(v, np.float64) for k, v in fields.items()}
        n = int(w.shape[0])
        self._check(lib().pic_set_state(self._h, n, _ptr(species, on_device), _ptr(x, on_device),
                                        _ptr(P, on_device), _ptr(w, on_device),
                                        *[_ptr(fields[k], on_device) for k in
                                          ("phi", "psi", "A", "U", "rho", "J")],
                                        float(E0), int(on_device)))

    # -- adjoint of a step (pic_step_vjp) --------------------------------------
    FIELD_ORDER = ("phi", "psi", "A", "U", "rho")

    def _pack_fields(self, f):
        """{phi, psi, A, U, rho} (missing = zero) -> the 9 Ng array of pic_step_vjp."""
        N = self.Ng
        out = np.zeros(9 * N)
        off = 0
        for k, nc in zip(self.FIELD_ORDER, (1, 1, 3, 3, 1)):
            if f is not None and f.get(k) is not None:
                out[off:off + nc * N] = np.asarray(f[k], np.float64).reshape(-1)
            off += nc * N
        return out

    def _unpack_fields(self, a):
        N = self.Ng
        out, off = {}, 0
        for k, nc in zip(self.FIELD_ORDER, (1, 1, 3, 3, 1)):
            out[k] = a[off:off + nc * N].copy()
            off += nc * N
        return out

    def step_vjp(self, tol, xbar=None, Pbar=None, fbar=None) -> dict:
        """Cotangents of the state before a step from those after it.

        xbar (dim x N), Pbar (3 x N) in load order and fbar (a dict of
        phi, psi, A, U, rho in real space, as :meth:`fields` returns them)
        are the cotangents of the state after one step at ``tol``; missing
        ones are zero.  Returns the cotangents of the current state in the
        same form (keys ``x``, ``P``, ``fields``) and ``gmres_iters``.  The
        state is left unchanged."""
        n = self.num_particles()
        x1 = None if xbar is None else np.ascontiguousarray(xbar, np.float64).reshape(self.dim, n)
        P1 = None if Pbar is None else np.ascontiguousarray(Pbar, np.float64).reshape(3, n)
        f1 = self._pack_fields(fbar) if fbar is not None else None
        x0 = np.zeros((self.dim, n))
        P0 = np.zeros((3, n))
        f0 = np.zeros(9 * self.Ng)
        its = C.c_int(0)
        self._check(lib().pic_step_vjp(self._h, float(tol), _ptr(x1, 0), _ptr(P1, 0), _ptr(f1, 0),
                                       _ptr(x0, 0), _ptr(P0, 0), _ptr(f0, 0), C.byref(its), 0))
        return {"x": x0, "P": P0, "fields": self._unpack_fields(f0), "gmres_iters": its.value}

    def run_adjoint(self, tol, steps, xbar=None, Pbar=None, fbar=None):
        """Reverse-mode gradient through ``steps`` steps from the current state.

        Runs the steps forward, keeping each step's checkpoint image on the
        host, then chains :meth:`step_vjp` from the last step back to the
        first.  The cotangents given are those of the final state; the
        result holds the cotangents of the current (initial) state and the
        forward reports.  The context ends in the final state."""
        images, reports = [], []
        for _ in range(steps):
            images.append(self.checkpoint())
            r = self.step(tol)
            if r["status"] != 0:
                raise PicError(r["status"], "forward step failed")
            reports.append(r)
        final = self.checkpoint()
        g = {"x": xbar, "P": Pbar, "fields": fbar}
        its = []
        for img in reversed(images):
            self.restore(img)
            g = self.step_vjp(tol, g["x"], g["P"], g["fields"])
            its.append(g["gmres_iters"])
        self.restore(final)
        g["gmres_iters"] = its[::-1]
        g["reports"] = reports
        return g

    # -- checkpoint / exact resume (pic_checkpoint_*) -------------------------
    def checkpoint(self) -> bytes:
        """The accepted state as a checkpoint image (header + raw sections)."""
        nb = C.c_uint64()
        self._check(lib().pic_checkpoint_bytes(self._h, C.byref(nb)))
        buf = np.empty(nb.value, np.uint8)
        self._check(lib().pic_checkpoint_save(self._h, C.c_void_p(buf.ctypes.data), nb.value))
        return buf.tobytes()

    def restore(self, image: bytes):
        """Replace the state with a checkpoint image from a context of the
        same mesh, precision and species."""
        buf = np.frombuffer(image, np.uint8)
        self._check(lib().pic_checkpoint_load(self._h, C.c_void_p(buf.ctypes.data), buf.size))

    def save_checkpoint(self, path):
        """Write the checkpoint image to a file (through a temporary name, so
        an interrupted write never leaves a partial image under `path`)."""
        data = self.checkpoint()
        tmp = f"{os.fspath(path)}.tmp{os.getpid()}"
        with open(tmp, "wb") as f:
            f.write(data)
        os.replace(tmp, path)

    def checkpoint_header(self) -> dict:
        """The header of the current state's checkpoint image (E0, step count, ...)."""
        return inspect_checkpoint(self.checkpoint())

    def load_checkpoint(self, path):
        with open(path, "rb") as f:
            self.restore(f.read())

    def knot_jumps(self, eps=1e-8):
        """(E_shape jump, grad A jump): the knot-jump regularity diagnostic of
        Sec. 5.3 on the accepted fields (pic_knot_jumps)."""
        Ej, Gj = C.c_double(0.0), C.c_double(0.0)
        self._check(lib().pic_knot_jumps(self._h, float(eps), C.byref(Ej), C.byref(Gj)))
        return Ej.value, Gj.value

    def stats(self) -> dict:
        st = Stats()
        self._check(lib().pic_get_stats(self._h, C.byref(st)))
        return st.as_dict()

    def reset_stats(self):
        self._check(lib().pic_reset_stats(self._h))

    # -- raw access for device-resident benchmarking ----------------------------
    @property
    def handle(self):
        return self._h


def _reports_view(arr):
    """The per-instance reports as a numpy structured array (no copy): field
    access by name, e.g. reps[b]["status"], as for the single-problem dicts."""
    return np.ctypeslib.as_array(arr)


class Batch:
    """An ensemble of independent 1D3V problems advanced together (pic_batch_*).

    ``n``, ``L``, ``x0`` and ``np_`` give every instance's mesh size, length,
    origin and particle count; the species, dt and options are shared."""

    def __init__(self, n, L, x0, np_, species, dt, precision=PIC_FP64, stream=None, **opts):
        self.B = len(n)
        self.n = np.ascontiguousarray(n, np.int32)
        self.L = np.ascontiguousarray(L, np.float64)
        self.x0 = np.ascontiguousarray(x0, np.float64)
        self.np_ = np.ascontiguousarray(np_, np.int64)
        sp = (Species * len(species))(*[Species(float(q), float(m)) for q, m in species])
        o = default_options()
        o.precision = precision
        for k, v in opts.items():
            setattr(o, "lambda_" if k == "lambda" else k, v)
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream().cuda_stream
            except Exception:
                stream = None
        o.cuda_stream = stream or None
        h = C.c_void_p()
        rc = lib().pic_batch_init(C.byref(h), self.B, _ptr(self.n, 0), _ptr(self.L, 0),
                                  _ptr(self.x0, 0), _ptr(self.np_, 0), sp, len(species),
                                  float(dt), C.byref(o))
        if rc:
            raise PicError(rc, "pic_batch_init rejected the arguments or could not allocate")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().pic_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, allow=()):
        if rc and rc not in allow:
            raise PicError(rc, lib().pic_batch_last_error(self._h).decode())
        return rc

    def set_instance(self, b, x, u, w, species=None, A=None, U=None):
        x = np.ascontiguousarray(x, np.float64).reshape(-1)
        u = np.ascontiguousarray(u, np.float64)
        w = np.ascontiguousarray(w, np.float64)
        species = None if species is None else np.ascontiguousarray(species, np.int32)
        A = None if A is None else np.ascontiguousarray(A, np.float64)
        U = None if U is None else np.ascontiguousarray(U, np.float64)
        self._check(lib().pic_batch_set_instance(self._h, int(b), _ptr(species, 0), _ptr(x, 0),
                                                 _ptr(u, 0), _ptr(w, 0), _ptr(A, 0), _ptr(U, 0)))

    def start(self):
        reps = (Report * self.B)()
        self._check(lib().pic_batch_start(self._h, reps))
        return _reports_view(reps)

    def step(self, tol):
        """One step of every instance; per-instance reports (status included)."""
        reps = (Report * self.B)()
        rc = lib().pic_batch_step(self._h, float(tol), reps)
        self._check(rc, allow=(PIC_EINNER, PIC_EOUTER))
        return _reports_view(reps)

    def particles(self, b):
        npart = int(self.np_[b])
        x = np.zeros(npart); P = np.zeros(3 * npart); w = np.zeros(npart)
        sp = np.zeros(npart, np.int32)
        self._check(lib().pic_batch_get_particles(self._h, int(b), _ptr(x, 0), _ptr(P, 0),
                                                  _ptr(w, 0), _ptr(sp, 0)))
        return x.reshape(1, npart), P.reshape(3, npart), w, sp

    def fields(self, b) -> dict:
        N = int(self.n[b])
        out = dict(phi=np.zeros(N), psi=np.zeros(N), A=np.zeros(3 * N), U=np.zeros(3 * N),
                   rho=np.zeros(N), J=np.zeros(3 * N))
        self._check(lib().pic_batch_get_potentials(self._h, int(b), *[_ptr(out[k], 0) for k in
                                                   ("phi", "psi", "A", "U", "rho", "J")]))
        return out

    def stats(self) -> dict:
        st = Stats()
        self._check(lib().pic_batch_get_stats(self._h, C.byref(st)))
        return st.as_dict()

    def reset_stats(self):
        self._check(lib().pic_batch_reset_stats(self._h))


def batch_from_configs(cfgs, precision=PIC_FP64, **opts) -> Batch:
    """Create and load a batch from a list of 1D ``pic_inputs`` recipes that
    share species, dt and rho_bg."""
    c0 = cfgs[0]
    bt = Batch([c["n"][0] for c in cfgs], [c["L"][0] for c in cfgs], [c["x0"][0] for c in cfgs],
               [c["w"].shape[0] for c in cfgs], c0["species"], c0["dt"], precision=precision,
               rho_bg=c0["rho_bg"], **opts)
    for b, c in enumerate(cfgs):
        bt.set_instance(b, c["x"], c["u"], c["w"], c["sp"], c["A"], c["U"])
    return bt


def fma_throughput(precision=PIC_FP64) -> float:
    """Measured FMA throughput of the current device, FLOP/s."""
    v = C.c_double()
    rc = lib().pic_fma_throughput(int(precision), C.byref(v))
    if rc:
        raise PicError(rc, "pic_fma_throughput failed")
    return v.value


def from_config(cfg, precision=PIC_FP64, **opts) -> Simulation:
    """Create, load and start a simulation from a ``pic_inputs`` recipe."""
    sim = Simulation(cfg["dim"], cfg["n"], cfg["L"], cfg["x0"], cfg["species"], cfg["dt"],
                     precision=precision, rho_bg=cfg["rho_bg"], **opts)
    sim.set_particles(cfg["x"], cfg["u"], cfg["w"], cfg["sp"])
    sim.set_potentials(cfg["A"], cfg["U"])
    return sim
