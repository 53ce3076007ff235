"""CPU checks of the C ABI: the library builds, loads, and exports every entry
point include/pic.h declares (no compute call: there is no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "pic.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pic_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpic():
    from paper_2609_36383_b300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for must in ("pic_init", "pic_step", "pic_start", "pic_set_particles", "pic_get_particles",
                 "pic_set_potentials", "pic_get_potentials", "pic_eval_map", "pic_set_state",
                 "pic_last_error", "pic_free"):
        assert must in names


def test_library_exports_every_declared_symbol(libpic):
    for name in declared_entry_points():
        assert hasattr(libpic, name), name


def test_binding_lists_every_symbol():
    import paper_2609_36383_b300 as P
    assert sorted(P.EXPORTS) == declared_entry_points()


def test_default_options_are_the_papers(libpic):
    import paper_2609_36383_b300 as P
    o = P.default_options()
    assert (o.inner_max, o.outer_max, o.anderson_m, o.anderson_start) == (64, 80, 4, 2)
    assert (o.beta, o.lambda_, o.decrease_coef, o.growth_limit) == (0.5, 1e-12, 1e-4, 1.2)
    assert o.backtrack_levels == 7 and o.project_nyquist == 1
    assert (o.kappa, o.sigma1, o.sigma2) == (1.0, 1.0, 1.0)
    assert o.order == 2 and o.refine_max == 0  # quadratic shapes, no refinement


def test_init_rejects_bad_grids_without_touching_the_gpu(libpic):
    import paper_2609_36383_b300 as P
    g = P.Grid()
    g.dim = 2
    g.n[0], g.n[1], g.n[2] = 100, 64, 1  # not a power of two
    g.L[0] = g.L[1] = g.L[2] = 1.0
    sp = (P.Species * 1)(P.Species(-1.0, 1.0))
    h = ctypes.c_void_p()
    assert P.lib().pic_init(ctypes.byref(h), ctypes.byref(g), sp, 1, 0.1, None) == P.PIC_EARG
    g.n[0] = 64
    assert P.lib().pic_init(ctypes.byref(h), ctypes.byref(g), sp, 1, -0.1, None) == P.PIC_EARG
    assert P.lib().pic_init(ctypes.byref(h), ctypes.byref(g), sp, 0, 0.1, None) == P.PIC_EARG


def test_batch_init_rejects_bad_sizes_without_touching_the_gpu(libpic):
    import paper_2609_36383_b300 as P
    h = ctypes.c_void_p()
    sp = (P.Species * 1)(P.Species(-1.0, 1.0))
    n = (ctypes.c_int * 2)(16, 24)  # 24 is not a power of two
    L = (ctypes.c_double * 2)(1.0, 1.0)
    npart = (ctypes.c_int64 * 2)(10, 10)
    assert P.lib().pic_batch_init(ctypes.byref(h), 2, n, L, None, npart, sp, 1, 0.1,
                                  None) == P.PIC_EARG
    n[1] = 2048  # above the largest instance mesh
    assert P.lib().pic_batch_init(ctypes.byref(h), 2, n, L, None, npart, sp, 1, 0.1,
                                  None) == P.PIC_EARG


def test_deterministic_deposit_rejected_where_unsupported_without_touching_the_gpu(libpic):
    """The deterministic deposit needs FP64, no refinement, at least 8 nodes
    per active dimension, and a single context; pic_init and pic_batch_init
    refuse it otherwise before any device call."""
    import paper_2609_36383_b300 as P
    sp = (P.Species * 1)(P.Species(-1.0, 1.0))
    g = P.Grid()
    g.dim = 2
    for a in range(3):
        g.n[a] = 16 if a < 2 else 1
        g.L[a] = 1.0
    h = ctypes.c_void_p()
    for field, value in (("precision", P.PIC_MIXED), ("refine_max", 1)):
        o = P.default_options()
        o.deterministic_deposit = 1
        setattr(o, field, value)
        assert P.lib().pic_init(ctypes.byref(h), ctypes.byref(g), sp, 1, 0.1,
                                ctypes.byref(o)) == P.PIC_EARG
    o = P.default_options()
    o.deterministic_deposit = 1
    g.n[1] = 4  # too small for the node gather's stencil
    assert P.lib().pic_init(ctypes.byref(h), ctypes.byref(g), sp, 1, 0.1,
                            ctypes.byref(o)) == P.PIC_EARG
    n = (ctypes.c_int * 2)(16, 32)
    L = (ctypes.c_double * 2)(1.0, 1.0)
    npart = (ctypes.c_int64 * 2)(10, 10)
    assert P.lib().pic_batch_init(ctypes.byref(h), 2, n, L, None, npart, sp, 1, 0.1,
                                  ctypes.byref(o)) == P.PIC_EARG


def test_new_entry_points_refuse_a_null_context_without_touching_the_gpu(libpic):
    """The checkpoint, step-adjoint and regularity calls check their context
    and arguments before any CUDA call: PIC_EARG (-1) for a null context or
    a null output."""
    import paper_2609_36383_b300 as P
    L = P.lib()
    nb = ctypes.c_uint64(0)
    assert L.pic_checkpoint_bytes(None, ctypes.byref(nb)) == P.PIC_EARG
    buf = ctypes.create_string_buffer(512)
    assert L.pic_checkpoint_save(None, buf, 512) == P.PIC_EARG
    assert L.pic_checkpoint_load(None, buf, 512) == P.PIC_EARG
    its = ctypes.c_int(0)
    assert L.pic_step_vjp(None, 1e-12, None, None, None, None, None, None,
                          ctypes.byref(its), 0) == P.PIC_EARG
    e, g = ctypes.c_double(0.0), ctypes.c_double(0.0)
    assert L.pic_knot_jumps(None, 1e-8, ctypes.byref(e), ctypes.byref(g)) == P.PIC_EARG
    # inspect needs no context at all: a zero-length image is refused with a reason
    why = ctypes.create_string_buffer(128)
    h = P.CheckpointHeader()
    assert L.pic_checkpoint_inspect(buf, 0, ctypes.byref(h), why, 128) == P.PIC_EARG
    assert b"shorter than its header" in why.value
