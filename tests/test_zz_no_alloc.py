"""GPU check of pic_kinetic_energy_noalloc, the entry point for callers that
cannot allocate device memory.

Some callers must not call cudaMalloc: a memory pool or arena may own the
whole device, an allocation inside a latency-critical loop would synchronize
the device, or a framework may forbid allocating on its hot path.  For them
the library offers a kinetic-energy reduction whose scratch lives in a fixed
array inside the library.  This test calls it through the C ABI, twice in a
row on the same data, and checks both results against the kinetic energy the
context reports from pic_start and pic_step (the existing entry points), at
the 1e-12 relative tolerance of the other FP64 parity tests.  The cases
span 1D, 2D and 3D, and one 2D set of 131,072 particles (512 blocks, so the
final pass strides over more partials than it has threads).  It also checks
that an input larger than the fixed scratch is rejected, and that a species
index out of range is refused without being used as an index.  The file is
named so that pytest collects it last.
"""
import ctypes as C

import pytest

import pic_inputs
from tests._common import make_gpu, small_1d, small_2d

pytestmark = pytest.mark.gpu


def _device_state(sim, torch):
    import paper_2609_36383_b300 as P
    n, Ng, d = sim.num_particles(), sim.Ng, sim.dim
    dev = dict(dtype=torch.float64, device="cuda")
    x = torch.empty(d * max(n, 1), **dev)
    Pm = torch.empty(3 * max(n, 1), **dev)
    w = torch.empty(max(n, 1), **dev)
    sp = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    A = torch.empty(3 * Ng, **dev)
    ptr = lambda t: C.c_void_p(t.data_ptr())
    assert P.lib().pic_get_particles(sim.handle, ptr(x), ptr(Pm), ptr(w), ptr(sp), 1) == 0
    assert P.lib().pic_get_potentials(sim.handle, None, None, ptr(A), None, None, None, 1) == 0
    return n, x, Pm, w, sp, A


def _noalloc_K(cfg, n, x, Pm, w, sp, A, torch, n_override=None):
    import paper_2609_36383_b300 as P
    g = P.Grid()
    g.dim = cfg["dim"]
    for a in range(3):
        g.n[a] = cfg["n"][a] if a < cfg["dim"] else 1
        g.L[a] = cfg["L"][a] if a < cfg["dim"] else 1.0
        g.x0[a] = cfg["x0"][a] if a < cfg["dim"] else 0.0
    sps = (P.Species * len(cfg["species"]))(*[P.Species(q, m) for q, m in cfg["species"]])
    K = C.c_double(float("nan"))
    ptr = lambda t: C.c_void_p(t.data_ptr())
    rc = P.lib().pic_kinetic_energy_noalloc(
        C.byref(g), sps, len(cfg["species"]), 1.0, n if n_override is None else n_override,
        ptr(sp), ptr(x), ptr(Pm), ptr(w), ptr(A), C.byref(K),
        C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, K.value


def _large_2d():  # 64 x 64 cells, 32 particles per cell: 131,072 particles
    return pic_inputs.weibel_2d(n=64, ppc_beam=16, u_drift=0.5, T=0.01, dt=0.05, tol=1e-12,
                                steps=2, seed=5, noise=1e-3, kmax=3)


def _small_3d():
    return pic_inputs.thermal_box(dim=3, n=8, ppc=2, T=0.05, u_drift=0.3, seed=2)


@pytest.mark.parametrize("make_cfg", [small_1d, small_2d, _large_2d, _small_3d],
                         ids=["1d", "2d", "2d_131k", "3d"])
def test_noalloc_kinetic_energy_matches_context(make_cfg):
    import torch
    import paper_2609_36383_b300 as P
    from paper_2609_36383_b300 import build
    build.build()
    cfg = make_cfg()
    sim = make_gpu(cfg)
    r0 = sim.start()
    state = _device_state(sim, torch)
    for _ in range(2):  # two calls in a row share the same scratch
        rc, K = _noalloc_K(cfg, *state, torch)
        assert rc == P.PIC_OK
        assert K == pytest.approx(r0["K"], rel=1e-12)
    r1 = sim.step(1e-12)
    assert r1["status"] == 0
    state = _device_state(sim, torch)
    rc, K = _noalloc_K(cfg, *state, torch)
    assert rc == P.PIC_OK and K == pytest.approx(r1["K"], rel=1e-12)
    rc, _ = _noalloc_K(cfg, *state, torch, n_override=P.NOALLOC_MAX_PARTICLES + 1)
    assert rc == P.PIC_ETOOBIG
    sim.close()


def test_noalloc_rejects_species_out_of_range():
    import torch
    import paper_2609_36383_b300 as P
    from paper_2609_36383_b300 import build
    build.build()
    cfg = small_2d()
    sim = make_gpu(cfg)
    r0 = sim.start()
    n, x, Pm, w, sp, A = _device_state(sim, torch)
    bad = sp.clone()
    bad[n // 2] = len(cfg["species"])  # one past the last species
    rc, _ = _noalloc_K(cfg, n, x, Pm, w, bad, A, torch)
    assert rc == P.PIC_EARG
    bad[n // 2] = -1
    rc, _ = _noalloc_K(cfg, n, x, Pm, w, bad, A, torch)
    assert rc == P.PIC_EARG
    # the error word is cleared by the next call: a valid input succeeds
    rc, K = _noalloc_K(cfg, n, x, Pm, w, sp, A, torch)
    assert rc == P.PIC_OK and K == pytest.approx(r0["K"], rel=1e-12)
    sim.close()
