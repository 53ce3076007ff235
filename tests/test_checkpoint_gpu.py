"""Checkpoint and exact resume (pic_checkpoint_*) on the CUDA path.

  * Round trip: a context loaded from an image holds the saving context's
    state bit for bit: its own image equals the loaded one byte for byte and
    pic_get_* return identical arrays (FP64 and FP32-mixed, 1D-3D).
  * Exact resume: with the deterministic deposit, a run checkpointed to a
    file after 2 steps and resumed in a fresh context repeats the
    uninterrupted run's steps 3-5 bit for bit (reports and state), through
    particle sorts after every step.  With the atomic deposit the resumed
    steps agree with the uninterrupted run to the rounding of the deposit's
    summation order (bounded at 1e-11 relative, the tolerance the steps
    converge to being 1e-12).
  * A foreign image (other mesh, other precision) is refused with PIC_EARG
    and leaves the context as it was.
"""
import numpy as np
import pytest

import paper_2609_36383_b300 as pic
import pic_inputs
from tests._common import make_gpu, small_1d, small_2d

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2609_36383_b300 import build
    build.build()


def _thermal_3d():
    return pic_inputs.thermal_box(dim=3, n=8, ppc=2, T=0.05, u_drift=0.3, dt=0.2, seed=4)


CASES = {"1d_two_stream": small_1d, "2d_weibel": small_2d, "3d_thermal": _thermal_3d}
TOL = 1e-12


def _state(s):
    x, P, w, sp = s.particles()
    return dict(x=x, P=P, w=w, sp=sp, **s.fields())


def _same(a, b):
    for k in a:
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("precision", [pic.PIC_FP64, pic.PIC_MIXED])
@pytest.mark.parametrize("name", sorted(CASES))
def test_loaded_context_holds_the_saved_state_bit_for_bit(name, precision):
    cfg = CASES[name]()
    s = make_gpu(cfg, precision=precision, sort_every=1)
    s.start()
    for _ in range(2):
        assert s.step(TOL)["status"] == 0
    img = s.checkpoint()
    h = pic.inspect_checkpoint(img)
    assert h["np"] == cfg["w"].shape[0] and h["steps_done"] == 2
    t = make_gpu(cfg, precision=precision, sort_every=0)
    t.restore(img)
    assert t.checkpoint() == img  # the whole device state, byte for byte
    _same(_state(s), _state(t))
    assert pic.inspect_checkpoint(t.checkpoint())["sort_every"] == 1


@pytest.mark.parametrize("name", sorted(CASES))
def test_resume_from_a_file_repeats_the_run_bit_for_bit(name, tmp_path):
    cfg = CASES[name]()
    ref = make_gpu(cfg, deterministic_deposit=1, sort_every=1)
    ref.start()
    rep_ref = [ref.step(TOL) for _ in range(5)]
    assert all(r["status"] == 0 for r in rep_ref)

    a = make_gpu(cfg, deterministic_deposit=1, sort_every=1)
    a.start()
    for _ in range(2):
        assert a.step(TOL)["status"] == 0
    path = tmp_path / f"{name}.ckpt"
    a.save_checkpoint(path)
    a.close()
    b = make_gpu(cfg, deterministic_deposit=1, sort_every=1)
    b.load_checkpoint(path)
    rep_b = [b.step(TOL) for _ in range(3)]
    for r0, r1 in zip(rep_ref[2:], rep_b):
        assert r0 == r1
    _same(_state(ref), _state(b))
    assert ref.checkpoint() == b.checkpoint()


@pytest.mark.parametrize("precision", [pic.PIC_FP64, pic.PIC_MIXED])
def test_resume_with_the_atomic_deposit_agrees_to_rounding(precision):
    cfg = small_2d()
    tol = TOL if precision == pic.PIC_FP64 else 1e-6
    ref = make_gpu(cfg, precision=precision)
    ref.start()
    for _ in range(2):
        assert ref.step(tol)["status"] == 0
    img = ref.checkpoint()
    rep_ref = [ref.step(tol) for _ in range(2)]
    b = make_gpu(cfg, precision=precision)
    b.restore(img)
    rep_b = [b.step(tol) for _ in range(2)]
    bound = 1e-11 if precision == pic.PIC_FP64 else 1e-4
    for r0, r1 in zip(rep_ref, rep_b):
        assert r1["status"] == 0
        for k in ("W", "K", "E_tot"):
            assert abs(r0[k] - r1[k]) <= bound * abs(r0[k]), k
    x0, P0, _, _ = ref.particles()
    x1, P1, _, _ = b.particles()
    assert np.abs(P1 - P0).max() <= bound * np.abs(P0).max()


def test_a_foreign_image_is_refused_and_changes_nothing():
    cfg = small_2d()
    s = make_gpu(cfg)
    s.start()
    assert s.step(TOL)["status"] == 0
    before = s.checkpoint()
    other_mesh = make_gpu(small_2d(n=32))
    other_mesh.start()
    other_prec = make_gpu(cfg, precision=pic.PIC_MIXED)
    other_prec.start()
    for img in (other_mesh.checkpoint(), other_prec.checkpoint()):
        with pytest.raises(pic.PicError) as ei:
            s.restore(img)
        assert ei.value.code == pic.PIC_EARG
        assert s.checkpoint() == before
    damaged = bytearray(before)
    damaged[-1] ^= 0xFF
    with pytest.raises(pic.PicError) as ei:
        s.restore(bytes(damaged))
    assert "checksum" in str(ei.value)
    assert s.checkpoint() == before
    assert s.step(TOL)["status"] == 0  # and the context keeps working


def test_load_drops_a_forward_sensitivity():
    cfg = small_2d()
    s = make_gpu(cfg)
    s.start()
    img = s.checkpoint()
    s.tangent_begin(du=np.zeros((3, cfg["u"].shape[1])))
    s.restore(img)
    with pytest.raises(RuntimeError):
        s.tangent()
    assert s.step(TOL)["status"] == 0


def test_report_log_records_the_steps_of_a_run(tmp_path):
    from paper_2609_36383_b300.reportlog import ReportLog, read_reports
    cfg = small_1d()
    s = make_gpu(cfg)
    s.start()
    with ReportLog(tmp_path / "run.jsonl", mode="w", workload="two_stream_1d") as log:
        reps = [log.write(s.step(TOL)) for _ in range(3)]
    recs = read_reports(tmp_path / "run.jsonl")
    assert [r["step"] for r in recs] == [0, 1, 2]
    for r, rep in zip(recs, reps):
        assert r == rep and r["status"] == 0 and r["workload"] == "two_stream_1d"
        assert abs(r["rel_dE"]) < 1e-11
