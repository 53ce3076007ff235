"""Checkpoint images (pic_checkpoint_*) and the JSON Lines report log, on CPU.

pic_checkpoint_inspect validates an image on the host, so it is exercised
here without a GPU against images this test writes itself from the layout
that include/pic.h documents (256-byte header; cell, off, P, w, sp, id,
phi, psi, rho, A, U in spectral form, A and J in real space, each section
starting on a 16-byte boundary) and from the published definition of the
64-bit FNV-1a hash.  A valid image must pass and report its header; every
kind of damage (magic, version, size, checksum, an index out of range, a
repeated load-order index, an offset outside its cell) must be refused with
PIC_EARG and a reason.  The round trip through a real context is in
tests/test_checkpoint_gpu.py.
"""
import json
import struct

import numpy as np
import pytest

import paper_2609_36383_b300 as pic
from paper_2609_36383_b300.reportlog import ReportLog, read_reports

FNV_OFFSET = 14695981039346656037
FNV_PRIME = 1099511628211


def fnv1a64(data: bytes) -> int:
    h = FNV_OFFSET
    for byte in data:
        h ^= byte
        h = (h * FNV_PRIME) % (1 << 64)
    return h


def test_fnv1a64_of_the_published_test_strings():
    # reference values of the FNV-1a 64-bit hash for "" and "a"
    assert fnv1a64(b"") == 0xCBF29CE484222325
    assert fnv1a64(b"a") == 0xAF63DC4C8601EC8C


def _pad16(b: bytes) -> bytes:
    return b + bytes((-len(b)) % 16)


def make_image(dim=2, n=(8, 8, 1), np_=5, precision=pic.PIC_FP64, nspecies=2, seed=0,
               mutate=None):
    """A checkpoint image written from the documented layout; `mutate` may
    edit the section arrays before they are packed."""
    rng = np.random.default_rng(seed)
    Ng = int(np.prod(n))
    rt = np.float64 if precision == pic.PIC_FP64 else np.float32
    sec = {
        "cell": np.stack([rng.integers(0, n[l], np_) for l in range(dim)]).astype(np.int32),
        "off": rng.uniform(-0.5, 0.5, (dim, np_)).astype(rt),
        "P": rng.standard_normal((3, np_)).astype(rt),
        "w": rng.uniform(0.5, 1.5, np_),
        "sp": rng.integers(0, nspecies, np_).astype(np.int32),
        "id": rng.permutation(np_).astype(np.int64),
        "phi": rng.standard_normal(2 * Ng), "psi": rng.standard_normal(2 * Ng),
        "rho": rng.standard_normal(2 * Ng), "A": rng.standard_normal(6 * Ng),
        "U": rng.standard_normal(6 * Ng), "A_real": rng.standard_normal(3 * Ng),
        "J": rng.standard_normal(3 * Ng),
    }
    if mutate:
        mutate(sec)
    order = ("cell", "off", "P", "w", "sp", "id", "phi", "psi", "rho", "A", "U", "A_real", "J")
    payload = b"".join(_pad16(np.ascontiguousarray(sec[k]).tobytes()) for k in order)
    L = [1.0, 2.0, 3.0][:dim] + [1.0] * (3 - dim)
    head = b"PICCKPT1" + struct.pack("<IIQQ", 1, 256, 256 + len(payload), fnv1a64(payload))
    head += struct.pack("<4i", dim, *n)
    head += struct.pack("<4i", precision, nspecies, 10, 0)
    head += struct.pack("<3d", *L) + struct.pack("<3d", 0, 0, 0)
    head += struct.pack("<4d", *([-1.0] * nspecies + [0.0] * (4 - nspecies)))
    head += struct.pack("<4d", *([1.0] * nspecies + [0.0] * (4 - nspecies)))
    head += struct.pack("<dd", 0.05, 123.5) + struct.pack("<qq", np_, 7)
    head += bytes(256 - len(head))
    assert len(head) == 256
    return head + payload


@pytest.mark.parametrize("precision", [pic.PIC_FP64, pic.PIC_MIXED])
@pytest.mark.parametrize("dim,n", [(1, (16, 1, 1)), (2, (8, 8, 1)), (3, (4, 8, 4))])
def test_a_valid_image_passes_and_reports_its_header(precision, dim, n):
    img = make_image(dim=dim, n=n, precision=precision)
    h = pic.inspect_checkpoint(img)
    assert h["magic"] == b"PICCKPT1" and h["version"] == 1 and h["header_bytes"] == 256
    assert h["total_bytes"] == len(img) and h["dim"] == dim and h["n"] == list(n)
    assert h["precision"] == precision and h["np"] == 5 and h["steps_done"] == 7
    assert h["E0"] == 123.5 and h["dt"] == 0.05 and h["sort_every"] == 10


def test_an_empty_particle_set_is_a_valid_image():
    h = pic.inspect_checkpoint(make_image(np_=0))
    assert h["np"] == 0


def _refused(img, reason):
    with pytest.raises(pic.PicError) as ei:
        pic.inspect_checkpoint(img)
    assert ei.value.code == pic.PIC_EARG
    assert reason in str(ei.value), str(ei.value)


def test_damaged_images_are_refused_with_the_reason():
    good = make_image()
    _refused(good[:100], "shorter than its header")
    _refused(b"NOTACKPT" + good[8:], "magic")
    _refused(good[:8] + struct.pack("<I", 2) + good[12:], "format version")
    _refused(good[:-16], "truncated")
    _refused(good + bytes(16), "truncated")
    flipped = bytearray(good)
    flipped[300] ^= 1
    _refused(bytes(flipped), "checksum")
    # a header claiming more particles than the payload holds
    bad_np = bytearray(good)
    bad_np[192:200] = struct.pack("<q", 6)
    _refused(bytes(bad_np), "size does not match")
    # a mesh size that is not a power of two
    bad_n = bytearray(good)
    bad_n[36:40] = struct.pack("<i", 12)
    _refused(bytes(bad_n), "mesh size")


def test_indices_are_checked_before_anything_reaches_a_device():
    def cell_out(s):
        s["cell"][1, 3] = 8
    def cell_neg(s):
        s["cell"][0, 0] = -1
    def off_out(s):
        s["off"][0, 2] = 0.75
    def off_nan(s):
        s["off"][1, 1] = np.nan
    def sp_out(s):
        s["sp"][4] = 2
    def id_dup(s):
        s["id"][:] = [0, 1, 2, 3, 3]
    def id_out(s):
        s["id"][:] = [0, 1, 2, 3, 5]
    for mut, reason in [(cell_out, "cell outside"), (cell_neg, "cell outside"),
                        (off_out, "offset outside"), (off_nan, "offset outside"),
                        (sp_out, "species"), (id_dup, "permutation"), (id_out, "permutation")]:
        _refused(make_image(mutate=mut), reason)


def test_report_log_writes_strict_json_lines(tmp_path):
    p = tmp_path / "steps.jsonl"
    with ReportLog(p, mode="w", run="weibel_2d", n=[128, 128]) as log:
        log.write({"E_tot": 1.5, "rel_dE": np.float64(2e-16), "outer_iters": np.int32(5),
                   "status": 0})
        log.write({"E_tot": float("nan"), "rel_dE": float("inf"), "status": -4}, wall_s=0.25)
    recs = read_reports(p)
    assert [r["step"] for r in recs] == [0, 1]
    assert recs[0] == {"run": "weibel_2d", "n": [128, 128], "step": 0, "E_tot": 1.5,
                       "rel_dE": 2e-16, "outer_iters": 5, "status": 0}
    assert recs[1]["E_tot"] is None and recs[1]["rel_dE"] is None and recs[1]["wall_s"] == 0.25
    for line in p.read_text().splitlines():
        json.loads(line, parse_constant=lambda c: pytest.fail(f"non-strict JSON {c}"))
    with ReportLog(p) as log:  # append
        log.write({"status": 0}, step=9)
    assert read_reports(p)[-1]["step"] == 9 and len(read_reports(p)) == 3
