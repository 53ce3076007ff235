"""Per-step diagnostics as JSON Lines.

A :class:`ReportLog` appends one JSON object per step: the report of
``Simulation.step`` (energies, the relative energy error, the Gauss and Lorenz
residuals, the work and chain-rule residuals, outer iterations, map
evaluations, inner iteration counts, status; the diagnostics of Sec. 5) plus a
step index and whatever fixed fields the caller attaches.  Non-finite numbers
are written as null, so every line is strict JSON.
"""
from __future__ import annotations

import json
import math
import os


def _clean(v):
    if isinstance(v, bool) or v is None or isinstance(v, str):
        return v
    if isinstance(v, (list, tuple)):
        return [_clean(x) for x in v]
    if isinstance(v, dict):
        return {str(k): _clean(x) for k, x in v.items()}
    if hasattr(v, "item") and not hasattr(v, "__len__"):  # numpy scalar
        v = v.item()
    if isinstance(v, int):
        return v
    f = float(v)
    return f if math.isfinite(f) else None


class ReportLog:
    """Append step reports to a JSON Lines file.

    ``meta`` holds fields written into every line (a run name, the workload).
    Each line is flushed as it is written, so a crashed run keeps every step
    it completed.
    """

    def __init__(self, path, mode: str = "a", **meta):
        if mode not in ("a", "w"):
            raise ValueError("mode must be 'a' or 'w'")
        self.path = os.fspath(path)
        self.meta = _clean(meta)
        self._f = open(self.path, mode, encoding="utf-8")
        self.count = 0

    def write(self, report: dict, step: int | None = None, **extra) -> dict:
        rec = dict(self.meta)
        rec["step"] = self.count if step is None else int(step)
        rec.update(_clean(report))
        rec.update(_clean(extra))
        self._f.write(json.dumps(rec, allow_nan=False, sort_keys=True) + "\n")
        self._f.flush()
        self.count += 1
        return rec

    def close(self):
        if self._f is not None:
            self._f.close()
            self._f = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def read_reports(path) -> list[dict]:
    """The records of a JSON Lines report file, in order."""
    with open(path, encoding="utf-8") as f:
        return [json.loads(line) for line in f if line.strip()]
