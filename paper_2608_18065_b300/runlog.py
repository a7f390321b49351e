"""Per-step metrics of a minSR run as JSON lines (host-side).

Each line holds the step index and the step's statistics as the library
reports them: E (Eq. energy), Var, the V-score (Eq. vscore), the damping
lambda and ||T||_F, the effective step size and ||tau|| (App. F), the
device status word, which factorisation produced x, and the
Levenberg-Marquardt ratio and next damping (App. G).  Given the exact
energy, the relative error (E - E_exact) / |E_exact| is added; given
per-stage times (nqs_timing_end), they are added in milliseconds.
"""
import json

from . import nqs


def step_record(step_index, stats, e_exact=None, stage_ms=None):
    """One step's record (a dict of plain numbers)."""
    rec = {"step": int(step_index)}
    rec.update(nqs.decode_stats(stats))
    if e_exact is not None:
        rec["rel_err"] = (rec["E_re"] - e_exact) / abs(e_exact)
    if stage_ms is not None:
        rec["stage_ms"] = {k: float(v) for k, v in stage_ms.items()}
    return rec


class StepLog:
    """Appends one JSON line per step to a file."""

    def __init__(self, path, e_exact=None):
        self.f = open(path, "a", encoding="utf-8")
        self.e_exact = e_exact

    def write(self, step_index, stats, stage_ms=None):
        self.f.write(json.dumps(step_record(step_index, stats, self.e_exact, stage_ms)) + "\n")
        self.f.flush()

    def close(self):
        self.f.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
