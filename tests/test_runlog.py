"""Per-step JSON lines: the fields of the step statistics as the library
lays them out (8 doubles, the int32 pair status / solve_fp64, rho,
lambda_next), the relative energy error and stage times."""
import json

import torch

from paper_2608_18065_b300 import runlog


def _stats(E, status, fp64):
    s = torch.zeros(11, dtype=torch.float64)
    s[:8] = torch.tensor([E, 0.0, 2.5, 0.125, 1e-3, 40.0, 0.05, 3.0], dtype=torch.float64)
    s[8:9].view(torch.int32)[0] = status
    s[8:9].view(torch.int32)[1] = fp64
    s[9], s[10] = 0.8, 1e-3
    return s


def test_lines(tmp_path):
    p = tmp_path / "run.jsonl"
    with runlog.StepLog(p, e_exact=-20.0) as log:
        log.write(0, _stats(-19.0, 0, 0), stage_ms={"sample": 0.2, "cholesky": 0.5})
        log.write(1, _stats(-19.5, 5, 1))
    recs = [json.loads(x) for x in open(p)]
    assert [r["step"] for r in recs] == [0, 1]
    assert recs[0]["E_re"] == -19.0 and abs(recs[0]["rel_err"] - 0.05) < 1e-15
    assert recs[0]["vscore"] == 0.125 and recs[0]["lambda_next"] == 1e-3 and recs[0]["rho"] == 0.8
    assert recs[0]["stage_ms"] == {"sample": 0.2, "cholesky": 0.5}
    assert recs[1]["status"] == 5 and recs[1]["solve_fp64"] == 1 and "stage_ms" not in recs[1]
