"""Failure detection by bounded waits, exercised on the GPU without a fault:
a test hook makes the streamed 2D local-energy engine's producer never
publish its first tile, with a short wait limit.  Every other role's wait
runs out, the kernel returns, the step reports NQS_ERR_TIMEOUT and leaves
theta and momentum unchanged, and the same context steps normally once the
hook is cleared."""
import numpy as np
import pytest
import torch

from paper_2608_18065_b300 import nqs
from paper_2608_18065_b300.inputs import HamSpec, HParams, ModelSpec, TAB1, init_theta

pytestmark = pytest.mark.gpu

NQS_ERR_TIMEOUT = 6


def test_wait_that_runs_out_reports_timeout_and_keeps_theta():
    model = ModelSpec(2, 4, 4, 128, cplx=1, marshall=1, zmask=1)
    hp = HParams(ns=64, **TAB1["j1j2"])
    c = nqs.Context(model, HamSpec("j1j2", J2=0.5), "mixed", hp.ns)
    th = torch.tensor(init_theta(model, 5), device="cuda")
    mo = torch.zeros_like(th) + 0.25
    th0, mo0 = th.clone(), mo.clone()
    c.test_wait_timeout(spin_limit=1 << 12, drop_tile=True)
    st = nqs.decode_stats(c.minsr_step(th, mo, hp, 0))
    torch.cuda.synchronize()
    assert st["status"] == NQS_ERR_TIMEOUT, st
    assert torch.equal(th, th0) and torch.equal(mo, mo0)
    # the context is still usable
    c.test_wait_timeout(0, False)
    st = nqs.decode_stats(c.minsr_step(th, mo, hp, 1))
    torch.cuda.synchronize()
    assert st["status"] == 0, st
    assert not torch.equal(th, th0)
    assert np.isfinite(st["E_re"])
