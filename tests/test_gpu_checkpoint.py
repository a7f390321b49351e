"""Hidden-state checkpoints every c sites (nqs_options.checkpoint_stride):
the reverse sweep recomputes each segment from its checkpoint and the
local energies restart from the last checkpoint before their first changed
site.  FP64: samples, log Psi and E_loc are bit-identical to the fully
cached context (same kernels, same arithmetic); O and the step agree with
the oracle to the FP64 tolerance.  Mixed: the same tolerances as the fully
cached mixed path."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2608_18065_b300 import nqs
from paper_2608_18065_b300.inputs import HamSpec, HParams, ModelSpec, TAB1, init_theta, random_spins
from tests.gpu_helpers import (RTOL64, TOL_MIXED_ELOC, TOL_MIXED_JAC, cplx, max_elem_err,
                               max_row_err, rel_err)

pytestmark = pytest.mark.gpu

CASES = [
    (ModelSpec(1, 20, 1, 16), HamSpec("tfim"), "fp64", 64, -1),
    (ModelSpec(1, 12, 1, 16, cplx=1), HamSpec("cluster_zxz"), "fp64", 48, 5),
    (ModelSpec(1, 33, 1, 64), HamSpec("tfim"), "mixed", 200, 6),
    (ModelSpec(1, 16, 1, 32, cplx=1), HamSpec("cluster_paper"), "mixed", 96, 1),
    (ModelSpec(1, 14, 1, 16), HamSpec("tfim"), "fp64", 40, 14),
]
IDS = ["tfim20-sqrt", "cluster12-c5", "tfim33-mixed-c6", "clusterP16-mixed-c1", "tfim14-one-seg"]


@pytest.mark.parametrize("model,ham,prec,ns,ck", CASES, ids=IDS)
def test_checkpointed_stages(model, ham, prec, ns, ck):
    th = init_theta(model, 3)
    thd = torch.tensor(th, device="cuda")
    full = nqs.Context(model, ham, prec, ns)
    chk = nqs.Context(model, ham, prec, ns, checkpoint_stride=ck)
    assert chk.checkpoint_stride() == (int(np.ceil(np.sqrt(model.N))) if ck == -1 else ck)
    if chk.checkpoint_stride() < model.N:
        assert chk.workspace_bytes < full.workspace_bytes
    spins = torch.tensor(random_spins(model, ns, 11), device="cuda")
    el_f = cplx(full.local_energy(thd, spins))
    el_c = cplx(chk.local_energy(thd, spins))
    O_f = full.jacobian(thd, spins).cpu().numpy()
    O_c = chk.jacobian(thd, spins).cpu().numpy()
    sp = spins.cpu().numpy()
    el_o = O.local_energy(model, ham, th, sp)
    O_o = O.jacobian(model, th, sp)
    if prec == "fp64":
        assert np.array_equal(el_c, el_f)
        assert rel_err(O_c, O_o) < RTOL64
        assert rel_err(O_c, O_f) < 1e-13
    else:
        assert rel_err(el_c, el_o) < TOL_MIXED_ELOC
        assert max_elem_err(el_c, el_o) < TOL_MIXED_ELOC
        assert rel_err(O_c, O_o) < TOL_MIXED_JAC
        assert max_row_err(O_c, O_o) < TOL_MIXED_JAC


@pytest.mark.parametrize("model,ham,prec,ns,ck", CASES[:3], ids=IDS[:3])
def test_checkpointed_step(model, ham, prec, ns, ck):
    col = {"tfim": "tfim", "cluster_zxz": "cluster", "cluster_paper": "cluster"}[ham.family]
    hp = HParams(ns=ns, **TAB1[col])
    th = init_theta(model, 4)
    res = []
    for stride in (0, ck):
        c = nqs.Context(model, ham, prec, ns, checkpoint_stride=stride)
        t = torch.tensor(th, device="cuda")
        m = torch.zeros_like(t)
        s = c.new_stats()
        c.minsr_step(t, m, hp, 0, s)
        torch.cuda.synchronize()
        res.append((t.cpu().numpy(), nqs.decode_stats(s)))
    (t0, s0), (t1, s1) = res
    assert s1["status"] == 0
    if prec == "fp64":
        th_o, _, st_o, _ = O.minsr_step(model, ham, th, np.zeros_like(th), hp, 0)
        np.testing.assert_allclose(t1, th_o, rtol=RTOL64, atol=RTOL64)
        assert s1["E_re"] == s0["E_re"]
    else:
        assert rel_err(t1 - th, t0 - th) < 5e-4


def test_checkpoints_rejected_in_2d():
    with pytest.raises(nqs.NqsError):
        nqs.Context(ModelSpec(2, 4, 4, 16, cplx=1, marshall=1, zmask=1), HamSpec("j1j2"),
                    "fp64", 32, checkpoint_stride=-1)
