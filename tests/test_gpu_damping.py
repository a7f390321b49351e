"""Levenberg-Marquardt damping (App. G) on the GPU against the oracle.

FP64: every step's samples are bit-exact, and the damping sequence, the gain
ratio and theta follow the oracle chained step by step (the oracle is
stateless: it takes lambda_t and returns lambda_{t+1}; the library keeps the
damping on the device).  Mixed: the update rule holds on the reported ratio,
and a graph replay gives the eager result bit for bit.
"""
import copy

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2608_18065_b300 import nqs
from paper_2608_18065_b300.inputs import HamSpec, HParams, ModelSpec, init_theta
from tests.gpu_helpers import RTOL64

pytestmark = pytest.mark.gpu

OMEGA = 1.5
CASES = [
    (ModelSpec(1, 16, 1, 16), HamSpec("tfim"), HParams(0.5, 1e3, 0.7, lam=1e-3, ns=64)),
    (ModelSpec(2, 4, 2, 8, cplx=1, marshall=1, zmask=1), HamSpec("j1j2", J2=0.5),
     HParams(0.1, 1e4, 0.1, lam=0.1, trust_region=1, ns=48)),
]


@pytest.mark.parametrize("model,ham,hp", CASES, ids=["tfim16", "j1j2_4x2_tr"])
def test_damping_fp64_against_oracle(model, ham, hp):
    th = init_theta(model, 8)
    c = nqs.Context(model, ham, "fp64", hp.ns)
    c.set_damping(OMEGA, hp.lam)
    thd = torch.tensor(th, device="cuda")
    md = torch.zeros_like(thd)
    th_o, mo_o = th.copy(), np.zeros_like(th)
    lam = hp.lam
    lams = set()
    for t in range(4):
        out = c.step_outputs(hp.ns)
        s = c.new_stats()
        c.minsr_step(thd, md, hp, t, s, outputs=out)
        torch.cuda.synchronize()
        d = nqs.decode_stats(s)
        h = copy.copy(hp)
        h.lam = lam
        h.lm_omega = OMEGA
        th_o, mo_o, st, b = O.minsr_step(model, ham, th_o, mo_o, h, t, want=("spins",))
        assert np.array_equal(out["spins"].cpu().numpy(), b["spins"])
        assert d["status"] == st["status"] == 0
        assert d["lam"] == pytest.approx(lam, rel=1e-12)
        assert d["rho"] == pytest.approx(st["rho"], rel=1e-8, abs=1e-12)
        assert d["lambda_next"] == pytest.approx(st["lambda_next"], rel=1e-12)
        np.testing.assert_allclose(thd.cpu().numpy(), th_o, rtol=RTOL64, atol=RTOL64)
        lams.add(round(lam / hp.lam, 6))
        lam = st["lambda_next"]


def test_damping_mixed_rule_and_graph():
    model, ham = ModelSpec(1, 20, 1, 64), HamSpec("tfim")
    hp = HParams(0.5, 1e3, 0.7, lam=1e-3, ns=300)
    th0 = torch.tensor(init_theta(model, 9), device="cuda")
    res = []
    for graph in (False, True):
        c = nqs.Context(model, ham, "mixed", hp.ns)
        c.use_graph(graph)
        c.set_damping(OMEGA, hp.lam)
        t_ = th0.clone()
        m_ = torch.zeros_like(t_)
        s = c.new_stats()
        hist = []
        for t in range(4):
            c.minsr_step(t_, m_, hp, t, s)
            torch.cuda.synchronize()
            hist.append(nqs.decode_stats(s))
        res.append((t_, hist))
        assert c.graph_active() == graph
    for d in res[0][1]:
        assert d["status"] == 0
        lam, rho = d["lam"], d["rho"]
        want = lam * OMEGA if rho < 0.25 else (lam / OMEGA if rho > 0.75 else lam)
        assert d["lambda_next"] == pytest.approx(want, rel=1e-15)
    for a, b in zip(res[0][1], res[1][1]):
        assert a["lam"] == b["lam"] and a["rho"] == b["rho"]
    assert torch.equal(res[0][0], res[1][0])
    # consecutive steps chain the damping on the device
    for a, b in zip(res[0][1][:-1], res[0][1][1:]):
        assert b["lam"] == a["lambda_next"]


def test_damping_off_and_arguments():
    model, ham = ModelSpec(1, 8, 1, 8), HamSpec("tfim")
    hp = HParams(0.5, 1e3, 0.7, lam=1e-3, ns=32)
    c = nqs.Context(model, ham, "fp64", hp.ns)
    with pytest.raises(nqs.NqsError):
        c.set_damping(2.0, -1.0)
    c.set_damping(2.0, 1e-2)
    c.set_damping(1.0, 0.0)  # off again: hp.lam is used
    th = torch.tensor(init_theta(model, 1), device="cuda")
    s = c.new_stats()
    c.minsr_step(th, torch.zeros_like(th), hp, 0, s)
    d = nqs.decode_stats(s)
    assert d["lam"] == hp.lam and d["rho"] == 0.0 and d["lambda_next"] == hp.lam
