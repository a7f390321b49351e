"""CUDA-graph replay of nqs_minsr_step gives bitwise the same trajectory as
eager launches, across consecutive and non-consecutive step indices."""
import numpy as np
import pytest
import torch

from paper_2608_18065_b300 import nqs
from paper_2608_18065_b300.inputs import HamSpec, HParams, ModelSpec, init_theta

pytestmark = pytest.mark.gpu

CASES = [
    ("mixed", ModelSpec(1, 24, 1, 64), HamSpec("tfim"), HParams(0.1, 1e3, 0.7, lam=1e-3, ns=256)),
    ("fp64", ModelSpec(1, 12, 1, 16), HamSpec("tfim"), HParams(0.1, 1e3, 0.7, lam=1e-3, ns=64)),
    ("mixed", ModelSpec(2, 4, 4, 16, cplx=1, marshall=1, zmask=1), HamSpec("j1j2", J2=0.5),
     HParams(0.1, 1e4, 0.1, lam=0.1, trust_region=1, ns=128)),
]


@pytest.mark.parametrize("prec,model,ham,hp", CASES, ids=["tfim-mixed", "tfim-fp64", "j1j2-mixed"])
def test_graph_replay_matches_eager(prec, model, ham, hp):
    th0 = init_theta(model, 5)
    runs = {}
    for mode in ("eager", "graph"):
        c = nqs.Context(model, ham, prec, hp.ns)
        if mode == "graph":
            c.use_graph(True)
        th = torch.tensor(th0, device="cuda")
        mo = torch.zeros_like(th)
        st = c.new_stats()
        traj = []
        for t in [0, 1, 2, 3, 7, 8]:  # a jump after step 3
            c.minsr_step(th, mo, hp, t, st)
            traj.append((th.cpu().numpy().copy(), nqs.decode_stats(st)))
        torch.cuda.synchronize()
        if mode == "graph":
            assert c.graph_active()
        runs[mode] = traj
    for (a, sa), (b, sb) in zip(runs["eager"], runs["graph"]):
        assert np.array_equal(a, b)
        assert sa == sb
