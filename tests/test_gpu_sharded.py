"""The sample-sharded step's library stages (nqs_shard_forward, _center,
_solve, _apply) on the GPU.

G = 1 runs sharded_step without a process group and must equal
nqs_minsr_step.  G = 2 and 3 run the ranks' stages one after another in
this process, one context per rank on the same GPU (no kernel of one rank
waits for another's: the exchanges are the sums, row and delta theta
concatenations done here between the calls), and must give the
single-rank oracle step: FP64 to 1e-10, every rank's theta identical.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2608_18065_b300 import nqs
from paper_2608_18065_b300.inputs import HamSpec, HParams, ModelSpec, TAB1, init_theta
from paper_2608_18065_b300.sharded import ShardBackend, partition, sharded_step
from tests.gpu_helpers import RTOL64, rel_err

pytestmark = pytest.mark.gpu

CASES = [
    (ModelSpec(1, 16, 1, 16), HamSpec("tfim"), HParams(ns=96, **TAB1["tfim"])),
    (ModelSpec(2, 4, 4, 16, cplx=1, marshall=1, zmask=1), HamSpec("j1j2", J2=0.5),
     HParams(ns=77, **TAB1["j1j2"])),
    (ModelSpec(2, 4, 4, 8, cplx=1, marshall=1, zmask=1), HamSpec("j1j2", J2=0.0),
     HParams(ns=64, **TAB1["heisenberg"])),
]
IDS = ["tfim16", "j1j2_4x4_trust", "heis4x4_normpow"]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("model,ham,hp", CASES, ids=IDS)
def test_sharded_one_rank_equals_step(model, ham, hp, prec):
    th0 = init_theta(model, 1234)
    a = nqs.Context(model, ham, prec, hp.ns)
    b = nqs.Context(model, ham, prec, hp.ns)
    tha = torch.tensor(th0, device="cuda")
    ma = torch.zeros_like(tha)
    thb, mb = tha.clone(), ma.clone()
    for t in range(2):
        sa = a.minsr_step(tha, ma, hp, t)
        sb = sharded_step(ShardBackend(b), thb, mb, hp, t)
        torch.cuda.synchronize()
        da, db = nqs.decode_stats(sa), nqs.decode_stats(sb)
        assert da["status"] == 0 and db["status"] == 0
        tol = 1e-12 if prec == "fp64" else 5e-4
        step_a = (tha - torch.tensor(th0, device="cuda")).cpu().numpy()
        step_b = (thb - torch.tensor(th0, device="cuda")).cpu().numpy()
        assert rel_err(step_b, step_a) < tol, (t, rel_err(step_b, step_a))
        assert abs(db["E_re"] - da["E_re"]) <= (1e-12 if prec == "fp64" else 2e-4) * abs(da["E_re"])


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("model,ham,hp", CASES, ids=IDS)
def test_sharded_ranks_equal_oracle_step(model, ham, hp, world):
    th0 = init_theta(model, 1234)
    ctxs = [nqs.Context(model, ham, "fp64", hp.ns) for _ in range(world)]
    bes = [ShardBackend(c) for c in ctxs]
    ths = [torch.tensor(th0, device="cuda") for _ in range(world)]
    mos = [torch.zeros_like(t) for t in ths]
    th_o, mo_o = th0.copy(), np.zeros_like(th0)
    nb = bes[0].blocks
    for t in range(2):
        stats = [be.new_stats() for be in bes]
        parts = [partition(hp.ns, world, r) for r in range(world)]
        sums = [be.forward(ths[r], hp, t, *parts[r]) for r, be in enumerate(bes)]
        tot = torch.stack(sums).sum(0)  # the allreduce
        cen = [be.center(tot, hp.ns, parts[r][1], stats[r]) for r, be in enumerate(bes)]
        rows = torch.cat([c[0] for c in cen], 0)  # the allgathers, rank order
        eps = torch.cat([c[1] for c in cen], 0)
        assert rows.shape[0] == nb * hp.ns
        pp = [partition(bes[0].np, world, r) for r in range(world)]
        dth = torch.cat([be.solve(rows, eps, hp, t, p0, p0 + n, stats[r])
                         for r, (be, (p0, n)) in enumerate(zip(bes, pp))], 0)
        for r, be in enumerate(bes):
            be.apply(ths[r], mos[r], dth, hp, t, stats[r])
        torch.cuda.synchronize()
        th_o, mo_o, st_o, _ = O.minsr_step(model, ham, th_o, mo_o, hp, t)
        for r in range(world):
            d = nqs.decode_stats(stats[r])
            assert d["status"] == 0
            assert abs(d["E_re"] - st_o["E_re"]) <= RTOL64 * abs(st_o["E_re"])
            assert rel_err(ths[r].cpu().numpy(), th_o) < RTOL64
            assert rel_err(mos[r].cpu().numpy(), mo_o) < RTOL64
            assert torch.equal(ths[r], ths[0])
