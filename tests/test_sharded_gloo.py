"""The sample-sharded minSR step (paper_2608_18065_b300.sharded) on CPU gloo
ranks: G = 2 and 3 ranks each draw their own range of the step's samples
(their own Philox counters), and after the allreduce of the centring sums,
the allgather of the centred rows and the allgather of the delta theta
ranges every rank holds the single-rank oracle step's theta and momentum
(FP64, 1e-12), over two chained steps.

The backend here does each rank's arithmetic with the oracle's sampler,
local energies, Jacobian and Cholesky solve; the decomposition and the
collectives under test are the product's (sharded_step).
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2608_18065_b300.inputs import HamSpec, HParams, ModelSpec, TAB1, init_theta
from paper_2608_18065_b300.sharded import partition

CASES = {
    "tfim16": (ModelSpec(1, 16, 1, 16), HamSpec("tfim"), HParams(ns=40, **TAB1["tfim"])),
    "heis4x4_c": (ModelSpec(2, 4, 4, 8, cplx=1, marshall=1, zmask=1), HamSpec("j1j2", J2=0.0),
                  HParams(ns=31, **TAB1["heisenberg"])),
    "j1j2_4x4_trust": (ModelSpec(2, 4, 4, 8, cplx=1, marshall=1, zmask=1),
                       HamSpec("j1j2", J2=0.5), HParams(ns=29, **TAB1["j1j2"])),
}


class OracleShardBackend:
    """A rank's stages computed with the FP64 oracle (CPU tensors)."""

    def __init__(self, model, ham):
        from oracle import oracle as O
        self.O = O
        self.model, self.ham = model, ham
        self.blocks = 2 if model.cplx else 1
        self.np = len(init_theta(model, 0))

    def new_stats(self):
        return {}

    def forward(self, theta, hp, t, s0, n):
        th = theta.numpy()
        sp, _ = self.O.sample(self.model, th, n, hp.seed, t, s0=s0)
        self.eloc = self.O.local_energy(self.model, self.ham, th, sp)
        self.J = self.O.jacobian(self.model, th, sp)
        nb, np_ = self.blocks, self.np
        col = np.concatenate([self.J[b * n:(b + 1) * n].sum(0) for b in range(nb)])
        e = self.eloc
        return torch.tensor(np.concatenate([col, [e.real.sum(), e.imag.sum(),
                                                  (np.abs(e) ** 2).sum()]]))

    def center(self, sums, ns, n, stats):
        s = sums.numpy()
        nb, np_ = self.blocks, self.np
        mean = s[:nb * np_].reshape(nb, np_) / ns
        E = (s[nb * np_] + 1j * s[nb * np_ + 1]) / ns
        stats["E"] = E
        rows = np.concatenate([(self.J[b * n:(b + 1) * n] - mean[b]) / np.sqrt(ns)
                               for b in range(nb)])
        d = (self.eloc - E) / np.sqrt(ns)
        eps = 2 * np.concatenate([d.real] + ([d.imag] if self.model.cplx else []))
        return torch.tensor(rows), torch.tensor(eps)

    def solve(self, rows, eps, hp, t, p0, p1, stats):
        A, b = rows.numpy(), eps.numpy()
        T = A @ A.T
        lam = hp.lam if hp.lambda_mode == 0 else hp.lambda_coeff * np.linalg.norm(T) ** hp.lambda_pow
        rc, x = self.O.cholesky_solve(T + lam * np.eye(len(b)), b)
        assert rc == 0
        tau = np.linalg.norm(b - lam * x)
        eta = hp.eta0 / (1.0 + t / hp.decay_T)
        if hp.trust_region:
            eta = eta / tau
        stats["lam"] = lam
        return torch.tensor(eta * (A[:, p0:p1].T @ x))

    def apply(self, theta, mom, dtheta, hp, t, stats):
        m = hp.mu * mom.numpy() + (1 - hp.mu) * dtheta.numpy()
        mom.copy_(torch.tensor(m))
        theta.sub_(torch.tensor(m))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, key, out):
    import torch.distributed as dist
    from paper_2608_18065_b300.sharded import Group, sharded_step
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        model, ham, hp = CASES[key]
        be = OracleShardBackend(model, ham)
        th = torch.tensor(init_theta(model, 1234))
        mo = torch.zeros_like(th)
        res = []
        for t in range(2):
            st = sharded_step(be, th, mo, hp, t, group=Group.current())
            res.append((th.numpy().tobytes(), mo.numpy().tobytes(), complex(st["E"])))
        out[rank] = res
    finally:
        dist.destroy_process_group()


def test_partition_covers_every_item_once():
    for total in (1, 7, 40, 1024, 13058):
        for world in (1, 2, 3, 8):
            if world > total:
                continue
            parts = [partition(total, world, r) for r in range(world)]
            assert parts[0][0] == 0
            for (a, n), (b, _) in zip(parts, parts[1:]):
                assert a + n == b
            assert sum(n for _, n in parts) == total
            assert max(n for _, n in parts) - min(n for _, n in parts) <= 1


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("key", list(CASES))
def test_sharded_step_equals_single_rank_oracle(key, world):
    from oracle import oracle as O
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, key, out))
                 for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(300)
            assert p.exitcode == 0
        res = dict(out)
    model, ham, hp = CASES[key]
    th = init_theta(model, 1234)
    mo = np.zeros_like(th)
    for t in range(2):
        th, mo, st, _ = O.minsr_step(model, ham, th, mo, hp, t)
        for r in range(world):
            th_r = np.frombuffer(res[r][t][0])
            mo_r = np.frombuffer(res[r][t][1])
            assert np.linalg.norm(th_r - th) <= 1e-12 * np.linalg.norm(th)
            assert np.linalg.norm(mo_r - mo) <= 1e-12 * np.linalg.norm(mo)
            assert abs(res[r][t][2].real - st["E_re"]) <= 1e-12 * abs(st["E_re"])
        # every rank holds the same parameters
        assert all(res[r][t][0] == res[0][t][0] for r in range(world))
