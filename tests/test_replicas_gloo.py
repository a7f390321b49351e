"""N > 1 benchmark path on CPU: two gloo ranks run the replica host logic.

Each replica steps its own instance (no data-path collective): the replica
of rank r is the single-rank oracle step with Philox key seed + r, the
timed region is reduced by MAX over ranks, and the whole-job rate sums the
replicas.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2608_18065_b300.replicas import aggregate_rate, max_over_ranks, replica_hparams


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    from oracle import oracle as O
    from paper_2608_18065_b300.inputs import init_theta, workloads
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = workloads()["tfim16"]
        hp = replica_hparams(w.hp, rank)
        hp.ns = 16
        th = init_theta(w.model, w.theta_seed)
        th1, _, st, bufs = O.minsr_step(w.model, w.ham, th, np.zeros_like(th), hp, 0,
                                        want=("spins",))
        ms = 10.0 + 5.0 * rank  # this rank's timed region
        dist.barrier()
        mx = max_over_ranks(ms, dist, "cpu")
        out[rank] = (hp.seed, float(st["E_re"]), bufs["spins"].tobytes(), mx,
                     aggregate_rate(world, 4, mx), th1.tobytes())
    finally:
        dist.destroy_process_group()


def test_two_replicas_on_gloo():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    from oracle import oracle as O
    from paper_2608_18065_b300.inputs import init_theta, workloads
    w = workloads()["tfim16"]
    th = init_theta(w.model, w.theta_seed)
    # every rank sees the slowest rank's time and the summed rate
    for r in range(world):
        assert res[r][3] == 15.0
        assert res[r][4] == pytest.approx(2 * 4 / 0.015)
    # distinct Philox keys, distinct samples
    assert res[0][0] != res[1][0]
    assert res[0][2] != res[1][2]
    # each replica is exactly the single-rank step with its own key
    for r in range(world):
        hp = replica_hparams(w.hp, r)
        hp.ns = 16
        th1, _, st, bufs = O.minsr_step(w.model, w.ham, th, np.zeros_like(th), hp, 0,
                                        want=("spins",))
        assert res[r][2] == bufs["spins"].tobytes()
        assert res[r][5] == th1.tobytes()


def test_single_rank_helpers():
    assert max_over_ranks(3.5) == 3.5
    assert aggregate_rate(1, 10, 500.0) == 20.0
