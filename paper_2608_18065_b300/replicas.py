"""Host logic of the N-GPU benchmark: independent replicas, no data-path
collective.

One minSR step of one instance does not split across GPUs without
exchanging the centring sums and the Gram matrix, so N GPUs run N
independent instances of the same workload (or N copies of the batched
workload): replica r keeps theta_0 and draws its samples from the Philox
key seed + r.  The only collectives are the timing barrier and the max over
ranks of the timed region; the reported rate is the sum over replicas.
"""
import copy


def replica_hparams(hp, rank: int):
    """Hyper-parameters of replica `rank`: its own Philox key."""
    h = copy.copy(hp)
    h.seed = h.seed + int(rank)
    return h


def max_over_ranks(ms: float, dist=None, device="cpu") -> float:
    """The slowest rank's time (every rank gets the same value)."""
    if dist is None or not dist.is_available() or not dist.is_initialized() \
            or dist.get_world_size() == 1:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(world: int, steps: int, ms: float) -> float:
    """Whole-job rate: every replica completed `steps` steps in `ms`."""
    return world * steps / (ms / 1000.0)
