"""Checkpoint / resume: the saved state round-trips (CPU), and a resumed run
equals an uninterrupted one bit for bit (GPU, FP64 and mixed contexts, with
Levenberg-Marquardt damping on, App. G)."""
import numpy as np
import pytest
import torch

from paper_2608_18065_b300 import checkpoint
from paper_2608_18065_b300.inputs import HamSpec, HParams, ModelSpec, init_theta

STATS_LEN = 11


class _Ctx:
    device = torch.device("cpu")

    def __init__(self):
        self.damping = None

    def set_damping(self, omega, lam):
        self.damping = (omega, lam)


def test_round_trip(tmp_path):
    hp = HParams(0.1, 1e4, 0.7, lam=2e-3, lambda_mode=1, lambda_coeff=3e-4, lambda_pow=2 / 3,
                 trust_region=1, seed=9, ns=40)
    th = torch.tensor(np.random.default_rng(1).standard_normal(50))
    m = torch.tensor(np.random.default_rng(2).standard_normal(50))
    st = torch.zeros(STATS_LEN, dtype=torch.float64)
    st[10] = 0.0375  # lambda_next
    p = tmp_path / "ck.npz"
    checkpoint.save(p, th, m, 17, hp, st, damping_omega=1.5)
    c = _Ctx()
    th2, m2, t, hp2 = checkpoint.load(p, c)
    assert torch.equal(th2, th) and torch.equal(m2, m) and t == 17 and hp2 == hp
    assert c.damping == (1.5, 0.0375)
    checkpoint.save(p, th, m, 3, hp, st)  # damping off in the saved run
    c = _Ctx()
    c.damping = (1.5, 0.02)  # ... but on in the target context: switched off
    checkpoint.load(p, c)
    assert c.damping is not None and c.damping[0] <= 1.0


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_resume_is_bit_exact(prec, tmp_path):
    from paper_2608_18065_b300 import nqs
    model, ham = ModelSpec(1, 16, 1, 16), HamSpec("tfim")
    hp = HParams(0.5, 1e3, 0.7, lam=1e-3, ns=64)
    omega = 1.5

    def fresh():
        c = nqs.Context(model, ham, prec, hp.ns)
        c.set_damping(omega, hp.lam)
        th = torch.tensor(init_theta(model, 5), device="cuda")
        return c, th, torch.zeros_like(th), c.new_stats()

    c, th, m, s = fresh()
    for t in range(6):
        c.minsr_step(th, m, hp, t, s)
    c2, th2, m2, s2 = fresh()
    for t in range(3):
        c2.minsr_step(th2, m2, hp, t, s2)
    p = tmp_path / "ck.npz"
    checkpoint.save(p, th2, m2, 3, hp, s2, damping_omega=omega)
    c3 = nqs.Context(model, ham, prec, hp.ns)
    th3, m3, t0, hp3 = checkpoint.load(p, c3)
    s3 = c3.new_stats()
    for t in range(t0, 6):
        c3.minsr_step(th3, m3, hp3, t, s3)
    torch.cuda.synchronize()
    assert torch.equal(th3, th) and torch.equal(m3, m)
    assert torch.equal(s3, s)
