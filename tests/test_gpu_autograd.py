"""torch.autograd through libnqs: LogPsi's backward (hand-written reverse
mode + on-device contraction) against the oracle's log-derivatives."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2608_18065_b300 import nqs
from paper_2608_18065_b300.inputs import HamSpec, ModelSpec, init_theta, random_spins
from tests.gpu_helpers import RTOL64, rel_err

pytestmark = pytest.mark.gpu

CASES = [(ModelSpec(1, 14, 1, 16), HamSpec("tfim")),
         (ModelSpec(2, 4, 4, 8, cplx=1, marshall=1, zmask=1), HamSpec("j1j2", J2=0.5))]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("model,ham", CASES, ids=["1d", "2d"])
def test_logpsi_autograd_backward(model, ham, prec):
    ns = 40
    c = nqs.Context(model, ham, prec, ns)
    th = init_theta(model, 2)
    sp = random_spins(model, ns, seed=3, zero_mag=bool(model.zmask))
    t = torch.tensor(th, device="cuda", requires_grad=True)
    spd = torch.tensor(sp, device="cuda")
    rng = np.random.default_rng(1)
    g = rng.standard_normal((ns, 2))
    out = nqs.logpsi(t, spd, c)
    loss = (out * torch.tensor(g, device="cuda")).sum()
    loss.backward()
    J = O.jacobian(model, th, sp)
    ref = g[:, 0] @ J[:ns] + (g[:, 1] @ J[ns:] if model.cplx else 0.0)
    assert rel_err(t.grad.cpu().numpy(), ref) < (RTOL64 if prec == "fp64" else 2e-4)
    np.testing.assert_allclose(out.detach().cpu().numpy()[:, 0],
                               O.logpsi(model, th, sp).real, atol=1e-4)
