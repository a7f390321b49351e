"""Pins of the oracle's per-sample log-derivatives O (Sec. II.C)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2608_18065_b300.inputs import HamSpec, ModelSpec, init_theta, random_spins
from tests.exact import all_configs, dense_tfim, torch_logpsi

CASES = [
    ModelSpec(1, 7, 1, 4),
    ModelSpec(1, 6, 1, 3, cplx=1),
    ModelSpec(2, 3, 3, 3, cplx=1, marshall=1),
    ModelSpec(2, 2, 4, 3, cplx=1, marshall=1, zmask=1),
]


@pytest.mark.parametrize("spec", CASES, ids=str)
def test_jacobian_central_differences(spec):
    """O against central finite differences of log Psi (step 1e-5): relative
    error <= 1e-7 on the gradient of each sample."""
    th = init_theta(spec, 21)
    sp = random_spins(spec, 4, seed=2, zero_mag=bool(spec.zmask))
    Oj = O.jacobian(spec, th, sp)
    h = 1e-5
    fd = np.zeros((2, len(sp), len(th)))
    for k in range(len(th)):
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        d = (O.logpsi(spec, tp, sp) - O.logpsi(spec, tm, sp)) / (2 * h)
        fd[0, :, k] = d.real
        fd[1, :, k] = d.imag
    ns = len(sp)
    for s in range(ns):
        err = np.linalg.norm(Oj[s] - fd[0, s]) / np.linalg.norm(fd[0, s])
        assert err < 1e-7
        if spec.cplx:
            err = np.linalg.norm(Oj[ns + s] - fd[1, s]) / np.linalg.norm(fd[1, s])
            assert err < 1e-7


@pytest.mark.parametrize("spec", CASES, ids=str)
def test_jacobian_equals_library_autodiff(spec):
    """O equals torch autograd through the library GRU cell, element by
    element."""
    th = init_theta(spec, 13)
    sp = random_spins(spec, 3, seed=5, zero_mag=bool(spec.zmask))
    Oj = O.jacobian(spec, th, sp)
    ns = len(sp)
    for s in range(ns):
        t = torch.tensor(th, requires_grad=True)
        re, im = torch_logpsi(spec, t, sp[s:s + 1])
        g, = torch.autograd.grad(re.sum(), t)
        np.testing.assert_allclose(Oj[s], g.numpy(), rtol=0, atol=1e-12)
        if spec.cplx:
            t = torch.tensor(th, requires_grad=True)
            re, im = torch_logpsi(spec, t, sp[s:s + 1])
            g, = torch.autograd.grad(im.sum(), t)
            np.testing.assert_allclose(Oj[ns + s], g.numpy(), rtol=0, atol=1e-12)


def test_score_mean_zero_and_exact_energy_gradient():
    """pRNN: sum_sigma P O = 0 (a normalised model's score has zero mean), and
    dE/dtheta = 2 Re sum_sigma P O* (eps - E) equals finite differences of the
    exact energy <Psi|H|Psi> (Sec. II.C)."""
    spec = ModelSpec(1, 7, 1, 3)
    ham = HamSpec("tfim", J=1.0, h=0.8)
    Hd = dense_tfim(7, 1.0, 0.8).real
    th = init_theta(spec, 30)
    allc = all_configs(spec.N)
    P = np.exp(2 * O.logpsi(spec, th, allc).real)
    Oj = O.jacobian(spec, th, allc)
    assert np.max(np.abs(P @ Oj)) < 1e-13
    el = O.local_energy(spec, ham, th, allc).real
    E = P @ el
    grad = 2 * (P * (el - E)) @ Oj

    def energy(t):
        psi = np.exp(O.logpsi(spec, t, allc).real)
        return psi @ Hd @ psi

    h = 1e-5
    for k in range(0, len(th), 7):
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        fd = (energy(tp) - energy(tm)) / (2 * h)
        assert abs(fd - grad[k]) < 1e-8 * max(1.0, abs(fd))
