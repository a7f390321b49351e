"""Pins of the Adam comparator and the loss-landscape energies (oracle/adam.py).

* The sampled gradient g = Obar'^T eps-bar' is the large-lambda limit of
  the minSR step (a separate code path, itself pinned against the
  parameter-space SR solve): delta theta = eta Obar'^T (T + lambda I)^{-1}
  eps-bar' -> (eta / lambda) g as lambda -> infinity.
* Adam's first iteration is sign descent: with m = (1 - b1) g and
  v = (1 - b2) g^2 the bias corrections give m^ = g, v^ = g^2, so
  theta_1 = theta_0 - eta g / (|g| + epsilon).
* The second iteration, from the two gradients, by the closed-form moments.
* A landscape point at (0, 0) is the minSR step's sampled energy at the same
  theta, key and step.
"""
import numpy as np
import pytest

from oracle import adam as A
from oracle import oracle as O
from paper_2608_18065_b300.inputs import (AdamParams, HamSpec, HParams, ModelSpec, TAB1_ADAM,
                                          init_theta)

CASES = [(ModelSpec(1, 8, 1, 8), HamSpec("tfim")),
         (ModelSpec(2, 3, 2, 8, cplx=1, marshall=1, zmask=1), HamSpec("j1j2", J2=0.5))]


@pytest.mark.parametrize("spec,ham", CASES, ids=["tfim8", "j1j2_3x2_c"])
def test_gradient_is_large_lambda_limit_of_minsr(spec, ham):
    th = init_theta(spec, 11)
    ns = 40
    E, g = A.gradient(spec, ham, th, ns, 42, 3)
    lam, eta = 1e9, 0.7
    hp = HParams(eta0=eta, decay_T=1e4, mu=0.0, lam=lam, ns=ns, seed=42)
    _, _, st, b = O.minsr_step(spec, ham, th, np.zeros_like(th), hp, 3, want=("dtheta",))
    lim = b["dtheta"] * lam / (eta / (1.0 + 3 / hp.decay_T))  # eta_t of Tab. I's decay at t = 3
    assert np.linalg.norm(lim - g) <= 1e-6 * np.linalg.norm(g)
    assert abs(E.real - st["E_re"]) <= 1e-12 * abs(st["E_re"])


@pytest.mark.parametrize("spec,ham", CASES, ids=["tfim8", "j1j2_3x2_c"])
def test_first_two_adam_iterations_closed_form(spec, ham):
    th0 = init_theta(spec, 12)
    ap = AdamParams(ns=32, **TAB1_ADAM["tfim"])
    z = np.zeros_like(th0)
    th1, m, v, _, g0 = A.adam_step(spec, ham, th0, z, z, ap, 0)
    np.testing.assert_allclose(th1, th0 - ap.eta0 * g0 / (np.abs(g0) + ap.eps), rtol=0,
                               atol=1e-15)
    th2, m2, v2, _, g1 = A.adam_step(spec, ham, th1, m, v, ap, 1)
    b1, b2 = ap.beta1, ap.beta2
    mh = (b1 * (1 - b1) * g0 + (1 - b1) * g1) / (1 - b1 ** 2)
    vh = (b2 * (1 - b2) * g0 ** 2 + (1 - b2) * g1 ** 2) / (1 - b2 ** 2)
    np.testing.assert_allclose(th2, th1 - ap.eta0 * mh / (np.sqrt(vh) + ap.eps), rtol=1e-12,
                               atol=1e-15)


def test_decay_follows_tab1():
    spec, ham = CASES[0]
    th0 = init_theta(spec, 13)
    ap = AdamParams(ns=16, eta0=0.01, decay_T=4.0)
    z = np.zeros_like(th0)
    # at t = 8 (the ninth iteration) from zero moments, eta_t = eta0 / (1 + 8 / 4)
    th1, m, v, _, g = A.adam_step(spec, ham, th0, z, z, ap, 8)
    b1, b2 = ap.beta1, ap.beta2
    mh = (1 - b1) * g / (1 - b1 ** 9)
    vh = (1 - b2) * g ** 2 / (1 - b2 ** 9)
    np.testing.assert_allclose(th1, th0 - ap.eta0 / 3.0 * mh / (np.sqrt(vh) + ap.eps),
                               rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("spec,ham", CASES, ids=["tfim8", "j1j2_3x2_c"])
def test_landscape_origin_is_the_step_energy(spec, ham):
    th = init_theta(spec, 14)
    rng = np.random.default_rng(0)
    v1, v2 = rng.standard_normal(len(th)), rng.standard_normal(len(th))
    E = A.landscape(spec, ham, th, v1, v2, [0.0, 0.3], [0.0, -0.2], 24, 9)
    hp = HParams(eta0=0.1, decay_T=1e4, mu=0.0, lam=1e-3, ns=24, seed=9)
    _, _, st, _ = O.minsr_step(spec, ham, th, np.zeros_like(th), hp, 0)
    assert abs(E[0].real - st["E_re"]) <= 1e-12 * abs(st["E_re"])
    # a displaced point is the step energy of the displaced parameters
    _, _, st2, _ = O.minsr_step(spec, ham, th + 0.3 * v1 - 0.2 * v2, np.zeros_like(th), hp, 0)
    assert abs(E[1].real - st2["E_re"]) <= 1e-12 * abs(st2["E_re"])
