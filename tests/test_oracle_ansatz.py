"""Pins of the oracle's ansatz (Sec. II.A-B, App. A) and Philox generator."""
import itertools
import os

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2608_18065_b300.inputs import ModelSpec, init_theta, param_count, workloads
from tests.exact import all_configs, torch_logpsi

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    """Philox4x32-10 against its published known-answer vectors."""
    rows = [l.split() for l in open(os.path.join(GOLD, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert O.philox(v[0:4], v[4:6]) == v[6:10]


def test_uniform_definition_and_moments():
    o = O.philox([5, 9, 3, 0], [42, 0])
    bits = (o[1] << 32) | o[0]
    assert O.uniform(42, 3, 9, 5) == (bits >> 11) * 2.0 ** -53
    u = np.array([O.uniform(7, 0, s, k) for s in range(40) for k in range(100)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.02 and abs(u.var() - 1 / 12) < 0.01


def test_param_counts_match_layout():
    # counts implied by the layout of App. A for the benchmark models
    expect = {"tfim16": 962, "tfim100": 13058, "tfim200": 3458, "cluster64": 13188,
              "heis10": 21764,
              # 1D, d_h 256, complex head: 2 (256 x 258) + 256^2 + 4 x 256 + 256 x 2 + 2 x (2 x 256 + 2)
              "cluster100p": 2 * 256 * 258 + 256 ** 2 + 4 * 256 + 256 * 2 + 2 * (2 * 256 + 2),
              # 2D, d_h 200: U1, U2, 2 (200 x 204), 200^2, 4 x 200, 200 x 4, heads (+ phase head)
              "heis10p": 2 * 200 ** 2 + 2 * 200 * 204 + 200 ** 2 + 4 * 200 + 200 * 4 + 2 * 200 + 2,
              "j1j2_10p": 2 * 200 ** 2 + 2 * 200 * 204 + 200 ** 2 + 4 * 200 + 200 * 4 +
              2 * (2 * 200 + 2)}
    for key, w in workloads().items():
        assert O.param_count(w.model) == param_count(w.model) == expect[key]
    assert O.param_count(ModelSpec(2, 6, 6, 32, cplx=1)) == 5764
    assert O.param_count(ModelSpec(2, 6, 6, 128, cplx=1)) == 84484


CASES = [
    ModelSpec(1, 9, 1, 5),
    ModelSpec(1, 8, 1, 4, cplx=1),
    ModelSpec(2, 3, 3, 4),
    ModelSpec(2, 4, 3, 3, cplx=1, marshall=1),
    ModelSpec(2, 3, 4, 4, cplx=1, marshall=1, zmask=1),
    ModelSpec(1, 8, 1, 4, zmask=1),
]


@pytest.mark.parametrize("spec", CASES, ids=str)
def test_logpsi_matches_library_gru_cell(spec):
    """log Psi of the oracle equals a log Psi assembled from torch's GRU cell
    (App. A mapped onto the library cell) on random configurations."""
    th = init_theta(spec, 11)
    rng = np.random.default_rng(3)
    sp = rng.integers(0, 2, size=(64, spec.N), dtype=np.uint8)
    if spec.zmask:
        for s in range(len(sp)):
            sp[s] = 0
            sp[s, rng.permutation(spec.N)[: spec.N // 2]] = 1
    lo = O.logpsi(spec, th, sp)
    re, im = torch_logpsi(spec, torch.tensor(th), sp)
    np.testing.assert_allclose(lo.real, re.numpy(), rtol=0, atol=1e-12)
    np.testing.assert_allclose(lo.imag, im.numpy(), rtol=0, atol=1e-12)


@pytest.mark.parametrize("spec", CASES, ids=str)
def test_normalisation_by_enumeration(spec):
    """sum_sigma |Psi|^2 = 1 (softmax conditionals, Sec. II.A), within the
    S^z = 0 sector when masked; masked configurations outside it vanish."""
    th = init_theta(spec, 5)
    allc = all_configs(spec.N)
    lp = O.logpsi(spec, th, allc)
    P = np.exp(2 * lp.real)
    assert abs(P.sum() - 1.0) < 1e-12
    if spec.zmask:
        out = allc.sum(1) != spec.N // 2
        assert np.all(P[out] == 0.0)


def test_conditionals_product_is_probability():
    spec = ModelSpec(1, 7, 1, 3)
    th = init_theta(spec, 2)
    sp = np.array([0, 1, 1, 0, 1, 0, 0], dtype=np.uint8)
    p0 = O.conditionals(spec, th, sp)
    p = np.where(sp == 0, p0, 1 - p0)
    assert abs(np.prod(p) - np.exp(2 * O.logpsi(spec, th, sp[None])[0].real)) < 1e-14
