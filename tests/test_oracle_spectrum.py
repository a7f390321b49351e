"""Pins of the spectrum oracle (App. E) against closed forms.

Each case fixes the answer independently of the eigensolver: a rank-one
Gram matrix, a diagonal matrix, a rotated diagonal, the null vectors that
centring puts into T, and the condition-number / digit formulas themselves
at values worked by hand.
"""
import numpy as np
import pytest

from oracle import spectrum as S


def test_rank_one_gram():
    # T = v v^T: lambda_max = |v|^2, every other eigenvalue 0, so
    # kappa = 1 + |v|^2 / lambda
    v = np.array([3.0, -4.0, 12.0])  # |v|^2 = 169
    d = S.spectrum(np.outer(v, v), 0.5)
    assert d["lambda_max"] == pytest.approx(169.0, rel=1e-14)
    assert abs(d["lambda_min"]) < 1e-12
    assert d["kappa"] == pytest.approx(1.0 + 169.0 / 0.5, rel=1e-12)


def test_diagonal_and_rotated():
    diag = np.array([5.0, 1e-3, 2.5, 7.25, 0.0])
    d = S.spectrum(np.diag(diag), 1e-2)
    assert d["lambda_max"] == 7.25 and d["lambda_min"] == 0.0
    assert d["kappa"] == pytest.approx((7.25 + 1e-2) / 1e-2, rel=1e-15)
    # an orthogonal change of basis keeps the spectrum
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((5, 5)))
    d2 = S.spectrum(Q @ np.diag(diag) @ Q.T, 1e-2)
    assert d2["lambda_max"] == pytest.approx(7.25, rel=1e-13)
    assert abs(d2["lambda_min"]) < 1e-13


def test_centred_gram_is_singular():
    # the columns of O are centred over the samples, so T = Obar^T Obar has
    # the all-ones vector in its null space and lambda_min(T) = 0 (App. E)
    rng = np.random.default_rng(7)
    O = rng.standard_normal((40, 12))          # 12 samples, 40 parameters
    Ob = O - O.mean(axis=1, keepdims=True)
    T = Ob.T @ Ob
    w = S.eigenvalues(T)
    assert abs(w[0]) < 1e-12 * w[-1]
    assert np.linalg.norm(T @ np.ones(12)) < 1e-12 * w[-1]
    lam = 1e-3
    d = S.spectrum(T, lam)
    assert d["kappa"] == pytest.approx(1.0 + w[-1] / lam, rel=1e-9)


def test_digits_worked_values():
    # kappa = 1e3 in FP64 (eps 2.22e-16): 12.65 digits; in FP32 (eps 1.19e-7): 3.92
    assert S.digits(1e3, S.EPS_FP64) == pytest.approx(-np.log10(1e3 * 2.0 ** -52), rel=1e-15)
    assert S.digits(1e3, S.EPS_FP64) == pytest.approx(12.6536, abs=1e-4)
    assert S.digits(1e3, S.EPS_FP32) == pytest.approx(3.9237, abs=1e-4)
    # one decade less damping costs one digit when lambda << lambda_max
    k1 = S.condition_number(100.0, 0.0, 1e-4)
    k2 = S.condition_number(100.0, 0.0, 1e-5)
    assert S.digits(k1, S.EPS_FP32) - S.digits(k2, S.EPS_FP32) == pytest.approx(1.0, abs=1e-5)
