"""Pins of the oracle's exact autoregressive sampler (Sec. II.A)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2608_18065_b300.inputs import ModelSpec, init_theta
from tests.exact import all_configs


def test_sampler_decisions_follow_shared_uniforms():
    """sigma_k = 0 iff u(seed, step, s, k) < p_k(0), site by site, and the
    returned log Psi equals log Psi of the returned configuration."""
    spec = ModelSpec(2, 3, 4, 4, cplx=1, marshall=1, zmask=1)
    th = init_theta(spec, 4)
    sp, lp = O.sample(spec, th, 20, seed=42, step=3)
    np.testing.assert_allclose(lp, O.logpsi(spec, th, sp), rtol=0, atol=1e-13)
    for s in range(20):
        p0 = O.conditionals(spec, th, sp[s])
        u = np.array([O.uniform(42, 3, s, k) for k in range(spec.N)])
        assert np.array_equal(sp[s], np.where(u < p0, 0, 1).astype(np.uint8))
    assert np.all(sp.sum(1) == spec.N // 2)


@pytest.mark.parametrize("spec", [ModelSpec(1, 6, 1, 3), ModelSpec(2, 2, 3, 3, zmask=1)],
                         ids=str)
def test_sampler_chi_square(spec):
    """Empirical frequencies of 40000 samples against exact P(sigma)."""
    th = init_theta(spec, 8) * 2.0
    n = 40000
    sp, _ = O.sample(spec, th, n, seed=123, step=0)
    idx = sp.astype(np.int64) @ (1 << np.arange(spec.N)[::-1])
    counts = np.bincount(idx, minlength=2 ** spec.N)
    P = np.exp(2 * O.logpsi(spec, th, all_configs(spec.N)).real)
    m = P > 0
    assert counts[~m].sum() == 0
    exp_ = n * P[m]
    chi2 = np.sum((counts[m] - exp_) ** 2 / exp_)
    dof = m.sum() - 1
    # 5-sigma bound on a chi-square with dof degrees of freedom
    assert chi2 < dof + 5 * np.sqrt(2 * dof)
