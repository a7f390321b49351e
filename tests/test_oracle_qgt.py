"""The subsampled SR-metric error of Fig. 5b (Sec. III, Prop. 1): the
oracle's direct definition pinned by a closed form and by invariances, and
the Gram-block algebra bench.py uses against it."""
import numpy as np

import bench
from oracle import qgt


def _rows(rng, n, p, cplx):
    re = rng.standard_normal((n, p)) * np.linspace(0.5, 2.0, p)
    if not cplx:
        return re
    return np.concatenate([re, rng.standard_normal((n, p))], 0)


def test_one_parameter_closed_form():
    # N_p = 1: S is the sample variance (1/N sum |O - mean|^2)
    rng = np.random.default_rng(1)
    a, b = rng.standard_normal(40), rng.standard_normal(9) * 1.7
    va, vb = np.mean((a - a.mean()) ** 2), np.mean((b - b.mean()) ** 2)
    e = qgt.subsampled_error(a[:, None], 40, b[:, None], 9, False)
    assert abs(e - abs(va - vb) / va) < 1e-14


def test_invariances():
    rng = np.random.default_rng(2)
    for cplx in (False, True):
        Jr, Js = _rows(rng, 50, 7, cplx), _rows(rng, 12, 7, cplx)
        assert qgt.subsampled_error(Jr, 50, Jr, 50, cplx) == 0.0
        e = qgt.subsampled_error(Jr, 50, Js, 12, cplx)
        assert e > 0
        # every sample counted twice: same mean, same metric
        k = 2 if cplx else 1
        Jd = np.concatenate([np.repeat(Js[i * 12:(i + 1) * 12], 2, axis=0) for i in range(k)], 0)
        assert abs(qgt.subsampled_error(Jr, 50, Jd, 24, cplx) - e) < 1e-13
        # a common scale of all log-derivatives cancels
        assert abs(qgt.subsampled_error(3.0 * Jr, 50, 3.0 * Js, 12, cplx) - e) < 1e-13


def test_gram_route_equals_the_definition():
    rng = np.random.default_rng(3)
    for cplx in (False, True):
        nr, ns, p = 60, 15, 11
        Jr, Js = _rows(rng, nr, p, cplx), _rows(rng, ns, p, cplx)

        def cen(J, n):
            k = 2 if cplx else 1
            return [(J[i * n:(i + 1) * n] - J[i * n:(i + 1) * n].mean(0)) / np.sqrt(n) for i in range(k)]

        X = np.concatenate(cen(Jr, nr) + cen(Js, ns), 0)
        e_g = bench.qgt_error_from_gram(X @ X.T, nr, ns, cplx)
        e_o = qgt.subsampled_error(Jr, nr, Js, ns, cplx)
        assert abs(e_g - e_o) < 1e-12 * max(1.0, e_o)
