"""Spectrum diagnostics (App. E) on the GPU against the oracle.

nqs_spectrum runs Lanczos with full reorthogonalisation in FP64; its top
Ritz value is compared with the oracle's dense eigensolver, kappa and the
digit counts with the oracle's formulas (App. E).  Matrices: a rotated
diagonal with a known spectrum (ragged size), the centred Gram matrix of a
real FP64 minSR step (lambda_min = 0 by centring), a rank-one matrix (the
Krylov space becomes invariant after two steps), a 1 x 1 matrix and a
matrix smaller than the step count (the Krylov space is the whole space, so
both ends are exact).
"""
import numpy as np
import pytest
import torch

from oracle import spectrum as S
from paper_2608_18065_b300 import nqs
from paper_2608_18065_b300.inputs import HamSpec, HParams, ModelSpec
from tests.gpu_helpers import ctx, theta_dev

pytestmark = pytest.mark.gpu

# Lanczos converges to the top eigenvalue to rounding when it is separated;
# 1e-10 relative leaves room for the FP64 sums over R terms
TOL = 1e-10


def _dev(A):
    return torch.tensor(np.ascontiguousarray(A), dtype=torch.float64, device="cuda")


def _rotated(d, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((len(d), len(d))))
    return (Q * d) @ Q.T


def test_known_spectrum_ragged_size():
    R = 300
    rng = np.random.default_rng(11)
    d = np.sort(rng.uniform(0.0, 1.0, R))
    d[-1], d[-2] = 50.0, 20.0            # separated top of the spectrum
    A = _rotated(d, 5)
    lam = 1e-3
    st = nqs.spectrum(_dev(A), lam, m=64, seed=3)
    o = S.spectrum(A, lam)
    assert st["status"] == 0 and st["iterations"] == 64
    assert st["lambda_max"] == pytest.approx(o["lambda_max"], rel=TOL)
    assert st["residual"] < 1e-8 * o["lambda_max"]
    # kappa of the centred Gram form: (lambda_max + lam) / lam
    assert st["kappa"] == pytest.approx((o["lambda_max"] + lam) / lam, rel=TOL)
    assert st["digits_fp32"] == pytest.approx(S.digits(st["kappa"], S.EPS_FP32), abs=1e-12)
    assert st["digits_fp64"] == pytest.approx(S.digits(st["kappa"], S.EPS_FP64), abs=1e-12)
    # the smallest Ritz value bounds lambda_min from above
    assert st["lambda_min_ritz"] >= o["lambda_min"] - TOL * o["lambda_max"]
    # deterministic: a second call gives the same bits
    st2 = nqs.spectrum(_dev(A), lam, m=64, seed=3)
    assert st2 == st


def test_gram_of_a_step():
    model, ham = ModelSpec(1, 12, 1, 16), HamSpec("tfim")
    hp = HParams(0.5, 1e3, 0.7, lam=1e-3, ns=96)
    c = ctx(model, ham, "fp64", hp.ns)
    _, thd = theta_dev(model, 21)
    outs = c.step_outputs(hp.ns)
    c.minsr_step(thd, torch.zeros_like(thd), hp, 0, outputs=outs)
    torch.cuda.synchronize()
    T = outs["T"].cpu().numpy()
    o = S.spectrum(T, hp.lam)
    # centring puts the all-ones vector into the null space (App. E)
    assert abs(o["lambda_min"]) < 1e-10 * o["lambda_max"]
    st = nqs.spectrum(outs["T"], hp.lam, m=96)
    assert st["status"] == 0
    assert st["lambda_max"] == pytest.approx(o["lambda_max"], rel=TOL)
    assert st["kappa"] == pytest.approx(o["kappa"], rel=1e-8)
    # m = R: the Krylov space is the whole space, both ends are exact
    assert abs(st["lambda_min_ritz"] - o["lambda_min"]) < 1e-9 * o["lambda_max"]


def test_rank_one_invariant_after_two_steps():
    u = np.linspace(-1.0, 2.0, 100)
    st = nqs.spectrum(_dev(np.outer(u, u)), 0.25, m=32)
    assert st["status"] == 0 and st["iterations"] == 2
    assert st["lambda_max"] == pytest.approx(float(u @ u), rel=TOL)
    assert abs(st["lambda_min_ritz"]) < 1e-12 * float(u @ u)


def test_small_sizes():
    st = nqs.spectrum(_dev(np.array([[5.0]])), 1.0, m=8)
    assert st["iterations"] == 1 and st["lambda_max"] == pytest.approx(5.0, rel=1e-15)
    assert st["kappa"] == pytest.approx(6.0, rel=1e-15)
    d = np.array([3.0, 1e-4, 0.5, 9.0, 2.0, 7.0, 0.0, 4.0])
    A = _rotated(d, 2)
    st = nqs.spectrum(_dev(A), 0.1, m=64)
    assert st["iterations"] <= 8
    assert st["lambda_max"] == pytest.approx(9.0, rel=TOL)
    assert abs(st["lambda_min_ritz"]) < 1e-12 * 9.0


def test_nonfinite_and_arguments():
    A = np.eye(40)
    A[3, 7] = A[7, 3] = np.nan
    st = nqs.spectrum(_dev(A), 0.1, m=8)
    assert st["status"] == 4  # NQS_ERR_NONFINITE
    with pytest.raises(nqs.NqsError):
        nqs.spectrum(_dev(np.eye(4)), -1.0)
    with pytest.raises(nqs.NqsError):
        nqs.spectrum(_dev(np.eye(4)), 0.1, m=0)


def test_subsampled_sr_metric_error_matches_oracle():
    """Fig. 5b: ||S - S~||_F / ||S||_F from the library's Jacobian rows and
    one FP64 Gram of the stacked centred rows (bench.py) against the oracle's
    explicit N_p x N_p metrics built from the oracle's Jacobian."""
    import bench
    from oracle import oracle as O
    from oracle import qgt
    from paper_2608_18065_b300.inputs import random_spins
    model, ham = ModelSpec(2, 3, 3, 8, cplx=1, marshall=1), HamSpec("j1j2", J2=0.5)
    n_ref, subs = 200, [20, 60]
    c = ctx(model, ham, "fp64", n_ref)
    th, thd = theta_dev(model, 3)
    sp_ref = random_spins(model, n_ref, seed=1)
    sp_sub = random_spins(model, max(subs), seed=2)
    dev = thd.device
    errs = bench.qgt_subsample_errors(c, thd, torch.tensor(sp_ref, device=dev),
                                      [torch.tensor(sp_sub[:n], device=dev) for n in subs])
    J_ref = O.jacobian(model, th, sp_ref)
    for n, e in zip(subs, errs):
        e_o = qgt.subsampled_error(J_ref, n_ref, O.jacobian(model, th, sp_sub[:n]), n, True)
        assert e_o > 0
        assert abs(e - e_o) < 1e-9 * e_o
