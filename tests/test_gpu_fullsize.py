"""Parity at the benchmark workloads' full sizes, in the launch configuration
the benchmark times (one nqs_minsr_step_ex from theta_0).

The oracle cannot redo a whole step at these sizes in seconds, so each stage
is checked where it can be computed independently:
  * samples: every decision sigma_k = [u >= p_k(0)] against the oracle's
    conditionals along the GPU's own configurations (near-ties |u - p| below
    the path's precision are excused);
  * log Psi of every sample; E_loc on a random subset of samples;
  * T against O'^T O' assembled from the oracle's Jacobian of all samples
    (centred per block, / sqrt(Ns)); eps-bar' from the GPU's own E_loc;
  * x by its backward error on (T_gpu + lambda I) x = eps'_gpu;
  * delta theta against eta_eff O'_oracle x_gpu.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2608_18065_b300 import nqs
from paper_2608_18065_b300.inputs import init_theta, workloads
from tests.gpu_helpers import RTOL64, TOL_MIXED_ELOC, TOL_MIXED_LOGPSI, cplx, rel_err

pytestmark = pytest.mark.gpu


def _check_decisions(model, th, spins, seed, step, tol, rows):
    bad = 0
    for s in rows:
        p0 = O.conditionals(model, th, spins[s])
        u = np.array([O.uniform(seed, step, int(s), k) for k in range(model.N)])
        dec = np.where(u < p0, 0, 1)
        bad += int(np.sum((dec != spins[s]) & (np.abs(u - p0) > tol)))
    return bad


def _centred_oracle_rows(model, th, spins):
    ns = len(spins)
    Oj = O.jacobian(model, th, spins)
    blocks = [Oj[:ns]] + ([Oj[ns:]] if model.cplx else [])
    return np.concatenate([(b - b.mean(0)) / np.sqrt(ns) for b in blocks], 0)


CASES = [("tfim100", "mixed"), ("tfim100", "fp64"), ("cluster64", "mixed"), ("heis10", "mixed")]


@pytest.mark.parametrize("key,prec", CASES, ids=[f"{k}-{p}" for k, p in CASES])
def test_full_size_step(key, prec):
    w = workloads()[key]
    model, ham, hp = w.model, w.ham, w.hp
    ns = hp.ns
    th = init_theta(model, w.theta_seed)
    c = nqs.Context(model, ham, prec, ns)
    thd = torch.tensor(th, device="cuda")
    md = torch.zeros_like(thd)
    outs = c.step_outputs(ns)
    stats = nqs.decode_stats(c.minsr_step(thd, md, hp, 0, outputs=outs))
    torch.cuda.synchronize()
    assert stats["status"] == 0, stats
    f64 = prec == "fp64"
    spins = outs["spins"].cpu().numpy()
    rng = np.random.default_rng(0)
    rows = rng.choice(ns, size=24, replace=False)
    # samples: all decisions of 24 random rows; for FP64 bit-exact over all rows
    if f64:
        sp_o, lp_o = O.sample(model, th, ns, hp.seed, 0)
        assert np.array_equal(spins, sp_o)
    else:
        assert _check_decisions(model, th, spins, hp.seed, 0, 1e-5, rows) == 0
    if model.zmask:
        assert np.all(spins.sum(1) == model.N // 2)
    # log Psi of every sample
    lp = cplx(outs["logpsi"])
    lp_o = O.logpsi(model, th, spins)
    if f64:
        np.testing.assert_allclose(lp, lp_o, rtol=RTOL64, atol=RTOL64)
    else:
        assert np.max(np.abs(lp - lp_o)) < TOL_MIXED_LOGPSI
    # E_loc on sampled rows
    el = cplx(outs["eloc"])
    el_o = O.local_energy(model, ham, th, spins[rows])
    assert rel_err(el[rows], el_o) < (RTOL64 if f64 else TOL_MIXED_ELOC)
    # T from the oracle's Jacobian of every sample
    A = _centred_oracle_rows(model, th, spins)
    T = outs["T"].cpu().numpy()
    T_o = A @ A.T
    scale = np.max(np.abs(T_o))
    assert np.array_equal(T, T.T)
    assert np.max(np.abs(T - T_o)) < (RTOL64 if f64 else 2e-4) * scale
    # eps-bar' from the GPU's local energies
    E = el.mean()
    ebar = np.conj(el - E) / np.sqrt(ns)
    eps = 2 * np.concatenate([ebar.real] + ([-ebar.imag] if model.cplx else []))
    np.testing.assert_allclose(outs["eps"].cpu().numpy(), eps, rtol=0, atol=1e-12 * np.max(np.abs(eps)))
    # x: backward error of the GPU's solve of its own system (FP64 level)
    lam = stats["lam"]
    Ts = T + lam * np.eye(len(eps))
    x = outs["x"].cpu().numpy()
    e_gpu = outs["eps"].cpu().numpy()
    berr = np.max(np.abs(Ts @ x - e_gpu)) / (np.max(np.abs(Ts).sum(1)) * np.max(np.abs(x)))
    assert berr < 100 * np.sqrt(len(x)) * 1.11e-16
    # delta theta = eta_eff O' x with the oracle's O'
    d_ref = stats["eta_eff"] * (A.T @ x)
    d = outs["dtheta"].cpu().numpy()
    assert rel_err(d, d_ref) < (1e-9 if f64 else 5e-4)
