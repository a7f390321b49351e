"""Shared helpers of the GPU parity tests: run the CUDA path through the
C-ABI binding and the oracle on the same seeded inputs."""
import json
import os

import numpy as np
import torch

from oracle import oracle as O
from paper_2608_18065_b300 import nqs
from paper_2608_18065_b300.inputs import init_theta

# Tolerances.
#  FP64 path: 1e-10 relative (the bound stated for the plain GPU path); the
#  kernels differ from the oracle only in summation order and libm ulps.
#  Mixed path: the recurrence runs in FP32 (unit roundoff u = 6e-8).  A
#  per-site error of a few u, accumulated over N <= 100 sites and amplified
#  by the recurrence Jacobian (O(1) for these initialisations), bounds the
#  error of log Psi at ~N * 10 u ~ 6e-5 absolute; local energies inherit it
#  through exp(log Psi' - log Psi) -> 1e-4 relative; O is a sum over N sites
#  of FP32 products -> 1e-4 relative in norm.
RTOL64 = 1e-10
TOL_MIXED_LOGPSI = 1e-4
#  At the benchmark lattices (N up to 144, |log Psi| up to ~70) the FP32 sum
#  of N per-site terms carries an error proportional to its magnitude:
#  |Delta log Psi| <= 1e-4 + 1e-5 |log Psi| (1e-5 ~ 80 u) per sample.
TOL_MIXED_LOGPSI_REL = 1e-5
TOL_MIXED_ELOC = 2e-4
TOL_MIXED_JAC = 2e-4


def ctx(model, ham, precision, max_samples):
    return nqs.Context(model, ham, precision, max_samples)


def theta_dev(model, seed=1234, scale=1.0):
    th = init_theta(model, seed) * scale
    return th, torch.tensor(th, dtype=torch.float64, device="cuda")


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def cplx(t):
    a = t.detach().cpu().numpy()
    return a[..., 0] + 1j * a[..., 1]


def near_ties(model, theta, spins, seed, step, tol):
    """Sites where |u - p_k(0)| < tol along each oracle configuration."""
    out = 0
    for s in range(spins.shape[0]):
        p0 = O.conditionals(model, theta, spins[s])
        u = np.array([O.uniform(seed, step, s, k) for k in range(model.N)])
        out += int(np.sum(np.abs(u - p0) < tol))
    return out


def max_elem_err(a, b):
    """Largest element-wise error, relative to the largest |b| (one sample
    or entry off by the tolerance fails, unlike a vector-norm bound)."""
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1e-300))


def max_row_err(a, b):
    """Largest element-wise error, each row relative to its own largest |b|."""
    a = np.asarray(a)
    b = np.asarray(b)
    scale = np.maximum(np.max(np.abs(b), axis=1, keepdims=True), 1e-300)
    return float(np.max(np.abs(a - b) / scale))


def record_error(case, **errors):
    """Append measured errors of the mixed path against the oracle to the
    JSON-lines file named by NQS_ERRORS_OUT (nothing when unset)."""
    path = os.environ.get("NQS_ERRORS_OUT")
    if not path:
        return
    with open(path, "a") as f:
        f.write(json.dumps({"case": case, **{k: float(v) for k, v in errors.items()}}) + "\n")


#  Mixed 2D models of hidden size 96 / 128 (rows of at most 16 sites) draw
#  their samples on the streamed tensor-core engine, whose gate products take
#  BF16 hi/lo splits of both operands (hi.hi + lo.hi + hi.lo): each product
#  term carries a relative error up to 3 * 2^-18 (two split residuals of
#  2^-18 and the dropped lo.lo term), about 2^-16.4, against FP32's 2^-24.
#  A state error of that order enters every site's logits; the sites'
#  log-probabilities add up to |Delta log Psi| <= 1e-4 + 2^-14 N, a per-site
#  budget of four such units (weights up to 1.5 times the initialisation
#  scale, whose row sums of |W h| stay below a few units).
TOL_TC_LOGPSI_SITE = 2.0 ** -14


def tc_sampled(model, precision):
    """Whether the context draws its samples on the streamed engine."""
    return (precision == "mixed" and model.dim == 2 and model.dh in (96, 128)
            and 2 * model.Lx - 1 <= 31)


def logpsi_err_tc(lp, lp_o, N):
    """Largest per-sample |Delta log Psi| in units of the tensor-core
    sampler's bound 1e-4 + 2^-14 N (<= 1 passes)."""
    return float(np.max(np.abs(lp - lp_o)) / (TOL_MIXED_LOGPSI + TOL_TC_LOGPSI_SITE * N))


def logpsi_err(lp, lp_o):
    """Largest per-sample |Delta log Psi| in units of the mixed path's bound
    1e-4 + 1e-5 |log Psi| (<= 1 passes)."""
    return float(np.max(np.abs(lp - lp_o) / (TOL_MIXED_LOGPSI + TOL_MIXED_LOGPSI_REL * np.abs(lp_o))))
