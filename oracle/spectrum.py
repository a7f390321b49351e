"""Spectrum diagnostics of the damped minSR system (App. E), FP64 on the CPU.

Test infrastructure only: tests, the package's smoke check and the
benchmark's CPU-baseline leg may import this module.  Nothing here is
shared with the CUDA path.

App. E bounds the attainable accuracy of the damped solve by the condition
number of S_lambda = S + lambda I:
    kappa_2(S_lambda) = (lambda_max(S) + lambda) / (lambda_min(S) + lambda),
and the sample-space matrix T = O'^T O' has the same nonzero eigenvalues as
S, so the same quantities follow from T.  A rule-of-thumb count of reliable
decimal digits in a precision with machine epsilon eps is
    d = -log10(kappa_2 * eps).
The definitions are written out directly: the eigenvalues come from a dense
symmetric eigensolver (numpy.linalg.eigvalsh, a library primitive).
"""
import numpy as np

# machine epsilon (spacing of 1.0 and the next number) of FP32 and FP64; the
# passage quotes about 1e-7 for single precision
EPS_FP32 = 2.0 ** -23
EPS_FP64 = 2.0 ** -52


def eigenvalues(T):
    """All eigenvalues of the symmetric matrix T, ascending."""
    T = np.asarray(T, dtype=np.float64)
    return np.linalg.eigvalsh(0.5 * (T + T.T))


def condition_number(lam_max, lam_min, lam):
    """kappa_2(T + lambda I) for a positive semi-definite T (App. E)."""
    return (lam_max + lam) / (lam_min + lam)


def digits(kappa, eps):
    """Reliable decimal digits -log10(kappa * eps) (App. E)."""
    return -np.log10(kappa * eps)


def spectrum(T, lam):
    """lambda_max, lambda_min, kappa_2 of T + lambda I and the digits in FP32
    and FP64, as a dict."""
    w = eigenvalues(T)
    lmax, lmin = float(w[-1]), float(w[0])
    k = condition_number(lmax, lmin, lam)
    return {"lambda_max": lmax, "lambda_min": lmin, "kappa": k,
            "digits_fp32": float(digits(k, EPS_FP32)),
            "digits_fp64": float(digits(k, EPS_FP64))}
