"""Error of the subsampled SR metric (Sec. III, Prop. 1, Fig. 5b), FP64 on the CPU.

Test infrastructure only: tests, the package's smoke check and the
benchmark's CPU-baseline leg may import this module.  Nothing here is
shared with the CUDA path.

The SR metric (the quantum geometric tensor) estimated from N samples is
    S = Obar^dagger Obar,   Obar_s,i = (O_i(sigma_s) - mean_s O_i) / sqrt(N),
with the sample-mean centring the paper uses in its simulations (App. of
the proof of Prop. 1).  Fig. 5b plots ||S - S~||_F / ||S||_F for a
subsampled estimate S~ (N_s samples) against a high-sample reference S,
versus alpha = sqrt(N_s) / N_p.  Here both matrices are formed explicitly
(N_p x N_p, complex for the complex head) and the Frobenius norms are taken
directly.

Jacobian rows follow the layout of the step (R13): a real head gives N rows
O_s; the complex head gives 2N rows, the real parts of O_s then the
imaginary parts.
"""
import numpy as np


def centred(J, n, cplx):
    """Obar (n x N_p, complex when cplx) from Jacobian rows J ([n or 2n][N_p])."""
    J = np.asarray(J, dtype=np.float64)
    O = J[:n] + 1j * J[n:2 * n] if cplx else J[:n].astype(np.complex128)
    return (O - O.mean(axis=0)) / np.sqrt(n)


def metric(J, n, cplx):
    """S = Obar^dagger Obar (N_p x N_p)."""
    Ob = centred(J, n, cplx)
    return Ob.conj().T @ Ob


def subsampled_error(J_ref, n_ref, J_sub, n_sub, cplx):
    """||S_ref - S_sub||_F / ||S_ref||_F (Fig. 5b)."""
    S = metric(J_ref, n_ref, cplx)
    St = metric(J_sub, n_sub, cplx)
    return float(np.linalg.norm(S - St) / np.linalg.norm(S))


def alpha(n_sub, n_params):
    """alpha = sqrt(N_s) / N_p, the abscissa of Fig. 5b (Eq. UB)."""
    return float(np.sqrt(n_sub) / n_params)
