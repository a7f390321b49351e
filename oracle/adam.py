"""The Adam comparator and the loss-landscape energies, FP64 on the CPU.

Test infrastructure only: tests, the package's smoke check and the
benchmark's CPU-baseline leg may import this module.  Nothing here is
shared with the CUDA path.

Adam (the first-order baseline of Sec. II.C, Tab. I's Adam column) moves
theta along the sampled energy gradient with Kingma and Ba's moment
estimates.  The gradient of E = <H> over the variational parameters is
    g_k = 2 Re (1/Ns) sum_s (O_k(sigma_s) - mean O_k)^* (E_loc(sigma_s) - E),
which in the real representation of the minSR step (Eq. real-valued:
centred rows Obar' stacked as real then imaginary parts, / sqrt(Ns), and
eps-bar' = 2 (Re eps-bar; -Im eps-bar), eps-bar_s = (E_loc - E)^* / sqrt(Ns))
is exactly Obar'^T eps-bar'.  The moments (defaults of Kingma and Ba, the
paper gives no other values: beta1 = 0.9, beta2 = 0.999, epsilon = 1e-8):
    m <- beta1 m + (1 - beta1) g,   v <- beta2 v + (1 - beta2) g^2,
    theta <- theta - eta_t (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + epsilon),
t = 1, 2, ... the iteration, eta_t = eta0 / (1 + (t - 1) / T) (Tab. I's decay).

Loss landscape (Sec. IV): E(theta + x v1 + y v2) estimated from Ns samples
per point; every point draws with the same Philox counters (step 0), so the
points share their random numbers.
"""
import numpy as np

from . import oracle as O


def centred_rows_eps(spec, hamspec, theta, ns, seed, step):
    """(E, Obar' [R x Np], eps-bar' [R]) of one draw, as in the minSR step."""
    sp, _ = O.sample(spec, theta, ns, seed, step)
    el = O.local_energy(spec, hamspec, theta, sp)
    J = O.jacobian(spec, theta, sp)
    E = el.mean()
    nb = 2 if spec.cplx else 1
    A = np.concatenate([(J[b * ns:(b + 1) * ns] - J[b * ns:(b + 1) * ns].mean(0)) / np.sqrt(ns)
                        for b in range(nb)])
    ebar = np.conj(el - E) / np.sqrt(ns)
    eps = 2 * np.concatenate([ebar.real] + ([-ebar.imag] if spec.cplx else []))
    return E, A, eps


def gradient(spec, hamspec, theta, ns, seed, step):
    """(E, g) with g = Obar'^T eps-bar' (the sampled energy gradient)."""
    E, A, eps = centred_rows_eps(spec, hamspec, theta, ns, seed, step)
    return E, A.T @ eps


def adam_step(spec, hamspec, theta, m, v, ap, step_index):
    """One Adam iteration; step_index t = 0, 1, ... (bias corrections use
    t + 1).  ap: eta0, decay_T, beta1, beta2, eps, seed, ns.  Returns
    (theta', m', v', E, g)."""
    E, g = gradient(spec, hamspec, theta, ap.ns, ap.seed, step_index)
    t = step_index + 1
    m = ap.beta1 * m + (1.0 - ap.beta1) * g
    v = ap.beta2 * v + (1.0 - ap.beta2) * g * g
    mh = m / (1.0 - ap.beta1 ** t)
    vh = v / (1.0 - ap.beta2 ** t)
    eta = ap.eta0 if not np.isfinite(ap.decay_T) or ap.decay_T <= 0 else \
        ap.eta0 / (1.0 + step_index / ap.decay_T)
    return theta - eta * mh / (np.sqrt(vh) + ap.eps), m, v, E, g


def landscape(spec, hamspec, theta, v1, v2, xs, ys, ns, seed):
    """E(theta + x v1 + y v2) for every (x, y) of the lists (complex mean of
    the local energies), samples drawn at Philox step 0 for every point."""
    out = np.zeros(len(xs), dtype=np.complex128)
    for i, (x, y) in enumerate(zip(xs, ys)):
        th = theta + x * v1 + y * v2
        sp, _ = O.sample(spec, th, ns, seed, 0)
        out[i] = O.local_energy(spec, hamspec, th, sp).mean()
    return out
