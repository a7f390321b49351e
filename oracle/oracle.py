"""ctypes front end of the FP64 CPU oracle (test infrastructure only).

Only tests, the package's smoke check and the benchmark's CPU-baseline leg
may import this module.  It builds the Hamiltonians of the paper as lists of
Pauli strings, written out from their definitions:
  TFIM (Sec. III.A):      H = -J sum_i Z_i Z_{i+1} - h sum_i X_i, open chain;
  cluster, ZXZ form:      H = -sum_{i=2}^{N-1} Z_{i-1} X_i Z_{i+1}, open chain;
  cluster, paper form (Sec. III.B):
        H = -sum_{k=2}^{N-2} X_{k-1} Z_k X_{k+1} - Z_1 X_2 - X_{N-1} X_N
            - X_{N-2} Z_{N-1} Z_N;
  J1-J2 (Sec. III.C):     H = J1/4 sum_<ij> (XX+YY+ZZ) + J2/4 sum_<<ij>> (...)
                          on an open Lx x Ly square lattice.
Sites of 2D lattices are addressed by their index k along the zig-zag path
pi(k) of Sec. II.B.
"""
import ctypes as C
import os

import numpy as np

from .build import build_oracle

_lib = None


class OrModel(C.Structure):
    _fields_ = [("dim", C.c_int), ("Lx", C.c_int), ("Ly", C.c_int),
                ("dh", C.c_int), ("cplx", C.c_int), ("marshall", C.c_int),
                ("zmask", C.c_int)]


class OrHam(C.Structure):
    _fields_ = [("n_terms", C.c_int), ("coeff", C.POINTER(C.c_double)),
                ("nops", C.POINTER(C.c_int)), ("site", C.POINTER(C.c_int)),
                ("op", C.c_char_p)]


class OrHParams(C.Structure):
    _fields_ = [("eta0", C.c_double), ("decay_T", C.c_double), ("mu", C.c_double),
                ("lam", C.c_double), ("lambda_coeff", C.c_double),
                ("lambda_pow", C.c_double), ("lambda_mode", C.c_int),
                ("trust_region", C.c_int), ("step_index", C.c_int64),
                ("seed", C.c_uint64), ("ns", C.c_int64), ("lm_omega", C.c_double)]


class OrStats(C.Structure):
    _fields_ = [("E_re", C.c_double), ("E_im", C.c_double), ("var", C.c_double),
                ("vscore", C.c_double), ("lam", C.c_double), ("normT", C.c_double),
                ("eta_eff", C.c_double), ("tau_norm", C.c_double),
                ("status", C.c_int), ("rho", C.c_double), ("lambda_next", C.c_double)]


class OrStepOut(C.Structure):
    _fields_ = [("spins", C.c_void_p), ("logpsi", C.c_void_p), ("eloc", C.c_void_p),
                ("T", C.c_void_p), ("eps", C.c_void_p), ("x", C.c_void_p),
                ("dtheta", C.c_void_p)]


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build_oracle())
        _lib.or_param_count.restype = C.c_int64
        _lib.or_uniform.restype = C.c_double
        _lib.or_uniform.argtypes = [C.c_uint64] * 4
        _lib.or_num_threads.restype = C.c_int
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def model_struct(spec) -> OrModel:
    return OrModel(spec.dim, spec.Lx, spec.Ly, spec.dh, spec.cplx,
                   spec.marshall, spec.zmask)


# ------------------------------------------------------------ Hamiltonians
class PauliSum:
    """Real combination of Pauli strings; each term = (coeff, [(site, op)])."""

    def __init__(self, N):
        self.N = N
        self.terms = []

    def add(self, coeff, ops):
        self.terms.append((float(coeff), list(ops)))

    def struct(self):
        n = len(self.terms)
        self._coeff = np.array([c for c, _ in self.terms], dtype=np.float64)
        self._nops = np.array([len(o) for _, o in self.terms], dtype=np.int32)
        self._site = np.zeros(4 * n, dtype=np.int32)
        ops = bytearray(b"I" * (4 * n))
        for t, (_, o) in enumerate(self.terms):
            assert len(o) <= 4
            for q, (k, p) in enumerate(o):
                self._site[4 * t + q] = k
                ops[4 * t + q] = ord(p)
        self._op = bytes(ops)
        return OrHam(n, self._coeff.ctypes.data_as(C.POINTER(C.c_double)),
                     self._nops.ctypes.data_as(C.POINTER(C.c_int)),
                     self._site.ctypes.data_as(C.POINTER(C.c_int)), self._op)


def path_coords(Lx, Ly):
    """pi(k) = (i_k, j_k) of the zig-zag path (Sec. II.B)."""
    out = []
    for k in range(Lx * Ly):
        j = k // Lx
        i = k % Lx if j % 2 == 0 else Lx - 1 - (k % Lx)
        out.append((i, j))
    return out


def hamiltonian(ham, spec) -> PauliSum:
    N = spec.N
    H = PauliSum(N)
    f = ham.family
    if f == "tfim":
        for i in range(N - 1):
            H.add(-ham.J, [(i, "Z"), (i + 1, "Z")])
        for i in range(N):
            H.add(-ham.h, [(i, "X")])
    elif f == "cluster_zxz":
        for i in range(1, N - 1):
            H.add(-1.0, [(i - 1, "Z"), (i, "X"), (i + 1, "Z")])
    elif f == "cluster_paper":
        # 1-indexed k = 2..N-2 acts on k-1, k, k+1 -> 0-indexed k-2, k-1, k
        for k in range(2, N - 1):
            H.add(-1.0, [(k - 2, "X"), (k - 1, "Z"), (k, "X")])
        H.add(-1.0, [(0, "Z"), (1, "X")])
        H.add(-1.0, [(N - 2, "X"), (N - 1, "X")])
        H.add(-1.0, [(N - 3, "X"), (N - 2, "Z"), (N - 1, "Z")])
    elif f == "j1j2":
        Lx, Ly = spec.Lx, spec.Ly
        index = {c: k for k, c in enumerate(path_coords(Lx, Ly))}
        bonds = []
        for (i, j), k in index.items():
            for di, dj, J in ((1, 0, ham.J1), (0, 1, ham.J1),
                              (1, 1, ham.J2), (1, -1, ham.J2)):
                q = index.get((i + di, j + dj))
                if q is not None and J != 0.0:
                    bonds.append((k, q, J))
        for k, q, J in bonds:
            for p in "XYZ":
                H.add(J / 4.0, [(k, p), (q, p)])
    else:
        raise ValueError(f)
    return H


# ------------------------------------------------------------- wrappers
def param_count(spec) -> int:
    m = model_struct(spec)
    return int(lib().or_param_count(C.byref(m)))


def uniform(seed, step, s, k) -> float:
    return float(lib().or_uniform(seed, step, s, k))


def philox(ctr, key):
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return list(o)


def logpsi(spec, theta, spins) -> np.ndarray:
    """log Psi per configuration as complex128."""
    m = model_struct(spec)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    sp = np.ascontiguousarray(spins, dtype=np.uint8).reshape(-1, spec.N)
    out = np.zeros((sp.shape[0], 2))
    rc = lib().or_logpsi(C.byref(m), _p(th), _p(sp), C.c_int64(sp.shape[0]), _p(out))
    assert rc == 0
    return out[:, 0] + 1j * out[:, 1]


def conditionals(spec, theta, spins) -> np.ndarray:
    m = model_struct(spec)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    sp = np.ascontiguousarray(spins, dtype=np.uint8).reshape(spec.N)
    out = np.zeros(spec.N)
    assert lib().or_conditionals(C.byref(m), _p(th), _p(sp), _p(out)) == 0
    return out


def sample(spec, theta, ns, seed, step, s0=0):
    """ns configurations drawn with the Philox counters of samples
    s0 .. s0 + ns - 1 (Sec. II.A inverse-CDF sampling)."""
    m = model_struct(spec)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    sp = np.zeros((ns, spec.N), dtype=np.uint8)
    lp = np.zeros((ns, 2))
    rc = lib().or_sample_range(C.byref(m), _p(th), C.c_int64(s0), C.c_int64(ns),
                               C.c_uint64(seed), C.c_uint64(step), _p(sp), _p(lp))
    assert rc == 0
    return sp, lp[:, 0] + 1j * lp[:, 1]


def local_energy(spec, hamspec, theta, spins) -> np.ndarray:
    m = model_struct(spec)
    H = hamiltonian(hamspec, spec)
    hs = H.struct()
    th = np.ascontiguousarray(theta, dtype=np.float64)
    sp = np.ascontiguousarray(spins, dtype=np.uint8).reshape(-1, spec.N)
    out = np.zeros((sp.shape[0], 2))
    rc = lib().or_local_energy(C.byref(m), C.byref(hs), _p(th), _p(sp),
                               C.c_int64(sp.shape[0]), _p(out))
    assert rc == 0
    return out[:, 0] + 1j * out[:, 1]


def jacobian(spec, theta, spins) -> np.ndarray:
    """Raw d log Psi / d theta, rows = samples (real rows, then imaginary
    rows for a complex head), no 1/sqrt(Ns)."""
    m = model_struct(spec)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    sp = np.ascontiguousarray(spins, dtype=np.uint8).reshape(-1, spec.N)
    ns = sp.shape[0]
    R = 2 * ns if spec.cplx else ns
    O = np.zeros((R, len(th)))
    rc = lib().or_jacobian(C.byref(m), _p(th), _p(sp), C.c_int64(ns), _p(O))
    assert rc == 0
    return O


def cholesky_solve(A, b):
    A = np.ascontiguousarray(A, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    rc = lib().or_cholesky_solve(_p(A), C.c_int64(len(b)), _p(b), _p(x))
    return rc, x


def hparams_struct(hp, step_index) -> OrHParams:
    return OrHParams(hp.eta0, hp.decay_T, hp.mu, hp.lam, hp.lambda_coeff,
                     hp.lambda_pow, hp.lambda_mode, hp.trust_region,
                     step_index, hp.seed, hp.ns, getattr(hp, "lm_omega", 0.0))


def minsr_step(spec, hamspec, theta, mom, hp, step_index, want=()):
    """One iteration of Algorithm 1.  Returns (theta', mom', stats dict,
    intermediates dict).  theta/mom arrays are not modified."""
    m = model_struct(spec)
    H = hamiltonian(hamspec, spec)
    hs = H.struct()
    th = np.array(theta, dtype=np.float64, copy=True)
    mo = np.array(mom, dtype=np.float64, copy=True)
    hps = hparams_struct(hp, step_index)
    st = OrStats()
    ns, np_ = hp.ns, len(th)
    R = 2 * ns if spec.cplx else ns
    bufs = {}
    shapes = dict(spins=((ns, spec.N), np.uint8), logpsi=((ns, 2), np.float64),
                  eloc=((ns, 2), np.float64), T=((R, R), np.float64),
                  eps=((R,), np.float64), x=((R,), np.float64),
                  dtheta=((np_,), np.float64))
    out = OrStepOut()
    for name in want:
        shp, dt = shapes[name]
        bufs[name] = np.zeros(shp, dtype=dt)
        setattr(out, name, bufs[name].ctypes.data)
    rc = lib().or_minsr_step(C.byref(m), C.byref(hs), _p(th), _p(mo), C.byref(hps),
                             C.byref(st), C.byref(out))
    assert rc == 0
    stats = {f: getattr(st, f) for f, _ in OrStats._fields_}
    for k in ("logpsi", "eloc"):
        if k in bufs:
            bufs[k] = bufs[k][:, 0] + 1j * bufs[k][:, 1]
    return th, mo, stats, bufs


def set_threads(n: int):
    lib().or_set_num_threads(int(n))


def num_threads() -> int:
    return int(lib().or_num_threads())
