"""Seeded synthetic inputs shared by the CUDA path, the tests and the bench.

This module holds no arithmetic of the method.  It fixes:
  * the model and Hamiltonian descriptions of the five benchmark workloads,
  * the initial parameters theta_0 ~ N(0, 1/fan_in) from a fixed seed,
  * the minSR hyper-parameters of Tab. I of the paper per workload family.

Parameter blocks follow the flat layout of the C-ABI (row-major, hidden-state
columns before one-hot columns):
  [U1 U2 (2D)] Wu bu Wr br Wh bh Win bin U c [Uphi cphi (complex head)].
fan_in of a matrix is its column count; a bias takes the fan_in of its matrix.
"""
from dataclasses import dataclass, field, asdict
from typing import List, Tuple

import numpy as np


@dataclass(frozen=True)
class ModelSpec:
    dim: int          # 1 or 2
    Lx: int
    Ly: int           # 1 in 1D
    dh: int
    cplx: int = 0     # softsign phase head (cRNN)
    marshall: int = 0 # Marshall sign (-1)^{sigma_A}
    zmask: int = 0    # zero-magnetisation masking

    @property
    def N(self) -> int:
        return self.Lx * self.Ly


@dataclass(frozen=True)
class HamSpec:
    family: str       # "tfim" | "cluster_zxz" | "cluster_paper" | "j1j2"
    J: float = 1.0
    h: float = 1.0
    J1: float = 1.0
    J2: float = 0.0


@dataclass
class HParams:
    eta0: float
    decay_T: float
    mu: float
    lam: float = 1e-3
    lambda_mode: int = 0          # 0: constant, 1: coeff*||T||_F^pow
    lambda_coeff: float = 0.0
    lambda_pow: float = 0.0
    trust_region: int = 0
    seed: int = 42
    ns: int = 128
    lm_omega: float = 0.0         # > 1: Levenberg-Marquardt damping factor (App. G)


def param_blocks(spec: ModelSpec) -> List[Tuple[str, int, int, int]]:
    """(name, rows, cols, fan_in) of every parameter block in layout order."""
    dh = spec.dh
    din = 4 if spec.dim == 2 else 2
    b = []
    if spec.dim == 2:
        b += [("U1", dh, dh, dh), ("U2", dh, dh, dh)]
    b += [("Wu", dh, dh + din, dh + din), ("bu", dh, 1, dh + din),
          ("Wr", dh, dh + din, dh + din), ("br", dh, 1, dh + din),
          ("Wh", dh, dh, dh), ("bh", dh, 1, dh),
          ("Win", dh, din, din), ("bin", dh, 1, din),
          ("U", 2, dh, dh), ("c", 2, 1, dh)]
    if spec.cplx:
        b += [("Uphi", 2, dh, dh), ("cphi", 2, 1, dh)]
    return b


def param_count(spec: ModelSpec) -> int:
    return sum(r * c for _, r, c, _ in param_blocks(spec))


def init_theta(spec: ModelSpec, seed: int = 1234) -> np.ndarray:
    """theta_0: every entry N(0, 1/fan_in), one PCG64 stream per seed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for _, r, c, fan in param_blocks(spec):
        parts.append(rng.standard_normal(r * c) / np.sqrt(fan))
    return np.concatenate(parts).astype(np.float64)


def random_spins(spec: ModelSpec, n: int, seed: int = 7,
                 zero_mag: bool = False) -> np.ndarray:
    """n configurations in path order, uint8 {0,1}; optionally S^z = 0."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if not zero_mag:
        return rng.integers(0, 2, size=(n, spec.N), dtype=np.uint8)
    out = np.zeros((n, spec.N), dtype=np.uint8)
    for s in range(n):
        out[s, rng.permutation(spec.N)[: spec.N // 2]] = 1
    return out


# ---------------------------------------------------------------- workloads
# Tab. I of the paper: (eta0, mu, lambda, decay time) per model column.
TAB1 = {
    "tfim": dict(eta0=0.5, mu=0.7, lam=1e-3, decay_T=1e3),
    "cluster": dict(eta0=5e-3, mu=0.1, lam=1e-3, decay_T=5e3),
    "heisenberg": dict(eta0=6e-2, mu=0.75, lambda_mode=1, lambda_coeff=3e-4,
                       lambda_pow=2.0 / 3.0, decay_T=1e4),
    "j1j2": dict(eta0=0.1, mu=0.1, lam=0.1, decay_T=1e4, trust_region=1),
}


# Tab. I, Adam column: (eta0, decay time); T = inf keeps eta constant.  The
# moment decays and epsilon are not given in the paper: Kingma and Ba's.
TAB1_ADAM = {
    "tfim": dict(eta0=5e-3, decay_T=float("inf")),
    "cluster": dict(eta0=5e-4, decay_T=float("inf")),
    "heisenberg": dict(eta0=5e-4, decay_T=1e4),
    "j1j2": dict(eta0=3e-3, decay_T=5e3),
}


@dataclass
class AdamParams:
    eta0: float
    decay_T: float = float("inf")
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    seed: int = 42
    ns: int = 128


@dataclass
class Workload:
    name: str
    model: ModelSpec
    ham: HamSpec
    hp: HParams
    precision: str            # "fp64" | "mixed"
    theta_seed: int = 1234

    def describe(self) -> dict:
        d = dict(workload=self.name, **asdict(self.model), **asdict(self.ham))
        d.update(ns=self.hp.ns, precision=self.precision,
                 n_params=param_count(self.model))
        return d


def workloads() -> dict:
    """The synthetic benchmark workloads (1D TFIM small/large and at the
    paper's own size, 1D cluster, 2D Heisenberg), each with Tab. I
    hyper-parameters."""
    w = {}
    w["tfim16"] = Workload(
        "tfim_N16_dh16_ns128_fp64", ModelSpec(1, 16, 1, 16),
        HamSpec("tfim", J=1.0, h=1.0), HParams(ns=128, **TAB1["tfim"]), "fp64")
    w["tfim100"] = Workload(
        "tfim_N100_dh64_ns1024_mixed", ModelSpec(1, 100, 1, 64),
        HamSpec("tfim", J=1.0, h=1.0), HParams(ns=1024, **TAB1["tfim"]), "mixed")
    # the paper's own 1D TFIM configuration (Sec. III.A, Tab. I)
    w["tfim200"] = Workload(
        "tfim_N200_dh32_ns100_mixed", ModelSpec(1, 200, 1, 32),
        HamSpec("tfim", J=1.0, h=1.0), HParams(ns=100, **TAB1["tfim"]), "mixed")
    # the paper's cluster-state configuration (Sec. III.A: XZX form with its
    # boundary terms, E_0 = -N; Tab. I: d_h = 256, N_s = 100)
    w["cluster100p"] = Workload(
        "cluster_paper_N100_dh256_ns100_mixed", ModelSpec(1, 100, 1, 256, cplx=1),
        HamSpec("cluster_paper"), HParams(ns=100, **TAB1["cluster"]), "mixed")
    # the paper's 2D configurations (Sec. III.C, Tab. I: 10 x 10 open lattice,
    # d_h = 200, N_s = 200): the Heisenberg point with a positive RNN and the
    # Marshall sign, J2 = 0.5 with a complex RNN on the Marshall prior
    w["heis10p"] = Workload(
        "heisenberg_10x10_dh200_ns200_prnn_mixed",
        ModelSpec(2, 10, 10, 200, cplx=0, marshall=1, zmask=1),
        HamSpec("j1j2", J1=1.0, J2=0.0), HParams(ns=200, **TAB1["heisenberg"]), "mixed")
    w["j1j2_10p"] = Workload(
        "j1j2_10x10_J2_0.5_dh200_ns200_mixed",
        ModelSpec(2, 10, 10, 200, cplx=1, marshall=1, zmask=1),
        HamSpec("j1j2", J1=1.0, J2=0.5), HParams(ns=200, **TAB1["j1j2"]), "mixed")
    w["cluster64"] = Workload(
        "cluster_zxz_N64_dh64_ns512_mixed", ModelSpec(1, 64, 1, 64, cplx=1),
        HamSpec("cluster_zxz"), HParams(ns=512, **TAB1["cluster"]), "mixed")
    w["heis10"] = Workload(
        "heisenberg_10x10_dh64_ns2048_mixed",
        ModelSpec(2, 10, 10, 64, cplx=1, marshall=1, zmask=1),
        HamSpec("j1j2", J1=1.0, J2=0.0), HParams(ns=2048, **TAB1["heisenberg"]),
        "mixed")
    return w


def batched_instances(n: int = 16, seed: int = 7) -> List[Workload]:
    """Heterogeneous J1-J2 instances: L in {6,8,10,12}, J2 in {0,.25,.5,.6},
    Ns in {256..4096}, dh in {32,64,96,128}; J2 = 0 uses the Heisenberg
    column of Tab. I, J2 > 0 the J1-J2 column."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n):
        L = int(rng.choice([6, 8, 10, 12]))
        J2 = float(rng.choice([0.0, 0.25, 0.5, 0.6]))
        ns = int(rng.choice([256, 512, 1024, 2048, 4096]))
        dh = int(rng.choice([32, 64, 96, 128]))
        fam = "heisenberg" if J2 == 0.0 else "j1j2"
        out.append(Workload(
            f"j1j2_L{L}_J2{J2}_dh{dh}_ns{ns}",
            ModelSpec(2, L, L, dh, cplx=1, marshall=1, zmask=1),
            HamSpec("j1j2", J1=1.0, J2=J2), HParams(ns=ns, **TAB1[fam]),
            "mixed", theta_seed=1000 + i))
    return out
