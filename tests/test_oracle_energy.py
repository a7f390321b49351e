"""Pins of the oracle's local energies (Sec. II.C) and Hamiltonians (Sec. III)
against exact diagonalisation, closed forms and the paper's printed values."""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2608_18065_b300.inputs import HamSpec, ModelSpec, init_theta
from tests.exact import (all_configs, dense_cluster_paper, dense_cluster_zxz,
                         dense_j1j2, dense_tfim, tfim_jw_energy)

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden():
    out = {}
    for l in open(os.path.join(GOLD, "reference_energies.txt")):
        if l.strip() and not l.startswith("#"):
            name, N, e, *_ = l.split()
            out[name] = (int(N), float(e))
    return out


def test_jw_closed_form_matches_paper_table():
    """The free-fermion closed form reproduces the TFIM E/N printed in
    Tab. II for N = 200 (J = h = 1, open chain)."""
    N, e = _golden()["tfim_obc_J1_h1"]
    assert abs(tfim_jw_energy(N) / N - e) < 1e-10


@pytest.mark.parametrize("N", [2, 5, 8, 10])
def test_tfim_ed_equals_jw(N):
    E0 = np.linalg.eigvalsh(dense_tfim(N))[0]
    assert abs(E0 - tfim_jw_energy(N)) < 1e-10


@pytest.mark.parametrize("N", [6, 8])
def test_cluster_ground_energies(N):
    assert abs(np.linalg.eigvalsh(dense_cluster_zxz(N))[0] + (N - 2)) < 1e-10
    assert abs(np.linalg.eigvalsh(dense_cluster_paper(N))[0] + N) < 1e-10


def test_heisenberg_small_exact_values():
    # two spins: singlet energy -3/4; 2x2 open plaquette: -2 (exact)
    assert abs(np.linalg.eigvalsh(dense_j1j2(2, 1))[0] + 0.75) < 1e-12
    assert abs(np.linalg.eigvalsh(dense_j1j2(2, 2))[0] + 2.0) < 1e-12


CASES = [
    (ModelSpec(1, 8, 1, 4), HamSpec("tfim", J=1.0, h=0.7), dense_tfim(8, 1.0, 0.7)),
    (ModelSpec(1, 8, 1, 4, cplx=1), HamSpec("cluster_zxz"), dense_cluster_zxz(8)),
    (ModelSpec(1, 7, 1, 3, cplx=1), HamSpec("cluster_paper"), dense_cluster_paper(7)),
    (ModelSpec(2, 3, 3, 3, cplx=1, marshall=1), HamSpec("j1j2", J1=1.0, J2=0.5),
     dense_j1j2(3, 3, 1.0, 0.5)),
    (ModelSpec(2, 4, 2, 3, cplx=1, marshall=1, zmask=1), HamSpec("j1j2", J1=1.0, J2=0.0),
     dense_j1j2(4, 2, 1.0, 0.0)),
]


@pytest.mark.parametrize("spec,ham,Hd", CASES, ids=lambda c: str(c)[:40])
def test_local_energy_equals_H_psi_over_psi(spec, ham, Hd):
    """eps(sigma) = (H Psi)(sigma) / Psi(sigma) for every configuration with
    Psi != 0, with H from Kronecker products; and sum P eps = <Psi|H|Psi>
    >= E_0 (variational bound)."""
    th = init_theta(spec, 9)
    allc = all_configs(spec.N)
    lp = O.logpsi(spec, th, allc)
    psi = np.exp(lp)
    keep = np.abs(psi) > 0
    el = O.local_energy(spec, ham, th, allc[keep])
    Hpsi = Hd @ psi
    np.testing.assert_allclose(el, Hpsi[keep] / psi[keep], rtol=1e-10, atol=1e-10)
    P = np.abs(psi) ** 2
    E = np.sum(P[keep] * el)
    assert abs(E - np.vdot(psi, Hpsi)) < 1e-10
    E0 = np.linalg.eigvalsh(Hd)[0]
    assert E.real >= E0 - 1e-10
