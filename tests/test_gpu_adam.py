"""nqs_adam_step and nqs_energy_scan (row f4: the Adam comparator of
Sec. II.C and the loss landscape of Sec. IV) against the oracle: FP64
chained Adam iterations and landscape energies to 1e-10 (same samples);
mixed: the gradient within the O and E_loc tolerances, the update where the
gradient is not near zero (Adam's update is g / |g|)."""
import numpy as np
import pytest
import torch

from oracle import adam as A
from paper_2608_18065_b300 import nqs
from paper_2608_18065_b300.inputs import (AdamParams, HamSpec, ModelSpec, TAB1_ADAM,
                                          init_theta)
from tests.gpu_helpers import RTOL64, TOL_MIXED_ELOC, max_elem_err, rel_err

pytestmark = pytest.mark.gpu

CASES = [
    (ModelSpec(1, 14, 1, 16), HamSpec("tfim"), AdamParams(ns=96, **TAB1_ADAM["tfim"])),
    (ModelSpec(2, 4, 4, 16, cplx=1, marshall=1, zmask=1), HamSpec("j1j2", J2=0.5),
     AdamParams(ns=70, **TAB1_ADAM["j1j2"])),
]
IDS = ["tfim14", "j1j2_4x4_c"]


@pytest.mark.parametrize("model,ham,ap", CASES, ids=IDS)
def test_adam_fp64_against_oracle(model, ham, ap):
    c = nqs.Context(model, ham, "fp64", ap.ns)
    th = init_theta(model, 21)
    m1, m2 = np.zeros_like(th), np.zeros_like(th)
    thd = torch.tensor(th, device="cuda")
    m1d, m2d = torch.zeros_like(thd), torch.zeros_like(thd)
    g = torch.empty_like(thd)
    for t in range(3):
        st = nqs.decode_stats(c.adam_step(thd, m1d, m2d, ap, t, grad=g))
        torch.cuda.synchronize()
        th, m1, m2, E, g_o = A.adam_step(model, ham, th, m1, m2, ap, t)
        assert st["status"] == 0
        assert abs(st["E_re"] - E.real) <= RTOL64 * abs(E.real)
        assert rel_err(g.cpu().numpy(), g_o) < RTOL64
        assert rel_err(thd.cpu().numpy(), th) < RTOL64
        assert rel_err(m1d.cpu().numpy(), m1) < RTOL64
        assert rel_err(m2d.cpu().numpy(), m2) < 1e-9


@pytest.mark.parametrize("model,ham,ap", CASES, ids=IDS)
def test_adam_mixed_against_oracle(model, ham, ap):
    c = nqs.Context(model, ham, "mixed", ap.ns)
    th = init_theta(model, 22)
    thd = torch.tensor(th, device="cuda")
    m1d, m2d = torch.zeros_like(thd), torch.zeros_like(thd)
    g = torch.empty_like(thd)
    st = nqs.decode_stats(c.adam_step(thd, m1d, m2d, ap, 0, grad=g))
    torch.cuda.synchronize()
    z = np.zeros_like(th)
    th1, _, _, E, g_o = A.adam_step(model, ham, th, z, z, ap, 0)
    assert st["status"] == 0
    assert abs(st["E_re"] - E.real) <= TOL_MIXED_ELOC * abs(E.real)
    gg = g.cpu().numpy()
    assert rel_err(gg, g_o) < 5e-4
    assert max_elem_err(gg, g_o) < 2e-3
    big = np.abs(g_o) > 1e-2 * np.max(np.abs(g_o))
    d = (thd.cpu().numpy() - th)[big]
    assert np.max(np.abs(d - (th1 - th)[big])) <= 1e-3 * ap.eta0


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("model,ham,ap", CASES, ids=IDS)
def test_energy_scan_against_oracle(model, ham, ap, prec):
    c = nqs.Context(model, ham, prec, ap.ns)
    th = init_theta(model, 23)
    rng = np.random.default_rng(5)
    v1 = rng.standard_normal(len(th)) * 0.1
    v2 = rng.standard_normal(len(th)) * 0.1
    xy = np.array([[0.0, 0.0], [0.5, -0.25], [-1.0, 0.75], [0.2, 0.2], [1.5, -1.5]])
    dev = lambda a: torch.tensor(a, device="cuda")
    out = c.energy_scan(dev(th), dev(v1), dev(v2), xy, ap.ns, 17).cpu().numpy()
    E_o = A.landscape(model, ham, th, v1, v2, xy[:, 0], xy[:, 1], ap.ns, 17)
    assert np.all(out[:, 3] == 0)
    tol = RTOL64 if prec == "fp64" else TOL_MIXED_ELOC
    np.testing.assert_allclose(out[:, 0], E_o.real, rtol=tol, atol=0)
