"""Sampling (Sec. II.A) on the streamed tensor-core engine: mixed-precision
2D models of hidden size 96 and 128 with every state cached draw their
samples on the same engine as their local energies.

Each decision sigma_k = [u_k >= p_k(0)] is taken in FP32 from conditionals
formed with BF16x3 products; it must agree with the oracle's FP64 p_k(0)
along the drawn configuration except where u lies within 1e-5 of it.  log Psi
of the samples is held to the BF16x3 bound 1e-4 + 2^-14 N; the caches the
engine writes for the local energies and the reverse sweep are checked
through whole steps against the oracle.  Sample ranges (s0 > 0, as a shard of the sample-sharded
step draws them) and lattices too wide for the engine's spin ring (which
fall back to the recurrence kernels' sampler) are covered too.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2608_18065_b300 import nqs
from paper_2608_18065_b300.inputs import HamSpec, HParams, ModelSpec, TAB1, init_theta
from paper_2608_18065_b300.sharded import ShardBackend, partition
from tests.gpu_helpers import (TOL_MIXED_ELOC, cplx, ctx, logpsi_err, logpsi_err_tc,
                               max_elem_err, record_error, rel_err, tc_sampled, theta_dev)

pytestmark = pytest.mark.gpu

# several 128-sample tiles with a ragged tail; odd row lengths; real and
# complex heads; the mask and the Marshall sign; a row of 16 sites (the
# widest the engine's 32-site spin ring holds) and one of 17 (recurrence
# kernels' sampler)
MODELS = [
    (ModelSpec(2, 4, 4, 128, cplx=1, marshall=1, zmask=1), 300, 1.0),
    (ModelSpec(2, 5, 3, 96), 130, 1.5),
    (ModelSpec(2, 3, 4, 128, cplx=1), 200, 1.5),
    (ModelSpec(2, 4, 3, 96, cplx=1, marshall=1, zmask=1), 260, 1.0),
    (ModelSpec(2, 16, 2, 128, cplx=1, marshall=1, zmask=1), 140, 1.0),
    (ModelSpec(2, 17, 2, 96, cplx=1), 40, 1.0),
]
IDS = ["4x4_dh128_cmask", "5x3_dh96", "3x4_dh128_c", "4x3_dh96_cmask", "16x2_dh128_cmask",
       "17x2_dh96_c_fallback"]


def _check_decisions(model, th, sp, seed, step, s0=0):
    bad = ties = 0
    for s in range(sp.shape[0]):
        p0 = O.conditionals(model, th, sp[s])
        u = np.array([O.uniform(seed, step, s0 + s, k) for k in range(model.N)])
        dec = np.where(u < p0, 0, 1)
        near = np.abs(u - p0) <= 1e-5
        bad += int(np.sum((dec != sp[s]) & ~near))
        ties += int(np.sum(near))
    assert bad == 0
    return ties


@pytest.mark.parametrize("model,ns,scale", MODELS, ids=IDS)
def test_tc_sampler_decisions_and_logpsi(model, ns, scale):
    c = ctx(model, HamSpec("j1j2", J2=0.5), "mixed", ns)
    th, thd = theta_dev(model, 21, scale=scale)
    spins, lp = c.sample(thd, ns, seed=5, step=3)
    sp = spins.cpu().numpy()
    assert sp.shape == (ns, model.N) and set(np.unique(sp)) <= {0, 1}
    if model.zmask:
        assert np.all(sp.sum(1) == model.N // 2)
    _check_decisions(model, th, sp, 5, 3)
    lp_o = O.logpsi(model, th, sp)
    if tc_sampled(model, "mixed"):
        assert logpsi_err_tc(cplx(lp), lp_o, model.N) <= 1.0
    else:
        assert logpsi_err(cplx(lp), lp_o) <= 1.0
    record_error(f"tc_sampler_{model.Lx}x{model.Ly}_dh{model.dh}_scale{scale}",
                 logpsi_abs=np.max(np.abs(cplx(lp) - lp_o)),
                 logpsi_abs_per_site=np.max(np.abs(cplx(lp) - lp_o)) / model.N)
    # drawing again is deterministic (same counters, same samples)
    spins2, lp2 = c.sample(thd, ns, seed=5, step=3)
    assert torch.equal(spins2, spins) and torch.equal(lp2, lp)


STEP_CASES = [
    (ModelSpec(2, 4, 4, 128, cplx=1, marshall=1, zmask=1), HamSpec("j1j2", J2=0.5),
     HParams(ns=150, **TAB1["j1j2"])),
    (ModelSpec(2, 4, 3, 96, cplx=1, marshall=1, zmask=1), HamSpec("j1j2", J2=0.0),
     HParams(ns=140, **TAB1["heisenberg"])),
]


@pytest.mark.parametrize("model,ham,hp", STEP_CASES, ids=["j1j2_4x4_dh128", "heis_4x3_dh96"])
def test_tc_sampler_step_against_oracle(model, ham, hp):
    """One mixed step from the engine's samples and caches: the samples equal
    the oracle's (a draw with a near-tie is retried at the next step index),
    E within the mixed E_loc bound, T element by element within 2e-4 of its
    largest entry (the Jacobian rows come from the engine's gate and state
    caches), delta theta against eta_eff O'^T x with the oracle's O'."""
    c = ctx(model, ham, "mixed", hp.ns)
    th, thd = theta_dev(model, 1234)
    momd = torch.zeros_like(thd)
    for t in range(8):
        outs = c.step_outputs(hp.ns)
        stats = c.minsr_step(thd.clone(), momd.clone(), hp, t, outputs=outs)
        torch.cuda.synchronize()
        st = nqs.decode_stats(stats)
        _, _, st_o, b = O.minsr_step(model, ham, th, np.zeros_like(th), hp, t,
                                     want=("spins", "eloc", "T", "eps", "x", "dtheta"))
        if np.array_equal(outs["spins"].cpu().numpy(), b["spins"]):
            break
    else:
        pytest.fail("eight draws in a row changed a mixed-precision sample")
    assert st["status"] == 0
    assert abs(st["E_re"] - st_o["E_re"]) < TOL_MIXED_ELOC * abs(st_o["E_re"])
    el = cplx(outs["eloc"])
    assert max_elem_err(el, b["eloc"]) < TOL_MIXED_ELOC
    assert max_elem_err(outs["T"].cpu().numpy(), b["T"]) < 2e-4
    ns = hp.ns
    Oj = O.jacobian(model, th, b["spins"])
    blocks = [Oj[:ns]] + ([Oj[ns:]] if model.cplx else [])
    A = np.concatenate([(q - q.mean(0)) / np.sqrt(ns) for q in blocks], 0)
    d = outs["dtheta"].cpu().numpy()
    d_ref = st["eta_eff"] * (A.T @ outs["x"].cpu().numpy())
    assert rel_err(d, d_ref) < 5e-4


def test_tc_sampler_sample_ranges_in_sharded_step():
    """Two ranks drawing samples [0, 75) and [75, 150) (s0 = 75 on the
    second) on the engine give the single-context step: a rank that ignored
    s0 would draw the first rank's samples again."""
    model = ModelSpec(2, 4, 4, 128, cplx=1, marshall=1, zmask=1)
    ham = HamSpec("j1j2", J2=0.5)
    hp = HParams(ns=150, **TAB1["j1j2"])
    th0 = init_theta(model, 77)
    one = nqs.Context(model, ham, "mixed", hp.ns)
    tha = torch.tensor(th0, device="cuda")
    ma = torch.zeros_like(tha)
    sa = nqs.decode_stats(one.minsr_step(tha, ma, hp, 0))
    bes = [ShardBackend(nqs.Context(model, ham, "mixed", hp.ns)) for _ in range(2)]
    ths = [torch.tensor(th0, device="cuda") for _ in range(2)]
    mos = [torch.zeros_like(t) for t in ths]
    stats = [be.new_stats() for be in bes]
    parts = [partition(hp.ns, 2, r) for r in range(2)]
    assert parts[1][0] == 75
    sums = [be.forward(ths[r], hp, 0, *parts[r]) for r, be in enumerate(bes)]
    tot = torch.stack(sums).sum(0)
    cen = [be.center(tot, hp.ns, parts[r][1], stats[r]) for r, be in enumerate(bes)]
    nb = bes[0].blocks
    # rank order within each block of rows (real rows, then imaginary rows)
    rows = torch.cat([c[0] for c in cen], 0)
    eps = torch.cat([c[1] for c in cen], 0)
    assert rows.shape[0] == nb * hp.ns
    pp = [partition(bes[0].np, 2, r) for r in range(2)]
    dth = torch.cat([be.solve(rows, eps, hp, 0, p0, p0 + n, stats[r])
                     for r, (be, (p0, n)) in enumerate(zip(bes, pp))], 0)
    for r, be in enumerate(bes):
        be.apply(ths[r], mos[r], dth, hp, 0, stats[r])
    torch.cuda.synchronize()
    d = nqs.decode_stats(stats[0])
    assert d["status"] == 0 and sa["status"] == 0
    assert abs(d["E_re"] - sa["E_re"]) <= 2e-4 * abs(sa["E_re"])
    step_a = (tha - torch.tensor(th0, device="cuda")).cpu().numpy()
    step_b = (ths[0] - torch.tensor(th0, device="cuda")).cpu().numpy()
    assert rel_err(step_b, step_a) < 5e-4
    assert torch.equal(ths[0], ths[1])


def test_tc_and_recurrence_samplers_agree():
    """The two samplers of a mixed 2D d_h 128 context (nqs_set_sampler) draw
    the same configurations from the same uniforms: a row may differ only
    where the first differing site is a near-tie of the oracle's p_k(0), and
    log Psi of the common rows agrees within the tensor-core bound."""
    model = ModelSpec(2, 4, 4, 128, cplx=1, marshall=1, zmask=1)
    ns = 300
    c = ctx(model, HamSpec("j1j2", J2=0.5), "mixed", ns)
    th, thd = theta_dev(model, 31)
    c.set_sampler(1)
    s1, l1 = c.sample(thd, ns, seed=9, step=4)
    c.set_sampler(0)
    s0, l0 = c.sample(thd, ns, seed=9, step=4)
    c.set_sampler(-1)
    a, b = s1.cpu().numpy(), s0.cpu().numpy()
    same = np.all(a == b, axis=1)
    for s in np.where(~same)[0]:
        k = int(np.argmax(a[s] != b[s]))
        p0 = O.conditionals(model, th, a[s])[k]
        assert abs(O.uniform(9, 4, int(s), k) - p0) <= 1e-5
    assert np.sum(~same) <= 0.02 * ns
    d = np.abs(cplx(l1)[same] - cplx(l0)[same])
    assert np.max(d) <= 1e-4 + 2.0 ** -14 * model.N
