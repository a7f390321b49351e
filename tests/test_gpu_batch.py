"""Batched heterogeneous instances and the launch-shape autotuner.

A batched step must give every instance exactly what its own
nqs_minsr_step gives (same kernels, same data, only the streams differ), so
the comparisons are bitwise; the FP64 instances are also checked against the
oracle.  Tuned launch shapes change only how work is spread over CTAs: two
contexts with the same shapes agree bitwise, and against the built-in shapes
the regrouped sums (K-slices of T, substitution partials) differ by rounding.
"""
import copy

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2608_18065_b300 import nqs
from paper_2608_18065_b300.inputs import TAB1, HamSpec, HParams, ModelSpec, init_theta
from tests.gpu_helpers import RTOL64

pytestmark = pytest.mark.gpu

# (model, Hamiltonian, precision, Ns, Tab. I column): lattices, hidden sizes,
# couplings, precisions and ragged sample counts all differ.
INSTANCES = [
    (ModelSpec(2, 4, 4, 32, cplx=1, marshall=1, zmask=1), HamSpec("j1j2", J2=0.5), "mixed", 256, "j1j2"),
    (ModelSpec(1, 20, 1, 64), HamSpec("tfim"), "mixed", 300, "tfim"),
    (ModelSpec(2, 4, 4, 64, cplx=1, marshall=1, zmask=1), HamSpec("j1j2", J2=0.0), "mixed", 130, "heisenberg"),
    (ModelSpec(1, 12, 1, 16, cplx=1), HamSpec("cluster_zxz"), "fp64", 64, "cluster"),
    (ModelSpec(2, 6, 6, 96, cplx=1, marshall=1, zmask=1), HamSpec("j1j2", J2=0.25), "mixed", 200, "j1j2"),
    (ModelSpec(2, 4, 2, 128, cplx=1, marshall=1, zmask=1), HamSpec("j1j2", J2=0.6), "fp64", 48, "j1j2"),
]


def _hp(col, ns, seed):
    return HParams(ns=ns, seed=seed, **TAB1[col])


def _setup(instances=INSTANCES):
    ctxs, th, mo, hps = [], [], [], []
    for i, (m, h, prec, ns, col) in enumerate(instances):
        ctxs.append(nqs.Context(m, h, prec, ns))
        th.append(torch.tensor(init_theta(m, 1000 + i), device="cuda"))
        mo.append(torch.zeros_like(th[-1]))
        hps.append(_hp(col, ns, 42 + i))
    return ctxs, th, mo, hps


def _solo(instances, steps, tuned=False):
    """Every instance stepped alone (eager), from the same start; tuned: with
    the launch shapes the process-wide autotune cache holds for it."""
    ctxs, th, mo, hps = _setup(instances)
    stats = []
    for c, t, m, hp in zip(ctxs, th, mo, hps):
        if tuned:
            c.autotune(t, hp, 0)
        s = c.new_stats()
        for k in range(steps):
            c.minsr_step(t, m, hp, k, s)
        stats.append(s)
    torch.cuda.synchronize()
    return th, mo, stats


@pytest.mark.parametrize("graph,conc", [(True, 0), (False, 0), (True, 2), (False, 1)],
                         ids=["graph-all", "eager-all", "graph-2streams", "eager-serial"])
def test_batched_equals_solo(graph, conc):
    steps = 3
    th0, mo0, st0 = _solo(INSTANCES, steps)
    ctxs, th, mo, hps = _setup()
    b = nqs.Batch(ctxs)
    b.use_graph(graph)
    b.set_concurrency(conc)
    stats = b.new_stats()
    for k in range(steps):
        b.step(th, mo, hps, k, stats)
    torch.cuda.synchronize()
    assert b.graph_active() == graph
    for i in range(len(INSTANCES)):
        d = nqs.decode_stats(stats[i])
        assert d["status"] == 0, (i, d)
        assert torch.equal(th[i], th0[i]), i
        assert torch.equal(mo[i], mo0[i]), i
        assert torch.equal(stats[i], st0[i]), i
    b.close()


def test_batched_step_index_out_of_sequence():
    """Graph replays with per-instance step indices that jump: the device
    counters are reset before the replay, as for a single context."""
    sub = INSTANCES[:3]
    ctxs, th, mo, hps = _setup(sub)
    b = nqs.Batch(ctxs)
    b.use_graph(True)
    stats = b.new_stats()
    seq = [[0, 5, 9], [1, 6, 2], [7, 7, 3]]
    for s in seq:
        b.step(th, mo, hps, s, stats)
    torch.cuda.synchronize()
    th0, mo0, _ = _setup(sub)[1:]
    c0 = _setup(sub)[0]
    for i, c in enumerate(c0):
        st = c.new_stats()
        for s in seq:
            c.minsr_step(th0[i], mo0[i], hps[i], s[i], st)
    torch.cuda.synchronize()
    for i in range(len(sub)):
        assert torch.equal(th[i], th0[i]), i


def test_batched_fp64_against_oracle():
    inst = [INSTANCES[3], INSTANCES[5]]
    ctxs, th, mo, hps = _setup(inst)
    b = nqs.Batch(ctxs)
    b.use_graph(True)
    stats = b.new_stats()
    b.step(th, mo, hps, 0, stats)
    torch.cuda.synchronize()
    for i, (m, h, prec, ns, col) in enumerate(inst):
        th0 = init_theta(m, 1000 + i)
        th_o, _, st_o, _ = O.minsr_step(m, h, th0, np.zeros_like(th0), hps[i], 0)
        np.testing.assert_allclose(th[i].cpu().numpy(), th_o, rtol=RTOL64, atol=RTOL64)
        d = nqs.decode_stats(stats[i])
        assert abs(d["E_re"] - st_o["E_re"]) <= RTOL64 * abs(st_o["E_re"])


def test_batched_failure_is_isolated():
    """A non-finite step size in one instance flags that instance only and
    leaves its theta and momentum unchanged."""
    sub = INSTANCES[:3]
    ctxs, th, mo, hps = _setup(sub)
    hps[1] = copy.copy(hps[1])
    hps[1].eta0 = float("inf")
    before = [t.clone() for t in th]
    b = nqs.Batch(ctxs)
    b.use_graph(True)
    stats = b.new_stats()
    b.step(th, mo, hps, 0, stats)
    torch.cuda.synchronize()
    d = [nqs.decode_stats(stats[i]) for i in range(3)]
    assert d[1]["status"] == 4  # NQS_ERR_NONFINITE
    assert torch.equal(th[1], before[1]) and not torch.any(mo[1] != 0)
    for i in (0, 2):
        assert d[i]["status"] == 0
        assert not torch.equal(th[i], before[i])


@pytest.mark.parametrize("k", [0, 1, 3, 4])
def test_autotune_keeps_results(k):
    m, h, prec, ns, col = INSTANCES[k]
    hp = _hp(col, ns, 42)
    th0 = torch.tensor(init_theta(m, 5), device="cuda")
    ref = nqs.Context(m, h, prec, ns)
    tuned = nqs.Context(m, h, prec, ns)
    info = tuned.autotune(th0, hp, 0, force=True)
    assert info["n_samples"] == ns
    assert info["eloc_grid"] >= 1 and info["solve_grid"] >= 1
    assert info["ms"]["eloc"] > 0 and info["ms"]["solve"] > 0
    assert info["ms"]["eloc"] <= info["ms_default"]["eloc"]
    assert info["ms"]["solve"] <= info["ms_default"]["solve"]
    # theta given to the tuner is untouched
    assert torch.equal(th0, torch.tensor(init_theta(m, 5), device="cuda"))
    # one step with the built-in and the tuned shapes: samples, log Psi and
    # E_loc do not depend on the shapes; T differs by the rounding of its
    # regrouped K-slices, x and delta theta by that times the conditioning
    outs, stats_ = [], []
    for c in (ref, tuned):
        o = c.step_outputs(ns)
        t = th0.clone()
        st = c.new_stats()
        c.minsr_step(t, torch.zeros_like(t), hp, 0, st, outputs=o)
        outs.append(o)
        stats_.append(st)
    torch.cuda.synchronize()
    for key in ("spins", "logpsi", "eloc", "eps"):
        assert torch.equal(outs[0][key], outs[1][key]), key
    f64 = prec == "fp64"
    T0, T1 = outs[0]["T"], outs[1]["T"]
    # FP32 accumulation over K-slices of another length: well inside the
    # 2e-4 parity tolerance of the mixed T
    assert (T0 - T1).abs().max().item() <= (1e-13 if f64 else 2e-5) * T0.abs().max().item()
    # each solve meets the FP64 backward-error bound on its own system
    for o, st in zip(outs, stats_):
        lam = nqs.decode_stats(st)["lam"]
        T = o["T"].double()
        Ts = T + lam * torch.eye(T.shape[0], dtype=T.dtype, device=T.device)
        x, e = o["x"], o["eps"]
        berr = ((Ts @ x - e).abs().max() / (Ts.abs().sum(1).max() * x.abs().max())).item()
        assert berr < 100 * np.sqrt(len(x)) * 1.11e-16, berr
    # a second context of the same shape takes the cached choice without
    # measuring and then reproduces the tuned context bit for bit
    other = nqs.Context(m, h, prec, ns)
    info2 = other.autotune(th0, hp, 0)
    knobs = ("eloc_grid", "gram_splits", "solve_grid")
    assert {k_: info2[k_] for k_ in knobs} == {k_: info[k_] for k_ in knobs}
    res = []
    for c in (tuned, other):
        t = th0.clone()
        mo = torch.zeros_like(t)
        st = c.new_stats()
        for step in range(2):
            c.minsr_step(t, mo, hp, step, st)
        res.append((t, mo, st))
    torch.cuda.synchronize()
    for j in range(3):
        assert torch.equal(res[0][j], res[1][j])


def test_batch_autotune_then_step():
    sub = INSTANCES[:4]
    ctxs, th, mo, hps = _setup(sub)
    b = nqs.Batch(ctxs)
    b.use_graph(True)
    before = [t.clone() for t in th]
    ms = b.autotune(th, hps, 0, force=True)
    assert ms > 0
    assert 1 <= b.concurrency() <= len(sub)
    for t, t0 in zip(th, before):
        assert torch.equal(t, t0)
    stats = b.new_stats()
    for k in range(2):
        b.step(th, mo, hps, k, stats)
    torch.cuda.synchronize()
    th0, mo0, st0 = _solo(sub, 2, tuned=True)
    for i in range(len(sub)):
        assert torch.equal(th[i], th0[i]), i


GROUPED = INSTANCES + [
    (ModelSpec(1, 16, 1, 32), HamSpec("tfim"), "mixed", 150, "tfim"),
    (ModelSpec(2, 4, 4, 128, cplx=1, marshall=1, zmask=1), HamSpec("j1j2", J2=0.5), "mixed", 150, "j1j2"),
    (ModelSpec(2, 5, 3, 96), HamSpec("j1j2", J2=0.0), "mixed", 130, "heisenberg"),
]


@pytest.mark.parametrize("graph,stages", [(True, 3), (False, 3), (False, 2), (False, 1)],
                         ids=["graph-both", "eager-both", "eager-eloc", "eager-solve"])
def test_grouped_stages_equal_solo(graph, stages):
    """The batched step by stage (one launch of the streamed local-energy
    engine per hidden size over the mixed 2D d_h 96 / 128 instances, one
    cooperative launch for the FP32 solves of all mixed instances, each
    instance on its own CTA range) gives every instance exactly what its own
    step gives with the same solve form (128-wide panels): a tile's local
    energies, the factor's tiles and the refinement's rows do not depend on
    how many CTAs share them.  Mixed instances outside the solve group
    (R = 150 and R = 130, not a multiple of 4) and the FP64 instances take
    their own solves in the last part of the step."""
    inst = GROUPED
    steps = 3
    ctxs0, th0, mo0, hps = _setup(inst)
    n00 = sum(c.launch_count() for c in ctxs0)
    st0 = []
    n_solve, eloc_dh, blk = 0, [], []
    for i, (c, t, m, hp, (mod, _, prec, ns, _)) in enumerate(zip(ctxs0, th0, mo0, hps, inst)):
        R = ns * (2 if c.model.cplx else 1)
        if prec == "mixed" and R >= 256 and R % 4 == 0:
            c.set_solve_form(2)
            n_solve += 1
            blk.append(i)
        if prec == "mixed" and mod.dim == 2 and mod.dh in (96, 128):
            eloc_dh.append(mod.dh)
        s = c.new_stats()
        for k in range(steps):
            c.minsr_step(t, m, hp, k, s)
        st0.append(s)
    torch.cuda.synchronize()
    assert n_solve == 5 and sorted(eloc_dh) == [96, 96, 128]
    ctxs, th, mo, hps = _setup(inst)
    for i in blk:  # the same solve form where the solves stay apart (stages without bit 1)
        ctxs[i].set_solve_form(2)
    b = nqs.Batch(ctxs)
    b.use_graph(graph)
    b.set_grouped(stages)
    assert b.grouped() == stages
    stats = b.new_stats()
    n0 = sum(c.launch_count() for c in ctxs)
    for k in range(steps):
        b.step(th, mo, hps, k, stats)
    torch.cuda.synchronize()
    assert b.graph_active() == graph
    for i in range(len(inst)):
        d = nqs.decode_stats(stats[i])
        assert d["status"] == 0, (i, d)
        assert d["solve_fp64"] == (inst[i][2] == "fp64"), (i, d)
        assert torch.equal(th[i], th0[i]), i
        assert torch.equal(mo[i], mo0[i]), i
        assert torch.equal(stats[i], st0[i]), i
    if not graph:
        # per step: one grouped solve instead of five cooperative factors, one
        # engine launch per hidden size instead of one per instance
        solo = sum(c.launch_count() for c in ctxs0) - n00
        saved = ((n_solve - 1) if stages & 1 else 0) + \
            ((len(eloc_dh) - len(set(eloc_dh))) if stages & 2 else 0)
        assert sum(c.launch_count() for c in ctxs) - n0 == solo - saved * steps
    b.close()


def test_batched_eloc_share_equals_solo():
    """Local-energy engines on 6/8 of their grids inside the batch (the
    other SMs free for the other instances' kernels): every instance's step
    is still the one it takes alone, bit for bit, since a tile's local
    energies do not depend on the CTA that runs it."""
    steps = 2
    th0, mo0, st0 = _solo(INSTANCES, steps)
    ctxs, th, mo, hps = _setup()
    b = nqs.Batch(ctxs)
    b.set_eloc_share(6)
    assert b.eloc_share() == 6
    stats = b.new_stats()
    for k in range(steps):
        b.step(th, mo, hps, k, stats)
    torch.cuda.synchronize()
    for i in range(len(INSTANCES)):
        assert torch.equal(th[i], th0[i]), i
        assert torch.equal(stats[i], st0[i]), i
    with pytest.raises(nqs.NqsError):
        b.set_eloc_share(9)
    b.close()
