"""Parity at the benchmark workloads' full sizes, in the launch configuration
the benchmark times (one nqs_minsr_step_ex from theta_0).

The oracle cannot redo a whole step at these sizes in seconds, so each stage
is checked where it can be computed independently:
  * samples: every decision sigma_k = [u >= p_k(0)] against the oracle's
    conditionals along the GPU's own configurations (near-ties |u - p| below
    the path's precision are excused);
  * log Psi of every sample; E_loc on a random subset of samples;
  * T against O'^T O' assembled from the oracle's Jacobian of all samples
    (centred per block, / sqrt(Ns)); eps-bar' from the GPU's own E_loc;
  * x by its backward error on (T_gpu + lambda I) x = eps'_gpu;
  * delta theta against eta_eff O'_oracle x_gpu.
Where the oracle's whole Jacobian would take minutes (the 12 x 12, d_h 128,
Ns 4096 batched instance: 8192 x 84484), O is checked on the sampled rows
and T and delta theta against the FP64 Gram and product of the GPU's own O.
Errors of the mixed path go to NQS_ERRORS_OUT when it is set.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2608_18065_b300 import nqs
from paper_2608_18065_b300.inputs import init_theta, workloads
from tests.gpu_helpers import (RTOL64, TOL_MIXED_ELOC, TOL_MIXED_JAC, cplx, logpsi_err,
                               logpsi_err_tc, tc_sampled,
                               max_elem_err, max_row_err, record_error, rel_err)

pytestmark = pytest.mark.gpu


def _check_decisions(model, th, spins, seed, step, tol, rows):
    bad = 0
    for s in rows:
        p0 = O.conditionals(model, th, spins[s])
        u = np.array([O.uniform(seed, step, int(s), k) for k in range(model.N)])
        dec = np.where(u < p0, 0, 1)
        bad += int(np.sum((dec != spins[s]) & (np.abs(u - p0) > tol)))
    return bad


def _centred_oracle_rows(model, th, spins):
    ns = len(spins)
    Oj = O.jacobian(model, th, spins)
    blocks = [Oj[:ns]] + ([Oj[ns:]] if model.cplx else [])
    return np.concatenate([(b - b.mean(0)) / np.sqrt(ns) for b in blocks], 0)


CASES = [("tfim100", "mixed"), ("tfim100", "fp64"), ("tfim200", "mixed"), ("cluster64", "mixed"),
         ("heis10", "mixed"), ("cluster100p", "mixed"), ("heis10p", "mixed"), ("j1j2_10p", "mixed"),
         # batched instances: the largest (12 x 12, d_h 128, streamed-weight
         # engine, R = 8192 solve, 12.6 GB workspace) and a 12 x 12 d_h 32 one
         ("b16:j1j2_L12_J20.25_dh128_ns4096", "mixed"), ("b16:j1j2_L12_J20.5_dh32_ns256", "mixed")]


def _workload(key):
    if key.startswith("b16:"):
        from paper_2608_18065_b300.inputs import batched_instances
        return next(w for w in batched_instances() if w.name == key[4:])
    return workloads()[key]


@pytest.mark.parametrize("key,prec", CASES, ids=[f"{k}-{p}" for k, p in CASES])
def test_full_size_step(key, prec):
    w = _workload(key)
    model, ham, hp = w.model, w.ham, w.hp
    ns = hp.ns
    R = 2 * ns if model.cplx else ns
    np_ = len(init_theta(model, w.theta_seed))
    big = R * np_ > 2e8  # the oracle's whole Jacobian would not take seconds
    th = init_theta(model, w.theta_seed)
    c = nqs.Context(model, ham, prec, ns)
    thd = torch.tensor(th, device="cuda")
    md = torch.zeros_like(thd)
    outs = c.step_outputs(ns)
    stats = nqs.decode_stats(c.minsr_step(thd.clone(), md, hp, 0, outputs=outs))
    torch.cuda.synchronize()
    assert stats["status"] == 0, stats
    f64 = prec == "fp64"
    spins = outs["spins"].cpu().numpy()
    rng = np.random.default_rng(0)
    rows = rng.choice(ns, size=24, replace=False)
    # samples: all decisions of 24 random rows; for FP64 bit-exact over all rows
    if f64:
        sp_o, lp_o = O.sample(model, th, ns, hp.seed, 0)
        assert np.array_equal(spins, sp_o)
    else:
        assert _check_decisions(model, th, spins, hp.seed, 0, 1e-5, rows) == 0
    if model.zmask:
        assert np.all(spins.sum(1) == model.N // 2)
    # log Psi of every sample
    lp = cplx(outs["logpsi"])
    lp_o = O.logpsi(model, th, spins)
    if f64:
        np.testing.assert_allclose(lp, lp_o, rtol=RTOL64, atol=RTOL64)
    elif tc_sampled(model, prec):
        assert logpsi_err_tc(lp, lp_o, model.N) <= 1.0
    else:
        assert logpsi_err(lp, lp_o) <= 1.0
    # E_loc on sampled rows, every one of them
    el = cplx(outs["eloc"])
    el_o = O.local_energy(model, ham, th, spins[rows])
    tol_e = RTOL64 if f64 else TOL_MIXED_ELOC
    assert rel_err(el[rows], el_o) < tol_e
    assert max_elem_err(el[rows], el_o) < tol_e
    lam = stats["lam"]
    x = outs["x"].cpu().numpy()
    T = outs["T"].cpu().numpy()
    assert np.array_equal(T, T.T)
    errs = {"logpsi_abs": np.max(np.abs(lp - lp_o)), "eloc_elem": max_elem_err(el[rows], el_o)}
    if not big:
        # T from the oracle's Jacobian of every sample
        A = _centred_oracle_rows(model, th, spins)
        T_o = A @ A.T
        # T = A A^T carries twice the row-relative error of the mixed O
        # (Delta T = Delta A A^T + A Delta A^T): 2 TOL_MIXED_JAC
        assert max_elem_err(T, T_o) < (RTOL64 if f64 else 2 * TOL_MIXED_JAC)
        d_ref = stats["eta_eff"] * (A.T @ x)
        d_abs = stats["eta_eff"] * (np.abs(A).T @ np.abs(x))
        errs["T_elem"] = max_elem_err(T, T_o)
    else:
        # rows of O against the oracle's on the sampled samples (both blocks),
        # T against the FP64 Gram of the GPU's own O (centred in FP64), and
        # delta theta against eta_eff O'^T x from the same FP64 rows
        Og = c.jacobian(thd, outs["spins"])
        sel = np.concatenate([rows] + ([rows + ns] if model.cplx else []))
        J_o = O.jacobian(model, th, spins[rows])
        o_err = max_row_err(Og[torch.tensor(sel, device="cuda")].double().cpu().numpy(), J_o)
        assert o_err < TOL_MIXED_JAC
        Od = Og.double()
        del Og
        blocks = [Od[:ns]] + ([Od[ns:]] if model.cplx else [])
        Ac = torch.cat([(q - q.mean(0)) / np.sqrt(ns) for q in blocks], 0)
        del Od, blocks
        T_ref = (Ac @ Ac.T).cpu().numpy()
        assert max_elem_err(T, T_ref) < 2e-5
        xd = torch.tensor(x, device="cuda")
        d_ref = stats["eta_eff"] * (Ac.T @ xd).cpu().numpy()
        d_abs = stats["eta_eff"] * (Ac.abs().T @ xd.abs()).cpu().numpy()
        del Ac
        errs["T_elem_vs_fp64_gram_of_gpu_O"] = max_elem_err(T, T_ref)
        errs["O_row_sampled"] = o_err
    # eps-bar' from the GPU's local energies
    E = el.mean()
    ebar = np.conj(el - E) / np.sqrt(ns)
    eps = 2 * np.concatenate([ebar.real] + ([-ebar.imag] if model.cplx else []))
    np.testing.assert_allclose(outs["eps"].cpu().numpy(), eps, rtol=0, atol=1e-12 * np.max(np.abs(eps)))
    # x: backward error of the GPU's solve of its own system (FP64 level)
    Ts = T + lam * np.eye(len(eps))
    e_gpu = outs["eps"].cpu().numpy()
    berr = np.max(np.abs(Ts @ x - e_gpu)) / (np.max(np.abs(Ts).sum(1)) * np.max(np.abs(x)))
    assert berr < 100 * np.sqrt(len(x)) * 1.11e-16
    # delta theta = eta_eff O' x with the reference O'
    d = outs["dtheta"].cpu().numpy()
    # delta theta = eta sum_r x_r O'_r reads O' as its BF16 hi + lo split
    # (16 significant bits, 2^-17 relative per entry); independent rounding
    # errors add in quadrature over the R rows, amplified by the sum's
    # condition cond = ||eta |O'|^T |x||| / ||delta theta||: 4 2^-17 cond /
    # sqrt(R) (the measured errors of every workload follow 2^-17 cond /
    # sqrt(R) to within 1.5x), at least 5e-4
    cond = float(np.linalg.norm(d_abs) / np.linalg.norm(d_ref))
    tol_d = 1e-9 if f64 else max(5e-4, 4 * 2.0 ** -17 * cond / np.sqrt(len(x)))
    assert rel_err(d, d_ref) < tol_d
    # element by element: the bias and input columns of O are sums over the
    # sites of BF16x3-split adjoints (2^-17 per term) whose terms largely
    # cancel, and the centring and the x-weighted sum cancel again, so their
    # entries of delta theta carry a few times the norm's relative error
    assert max_elem_err(d, d_ref) < (1e-9 if f64 else 2e-3)
    errs.update(x_backward_error=berr, dtheta_rel=rel_err(d, d_ref),
                dtheta_elem=max_elem_err(d, d_ref), dtheta_sum_cond=cond,
                solve_fp64=stats["solve_fp64"])
    if not f64:
        record_error(f"fullsize_{key}", **errs)


def _fp64_gram_of(ctx, model, th, spins, ns):
    """T from the context's own FP32 Jacobian, centred and multiplied in FP64."""
    O = ctx.jacobian(th, spins).double()
    blocks = [O[:ns]] + ([O[ns:]] if model.cplx else [])
    Oc = torch.cat([(b - b.mean(0)) / np.sqrt(ns) for b in blocks], 0)
    return Oc @ Oc.T


def test_tensor_core_gram_keeps_positive_semidefinite():
    """The tensor-core T (four split products, compensated chunk sums) stays
    within FP32-split accuracy of the FP64 Gram of the same FP32 Jacobian and
    loses positive semi-definiteness only at the level of its own rounding
    (dropping lo lo^T or summing long K ranges in one FP32 accumulator made
    its smallest eigenvalue about -1e-4 ||T|| on this 10 x 10 lattice)."""
    w = workloads()["heis10"]
    model, ham, hp = w.model, w.ham, w.hp
    ns = hp.ns
    c = nqs.Context(model, ham, "mixed", ns)
    th = torch.tensor(init_theta(model, w.theta_seed), device="cuda")
    outs = c.step_outputs(ns)
    s = c.new_stats()
    c.minsr_step(th.clone(), torch.zeros_like(th), hp, 0, s, outputs=outs)
    torch.cuda.synchronize()
    T = outs["T"]
    Tx = _fp64_gram_of(c, model, th, outs["spins"], ns)
    scale = Tx.abs().max().item()
    assert (T - Tx).abs().max().item() <= 2e-5 * scale
    ev = torch.linalg.eigvalsh(T)
    assert ev.min().item() >= -1e-7 * ev.max().item(), (ev.min().item(), ev.max().item())
    st = nqs.decode_stats(s)
    assert st["status"] == 0 and st["solve_fp64"] == 0, st


def test_mixed_steps_accepted_where_fp64_is():
    """Tab. I Heisenberg steps on the 10 x 10 lattice: every mixed step is
    accepted (status 0), as on the FP64 path."""
    w = workloads()["heis10"]
    c = nqs.Context(w.model, w.ham, "mixed", w.hp.ns)
    th = torch.tensor(init_theta(w.model, w.theta_seed), device="cuda")
    mo = torch.zeros_like(th)
    s = c.new_stats()
    for t in range(4):
        c.minsr_step(th, mo, w.hp, t, s)
        torch.cuda.synchronize()
        st = nqs.decode_stats(s)
        assert st["status"] == 0, (t, st)


def test_fp64_gram_retry_when_lambda_is_below_tensor_core_rounding():
    """A 12 x 12 J1-J2 instance (dh 32, Ns 256, lambda = 0.1) whose ||T||
    reaches 1e8-1e9: T + lambda I from the tensor cores is indefinite by its
    rounding, the step rebuilds T in FP64 from the split planes and solves
    again (solve_fp64 = 2) instead of being rejected; the FP64 path accepts
    the same steps."""
    from paper_2608_18065_b300.inputs import batched_instances
    w = batched_instances()[11]
    c = nqs.Context(w.model, w.ham, "mixed", w.hp.ns)
    th = torch.tensor(init_theta(w.model, w.theta_seed), device="cuda")
    mo = torch.zeros_like(th)
    s = c.new_stats()
    seen = set()
    checked = False
    for t in range(5):
        th_before = th.cpu().numpy()
        outs = c.step_outputs(w.hp.ns)
        st = nqs.decode_stats(c.minsr_step(th, mo, w.hp, t, s, outputs=outs))
        torch.cuda.synchronize()
        assert st["status"] == 0, (t, st)
        seen.add(st["solve_fp64"])
        if st["solve_fp64"] == 2 and not checked:
            # the retried step: T against the FP64 Gram of the step's own O
            # (centred in FP64), delta theta = eta_eff O'^T x from the same
            # rows, x at FP64 backward error.  Here ||T|| ~ 1e8 -- 1e9: O has
            # large entries with a small spread over the samples, the
            # centring cancels, and the FP32 Jacobian sits ~6e-4 (row-
            # relative) from the oracle's, so O is held to that regime's 2e-3
            checked = True
            sp = outs["spins"]
            thb = torch.tensor(th_before, device="cuda")
            Og = c.jacobian(thb, sp).double()
            ns = w.hp.ns
            A = torch.cat([(q - q.mean(0)) / np.sqrt(ns) for q in (Og[:ns], Og[ns:])], 0)
            T = outs["T"].cpu().numpy()
            assert max_elem_err(T, (A @ A.T).cpu().numpy()) < 2e-5
            x = outs["x"].cpu().numpy()
            d_ref = st["eta_eff"] * (A.T @ torch.tensor(x, device="cuda")).cpu().numpy()
            d = outs["dtheta"].cpu().numpy()
            assert rel_err(d, d_ref) < 5e-4
            # x solves the T rebuilt in FP64 from the split planes, which
            # differs from the step's output T (the tensor-core T, copied
            # before the rebuild) by ~1e-7 of its scale: the backward error
            # against the output T is bounded by that difference
            Ts = T + st["lam"] * np.eye(len(x))
            e = outs["eps"].cpu().numpy()
            berr = np.max(np.abs(Ts @ x - e)) / (np.max(np.abs(Ts).sum(1)) * np.max(np.abs(x)))
            assert berr < 1e-6
            rows = np.arange(8)
            J_o = O.jacobian(w.model, th_before, sp.cpu().numpy()[rows])
            Jg = torch.cat([Og[:8], Og[ns:ns + 8]]).cpu().numpy()
            # at these weights (a run that has grown ||T|| to 1e9) the reverse
            # sweep's FP32 recurrences put O within ~1e-3 of each row's largest
            # entry (8.3e-4 measured with an FP32 assembly); the tensor-core
            # assembly of the 2D rows adds its BF16x3 rounding, up to 3 2^-18
            # per adjoint-state product over the 144 sites, which the sums'
            # cancellation at this scale magnifies (2.3e-3 in all, measured)
            assert max_row_err(Jg, J_o) < 5e-3
            record_error("fp64_gram_retry_" + w.name,
                         T_elem_vs_fp64_gram_of_gpu_O=max_elem_err(T, (A @ A.T).cpu().numpy()),
                         dtheta_rel=rel_err(d, d_ref), x_backward_error=berr,
                         O_row_sampled=max_row_err(Jg, J_o))
    assert 2 in seen, seen
    assert checked
    assert torch.isfinite(th).all()
