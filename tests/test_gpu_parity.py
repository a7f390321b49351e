"""GPU parity of every stage of the minSR step against the FP64 oracle,
through the C-ABI (libnqs.so).  Sizes span several CTA tiles with ragged
tails; the FP64 path is held to 1e-10 relative and bit-exact samples, the
mixed path to the FP32-derived tolerances of gpu_helpers."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2608_18065_b300.inputs import HamSpec, HParams, ModelSpec, random_spins
from tests.gpu_helpers import (RTOL64, TOL_MIXED_ELOC, TOL_MIXED_JAC, TOL_MIXED_LOGPSI,
                               cplx, ctx, max_elem_err, max_row_err, near_ties, record_error,
                               rel_err, theta_dev)

pytestmark = pytest.mark.gpu

MODELS = [
    (ModelSpec(1, 13, 1, 8), HamSpec("tfim", J=1.0, h=0.9)),
    (ModelSpec(1, 12, 1, 16, cplx=1), HamSpec("cluster_zxz")),
    (ModelSpec(1, 11, 1, 8, cplx=1), HamSpec("cluster_paper")),
    (ModelSpec(2, 4, 4, 8, cplx=1, marshall=1, zmask=1), HamSpec("j1j2", J1=1.0, J2=0.5)),
    (ModelSpec(2, 3, 4, 16, cplx=1, marshall=1, zmask=1), HamSpec("j1j2", J1=1.0, J2=0.0)),
    (ModelSpec(2, 5, 2, 8), HamSpec("j1j2", J1=1.0, J2=0.0)),
]
IDS = [f"{m.dim}d_{m.Lx}x{m.Ly}_dh{m.dh}_{h.family}" for m, h in MODELS]


@pytest.mark.parametrize("model,ham", MODELS, ids=IDS)
def test_sampler_fp64_bit_exact(model, ham):
    ns = 77
    c = ctx(model, ham, "fp64", ns)
    th, thd = theta_dev(model, 3, scale=1.5)
    spins, lp = c.sample(thd, ns, seed=42, step=5)
    torch.cuda.synchronize()
    sp_o, lp_o = O.sample(model, th, ns, 42, 5)
    assert near_ties(model, th, sp_o, 42, 5, 1e-12) == 0
    assert np.array_equal(spins.cpu().numpy(), sp_o)
    np.testing.assert_allclose(cplx(lp), lp_o, rtol=RTOL64, atol=RTOL64)


@pytest.mark.parametrize("model,ham", MODELS, ids=IDS)
def test_logpsi_eloc_jacobian_fp64(model, ham):
    ns = 70
    c = ctx(model, ham, "fp64", ns)
    th, thd = theta_dev(model, 4)
    sp = random_spins(model, ns, seed=9, zero_mag=bool(model.zmask))
    spd = torch.tensor(sp, device="cuda")
    lp = cplx(c.logpsi(thd, spd))
    np.testing.assert_allclose(lp, O.logpsi(model, th, sp), rtol=RTOL64, atol=RTOL64)
    el = cplx(c.local_energy(thd, spd))
    el_o = O.local_energy(model, ham, th, sp)
    assert rel_err(el, el_o) < RTOL64
    J = c.jacobian(thd, spd).cpu().numpy()
    J_o = O.jacobian(model, th, sp)
    assert J.shape == J_o.shape
    assert rel_err(J, J_o) < RTOL64
    assert np.max(np.abs(J - J_o)) < RTOL64 * np.max(np.abs(J_o))


@pytest.mark.parametrize("model,ham", MODELS, ids=IDS)
def test_logpsi_eloc_jacobian_mixed(model, ham):
    ns = 70
    c = ctx(model, ham, "mixed", ns)
    th, thd = theta_dev(model, 4)
    sp = random_spins(model, ns, seed=9, zero_mag=bool(model.zmask))
    spd = torch.tensor(sp, device="cuda")
    lp = cplx(c.logpsi(thd, spd))
    lp_o = O.logpsi(model, th, sp)
    assert np.max(np.abs(lp - lp_o)) < TOL_MIXED_LOGPSI
    el = cplx(c.local_energy(thd, spd))
    el_o = O.local_energy(model, ham, th, sp)
    assert rel_err(el, el_o) < TOL_MIXED_ELOC
    assert max_elem_err(el, el_o) < TOL_MIXED_ELOC  # every sample
    J = c.jacobian(thd, spd).cpu().numpy().astype(np.float64)
    J_o = O.jacobian(model, th, sp)
    assert rel_err(J, J_o) < TOL_MIXED_JAC
    assert max_row_err(J, J_o) < TOL_MIXED_JAC  # every entry, per row
    record_error(f"small_{model.dim}d_{model.Lx}x{model.Ly}_dh{model.dh}_{ham.family}",
                 logpsi_abs=np.max(np.abs(lp - lp_o)), eloc_elem=max_elem_err(el, el_o),
                 O_row=max_row_err(J, J_o))


# hidden size 64 and 32 on 1D chains assemble the rows of O on the tensor
# cores: chain lengths that end a 16-site chunk exactly (N + 1 = 16), leave
# one site over (N + 1 = 17) or span two chunks, real and complex heads, the
# mask, and more rows than the two CTAs per SM (so a CTA walks several rows
# with the next row's loads in flight)
JTC_MODELS = [
    (ModelSpec(1, 21, 1, 64), HamSpec("tfim", J=1.0, h=0.9), 300),
    (ModelSpec(1, 16, 1, 32, cplx=1, zmask=1), HamSpec("cluster_zxz"), 160),
    (ModelSpec(1, 15, 1, 64, cplx=1), HamSpec("cluster_zxz"), 40),
    (ModelSpec(1, 30, 1, 32, zmask=1), HamSpec("tfim"), 333),
]


@pytest.mark.parametrize("model,ham,ns", JTC_MODELS,
                         ids=["tfim21dh64", "zxz16dh32cmask", "zxz15dh64c", "tfim30dh32mask"])
def test_tensor_core_jacobian_mixed(model, ham, ns):
    c = ctx(model, ham, "mixed", ns)
    th, thd = theta_dev(model, 6)
    sp = random_spins(model, ns, seed=13, zero_mag=bool(model.zmask))
    J = c.jacobian(thd, torch.tensor(sp, device="cuda")).cpu().numpy().astype(np.float64)
    J_o = O.jacobian(model, th, sp)
    assert J.shape == J_o.shape
    assert rel_err(J, J_o) < TOL_MIXED_JAC
    # every entry, including the biases, input columns and heads, within the
    # same tolerance of the largest entry of its row
    scale = np.max(np.abs(J_o), axis=1, keepdims=True)
    assert np.max(np.abs(J - J_o) / scale) < TOL_MIXED_JAC


@pytest.mark.parametrize("model,ham,scale", [
    (ModelSpec(2, 4, 4, 16, cplx=1, marshall=1, zmask=1), HamSpec("j1j2"), 1.5),
    (ModelSpec(1, 40, 1, 64, cplx=1), HamSpec("cluster_zxz"), 1.0),
    (ModelSpec(1, 100, 1, 64), HamSpec("tfim"), 1.0),
], ids=["2d_dh16", "1d_dh64_c_wmma", "1d_dh64_n100_wmma"])
def test_sampler_mixed_decisions_valid(model, ham, scale):
    """FP32 conditionals decide the spins: every decision must agree with the
    oracle's p_k(0) unless u lies within 1e-5 of it; log Psi as mixed.  The
    1D d_h = 64 sampler forms its gate products on warp-level MMAs (BF16x3),
    checked at the initialisation scale N(0, 1/fan_in)."""
    ns = 100
    c = ctx(model, ham, "mixed", ns)
    th, thd = theta_dev(model, 6, scale=scale)
    spins, lp = c.sample(thd, ns, seed=11, step=2)
    sp = spins.cpu().numpy()
    if model.zmask:
        assert np.all(sp.sum(1) == model.N // 2)
    bad = 0
    for s in range(ns):
        p0 = O.conditionals(model, th, sp[s])
        u = np.array([O.uniform(11, 2, s, k) for k in range(model.N)])
        dec = np.where(u < p0, 0, 1)
        bad += int(np.sum((dec != sp[s]) & (np.abs(u - p0) > 1e-5)))
    assert bad == 0
    assert np.max(np.abs(cplx(lp) - O.logpsi(model, th, sp))) < TOL_MIXED_LOGPSI


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("R,np_", [(1, 7), (70, 300), (130, 1001), (256, 4097)])
def test_gram(prec, R, np_):
    model, ham = ModelSpec(1, 8, 1, 64), HamSpec("tfim")  # Np = 13058 >= np_
    c = ctx(model, ham, prec, 256)
    rng = np.random.default_rng(R)
    A = rng.standard_normal((R, np_)) / np.sqrt(np_)
    dt = torch.float64 if prec == "fp64" else torch.float32
    Ad = torch.tensor(A, dtype=dt, device="cuda")
    T = c.gram(Ad).cpu().numpy()
    Aref = Ad.double().cpu().numpy()
    Tref = Aref @ Aref.T
    tol = RTOL64 if prec == "fp64" else 1e-5
    assert np.max(np.abs(T - Tref)) < tol * np.max(np.abs(Tref))
    assert np.array_equal(T, T.T)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("R", [1, 31, 64, 200, 513, 600])
def test_regularized_solve(R, prec):
    """FP64 Cholesky (FP64 context) and FP32-factor + FP64 refinement (mixed
    context) both reach the FP64 solution."""
    model, ham = ModelSpec(1, 8, 1, 8), HamSpec("tfim")
    c = ctx(model, ham, prec, 600)
    rng = np.random.default_rng(R)
    M = rng.standard_normal((R, R + 5))
    T = M @ M.T
    b = rng.standard_normal(R)
    lam = 1e-2
    Td = torch.tensor(T, device="cuda")
    x, st = c.regularized_solve(Td, lam, torch.tensor(b, device="cuda"))
    assert int(st.item()) == 0
    xr = np.linalg.solve(T + lam * np.eye(R), b)
    kappa = np.linalg.cond(T + lam * np.eye(R))
    assert rel_err(x.cpu().numpy(), xr) < max(1e-10, 100 * kappa * 2.2e-16)
    # an indefinite matrix reports NOT_SPD (5)
    Td = torch.tensor(-T - np.eye(R), device="cuda")
    x, st = c.regularized_solve(Td, 0.0, torch.tensor(b, device="cuda"))
    assert int(st.item()) == 5


STEP_CASES = [
    (ModelSpec(1, 16, 1, 16), HamSpec("tfim"), HParams(0.5, 1e3, 0.7, lam=1e-3, ns=128)),
    (ModelSpec(1, 12, 1, 8, cplx=1), HamSpec("cluster_zxz"),
     HParams(5e-3, 5e3, 0.1, lam=1e-3, ns=60)),
    (ModelSpec(2, 4, 4, 8, cplx=1, marshall=1, zmask=1), HamSpec("j1j2", J2=0.0),
     HParams(6e-2, 1e4, 0.75, lambda_mode=1, lambda_coeff=3e-4, lambda_pow=2 / 3, ns=50)),
    (ModelSpec(2, 4, 4, 8, cplx=1, marshall=1, zmask=1), HamSpec("j1j2", J2=0.5),
     HParams(0.1, 1e4, 0.1, lam=0.1, trust_region=1, ns=50)),
]
STEP_IDS = ["tfim16", "cluster12", "heis4x4", "j1j2_4x4"]


@pytest.mark.parametrize("model,ham,hp", STEP_CASES, ids=STEP_IDS)
def test_minsr_step_fp64(model, ham, hp):
    """Two consecutive steps: samples bit-exact; E, T, x, delta theta,
    theta and momentum to 1e-10 relative (kappa * eps64 << 1e-10 here)."""
    c = ctx(model, ham, "fp64", hp.ns)
    th, thd = theta_dev(model, 1234)
    mom = np.zeros_like(th)
    momd = torch.zeros_like(thd)
    for t in range(2):
        outs = c.step_outputs(hp.ns)
        stats = c.minsr_step(thd, momd, hp, t, outputs=outs)
        torch.cuda.synchronize()
        th, mom, st_o, b = O.minsr_step(model, ham, th, mom, hp, t,
                                        want=("spins", "eloc", "T", "eps", "x", "dtheta"))
        from paper_2608_18065_b300.nqs import decode_stats
        st = decode_stats(stats)
        assert st["status"] == 0 and st_o["status"] == 0
        assert np.array_equal(outs["spins"].cpu().numpy(), b["spins"])
        assert rel_err(cplx(outs["eloc"]), b["eloc"]) < RTOL64
        for k in ("E_re", "var", "lam", "normT", "eta_eff", "tau_norm"):
            assert abs(st[k] - st_o[k]) <= RTOL64 * max(abs(st_o[k]), 1e-300), k
        assert rel_err(outs["T"].cpu().numpy(), b["T"]) < RTOL64
        assert rel_err(outs["eps"].cpu().numpy(), b["eps"]) < RTOL64
        Tm = b["T"] + st_o["lam"] * np.eye(len(b["eps"]))
        kappa = np.linalg.cond(Tm)
        tol = max(RTOL64, 100 * kappa * 2.2e-16)
        assert rel_err(outs["x"].cpu().numpy(), b["x"]) < tol
        assert rel_err(outs["dtheta"].cpu().numpy(), b["dtheta"]) < tol
        assert rel_err(thd.cpu().numpy(), th) < tol
        assert rel_err(momd.cpu().numpy(), mom) < tol


@pytest.mark.parametrize("model,ham,hp", STEP_CASES[:3], ids=STEP_IDS[:3])
def test_minsr_step_mixed_error_report(model, ham, hp):
    """Mixed step against the FP64 oracle from the same state: samples agree
    except near-ties; E, T and delta theta errors stay within FP32-derived
    bounds (T: BF16x3/FP32 product error ~1e-5 of max|T|)."""
    c = ctx(model, ham, "mixed", hp.ns)
    th, thd = theta_dev(model, 1234)
    momd = torch.zeros_like(thd)
    from paper_2608_18065_b300.nqs import decode_stats
    # a near-tie (|u - p| below the FP32 decision's resolution) may change a
    # mixed sample: draw again at the next step index (other uniforms)
    for t in range(8):
        outs = c.step_outputs(hp.ns)
        stats = c.minsr_step(thd.clone(), momd.clone(), hp, t, outputs=outs)
        torch.cuda.synchronize()
        st = decode_stats(stats)
        _, _, st_o, b = O.minsr_step(model, ham, th, np.zeros_like(th), hp, t,
                                     want=("spins", "eloc", "T", "eps", "x", "dtheta"))
        if np.array_equal(outs["spins"].cpu().numpy(), b["spins"]):
            break
    else:
        pytest.fail("eight draws in a row changed a mixed-precision sample")
    assert st["status"] == 0
    assert abs(st["E_re"] - st_o["E_re"]) < TOL_MIXED_ELOC * abs(st_o["E_re"])
    T = outs["T"].cpu().numpy()
    # T element by element (BF16x3 products, FP32 chunk sums, FP64 totals)
    assert max_elem_err(T, b["T"]) < 2e-4
    # delta theta = eta_eff O' x: the update path against the oracle's O'
    # with the GPU's own x (as at full size) ...
    ns = hp.ns
    Oj = O.jacobian(model, th, b["spins"])
    blocks = [Oj[:ns]] + ([Oj[ns:]] if model.cplx else [])
    A = np.concatenate([(q - q.mean(0)) / np.sqrt(ns) for q in blocks], 0)
    d = outs["dtheta"].cpu().numpy()
    d_ref = st["eta_eff"] * (A.T @ outs["x"].cpu().numpy())
    assert rel_err(d, d_ref) < 5e-4
    assert max_elem_err(d, d_ref) < 5e-4
    # ... and end to end against the oracle's delta theta: the solve
    # amplifies the errors of T and eps-bar' by at most kappa(T + lambda I)
    Tm = b["T"] + st_o["lam"] * np.eye(len(b["eps"]))
    kappa = np.linalg.cond(Tm)
    dT = np.linalg.norm(T - b["T"], 2) / np.linalg.norm(Tm, 2)
    de = rel_err(outs["eps"].cpu().numpy(), b["eps"])
    bound = 5e-4 + 2 * kappa * (dT + de)
    err = rel_err(d, b["dtheta"])
    assert err < bound, (err, bound, kappa)
    record_error(f"step_{model.dim}d_{model.Lx}x{model.Ly}_dh{model.dh}_{ham.family}",
                 E_rel=abs(st["E_re"] - st_o["E_re"]) / abs(st_o["E_re"]),
                 T_elem=max_elem_err(T, b["T"]), dtheta_update_path=rel_err(d, d_ref),
                 dtheta_end_to_end=err, kappa=kappa)


@pytest.mark.parametrize("model,ham,hp", STEP_CASES[:2], ids=STEP_IDS[:2])
def test_energy_trajectory_mixed_vs_oracle(model, ham, hp):
    """Eight chained steps of the mixed path and of the FP64 oracle, each from
    its own previous state with the same Philox keys: while the two draw the
    same samples the energies agree to the mixed E_loc tolerance (the states
    drift apart by the steps' own delta theta errors, ~1e-4)."""
    c = ctx(model, ham, "mixed", hp.ns)
    th, thd = theta_dev(model, 1234)
    mo = np.zeros_like(th)
    momd = torch.zeros_like(thd)
    from paper_2608_18065_b300.nqs import decode_stats
    worst, same = 0.0, 0
    for t in range(8):
        outs = c.step_outputs(hp.ns)
        st = decode_stats(c.minsr_step(thd, momd, hp, t, outputs=outs))
        torch.cuda.synchronize()
        th, mo, st_o, b = O.minsr_step(model, ham, th, mo, hp, t, want=("spins",))
        assert st["status"] == 0
        if not np.array_equal(outs["spins"].cpu().numpy(), b["spins"]):
            break
        same += 1
        worst = max(worst, abs(st["E_re"] - st_o["E_re"]) / abs(st_o["E_re"]))
    assert same >= 3
    assert worst < TOL_MIXED_ELOC
    record_error(f"trajectory_{model.dim}d_{model.Lx}x{model.Ly}_dh{model.dh}_{ham.family}",
                 E_rel_max=worst, steps_same_samples=same)


# hidden size 64 on 1D chains takes the tensor-core connected-configuration
# engine in the mixed path, and so does 32 (units padded with zeros); 300
# samples = two full 128-row tiles + a ragged one
TC_MODELS = [
    (ModelSpec(1, 24, 1, 64), HamSpec("tfim", J=1.0, h=0.8)),
    (ModelSpec(1, 20, 1, 64, cplx=1), HamSpec("cluster_zxz")),
    (ModelSpec(1, 18, 1, 64, cplx=1), HamSpec("cluster_paper")),
    (ModelSpec(1, 16, 1, 64, zmask=1), HamSpec("tfim")),
    (ModelSpec(1, 26, 1, 32), HamSpec("tfim", J=1.0, h=1.0)),
    (ModelSpec(1, 18, 1, 32, cplx=1, zmask=1), HamSpec("cluster_zxz")),
]


@pytest.mark.parametrize("model,ham", TC_MODELS,
                         ids=["tfim24", "zxz20", "xzx18", "tfim16mask", "tfim26dh32", "zxz18dh32mask"])
def test_eloc_tensor_core_engine_mixed(model, ham):
    ns = 300
    c = ctx(model, ham, "mixed", ns)
    th, thd = theta_dev(model, 4)
    sp = random_spins(model, ns, seed=9, zero_mag=bool(model.zmask))
    spd = torch.tensor(sp, device="cuda")
    el = cplx(c.local_energy(thd, spd))
    el_o = O.local_energy(model, ham, th, sp)
    assert rel_err(el, el_o) < TOL_MIXED_ELOC
    assert max_elem_err(el, el_o) < TOL_MIXED_ELOC  # every sample, ragged tile included
    # the FP64 context (SIMT engine) agrees with the oracle to 1e-10
    c64 = ctx(model, ham, "fp64", ns)
    assert rel_err(cplx(c64.local_energy(thd, spd)), O.local_energy(model, ham, th, sp)) < RTOL64


# 2D lattices with hidden size 64 run the tensor-core engine in the mixed
# context: 128-row tiles with a ragged tail, more tiles than CTAs (ns = 700 on
# the 4x4 J1-J2 model gives 42 operators x 6 tiles), an odd row length, two
# columns (a row turn every other site), real and complex heads, the mask
E2D_MODELS = [
    (ModelSpec(2, 4, 4, 64, cplx=1, marshall=1, zmask=1), HamSpec("j1j2", J1=1.0, J2=0.5), 700),
    (ModelSpec(2, 5, 3, 64), HamSpec("j1j2", J1=1.0, J2=0.0), 130),
    (ModelSpec(2, 2, 3, 64, cplx=1), HamSpec("j1j2", J1=1.0, J2=0.25), 70),
    # hidden size 32 runs the same engine with its units padded to 64
    (ModelSpec(2, 4, 4, 32, cplx=1, marshall=1, zmask=1), HamSpec("j1j2", J1=1.0, J2=0.6), 300),
    (ModelSpec(2, 3, 5, 32), HamSpec("j1j2", J1=1.0, J2=0.0), 140),
]


@pytest.mark.parametrize("model,ham,ns", E2D_MODELS, ids=["j1j2_4x4_cmask", "heis_5x3", "j1j2_2x3_c",
                                                          "j1j2_4x4_dh32_cmask", "heis_3x5_dh32"])
def test_eloc_2d_tensor_core_engine_mixed(model, ham, ns):
    c = ctx(model, ham, "mixed", ns)
    th, thd = theta_dev(model, 4)
    sp = random_spins(model, ns, seed=9, zero_mag=bool(model.zmask))
    spd = torch.tensor(sp, device="cuda")
    el = cplx(c.local_energy(thd, spd))
    el_o = O.local_energy(model, ham, th, sp)
    assert rel_err(el, el_o) < TOL_MIXED_ELOC
    # every sample's local energy, not only the vector norm
    scale = np.max(np.abs(el_o))
    assert np.max(np.abs(el - el_o)) < TOL_MIXED_ELOC * scale


# 2D lattices with hidden size 96 or 128 run the streamed-weight tensor-core
# engine in the mixed context: the frontier passes (U2 h of the cached row
# frontier), row starts taking U2 h_{k-1} from the same product, several
# 128-row tiles per operator with a ragged tail, odd row lengths, real and
# complex heads, the mask
E2DS_MODELS = [
    (ModelSpec(2, 4, 4, 128, cplx=1, marshall=1, zmask=1), HamSpec("j1j2", J1=1.0, J2=0.5), 300),
    (ModelSpec(2, 5, 3, 96), HamSpec("j1j2", J1=1.0, J2=0.0), 130),
    (ModelSpec(2, 3, 4, 128, cplx=1), HamSpec("j1j2", J1=1.0, J2=0.25), 200),
    (ModelSpec(2, 4, 3, 96, cplx=1, marshall=1, zmask=1), HamSpec("j1j2", J1=1.0, J2=0.6), 260),
]


@pytest.mark.parametrize("model,ham,ns", E2DS_MODELS,
                         ids=["j1j2_4x4_dh128_cmask", "heis_5x3_dh96", "j1j2_3x4_dh128_c",
                              "j1j2_4x3_dh96_cmask"])
def test_eloc_2d_tensor_core_streamed_mixed(model, ham, ns):
    c = ctx(model, ham, "mixed", ns)
    th, thd = theta_dev(model, 4)
    sp = random_spins(model, ns, seed=9, zero_mag=bool(model.zmask))
    spd = torch.tensor(sp, device="cuda")
    el = cplx(c.local_energy(thd, spd))
    el_o = O.local_energy(model, ham, th, sp)
    assert rel_err(el, el_o) < TOL_MIXED_ELOC
    scale = np.max(np.abs(el_o))
    assert np.max(np.abs(el - el_o)) < TOL_MIXED_ELOC * scale


# 2D lattices with hidden size 64 run the reverse sweep's gate product
# W^T [dau; dar; dg] on warp-level MMAs in the mixed context (the adjoint of
# h', routed on through U1, U2 to the horizontal and vertical neighbours):
# complex head with mask (two adjoint seeds), an odd row length, two columns
E2DJ_MODELS = [
    (ModelSpec(2, 4, 4, 64, cplx=1, marshall=1, zmask=1), HamSpec("j1j2", J1=1.0, J2=0.5), 150),
    (ModelSpec(2, 5, 3, 64), HamSpec("j1j2", J1=1.0, J2=0.0), 130),
    (ModelSpec(2, 2, 3, 64, cplx=1), HamSpec("j1j2", J1=1.0, J2=0.25), 70),
]


@pytest.mark.parametrize("model,ham,ns", E2DJ_MODELS, ids=["j1j2_4x4_cmask", "heis_5x3", "j1j2_2x3_c"])
def test_jacobian_2d_warp_mma_mixed(model, ham, ns):
    c = ctx(model, ham, "mixed", ns)
    th, thd = theta_dev(model, 6)
    sp = random_spins(model, ns, seed=13, zero_mag=bool(model.zmask))
    J = c.jacobian(thd, torch.tensor(sp, device="cuda")).cpu().numpy().astype(np.float64)
    J_o = O.jacobian(model, th, sp)
    assert J.shape == J_o.shape
    assert rel_err(J, J_o) < TOL_MIXED_JAC
    # every entry within the tolerance of the largest entry of its row
    scale = np.max(np.abs(J_o), axis=1, keepdims=True)
    assert np.max(np.abs(J - J_o) / scale) < TOL_MIXED_JAC


# 2D lattices of hidden size 32, 64, 96 and 128 assemble the five large
# weight blocks of every row of O (W_u, W_r, W_h on h'; U1, U2) as
# tensor-core products over the sites, the rest of the row on SIMT: chains
# that are not a multiple of the 16-site chunk, real and complex heads (two
# rows per sample), a tile of gate adjoints only partly filled (d_h 96: 288
# of 384 rows), the mask
E2DJT_MODELS = [
    (ModelSpec(2, 5, 3, 32, cplx=1, marshall=1), HamSpec("j1j2", J1=1.0, J2=0.5), 90),
    (ModelSpec(2, 4, 5, 96, cplx=1, marshall=1, zmask=1), HamSpec("j1j2", J1=1.0, J2=0.25), 70),
    (ModelSpec(2, 3, 7, 128), HamSpec("j1j2", J1=1.0, J2=0.0), 60),
    (ModelSpec(2, 4, 4, 128, cplx=1, marshall=1, zmask=1), HamSpec("j1j2", J1=1.0, J2=0.5), 50),
]


@pytest.mark.parametrize("model,ham,ns", E2DJT_MODELS,
                         ids=["5x3_dh32_c", "4x5_dh96_cmask", "3x7_dh128", "4x4_dh128_cmask"])
def test_jacobian_2d_tensor_core_blocks_mixed(model, ham, ns):
    from paper_2608_18065_b300.inputs import param_blocks
    c = ctx(model, ham, "mixed", ns)
    th, thd = theta_dev(model, 8)
    sp = random_spins(model, ns, seed=17, zero_mag=bool(model.zmask))
    J = c.jacobian(thd, torch.tensor(sp, device="cuda")).cpu().numpy().astype(np.float64)
    J_o = O.jacobian(model, th, sp)
    assert J.shape == J_o.shape
    scale = np.max(np.abs(J_o), axis=1, keepdims=True)
    assert np.max(np.abs(J - J_o) / scale) < TOL_MIXED_JAC
    # block by block against each block's own largest entry
    off = 0
    for name, r, cols, _ in param_blocks(model):
        sl = slice(off, off + r * cols)
        off += r * cols
        bmax = np.max(np.abs(J_o[:, sl]))
        assert np.max(np.abs(J[:, sl] - J_o[:, sl])) <= 5e-3 * bmax, name
    record_error(f"jac2d_tc_{model.Lx}x{model.Ly}_dh{model.dh}", O_row=max_row_err(J, J_o))


def test_refinement_falls_back_to_fp64_when_fp32_factor_fails():
    """A matrix whose FP32 Cholesky breaks down (kappa ~ 1e12) but is SPD in
    FP64: the mixed context must still return the FP64 solution."""
    model, ham = ModelSpec(1, 8, 1, 8), HamSpec("tfim")
    c = ctx(model, ham, "mixed", 64)
    R = 64
    rng = np.random.default_rng(1)
    Q, _ = np.linalg.qr(rng.standard_normal((R, R)))
    ev = np.logspace(0, -12, R)
    T = (Q * ev) @ Q.T
    T = 0.5 * (T + T.T)
    b = rng.standard_normal(R)
    x, st = c.regularized_solve(torch.tensor(T, device="cuda"), 0.0,
                                torch.tensor(b, device="cuda"))
    assert int(st.item()) == 0
    xr = np.linalg.solve(T, b)
    kappa = np.linalg.cond(T)
    assert rel_err(x.cpu().numpy(), xr) < 100 * kappa * 2.2e-16


@pytest.mark.parametrize("R", [256, 260, 1000, 2304])
def test_regularized_solve_128_wide_panels(R):
    """Mixed context, the 128-wide panel form (two panels at R = 256; ragged
    last blocks of 4 and 104 rows at 260 and 1000): the FP32 factor with
    explicitly inverted 128 x 128 diagonal blocks and the FP64 refinement
    reach the FP64 solution at FP64 backward error; an indefinite matrix
    reports NOT_SPD; a matrix whose FP32 factor breaks down (kappa ~ 1e12)
    is solved by the FP64 Cholesky that follows."""
    model, ham = ModelSpec(1, 8, 1, 8), HamSpec("tfim")
    c = ctx(model, ham, "mixed", R)
    c.set_solve_form(2)
    rng = np.random.default_rng(R + 7)
    M = rng.standard_normal((R, R + 5))
    T = M @ M.T / R
    b = rng.standard_normal(R)
    lam = 1e-2
    x, st = c.regularized_solve(torch.tensor(T, device="cuda"), lam, torch.tensor(b, device="cuda"))
    assert int(st.item()) == 0
    A = T + lam * np.eye(R)
    xr = np.linalg.solve(A, b)
    kappa = np.linalg.cond(A)
    xg = x.cpu().numpy()
    assert rel_err(xg, xr) < max(1e-10, 100 * kappa * 2.2e-16)
    berr = np.max(np.abs(A @ xg - b)) / (np.max(np.abs(A).sum(1)) * np.max(np.abs(xg)))
    assert berr < 100 * np.sqrt(R) * 1.11e-16
    x, st = c.regularized_solve(torch.tensor(-T - np.eye(R), device="cuda"), 0.0,
                                torch.tensor(b, device="cuda"))
    assert int(st.item()) == 5
    Q, _ = np.linalg.qr(rng.standard_normal((R, R)))
    Ts = (Q * np.logspace(0, -12, R)) @ Q.T
    Ts = 0.5 * (Ts + Ts.T)
    x, st = c.regularized_solve(torch.tensor(Ts, device="cuda"), 0.0, torch.tensor(b, device="cuda"))
    assert int(st.item()) == 0
    xr = np.linalg.solve(Ts, b)
    assert rel_err(x.cpu().numpy(), xr) < 100 * np.linalg.cond(Ts) * 2.2e-16


# hidden sizes whose weights do not fit shared memory (read through L1)
BIG = [
    (ModelSpec(1, 10, 1, 96), HamSpec("tfim")),
    (ModelSpec(1, 9, 1, 128, cplx=1), HamSpec("cluster_zxz")),
    (ModelSpec(2, 4, 4, 128, cplx=1, marshall=1, zmask=1), HamSpec("j1j2", J2=0.25)),
    (ModelSpec(2, 4, 3, 96, cplx=1, marshall=1, zmask=1), HamSpec("j1j2", J2=0.6)),
    # the paper's cluster-state hidden size (Tab. I): 32 lanes x 8 units per
    # thread in the sweeps, 2 x 2 sub-blocks per pass in the O assembly
    (ModelSpec(1, 8, 1, 256, cplx=1), HamSpec("cluster_paper")),
    (ModelSpec(2, 3, 4, 256, cplx=1, marshall=1, zmask=1), HamSpec("j1j2", J2=0.5)),
    # and the 2D one (200 = 8 lanes x 25 units; O in 10 x 10 tiles)
    (ModelSpec(2, 4, 3, 200, marshall=1, zmask=1), HamSpec("j1j2", J2=0.0)),
    (ModelSpec(1, 9, 1, 200), HamSpec("tfim")),
]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("model,ham", BIG, ids=["1d96", "1d128", "2d128", "2d96", "1d256", "2d256",
                                                "2d200", "1d200"])
def test_large_hidden_sizes(model, ham, prec):
    ns = 37
    c = ctx(model, ham, prec, ns)
    th, thd = theta_dev(model, 8)
    sp = random_spins(model, ns, seed=2, zero_mag=bool(model.zmask))
    spd = torch.tensor(sp, device="cuda")
    lp = cplx(c.logpsi(thd, spd))
    el = cplx(c.local_energy(thd, spd))
    J = c.jacobian(thd, spd).cpu().numpy().astype(np.float64)
    lp_o, el_o, J_o = O.logpsi(model, th, sp), O.local_energy(model, ham, th, sp), O.jacobian(model, th, sp)
    if prec == "fp64":
        np.testing.assert_allclose(lp, lp_o, rtol=RTOL64, atol=RTOL64)
        assert rel_err(el, el_o) < RTOL64
        assert rel_err(J, J_o) < RTOL64
    else:
        assert np.max(np.abs(lp - lp_o)) < TOL_MIXED_LOGPSI
        assert rel_err(el, el_o) < TOL_MIXED_ELOC
        assert max_elem_err(el, el_o) < TOL_MIXED_ELOC
        assert rel_err(J, J_o) < TOL_MIXED_JAC
        assert max_row_err(J, J_o) < TOL_MIXED_JAC


def test_large_hidden_size_step_fp64():
    model, ham = ModelSpec(2, 4, 4, 128, cplx=1, marshall=1, zmask=1), HamSpec("j1j2", J2=0.5)
    hp = HParams(0.1, 1e4, 0.1, lam=0.1, trust_region=1, ns=48)
    c = ctx(model, ham, "fp64", hp.ns)
    th, thd = theta_dev(model, 1234)
    momd = torch.zeros_like(thd)
    outs = c.step_outputs(hp.ns)
    c.minsr_step(thd, momd, hp, 0, outputs=outs)
    torch.cuda.synchronize()
    th1, _, st_o, b = O.minsr_step(model, ham, th, np.zeros_like(th), hp, 0, want=("spins", "dtheta"))
    assert np.array_equal(outs["spins"].cpu().numpy(), b["spins"])
    assert rel_err(outs["dtheta"].cpu().numpy(), b["dtheta"]) < 1e-9
    assert rel_err(thd.cpu().numpy(), th1) < 1e-9


@pytest.mark.parametrize("R", [2090, 2304])
def test_regularized_solve_block_substitution(R):
    """Mixed context, R >= 2048: refinement sweeps by block substitution with
    the inverted 32 x 32 diagonal blocks (ragged last block for R = 2090)
    reach the FP64 solution; an indefinite matrix still reports NOT_SPD."""
    model, ham = ModelSpec(1, 8, 1, 8), HamSpec("tfim")
    c = ctx(model, ham, "mixed", R)
    rng = np.random.default_rng(R)
    M = rng.standard_normal((R, R + 5))
    T = M @ M.T / R
    b = rng.standard_normal(R)
    lam = 1e-2
    x, st = c.regularized_solve(torch.tensor(T, device="cuda"), lam, torch.tensor(b, device="cuda"))
    assert int(st.item()) == 0
    A = T + lam * np.eye(R)
    xr = np.linalg.solve(A, b)
    kappa = np.linalg.cond(A)
    xg = x.cpu().numpy()
    assert rel_err(xg, xr) < max(1e-10, 100 * kappa * 2.2e-16)
    berr = np.max(np.abs(A @ xg - b)) / (np.max(np.abs(A).sum(1)) * np.max(np.abs(xg)))
    assert berr < 100 * np.sqrt(R) * 1.11e-16
