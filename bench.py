#!/usr/bin/env python
"""Benchmark: regularized minSR steps/s on one B300 (and N replicas).

Workload (default): 1D transverse-field Ising open chain, N = 100, h = J = 1,
GRU hidden size 64 (Np = 13058), Ns = 1024 samples, mixed precision (FP32
recurrence and Jacobian, BF16x3 tensor-core Gram, FP64 centring and solve),
Tab. I TFIM hyper-parameters.  One step = one iteration of Algorithm 1
(sampling, local energies, O, centring, T, regularized solve, momentum,
update) through nqs_minsr_step.

Prints one JSON line.  `--impl reference` times the FP64 CPU oracle instead
(bounded per-step sample of the same workload, scaled to steps/s).
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "minSR steps/s & Gram TFLOP/s vs plain FP64 GPU path at matched energy error"
UNIT = "steps/s"
FP32_ALU_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12  # SMs x FP32 lanes x 2 x max SM clock
FP64_PEAK_TFLOPS = 148 * 2 * 2 * 2.032e9 / 1e12    # SMs x FP64 lane-FMAs x 2 x max SM clock


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="tfim100")
    p.add_argument("--matched-steps", type=int, default=60,
                   help="steps of the mixed and FP64 paths for the matched-energy check (0: skip)")
    p.add_argument("--matched-eta0", type=float, default=0.1,
                   help="eta0 of the matched-energy runs (Tab. I's 0.5 collapses this model "
                        "onto the product state within ~30 steps for both paths)")
    p.add_argument("--fp64-steps", type=int, default=3)
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-spectrum", action="store_true",
                   help="skip the conditioning diagnostics of T (App. E)")
    p.add_argument("--spectrum-steps", type=int, default=64,
                   help="Lanczos steps of the conditioning diagnostics")
    p.add_argument("--no-graph", action="store_true", help="launch every kernel eagerly")
    return p.parse_args()


# ----------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.path = tempfile.mktemp(suffix=".csv")
        self.idx = gpu_index
        self.proc = None

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------- algorithmic
def site_flops(model):
    """FMA-pipe flops of one site of one configuration (x2 per FMA): the
    gate products 3dh x dh, the 2D state mix 2 dh x dh, the output heads."""
    dh = model.dh
    f = 2 * 3 * dh * dh + 2 * 2 * dh * (2 if model.cplx else 1)
    if model.dim == 2:
        f += 2 * 2 * dh * dh
    return f


def eloc_suffix_sites(w):
    """Sites recomputed per step by the connected-configuration engine for
    Hamiltonians whose connectivity does not depend on the sample."""
    N, ns = w.model.N, w.hp.ns
    if w.ham.family == "tfim":
        return ns * sum(N - j for j in range(N))
    if w.ham.family == "cluster_zxz":
        return ns * sum(N - i for i in range(1, N - 1))
    return None


def src_sha(*rel):
    h = hashlib.sha256()
    for r in rel:
        h.update(open(os.path.join(ROOT, r), "rb").read())
    return h.hexdigest()[:16]


def load_traffic(kernel, sha, workload):
    p = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p)).get(kernel)
    except (ValueError, OSError):
        return None
    if d and d.get("src_sha") == sha and d.get("workload") == workload:
        return d.get("bytes_per_launch")
    return None


def spectrum_diagnostics(ctx, w, hp, th0, dev, m=64, reps=5):
    """kappa_2(T + lambda I), lambda_max(T) and the reliable digits (App. E)
    of the T of one eager step from theta_0 (nqs_spectrum, m Lanczos steps,
    the step's own lambda), with the kernel's CUDA-event time over reps
    back-to-back launches and the rate of its dominant traffic: one product
    T v per Lanczos step, R^2 FP64 reads each (T stays resident in L2)."""
    import ctypes as C
    import torch
    from paper_2608_18065_b300 import nqs
    th = torch.tensor(th0, device=dev)
    outs = ctx.step_outputs(hp.ns)
    stats = ctx.minsr_step(th, torch.zeros_like(th), hp, 0, outputs=outs)
    torch.cuda.synchronize()
    lam = nqs.decode_stats(stats)["lam"]
    T = outs["T"]
    R = T.shape[0]
    st = nqs.spectrum(T, lam, m=m)
    lib = nqs.lib()
    wb = lib.nqs_spectrum_workspace(R, m)
    work = torch.empty(wb, dtype=torch.uint8, device=dev)
    out = torch.zeros(C.sizeof(nqs.SpectrumStats), dtype=torch.uint8, device=dev)
    args = (nqs._ptr(T), C.c_int64(R), C.c_double(lam), C.c_int(m), C.c_uint64(1),
            nqs._ptr(work), C.c_size_t(wb), nqs._ptr(out), nqs._stream())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        nqs._check(lib.nqs_spectrum(*args))
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    byts = st["iterations"] * R * R * 8
    return {"kernel": "k_lanczos", "R": R, "m": m, "iterations": st["iterations"],
            "lambda": lam, "lambda_max": st["lambda_max"],
            "lambda_min_ritz": st["lambda_min_ritz"], "kappa": st["kappa"],
            "digits_fp32": st["digits_fp32"], "digits_fp64": st["digits_fp64"],
            "ritz_residual": st["residual"], "status": st["status"],
            "ms": ms, "tv_bytes": byts, "tv_gbs": byts / (ms * 1e-3) / 1e9}


def measured_peak(key, fallback):
    """A peak from the measured MEASURED_PEAKS.json beside this file,
    else the stated fallback; returns (value, source)."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        v = json.load(open(p)).get(key)
        if v:
            return float(v), f"measured ({key})"
    except (ValueError, OSError):
        pass
    return fallback, "fallback"


def eloc_tc_used(model, precision):
    """The connected-configuration engine runs on tcgen05 for mixed 1D chains
    of hidden size 64, and 32 (run with its units padded to 64: the issued
    tensor work per site is that of 64), and for mixed 2D lattices of hidden
    size 64."""
    if precision != "mixed":
        return False
    return (model.dim == 1 and model.dh in (32, 64)) or (model.dim == 2 and model.dh == 64)


def eloc_tc_site_flops(model):
    """Tensor-pipe flops issued per recomputed site of one configuration:
    three BF16 products (hi.hi + hi.lo + lo.hi) of the gate product
    [1 x 64] x [64 x 192], and in 2D also of the state mix [1 x 128] x [128 x 64]."""
    k = 3 * 64 + (2 * 64 if model.dim == 2 else 0)
    return 3 * 2 * 64 * k


def eloc_roofline(w, ms, sites=None):
    """Roofline of the connected-configuration engine for one launch.

    Tensor-core engine: per recomputed site of one connected configuration
    the gate product [1 x dh] x [dh x 3dh] is issued as three BF16 MMAs
    (hi.hi + hi.lo + lo.hi), 3 * 2 * dh * 3dh tensor-pipe flops; bound by
    the measured sustained BF16 rate.  SIMT engine: FP32 FMA-pipe flops of
    the recurrence against the derived FP32 peak."""
    if sites is None:
        sites = eloc_suffix_sites(w)
    if sites is None:
        return None
    dh = w.model.dh
    alg = sites * site_flops(w.model)
    if eloc_tc_used(w.model, w.precision):
        fl = sites * eloc_tc_site_flops(w.model)
        peak, src = measured_peak("bf16_tflops_sustained", 1400.0)
        ach = fl / (ms * 1e-3) / 1e12
        kern = "k_eloc_tc" if w.model.dim == 1 else "k_eloc2d_tc"
        sha = src_sha("paper_2608_18065_b300/csrc/%s.cu" % kern[2:],
                      "paper_2608_18065_b300/csrc/tc_common.cuh")
        return {"kernel": kern + " (eloc_suffix)", "bound": "tensor", "achieved": ach,
                "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": load_traffic(kern, sha, w.name),
                "peak_source": src + ", BF16 dense, sustained",
                "flops_per_launch": fl, "fp32_equiv_flops_per_launch": alg,
                "fp32_equiv_tflops": alg / (ms * 1e-3) / 1e12, "ms_per_launch": ms}
    ach = alg / (ms * 1e-3) / 1e12
    sha = src_sha("paper_2608_18065_b300/csrc/recurrence.cuh",
                  "paper_2608_18065_b300/csrc/recur_impl.cuh")
    return {"kernel": "k_forward<MODE_ELOC> (eloc_suffix)", "bound": "alu",
            "achieved": ach, "peak": FP32_ALU_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": ach / FP32_ALU_PEAK_TFLOPS,
            "traffic": load_traffic("k_forward_eloc", sha, w.name),
            "peak_source": "148 SMs x 128 FP32 lanes x 2 flop x 2032 MHz (derived)",
            "flops_per_launch": alg, "ms_per_launch": ms}


def stage_rooflines(w, ms, sites, R, np_):
    """Per-stage rooflines of one step (ms: stage -> ms per step).

    eloc_suffix: see eloc_roofline (sites = recomputed sites counted by the
    library).  sample, jac_bwd, jac_grad: FP32 (FP64) FMA-pipe work of the
    recurrence, N_s N (sample) or R N (reverse sweep, O assembly) sites of
    site_flops each (the mixed 1D O assembly on the tensor cores is
    reported by its HBM bytes).  cholesky: n^3/3 factor + n^3/3 triangular inverse
    (n = R) in FP32 for the mixed path (refinement sweeps: 2n^2 each, not
    counted).  gram: BF16x3 tensor work 3 R(R+1) Np.  center: HBM bytes of
    the column sums and the split (read O twice, write hi and lo)."""
    out = {}
    f32 = w.precision == "mixed"
    alu_peak = FP32_ALU_PEAK_TFLOPS if f32 else FP64_PEAK_TFLOPS
    alu_src = ("148 SMs x 128 FP32 lanes x 2 flop x 2032 MHz (derived)" if f32 else
               "148 SMs x 2 FP64 lane-FMAs x 2 flop x 2032 MHz (derived; 0.94 measured)")
    sf = site_flops(w.model)
    N = w.model.N

    def alu(name, kernel, flops):
        t = ms.get(name, 0.0)
        if t <= 0:
            return
        a = flops / (t * 1e-3) / 1e12
        out[name] = {"kernel": kernel, "bound": "alu", "achieved": a, "peak": alu_peak,
                     "unit": "TFLOP/s", "frac": a / alu_peak, "traffic": None,
                     "peak_source": alu_src, "flops_per_launch": flops, "ms_per_launch": t}

    if ms.get("eloc_suffix", 0) > 0 and sites:
        if eloc_tc_used(w.model, w.precision):
            out["eloc_suffix"] = eloc_roofline(w, ms["eloc_suffix"], sites)
        else:
            alu("eloc_suffix", "k_forward<MODE_ELOC>", sites * sf)
    alu("sample", "k_forward<MODE_SAMPLE>", w.hp.ns * N * sf)
    alu("jac_bwd", "k_jac_bwd", R * N * sf)
    if f32 and w.model.dim == 1 and w.model.dh in (32, 64) and ms.get("jac_grad", 0) > 0:
        # tensor-core O assembly: HBM-bound reads of the adjoint records and
        # states, write of O
        t = ms["jac_grad"]
        dh = w.model.dh
        byts = R * N * (4 * dh + 4) * 4 + w.hp.ns * N * dh * 4 + R * np_ * 4
        pk, src = measured_peak("hbm_gbs", 6400.0)
        a = byts / (t * 1e-3) / 1e9
        out["jac_grad"] = {"kernel": "k_jac_tc", "bound": "hbm", "achieved": a, "peak": pk,
                           "unit": "GB/s", "frac": a / pk, "traffic": None, "peak_source": src,
                           "bytes_per_launch": byts, "ms_per_launch": t}
    else:
        alu("jac_grad", "k_jac_grad", R * N * sf)
    alu("cholesky", "k_chol_ir" if f32 else "k_chol_coop", 2 * R ** 3 / 3)
    if ms.get("gram", 0) > 0:
        t = ms["gram"]
        if f32:
            pk, src = measured_peak("bf16_tflops_sustained", 1400.0)
            a = 3 * R * (R + 1) * np_ / (t * 1e-3) / 1e12
            out["gram"] = {"kernel": "k_gram_bf16x3 + k_gram_reduce", "bound": "tensor",
                           "achieved": a, "peak": pk, "unit": "TFLOP/s", "frac": a / pk,
                           "traffic": None, "peak_source": src + ", BF16 dense, sustained",
                           "ms_per_launch": t}
        else:
            alu("gram", "k_gram_simt<double>", R * (R + 1) * np_)
    if ms.get("center", 0) > 0:
        t = ms["center"]
        kpad = (np_ + 63) // 64 * 64
        byts = R * np_ * (4 if f32 else 8) * 2 + (R * kpad * 4 if f32 else R * np_ * 8)
        pk, src = measured_peak("hbm_gbs", 6400.0)
        a = byts / (t * 1e-3) / 1e9
        out["center"] = {"kernel": "k_colsum_part + k_colmean_fin + " +
                         ("k_center_split" if f32 else "k_center"), "bound": "hbm",
                         "achieved": a, "peak": pk, "unit": "GB/s", "frac": a / pk,
                         "traffic": None, "peak_source": src, "bytes_per_launch": byts,
                         "ms_per_launch": t}
    return out


# ------------------------------------------------------------------ oracle
def oracle_bounded(w, budget_s, seed_step=0):
    """Time oracle steps on a sample of Ns_sub configurations sized to the
    budget; returns (steps/s scaled to the full Ns, Ns_sub, seconds, threads)."""
    import copy
    from oracle import oracle as O
    from paper_2608_18065_b300.inputs import init_theta
    th = init_theta(w.model, w.theta_seed)
    hp = copy.copy(w.hp)
    hp.ns = 8
    t0 = time.perf_counter()
    O.minsr_step(w.model, w.ham, th, np.zeros_like(th), hp, seed_step)
    per_sample = (time.perf_counter() - t0) / 8
    ns_sub = int(max(8, min(w.hp.ns, budget_s / max(per_sample, 1e-9))))
    hp.ns = ns_sub
    t0 = time.perf_counter()
    O.minsr_step(w.model, w.ham, th, np.zeros_like(th), hp, seed_step)
    dt = time.perf_counter() - t0
    scale = w.hp.ns / ns_sub
    return 1.0 / (dt * scale), ns_sub, dt, O.num_threads()


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2608_18065_b300.inputs import batched_instances, workloads
    if args.workload == "batched16":
        return run_reference_batched(args)
    w = workloads()[args.workload]
    budget = max(2.0, 150.0 / max(1, args.steps + args.warmup))
    for t in range(args.warmup):
        oracle_bounded(w, budget, t)
    vals, subs, secs, thr = [], [], [], 1
    for t in range(args.steps):
        v, sub, dt, thr = oracle_bounded(w, budget, args.warmup + t)
        vals.append(v); subs.append(sub); secs.append(dt)
    value = float(np.mean(vals))
    sample = (f"one oracle step per timed step on Ns_sub={min(subs)}..{max(subs)} of the "
              f"{w.hp.ns} samples (same model, Hamiltonian, theta_0), time scaled by "
              f"{w.hp.ns}/Ns_sub (sampling, local energies and O are linear in Ns)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 / value, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": w.describe(),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": thr, "kind": "oracle",
                             "sample": sample, "cpu": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_reference_batched(args):
    """Oracle arm of the batched workload: per timed step one bounded oracle
    step of every instance, each scaled to its full Ns, summed."""
    from paper_2608_18065_b300.inputs import batched_instances
    insts = batched_instances()
    budget = max(0.3, 150.0 / max(1, args.steps + args.warmup) / len(insts))
    vals, thr, subs = [], 1, []
    for t in range(args.warmup + args.steps):
        tot = 0.0
        for w in insts:
            v, sub, dt, thr = oracle_bounded(w, budget, t)
            tot += 1.0 / v
            subs.append(sub)
        if t >= args.warmup:
            vals.append(1.0 / tot)
    value = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "batched steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 / value, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "batched16_j1j2", "instances": [w.name for w in insts],
                       "n_instances": len(insts), "precision": "fp64"},
            "cpu_baseline": {"value": value, "unit": "batched steps/s", "cores": thr,
                             "kind": "oracle",
                             "sample": (f"one oracle step per instance per timed step on "
                                        f"Ns_sub={min(subs)}..{max(subs)} samples, each scaled "
                                        "to its full Ns, summed over the 16 instances"),
                             "cpu": cpu_model()},
            "e2e": {"value": value, "unit": "batched steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# -------------------------------------------------------------------- ours
def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2608_18065_b300 import nqs
    from paper_2608_18065_b300.inputs import init_theta, workloads
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workloads()[args.workload]
    hp = w.hp
    K, Wu = args.steps, args.warmup

    def barrier():
        if world > 1:
            dist.barrier()

    # replica r: its own Philox key (seed + r), same theta_0
    import copy
    from paper_2608_18065_b300.replicas import aggregate_rate, max_over_ranks, replica_hparams
    hp = replica_hparams(hp, rank)
    ctx = nqs.Context(w.model, w.ham, w.precision, hp.ns, device=dev)
    ctx.use_graph(not args.no_graph)
    th0 = init_theta(w.model, w.theta_seed)
    thd = torch.tensor(th0, device=dev)
    momd = torch.zeros_like(thd)
    stats = ctx.new_stats()
    for t in range(Wu):
        ctx.minsr_step(thd, momd, hp, t, stats)
    torch.cuda.synchronize()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = ctx.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier()
    e0.record()
    for t in range(Wu, Wu + K):
        ctx.minsr_step(thd, momd, hp, t, stats)
    e1.record()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    graph_used = ctx.graph_active()
    # kernels per step, counted by the library on the eager path (a graph
    # replay launches the same kernels as one graph)
    ctx.timing_begin(min(K, 10))
    lt0 = ctx.launch_count()
    for t in range(Wu + K, Wu + K + min(K, 10)):
        ctx.minsr_step(thd, momd, hp, t, stats)
    torch.cuda.synchronize()
    per_step = (ctx.launch_count() - lt0) / min(K, 10)
    launches = int(round(per_step * K))
    stage_ms, nt = ctx.timing_end()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    st = nqs.decode_stats(stats)
    value = aggregate_rate(world, K, ms)
    ms_step = ms / K

    # Gram throughput (symmetric algorithmic count R(R+1)Np)
    R = hp.ns * (2 if w.model.cplx else 1)
    gram_ms = stage_ms["gram"] / max(nt, 1)
    gram_tflops = R * (R + 1) * ctx.np / (gram_ms * 1e-3) / 1e12 if gram_ms > 0 else None
    gram = None
    if gram_tflops:
        pk, src = measured_peak("bf16_tflops_sustained", 1400.0)
        tc = w.precision == "mixed"
        gram = {"tflops_symmetric": gram_tflops, "ms": gram_ms,
                "mma_tflops": 3 * gram_tflops if tc else None,
                "frac_of_bf16": 3 * gram_tflops / pk if tc else None,
                "peak_source": src if tc else None}

    # roofline of every large stage; the dominant one is the headline
    cfg, sites = ctx.eloc_work()
    kernels = stage_rooflines(w, {k: v / max(nt, 1) for k, v in stage_ms.items()}, sites, R,
                              ctx.np)
    dom = max(stage_ms, key=lambda k: stage_ms[k])
    roof = kernels.get(dom) or {"kernel": dom, "bound": None, "achieved": None, "peak": None,
                                "unit": None, "frac": None, "traffic": None,
                                "ms_per_launch": stage_ms[dom] / max(nt, 1)}

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        th_h = thd.cpu().pin_memory()
        m_h = momd.cpu().pin_memory()
        st_h = torch.empty_like(stats, device="cpu").pin_memory()
        torch.cuda.synchronize()
        barrier()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record()
        for t in range(Wu + K + 10, Wu + 2 * K + 10):
            thd.copy_(th_h, non_blocking=True)
            momd.copy_(m_h, non_blocking=True)
            ctx.minsr_step(thd, momd, hp, t, stats)
            th_h.copy_(thd, non_blocking=True)
            m_h.copy_(momd, non_blocking=True)
            st_h.copy_(stats, non_blocking=True)
        a1.record()
        torch.cuda.synchronize()
        ems = max_over_ranks(a0.elapsed_time(a1), dist, dev)
        e2e = {"value": aggregate_rate(world, K, ems), "unit": UNIT,
               "h2d_bytes_per_step": 2 * ctx.np * 8,
               "d2h_bytes_per_step": 2 * ctx.np * 8 + stats.numel() * 8}

    # plain FP64 GPU path on the same workload
    fp64 = None
    if args.fp64_steps > 0:
        c64 = nqs.Context(w.model, w.ham, "fp64", hp.ns, device=dev)
        t64 = torch.tensor(th0, device=dev)
        m64 = torch.zeros_like(t64)
        s64 = c64.new_stats()
        c64.minsr_step(t64, m64, hp, 0, s64)
        torch.cuda.synchronize()
        c64.timing_begin(args.fp64_steps)
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record()
        for t in range(1, 1 + args.fp64_steps):
            c64.minsr_step(t64, m64, hp, t, s64)
        b1.record()
        torch.cuda.synchronize()
        sm64, n64 = c64.timing_end()
        f_ms = b0.elapsed_time(b1) / args.fp64_steps
        g64 = sm64["gram"] / max(n64, 1)
        fp64 = {"steps_per_s": 1000.0 / f_ms, "ms_per_step": f_ms,
                "gram_tflops": R * (R + 1) * ctx.np / (g64 * 1e-3) / 1e12 if g64 > 0 else None,
                "stage_ms": {k: v / max(n64, 1) for k, v in sm64.items()},
                "speedup_mixed_over_fp64": (1000.0 / ms_step) / (1000.0 / f_ms)}
        del c64

    # conditioning diagnostics of the step's T (App. E), outside the timed
    # region: lambda_max by Lanczos, kappa_2 and the reliable digits
    spec = None
    if not args.no_spectrum and rank == 0:
        spec = spectrum_diagnostics(ctx, w, hp, th0, dev, m=args.spectrum_steps)

    # matched energy error: both paths from theta_0 with the same seeds
    matched = None
    if args.matched_steps > 0 and rank == 0:
        hpm = copy.copy(hp)
        hpm.eta0 = args.matched_eta0
        matched = matched_energy(w, hpm, args.matched_steps, dev)

    cpu = None
    if not args.no_cpu and rank == 0:
        v, sub, dt, thr = oracle_bounded(w, 20.0)
        cpu = {"value": v, "unit": UNIT, "cores": thr, "kind": "oracle",
               "sample": (f"one FP64 oracle step on Ns_sub={sub} of the {hp.ns} samples "
                          f"({dt:.1f} s), scaled by {hp.ns}/{sub}"), "cpu": cpu_model()}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
                "warmup": Wu, "ms_per_step": ms_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16x3+f64",
                "data": "synthetic",
                "config": dict(w.describe(), l2="step working set > 126 MB L2 (O, caches, adjoints)",
                               replicas=world, workspace_mb=ctx.workspace_bytes / 2**20),
                "gram_tflops": gram_tflops, "gram": gram,
                "roofline": roof, "kernels": kernels, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches,
                "clocks": clk, "cuda_graph": graph_used, "fp64_path": fp64,
                "matched_energy": matched, "spectrum": spec,
                "stage_ms": {k: v / max(nt, 1) for k, v in stage_ms.items()},
                "final_stats": st}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_batched(args):
    """Batched J1-J2 workload: 16 heterogeneous 2D instances (L in {6..12},
    J2 in {0, .25, .5, .6}, Ns in {256..4096}, dh in {32..128}) stepped
    together by nqs_minsr_step_batched (one graph per batched step, launch
    shapes from the autotuner); value = batched steps/s (x16 instance steps)."""
    import copy
    import torch
    import torch.distributed as dist
    from paper_2608_18065_b300 import nqs
    from paper_2608_18065_b300.inputs import batched_instances, init_theta, param_count
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    insts = batched_instances()
    n = len(insts)
    K, Wu = args.steps, args.warmup

    def barrier():
        if world > 1:
            dist.barrier()

    ctxs = [nqs.Context(w.model, w.ham, "mixed", w.hp.ns, device=dev) for w in insts]
    th0 = [init_theta(w.model, w.theta_seed) for w in insts]
    thd = [torch.tensor(t, device=dev) for t in th0]
    mod = [torch.zeros_like(t) for t in thd]
    from paper_2608_18065_b300.replicas import aggregate_rate, max_over_ranks, replica_hparams
    hps = [replica_hparams(w.hp, rank) for w in insts]
    b = nqs.Batch(ctxs)
    b.use_graph(not args.no_graph)
    t0 = time.perf_counter()
    tune_ms = b.autotune(thd, hps, 0)
    tune_s = time.perf_counter() - t0
    tuning = [c.tuning() for c in ctxs]
    stats = b.new_stats()
    for t in range(Wu):
        b.step(thd, mod, hps, t, stats)
    torch.cuda.synchronize()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier()
    e0.record()
    for t in range(Wu, Wu + K):
        b.step(thd, mod, hps, t, stats)
    e1.record()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    value = aggregate_rate(world, K, ms)
    st = [nqs.decode_stats(stats[i]) for i in range(n)]

    # per-instance stage times: every instance alone, eager, one step
    solo = []
    tot_stage = {}
    eloc_ms = eloc_flops = gram_ms = gram_fl = 0.0
    launches = 0
    for i, (c, w) in enumerate(zip(ctxs, insts)):
        c.timing_begin(1)
        l0 = c.launch_count()
        s1 = c.new_stats()
        c.minsr_step(thd[i], mod[i], hps[i], Wu + K, s1)
        torch.cuda.synchronize()
        launches += c.launch_count() - l0
        sm, nt = c.timing_end()
        cfg, sites = c.eloc_work()
        R = w.hp.ns * (2 if w.model.cplx else 1)
        np_ = param_count(w.model)
        for k, v in sm.items():
            tot_stage[k] = tot_stage.get(k, 0.0) + v
        eloc_ms += sm["eloc_suffix"]
        eloc_flops += sites * site_flops(w.model)
        gram_ms += sm["gram"]
        gram_fl += R * (R + 1) * np_
        solo.append({"instance": w.name, "ms": sum(sm.values()), "eloc_configs": cfg,
                     "workspace_mb": round(c.workspace_bytes / 2**20, 1),
                     "eloc_sites": sites, "E_re": st[i]["E_re"], "status": st[i]["status"],
                     "tuning": {k: tuning[i][k] for k in ("eloc_grid", "gram_splits", "solve_grid")}})
    solo_ms = sum(x["ms"] for x in solo)
    dom = max(tot_stage, key=lambda k: tot_stage[k])
    roof = None
    if dom == "eloc_suffix" and eloc_ms > 0:
        ach = eloc_flops / (eloc_ms * 1e-3) / 1e12
        roof = {"kernel": "2D E_loc engines (eloc_suffix, all instances; k_eloc2d_tc for "
                          "mixed d_h = 64, k_forward<MODE_ELOC> otherwise; FP32-equivalent flops)",
                "bound": "alu",
                "achieved": ach, "peak": FP32_ALU_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / FP32_ALU_PEAK_TFLOPS, "traffic": None,
                "peak_source": "148 SMs x 128 FP32 lanes x 2 flop x 2032 MHz (derived)",
                "flops_per_batch": eloc_flops, "ms_per_batch": eloc_ms}
    if roof is None:
        roof = {"kernel": dom, "bound": None, "achieved": None, "peak": None, "unit": None,
                "frac": None, "traffic": None, "ms_per_batch": tot_stage[dom]}

    # end to end: every instance's theta and momentum from and back to pinned host memory
    e2e = None
    if not args.no_e2e:
        th_h = [t.cpu().pin_memory() for t in thd]
        m_h = [m.cpu().pin_memory() for m in mod]
        st_h = torch.empty_like(stats, device="cpu").pin_memory()
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record()
        for t in range(Wu + K + 1, Wu + 2 * K + 1):
            for i in range(n):
                thd[i].copy_(th_h[i], non_blocking=True)
                mod[i].copy_(m_h[i], non_blocking=True)
            b.step(thd, mod, hps, t, stats)
            for i in range(n):
                th_h[i].copy_(thd[i], non_blocking=True)
                m_h[i].copy_(mod[i], non_blocking=True)
            st_h.copy_(stats, non_blocking=True)
        a1.record()
        torch.cuda.synchronize()
        ems = max_over_ranks(a0.elapsed_time(a1), dist, dev)
        nbytes = sum(t.numel() * 8 for t in thd) * 2
        e2e = {"value": aggregate_rate(world, K, ems), "unit": "batched steps/s",
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes + stats.numel() * 8}

    # the same instances one at a time on the plain FP64 GPU path
    fp64 = None
    if args.fp64_steps > 0:
        f_ms = 0.0
        per = []
        for i, w in enumerate(insts):
            c64 = nqs.Context(w.model, w.ham, "fp64", w.hp.ns, device=dev)
            t64 = torch.tensor(th0[i], device=dev)
            m64 = torch.zeros_like(t64)
            s64 = c64.new_stats()
            b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            b0.record()
            for t in range(args.fp64_steps):
                c64.minsr_step(t64, m64, hps[i], t, s64)
            b1.record()
            torch.cuda.synchronize()
            d = b0.elapsed_time(b1) / args.fp64_steps
            f_ms += d
            per.append(round(d, 3))
            del c64
        fp64 = {"batched_steps_per_s": 1000.0 / f_ms, "ms_per_batched_step": f_ms,
                "instance_ms": per, "steps_per_instance": args.fp64_steps,
                "speedup_mixed_batched_over_fp64": (1000.0 * K / ms) / (1000.0 / f_ms)}

    cpu = None
    if not args.no_cpu and rank == 0:
        tot_s, subs, thr = 0.0, [], 1
        for w in insts:
            v, sub, dt, thr = oracle_bounded(w, 1.5)
            tot_s += 1.0 / v
            subs.append(sub)
        cpu = {"value": 1.0 / tot_s, "unit": "batched steps/s", "cores": thr, "kind": "oracle",
               "sample": (f"one FP64 oracle step per instance on Ns_sub={min(subs)}..{max(subs)} "
                          "samples, each scaled to its full Ns, summed over the 16 instances"),
               "cpu": cpu_model()}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "batched steps/s", "n_gpus": world,
                "steps": K, "warmup": Wu, "ms_per_step": ms / K, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16x3+f64",
                "data": "synthetic",
                "config": {"workload": "batched16_j1j2", "instances": [w.name for w in insts],
                           "n_instances": n, "precision": "mixed",
                           "l2": "step working set > 126 MB L2", "replicas": world},
                "instance_steps_per_s": n * value,
                "solo_sum_ms": solo_ms, "concurrency_gain": solo_ms / (ms / K),
                "gram_tflops": gram_fl / (gram_ms * 1e-3) / 1e12 if gram_ms > 0 else None,
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(launches * K), "clocks": clk,
                "cuda_graph": b.graph_active(), "concurrency": b.concurrency(),
                "autotune": {"seconds": tune_s, "best_batched_ms": tune_ms},
                "fp64_path": fp64,
                "stage_ms_solo_sum": tot_stage, "instances": solo}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def matched_energy(w, hp, steps, dev):
    """Run the mixed and the FP64 GPU paths for `steps` steps from theta_0
    with the same Philox seeds; report the mean relative error of E over the
    last 10 steps against the exact energy (Jordan-Wigner for the TFIM)."""
    import torch
    from paper_2608_18065_b300 import nqs
    from paper_2608_18065_b300.inputs import init_theta
    if w.ham.family != "tfim":
        return None
    N = w.model.N
    B = np.diag(np.full(N, w.ham.h)) + np.diag(np.full(N - 1, w.ham.J), 1)
    E0 = -float(np.sum(np.linalg.svd(B, compute_uv=False)))
    out = {"E_exact": E0, "steps": steps, "eta0": hp.eta0}
    for prec in ("mixed", "fp64"):
        c = nqs.Context(w.model, w.ham, prec, hp.ns, device=dev)
        th = torch.tensor(init_theta(w.model, w.theta_seed), device=dev)
        m = torch.zeros_like(th)
        es, se = [], []
        s = c.new_stats()
        for t in range(steps):
            c.minsr_step(th, m, hp, t, s)
            d = nqs.decode_stats(s)
            es.append(d["E_re"])
            se.append(np.sqrt(d["var"] / hp.ns))
        last = np.array(es[-10:])
        rel = (last - E0) / abs(E0)
        out[prec] = {"rel_err_last10": float(rel.mean()),
                     "stderr": float(np.mean(se[-10:]) / abs(E0) / np.sqrt(10)),
                     "E_first": es[0], "E_last": es[-1]}
        del c
    d = abs(out["mixed"]["rel_err_last10"] - out["fp64"]["rel_err_last10"])
    out["matched"] = bool(d <= max(out["mixed"]["stderr"], out["fp64"]["stderr"]))
    return out


def run_lambda_grid(args):
    """Stability grid of App. E / Fig. 6: a 1D TFIM network (N = 20, d_h = 32,
    Tab. I's TFIM column) trained for 100 steps from theta_0 for every
    (lambda, N_s) of the grid, in the mixed and the FP64 contexts.  Per point:
    steps the library rejected (non-finite E, eps or delta theta; theta left
    unchanged), solves that fell back from FP32-factor refinement to the FP64
    factorisation, lambda_max and kappa_2 of the last step's T + lambda I
    (nqs_spectrum; lambda_max = 0 means every sample was the same
    configuration and training has stalled), and the final relative energy
    error against the Jordan-Wigner energy."""
    import torch
    from paper_2608_18065_b300 import nqs
    from paper_2608_18065_b300.inputs import HamSpec, HParams, ModelSpec, TAB1, init_theta
    dev = torch.device("cuda", 0)
    model, ham = ModelSpec(1, 20, 1, 32), HamSpec("tfim", J=1.0, h=1.0)
    N = model.N
    B = np.diag(np.full(N, ham.h)) + np.diag(np.full(N - 1, ham.J), 1)
    E0 = -float(np.sum(np.linalg.svd(B, compute_uv=False)))
    lams = [1e-1, 1e-2, 1e-3, 1e-4, 1e-5, 1e-6]
    nss = [16, 64, 256, 1024]
    steps = 100
    grid = []
    t0 = time.time()
    for prec in ("mixed", "fp64"):
        for ns in nss:
            c = nqs.Context(model, ham, prec, ns, device=dev)
            for lam in lams:
                tab = dict(TAB1["tfim"])
                tab["lam"] = lam
                hp = HParams(ns=ns, **tab)
                th = torch.tensor(init_theta(model, 5), device=dev)
                m = torch.zeros_like(th)
                s = c.new_stats()
                rejected = fallback = 0
                E = float("nan")
                for t in range(steps):
                    outs = c.step_outputs(ns) if t == steps - 1 else None
                    c.minsr_step(th, m, hp, t, s, outputs=outs)
                    d = nqs.decode_stats(s)
                    rejected += int(d["status"] != 0)
                    fallback += int(d["solve_fp64"] != 0)
                    if d["status"] == 0:
                        E = d["E_re"]
                sp = nqs.spectrum(outs["T"], lam, m=min(64, outs["T"].shape[0]))
                grid.append({"precision": prec, "ns": ns, "lambda": lam, "rejected": rejected,
                             # the FP64 context always factors in FP64
                             "fp64_fallback": fallback if prec == "mixed" else None,
                             "lambda_max_last": sp["lambda_max"], "kappa_last": sp["kappa"],
                             "rel_err_final": (E - E0) / abs(E0),
                             "finite_theta": bool(torch.isfinite(th).all().item())})
            del c
    line = {"metric": "minSR stability grid (App. E, Fig. 6)", "workload": "lambda_grid",
            "model": "tfim_N20_dh32", "steps_per_point": steps, "E_exact": E0,
            "seconds": time.time() - t0, "grid": grid}
    print(json.dumps(line))
    return 0


def qgt_error_from_gram(G, n_ref, n_sub, cplx):
    """||S_ref - S_sub||_F / ||S_ref||_F of Fig. 5b from the Gram G = X X^T of
    the stacked centred rows X = [Re Obar_ref; (Im Obar_ref;) Re Obar_sub;
    (Im Obar_sub)], without the N_p x N_p metrics: S = Obar^dagger Obar has
    ||S||_F = ||Obar Obar^dagger||_F and tr(S_ref S_sub) =
    ||Obar_ref Obar_sub^dagger||_F^2, and each complex Gram block follows from
    the real ones, (A + iB)(C + iD)^dagger = A C^T + B D^T + i (B C^T - A D^T)."""
    G = np.asarray(G, dtype=np.float64)
    k = 2 if cplx else 1
    r0, s0 = 0, k * n_ref
    def blk(i0, ni, j0, nj):
        a = G[i0:i0 + ni, j0:j0 + nj]
        if not cplx:
            return a.astype(np.complex128)
        ar, br = i0, i0 + ni
        ac, bc = j0, j0 + nj
        re = G[ar:ar + ni, ac:ac + nj] + G[br:br + ni, bc:bc + nj]
        im = G[br:br + ni, ac:ac + nj] - G[ar:ar + ni, bc:bc + nj]
        return re + 1j * im
    rr = blk(r0, n_ref, r0, n_ref)
    ss = blk(s0, n_sub, s0, n_sub)
    rs = blk(r0, n_ref, s0, n_sub)
    nr2 = float(np.sum(np.abs(rr) ** 2))
    d2 = nr2 + float(np.sum(np.abs(ss) ** 2)) - 2.0 * float(np.sum(np.abs(rs) ** 2))
    return float(np.sqrt(max(d2, 0.0) / nr2))


def qgt_subsample_errors(ctx, theta, sp_ref, sp_subs):
    """Fig. 5b errors of the subsampled SR metric for each spin set of
    sp_subs against the reference spins sp_ref: Jacobian rows from the
    library (nqs_jacobian), centred and scaled, stacked, and one FP64 Gram
    (nqs_gram) per subsample."""
    import torch
    cplx = bool(ctx.model.cplx)

    def rows(sp):
        n = sp.shape[0]
        J = ctx.jacobian(theta, sp)
        blocks = [J[:n]] + ([J[n:2 * n]] if cplx else [])
        return [(b - b.mean(0)) / math.sqrt(n) for b in blocks]

    ref = rows(sp_ref)
    out = []
    for sp in sp_subs:
        X = torch.cat(ref + rows(sp), 0).contiguous()
        G = ctx.gram(X).cpu().numpy()
        out.append(qgt_error_from_gram(G, sp_ref.shape[0], sp.shape[0], cplx))
    return out


def run_qgt_subsample(args):
    """Fig. 5b: relative error ||S - S~||_F / ||S||_F of the SR metric from
    N_s samples against a reference from 4096 samples (>= N_p), for the 6 x 6
    J1-J2 model (J2 = 0.5, complex head, Marshall sign, zero magnetisation)
    at theta_0, versus alpha = sqrt(N_s) / N_p.  The paper uses d_h = 10;
    the library builds hidden sizes 8, 16, 32, ..., and this run takes 16.
    FP64 context: exact samples, FP64 Jacobian and Gram.  Reports the fitted
    slope of log(error) against log(alpha) (Eq. UB predicts -1 for the
    bound)."""
    import torch
    from paper_2608_18065_b300 import nqs
    from paper_2608_18065_b300.inputs import HamSpec, ModelSpec, init_theta
    dev = torch.device("cuda", 0)
    model, ham = ModelSpec(2, 6, 6, 16, cplx=1, marshall=1, zmask=1), HamSpec("j1j2", J1=1.0, J2=0.5)
    n_ref, subs = 4096, [16, 32, 64, 128, 256, 512, 1024, 2048]
    t0 = time.time()
    c = nqs.Context(model, ham, "fp64", n_ref, device=dev)
    th = torch.tensor(init_theta(model, 7), device=dev)
    sp_ref, _ = c.sample(th, n_ref, seed=101, step=0)
    sp_all, _ = c.sample(th, max(subs), seed=202, step=0)
    errs = qgt_subsample_errors(c, th, sp_ref, [sp_all[:n] for n in subs])
    npar = c.np
    alphas = [math.sqrt(n) / npar for n in subs]
    slope = float(np.polyfit(np.log(alphas), np.log(errs), 1)[0])
    line = {"metric": "subsampled SR-metric error (Sec. III, Fig. 5b)", "workload": "qgt_subsample",
            "model": "j1j2_6x6_dh16_cplx", "n_params": npar, "n_ref": n_ref,
            "points": [{"ns": n, "alpha": a, "rel_err": e} for n, a, e in zip(subs, alphas, errs)],
            "loglog_slope": slope, "seconds": time.time() - t0}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched16":
        return run_batched(args)
    if args.workload == "lambda_grid":
        return run_lambda_grid(args)
    if args.workload == "qgt_subsample":
        return run_qgt_subsample(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
