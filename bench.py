#!/usr/bin/env python
"""Benchmark: regularized minSR steps/s on one B300 (and N replicas).

Workload (default, `batched16`): 16 independent 2D J1-J2 instances on open
L x L lattices (L in {6, 8, 10, 12}, J2/J1 in {0, .25, .5, .6}, Ns in
{256 .. 4096}, GRU hidden size 32 .. 128, complex head, Marshall sign,
zero-magnetisation mask), mixed precision (FP32 recurrence and Jacobian,
BF16x3 tensor-core local energies and Gram, FP64 centring and solve), each
with Tab. I's hyper-parameters, stepped together: one batched step = one
iteration of Algorithm 1 (sampling, local energies, O, centring, T,
regularized solve, momentum, update) of every instance, one CUDA graph.
Beside it: the same instances one at a time on the plain FP64 GPU path,
matched energies, and a summary of each single-instance workload.
Other workloads by --workload (tfim100, heis10, ...).

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



# NVTX range around the timed steps (ncu --nvtx --nvtx-include "nqs_timed_steps/"
# lists exactly the kernels of the timed region)
TIMED_RANGE = "nqs_timed_steps"

def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="batched16",
                   help="batched16 (the headline: 16 J1-J2 instances), tfim16, tfim100, "
                        "tfim200, cluster64, heis10, lambda_grid, qgt_subsample")
    p.add_argument("--matched-steps", type=int, default=50,
                   help="steps of the mixed and FP64 paths for the matched-energy check (0: skip)")
    p.add_argument("--matched-eta0", type=float, default=0.1,
                   help="eta0 of the matched-energy runs (Tab. I's 0.5 collapses this model "
                        "onto the product state within ~30 steps for both paths)")
    p.add_argument("--fp64-steps", type=int, default=1,
                   help="timed steps of the plain FP64 GPU path (per instance)")
    p.add_argument("--no-per-config", action="store_true",
                   help="batched16: skip the summary lines of the other workloads")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-spectrum", action="store_true",
                   help="skip the conditioning diagnostics of T (App. E)")
    p.add_argument("--spectrum-steps", type=int, default=64,
                   help="Lanczos steps of the conditioning diagnostics")
    p.add_argument("--no-graph", action="store_true", help="launch every kernel eagerly")
    p.add_argument("--instances", default="",
                   help="batched16: only these instances (comma-separated names; for profiles)")
    p.add_argument("--grouped", type=int, default=-1,
                   help="batched16: grouped stages after the autotuner (nqs_batch_set_grouped "
                        "mask; -1: the autotuner's choice)")
    p.add_argument("--train-steps", type=int, default=10000,
                   help="train:<workload>: minSR steps of the training run")
    p.add_argument("--train-eta0", type=float, default=None,
                   help="train:<workload>: eta0 instead of Tab. I's")
    p.add_argument("--train-window", type=int, default=300,
                   help="train:<workload>: steps averaged at the end (the paper's window)")
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
    """A peak from MEASURED_PEAKS.json beside this file (a copy bandwidth and
    BF16 GEMM rates measured on this GPU model), else the stated fallback;
    returns (value, source)."""
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
    of hidden size 64 and 32 (units padded to 64), and for mixed 2D lattices
    of hidden size 64 (weights in shared memory; 32 padded to 64) and 96 or
    128 (weights streamed from L2)."""
    if precision != "mixed":
        return False
    return ((model.dim == 1 and model.dh in (32, 64)) or
            (model.dim == 2 and model.dh in ENGINE2D_DH))


# 2D hidden sizes served by the tensor-core engines
ENGINE2D_DH = (32, 64, 96, 128)


def eloc_tc_site_flops(model):
    """Tensor-pipe flops issued per recomputed site of one configuration
    (three BF16 products hi.hi + hi.lo + lo.hi of each product):
    1D: the gate product [1 x 64] x [64 x 192];
    2D, d_h 64 (32 padded): the state mix [1 x 128] x [128 x 64] and the
    gates [1 x 64] x [64 x 192];
    2D, d_h 96 / 128: [U1; U2] h_{k-1}, [1 x dh] x [dh x 2dh], and the gates
    [1 x dh] x [dh x 3dh] (the padded k-steps are not issued)."""
    if model.dim == 1:
        return 3 * 2 * 64 * 3 * 64
    if model.dh in (32, 64):
        return 3 * 2 * 64 * (3 * 64 + 2 * 64)
    dh = model.dh
    return 3 * 2 * dh * (2 * dh + 3 * dh)


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
        kern = ("k_eloc_tc" if w.model.dim == 1 else
                "k_eloc2d_tc" if w.model.dh in (32, 64) else "k_eloc2d_tcs")
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
    reported by its HBM bytes, as is the mixed 2D one; mixed 2D sampling at
    d_h 96 / 128 runs on the tensor cores and is reported by its BF16x3
    products).  cholesky: n^3/3 factor (128-wide panels, R >= 3072) or n^3/3
    factor + n^3/3 triangular inverse (32-wide panels) in FP32 for the mixed
    path (refinement sweeps: 2n^2 each, not counted).  gram: BF16x3 tensor work 3 R(R+1) Np.  center: HBM bytes of
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
    dh = w.model.dh
    if f32 and w.model.dim == 2 and dh in (96, 128) and 2 * w.model.Lx - 1 <= 31 \
            and ms.get("sample", 0) > 0:
        # sampling on the streamed tensor-core engine: per sample and site the
        # products [U1; U2] h (2 dh x dh) and W h' (3 dh x dh), BF16x3
        t = ms["sample"]
        fl = w.hp.ns * N * 3 * 2 * (2 * dh * dh + 3 * dh * dh)
        pk, src = measured_peak("bf16_tflops_sustained", 1400.0)
        a = fl / (t * 1e-3) / 1e12
        out["sample"] = {"kernel": "k_eloc2d_tcs (sampling)", "bound": "tensor", "achieved": a,
                         "peak": pk, "unit": "TFLOP/s", "frac": a / pk, "traffic": None,
                         "peak_source": src + ", BF16 dense, sustained", "flops_per_launch": fl,
                         "ms_per_launch": t}
    else:
        alu("sample", "k_forward<MODE_SAMPLE>", w.hp.ns * N * sf)
    alu("jac_bwd", "k_jac_bwd", R * N * sf)
    if f32 and w.model.dim == 2 and dh in (32, 64, 96, 128) and ms.get("jac_grad", 0) > 0:
        # tensor-core rows of O: HBM reads of the adjoint records (6 dh + 4
        # per site and row) and the states, write of O
        t = ms["jac_grad"]
        byts = R * N * (6 * dh + 4) * 4 + w.hp.ns * N * dh * 4 + R * np_ * 4
        pk, src = measured_peak("hbm_gbs", 6400.0)
        a = byts / (t * 1e-3) / 1e9
        out["jac_grad"] = {"kernel": "k_jac2d_tc", "bound": "hbm", "achieved": a, "peak": pk,
                           "unit": "GB/s", "frac": a / pk, "traffic": None, "peak_source": src,
                           "bytes_per_launch": byts, "ms_per_launch": t}
    elif f32 and w.model.dim == 1 and w.model.dh in (32, 64) and ms.get("jac_grad", 0) > 0:
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
    if f32 and R >= 3072 and R % 4 == 0:
        alu("cholesky", "k_chol_blk", R ** 3 / 3)  # 128-wide panels: the factor
    else:
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
def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


L2_NOTE = "working set > 126 MB L2 per step (O, caches, adjoints); no flush"


def workload_config(args, w=None, insts=None):
    """The config dict of a bench line: the same for the repo arm and the
    reference arm (precision and buffer sizes are reported beside it)."""
    if insts is not None:
        return {"workload": "batched16_j1j2", "n_instances": len(insts),
                "instances": [x.name for x in insts],
                "draw": "PCG64(7): L in {6,8,10,12}, J2 in {0,.25,.5,.6}, "
                        "Ns in {256..4096}, dh in {32,64,96,128}; theta_0 seed 1000+i",
                "l2": L2_NOTE, "replicas": args.gpus}
    d = w.describe()
    d.pop("precision", None)
    d.update(l2=L2_NOTE, replicas=args.gpus)
    return d


def oracle_instance_step(w, ns_sub, step):
    """One FP64 oracle step of instance w on ns_sub of its samples; returns
    (measured seconds, seconds scaled to its full Ns)."""
    import copy
    from oracle import oracle as O
    from paper_2608_18065_b300.inputs import init_theta
    th = init_theta(w.model, w.theta_seed)
    hp = copy.copy(w.hp)
    hp.ns = ns_sub
    t0 = time.perf_counter()
    O.minsr_step(w.model, w.ham, th, np.zeros_like(th), hp, step)
    dt = time.perf_counter() - t0
    return dt, dt * w.hp.ns / ns_sub


def oracle_sample_size(w, budget_s):
    """Samples of a bounded oracle step of w: at least as many as the oracle
    has threads (every core works), else as many as fit budget_s by a probe
    at that size, at most Ns."""
    from oracle import oracle as O
    nmin = min(w.hp.ns, max(4, O.num_threads()))
    dt, _ = oracle_instance_step(w, nmin, 0)
    return int(min(w.hp.ns, max(nmin, nmin * budget_s / max(dt, 1e-9))))


def run_reference(args):
    """The reference arm: the FP64 CPU oracle on the host cores, on the same
    workload.  Every timed step is one oracle step on a bounded sample of
    configurations: for the batched workload, instance t mod 16 (so that the
    timed steps walk through the instances) on as many samples as the oracle
    has threads; for one instance, as many samples as fit about
    150 s / (W + K).  ms_per_step is the measured time of that bounded step;
    value is the rate of whole steps, each instance's time scaled to its
    full Ns (sampling, local energies and O are linear in Ns and dominate
    the oracle's time; its Gram and solve grow faster, so the scaling
    flatters the oracle)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import oracle as O
    from paper_2608_18065_b300.inputs import batched_instances, workloads
    if args.workload == "batched16":
        insts = batched_instances()
        if args.instances:
            insts = [w for w in insts if w.name in args.instances.split(",")]
        cfg = workload_config(args, insts=insts)
        unit = "batched steps/s"
        nsub = [min(w.hp.ns, max(4, O.num_threads())) for w in insts]
    else:
        w = resolve_workload(args.workload)
        insts = [w]
        cfg = workload_config(args, w=w)
        unit = UNIT
        nsub = [oracle_sample_size(w, max(1.0, 150.0 / max(1, args.steps + args.warmup)))]
    n = len(insts)
    for t in range(args.warmup):
        oracle_instance_step(insts[t % n], nsub[t % n], t)
    meas = []
    full = [[] for _ in range(n)]
    for t in range(args.warmup, args.warmup + args.steps):
        m, f = oracle_instance_step(insts[t % n], nsub[t % n], t)
        meas.append(m)
        full[t % n].append(f)
    for i in range(n):  # fewer timed steps than instances: the rest once, untimed
        if not full[i]:
            full[i].append(oracle_instance_step(insts[i], nsub[i], 0)[1])
    per_full = sum(float(np.mean(x)) for x in full)
    value = 1.0 / per_full
    whole = all(ns == w.hp.ns for ns, w in zip(nsub, insts))
    sample = ("one whole FP64 oracle step per timed step" if whole and n == 1 else
              (f"one FP64 oracle step per timed step of instance t mod {n} on "
               f"{min(nsub)}..{max(nsub)} of its samples (same models, Hamiltonians, "
               "theta_0); each instance's time scaled to its full Ns and summed"
               if n > 1 else
               f"one FP64 oracle step per timed step on {nsub[0]} of the {insts[0].hp.ns} "
               "samples, time scaled to the full Ns"))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": unit,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * float(np.mean(meas)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "precision": "fp64",
            "data": "synthetic", "config": cfg,
            "ms_per_full_step_scaled": 1000.0 * per_full,
            "samples_per_instance": nsub,
            "cpu_baseline": {"value": value, "unit": unit, "cores": O.num_threads(),
                             "kind": "oracle", "sample": sample, "cpu": cpu_model()},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def cpu_baseline_leg(insts, unit, budget_s=20.0):
    """cpu_baseline of the repo arm: one bounded FP64 oracle step of every
    instance on the host cores (as many samples as the oracle has threads
    for the batched workload; as many as fit budget_s for one instance),
    each scaled to its full Ns, summed."""
    from oracle import oracle as O
    if len(insts) > 1:
        nsub = [min(w.hp.ns, max(4, O.num_threads())) for w in insts]
    else:
        nsub = [oracle_sample_size(insts[0], budget_s)]
    meas = full = 0.0
    for w, ns in zip(insts, nsub):
        m, f = oracle_instance_step(w, ns, 0)
        meas += m
        full += f
    return {"value": 1.0 / full, "unit": unit, "cores": O.num_threads(), "kind": "oracle",
            "sample": (f"one FP64 oracle step of each of the {len(insts)} instances on "
                       f"{min(nsub)}..{max(nsub)} of its samples, {meas:.1f} s measured, "
                       "each scaled to its full Ns and summed"
                       if len(insts) > 1 else
                       f"one FP64 oracle step on {nsub[0]} of the {insts[0].hp.ns} samples "
                       f"({meas:.1f} s), scaled to the full Ns"),
            "cpu": cpu_model()}


# -------------------------------------------------------------------- ours
def resolve_workload(name):
    """A single-instance workload: a key of inputs.workloads(), or
    b16:<instance name> for one of the batched instances."""
    from paper_2608_18065_b300.inputs import batched_instances, workloads
    if name.startswith("b16:"):
        for w in batched_instances():
            if w.name == name[4:]:
                return w
        raise SystemExit(f"no batched instance named {name[4:]}")
    return workloads()[name]


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
    w = resolve_workload(args.workload)
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
    torch.cuda.nvtx.range_push(TIMED_RANGE)
    e0.record()
    for t in range(Wu, Wu + K):
        ctx.minsr_step(thd, momd, hp, t, stats)
    e1.record()
    torch.cuda.nvtx.range_pop()
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
        if w.ham.family == "tfim":
            hpm.eta0 = args.matched_eta0
        matched = matched_energy(w, hpm, args.matched_steps, dev, reference_energy(w))

    cpu = None
    if not args.no_cpu and rank == 0:
        cpu = cpu_baseline_leg([w], UNIT, 20.0)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
                "warmup": Wu, "ms_per_step": ms_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+bf16x3+f64" if w.precision == "mixed" else "f64",
                "precision": w.precision, "data": "synthetic",
                "config": workload_config(args, w=w),
                "workspace_mb": ctx.workspace_bytes / 2**20,
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


MATCHED_SUBSET = ("j1j2_L6_J20.6_dh64_ns256", "j1j2_L6_J20.25_dh128_ns512",
                  "j1j2_L8_J20.0_dh96_ns256", "j1j2_L8_J20.25_dh32_ns512")


def instance_roofline(insts, stage_ms_list, sites_list):
    """Roofline of the batch's dominant stage, summed over the instances:
    the local-energy engines by issued tensor flops against the sustained
    BF16 peak when every instance runs on tcgen05 (else FP32-equivalent
    flops against the derived FP32 peak), other stages by the per-stage
    counts of stage_rooflines."""
    tot = {}
    for sm in stage_ms_list:
        for k, v in sm.items():
            tot[k] = tot.get(k, 0.0) + v
    dom = max(tot, key=lambda k: tot[k])
    if dom == "eloc_suffix":
        ms = tot[dom]
        alg = sum(n * site_flops(w.model) for w, n in zip(insts, sites_list))
        if all(eloc_tc_used(w.model, w.precision) for w in insts):
            fl = sum(n * eloc_tc_site_flops(w.model) for w, n in zip(insts, sites_list))
            peak, src = measured_peak("bf16_tflops_sustained", 1400.0)
            ach = fl / (ms * 1e-3) / 1e12
            return dom, {"kernel": "k_eloc2d_tc (d_h 32, 64) + k_eloc2d_tcs (d_h 96, 128), "
                                   "all instances (eloc_suffix)",
                         "bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                         "frac": ach / peak, "traffic": None,
                         "peak_source": src + ", BF16 dense, sustained",
                         "flops_per_batch": fl, "fp32_equiv_flops_per_batch": alg,
                         "fp32_equiv_tflops": alg / (ms * 1e-3) / 1e12, "ms_per_batch": ms}
        ach = alg / (ms * 1e-3) / 1e12
        return dom, {"kernel": "2D E_loc engines, all instances (eloc_suffix; FP32-equivalent)",
                     "bound": "alu", "achieved": ach, "peak": FP32_ALU_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": ach / FP32_ALU_PEAK_TFLOPS, "traffic": None,
                     "peak_source": "148 SMs x 128 FP32 lanes x 2 flop x 2032 MHz (derived)",
                     "flops_per_batch": alg, "ms_per_batch": ms}
    # other stages: sum the per-instance work of the stage's own count
    work = ms = 0.0
    first = None
    for w, sm, n in zip(insts, stage_ms_list, sites_list):
        R = w.hp.ns * (2 if w.model.cplx else 1)
        from paper_2608_18065_b300.inputs import param_count
        k = stage_rooflines(w, sm, n, R, param_count(w.model)).get(dom)
        if not k:
            continue
        first = first or k
        t = k["ms_per_launch"]
        ms += t
        work += k["achieved"] * t
    if not first:
        return dom, {"kernel": dom, "bound": None, "achieved": None, "peak": None, "unit": None,
                     "frac": None, "traffic": None, "ms_per_batch": tot[dom]}
    ach = work / ms
    out = dict(first)
    out.update(kernel=first["kernel"] + ", all instances", achieved=ach,
               frac=ach / first["peak"], ms_per_batch=ms)
    out.pop("ms_per_launch", None)
    out.pop("flops_per_launch", None)
    out.pop("bytes_per_launch", None)
    return dom, out


def run_batched(args):
    """The headline: 16 heterogeneous 2D J1-J2 instances (L in {6..12}, J2 in
    {0, .25, .5, .6}, Ns in {256..4096}, dh in {32..128}) stepped together by
    nqs_minsr_step_batched (one graph per batched step, launch shapes from
    the autotuner); value = batched steps/s (x16 instance steps).  Beside it:
    the same instances one at a time on the plain FP64 GPU path, the
    matched-energy leg (mixed batched vs FP64 one at a time from the same
    theta_0 and Philox keys, on four L <= 8 instances), the FP64 oracle on
    the host cores, the end-to-end rate through host buffers, and a summary
    line of each other workload (configs 1-4)."""
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
    if args.instances:
        keep = args.instances.split(",")
        insts = [w for w in insts if w.name in keep]
        if len(insts) != len(keep):
            raise SystemExit(f"--instances: unknown names in {args.instances}")
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
    if args.grouped >= 0:
        b.set_grouped(args.grouped)
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
    torch.cuda.nvtx.range_push(TIMED_RANGE)
    e0.record()
    for t in range(Wu, Wu + K):
        b.step(thd, mod, hps, t, stats)
    e1.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    batch_graph = bool(b.graph_active())
    batch_grouped = b.grouped()
    batch_eloc_share = b.eloc_share()
    # by stage, the FP32 solves of the mixed instances with R % 4 == 0 and
    # R >= 256 are one launch (bit 1), the streamed local-energy engines one
    # launch per hidden size (bit 2)
    n_group = sum(1 for w in insts
                  if (lambda R: R >= 256 and R % 4 == 0)(w.hp.ns * (2 if w.model.cplx else 1)))
    tcs_dh = [w.model.dh for w in insts if w.model.dim == 2 and w.model.dh in (96, 128)]
    saved = ((max(n_group - 1, 0) if batch_grouped & 1 else 0) +
             (len(tcs_dh) - len(set(tcs_dh)) if batch_grouped & 2 else 0))
    ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    value = aggregate_rate(world, K, ms)
    st = [nqs.decode_stats(stats[i]) for i in range(n)]

    # per-instance stage times: every instance alone, eager, one step
    solo, stage_list, sites_list = [], [], []
    gram_ms = gram_fl = 0.0
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
        stage_list.append(sm)
        sites_list.append(sites)
        gram_ms += sm["gram"]
        gram_fl += R * (R + 1) * param_count(w.model)
        solo.append({"instance": w.name, "ms": sum(sm.values()), "eloc_configs": cfg,
                     "eloc_sites": sites, "workspace_mb": round(c.workspace_bytes / 2**20, 1),
                     "stage_ms": {k: round(v, 3) for k, v in sm.items()},
                     "E_re": st[i]["E_re"], "status": st[i]["status"],
                     "solve_fp64": st[i].get("solve_fp64"),
                     "tuning": {k: tuning[i][k] for k in ("eloc_grid", "gram_splits", "solve_grid")}})
    solo_ms = sum(x["ms"] for x in solo)
    tot_stage = {}
    for sm in stage_list:
        for k, v in sm.items():
            tot_stage[k] = tot_stage.get(k, 0.0) + v
    dom, roof = instance_roofline(insts, stage_list, sites_list)

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
    del b
    for c in ctxs:
        c.close()
    torch.cuda.empty_cache()

    # the same instances one at a time on the plain FP64 GPU path (graphs on)
    fp64 = None
    if args.fp64_steps > 0:
        f_ms = 0.0
        per = []
        for i, w in enumerate(insts):
            c64 = nqs.Context(w.model, w.ham, "fp64", w.hp.ns, device=dev)
            t64 = torch.tensor(th0[i], device=dev)
            m64 = torch.zeros_like(t64)
            s64 = c64.new_stats()
            c64.minsr_step(t64, m64, hps[i], 0, s64)  # warm-up (not timed)
            torch.cuda.synchronize()
            b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            b0.record()
            for t in range(1, 1 + args.fp64_steps):
                c64.minsr_step(t64, m64, hps[i], t, s64)
            b1.record()
            torch.cuda.synchronize()
            d = b0.elapsed_time(b1) / args.fp64_steps
            f_ms += d
            per.append(round(d, 3))
            c64.close()
            del c64
        torch.cuda.empty_cache()
        fp64 = {"batched_steps_per_s": 1000.0 / f_ms, "ms_per_batched_step": f_ms,
                "instance_ms": per, "steps_per_instance": args.fp64_steps,
                "speedup_mixed_batched_over_fp64": (1000.0 * K / ms) / (1000.0 / f_ms)}

    matched = None
    if args.matched_steps > 0 and rank == 0:
        matched = matched_energy_batched([w for w in insts if w.name in MATCHED_SUBSET],
                                         args.matched_steps, dev)

    per_config = None
    if not args.no_per_config and rank == 0:
        per_config = {}
        for key in ("tfim16", "tfim100", "cluster64", "heis10"):
            per_config[key] = config_summary(key, args, dev)
            torch.cuda.empty_cache()

    cpu = None
    if not args.no_cpu and rank == 0:
        cpu = cpu_baseline_leg(insts, "batched steps/s", 20.0)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "batched steps/s", "n_gpus": world,
                "steps": K, "warmup": Wu, "ms_per_step": ms / K, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16x3+f64",
                "precision": "mixed", "data": "synthetic",
                "config": workload_config(args, insts=insts),
                "instance_steps_per_s": n * value,
                "solo_sum_ms": solo_ms, "concurrency_gain": solo_ms / (ms / K),
                "gram_tflops": gram_fl / (gram_ms * 1e-3) / 1e12 if gram_ms > 0 else None,
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int((launches - saved) * K),
                "clocks": clk, "cuda_graph": batch_graph, "grouped_stages": {"solve": bool(batch_grouped & 1), "eloc": bool(batch_grouped & 2)},
                "eloc_share_eighths": batch_eloc_share,
                "autotune": {"seconds": tune_s, "best_batched_ms": tune_ms},
                "fp64_path": fp64, "matched_energy": matched, "per_config": per_config,
                "errors_vs_oracle": load_errors(),
                "stage_ms_solo_sum": tot_stage, "dominant_stage": dom, "instances": solo}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def load_errors():
    """Maxima of the mixed path's errors against the FP64 oracle (log Psi,
    E_loc, T, delta theta, energy trajectory) as measured by the full-size
    parity tests on a B300 and recorded in profiles/errors_vs_oracle.json."""
    p = os.path.join(ROOT, "profiles", "errors_vs_oracle.json")
    try:
        return json.load(open(p))
    except (ValueError, OSError):
        return None


def _mean_stderr(es, vs, ns):
    """Mean of E over the last 10 steps and its standard error: the larger
    of the sampling error (sqrt(mean Var / Ns / 10)) and the spread of the
    10 values themselves (std / sqrt(10): the trajectory still moves)."""
    last = np.array(es[-10:])
    se_s = float(np.sqrt(np.mean(np.array(vs[-10:]) / ns) / 10.0))
    se_e = float(np.std(last, ddof=1) / np.sqrt(len(last))) if len(last) > 1 else 0.0
    return float(last.mean()), max(se_s, se_e)


def _match(a, b):
    """Matched energies: the two means differ by no more than the larger
    standard error (the criterion of the measurement plan); also reported,
    within three combined standard errors."""
    d = abs(a["E_last10"] - b["E_last10"])
    return (bool(d <= max(a["stderr"], b["stderr"])),
            bool(d <= 3.0 * np.hypot(a["stderr"], b["stderr"])))


def matched_energy(w, hp, steps, dev, E_ref=None):
    """Mixed and plain FP64 GPU paths for `steps` steps from theta_0 with the
    same Philox keys.  Reported: the mean of E over the last 10 steps and its
    standard error (sqrt(mean Var / Ns / 10)), the relative error against
    E_ref when one exists; matched when the two paths' means (or relative
    errors) differ by no more than the larger standard error."""
    import torch
    from paper_2608_18065_b300 import nqs
    from paper_2608_18065_b300.inputs import init_theta
    out = {"E_ref": E_ref, "steps": steps, "eta0": hp.eta0}
    for prec in ("mixed", "fp64"):
        c = nqs.Context(w.model, w.ham, prec, hp.ns, device=dev)
        th = torch.tensor(init_theta(w.model, w.theta_seed), device=dev)
        m = torch.zeros_like(th)
        es, vs = [], []
        s = c.new_stats()
        t0 = time.perf_counter()
        for t in range(steps):
            c.minsr_step(th, m, hp, t, s)
            d = nqs.decode_stats(s)
            es.append(d["E_re"])
            vs.append(d["var"])
        mean, se = _mean_stderr(es, vs, hp.ns)
        r = {"E_last10": mean, "stderr": se, "E_first": es[0], "E_last": es[-1],
             "seconds": time.perf_counter() - t0}
        if E_ref is not None:
            r["rel_err_last10"] = (mean - E_ref) / abs(E_ref)
            r["rel_stderr"] = se / abs(E_ref)
        out[prec] = r
        c.close()
        del c
    out["matched"], out["within_3sigma"] = _match(out["mixed"], out["fp64"])
    return out


def matched_energy_batched(insts, steps, dev):
    """Matched-energy leg of the batched workload: the given instances
    stepped together in the mixed batched form and one at a time on the FP64
    GPU path, from theta_0 with the same Philox keys, `steps` steps each;
    per instance the mean E over the last 10 steps with its standard error,
    matched when the two differ by no more than the larger one.  (No exact
    energy exists for these lattices; the paper's reference values per site
    are -0.628656 (J2 = 0, QMC, 10 x 10 and larger) and -0.48654 (J2 = 0.5,
    PEPS), context only.)"""
    import torch
    from paper_2608_18065_b300 import nqs
    from paper_2608_18065_b300.inputs import init_theta
    n = len(insts)
    ctxs = [nqs.Context(w.model, w.ham, "mixed", w.hp.ns, device=dev) for w in insts]
    ths = [torch.tensor(init_theta(w.model, w.theta_seed), device=dev) for w in insts]
    ms_ = [torch.zeros_like(t) for t in ths]
    b = nqs.Batch(ctxs)
    b.use_graph(True)
    stats = b.new_stats()
    es = [[] for _ in range(n)]
    vs = [[] for _ in range(n)]
    t0 = time.perf_counter()
    for t in range(steps):
        b.step(ths, ms_, [w.hp for w in insts], t, stats)
        for i in range(n):
            d = nqs.decode_stats(stats[i])
            es[i].append(d["E_re"])
            vs[i].append(d["var"])
    mixed_s = time.perf_counter() - t0
    del b
    for c in ctxs:
        c.close()
    out = {"steps": steps, "instances": [], "mixed_batched_seconds": mixed_s}
    t0 = time.perf_counter()
    allm = True
    for i, w in enumerate(insts):
        c = nqs.Context(w.model, w.ham, "fp64", w.hp.ns, device=dev)
        th = torch.tensor(init_theta(w.model, w.theta_seed), device=dev)
        m = torch.zeros_like(th)
        s = c.new_stats()
        e64, v64 = [], []
        for t in range(steps):
            c.minsr_step(th, m, w.hp, t, s)
            d = nqs.decode_stats(s)
            e64.append(d["E_re"])
            v64.append(d["var"])
        c.close()
        mm, ms1 = _mean_stderr(es[i], vs[i], w.hp.ns)
        fm, fs = _mean_stderr(e64, v64, w.hp.ns)
        a = {"E_last10": mm, "stderr": ms1, "E_first": es[i][0]}
        f = {"E_last10": fm, "stderr": fs, "E_first": e64[0]}
        ok, ok3 = _match(a, f)
        allm &= ok
        out["instances"].append({"instance": w.name, "N": w.model.N, "mixed": a, "fp64": f,
                                 "matched": ok, "within_3sigma": ok3})
    out["fp64_one_at_a_time_seconds"] = time.perf_counter() - t0
    out["matched"] = allm
    return out


def reference_energy(w):
    """Exact ground energy where one exists: Jordan-Wigner for the open TFIM
    chain, -(N - 2) for the ZXZ cluster chain (None otherwise)."""
    if w.ham.family == "tfim":
        N = w.model.N
        B = np.diag(np.full(N, w.ham.h)) + np.diag(np.full(N - 1, w.ham.J), 1)
        return -float(np.sum(np.linalg.svd(B, compute_uv=False)))
    if w.ham.family == "cluster_zxz":
        return -float(w.model.N - 2)
    if w.ham.family == "cluster_paper":
        return -float(w.model.N)
    return None


def config_summary(key, args, dev):
    """One line per other workload (configs 1-4): steps/s of its own
    precision with graphs, the plain FP64 path's ms/step and the ratio, the
    dominant stage's roofline fraction, and the matched-energy comparison
    (50 steps; 500 for the 1D TFIM N = 100 workload, at eta0 = 0.1 for the
    TFIM where Tab. I's 0.5 collapses onto the product state).  The FP64-only
    workload reports its us/step with and without graph replay."""
    import copy
    import torch
    from paper_2608_18065_b300 import nqs
    from paper_2608_18065_b300.inputs import init_theta, workloads
    w = workloads()[key]
    hp = w.hp
    out = {"workload": w.name, "precision": w.precision}
    th0 = init_theta(w.model, w.theta_seed)

    def timed(ctx, graph, steps=20, warm=3):
        ctx.use_graph(graph)
        th = torch.tensor(th0, device=dev)
        m = torch.zeros_like(th)
        s = ctx.new_stats()
        for t in range(warm):
            ctx.minsr_step(th, m, hp, t, s)
        torch.cuda.synchronize()
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for t in range(warm, warm + steps):
            ctx.minsr_step(th, m, hp, t, s)
        z.record()
        torch.cuda.synchronize()
        return a.elapsed_time(z) / steps, th, m

    c = nqs.Context(w.model, w.ham, w.precision, hp.ns, device=dev)
    ms, th, m = timed(c, True)
    out["steps_per_s"] = 1000.0 / ms
    out["ms_per_step"] = ms
    if w.precision == "fp64":
        ms_eager, _, _ = timed(c, False)
        out["us_per_step_graph"] = 1000.0 * ms
        out["us_per_step_eager"] = 1000.0 * ms_eager
        out["graph_replay_saving_us"] = 1000.0 * (ms_eager - ms)
    c.timing_begin(3)
    s = c.new_stats()
    for t in range(3):
        c.minsr_step(th, m, hp, 100 + t, s)
    torch.cuda.synchronize()
    sm, nt = c.timing_end()
    cfg, sites = c.eloc_work()
    R = hp.ns * (2 if w.model.cplx else 1)
    sm = {k: v / max(nt, 1) for k, v in sm.items()}
    kern = stage_rooflines(w, sm, sites, R, c.np)
    dom = max(sm, key=lambda k: sm[k])
    k = kern.get(dom)
    out["dominant_stage"] = dom
    out["roofline"] = ({x: k[x] for x in ("kernel", "bound", "achieved", "peak", "unit", "frac")}
                       if k else None)
    out["stage_ms"] = {x: round(v, 4) for x, v in sm.items()}
    c.close()
    if w.precision != "fp64":
        c64 = nqs.Context(w.model, w.ham, "fp64", hp.ns, device=dev)
        ms64, _, _ = timed(c64, True, steps=3, warm=1)
        c64.close()
        out["fp64_ms_per_step"] = ms64
        out["speedup_over_fp64"] = ms64 / ms
    if args.matched_steps > 0:
        hpm = copy.copy(hp)
        steps = 50
        if w.ham.family == "tfim":
            hpm.eta0 = args.matched_eta0
            if w.model.N == 100:
                steps = 500
        E_ref = reference_energy(w)
        if w.precision == "fp64":
            # config 1 is the plain FP64 method itself: its energy after the run
            c = nqs.Context(w.model, w.ham, "fp64", hp.ns, device=dev)
            th = torch.tensor(th0, device=dev)
            m = torch.zeros_like(th)
            s = c.new_stats()
            es, vs = [], []
            for t in range(steps):
                c.minsr_step(th, m, hpm, t, s)
                d = nqs.decode_stats(s)
                es.append(d["E_re"])
                vs.append(d["var"])
            c.close()
            mean, se = _mean_stderr(es, vs, hp.ns)
            out["energy"] = {"E_ref": E_ref, "steps": steps, "eta0": hpm.eta0,
                             "E_last10": mean, "stderr": se,
                             "rel_err_last10": (mean - E_ref) / abs(E_ref)}
        else:
            out["matched_energy"] = matched_energy(w, hpm, steps, dev, E_ref)
            if w.model.dim == 2:
                out["matched_energy"]["context"] = ("Tab. II QMC value for the 2D Heisenberg "
                                                    "model: -0.628656 per site")
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


# Tab. II: final minSR energies per site and the reference energies per site
TAB2 = {"tfim": (-1.2714254, -1.27142590795), "cluster_paper": (-0.999947, -1.0),
        "heisenberg": (-0.628486, -0.628656), "j1j2": (-0.48514, -0.48654)}


def run_train(args):
    """A training run of one workload (train:<key>): --train-steps minSR steps
    from theta_0 with graphs, E/N averaged over the last --train-window
    steps against Tab. II's minSR result and reference energy."""
    import copy
    import torch
    from paper_2608_18065_b300 import nqs
    from paper_2608_18065_b300.inputs import init_theta
    w = resolve_workload(args.workload[6:])
    hp = copy.copy(w.hp)
    if args.train_eta0 is not None:
        hp.eta0 = args.train_eta0
    dev = torch.device("cuda", 0)
    c = nqs.Context(w.model, w.ham, w.precision, hp.ns, device=dev)
    c.use_graph(True)
    th = torch.tensor(init_theta(w.model, w.theta_seed), device=dev)
    m = torch.zeros_like(th)
    K = args.train_steps
    stats = torch.zeros((K, 11), dtype=torch.float64, device=dev)
    one = c.new_stats()
    t0 = time.perf_counter()
    for t in range(K):
        c.minsr_step(th, m, hp, t, one)
        stats[t].copy_(one)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    st = stats.cpu().numpy()
    status = st[:, 8:9].copy().view(np.int32)[:, 0]
    E = st[:, 0] / w.model.N
    win = min(args.train_window, K)
    key = ("heisenberg" if w.ham.J2 == 0.0 else "j1j2") if w.ham.family == "j1j2" else w.ham.family
    E_ref = reference_energy(w)
    line = {"metric": "minSR training run (E per site after K steps)", "workload": w.name,
            "steps": K, "eta0": hp.eta0, "seconds": secs, "steps_per_s": K / secs,
            "E_per_site_last_window": float(E[-win:].mean()),
            "stderr": float(E[-win:].std(ddof=1) / np.sqrt(win)) if win > 1 else None,
            "window": win, "rejected_steps": int(np.sum(status != 0)),
            "E_exact_per_site": E_ref / w.model.N if E_ref is not None else None,
            "tab2_minsr_per_site": TAB2.get(key, (None, None))[0],
            "tab2_reference_per_site": TAB2.get(key, (None, None))[1],
            "trajectory_every_10pct": [float(E[min(K - 1, i * K // 10)]) for i in range(11)]}
    ref = line["E_exact_per_site"] or line["tab2_reference_per_site"]
    if ref:
        line["rel_err_last_window"] = (line["E_per_site_last_window"] - ref) / abs(ref)
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.workload.startswith("train:"):
        return run_train(args)
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
