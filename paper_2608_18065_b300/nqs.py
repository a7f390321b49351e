"""Thin ctypes binding of libnqs (include/nqs.h).

Argument marshalling only: every stage runs in the CUDA kernels of
libnqs.so.  torch supplies device memory (the workspace and the output
tensors) and streams.  Loading fails loudly if the library is missing.
"""
import ctypes as C
import os

import torch

from .inputs import HamSpec, HParams, ModelSpec

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnqs.so")
_lib = None

PREC = {"fp64": 0, "mixed": 1}
FAMILY = {"tfim": 0, "cluster_zxz": 1, "cluster_paper": 2, "j1j2": 3}


class NqsError(RuntimeError):
    pass


class ModelDesc(C.Structure):
    _fields_ = [("dim", C.c_int), ("Lx", C.c_int), ("Ly", C.c_int), ("dh", C.c_int),
                ("cplx", C.c_int), ("marshall", C.c_int), ("zmask", C.c_int)]


class HamDesc(C.Structure):
    _fields_ = [("family", C.c_int), ("J", C.c_double), ("h", C.c_double),
                ("J1", C.c_double), ("J2", C.c_double)]


class StepHParams(C.Structure):
    _fields_ = [("eta0", C.c_double), ("decay_T", C.c_double), ("mu", C.c_double),
                ("lam", C.c_double), ("lambda_coeff", C.c_double),
                ("lambda_pow", C.c_double), ("lambda_mode", C.c_int32),
                ("trust_region", C.c_int32), ("step_index", C.c_int64),
                ("seed", C.c_uint64), ("n_samples", C.c_int64)]


STATS_FIELDS = ["E_re", "E_im", "var", "vscore", "lam", "normT", "eta_eff", "tau_norm"]
STATS_DOUBLES = 11  # 8 doubles, (status, solve_fp64) as an int32 pair, rho, lambda_next


class Options(C.Structure):
    _fields_ = [("checkpoint_stride", C.c_int)]


class StepOutputs(C.Structure):
    _fields_ = [("spins", C.c_void_p), ("logpsi", C.c_void_p), ("eloc", C.c_void_p),
                ("T", C.c_void_p), ("eps", C.c_void_p), ("x", C.c_void_p),
                ("dtheta", C.c_void_p)]


N_STAGES = 14
SYMBOLS = ["nqs_create", "nqs_destroy", "nqs_param_count", "nqs_workspace_size",
           "nqs_set_workspace", "nqs_sample", "nqs_logpsi", "nqs_local_energy",
           "nqs_jacobian", "nqs_logpsi_vjp", "nqs_gram", "nqs_regularized_solve", "nqs_minsr_step",
           "nqs_minsr_step_ex", "nqs_set_graph", "nqs_graph_active", "nqs_timing_begin", "nqs_timing_end", "nqs_launch_count",
           "nqs_autotune", "nqs_get_tuning", "nqs_clear_tuning", "nqs_batch_create",
           "nqs_batch_destroy", "nqs_minsr_step_batched", "nqs_batch_set_graph",
           "nqs_batch_graph_active", "nqs_batch_set_concurrency", "nqs_batch_get_concurrency",
           "nqs_batch_autotune", "nqs_eloc_work", "nqs_create_ex", "nqs_checkpoint_stride",
           "nqs_set_damping", "nqs_spectrum", "nqs_shard_forward", "nqs_shard_center",
           "nqs_shard_solve", "nqs_shard_apply", "nqs_test_wait_timeout", "nqs_adam_step",
           "nqs_energy_scan", "nqs_set_solve_form", "nqs_set_sampler", "nqs_batch_set_grouped",
           "nqs_batch_get_grouped", "nqs_batch_set_eloc_share", "nqs_batch_get_eloc_share",
           "nqs_stage_name", "nqs_last_cuda_error", "nqs_status_string"]
TUNE_FORCE = 1


class AdamHParams(C.Structure):
    _fields_ = [("eta0", C.c_double), ("decay_T", C.c_double), ("beta1", C.c_double),
                ("beta2", C.c_double), ("epsilon", C.c_double), ("step_index", C.c_int64),
                ("seed", C.c_uint64), ("n_samples", C.c_int64)]


class SpectrumStats(C.Structure):
    _fields_ = [("lambda_max", C.c_double), ("lambda_min_ritz", C.c_double),
                ("kappa", C.c_double), ("digits_fp32", C.c_double),
                ("digits_fp64", C.c_double), ("residual", C.c_double),
                ("iterations", C.c_int32), ("status", C.c_int32)]


class Tuning(C.Structure):
    _fields_ = [("n_samples", C.c_int64), ("eloc_grid", C.c_int), ("gram_splits", C.c_int),
                ("solve_grid", C.c_int), ("solve_form", C.c_int),
                ("solve_substitution", C.c_int), ("reserved", C.c_int),
                ("ms", C.c_double * 3), ("ms_default", C.c_double * 3)]


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libnqs.so not built ({LIB_PATH}); run "
                              "python -m paper_2608_18065_b300.build")
        _lib = C.CDLL(LIB_PATH)
        _lib.nqs_status_string.restype = C.c_char_p
        _lib.nqs_stage_name.restype = C.c_char_p
        _lib.nqs_last_cuda_error.restype = C.c_char_p
        for name in SYMBOLS[:-3]:
            getattr(_lib, name).restype = C.c_int
        _lib.nqs_spectrum_workspace.restype = C.c_size_t
        _lib.nqs_spectrum_workspace.argtypes = [C.c_int64, C.c_int]
    return _lib


def _check(rc):
    if rc != 0:
        msg = f"libnqs: {lib().nqs_status_string(rc).decode()} ({rc})"
        if rc == 2:  # NQS_ERR_CUDA
            msg += ": " + lib().nqs_last_cuda_error().decode()
        raise NqsError(msg)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def model_desc(m: ModelSpec) -> ModelDesc:
    return ModelDesc(m.dim, m.Lx, m.Ly, m.dh, m.cplx, m.marshall, m.zmask)


def ham_desc(h: HamSpec) -> HamDesc:
    return HamDesc(FAMILY[h.family], h.J, h.h, h.J1, h.J2)


def step_hparams(hp: HParams, step_index: int) -> StepHParams:
    return StepHParams(hp.eta0, hp.decay_T, hp.mu, hp.lam, hp.lambda_coeff, hp.lambda_pow,
                       hp.lambda_mode, hp.trust_region, step_index, hp.seed, hp.ns)


class Context:
    """A libnqs context plus its torch-owned device workspace."""

    def __init__(self, model: ModelSpec, ham: HamSpec, precision: str, max_samples: int,
                 device="cuda", checkpoint_stride: int = 0):
        """checkpoint_stride: 0 caches every hidden state; c > 0 (or -1 for
        ceil(sqrt(N))) keeps every c-th and recomputes the rest (1D)."""
        self.model, self.ham, self.precision = model, ham, precision
        self.max_samples = int(max_samples)
        self.device = torch.device(device)
        with torch.cuda.device(self.device):
            h = C.c_void_p()
            opt = Options(int(checkpoint_stride))
            _check(lib().nqs_create_ex(C.byref(model_desc(model)), C.byref(ham_desc(ham)),
                                       PREC[precision], C.c_int64(self.max_samples),
                                       C.byref(opt), C.byref(h)))
            self._h = h
            n = C.c_int64()
            _check(lib().nqs_param_count(h, C.byref(n)))
            self.np = n.value
            b = C.c_size_t()
            _check(lib().nqs_workspace_size(h, C.byref(b)))
            self.workspace_bytes = b.value
            self.workspace = torch.empty(max(b.value, 256) + 256, dtype=torch.uint8,
                                         device=self.device)
            base = self.workspace.data_ptr()
            off = (-base) % 256
            _check(lib().nqs_set_workspace(h, C.c_void_p(base + off), C.c_size_t(b.value)))
        self.odtype = torch.float32 if precision == "mixed" else torch.float64
        self.rows_per_sample = 2 if model.cplx else 1

    def checkpoint_stride(self):
        v = C.c_int()
        _check(lib().nqs_checkpoint_stride(self._h, C.byref(v)))
        return v.value

    def close(self):
        if getattr(self, "_h", None):
            lib().nqs_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -------------------------------------------------------------- stages
    def sample(self, theta, ns, seed, step, stream=None):
        spins = torch.empty((ns, self.model.N), dtype=torch.uint8, device=self.device)
        lp = torch.empty((ns, 2), dtype=torch.float64, device=self.device)
        _check(lib().nqs_sample(self._h, _ptr(theta), C.c_int64(ns), C.c_uint64(seed),
                                C.c_uint64(step), _ptr(spins), _ptr(lp), _stream(stream)))
        return spins, lp

    def logpsi(self, theta, spins, stream=None):
        spins = spins.contiguous()
        n = spins.shape[0]
        lp = torch.empty((n, 2), dtype=torch.float64, device=self.device)
        _check(lib().nqs_logpsi(self._h, _ptr(theta), _ptr(spins), C.c_int64(n), _ptr(lp),
                                _stream(stream)))
        return lp

    def local_energy(self, theta, spins, stream=None):
        spins = spins.contiguous()
        n = spins.shape[0]
        el = torch.empty((n, 2), dtype=torch.float64, device=self.device)
        _check(lib().nqs_local_energy(self._h, _ptr(theta), _ptr(spins), C.c_int64(n),
                                      _ptr(el), _stream(stream)))
        return el

    def jacobian(self, theta, spins, stream=None):
        spins = spins.contiguous()
        n = spins.shape[0]
        O = torch.empty((n * self.rows_per_sample, self.np), dtype=self.odtype,
                        device=self.device)
        _check(lib().nqs_jacobian(self._h, _ptr(theta), _ptr(spins), C.c_int64(n), _ptr(O),
                                  _stream(stream)))
        return O

    def logpsi_vjp(self, theta, spins, grad_logpsi, stream=None):
        spins = spins.contiguous()
        g = grad_logpsi.to(torch.float64).contiguous()
        out = torch.empty(self.np, dtype=torch.float64, device=self.device)
        _check(lib().nqs_logpsi_vjp(self._h, _ptr(theta), _ptr(spins), C.c_int64(spins.shape[0]),
                                    _ptr(g), _ptr(out), _stream(stream)))
        return out

    def gram(self, A, stream=None):
        A = A.contiguous()
        R, np_ = A.shape
        T = torch.empty((R, R), dtype=torch.float64, device=self.device)
        _check(lib().nqs_gram(self._h, _ptr(A), C.c_int64(R), C.c_int64(np_), _ptr(T),
                              _stream(stream)))
        return T

    def regularized_solve(self, T, lam, b, stream=None):
        """Returns (x, device status); T is overwritten by its factor."""
        R = T.shape[0]
        x = torch.empty(R, dtype=torch.float64, device=self.device)
        status = torch.zeros(1, dtype=torch.int32, device=self.device)
        _check(lib().nqs_regularized_solve(self._h, _ptr(T), C.c_int64(R), C.c_double(lam),
                                           _ptr(b), _ptr(x), _ptr(status), _stream(stream)))
        return x, status

    def new_stats(self):
        return torch.zeros(STATS_DOUBLES, dtype=torch.float64, device=self.device)

    def minsr_step(self, theta, mom, hp: HParams, step_index, stats=None, outputs=None,
                   stream=None):
        """One step of Algorithm 1 in place on theta/mom (device FP64)."""
        if stats is None:
            stats = self.new_stats()
        hps = step_hparams(hp, step_index)
        if outputs is None:
            _check(lib().nqs_minsr_step(self._h, _ptr(theta), _ptr(mom), C.byref(hps),
                                        _ptr(stats), _stream(stream)))
        else:
            o = StepOutputs(*[(outputs[k].data_ptr() if k in outputs else None)
                              for k in ("spins", "logpsi", "eloc", "T", "eps", "x", "dtheta")])
            _check(lib().nqs_minsr_step_ex(self._h, _ptr(theta), _ptr(mom), C.byref(hps),
                                           _ptr(stats), C.byref(o), _stream(stream)))
        return stats

    # ------------------------------------------------ sample-sharded step
    def shard_sums_len(self):
        return self.rows_per_sample * self.np + 3

    def shard_forward(self, theta, hp: HParams, step_index, s0, n, sums=None, stream=None):
        """Sampling, E_loc and O of samples s0 .. s0 + n - 1; partial sums."""
        if sums is None:
            sums = torch.empty(self.shard_sums_len(), dtype=torch.float64, device=self.device)
        hps = step_hparams(hp, step_index)
        _check(lib().nqs_shard_forward(self._h, _ptr(theta), C.byref(hps), C.c_int64(s0),
                                       C.c_int64(n), _ptr(sums), _stream(stream)))
        return sums

    def shard_center(self, sums, ns, n, stats, stream=None):
        """This rank's centred rows O' [nblk*n, Np] and eps-bar' [nblk*n]."""
        rows = torch.empty((self.rows_per_sample * n, self.np), dtype=self.odtype,
                           device=self.device)
        eps = torch.empty(self.rows_per_sample * n, dtype=torch.float64, device=self.device)
        _check(lib().nqs_shard_center(self._h, _ptr(sums), C.c_int64(ns), C.c_int64(n),
                                      _ptr(rows), _ptr(eps), _ptr(stats), _stream(stream)))
        return rows, eps

    def shard_solve(self, rows, eps, hp: HParams, step_index, p0, p1, stats, stream=None):
        """T, lambda, x, eta from the gathered rows; delta theta [p0, p1)."""
        dth = torch.empty(max(p1 - p0, 1), dtype=torch.float64, device=self.device)
        hps = step_hparams(hp, step_index)
        _check(lib().nqs_shard_solve(self._h, _ptr(rows), C.c_int64(rows.shape[0]), _ptr(eps),
                                     C.byref(hps), C.c_int64(p0), C.c_int64(p1), _ptr(dth),
                                     _ptr(stats), _stream(stream)))
        return dth[:p1 - p0]

    def shard_apply(self, theta, mom, dtheta, hp: HParams, step_index, stats, stream=None):
        hps = step_hparams(hp, step_index)
        _check(lib().nqs_shard_apply(self._h, _ptr(theta), _ptr(mom), _ptr(dtheta),
                                     C.byref(hps), _ptr(stats), _stream(stream)))

    def adam_step(self, theta, m1, m2, ap, step_index, stats=None, grad=None, stream=None):
        """One Adam iteration (Sec. II.C baseline) in place on theta, m1, m2."""
        if stats is None:
            stats = self.new_stats()
        a = AdamHParams(ap.eta0, ap.decay_T, ap.beta1, ap.beta2, ap.eps, step_index, ap.seed,
                        ap.ns)
        _check(lib().nqs_adam_step(self._h, _ptr(theta), _ptr(m1), _ptr(m2), C.byref(a),
                                   _ptr(stats), _ptr(grad), _stream(stream)))
        return stats

    def energy_scan(self, theta0, v1, v2, xy, ns, seed, stream=None):
        """E(theta0 + x v1 + y v2) for the host (x, y) pairs xy [n, 2] (Sec. IV);
        returns a device [n, 4] tensor (Re E, Im E, Var, status)."""
        import numpy as np
        xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
        out = torch.empty((len(xy), 4), dtype=torch.float64, device=self.device)
        _check(lib().nqs_energy_scan(self._h, _ptr(theta0), _ptr(v1), _ptr(v2),
                                     xy.ctypes.data_as(C.c_void_p), C.c_int64(len(xy)),
                                     C.c_int64(ns), C.c_uint64(seed), _ptr(out),
                                     _stream(stream)))
        return out

    def test_wait_timeout(self, spin_limit=0, drop_tile=False):
        """Failure-detection test hook of the streamed 2D local-energy engine
        (see nqs_test_wait_timeout); (0, False) restores normal operation."""
        _check(lib().nqs_test_wait_timeout(self._h, C.c_uint64(spin_limit), int(drop_tile)))

    def set_damping(self, omega, lambda0):
        """Levenberg-Marquardt damping (App. G): omega > 1 on, else off."""
        _check(lib().nqs_set_damping(self._h, C.c_double(omega), C.c_double(lambda0)))

    def use_graph(self, enable=True):
        _check(lib().nqs_set_graph(self._h, 1 if enable else 0))

    def graph_active(self):
        v = C.c_int()
        _check(lib().nqs_graph_active(self._h, C.byref(v)))
        return bool(v.value)

    # ------------------------------------------------------ instrumentation
    def timing_begin(self, max_steps):
        _check(lib().nqs_timing_begin(self._h, int(max_steps)))

    def timing_end(self):
        """{stage name: summed ms}, number of timed steps."""
        ms = (C.c_double * N_STAGES)()
        n = C.c_int()
        _check(lib().nqs_timing_end(self._h, ms, C.byref(n)))
        return {lib().nqs_stage_name(i).decode(): ms[i] for i in range(N_STAGES)}, n.value

    def eloc_work(self):
        """(connected configurations, recomputed sites) of the last E_loc pass."""
        a, b = C.c_int64(), C.c_int64()
        _check(lib().nqs_eloc_work(self._h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def launch_count(self):
        n = C.c_int64()
        _check(lib().nqs_launch_count(self._h, C.byref(n)))
        return n.value

    # ------------------------------------------------------------ autotuner
    def autotune(self, theta, hp: HParams, step_index=0, force=False, stream=None):
        """Measure and keep the launch shapes for hp.ns samples (synchronous;
        theta is not modified)."""
        hps = step_hparams(hp, step_index)
        _check(lib().nqs_autotune(self._h, _ptr(theta), C.byref(hps),
                                  TUNE_FORCE if force else 0, _stream(stream)))
        return self.tuning()

    def tuning(self):
        t = Tuning()
        _check(lib().nqs_get_tuning(self._h, C.byref(t)))
        names = ("eloc", "gram", "solve")
        return {"n_samples": t.n_samples, "eloc_grid": t.eloc_grid,
                "gram_splits": t.gram_splits, "solve_grid": t.solve_grid,
                "solve_form": t.solve_form,
                "solve_substitution": t.solve_substitution,
                "ms": dict(zip(names, list(t.ms))),
                "ms_default": dict(zip(names, list(t.ms_default)))}

    def clear_tuning(self):
        _check(lib().nqs_clear_tuning(self._h))

    def set_sampler(self, form):
        """Sampler of a mixed 2D d_h 96/128 context: 1 tensor-core engine,
        0 recurrence kernels, -1 built-in (nqs_set_sampler)."""
        _check(lib().nqs_set_sampler(self._h, int(form)))

    def set_solve_form(self, form):
        """Form of the mixed regularized solve: 0 / 1 32-wide panels (tiles
        per CTA / per warp), 2 128-wide panels, -1 built-in (nqs_set_solve_form)."""
        _check(lib().nqs_set_solve_form(self._h, int(form)))

    def step_outputs(self, ns):
        R = ns * self.rows_per_sample
        d = self.device
        return dict(spins=torch.empty((ns, self.model.N), dtype=torch.uint8, device=d),
                    logpsi=torch.empty((ns, 2), dtype=torch.float64, device=d),
                    eloc=torch.empty((ns, 2), dtype=torch.float64, device=d),
                    T=torch.empty((R, R), dtype=torch.float64, device=d),
                    eps=torch.empty(R, dtype=torch.float64, device=d),
                    x=torch.empty(R, dtype=torch.float64, device=d),
                    dtheta=torch.empty(self.np, dtype=torch.float64, device=d))


class Batch:
    """n independent contexts stepped together (nqs_minsr_step_batched)."""

    def __init__(self, contexts):
        self.contexts = list(contexts)
        n = len(self.contexts)
        arr = (C.c_void_p * n)(*[c._h for c in self.contexts])
        h = C.c_void_p()
        _check(lib().nqs_batch_create(n, arr, C.byref(h)))
        self._h = h
        self.device = self.contexts[0].device

    def close(self):
        if getattr(self, "_h", None):
            lib().nqs_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def new_stats(self):
        return torch.zeros((len(self.contexts), STATS_DOUBLES), dtype=torch.float64,
                           device=self.device)

    def _arrays(self, thetas, hps, step_index):
        n = len(self.contexts)
        if len(thetas) != n or len(hps) != n:
            raise ValueError("one theta and one HParams per instance")
        steps = step_index if isinstance(step_index, (list, tuple)) else [step_index] * n
        th = (C.c_void_p * n)(*[t.data_ptr() for t in thetas])
        hp = (StepHParams * n)(*[step_hparams(h, int(s)) for h, s in zip(hps, steps)])
        return th, hp

    def step(self, thetas, moms, hps, step_index, stats=None, stream=None):
        """One step of every instance; stats: device [n, 9] doubles."""
        if stats is None:
            stats = self.new_stats()
        th, hp = self._arrays(thetas, hps, step_index)
        mo = (C.c_void_p * len(moms))(*[m.data_ptr() for m in moms])
        _check(lib().nqs_minsr_step_batched(self._h, th, mo, hp, _ptr(stats), _stream(stream)))
        return stats

    def autotune(self, thetas, hps, step_index=0, force=False, stream=None):
        """Tune every instance, then the concurrency; returns the best batched
        step time in ms (thetas are not modified)."""
        th, hp = self._arrays(thetas, hps, step_index)
        ms = C.c_double()
        _check(lib().nqs_batch_autotune(self._h, th, hp, TUNE_FORCE if force else 0,
                                        C.byref(ms), _stream(stream)))
        return ms.value

    def use_graph(self, enable=True):
        _check(lib().nqs_batch_set_graph(self._h, 1 if enable else 0))

    def graph_active(self):
        v = C.c_int()
        _check(lib().nqs_batch_graph_active(self._h, C.byref(v)))
        return bool(v.value)

    def set_concurrency(self, streams):
        _check(lib().nqs_batch_set_concurrency(self._h, int(streams)))

    def concurrency(self):
        v = C.c_int()
        _check(lib().nqs_batch_get_concurrency(self._h, C.byref(v)))
        return v.value

    def set_grouped(self, stages=3):
        """Batched step by stage (nqs_batch_set_grouped): bit 1 the FP32
        solves of all instances in one cooperative launch, bit 2 the
        streamed local-energy engines in one launch per hidden size; True
        is both, False neither."""
        stages = 3 if stages is True else 0 if stages is False else int(stages)
        _check(lib().nqs_batch_set_grouped(self._h, stages))

    def grouped(self):
        v = C.c_int()
        _check(lib().nqs_batch_get_grouped(self._h, C.byref(v)))
        return v.value

    def set_eloc_share(self, eighths):
        """Eighths of its grid each instance's local-energy engine takes in
        a batched step (nqs_batch_set_eloc_share)."""
        _check(lib().nqs_batch_set_eloc_share(self._h, int(eighths)))

    def eloc_share(self):
        v = C.c_int()
        _check(lib().nqs_batch_get_eloc_share(self._h, C.byref(v)))
        return v.value


def decode_stats(stats: torch.Tensor) -> dict:
    v = stats.detach().cpu()
    d = {k: float(v[i]) for i, k in enumerate(STATS_FIELDS)}
    d["status"] = int(v[8:9].view(torch.int32)[0])
    d["solve_fp64"] = int(v[8:9].view(torch.int32)[1])
    d["rho"] = float(v[9])
    d["lambda_next"] = float(v[10])
    return d


class LogPsi(torch.autograd.Function):
    """log Psi(sigma; theta) as a differentiable torch function.

    forward: nqs_logpsi -> (n, 2) FP64 tensor (Re, Im of log Psi).
    backward: nqs_logpsi_vjp, the hand-written reverse-mode Jacobian kernels
    contracted with the incoming cotangent on the device.  Gradients flow to
    theta only (spins are discrete)."""

    @staticmethod
    def forward(fctx, theta, spins, context):
        fctx.context = context
        fctx.save_for_backward(theta, spins)
        return context.logpsi(theta, spins)

    @staticmethod
    def backward(fctx, grad_out):
        theta, spins = fctx.saved_tensors
        g = fctx.context.logpsi_vjp(theta, spins, grad_out)
        return g, None, None


def logpsi(theta, spins, context):
    return LogPsi.apply(theta, spins, context)


def spectrum(T, lam, m=64, seed=1, stream=None):
    """Conditioning diagnostics of T + lam I (App. E) through nqs_spectrum:
    lambda_max(T), the smallest Ritz value, kappa_2 = (lambda_max + lam)/lam
    (lambda_min(T) = 0 for the centred Gram matrix), the reliable digits in
    FP32 and FP64, the Ritz residual, the Lanczos steps and the device
    status.  T: square contiguous FP64 CUDA tensor (not modified)."""
    assert T.dtype == torch.float64 and T.is_cuda and T.is_contiguous()
    R = T.shape[0]
    wb = lib().nqs_spectrum_workspace(R, m)
    if wb == 0:
        raise NqsError("libnqs: invalid argument (spectrum size)")
    work = torch.empty(wb, dtype=torch.uint8, device=T.device)
    out = torch.zeros(C.sizeof(SpectrumStats), dtype=torch.uint8, device=T.device)
    _check(lib().nqs_spectrum(_ptr(T), C.c_int64(R), C.c_double(lam), C.c_int(m),
                              C.c_uint64(seed), _ptr(work), C.c_size_t(wb), _ptr(out),
                              _stream(stream)))
    st = SpectrumStats.from_buffer_copy(out.cpu().numpy().tobytes())
    return {f: getattr(st, f) for f, _ in SpectrumStats._fields_}
