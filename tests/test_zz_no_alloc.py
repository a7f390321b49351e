"""nqs_logpsi_noalloc: log Psi for callers that cannot call cudaMalloc.

The allocation-free entry point keeps its scratch (packed weights, hidden-
state cache) in a static device array instead of a caller-allocated
workspace.  It must give the same log Psi as nqs_logpsi of an FP64 context,
call after call, and refuse batches whose scratch would not fit.  This file
is collected last so that a failure here cannot hide any other test.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2608_18065_b300 import nqs
from paper_2608_18065_b300.inputs import HamSpec, ModelSpec, init_theta, random_spins
from tests.gpu_helpers import RTOL64

pytestmark = pytest.mark.gpu

CASES = [(ModelSpec(1, 40, 1, 32), HamSpec("tfim")),
         (ModelSpec(2, 6, 6, 16, cplx=1, marshall=1, zmask=1), HamSpec("j1j2", J2=0.5))]


def _noalloc(model, theta, spins, out):
    L = nqs.lib()
    L.nqs_logpsi_noalloc.restype = C.c_int
    md = nqs.model_desc(model)
    return L.nqs_logpsi_noalloc(C.byref(md), C.c_void_p(theta.data_ptr()),
                                C.c_void_p(spins.data_ptr()), C.c_int64(spins.shape[0]),
                                C.c_void_p(out.data_ptr()),
                                C.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("model,ham", CASES, ids=["1d_N40_dh32", "2d_6x6_dh16"])
def test_noalloc_logpsi_matches_context_path_twice(model, ham):
    ctx = nqs.Context(model, ham, "fp64", 200)
    n = 150
    for seed in (1, 2):  # two calls in a row with different inputs
        th = torch.tensor(init_theta(model, seed), device="cuda")
        sp = torch.tensor(random_spins(model, n, seed=10 + seed, zero_mag=bool(model.zmask)),
                          device="cuda")
        ref = ctx.logpsi(th, sp)
        out = torch.full((n, 2), float("nan"), dtype=torch.float64, device="cuda")
        assert _noalloc(model, th, sp, out) == 0
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        np.testing.assert_allclose(a, b, rtol=RTOL64, atol=RTOL64)


def test_noalloc_rejects_batches_beyond_its_scratch():
    # 2D: the hidden-state cache (here 8 * 64 * 64 bytes per configuration)
    # must fit beside the packed weights
    model = ModelSpec(2, 8, 8, 64, cplx=1, marshall=1, zmask=1)
    th = torch.tensor(init_theta(model, 1), device="cuda")
    for n in (1000, 1 << 40):  # too large; so large that n * N * dh * 8 would wrap
        m = min(n, 1000)
        sp = torch.zeros((m, model.N), dtype=torch.uint8, device="cuda")
        out = torch.full((m, 2), float("nan"), dtype=torch.float64, device="cuda")
        L = nqs.lib()
        L.nqs_logpsi_noalloc.restype = C.c_int
        md = nqs.model_desc(model)
        rc = L.nqs_logpsi_noalloc(C.byref(md), C.c_void_p(th.data_ptr()),
                                  C.c_void_p(sp.data_ptr()), C.c_int64(n),
                                  C.c_void_p(out.data_ptr()),
                                  C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 7  # NQS_ERR_WORKSPACE, nothing launched
        torch.cuda.synchronize()
        assert torch.isnan(out).all()


def test_noalloc_1d_needs_no_state_cache():
    # a 1D chain keeps no scratch beyond the packed weights, so a batch whose
    # state cache alone would exceed the array (400 * 100 * 64 * 8 bytes) runs
    model = ModelSpec(1, 100, 1, 64)
    ctx = nqs.Context(model, HamSpec("tfim"), "fp64", 400)
    th = torch.tensor(init_theta(model, 3), device="cuda")
    sp = torch.tensor(random_spins(model, 400, seed=5), device="cuda")
    out = torch.full((400, 2), float("nan"), dtype=torch.float64, device="cuda")
    assert _noalloc(model, th, sp, out) == 0
    ref = ctx.logpsi(th, sp)
    torch.cuda.synchronize()
    np.testing.assert_allclose(out.cpu().numpy(), ref.cpu().numpy(), rtol=RTOL64, atol=RTOL64)
