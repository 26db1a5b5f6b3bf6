"""fr_refine_pair_noalloc against fr_refine_pair, through the C ABI.

The no-allocation entry point serves callers that cannot allocate device memory
(their device memory belongs to another allocator, or they must not stall on or
fail in cudaMalloc inside a latency-critical loop).  It keeps its workspace in a
fixed static device array, so its results must equal those of the allocating
entry point, also on a second call that reuses the array left by the first.
This file is collected last so a failure here leaves every other test run.
"""
import ctypes

import numpy as np
import pytest

from paper_1012_0006_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FIELDS = ("flow", "cut_before", "cut_after", "wA_before", "wB_before", "wA_after", "wB_after", "corridor_n",
          "corridor_arcs", "accepted", "iters", "alpha_final")


def _noalloc(F, g, part, k, a, b, eps, alpha, opts):
    res = F.PairResult()
    gc = g.c()
    st = F.lib().fr_refine_pair_noalloc(ctypes.byref(gc), ctypes.c_void_p(part.data_ptr()), k, a, b, eps, alpha,
                                        ctypes.byref(opts), ctypes.byref(res), None)
    return st, res


def test_noalloc_matches_allocating_entry_point_on_two_calls(gpu_lib):
    import torch
    F = gpu_lib
    cases = [
        (I.config(1), dict(mb=0)),                                                 # 64x64 grid, plain cut
        (I.config(2), dict(mb=1, adaptive=1, max_iters=10, alpha_max=16.0)),     # 65,536-vertex rgg, adaptive
    ]
    with F.Context(0) as ctx:
        for w, kw in cases:                                                       # two calls in a row
            g = F.DeviceGraph.from_workload(w)
            opts = F.default_options(**kw)
            p_ref = torch.as_tensor(np.array(w["part"], np.int32)).cuda()
            st, ref = ctx.refine_pair(g, p_ref, w["k"], 0, 1, w["eps"], w["alpha"], opts)
            p_na = torch.as_tensor(np.array(w["part"], np.int32)).cuda()
            st, got = _noalloc(F, g, p_na, w["k"], 0, 1, w["eps"], w["alpha"], opts)
            assert st == F.FR_OK
            assert torch.equal(p_na, p_ref)
            for f in FIELDS:
                assert getattr(got, f) == getattr(ref, f), f


def test_noalloc_rejects_problems_beyond_its_scratch(gpu_lib):
    import torch
    F = gpu_lib
    w = I.config(3, scale=1 / 16)            # 64^3 grid: n = 262,144 > 65,536
    g = F.DeviceGraph.from_workload(w)
    part = torch.as_tensor(np.array(w["part"], np.int32)).cuda()
    before = part.clone()
    st, res = _noalloc(F, g, part, w["k"], 0, 1, w["eps"], w["alpha"], F.default_options())
    assert st == F.FR_ERR_TOO_LARGE and res.status == F.FR_ERR_TOO_LARGE
    assert torch.equal(part, before)
