"""fr_refine_pair_noalloc against the oracle and fr_refine_pair, through the C ABI.

The no-allocation entry point serves callers that cannot allocate device memory
(their device memory belongs to another allocator, or they must not stall on or
fail in cudaMalloc inside a latency-critical loop).  It keeps its workspace in a
fixed static device array shared by every call, so its results must equal the
oracle's and those of the allocating entry point on every call of a sequence that
reuses the array: large problem, small one, large again, the same input twice, and a
normal call right after one that failed.  Device memory must not change across a
call.  This file is collected last so a failure here leaves every other test run.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_1012_0006_gb300 import inputs as I
from tests.pulse_caps import later_iteration_cap

pytestmark = pytest.mark.gpu

FIELDS = ("flow", "cut_before", "cut_after", "wA_before", "wB_before", "wA_after", "wB_after", "corridor_n",
          "corridor_arcs", "accepted", "iters", "alpha_final")
ORACLE_FIELDS = ("flow", "cut_before", "cut_after", "wA_before", "wB_before", "wA_after", "wB_after",
                 "corridor_n", "corridor_arcs", "accepted", "iters", "alpha_final")

PLAIN = dict(mb=0)
ADAPTIVE_MB = dict(mb=1, adaptive=1, max_iters=10, alpha_max=16.0)


def _noalloc(F, g, part, k, a, b, eps, alpha, opts):
    res = F.PairResult()
    gc = g.c()
    st = F.lib().fr_refine_pair_noalloc(ctypes.byref(gc), ctypes.c_void_p(part.data_ptr()), k, a, b, eps, alpha,
                                        ctypes.byref(opts), ctypes.byref(res), None)
    return st, res


def _part(w):
    import torch
    return torch.as_tensor(np.array(w["part"], np.int32)).cuda()


def _oracle_opts(kw):
    return O.options(mb=kw.get("mb", 0), adaptive=kw.get("adaptive", 0), max_iters=kw.get("max_iters", 1),
                     alpha_max=kw.get("alpha_max", 1.0))


def test_noalloc_matches_oracle_and_allocating_entry_point_large_small_large(gpu_lib):
    """65,536-vertex rgg (adaptive, most balanced), 64x64 grid (plain), the rgg again, and
    the grid twice more with the same input: every call against the oracle and against
    fr_refine_pair, so stale scratch beyond a smaller n would show."""
    import torch
    F = gpu_lib
    c1, c2 = I.config(1), I.config(2)
    seq = [(c2, ADAPTIVE_MB), (c1, PLAIN), (c2, ADAPTIVE_MB), (c1, PLAIN), (c1, PLAIN)]
    expect = {}
    with F.Context(0) as ctx:
        for w, kw in seq:
            key = (w["n"], tuple(sorted(kw.items())))
            if key not in expect:
                st, pref, rref = O.refine_pair(w, 0, 1, opts=_oracle_opts(kw))
                assert st == 0
                expect[key] = (pref, rref)
            pref, rref = expect[key]
            g = F.DeviceGraph.from_workload(w)
            opts = F.default_options(**kw)
            p_ref = _part(w)
            st, ref = ctx.refine_pair(g, p_ref, w["k"], 0, 1, w["eps"], w["alpha"], opts)
            assert st == F.FR_OK
            p_na = _part(w)
            st, got = _noalloc(F, g, p_na, w["k"], 0, 1, w["eps"], w["alpha"], opts)
            assert st == F.FR_OK and got.status == F.FR_OK
            assert np.array_equal(p_na.cpu().numpy(), pref)
            assert torch.equal(p_na, p_ref)
            for f in ORACLE_FIELDS:
                assert getattr(got, f) == getattr(rref, f), f
            for f in FIELDS:
                assert getattr(got, f) == getattr(ref, f), f


def test_noalloc_allocates_no_device_memory(gpu_lib):
    """After a first call (which loads the library's kernels and its static array onto
    the device), calls leave the device's free memory exactly as it was."""
    import torch
    F = gpu_lib
    w = I.config(2)
    g = F.DeviceGraph.from_workload(w)
    opts = F.default_options(**ADAPTIVE_MB)
    parts = [_part(w) for _ in range(3)]
    torch.cuda.synchronize()
    st, _ = _noalloc(F, g, parts[0], w["k"], 0, 1, w["eps"], w["alpha"], opts)
    assert st == F.FR_OK
    torch.cuda.synchronize()
    for p in parts[1:]:
        free0, _ = torch.cuda.mem_get_info()
        st, _ = _noalloc(F, g, p, w["k"], 0, 1, w["eps"], w["alpha"], opts)
        free1, _ = torch.cuda.mem_get_info()
        assert st == F.FR_OK
        assert free1 == free0
    assert torch.equal(parts[1], parts[2])


def test_noalloc_after_a_failed_call(gpu_lib):
    """A call stopped by the pulse cap (a host-side bound, no fault) fails with part
    unchanged; the next call on the same array matches a fresh fr_refine_pair."""
    import torch
    F = gpu_lib
    w = I.config(2)
    g = F.DeviceGraph.from_workload(w)
    part = _part(w)
    before = part.clone()
    st, res = _noalloc(F, g, part, w["k"], 0, 1, w["eps"], w["alpha"], F.default_options(mb=1, pulse_cap=1))
    assert st == F.FR_ERR_ITER_LIMIT and res.status == F.FR_ERR_ITER_LIMIT
    assert torch.equal(part, before)
    opts = F.default_options(**ADAPTIVE_MB)
    st, got = _noalloc(F, g, part, w["k"], 0, 1, w["eps"], w["alpha"], opts)
    assert st == F.FR_OK
    p_ref = _part(w)
    with F.Context(0) as ctx:
        st, ref = ctx.refine_pair(g, p_ref, w["k"], 0, 1, w["eps"], w["alpha"], opts)
    assert torch.equal(part, p_ref)
    for f in FIELDS:
        assert getattr(got, f) == getattr(ref, f), f


@pytest.mark.parametrize("mb", [0, 1])
def test_noalloc_error_in_a_later_adaptive_iteration_leaves_part_unchanged(gpu_lib, mb):
    """Iteration 1 is accepted and written; iteration 2 hits the pulse cap: the call
    fails and part is as it came in (the array's copy of it is written back)."""
    import torch
    F = gpu_lib
    tried = 0
    for w in (I.config(2, scale=0.5), I.config(2, scale=0.25), I.config(2)):
        g = F.DeviceGraph.from_workload(w)
        cap = later_iteration_cap(
            lambda p, al, kw: _noalloc(F, g, p, w["k"], 0, 1, w["eps"], al, F.default_options(**kw))[1], w,
            dict(mb=mb))
        if cap is None:
            continue
        tried += 1
        part = _part(w)
        before = part.clone()
        st, res = _noalloc(F, g, part, w["k"], 0, 1, w["eps"], 1.0,
                           F.default_options(mb=mb, adaptive=1, max_iters=10, alpha_max=16.0, pulse_cap=cap))
        assert st == F.FR_ERR_ITER_LIMIT and res.status == F.FR_ERR_ITER_LIMIT
        assert res.iters >= 2
        assert torch.equal(part, before)
        break
    assert tried, "no workload separates the pulse counts of the first two iterations"


def test_noalloc_rejects_problems_beyond_its_scratch(gpu_lib):
    import torch
    F = gpu_lib
    w = I.config(3, scale=1 / 16)            # 64^3 grid: n = 262,144 > 65,536
    g = F.DeviceGraph.from_workload(w)
    part = _part(w)
    before = part.clone()
    st, res = _noalloc(F, g, part, w["k"], 0, 1, w["eps"], w["alpha"], F.default_options())
    assert st == F.FR_ERR_TOO_LARGE and res.status == F.FR_ERR_TOO_LARGE
    assert torch.equal(part, before)


def test_noalloc_checks_options_as_the_allocating_entry_point_does(gpu_lib):
    """Options fr_refine_pair rejects are rejected here too, before any device work."""
    import torch
    F = gpu_lib
    w = I.config(1)
    g = F.DeviceGraph.from_workload(w)
    part = _part(w)
    before = part.clone()
    bad = [dict(block_threads=128), dict(pulse_cap=-1), dict(pre_waves=7), dict(cluster_ctas=5),
           dict(fm_permille=10), dict(mt_alpha=10)]
    for kw in bad:
        st, res = _noalloc(F, g, part, w["k"], 0, 1, w["eps"], w["alpha"], F.default_options(**kw))
        assert st == F.FR_ERR_INVALID_ARG, kw
        assert torch.equal(part, before)
