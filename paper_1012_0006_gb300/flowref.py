"""Python binding of libflowref (include/flowref.h).

Argument marshalling only: every step of the refinement runs in the CUDA kernels
of lib/libflowref.so.  PyTorch provides device memory and streams.  There is no
fallback: if the library or a CUDA device is missing, loading fails loudly.

The C entry points are exposed under their own names (fr_create,
fr_refine_pair, ...) on the loaded library `lib()`; `Context` wraps them for
torch tensors.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libflowref.so")

FR_OK, FR_ERR_INVALID_ARG, FR_ERR_CUDA, FR_ERR_OOM = 0, 1, 2, 3
FR_ERR_ITER_LIMIT, FR_ERR_TOO_LARGE, FR_ERR_ABORTED, FR_ERR_INTERNAL = 4, 5, 6, 7

i8p = ctypes.POINTER(ctypes.c_int8)
i32p = ctypes.POINTER(ctypes.c_int32)
i64p = ctypes.POINTER(ctypes.c_int64)
vp = ctypes.c_void_p


class Graph(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int32), ("xadj", vp), ("adjncy", vp), ("adjwgt", vp),
                ("vwgt", vp)]


class Options(ctypes.Structure):
    _fields_ = [("mb", ctypes.c_int32), ("mb_reps", ctypes.c_int32), ("adaptive", ctypes.c_int32),
                ("max_iters", ctypes.c_int32), ("alpha_max", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("pulse_cap", ctypes.c_int64), ("checked", ctypes.c_int32), ("block_threads", ctypes.c_int32),
                ("grid_blocks", ctypes.c_int32), ("gr_interval", ctypes.c_int32), ("inner_ops", ctypes.c_int32),
                ("pulse_passes", ctypes.c_int32), ("flow_sched", ctypes.c_int32), ("cluster_ctas", ctypes.c_int32),
                ("pre_waves", ctypes.c_int32), ("fm_permille", ctypes.c_int32), ("mt_alpha", ctypes.c_int32),
                ("sweep_sched", ctypes.c_int32), ("gap_interval", ctypes.c_int32)]


class PairResult(ctypes.Structure):
    _fields_ = [("flow", ctypes.c_int64), ("cut_before", ctypes.c_int64), ("cut_after", ctypes.c_int64),
                ("wA_before", ctypes.c_int64), ("wB_before", ctypes.c_int64), ("wA_after", ctypes.c_int64),
                ("wB_after", ctypes.c_int64), ("corridor_n", ctypes.c_int32), ("corridor_arcs", ctypes.c_int32),
                ("accepted", ctypes.c_int32), ("iters", ctypes.c_int32), ("alpha_final", ctypes.c_double),
                ("status", ctypes.c_int32), ("a", ctypes.c_int32), ("b", ctypes.c_int32), ("round", ctypes.c_int32),
                ("pulses", ctypes.c_int64), ("relabels", ctypes.c_int64), ("bfs_levels", ctypes.c_int32),
                ("scc_rounds", ctypes.c_int32), ("ncomp", ctypes.c_int32), ("fm_moves", ctypes.c_int32),
                ("cut_fm", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "pad0"}


class BatchResult(ctypes.Structure):
    _fields_ = [("npairs", ctypes.c_int32), ("nrounds", ctypes.c_int32), ("accepted", ctypes.c_int32),
                ("status", ctypes.c_int32), ("cut_before", ctypes.c_int64), ("cut_after", ctypes.c_int64),
                ("corridor_arcs", ctypes.c_int64), ("device_ns", ctypes.c_int64), ("flow_ns", ctypes.c_int64),
                ("mt_gain", ctypes.c_int64), ("mt_searches", ctypes.c_int32), ("mt_tried", ctypes.c_int32),
                ("mt_kept", ctypes.c_int32), ("pad0", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "pad0"}


class VcycleResult(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("status", ctypes.c_int32), ("cut_before", ctypes.c_int64),
                ("cut_after", ctypes.c_int64), ("level_n", ctypes.c_int32 * 64), ("level_pairs", ctypes.c_int32 * 64),
                ("level_cut", ctypes.c_int64 * 64), ("coarsen_ms", ctypes.c_double), ("refine_ms", ctypes.c_double)]

    def as_dict(self):
        L = self.levels
        return dict(levels=L, status=self.status, cut_before=self.cut_before, cut_after=self.cut_after,
                    level_n=list(self.level_n[:L]), level_pairs=list(self.level_pairs[:L]),
                    level_cut=list(self.level_cut[:L]), coarsen_ms=self.coarsen_ms, refine_ms=self.refine_ms)


class CycleResult(ctypes.Structure):
    _fields_ = [("coarsenings", ctypes.c_int32), ("refinements", ctypes.c_int32), ("depth", ctypes.c_int32),
                ("status", ctypes.c_int32), ("cut_before", ctypes.c_int64), ("cut_after", ctypes.c_int64),
                ("level_coarsenings", ctypes.c_int32 * 64), ("ms", ctypes.c_double)]

    def as_dict(self):
        return dict(coarsenings=self.coarsenings, refinements=self.refinements, depth=self.depth,
                    status=self.status, cut_before=self.cut_before, cut_after=self.cut_after,
                    level_coarsenings=list(self.level_coarsenings[:max(self.depth, 1)]), ms=self.ms)


class MtResult(ctypes.Structure):
    _fields_ = [("gain", ctypes.c_int64), ("searches", ctypes.c_int32), ("tried", ctypes.c_int32),
                ("kept", ctypes.c_int32), ("status", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ProfileInfo(ctypes.Structure):
    _fields_ = [("nrounds", ctypes.c_int32), ("launches", ctypes.c_int32), ("scan_ms", ctypes.c_double),
                ("step_ms", ctypes.c_double), ("cluster_ms", ctypes.c_double), ("phase_ms", ctypes.c_double * 12), ("n", ctypes.c_int64),
                ("nnz", ctypes.c_int64), ("bfs_visited", ctypes.c_int64), ("bfs_arcs", ctypes.c_int64),
                ("corridor_n", ctypes.c_int64), ("corridor_arcs", ctypes.c_int64), ("pulses", ctypes.c_int64),
                ("relabels", ctypes.c_int64), ("gr_arcs", ctypes.c_int64), ("pr_arcs", ctypes.c_int64),
                ("pushes", ctypes.c_int64), ("scc_rounds", ctypes.c_int64), ("barriers", ctypes.c_int64),
                ("cluster_phase_ms", ctypes.c_double * 7), ("cluster_syncs", ctypes.c_int64),
                ("cluster_remote_arcs", ctypes.c_int64),
                ("fallback_pairs", ctypes.c_int64),
                ("scan_listed", ctypes.c_int64), ("scan_rows", ctypes.c_int64), ("scan_arcs", ctypes.c_int64),
                ("fm_ms", ctypes.c_double * 3), ("cluster_sizes", ctypes.c_int32 * 5), ("cluster_max_active", ctypes.c_int32 * 5),
                ("queue", ctypes.c_int32), ("queue_ctas", ctypes.c_int32), ("queue_clusters", ctypes.c_int32),
                ("queue_fallbacks", ctypes.c_int32), ("queue_scan_ms", ctypes.c_double),
                ("gaps", ctypes.c_int64), ("gap_lifted", ctypes.c_int64)]

    PHASES = ("bfs", "select", "lid", "build", "flow", "relabel", "return", "reach", "scc", "sweep", "eval",
              "commit")

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_
             if f not in ("phase_ms", "cluster_phase_ms", "cluster_sizes", "cluster_max_active", "fm_ms")}
        d["fm_ms"] = dict(zip(("sort", "moves", "finish"), list(self.fm_ms)))
        d["phase_ms"] = dict(zip(self.PHASES, list(self.phase_ms)))
        d["cluster_phase_ms"] = dict(zip(("load", "flow", "return", "reach", "scc", "members", "relabel"),
                                         list(self.cluster_phase_ms)))
        d["cluster_sizes"] = list(self.cluster_sizes)
        d["cluster_max_active"] = list(self.cluster_max_active)
        return d


class ServerConfig(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("max_inflight", ctypes.c_int32), ("arena_bytes", ctypes.c_size_t),
                ("opt", Options)]


class Request(ctypes.Structure):
    _fields_ = [("graph_id", ctypes.c_int32), ("k", ctypes.c_int32), ("eps", ctypes.c_double),
                ("alpha", ctypes.c_double), ("part_host", i32p), ("tag", ctypes.c_uint64)]


class Response(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("status", ctypes.c_int32), ("npairs", ctypes.c_int32),
                ("nrounds", ctypes.c_int32), ("accepted", ctypes.c_int32), ("cut_before", ctypes.c_int64),
                ("cut_after", ctypes.c_int64), ("latency_ms", ctypes.c_double), ("queue_ms", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


# Every symbol declared in include/flowref.h (checked by the CPU test suite).
SYMBOLS = {
    "fr_default_options": (None, [ctypes.POINTER(Options)]),
    "fr_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int32, ctypes.c_size_t, vp]),
    "fr_destroy": (ctypes.c_int, [vp]),
    "fr_last_error": (ctypes.c_char_p, [vp]),
    "fr_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "fr_workspace_bytes": (ctypes.c_size_t, [vp]),
    "fr_build_corridor": (ctypes.c_int, [vp, ctypes.POINTER(Graph), vp, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.POINTER(vp)]),
    "fr_corridor_info": (ctypes.c_int, [vp, i32p, i32p]),
    "fr_corridor_export": (ctypes.c_int, [vp, vp, i32p, i32p, i32p, i32p, i8p, i32p, i8p, i32p]),
    "fr_maxflow": (ctypes.c_int, [vp, vp, i64p]),
    "fr_corridor_flow": (ctypes.c_int, [vp, vp, i64p, i64p]),
    "fr_extract_cut": (ctypes.c_int, [vp, vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, vp,
                                      ctypes.POINTER(PairResult)]),
    "fr_corridor_sets": (ctypes.c_int, [vp, vp, i8p, i8p, i32p, i8p]),
    "fr_corridor_free": (ctypes.c_int, [vp, vp]),
    "fr_refine_pair": (ctypes.c_int, [vp, ctypes.POINTER(Graph), vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_double, ctypes.c_double, ctypes.POINTER(Options),
                                      ctypes.POINTER(PairResult)]),
    "fr_refine_batch": (ctypes.c_int, [vp, ctypes.POINTER(Graph), vp, ctypes.c_int32, ctypes.c_double,
                                       ctypes.c_double, ctypes.POINTER(Options), ctypes.c_int32,
                                       ctypes.POINTER(PairResult), ctypes.POINTER(BatchResult)]),
    "fr_refine_active": (ctypes.c_int, [vp, ctypes.POINTER(Graph), vp, ctypes.c_int32, ctypes.c_double,
                                        ctypes.c_double, ctypes.POINTER(Options), ctypes.c_int32, ctypes.c_int32,
                                        ctypes.POINTER(PairResult), ctypes.POINTER(BatchResult),
                                        ctypes.POINTER(ctypes.c_int32)]),
    "fr_multitry": (ctypes.c_int, [vp, ctypes.POINTER(Graph), vp, ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                   i32p, i32p, ctypes.c_int32, ctypes.c_uint64, ctypes.POINTER(MtResult), i8p]),
    "fr_kway_global": (ctypes.c_int, [vp, ctypes.POINTER(Graph), vp, ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                      ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, ctypes.POINTER(MtResult)]),
    "fr_match": (ctypes.c_int, [vp, ctypes.POINTER(Graph), vp, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, vp,
                                ctypes.POINTER(ctypes.c_int32)]),
    "fr_contract": (ctypes.c_int, [vp, ctypes.POINTER(Graph), vp, vp, ctypes.POINTER(ctypes.c_int32),
                                   ctypes.POINTER(ctypes.c_int32), vp, vp, vp, vp]),
    "fr_vcycle": (ctypes.c_int, [vp, ctypes.POINTER(Graph), vp, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                 ctypes.POINTER(Options), ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(VcycleResult)]),
    "fr_cycle": (ctypes.c_int, [vp, ctypes.POINTER(Graph), vp, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                ctypes.POINTER(Options), ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                ctypes.POINTER(CycleResult)]),
    "fr_refine_batch_host": (ctypes.c_int, [vp, ctypes.c_int32, ctypes.c_int32, vp, vp, vp, vp, vp, ctypes.c_int32,
                                            ctypes.c_double, ctypes.c_double, ctypes.POINTER(Options),
                                            ctypes.c_int32, ctypes.POINTER(PairResult),
                                            ctypes.POINTER(BatchResult)]),
    "fr_rounds": (ctypes.c_int, [vp, ctypes.POINTER(Graph), vp, ctypes.c_int32, ctypes.c_int32, i32p, i32p, i32p,
                                 i32p, i32p]),
    "fr_autotune": (ctypes.c_int, [vp, ctypes.POINTER(Graph), vp, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                   ctypes.POINTER(Options), ctypes.c_int32, ctypes.POINTER(Options),
                                   ctypes.POINTER(ctypes.c_double)]),
    "fr_refine_pair_noalloc": (ctypes.c_int, [ctypes.POINTER(Graph), vp, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                              ctypes.POINTER(Options), ctypes.POINTER(PairResult), vp]),
    "fr_set_profiling": (ctypes.c_int, [vp, ctypes.c_int32]),
    "fr_struct_size": (ctypes.c_int32, [ctypes.c_int32]),
    "fr_profile_last": (ctypes.c_int, [vp, ctypes.POINTER(ProfileInfo)]),
    "fr_profile_rounds": (ctypes.c_int32, [vp, ctypes.POINTER(ctypes.c_float), ctypes.c_int32]),
    "fr_profile_pairs": (ctypes.c_int32, [vp, ctypes.POINTER(ctypes.c_float), ctypes.c_int32]),
    "fr_server_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.POINTER(ServerConfig)]),
    "fr_server_add_graph": (ctypes.c_int, [vp, ctypes.c_int32, ctypes.c_int32, vp, vp, vp, vp, i32p]),
    "fr_server_submit": (ctypes.c_int, [vp, ctypes.POINTER(Request)]),
    "fr_server_next": (ctypes.c_int, [vp, ctypes.POINTER(Response), i32p, ctypes.c_int32, ctypes.c_int32]),
    "fr_server_stats": (ctypes.c_int, [vp, i64p, i64p, i64p, i32p]),
    "fr_server_destroy": (ctypes.c_int, [vp]),
}

_LIB = None


def lib():
    """The loaded CUDA library; raises if it has not been built (no fallback)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(the CUDA path has no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SYMBOLS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        L.fr_last_launch_count.restype = ctypes.c_int64
        L.fr_last_launch_count.argtypes = [vp]
        _LIB = L
    return _LIB


class FlowRefError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{status}: {msg}")
        self.status = status


def default_options(**kw):
    o = Options()
    lib().fr_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _np32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


class DeviceGraph:
    """CSR graph held in torch int32 CUDA tensors (the caller-owned device arrays of fr_graph)."""

    def __init__(self, xadj, adjncy, adjwgt, vwgt, device="cuda"):
        import torch
        self.xadj = torch.as_tensor(_np32(xadj)).to(device)
        self.adjncy = torch.as_tensor(_np32(adjncy)).to(device)
        self.adjwgt = torch.as_tensor(_np32(adjwgt)).to(device)
        self.vwgt = torch.as_tensor(_np32(vwgt)).to(device)
        self.n = int(self.vwgt.numel())
        self.nnz = int(self.adjncy.numel())

    @classmethod
    def from_workload(cls, w, device="cuda"):
        return cls(w["xadj"], w["adjncy"], w["adjwgt"], w["vwgt"], device)

    def c(self):
        return Graph(self.n, self.nnz, self.xadj.data_ptr(), self.adjncy.data_ptr(), self.adjwgt.data_ptr(),
                     self.vwgt.data_ptr())


class Corridor:
    def __init__(self, ctx, handle):
        self.ctx = ctx
        self.h = handle

    @property
    def info(self):
        nc, m = ctypes.c_int32(), ctypes.c_int32()
        lib().fr_corridor_info(self.h, ctypes.byref(nc), ctypes.byref(m))
        return nc.value, m.value

    def export(self, with_dist=True):
        nc, m = self.info
        out = dict(gid=np.empty(nc, np.int32), off=np.empty(nc + 1, np.int32), head=np.empty(m, np.int32),
                   cap=np.empty(m, np.int32), border=np.empty(nc, np.int8), infcap=np.empty(nc, np.int32),
                   side0=np.empty(nc, np.int8), dist=np.empty(nc, np.int32))
        P = lambda a, t=i32p: a.ctypes.data_as(t)
        st = lib().fr_corridor_export(self.ctx.h, self.h, P(out["gid"]), P(out["off"]), P(out["head"]),
                                      P(out["cap"]), P(out["border"], i8p), P(out["infcap"]), P(out["side0"], i8p),
                                      P(out["dist"]) if with_dist else None)
        self.ctx._check(st)
        if not with_dist:
            out.pop("dist")
        return out

    def maxflow(self):
        f = ctypes.c_int64()
        self.ctx._check(lib().fr_maxflow(self.ctx.h, self.h, ctypes.byref(f)))
        return f.value

    def flow(self):
        nc, m = self.info
        af, sf = np.empty(m, np.int64), np.empty(nc, np.int64)
        self.ctx._check(lib().fr_corridor_flow(self.ctx.h, self.h, af.ctypes.data_as(i64p),
                                               sf.ctypes.data_as(i64p)))
        return af, sf

    def extract_cut(self, part, mb=0, reps=1, seed=0):
        res = PairResult()
        st = lib().fr_extract_cut(self.ctx.h, self.h, mb, reps, seed & 0xFFFFFFFFFFFFFFFF, _ptr(part),
                                  ctypes.byref(res))
        self.ctx._check(st)
        return res

    def sets(self):
        nc, _ = self.info
        ins, tot, comp, side = (np.empty(nc, np.int8), np.empty(nc, np.int8), np.empty(nc, np.int32),
                                np.empty(nc, np.int8))
        self.ctx._check(lib().fr_corridor_sets(self.ctx.h, self.h, ins.ctypes.data_as(i8p), tot.ctypes.data_as(i8p),
                                               comp.ctypes.data_as(i32p), side.ctypes.data_as(i8p)))
        return ins.astype(bool), tot.astype(bool), comp, side

    def free(self):
        if self.h:
            lib().fr_corridor_free(self.ctx.h, self.h)
            self.h = None


class Context:
    """One fr_ctx on a CUDA device (and a stream)."""

    def __init__(self, device=0, arena_bytes=0, stream=None):
        h = ctypes.c_void_p()
        st = lib().fr_create(ctypes.byref(h), device, arena_bytes, stream)
        if st != FR_OK:
            raise FlowRefError(st, "fr_create failed (no CUDA device?)")
        self.h = h

    def close(self):
        if self.h:
            lib().fr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def last_error(self):
        m = lib().fr_last_error(self.h)
        return m.decode() if m else ""

    def _check(self, st):
        if st != FR_OK:
            raise FlowRefError(st, self.last_error())

    @property
    def workspace_bytes(self):
        return lib().fr_workspace_bytes(self.h)

    @property
    def last_launches(self):
        return lib().fr_last_launch_count(self.h)

    def build_corridor(self, g: DeviceGraph, part, k, a, b, eps, alpha):
        h = ctypes.c_void_p()
        gc = g.c()
        st = lib().fr_build_corridor(self.h, ctypes.byref(gc), _ptr(part), k, a, b, eps, alpha, ctypes.byref(h))
        self._check(st)
        return Corridor(self, h)

    def refine_pair(self, g: DeviceGraph, part, k, a, b, eps, alpha, opts=None, check=True):
        res = PairResult()
        gc = g.c()
        o = opts if opts is not None else default_options()
        st = lib().fr_refine_pair(self.h, ctypes.byref(gc), _ptr(part), k, a, b, eps, alpha, ctypes.byref(o),
                                  ctypes.byref(res))
        if check:
            self._check(st)
        return st, res

    def refine_batch(self, g: DeviceGraph, part, k, eps, alpha, opts=None, check=True, results=True):
        cap = k * (k - 1) // 2 if results else 0
        res = (PairResult * max(cap, 1))()
        summ = BatchResult()
        gc = g.c()
        o = opts if opts is not None else default_options()
        st = lib().fr_refine_batch(self.h, ctypes.byref(gc), _ptr(part), k, eps, alpha, ctypes.byref(o), cap, res,
                                   ctypes.byref(summ))
        if check:
            self._check(st)
        pairs = [res[i].as_dict() for i in range(min(summ.npairs, cap))]
        return st, pairs, summ.as_dict()

    def refine_active(self, g: DeviceGraph, part, k, eps, alpha, opts=None, max_outer=16, cap=None, check=True):
        """Active block scheduling (fr_refine_active); returns (status, per-refinement
        results in processing order, summary, outer rounds run)."""
        cap = cap if cap is not None else max(1, max_outer * k * (k - 1) // 2)
        res = (PairResult * max(cap, 1))()
        summ = BatchResult()
        nouter = ctypes.c_int32()
        gc = g.c()
        o = opts if opts is not None else default_options()
        st = lib().fr_refine_active(self.h, ctypes.byref(gc), _ptr(part), k, eps, alpha, ctypes.byref(o), max_outer,
                                    cap, res, ctypes.byref(summ), ctypes.byref(nouter))
        if check:
            self._check(st)
        pairs = [res[i].as_dict() for i in range(min(summ.npairs, cap))]
        return st, pairs, summ.as_dict(), nouter.value

    def multitry(self, g: DeviceGraph, part, k, eps, pairs, alpha, seed=0, check=True):
        """One multi-try FM pass over block-disjoint pairs (fr_multitry); returns
        (status, totals, changed-block flags)."""
        pa = np.ascontiguousarray([p[0] for p in pairs], np.int32)
        pb = np.ascontiguousarray([p[1] for p in pairs], np.int32)
        out = MtResult()
        changed = np.zeros(k, np.int8)
        gc = g.c()
        st = lib().fr_multitry(self.h, ctypes.byref(gc), _ptr(part), k, eps, len(pairs), pa.ctypes.data_as(i32p),
                               pb.ctypes.data_as(i32p), alpha, seed & 0xFFFFFFFFFFFFFFFF, ctypes.byref(out),
                               changed.ctypes.data_as(i8p))
        if check:
            self._check(st)
        return st, out.as_dict(), changed.astype(bool)

    def kway_global(self, g: DeviceGraph, part, k, eps, init_mode=0, alpha=10, max_rounds=10, seed=0, check=True):
        """Global k-way refinement rounds (fr_kway_global); returns (status, totals
        with searches = rounds run)."""
        out = MtResult()
        gc = g.c()
        st = lib().fr_kway_global(self.h, ctypes.byref(gc), _ptr(part), k, eps, init_mode, alpha, max_rounds,
                                  seed & 0xFFFFFFFFFFFFFFFF, ctypes.byref(out))
        if check:
            self._check(st)
        return st, out.as_dict()

    def match(self, g: DeviceGraph, part, k, W, seed_l=0, check=True):
        """Greedy matching of one level (fr_match); returns (status, pairs, mate as a device tensor)."""
        import torch
        mate = torch.empty(g.n, dtype=torch.int32, device=part.device)
        pairs = ctypes.c_int32()
        gc = g.c()
        st = lib().fr_match(self.h, ctypes.byref(gc), _ptr(part), k, W, seed_l & 0xFFFFFFFFFFFFFFFF, _ptr(mate),
                            ctypes.byref(pairs))
        if check:
            self._check(st)
        return st, pairs.value, mate

    def contract(self, g: DeviceGraph, mate, check=True):
        """Contraction of a matching (fr_contract); returns (status, cmap, coarse arrays as numpy)."""
        import torch
        dev = mate.device
        cmap = torch.empty(g.n, dtype=torch.int32, device=dev)
        cx = torch.empty(g.n + 1, dtype=torch.int32, device=dev)
        ca = torch.empty(max(g.nnz, 1), dtype=torch.int32, device=dev)
        cw = torch.empty(max(g.nnz, 1), dtype=torch.int32, device=dev)
        cv = torch.empty(g.n, dtype=torch.int32, device=dev)
        cn, cnnz = ctypes.c_int32(), ctypes.c_int32()
        gc = g.c()
        st = lib().fr_contract(self.h, ctypes.byref(gc), _ptr(mate), _ptr(cmap), ctypes.byref(cn), ctypes.byref(cnnz),
                               _ptr(cx), _ptr(ca), _ptr(cw), _ptr(cv))
        if check:
            self._check(st)
        c, m = cn.value, cnnz.value
        return st, cmap.cpu().numpy(), dict(n=c, nnz=m, xadj=cx[:c + 1].cpu().numpy(), adjncy=ca[:m].cpu().numpy(),
                                            adjwgt=cw[:m].cpu().numpy(), vwgt=cv[:c].cpu().numpy())

    def vcycle(self, g: DeviceGraph, part, k, eps, alpha, opts=None, max_levels=64, active_outer=0, check=True):
        """One V-cycle with the given partition (fr_vcycle); returns (status, result dict)."""
        res = VcycleResult()
        gc = g.c()
        o = opts if opts is not None else default_options()
        st = lib().fr_vcycle(self.h, ctypes.byref(gc), _ptr(part), k, eps, alpha, ctypes.byref(o), max_levels,
                             active_outer, ctypes.byref(res))
        if check:
            self._check(st)
        return st, res.as_dict()

    def cycle(self, g: DeviceGraph, part, k, eps, alpha, kind="F", d=2, opts=None, max_levels=64, active_outer=0,
              check=True):
        """A global search cycle with the given partition (fr_cycle; kind V, W or F);
        returns (status, result dict)."""
        res = CycleResult()
        gc = g.c()
        o = opts if opts is not None else default_options()
        st = lib().fr_cycle(self.h, ctypes.byref(gc), _ptr(part), k, eps, alpha, ctypes.byref(o),
                            {"V": 0, "W": 1, "F": 2}[kind], d, max_levels, active_outer, ctypes.byref(res))
        if check:
            self._check(st)
        return st, res.as_dict()

    def refine_batch_host(self, xadj, adjncy, adjwgt, vwgt, part, k, eps, alpha, opts=None, cap=0):
        """Host-buffer form: arrays are numpy or (pinned) CPU tensors; part is updated in place."""
        def p(a):
            return ctypes.c_void_p(a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data)
        res = (PairResult * max(cap, 1))()
        summ = BatchResult()
        o = opts if opts is not None else default_options()
        n = len(vwgt)
        nnz = len(adjncy)
        st = lib().fr_refine_batch_host(self.h, n, nnz, p(xadj), p(adjncy), p(adjwgt), p(vwgt), p(part), k, eps,
                                        alpha, ctypes.byref(o), cap, res, ctypes.byref(summ))
        self._check(st)
        return summ.as_dict()

    def rounds(self, g: DeviceGraph, part, k):
        cap = k * (k - 1) // 2
        pa, pb, pr = np.empty(cap, np.int32), np.empty(cap, np.int32), np.empty(cap, np.int32)
        npairs, nrounds = ctypes.c_int32(), ctypes.c_int32()
        gc = g.c()
        st = lib().fr_rounds(self.h, ctypes.byref(gc), _ptr(part), k, cap, pa.ctypes.data_as(i32p),
                             pb.ctypes.data_as(i32p), pr.ctypes.data_as(i32p),
                             ctypes.byref(npairs), ctypes.byref(nrounds))
        self._check(st)
        return pa[:npairs.value], pb[:npairs.value], pr[:npairs.value], nrounds.value

    def set_profiling(self, on=True):
        self._check(lib().fr_set_profiling(self.h, 1 if on else 0))

    def profile(self):
        info = ProfileInfo()
        self._check(lib().fr_profile_last(self.h, ctypes.byref(info)))
        return info.as_dict()

    def profile_rounds(self):
        """Per round of the last profiled batch: [scan, step 1, cluster, step 2] in ms."""
        nr = lib().fr_profile_rounds(self.h, None, 0)
        buf = (ctypes.c_float * max(4 * nr, 1))()
        lib().fr_profile_rounds(self.h, buf, nr)
        return [[round(buf[4 * r + i], 4) for i in range(4)] for r in range(nr)]

    def profile_pairs(self):
        """Per pair of the last profiled batch: (round, cluster start ms, end ms) after
        the round's first start; -1 where no cluster solved the pair."""
        np_ = lib().fr_profile_pairs(self.h, None, 0)
        buf = (ctypes.c_float * max(3 * np_, 1))()
        lib().fr_profile_pairs(self.h, buf, np_)
        return [(int(buf[3 * i]), round(buf[3 * i + 1], 4), round(buf[3 * i + 2], 4)) for i in range(np_)]

    def autotune(self, g: DeviceGraph, part, k, eps, alpha, opts=None, trials=2):
        best = Options()
        ms = ctypes.c_double()
        gc = g.c()
        o = opts if opts is not None else default_options()
        st = lib().fr_autotune(self.h, ctypes.byref(gc), _ptr(part), k, eps, alpha, ctypes.byref(o), trials,
                               ctypes.byref(best), ctypes.byref(ms))
        self._check(st)
        return best, ms.value


class Server:
    """Continuous-batching refinement server (fr_server_*): graphs stay on the device,
    requests are admitted by free slots and arena bytes, each device step advances
    every in-flight request by one round."""

    def __init__(self, device=0, max_inflight=16, arena_bytes=0, opts=None):
        cfg = ServerConfig()
        cfg.device = device
        cfg.max_inflight = max_inflight
        cfg.arena_bytes = arena_bytes
        cfg.opt = opts if opts is not None else default_options()
        h = ctypes.c_void_p()
        st = lib().fr_server_create(ctypes.byref(h), ctypes.byref(cfg))
        if st != FR_OK:
            raise FlowRefError(st, "fr_server_create failed")
        self.h = h
        self.sizes = []

    def add_graph(self, xadj, adjncy, adjwgt, vwgt):
        xadj, adjncy, adjwgt, vwgt = (_np32(a) for a in (xadj, adjncy, adjwgt, vwgt))
        gid = ctypes.c_int32()
        st = lib().fr_server_add_graph(self.h, len(vwgt), len(adjncy), xadj.ctypes.data, adjncy.ctypes.data,
                                       adjwgt.ctypes.data, vwgt.ctypes.data, ctypes.byref(gid))
        if st != FR_OK:
            raise FlowRefError(st, "fr_server_add_graph failed")
        self.sizes.append(len(vwgt))
        return gid.value

    def submit(self, graph_id, part, k, eps, alpha, tag):
        part = _np32(part)
        req = Request(graph_id, k, eps, alpha, part.ctypes.data_as(i32p), tag)
        st = lib().fr_server_submit(self.h, ctypes.byref(req))
        if st != FR_OK:
            raise FlowRefError(st, "fr_server_submit failed")

    def next(self, n_max, timeout_ms=-1):
        resp = Response()
        out = np.empty(n_max, np.int32)
        st = lib().fr_server_next(self.h, ctypes.byref(resp), out.ctypes.data_as(i32p), n_max, timeout_ms)
        if st != FR_OK:
            raise FlowRefError(st, "fr_server_next: nothing completed in time")
        return resp.as_dict(), out

    def stats(self):
        s, a, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        m = ctypes.c_int32()
        lib().fr_server_stats(self.h, ctypes.byref(s), ctypes.byref(a), ctypes.byref(c), ctypes.byref(m))
        return dict(steps=s.value, admitted=a.value, completed=c.value, max_concurrent=m.value)

    def close(self):
        if self.h:
            lib().fr_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
