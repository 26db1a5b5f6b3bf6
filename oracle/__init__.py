"""ctypes view of the CPU oracle (liboracle.so).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py.  The product path never imports this package.
Every function mirrors one in fro.h; the docstrings there cite the paper.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None
i8p = ctypes.POINTER(ctypes.c_int8)
i32p = ctypes.POINTER(ctypes.c_int32)
i64p = ctypes.POINTER(ctypes.c_int64)


class Options(ctypes.Structure):
    _fields_ = [("mb", ctypes.c_int32), ("mb_reps", ctypes.c_int32), ("adaptive", ctypes.c_int32),
                ("max_iters", ctypes.c_int32), ("alpha_max", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("fm_permille", ctypes.c_int32), ("mt_alpha", ctypes.c_int32)]


class PairResult(ctypes.Structure):
    _fields_ = [("flow", ctypes.c_int64), ("cut_before", ctypes.c_int64), ("cut_after", ctypes.c_int64),
                ("wA_before", ctypes.c_int64), ("wB_before", ctypes.c_int64), ("wA_after", ctypes.c_int64),
                ("wB_after", ctypes.c_int64), ("corridor_n", ctypes.c_int32), ("corridor_arcs", ctypes.c_int32),
                ("accepted", ctypes.c_int32), ("iters", ctypes.c_int32), ("alpha_final", ctypes.c_double),
                ("status", ctypes.c_int32), ("a", ctypes.c_int32), ("b", ctypes.c_int32), ("round", ctypes.c_int32),
                ("cut_fm", ctypes.c_int64), ("fm_moves", ctypes.c_int32), ("pad0", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "pad0"}


class KwayResult(ctypes.Structure):
    _fields_ = [("gain", ctypes.c_int64), ("tried", ctypes.c_int32), ("kept", ctypes.c_int32),
                ("stop", ctypes.c_int32), ("pad0", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "pad0"}


class MTResult(ctypes.Structure):
    _fields_ = [("gain", ctypes.c_int64), ("searches", ctypes.c_int32), ("tried", ctypes.c_int32),
                ("kept", ctypes.c_int32), ("pad0", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "pad0"}


class VcycleResult(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("pad0", ctypes.c_int32), ("cut_before", ctypes.c_int64),
                ("cut_after", ctypes.c_int64), ("level_n", ctypes.c_int32 * 64), ("level_pairs", ctypes.c_int32 * 64),
                ("level_cut", ctypes.c_int64 * 64)]

    def as_dict(self):
        L = self.levels
        return dict(levels=L, cut_before=self.cut_before, cut_after=self.cut_after,
                    level_n=list(self.level_n[:L]), level_pairs=list(self.level_pairs[:L]),
                    level_cut=list(self.level_cut[:L]))


class CycleResult(ctypes.Structure):
    _fields_ = [("coarsenings", ctypes.c_int32), ("refinements", ctypes.c_int32), ("depth", ctypes.c_int32),
                ("pad0", ctypes.c_int32), ("cut_before", ctypes.c_int64), ("cut_after", ctypes.c_int64),
                ("level_coarsenings", ctypes.c_int32 * 64)]

    def as_dict(self):
        return dict(coarsenings=self.coarsenings, refinements=self.refinements, depth=self.depth,
                    cut_before=self.cut_before, cut_after=self.cut_after,
                    level_coarsenings=list(self.level_coarsenings[:max(self.depth, 1)]))


class FMResult(ctypes.Structure):
    _fields_ = [("cut_before", ctypes.c_int64), ("cut_after", ctypes.c_int64), ("wA_after", ctypes.c_int64),
                ("wB_after", ctypes.c_int64), ("tried", ctypes.c_int32), ("kept", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.fro_validate.restype = ctypes.c_int32
        L.fro_validate.argtypes = [ctypes.c_int32, i32p, i32p, i32p, i32p, i32p, ctypes.c_int32]
        for f in ("fro_total_weight", "fro_max_weight"):
            getattr(L, f).restype = ctypes.c_int64
            getattr(L, f).argtypes = [ctypes.c_int32, i32p]
        L.fro_lmax.restype = ctypes.c_int64
        L.fro_lmax.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.c_double]
        L.fro_budget_base.restype = ctypes.c_int64
        L.fro_budget_base.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_double]
        L.fro_pair_cut.restype = ctypes.c_int64
        L.fro_pair_cut.argtypes = [ctypes.c_int32, i32p, i32p, i32p, i32p, ctypes.c_int32, ctypes.c_int32]
        L.fro_build.restype = ctypes.c_void_p
        L.fro_build.argtypes = [ctypes.c_int32, i32p, i32p, i32p, i32p, i32p, ctypes.c_int32, ctypes.c_int32,
                                ctypes.c_int64]
        L.fro_from_network.restype = ctypes.c_void_p
        L.fro_from_network.argtypes = [ctypes.c_int32, i32p, i32p, i32p, i8p, i32p, i32p, i8p, ctypes.c_int64,
                                       ctypes.c_int64]
        L.fro_free.argtypes = [ctypes.c_void_p]
        L.fro_nc.restype = ctypes.c_int32
        L.fro_nc.argtypes = [ctypes.c_void_p]
        L.fro_m.restype = ctypes.c_int32
        L.fro_m.argtypes = [ctypes.c_void_p]
        L.fro_export.argtypes = [ctypes.c_void_p, i32p, i32p, i32p, i32p, i8p, i32p, i8p, i32p]
        L.fro_maxflow.restype = ctypes.c_int64
        L.fro_maxflow.argtypes = [ctypes.c_void_p, ctypes.c_int32]
        L.fro_flow.argtypes = [ctypes.c_void_p, i64p, i64p]
        L.fro_residual_sets.argtypes = [ctypes.c_void_p, i8p, i8p, i32p]
        L.fro_sweep.restype = ctypes.c_int32
        L.fro_sweep.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64, i32p, i64p]
        L.fro_cut.restype = ctypes.c_int64
        L.fro_cut.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, i8p, i32p, i32p]
        L.fro_refine_pair.restype = ctypes.c_int32
        L.fro_refine_pair.argtypes = [ctypes.c_int32, i32p, i32p, i32p, i32p, i32p, ctypes.c_int32,
                                      ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                      ctypes.POINTER(Options), ctypes.POINTER(PairResult)]
        L.fro_rounds.restype = ctypes.c_int32
        L.fro_rounds.argtypes = [ctypes.c_int32, i32p, i32p, i32p, ctypes.c_int32, ctypes.c_int32, i32p, i32p,
                                 i32p, i32p]
        L.fro_refine_batch.restype = ctypes.c_int32
        L.fro_refine_batch.argtypes = [ctypes.c_int32, i32p, i32p, i32p, i32p, i32p, ctypes.c_int32,
                                       ctypes.c_double, ctypes.c_double, ctypes.POINTER(Options), ctypes.c_int32,
                                       ctypes.POINTER(PairResult), i32p, i32p]
        L.fro_refine_batch_sample.restype = ctypes.c_int32
        L.fro_refine_batch_sample.argtypes = [ctypes.c_int32, i32p, i32p, i32p, i32p, i32p, ctypes.c_int32,
                                              ctypes.c_double, ctypes.c_double, ctypes.POINTER(Options),
                                              ctypes.c_int32, i32p]
        L.fro_refine_batch_mt.restype = ctypes.c_int32
        L.fro_refine_batch_mt.argtypes = [ctypes.c_int32, i32p, i32p, i32p, i32p, i32p, ctypes.c_int32,
                                          ctypes.c_double, ctypes.c_double, ctypes.POINTER(Options), ctypes.c_int32,
                                          ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(PairResult), i32p, i32p,
                                          i32p]
        L.fro_refine_active.restype = ctypes.c_int32
        L.fro_refine_active.argtypes = [ctypes.c_int32, i32p, i32p, i32p, i32p, i32p, ctypes.c_int32,
                                        ctypes.c_double, ctypes.c_double, ctypes.POINTER(Options), ctypes.c_int32,
                                        ctypes.c_int32, ctypes.POINTER(PairResult), i32p, i32p,
                                        ctypes.POINTER(MTResult)]
        L.fro_kaspar_stop.restype = ctypes.c_int32
        L.fro_kaspar_stop.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.c_double]
        L.fro_kway_search.restype = ctypes.c_int32
        L.fro_kway_search.argtypes = [ctypes.c_int32, i32p, i32p, i32p, i32p, i32p, ctypes.c_int32, i64p,
                                      ctypes.c_int64, i32p, ctypes.c_int32, i32p, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_double, ctypes.c_uint64, ctypes.POINTER(KwayResult), i32p, i32p, i64p,
                                      ctypes.c_int32]
        L.fro_multitry.restype = ctypes.c_int32
        L.fro_multitry.argtypes = [ctypes.c_int32, i32p, i32p, i32p, i32p, i32p, ctypes.c_int32, ctypes.c_int64,
                                   ctypes.c_int32, i32p, i32p, ctypes.c_int32, ctypes.c_uint64,
                                   ctypes.POINTER(MTResult), i8p]
        L.fro_mt_seed.restype = ctypes.c_uint64
        L.fro_mt_seed.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32]
        L.fro_kway_global.restype = ctypes.c_int32
        L.fro_kway_global.argtypes = [ctypes.c_int32, i32p, i32p, i32p, i32p, i32p, ctypes.c_int32, ctypes.c_double,
                                      ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                                      ctypes.POINTER(KwayResult), i32p]
        L.fro_match.restype = ctypes.c_int32
        L.fro_match.argtypes = [ctypes.c_int32, i32p, i32p, i32p, i32p, i32p, ctypes.c_int32, ctypes.c_int64,
                                ctypes.c_uint64, i32p]
        L.fro_contract.restype = ctypes.c_int32
        L.fro_contract.argtypes = [ctypes.c_int32, i32p, i32p, i32p, i32p, i32p, i32p, i32p, i32p, i32p, i32p, i32p]
        L.fro_vcycle.restype = ctypes.c_int32
        L.fro_vcycle.argtypes = [ctypes.c_int32, i32p, i32p, i32p, i32p, i32p, ctypes.c_int32, ctypes.c_double,
                                 ctypes.c_double, ctypes.POINTER(Options), ctypes.c_int32, ctypes.c_int32,
                                 ctypes.POINTER(VcycleResult)]
        L.fro_cycle.restype = ctypes.c_int32
        L.fro_cycle.argtypes = [ctypes.c_int32, i32p, i32p, i32p, i32p, i32p, ctypes.c_int32, ctypes.c_double,
                                ctypes.c_double, ctypes.POINTER(Options), ctypes.c_int32, ctypes.c_int32,
                                ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(CycleResult)]
        L.fro_fm_pair.restype = ctypes.c_int32
        L.fro_fm_pair.argtypes = [ctypes.c_int32, i32p, i32p, i32p, i32p, i32p, ctypes.c_int32, ctypes.c_int32,
                                  ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.POINTER(FMResult), i32p,
                                  ctypes.c_int32]
        L.fro_fm_seed.restype = ctypes.c_uint64
        L.fro_fm_seed.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32]
        L.fro_splitmix64.restype = ctypes.c_uint64
        L.fro_splitmix64.argtypes = [ctypes.c_uint64]
        _LIB = L
    return _LIB


def _p(a, t=i32p):
    return a.ctypes.data_as(t)


def _c32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def options(mb=0, mb_reps=1, adaptive=0, max_iters=1, alpha_max=1.0, seed=0, fm_permille=0, mt_alpha=0):
    return Options(mb, mb_reps, adaptive, max_iters, alpha_max, seed, fm_permille, mt_alpha)


def validate(w):
    return lib().fro_validate(w["n"], _p(w["xadj"]), _p(w["adjncy"]), _p(w["adjwgt"]), _p(w["vwgt"]),
                              _p(w["part"]), w["k"])


def total_weight(vwgt):
    return lib().fro_total_weight(len(vwgt), _p(_c32(vwgt)))


def lmax(W, maxc, k, eps):
    return lib().fro_lmax(W, maxc, k, eps)


def budget_base(W, k, eps, alpha):
    return lib().fro_budget_base(W, k, eps, alpha)


def pair_cut(w, part, a, b):
    return lib().fro_pair_cut(w["n"], _p(w["xadj"]), _p(w["adjncy"]), _p(w["adjwgt"]), _p(_c32(part)), a, b)


def splitmix64(x):
    return lib().fro_splitmix64(x & 0xFFFFFFFFFFFFFFFF)


class Problem:
    """One corridor flow problem (corridor, network, max flow, residual structure)."""

    def __init__(self, handle):
        self.h = handle

    def __del__(self):
        if getattr(self, "h", None):
            lib().fro_free(self.h)
            self.h = None

    @classmethod
    def build(cls, w, a, b, Ubase, part=None):
        part = _c32(w["part"] if part is None else part)
        return cls(lib().fro_build(w["n"], _p(w["xadj"]), _p(w["adjncy"]), _p(w["adjwgt"]), _p(w["vwgt"]),
                                   _p(part), a, b, Ubase))

    @classmethod
    def from_network(cls, off, head, cap, border, infcap, vw, side0, cA, cB):
        off, head, cap, infcap, vw = map(_c32, (off, head, cap, infcap, vw))
        border = np.ascontiguousarray(border, np.int8)
        side0 = np.ascontiguousarray(side0, np.int8)
        return cls(lib().fro_from_network(len(off) - 1, _p(off), _p(head), _p(cap), _p(border, i8p), _p(infcap),
                                          _p(vw), _p(side0, i8p), cA, cB))

    @property
    def nc(self):
        return lib().fro_nc(self.h)

    @property
    def m(self):
        return lib().fro_m(self.h)

    def export(self):
        nc, m = self.nc, self.m
        out = dict(gid=np.empty(nc, np.int32), off=np.empty(nc + 1, np.int32), head=np.empty(m, np.int32),
                   cap=np.empty(m, np.int32), border=np.empty(nc, np.int8), infcap=np.empty(nc, np.int32),
                   side0=np.empty(nc, np.int8), dist=np.empty(nc, np.int32))
        lib().fro_export(self.h, _p(out["gid"]), _p(out["off"]), _p(out["head"]), _p(out["cap"]),
                         _p(out["border"], i8p), _p(out["infcap"]), _p(out["side0"], i8p), _p(out["dist"]))
        return out

    def maxflow(self, method=0):
        return lib().fro_maxflow(self.h, method)

    def flow(self):
        af = np.empty(self.m, np.int64)
        sf = np.empty(self.nc, np.int64)
        lib().fro_flow(self.h, _p(af, i64p), _p(sf, i64p))
        return af, sf

    def residual_sets(self):
        nc = self.nc
        in_s, to_t, comp = np.empty(nc, np.int8), np.empty(nc, np.int8), np.empty(nc, np.int32)
        lib().fro_residual_sets(self.h, _p(in_s, i8p), _p(to_t, i8p), _p(comp))
        return in_s.astype(bool), to_t.astype(bool), comp

    def sweep(self, r=0, seed=0):
        nc = self.nc
        order = np.empty(nc + 1, np.int32)
        d = np.empty(nc + 2, np.int64)
        c = lib().fro_sweep(self.h, r, seed & 0xFFFFFFFFFFFFFFFF, _p(order), _p(d, i64p))
        return order[:max(c, 0)], d[:max(c, 0) + 1]

    def cut(self, mb=0, reps=1, seed=0):
        side = np.empty(self.nc, np.int8)
        bj, br = ctypes.c_int32(), ctypes.c_int32()
        capv = lib().fro_cut(self.h, mb, reps, seed & 0xFFFFFFFFFFFFFFFF, _p(side, i8p), ctypes.byref(bj),
                             ctypes.byref(br))
        return capv, side, bj.value, br.value


def refine_pair(w, a=0, b=1, part=None, eps=None, alpha=None, opts=None):
    part = np.array(w["part"] if part is None else part, np.int32, copy=True)
    eps = w["eps"] if eps is None else eps
    alpha = w["alpha"] if alpha is None else alpha
    if opts is None:
        opts = options(mb=w.get("mb", 0), adaptive=w.get("adaptive", 0), max_iters=w.get("max_iters", 1),
                       alpha_max=w.get("alpha_max", alpha))
    res = PairResult()
    st = lib().fro_refine_pair(w["n"], _p(w["xadj"]), _p(w["adjncy"]), _p(w["adjwgt"]), _p(w["vwgt"]), _p(part),
                               w["k"], a, b, eps, alpha, ctypes.byref(opts), ctypes.byref(res))
    return st, part, res


def rounds(w, part=None):
    part = _c32(w["part"] if part is None else part)
    k = w["k"]
    cap = k * (k - 1) // 2
    pa, pb, pr = np.empty(cap, np.int32), np.empty(cap, np.int32), np.empty(cap, np.int32)
    nr = ctypes.c_int32()
    np_ = lib().fro_rounds(w["n"], _p(w["xadj"]), _p(w["adjncy"]), _p(part), k, cap, _p(pa), _p(pb), _p(pr),
                           ctypes.byref(nr))
    return pa[:np_], pb[:np_], pr[:np_], nr.value


def refine_batch(w, part=None, eps=None, alpha=None, opts=None):
    part = np.array(w["part"] if part is None else part, np.int32, copy=True)
    eps = w["eps"] if eps is None else eps
    alpha = w["alpha"] if alpha is None else alpha
    if opts is None:
        opts = options(mb=w.get("mb", 0), adaptive=w.get("adaptive", 0), max_iters=w.get("max_iters", 1),
                       alpha_max=w.get("alpha_max", alpha))
    k = w["k"]
    cap = k * (k - 1) // 2
    res = (PairResult * max(cap, 1))()
    npairs, nrounds = ctypes.c_int32(), ctypes.c_int32()
    st = lib().fro_refine_batch(w["n"], _p(w["xadj"]), _p(w["adjncy"]), _p(w["adjwgt"]), _p(w["vwgt"]), _p(part),
                                k, eps, alpha, ctypes.byref(opts), cap, res, ctypes.byref(npairs),
                                ctypes.byref(nrounds))
    return st, part, [res[i].as_dict() for i in range(npairs.value)], nrounds.value


def refine_active(w, part=None, eps=None, alpha=None, opts=None, max_outer=16, cap=None, mt_out=None):
    """Active block scheduling with flow refinement (fro_refine_active); returns
    (status, part, per-refinement results in processing order, outer rounds run).
    mt_out (a dict, optional) receives the totals of the multi-try passes."""
    part = np.array(w["part"] if part is None else part, np.int32, copy=True)
    eps = w["eps"] if eps is None else eps
    alpha = w["alpha"] if alpha is None else alpha
    if opts is None:
        opts = options(mb=w.get("mb", 0))
    k = w["k"]
    cap = cap if cap is not None else max(1, max_outer * k * (k - 1) // 2)
    res = (PairResult * cap)()
    npairs, nouter = ctypes.c_int32(), ctypes.c_int32()
    mt = MTResult()
    st = lib().fro_refine_active(w["n"], _p(w["xadj"]), _p(w["adjncy"]), _p(w["adjwgt"]), _p(w["vwgt"]), _p(part),
                                 k, eps, alpha, ctypes.byref(opts), max_outer, cap, res,
                                 ctypes.byref(npairs), ctypes.byref(nouter), ctypes.byref(mt))
    if mt_out is not None:
        mt_out.update(mt.as_dict())
    return st, part, [res[i].as_dict() for i in range(min(npairs.value, cap))], nouter.value


def refine_batch_sample(w, max_pairs, part=None, opts=None):
    """The oracle's sweep stopped after max_pairs pairs; returns (status, part, pairs done)."""
    part = np.array(w["part"] if part is None else part, np.int32, copy=True)
    if opts is None:
        opts = options(mb=w.get("mb", 0))
    done = ctypes.c_int32()
    st = lib().fro_refine_batch_sample(w["n"], _p(w["xadj"]), _p(w["adjncy"]), _p(w["adjwgt"]), _p(w["vwgt"]),
                                       _p(part), w["k"], w["eps"], w["alpha"], ctypes.byref(opts), max_pairs,
                                       ctypes.byref(done))
    return st, part, done.value


def refine_batch_mt(w, nthreads, max_rounds=-1, part=None, eps=None, alpha=None, opts=None):
    """The sweep with the pairs of each round on up to nthreads threads
    (fro_refine_batch_mt); returns (status, part, results, rounds, pairs done)."""
    part = np.array(w["part"] if part is None else part, np.int32, copy=True)
    eps = w["eps"] if eps is None else eps
    alpha = w["alpha"] if alpha is None else alpha
    if opts is None:
        opts = options(mb=w.get("mb", 0), adaptive=w.get("adaptive", 0), max_iters=w.get("max_iters", 1),
                       alpha_max=w.get("alpha_max", alpha))
    k = w["k"]
    cap = max(1, k * (k - 1) // 2)
    res = (PairResult * cap)()
    npairs, nrounds, done = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    st = lib().fro_refine_batch_mt(w["n"], _p(w["xadj"]), _p(w["adjncy"]), _p(w["adjwgt"]), _p(w["vwgt"]),
                                   _p(part), k, eps, alpha, ctypes.byref(opts), nthreads, max_rounds, cap, res,
                                   ctypes.byref(npairs), ctypes.byref(nrounds), ctypes.byref(done))
    return st, part, [res[i].as_dict() for i in range(min(done.value, cap))], nrounds.value, done.value


def fm_seed(seed, a, b):
    return lib().fro_fm_seed(seed & 0xFFFFFFFFFFFFFFFF, a, b)


def fm_pair(w, a, b, permille, seed=0, part=None, Lmax=None):
    """Two-way FM with TopGain on pair (a, b) (fro_fm_pair); returns (status, part,
    result dict, vertices moved in order before the rollback)."""
    part = np.array(w["part"] if part is None else part, np.int32, copy=True)
    if Lmax is None:
        W = int(np.asarray(w["vwgt"], np.int64).sum())
        Lmax = lmax(W, int(np.asarray(w["vwgt"]).max()), w["k"], w["eps"])
    res = FMResult()
    moves = np.zeros(w["n"], np.int32)
    st = lib().fro_fm_pair(w["n"], _p(w["xadj"]), _p(w["adjncy"]), _p(w["adjwgt"]), _p(w["vwgt"]), _p(part),
                           a, b, Lmax, permille, seed & 0xFFFFFFFFFFFFFFFF, ctypes.byref(res), _p(moves), w["n"])
    d = res.as_dict()
    return st, part, d, moves[:d["tried"]]


def kaspar_stop(p, S1, S2, alpha, beta):
    """KaSPar stopping rule of the k-way search (fro_kaspar_stop)."""
    return lib().fro_kaspar_stop(p, S1, S2, alpha, beta)


def mt_seed(seed, a, b):
    return lib().fro_mt_seed(seed & 0xFFFFFFFFFFFFFFFF, a, b)


def kway_search(w, init, alpha, beta=None, tseed=0, part=None, blockw=None, Lmax=None, touched=None, sid=1):
    """One k-way local search (fro_kway_search) from the start set init; returns
    (status, part, blockw, result dict, log) with log = (vertices, targets, gains)
    of every move made, in order, before the rollback."""
    part = np.array(w["part"] if part is None else part, np.int32, copy=True)
    k = w["k"]
    if blockw is None:
        blockw = np.bincount(part, weights=np.asarray(w["vwgt"], np.int64), minlength=k).astype(np.int64)
    blockw = np.array(blockw, np.int64, copy=True)
    if Lmax is None:
        W = int(np.asarray(w["vwgt"], np.int64).sum())
        Lmax = lmax(W, int(np.asarray(w["vwgt"]).max()), k, w["eps"])
    if beta is None:
        beta = float(np.log(w["n"]))
    init = _c32(init)
    n = w["n"]
    lv, lt, lg = np.zeros(n, np.int32), np.zeros(n, np.int32), np.zeros(n, np.int64)
    res = KwayResult()
    tp = _p(touched) if touched is not None else None
    st = lib().fro_kway_search(n, _p(w["xadj"]), _p(w["adjncy"]), _p(w["adjwgt"]), _p(w["vwgt"]), _p(part), k,
                               _p(blockw, i64p), Lmax, _p(init), len(init), tp, sid, alpha, beta,
                               tseed & 0xFFFFFFFFFFFFFFFF, ctypes.byref(res), _p(lv), _p(lt), _p(lg, i64p), n)
    d = res.as_dict()
    t = d["tried"]
    return st, part, blockw, d, (lv[:t], lt[:t], lg[:t])


def multitry(w, pairs, alpha, seed=0, part=None, Lmax=None):
    """One multi-try FM pass over the pairs of a matching (fro_multitry); returns
    (status, part, totals dict, changed-block flags)."""
    part = np.array(w["part"] if part is None else part, np.int32, copy=True)
    k = w["k"]
    if Lmax is None:
        W = int(np.asarray(w["vwgt"], np.int64).sum())
        Lmax = lmax(W, int(np.asarray(w["vwgt"]).max()), k, w["eps"])
    pa = _c32([p[0] for p in pairs])
    pb = _c32([p[1] for p in pairs])
    res = MTResult()
    changed = np.zeros(k, np.int8)
    st = lib().fro_multitry(w["n"], _p(w["xadj"]), _p(w["adjncy"]), _p(w["adjwgt"]), _p(w["vwgt"]), _p(part), k,
                            Lmax, len(pairs), _p(pa), _p(pb), alpha, seed & 0xFFFFFFFFFFFFFFFF, ctypes.byref(res),
                            _p(changed, i8p))
    return st, part, res.as_dict(), changed.astype(bool)


def kway_global(w, alpha=10, init_mode=0, max_rounds=10, seed=0, part=None, eps=None):
    """Global k-way refinement rounds (fro_kway_global); returns (status, part, totals, rounds)."""
    part = np.array(w["part"] if part is None else part, np.int32, copy=True)
    eps = w["eps"] if eps is None else eps
    res = KwayResult()
    nr = ctypes.c_int32()
    st = lib().fro_kway_global(w["n"], _p(w["xadj"]), _p(w["adjncy"]), _p(w["adjwgt"]), _p(w["vwgt"]), _p(part),
                               w["k"], eps, init_mode, alpha, max_rounds, seed & 0xFFFFFFFFFFFFFFFF,
                               ctypes.byref(res), ctypes.byref(nr))
    return st, part, res.as_dict(), nr.value


def match(w, seed_l=0, part=None, W=None):
    """Greedy matching of one level (fro_match); returns (pairs, mate)."""
    part = _c32(w["part"] if part is None else part)
    if W is None:
        W = int(np.asarray(w["vwgt"], np.int64).sum())
    mate = np.empty(w["n"], np.int32)
    pairs = lib().fro_match(w["n"], _p(w["xadj"]), _p(w["adjncy"]), _p(w["adjwgt"]), _p(w["vwgt"]), _p(part),
                            w["k"], W, seed_l & 0xFFFFFFFFFFFFFFFF, _p(mate))
    return pairs, mate


def contract(w, mate):
    """Contraction of a matching (fro_contract); returns (cmap, coarse workload arrays)."""
    n, nnz = w["n"], len(w["adjncy"])
    cmap = np.empty(n, np.int32)
    cx, ca, cw, cv = (np.empty(n + 1, np.int32), np.empty(max(nnz, 1), np.int32), np.empty(max(nnz, 1), np.int32),
                      np.empty(n, np.int32))
    cn = ctypes.c_int32()
    cnnz = lib().fro_contract(n, _p(w["xadj"]), _p(w["adjncy"]), _p(w["adjwgt"]), _p(w["vwgt"]), _p(_c32(mate)),
                              _p(cmap), ctypes.byref(cn), _p(cx), _p(ca), _p(cw), _p(cv))
    c = cn.value
    return cmap, dict(n=c, nnz=cnnz, xadj=cx[:c + 1].copy(), adjncy=ca[:cnnz].copy(), adjwgt=cw[:cnnz].copy(),
                      vwgt=cv[:c].copy())


def vcycle(w, opts=None, max_levels=64, active_outer=0, part=None, eps=None, alpha=None):
    """One V-cycle with the given partition (fro_vcycle); returns (status, part, result dict)."""
    part = np.array(w["part"] if part is None else part, np.int32, copy=True)
    eps = w["eps"] if eps is None else eps
    alpha = w["alpha"] if alpha is None else alpha
    if opts is None:
        opts = options(mb=w.get("mb", 0))
    res = VcycleResult()
    st = lib().fro_vcycle(w["n"], _p(w["xadj"]), _p(w["adjncy"]), _p(w["adjwgt"]), _p(w["vwgt"]), _p(part), w["k"],
                          eps, alpha, ctypes.byref(opts), max_levels, active_outer, ctypes.byref(res))
    return st, part, res.as_dict()


CYCLES = {"V": 0, "W": 1, "F": 2}


def cycle(w, kind="F", d=2, opts=None, max_levels=64, active_outer=0, part=None, eps=None, alpha=None):
    """A global search cycle with the given partition (fro_cycle); returns (status, part, result dict)."""
    part = np.array(w["part"] if part is None else part, np.int32, copy=True)
    eps = w["eps"] if eps is None else eps
    alpha = w["alpha"] if alpha is None else alpha
    if opts is None:
        opts = options(mb=w.get("mb", 0))
    res = CycleResult()
    st = lib().fro_cycle(w["n"], _p(w["xadj"]), _p(w["adjncy"]), _p(w["adjwgt"]), _p(w["vwgt"]), _p(part), w["k"],
                         eps, alpha, ctypes.byref(opts), CYCLES[kind], d, max_levels, active_outer, ctypes.byref(res))
    return st, part, res.as_dict()
