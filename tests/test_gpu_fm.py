"""Two-way FM with TopGain before each pair's flow (fm_permille > 0) on the CUDA
path against the oracle: the same partition and the same per-pair results
(cut before FM, cut after FM, moves kept, flow results) for the batched sweep,
the single-pair call and active block scheduling; all integers, so bit-exact."""
import numpy as np
import pytest

import oracle as O
from paper_1012_0006_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FIELDS = ("a", "b", "round", "flow", "cut_before", "cut_fm", "fm_moves", "cut_after", "wA_before", "wB_before",
          "wA_after", "wB_after", "corridor_n", "corridor_arcs", "accepted", "iters")


@pytest.fixture(scope="module")
def F(gpu_lib):
    return gpu_lib


@pytest.fixture(scope="module")
def ctx(F):
    c = F.Context(0)
    yield c
    c.close()


def _dev(F, w):
    import torch
    return F.DeviceGraph.from_workload(w), torch.as_tensor(np.array(w["part"], np.int32)).cuda()


def _batch(F, ctx, w, okw, alpha=None):
    alpha = w["alpha"] if alpha is None else alpha
    st, pref, rref, nr = O.refine_batch(w, alpha=alpha, opts=O.options(**okw))
    assert st == 0
    g, part = _dev(F, w)
    st, res, summ = ctx.refine_batch(g, part, w["k"], w["eps"], alpha, F.default_options(**okw))
    assert summ["npairs"] == len(rref) and summ["nrounds"] == nr
    for rg, rc in zip(res, rref):
        for f in FIELDS:
            assert rg[f] == rc[f], (f, rg["a"], rg["b"], rg["round"])
    assert np.array_equal(part.cpu().numpy(), pref)
    assert summ["cut_after"] == summ["cut_before"] + sum(r["cut_after"] - r["cut_before"] for r in rref)
    return rref


@pytest.mark.parametrize("seed", range(16))
def test_batch_fm_random_small(F, ctx, seed):
    w = I.random_small(6000 + seed, n_max=2500, k_max=8)
    rref = _batch(F, ctx, w, dict(mb=seed % 2, mb_reps=1 + seed % 3, seed=seed, fm_permille=(10, 50, 300)[seed % 3]))
    assert len(rref) > 0


@pytest.mark.parametrize("cfg,scale,pm", [(1, 1.0, 50), (2, 1 / 16, 50), (3, 1 / 64, 10), (3, 1 / 8, 50),
                                          (4, 1 / 64, 50), (4, 1 / 16, 10)])
def test_batch_fm_workloads(F, ctx, cfg, scale, pm):
    w = I.config(cfg, scale=scale)
    rref = _batch(F, ctx, w, dict(mb=int(w.get("mb", 0)), fm_permille=pm))
    assert any(r["fm_moves"] > 0 for r in rref)


def test_batch_fm_boundary_sorted_in_global_memory(F, ctx):
    """A pair whose boundary exceeds what one CTA sorts in shared memory (4096
    entries): 32 x 160 x 160 grid split in two across a 32 x 160 face per side."""
    w = I.grid3d_rcb(32, 160, 160, k=2, alpha=1.0)
    rref = _batch(F, ctx, w, dict(mb=1, fm_permille=10))
    assert rref[0]["cut_fm"] < rref[0]["cut_before"]


@pytest.mark.parametrize("seed", range(6))
def test_pair_fm_adaptive(F, ctx, seed):
    w = I.random_small(6100 + seed, n_max=2000, k_max=4)
    pa, pb, _, _ = O.rounds(w)
    a, b = int(pa[0]), int(pb[0])
    okw = dict(mb=1, adaptive=seed % 2, max_iters=6, alpha_max=8.0, seed=seed, fm_permille=50)
    st, pref, rref = O.refine_pair(w, a, b, alpha=1.0, opts=O.options(**okw))
    rref = rref.as_dict()
    g, part = _dev(F, w)
    st, res = ctx.refine_pair(g, part, w["k"], a, b, w["eps"], 1.0, F.default_options(**okw))
    rg = res.as_dict()
    for f in FIELDS:
        if f in ("round",):
            continue
        assert rg[f] == rref[f], f
    assert np.array_equal(part.cpu().numpy(), pref)


@pytest.mark.parametrize("okw", [dict(mb=1, fm_permille=50),
                                 dict(mb=1, adaptive=1, max_iters=6, alpha_max=8.0, fm_permille=10)])
def test_active_fm(F, ctx, okw):
    import torch
    for w in (I.config(2, scale=1 / 16), I.random_small(6200, n_max=2500, k_max=6)):
        st, pref, rref, nref = O.refine_active(w, alpha=1.0, opts=O.options(**okw), max_outer=12)
        assert st == 0
        g = F.DeviceGraph.from_workload(w)
        part = torch.as_tensor(np.array(w["part"], np.int32)).cuda()
        st, res, summ, nouter = ctx.refine_active(g, part, w["k"], w["eps"], 1.0, F.default_options(**okw),
                                                  max_outer=12)
        assert nouter == nref and len(res) == len(rref)
        for rg, rc in zip(res, rref):
            for f in FIELDS:
                assert rg[f] == rc[f], (f, rg["a"], rg["b"], rg["round"])
        assert np.array_equal(part.cpu().numpy(), pref)


def test_fm_gain_range_is_checked(F, ctx):
    """Weighted degrees above 1023 do not fit the gain buckets: FR_ERR_TOO_LARGE, part untouched."""
    w = I.random_small(6300, n_max=400, k_max=3)
    w = dict(w, adjwgt=np.full(len(w["adjncy"]), 2000, np.int32))
    g, part = _dev(F, w)
    before = part.clone()
    st, _, _ = ctx.refine_batch(g, part, w["k"], w["eps"], w["alpha"], F.default_options(fm_permille=50),
                                check=False)
    assert st == F.FR_ERR_TOO_LARGE
    assert (part == before).all()


def test_fm_option_rejected_where_unsupported(F, ctx):
    import ctypes
    w = I.random_small(6301, n_max=200, k_max=3)
    g, part = _dev(F, w)
    st, _ = ctx.refine_pair(g, part, w["k"], 0, 1, w["eps"], w["alpha"], F.default_options(fm_permille=1001),
                            check=False)
    assert st == F.FR_ERR_INVALID_ARG
    cfg = F.ServerConfig()
    cfg.device, cfg.max_inflight, cfg.arena_bytes = 0, 2, 1 << 26
    F.lib().fr_default_options(ctypes.byref(cfg.opt))
    cfg.opt.fm_permille = 50
    srv = ctypes.c_void_p()
    assert F.lib().fr_server_create(ctypes.byref(srv), ctypes.byref(cfg)) == F.FR_ERR_INVALID_ARG


def test_batch_fm_full_rgg3d_bench_configuration(F, ctx):
    """The full 4,194,304-vertex 3D rgg (k = 64, the bench workload) with the FM step at
    the 1 % stopping rule, against the oracle's sweep run pair-parallel on the host cores
    (identical to the sequential sweep, pinned on CPU)."""
    import os
    w = I.config(4)
    okw = dict(mb=1, fm_permille=10)
    st, pref, rref, nr, done = O.refine_batch_mt(w, len(os.sched_getaffinity(0)), opts=O.options(**okw))
    assert st == 0 and done == len(rref)
    g, part = _dev(F, w)
    st, res, summ = ctx.refine_batch(g, part, w["k"], w["eps"], w["alpha"], F.default_options(**okw))
    assert summ["npairs"] == len(rref) and summ["nrounds"] == nr
    for rg, rc in zip(res, rref):
        for f in FIELDS:
            assert rg[f] == rc[f], (f, rg["a"], rg["b"], rg["round"])
    assert np.array_equal(part.cpu().numpy(), pref)
