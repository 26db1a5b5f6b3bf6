"""Multi-try FM (k-way searches with the KaSPar stopping rule) on the CUDA path
against the oracle: one pass over a matching's pairs (fr_multitry) and active block
scheduling with a pass after every matching (mt_alpha > 0).  Partitions, totals and
changed-block flags are integers: bit-exact."""
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


def _pass(F, ctx, w, pairs, alpha, seed):
    st, pref, tref, cref = O.multitry(w, pairs, alpha, seed=seed)
    assert st == 0
    g, part = _dev(F, w)
    st, tot, changed = ctx.multitry(g, part, w["k"], w["eps"], pairs, alpha, seed=seed)
    assert tot["status"] == 0
    assert {f: tot[f] for f in ("gain", "searches", "tried", "kept")} == tref
    assert np.array_equal(changed, cref)
    assert np.array_equal(part.cpu().numpy(), pref)
    return tref


def _matching(w, r):
    pa, pb, pr, nr = O.rounds(w)
    r = r % max(nr, 1)
    return [(int(a), int(b)) for a, b, c in zip(pa, pb, pr) if c == r]


@pytest.mark.parametrize("seed", range(20))
def test_pass_random_small(F, ctx, seed):
    w = I.random_small(7000 + seed, n_max=2500, k_max=9)
    pairs = _matching(w, seed)
    tref = _pass(F, ctx, w, pairs, (1, 10, 0, 100)[seed % 4], seed)
    assert tref["searches"] > 0


@pytest.mark.parametrize("cfg,scale", [(1, 1.0), (2, 1 / 16), (3, 1 / 64), (4, 1 / 64), (4, 1 / 16)])
def test_pass_workloads(F, ctx, cfg, scale):
    w = I.config(cfg, scale=scale)
    for r in range(2):
        _pass(F, ctx, w, _matching(w, r), 10, 1 + r)


def test_pass_empty_and_single_pair(F, ctx):
    w = I.random_small(7100, n_max=600, k_max=4)
    g, part = _dev(F, w)
    st, tot, changed = ctx.multitry(g, part, w["k"], w["eps"], [], 10)
    assert st == 0 and tot["searches"] == 0 and not changed.any()
    assert np.array_equal(part.cpu().numpy(), w["part"])
    _pass(F, ctx, w, _matching(w, 0)[:1], 10, 3)


def test_pass_quadrant_grid(F, ctx):
    xadj, adj, coords = I.grid2d(64, 64)
    x, y = coords[:, 0].astype(int), coords[:, 1].astype(int)
    part = (2 * (y >= 32) + (x >= 32)).astype(np.int32)
    for yy in range(2, 30, 5):   # bumps across the vertical line
        v = int(np.flatnonzero((x == 31) & (y == yy))[0])
        part[v] += 1
    n = 64 * 64
    w = dict(name="quadrants 64x64", n=n, nnz=len(adj), xadj=xadj, adjncy=adj,
             adjwgt=np.ones(len(adj), np.int32), vwgt=np.ones(n, np.int32), part=part, k=4, eps=0.03)
    _pass(F, ctx, w, [(0, 1), (2, 3)], 10, 9)


def _active(F, ctx, w, okw, max_outer=8, alpha=1.0):
    mt = {}
    st, pref, rref, nref = O.refine_active(w, alpha=alpha, opts=O.options(**okw), max_outer=max_outer, mt_out=mt)
    assert st == 0
    g, part = _dev(F, w)
    st, res, summ, nouter = ctx.refine_active(g, part, w["k"], w["eps"], alpha, F.default_options(**okw),
                                              max_outer=max_outer)
    assert nouter == nref and len(res) == len(rref)
    for rg, rc in zip(res, rref):
        for f in FIELDS:
            assert rg[f] == rc[f], (f, rg["a"], rg["b"], rg["round"])
    assert np.array_equal(part.cpu().numpy(), pref)
    assert (summ["mt_gain"], summ["mt_searches"], summ["mt_tried"], summ["mt_kept"]) == \
        (mt["gain"], mt["searches"], mt["tried"], mt["kept"])
    assert summ["cut_after"] == summ["cut_before"] + sum(r["cut_after"] - r["cut_before"] for r in rref) - mt["gain"]
    return summ


@pytest.mark.parametrize("seed", range(6))
def test_active_with_multitry_random_small(F, ctx, seed):
    w = I.random_small(7200 + seed, n_max=2000, k_max=7)
    okw = dict(mb=seed % 2, seed=seed, mt_alpha=10, fm_permille=(0, 50)[seed % 2])
    summ = _active(F, ctx, w, okw)
    assert summ["mt_searches"] > 0


@pytest.mark.parametrize("okw", [dict(mb=1, mt_alpha=10),
                                 dict(mb=1, adaptive=1, max_iters=6, alpha_max=8.0, fm_permille=50, mt_alpha=10)])
def test_active_with_multitry_workloads(F, ctx, okw):
    for w in (I.config(2, scale=1 / 16), I.config(4, scale=1 / 64)):
        _active(F, ctx, w, okw, max_outer=4)


def test_multitry_option_checks(F, ctx):
    w = I.random_small(7300, n_max=300, k_max=4)
    g, part = _dev(F, w)
    before = part.clone()
    st, _, _ = ctx.refine_batch(g, part, w["k"], w["eps"], w["alpha"], F.default_options(mt_alpha=10), check=False)
    assert st == F.FR_ERR_INVALID_ARG
    st, _ = ctx.refine_pair(g, part, w["k"], 0, 1, w["eps"], w["alpha"], F.default_options(mt_alpha=10),
                            check=False)
    assert st == F.FR_ERR_INVALID_ARG
    st, *_ = ctx.refine_active(g, part, w["k"], w["eps"], 1.0, F.default_options(mt_alpha=-1), check=False)
    assert st == F.FR_ERR_INVALID_ARG
    st, _, _ = ctx.multitry(g, part, w["k"], w["eps"], [(0, 1), (1, 2)], 10, check=False)   # not disjoint
    assert st == F.FR_ERR_INVALID_ARG
    assert (part == before).all()
    # gains beyond +-1023 do not fit the buckets
    w2 = dict(w, adjwgt=np.full(len(w["adjncy"]), 2000, np.int32))
    g2, part2 = _dev(F, w2)
    st, _, _ = ctx.multitry(g2, part2, w["k"], w["eps"], [(0, 1)], 10, check=False)
    assert st == F.FR_ERR_TOO_LARGE
    st, *_ = ctx.refine_active(g2, part2, w["k"], w["eps"], 1.0, F.default_options(mt_alpha=10), check=False)
    assert st == F.FR_ERR_TOO_LARGE
    assert (part2 == before).all()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_pass_hub_graph(F, ctx, seed):
    # hubs of degree 33-110 with neighbours in up to 16 blocks: the searches' serial gain
    # path (degree > 32) and its re-summing fallback (more than eight adjacent blocks)
    from tests.hub_graph import hub_workload
    w = hub_workload(seed, weighted=seed != 2)
    for r in range(2):
        _pass(F, ctx, w, _matching(w, r), (10, 1)[r], seed + r)
