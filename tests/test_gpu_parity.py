"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

All results are integers, so the bar is bit-exact equality: corridor networks,
flow values, residual sets, output sides, partitions and result fields.  Where
several answers are correct (which maximum flow), only what is unique is
compared (the flow value and everything derived from the residual closed-set
lattice), and the rest is checked for validity (conservation, capacities).
"""
import zlib

import numpy as np
import pytest

import oracle as O
from paper_1012_0006_gb300 import inputs as I
from tests.pulse_caps import later_iteration_cap

pytestmark = pytest.mark.gpu

RESULT_FIELDS = ("flow", "cut_before", "cut_after", "wA_before", "wB_before", "wA_after", "wB_after",
                 "corridor_n", "corridor_arcs", "accepted", "iters")


@pytest.fixture(scope="module")
def F(gpu_lib):
    return gpu_lib


@pytest.fixture(scope="module")
def ctx(F):
    c = F.Context(0)
    yield c
    c.close()


def _torch():
    import torch
    return torch


def _dev(F, w):
    torch = _torch()
    return F.DeviceGraph.from_workload(w), torch.as_tensor(np.array(w["part"], np.int32)).cuda()


def _adjacent_pair(w):
    pa, pb, pr, nr = O.rounds(w)
    return (int(pa[0]), int(pb[0])) if len(pa) else (0, 1)


def _small(seed, **kw):
    w = I.random_small(seed, **kw)
    w["pair"] = _adjacent_pair(w)
    return w


def _oracle_problem(w, a, b, alpha=None):
    W = O.total_weight(w["vwgt"])
    Ub = O.budget_base(W, w["k"], w["eps"], w["alpha"] if alpha is None else alpha)
    return O.Problem.build(w, a, b, Ub)


def _flow_valid(ex, af, sf, F_val):
    """Flow on the GPU's network: antisymmetric, within capacity, conserved, value F."""
    nc = len(ex["gid"])
    net = np.zeros(nc, np.int64)
    for i in range(nc):
        for j in range(ex["off"][i], ex["off"][i + 1]):
            assert af[j] <= ex["cap"][j]
            net[i] += af[j]
        if ex["border"][i] == 1:
            assert 0 <= sf[i] < ex["infcap"][i]
            net[i] -= sf[i]
        elif ex["border"][i] == 2:
            assert 0 <= sf[i] < ex["infcap"][i]
            net[i] += sf[i]
    assert np.all(net == 0)
    assert sf[ex["border"] == 2].sum() == F_val


# ------------------------------------------------------------ corridor steps --

def _corridor_cases():
    cases = [("grid2d-64", I.config(1), (0, 1), None)]
    w2 = I.config(2)
    for al in (1.0, 4.0, 16.0):
        cases.append((f"rgg2d-65536-a{al:g}", w2, (0, 1), al))
    for seed in range(40):
        w = _small(seed, n_max=500, k_max=5)
        cases.append((f"small-{seed}", w, w["pair"], None))
    w3 = I.config(3, scale=1 / 64)
    cases.append(("grid3d-32", w3, _adjacent_pair(w3), None))
    return cases


@pytest.mark.parametrize("case", _corridor_cases(), ids=lambda c: c[0])
def test_corridor_flow_cut_parity(F, ctx, case):
    name, w, (a, b), alpha = case
    alpha = w["alpha"] if alpha is None else alpha
    p = _oracle_problem(w, a, b, alpha)
    ex = p.export()
    Fo = p.maxflow(0)
    g, part = _dev(F, w)
    c = ctx.build_corridor(g, part, w["k"], a, b, w["eps"], alpha)
    eg = c.export()
    for key in ex:
        assert np.array_equal(ex[key], eg[key]), f"corridor field {key}"
    assert c.maxflow() == Fo
    af, sf = c.flow()
    _flow_valid(eg, af, sf, Fo)
    mb = 1 if (name.endswith("16") or (zlib.crc32(name.encode()) & 1)) else 0
    res = c.extract_cut(part, mb=mb, reps=2, seed=7)
    in_s, to_t, comp, side = c.sets()
    oi, ot, oc = p.residual_sets()
    assert np.array_equal(in_s, oi) and np.array_equal(to_t, ot)
    if mb:
        assert np.array_equal(comp, oc)
    _, oside, _, _ = p.cut(mb, reps=2, seed=7)
    assert np.array_equal(side, oside)
    assert res.flow == Fo
    c.free()


def test_stale_corridor_handle_is_rejected(F, ctx):
    w = I.config(1)
    g, part = _dev(F, w)
    c1 = ctx.build_corridor(g, part, 2, 0, 1, w["eps"], 1.0)
    c2 = ctx.build_corridor(g, part, 2, 0, 1, w["eps"], 1.0)   # invalidates c1
    with pytest.raises(F.FlowRefError) as e:
        c1.maxflow()
    assert e.value.status == F.FR_ERR_INVALID_ARG
    c2.maxflow()
    c2.extract_cut(part)
    c1.free()
    c2.free()


# ---------------------------------------------------------------- one pair --

def _check_pair(F, ctx, w, a, b, opts_kw, oracle_opts):
    st, pref, rref = O.refine_pair(w, a, b, opts=oracle_opts)
    assert st == 0
    g, part = _dev(F, w)
    st, res = ctx.refine_pair(g, part, w["k"], a, b, w["eps"], w["alpha"], F.default_options(**opts_kw))
    assert np.array_equal(part.cpu().numpy(), pref)
    for f in RESULT_FIELDS:
        assert getattr(res, f) == getattr(rref, f), f
    assert res.alpha_final == rref.alpha_final


@pytest.mark.parametrize("mb", [0, 1])
def test_pair_grid64(F, ctx, mb):
    w = I.config(1)
    _check_pair(F, ctx, w, 0, 1, dict(mb=mb), O.options(mb=mb))


@pytest.mark.parametrize("mb", [0, 1])
def test_pair_rgg2d_65536_adaptive(F, ctx, mb):
    """Full-size 2D rgg, adaptive alpha up to 16 (at most 10 iterations)."""
    w = I.config(2)
    _check_pair(F, ctx, w, 0, 1, dict(mb=mb, adaptive=1, max_iters=10, alpha_max=16.0),
                O.options(mb=mb, adaptive=1, max_iters=10, alpha_max=16.0))


@pytest.mark.parametrize("alpha", [1.0, 2.0, 4.0, 8.0, 16.0])
def test_pair_rgg2d_fixed_alpha(F, ctx, alpha):
    w = dict(I.config(2), alpha=alpha)
    _check_pair(F, ctx, w, 0, 1, dict(mb=1), O.options(mb=1))


@pytest.mark.parametrize("seed", range(60))
def test_pair_random_small(F, ctx, seed):
    w = _small(1000 + seed, n_max=2000, k_max=6)
    a, b = w["pair"]
    adaptive = seed % 3 == 0
    kw = dict(mb=w["mb"], mb_reps=1 + seed % 3, seed=seed)
    ok = dict(mb=w["mb"], mb_reps=1 + seed % 3, seed=seed)
    if adaptive:
        kw.update(adaptive=1, max_iters=6, alpha_max=8.0)
        ok.update(adaptive=1, max_iters=6, alpha_max=8.0)
    _check_pair(F, ctx, w, a, b, kw, O.options(**ok))


# ------------------------------------------------------------------- batches --

def _check_batch(F, ctx, w, opts_kw=None, **okw):
    opts_kw = opts_kw or {}
    ok = dict(mb=w.get("mb", 0), mb_reps=opts_kw.get("mb_reps", 1), seed=opts_kw.get("seed", 0))
    st, pref, rref, nr = O.refine_batch(w, opts=O.options(**ok))
    assert st == 0
    g, part = _dev(F, w)
    st, res, summ = ctx.refine_batch(g, part, w["k"], w["eps"], w["alpha"],
                                     F.default_options(mb=w.get("mb", 0), **opts_kw))
    assert np.array_equal(part.cpu().numpy(), pref)
    assert summ["npairs"] == len(rref) and summ["nrounds"] == nr
    for r_gpu, r_cpu in zip(res, rref):
        assert (r_gpu["a"], r_gpu["b"], r_gpu["round"]) == (r_cpu["a"], r_cpu["b"], r_cpu["round"])
        for f in RESULT_FIELDS:
            assert r_gpu[f] == r_cpu[f], (f, r_gpu["a"], r_gpu["b"])
    assert summ["accepted"] == sum(r["accepted"] for r in rref)
    return part, summ


@pytest.mark.parametrize("seed", range(30))
def test_batch_random_small(F, ctx, seed):
    w = I.random_small(2000 + seed, n_max=2000, k_max=8)
    _check_batch(F, ctx, w, dict(mb_reps=1 + seed % 2, seed=seed))


def test_batch_grid3d_64(F, ctx):
    _check_batch(F, ctx, I.config(3, scale=1 / 8))


def test_batch_rgg3d_small(F, ctx):
    _check_batch(F, ctx, I.config(4, scale=1 / 64))


def test_batch_grid3d_128_full(F, ctx):
    """The full 128^3 grid, k = 16, alpha = 2, most balanced cuts."""
    _check_batch(F, ctx, I.config(3))


def test_batch_rgg3d_4M_full(F, ctx):
    """The full 3D rgg (n = 4,194,304, k = 64, alpha = 4, weighted) in the bench's launch configuration."""
    _check_batch(F, ctx, I.config(4))


# --------------------------------------------------------- queue sweep --

def _queue_ran(ctx):
    p = ctx.profile()
    return p["queue"], p["queue_fallbacks"]


@pytest.mark.parametrize("sched", [0, 1])
def test_batch_random_small_both_schedules(F, ctx, sched):
    """The queue sweep (0) and the round-by-round sweep (1) both give the oracle's
    partition and per-pair results on random graphs of up to 2,000 vertices and k <= 8."""
    for seed in range(12):
        w = I.random_small(2100 + seed, n_max=2000, k_max=8)
        _check_batch(F, ctx, w, dict(mb_reps=1 + seed % 2, seed=seed, sweep_sched=sched))


@pytest.mark.parametrize("case", ["grid3d64", "rgg3d262K", "grid2d", "weighted_rgg3d_k128"])
def test_queue_sweep_equals_round_sweep(F, ctx, case):
    """Same partition, per-pair results and totals from both schedules, and the oracle's."""
    if case == "grid3d64":
        w = I.config(3, scale=1 / 8)
    elif case == "rgg3d262K":
        w = I.config(4, scale=1 / 16)
    elif case == "grid2d":
        w = I.config(1)
    else:
        n = 65536
        xadj, adj, coords = I.rgg(3, n, I.rgg_radius(3, n, 12.0), 777)
        wgt = I.edge_weights(xadj, adj, 1, 10, 778)
        vw = I.uniform_i32(n, 1, 4, 779)
        part = I.rcb(coords, vw, 128)
        I.noise(xadj, adj, vw, 128, part, -10000, 780)
        w = dict(name="rgg3d k128", n=n, nnz=len(adj), xadj=xadj, adjncy=adj, adjwgt=wgt, vwgt=vw, part=part,
                 k=128, eps=0.03, alpha=2.0, mb=1)
    pq, sq = _check_batch(F, ctx, w, dict(sweep_sched=0))
    ran, _ = _queue_ran(ctx)
    assert ran == 1
    pr, sr = _check_batch(F, ctx, w, dict(sweep_sched=1))
    assert _queue_ran(ctx)[0] == 0
    assert _torch().equal(pq, pr)
    assert (sq["cut_after"], sq["accepted"], sq["corridor_arcs"]) == (sr["cut_after"], sr["accepted"],
                                                                         sr["corridor_arcs"])


def test_queue_sweep_that_outgrows_its_clusters_runs_round_by_round(F):
    """Forced 4-CTA clusters on the 2D rgg at alpha = 16 (corridors of ~31,000 vertices,
    far beyond 4 CTAs' shared memory): the queue sweep stops, part is restored, and the
    sweep runs round by round -- the oracle's partition all the same."""
    w = dict(I.config(2), alpha=16.0, mb=1)
    with F.Context(0) as c:
        _check_batch(F, c, w, dict(cluster_ctas=4))
        ran, fallbacks = _queue_ran(c)
        assert ran == 0 and fallbacks == 1


def test_queue_sweep_repeated_runs_are_identical(F, ctx):
    """Pairs start in an order that depends on timing; the results may not."""
    w = I.config(4, scale=1 / 16)
    g, part0 = _dev(F, w)
    parts = []
    for _ in range(4):
        part = part0.clone()
        ctx.refine_batch(g, part, w["k"], w["eps"], w["alpha"], F.default_options(mb=1))
        assert _queue_ran(ctx)[0] == 1
        parts.append(part)
    assert all(_torch().equal(parts[0], p) for p in parts[1:])


def test_batch_equals_pairs_in_round_order(F, ctx):
    w = I.config(3, scale=1 / 64)
    g, part = _dev(F, w)
    st, res, summ = ctx.refine_batch(g, part, w["k"], w["eps"], w["alpha"], F.default_options(mb=1))
    torch = _torch()
    part2 = torch.as_tensor(np.array(w["part"], np.int32)).cuda()
    for r in res:   # in round order
        ctx.refine_pair(g, part2, w["k"], r["a"], r["b"], w["eps"], w["alpha"], F.default_options(mb=1))
    assert torch.equal(part, part2)


def test_rounds_parity(F, ctx):
    for seed in range(10):
        w = I.random_small(3000 + seed, n_max=1500, k_max=12)
        g, part = _dev(F, w)
        pa, pb, pr, nr = ctx.rounds(g, part, w["k"])
        oa, ob, orr, onr = O.rounds(w)
        # the device lists are sorted by round; the oracle's lexicographically
        got = sorted(zip(pa.tolist(), pb.tolist(), pr.tolist()))
        exp = sorted(zip(oa.tolist(), ob.tolist(), orr.tolist()))
        assert got == exp and nr == onr
        assert list(pr) == sorted(pr)


@pytest.mark.parametrize("k,dense", [(2, False), (31, False), (64, True), (89, True), (90, True), (91, True),
                                     (130, False), (130, True)])
def test_rounds_parity_many_blocks(F, ctx, k, dense):
    # the colouring runs in one CTA's shared memory up to k = 90 and on one thread
    # beyond; dense: a random partition, so that every pair of blocks is adjacent
    # (k (k - 1) / 2 pairs, up to 2k - 1 colours)
    xadj, adj, coords = I.rgg(2, 20000, I.rgg_radius(2, 20000, 10.0), 77 + k)
    n = len(xadj) - 1
    vwgt = np.ones(n, np.int32)
    if dense:
        part = np.random.Generator(np.random.Philox(k)).integers(0, k, n).astype(np.int32)
    else:
        part = I.rcb(coords, vwgt, k)
    w = dict(name=f"rgg2d k={k}", n=n, nnz=len(adj), xadj=xadj, adjncy=adj, adjwgt=np.ones(len(adj), np.int32),
             vwgt=vwgt, part=part, k=k, eps=0.03)
    g, dpart = _dev(F, w)
    pa, pb, pr, nr = ctx.rounds(g, dpart, k)
    oa, ob, orr, onr = O.rounds(w)
    got = sorted(zip(pa.tolist(), pb.tolist(), pr.tolist()))
    exp = sorted(zip(oa.tolist(), ob.tolist(), orr.tolist()))
    assert got == exp and nr == onr
    assert list(pr) == sorted(pr)
    # inside a round the pairs keep their lexicographic order
    rows = list(zip(pr.tolist(), pa.tolist(), pb.tolist()))
    assert rows == sorted(rows)


def test_launch_shapes_give_identical_partitions(F, ctx):
    """Races would show as shape-dependent results: grid, block size, relabel interval, ops per pulse."""
    w = I.config(4, scale=1 / 128)
    ref = None
    for shape in [dict(), dict(grid_blocks=1), dict(grid_blocks=3, block_threads=256), dict(gr_interval=1),
                  dict(gr_interval=32, inner_ops=1), dict(inner_ops=16, block_threads=256), dict(pulse_passes=8),
                  dict(pulse_passes=1, grid_blocks=300)]:
        g, part = _dev(F, w)
        ctx.refine_batch(g, part, w["k"], w["eps"], w["alpha"], F.default_options(mb=1, **shape))
        got = part.cpu().numpy()
        if ref is None:
            ref = got
        assert np.array_equal(got, ref), shape


@pytest.mark.parametrize("scale", [32767, 40000])
def test_edge_weights_at_and_above_the_packed_range(F, ctx, scale):
    """Edge weights up to 32767 keep residual and capacity sum in one 32-bit word in
    the cluster kernel; larger ones use separate words.  Both layouts against the
    oracle (weights rescaled so that the largest is `scale`)."""
    for seed in range(4):
        w = I.random_small(6100 + seed, n_max=3000, k_max=6)
        adjw = np.asarray(w["adjwgt"], np.int64)
        w["adjwgt"] = np.ascontiguousarray(np.maximum(1, adjw * scale // adjw.max()), np.int32)
        w["mb"] = seed % 2
        _check_batch(F, ctx, w, dict(mb_reps=1 + seed % 2, seed=seed))


@pytest.mark.parametrize("seed", range(12))
def test_tiny_networks_in_large_clusters(F, ctx, seed):
    """Small corridors in 16-CTA clusters: most CTAs hold no vertex, and most
    balanced cuts take several colouring rounds; every CTA must leave each loop
    after the same barrier."""
    w = I.random_small(5000 + seed, n_max=300, k_max=6)
    w["mb"] = 1
    _check_batch(F, ctx, w, dict(mb_reps=2, seed=seed, cluster_ctas=16))


@pytest.mark.parametrize("ctas,sched", [(4, 0), (6, 0), (8, 0), (12, 0), (16, 0), (4, 1)])
def test_cluster_sizes_parity(F, ctx, ctas, sched):
    """Each first-tier cluster size (and the wave schedule) against the oracle."""
    _check_batch(F, ctx, I.config(4, scale=1 / 16), dict(cluster_ctas=ctas, flow_sched=sched))


@pytest.mark.parametrize("k,alpha,grid_pairs", [(6, 4.0, False), (4, 16.0, True)])
def test_cluster_tiers_and_grid_fallback(F, ctx, k, alpha, grid_pairs):
    """64^3 grid.  k = 6, alpha = 4: networks of 0.4-1 MB, so with 4-CTA clusters
    first some pairs fit and the rest go to 16-CTA clusters.  k = 4, alpha = 16:
    ~6 MB networks fit no cluster and go to the grid-wide flow.  The partition is
    the oracle's either way."""
    w = I.grid3d_rcb(64, 64, 64, k=k, alpha=alpha)
    ctx.set_profiling(True)
    try:
        _, summ = _check_batch(F, ctx, w, dict(cluster_ctas=4))
        prof = ctx.profile()
    finally:
        ctx.set_profiling(False)
    assert (prof["fallback_pairs"] > 0) == grid_pairs
    if not grid_pairs:
        assert prof["cluster_syncs"] > 0
    rounds = ctx.profile_rounds()
    assert len(rounds) == prof["nrounds"] and all(min(r) >= 0 for r in rounds)
    assert abs(sum(r[0] for r in rounds) - prof["scan_ms"]) < 1e-3 * max(1.0, prof["scan_ms"])
    assert abs(sum(r[2] for r in rounds) - prof["cluster_ms"]) < 1e-3 * max(1.0, prof["cluster_ms"])
    pairs = ctx.profile_pairs()
    assert len(pairs) > 0 and [r for r, _, _ in pairs] == sorted(r for r, _, _ in pairs)
    assert all(e >= s >= 0 for _, s, e in pairs if e >= 0)
    solved = [(r, s, e) for r, s, e in pairs if e >= 0]
    if not grid_pairs:
        assert solved and all(e <= rounds[r][2] + 1e-3 for r, _, e in solved)
    _check_batch(F, ctx, w, dict(cluster_ctas=4))   # unprofiled: no per-round or per-pair times
    assert ctx.profile_rounds() == [] and ctx.profile_pairs() == []


def test_repeated_runs_are_identical(F, ctx):
    w = I.config(3, scale=1 / 64)
    outs = []
    for _ in range(5):
        g, part = _dev(F, w)
        ctx.refine_batch(g, part, w["k"], w["eps"], w["alpha"], F.default_options(mb=1))
        outs.append(part.cpu().numpy())
    assert all(np.array_equal(o, outs[0]) for o in outs)


def test_host_buffer_batch_matches_device_batch(F, ctx):
    w = I.config(4, scale=1 / 64)
    g, part = _dev(F, w)
    ctx.refine_batch(g, part, w["k"], w["eps"], w["alpha"], F.default_options(mb=1))
    hp = np.array(w["part"], np.int32)
    ctx.refine_batch_host(w["xadj"], w["adjncy"], w["adjwgt"], w["vwgt"], hp, w["k"], w["eps"], w["alpha"],
                          F.default_options(mb=1))
    assert np.array_equal(hp, part.cpu().numpy())


def test_autotune_returns_a_shape(F, ctx):
    w = I.config(3, scale=1 / 64)
    g, part = _dev(F, w)
    best, ms = ctx.autotune(g, part, w["k"], w["eps"], w["alpha"], F.default_options(mb=1), trials=1)
    assert best.block_threads in (256, 512) and ms > 0
    # tuned shape still gives the oracle's partition
    _check_batch(F, ctx, w)


# --------------------------------------------------------------- edge cases --

def test_pair_without_common_boundary(F, ctx):
    # blocks 0 and 2 of a strip never touch: empty corridor, zero flow, nothing changes
    W, H, k = 30, 4, 3
    xadj, adj, coords = I.grid2d(W, H)
    w = dict(n=W * H, xadj=xadj, adjncy=adj, adjwgt=np.ones(len(adj), np.int32), vwgt=np.ones(W * H, np.int32),
             part=(coords[:, 0] // 10).astype(np.int32), k=k, eps=0.03, alpha=1.0)
    _check_pair(F, ctx, w, 0, 2, {}, O.options())


def test_zero_weight_vertices_and_whole_block_corridor(F, ctx):
    W, H = 12, 3
    xadj, adj, coords = I.grid2d(W, H)
    vw = np.zeros(W * H, np.int32)
    vw[::5] = 1
    w = dict(n=W * H, xadj=xadj, adjncy=adj, adjwgt=np.ones(len(adj), np.int32), vwgt=vw,
             part=(coords[:, 0] >= 6).astype(np.int32), k=2, eps=0.5, alpha=4.0)
    for mb in (0, 1):
        _check_pair(F, ctx, w, 0, 1, dict(mb=mb), O.options(mb=mb))


def test_single_vertex_blocks(F, ctx):
    xadj, adj, coords = I.grid2d(2, 1)
    w = dict(n=2, xadj=xadj, adjncy=adj, adjwgt=np.array([3, 3], np.int32), vwgt=np.array([1, 1], np.int32),
             part=np.array([0, 1], np.int32), k=2, eps=0.5, alpha=1.0)
    _check_pair(F, ctx, w, 0, 1, dict(mb=1), O.options(mb=1))
    _check_batch(F, ctx, dict(w, mb=1))


# -------------------------------------------------------------- error paths --

def test_invalid_arguments(F, ctx):
    w = I.config(1)
    g, part = _dev(F, w)
    before = part.clone()
    for args in [dict(k=1), dict(a=1, b=1), dict(eps=0.0), dict(alpha=0.5), dict(a=2)]:
        kw = dict(k=2, a=0, b=1, eps=0.03, alpha=1.0)
        kw.update(args)
        st, res = ctx.refine_pair(g, part, kw["k"], kw["a"], kw["b"], kw["eps"], kw["alpha"], check=False)
        assert st == F.FR_ERR_INVALID_ARG, args
    bad = part.clone()
    bad[17] = 5                                   # block id >= k, found by the device check
    st, res = ctx.refine_pair(g, bad, 2, 0, 1, 0.03, 1.0, check=False)
    assert st == F.FR_ERR_INVALID_ARG
    st, res, summ = ctx.refine_batch(g, bad, 2, 0.03, 1.0, check=False)
    assert st == F.FR_ERR_INVALID_ARG
    assert bad[17].item() == 5 and _torch().equal(part, before)


def test_asymmetric_graph_rejected_in_checked_mode(F, ctx):
    w = I.config(1)
    wgt = w["adjwgt"].copy()
    wgt[5] = 7
    g = F.DeviceGraph(w["xadj"], w["adjncy"], wgt, w["vwgt"])
    part = _torch().as_tensor(w["part"]).cuda()
    st, _ = ctx.refine_pair(g, part, 2, 0, 1, 0.03, 1.0, F.default_options(checked=1), check=False)
    assert st == F.FR_ERR_INVALID_ARG


def test_iteration_cap_leaves_part_unchanged(F, ctx):
    w = I.config(3, scale=1 / 64)
    g, part = _dev(F, w)
    before = part.clone()
    st, res, summ = ctx.refine_batch(g, part, w["k"], w["eps"], w["alpha"],
                                     F.default_options(mb=1, pulse_cap=1), check=False)
    assert st == F.FR_ERR_ITER_LIMIT
    assert _torch().equal(part, before)
    st, res = ctx.refine_pair(g, part, w["k"], *_adjacent_pair(w), w["eps"], w["alpha"],
                              F.default_options(pulse_cap=1), check=False)
    assert st == F.FR_ERR_ITER_LIMIT
    assert _torch().equal(part, before)
    # the context stays usable
    _check_batch(F, ctx, w)


@pytest.mark.parametrize("mb", [0, 1])
def test_error_in_a_later_adaptive_iteration_leaves_part_unchanged(F, ctx, mb):
    """Iteration 1 is accepted and written to part; iteration 2 hits the pulse cap
    (a host-side bound, no fault): the call fails and part is as it came in."""
    torch = _torch()
    tried = 0
    for w in (I.config(2, scale=0.5), I.config(2, scale=0.25), I.config(2)):
        if tried:
            break
        g = F.DeviceGraph.from_workload(w)
        kw = dict(mb=mb, flow_sched=1)   # level-ordered waves: counts that do not vary between runs
        cap = later_iteration_cap(
            lambda p, al, k_: ctx.refine_pair(g, p, w["k"], 0, 1, w["eps"], al, F.default_options(**k_))[1], w, kw,
            exact=True)
        if cap is None:
            continue
        tried += 1
        part = torch.as_tensor(np.array(w["part"], np.int32)).cuda()
        before = part.clone()
        st, res = ctx.refine_pair(g, part, w["k"], 0, 1, w["eps"], 1.0,
                                  F.default_options(mb=mb, flow_sched=1, adaptive=1, max_iters=10, alpha_max=16.0,
                                                    pulse_cap=cap), check=False)
        assert st == F.FR_ERR_ITER_LIMIT and res.status == F.FR_ERR_ITER_LIMIT
        assert res.iters >= 2
        assert torch.equal(part, before)
        # the context stays usable: a normal call gives the oracle's partition
        _check_pair(F, ctx, w, 0, 1, dict(mb=mb, adaptive=1, max_iters=10, alpha_max=16.0),
                    O.options(mb=mb, adaptive=1, max_iters=10, alpha_max=16.0))
    assert tried, "no workload separates the pulse counts of the first two iterations"


def test_arena_bound_gives_oom(F):
    w = I.config(3, scale=1 / 64)
    g, part = _dev(F, w)
    with F.Context(0, arena_bytes=1 << 16) as small:
        st, res, summ = small.refine_batch(g, part, w["k"], w["eps"], w["alpha"], check=False)
        assert st == F.FR_ERR_OOM


def test_captured_sweeps_survive_workspace_growth(F):
    """A captured sweep is replayed only while the workspace it points into lives:
    small graph (captured, replayed), larger graph (workspaces reallocated), small
    graph again -- the oracle's partition every time."""
    small, big = I.config(3, scale=1 / 64), I.config(4, scale=1 / 16)
    with F.Context(0) as c:
        for w in (small, small, big, small, big, small):
            _check_batch(F, c, w)


def test_batch_with_the_largest_block_count(F, ctx):
    """k = 1024 (the largest the library takes): a 3D rgg of 32,768 vertices cut by RCB
    into 1,024 blocks of 32, a quotient graph of thousands of pairs in many rounds; k =
    1025 is refused."""
    n = 32768
    xadj, adj, coords = I.rgg(3, n, I.rgg_radius(3, n, 12.0), 4242)
    vwgt = np.ones(n, np.int32)
    part = I.rcb(coords, vwgt, 1024)
    I.noise(xadj, adj, vwgt, 1024, part, 300, 77)
    w = I._workload("rgg3d 32768 k=1024", xadj, adj, I.edge_weights(xadj, adj, 1, 10, 5), vwgt, part, 1024,
                    eps=0.05, alpha=2.0, mb=1)
    _, summ = _check_batch(F, ctx, w)
    assert summ["npairs"] > 2000 and summ["nrounds"] > 10
    g, p = _dev(F, w)
    st, _, _ = ctx.refine_batch(g, p, 1025, w["eps"], w["alpha"], F.default_options(), check=False)
    assert st == F.FR_ERR_INVALID_ARG
