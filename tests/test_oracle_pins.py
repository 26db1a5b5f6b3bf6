"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself.  Each test checks the oracle
against something independent: a hand-derived worked example, a closed form on
grids, brute-force enumeration of all cuts, max-flow/min-cut duality, flow
conservation, the Picard-Queyranne correspondence, a second max-flow algorithm,
an independent BFS, or exact rational arithmetic.
"""
import os
from fractions import Fraction
import math

import numpy as np
import pytest

import oracle as O
from paper_1012_0006_gb300 import inputs as I
from tests import bruteforce as BF

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _grid_halves(W, H, c0, eps):
    xadj, adj, coords = I.grid2d(W, H)
    n = W * H
    return dict(n=n, nnz=len(adj), xadj=xadj, adjncy=adj, adjwgt=np.ones(len(adj), np.int32),
                vwgt=np.ones(n, np.int32), part=(coords[:, 0] >= c0).astype(np.int32), k=2, eps=eps, alpha=1.0)


def _read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *rest = line.split()
            vals[key] = [int(x) for x in rest]
    return vals


# ------------------------------------------------------------------ generators --

def test_splitmix64_published_vector():
    # First output of splitmix64 seeded with 0 (Vigna's reference generator).
    assert O.splitmix64(0) == 0xE220A8397B1DCDAF


# ------------------------------------------------------------- Section 2.1 ----

@pytest.mark.parametrize("W,k,eps,alpha,maxc", [(100, 2, 0.5, 1.0, 1), (1024, 2, 0.125, 1.0, 1),
                                                 (4096, 16, 0.25, 2.0, 3), (777, 3, 0.125, 4.0, 0),
                                                 (2 ** 40 + 12345, 64, 0.0625, 8.0, 7)])
def test_budget_and_lmax_exact_rationals(W, k, eps, alpha, maxc):
    # eps and alpha are dyadic, so (1 + alpha*eps) W / k is an exact rational here.
    e, a = Fraction(eps), Fraction(alpha)
    assert O.budget_base(W, k, eps, alpha) == math.floor((1 + a * e) * W / k)
    assert O.lmax(W, maxc, k, eps) == math.floor((1 + e) * W / k) + maxc


def test_validation_rejects_bad_inputs():
    w = _grid_halves(6, 4, 3, 0.1)
    assert O.validate(w) == 0
    bad = dict(w, part=w["part"].copy())
    bad["part"][3] = 2                        # block id >= k
    assert O.validate(bad) == 1
    asym = dict(w, adjwgt=w["adjwgt"].copy())
    asym["adjwgt"][0] = 5                     # omega(u,v) != omega(v,u)
    assert O.validate(asym) == 1
    zero = dict(w, adjwgt=np.zeros_like(w["adjwgt"]))   # omega must be > 0
    assert O.validate(zero) == 1
    negc = dict(w, vwgt=w["vwgt"].copy())
    negc["vwgt"][0] = -1                      # c >= 0
    assert O.validate(negc) == 1
    st, _, _ = O.refine_pair(w, 0, 1, eps=0.0)
    assert st == 1                            # epsilon must be positive
    st, _, _ = O.refine_pair(w, 0, 1, alpha=0.5)
    assert st == 1                            # alpha >= 1
    st, _, _ = O.refine_pair(w, 1, 1)
    assert st == 1                            # a != b


# ------------------------------------------------------- the worked example --

def test_worked_example_grid_64x16():
    g = _read_golden("p5_grid64x16.txt")
    w = _grid_halves(64, 16, 30, 0.125)
    Ub = O.budget_base(1024, 2, 0.125, 1.0)
    assert Ub - 544 == g["U0"][0] and Ub - 480 == g["U1"][0]
    p = O.Problem.build(w, 0, 1, Ub)
    ex = p.export()
    cols = ex["gid"] % 64
    assert sorted(set(cols.tolist())) == g["corridor_columns"]
    assert sorted(set(cols[ex["border"] == 1].tolist())) == g["s_border_column"]
    assert sorted(set(cols[ex["border"] == 2].tolist())) == g["t_border_column"]
    assert p.maxflow(0) == g["flow"][0]
    in_s, to_t, comp = p.residual_sets()
    assert sorted(set(cols[in_s].tolist())) == g["smallest_source_columns"]
    assert sorted(set(cols[to_t].tolist())) == g["sink_reaching_columns"]
    order, d = p.sweep(0)
    assert [int(o) % 64 for o in order] == g["sweep_order_columns"]
    assert d.tolist() == g["sweep_d"]
    _, _, bj, br = p.cut(1)
    assert bj == g["mb_best_j"][0] and br == 0
    st, part, res = O.refine_pair(w, 0, 1, opts=O.options(mb=0))
    assert (res.accepted, res.wA_after, res.wB_after) == (g["plain_accepted"][0], *g["plain_weights"])
    assert np.array_equal(part, w["part"])
    st, part, res = O.refine_pair(w, 0, 1, opts=O.options(mb=1))
    assert (res.accepted, res.wA_after, res.wB_after) == (g["mb_accepted"][0], *g["mb_weights"])
    assert (res.cut_before, res.cut_after) == (g["cut_before"][0], g["cut_after"][0])
    assert np.array_equal(part, (np.arange(1024) % 64 >= 32).astype(np.int32))


@pytest.mark.parametrize("W,H,c0,eps", [(64, 16, 30, 0.125), (40, 8, 18, 0.25), (48, 5, 22, 0.25),
                                         (32, 12, 17, 0.25), (64, 3, 33, 0.125)])
def test_closed_form_grid_family(W, H, c0, eps):
    """Unit grid split by columns: every quantity follows from the geometry."""
    w = _grid_halves(W, H, c0, eps)
    total = W * H
    Ub = math.floor((1 + Fraction(eps)) * total / 2)
    UA, UB = max(0, Ub - (W - c0) * H), max(0, Ub - c0 * H)
    ca, cb = min(UA // H, c0), min(UB // H, W - c0)      # full columns per side
    assert UA % H == 0 and UB % H == 0 and ca >= 1 and cb >= 1, "choose whole-column budgets"
    p = O.Problem.build(w, 0, 1, O.budget_base(total, 2, eps, 1.0))
    ex = p.export()
    cols = sorted(set((ex["gid"] % W).tolist()))
    assert cols == list(range(c0 - ca, c0 + cb))
    F = p.maxflow(0)
    assert F == H                                        # one cut edge per row
    in_s, to_t, comp = p.residual_sets()
    colv = ex["gid"] % W
    assert set(colv[in_s].tolist()) == {c0 - ca}          # only the s-border column
    assert set(colv[to_t].tolist()) == {c0 + cb - 1}      # only the t-border column
    order, d = p.sweep(0)
    # SCCs are whole columns; the sweep moves them to the sink side right to left
    assert [int(o) % W for o in order] == list(range(c0 + cb - 2, c0 - ca, -1))
    # A' after j moves holds c0 + cb - 1 - j columns
    assert d.tolist() == [(2 * (c0 + cb - 1 - j) - W) * H for j in range(len(order) + 1)]
    best = min(range(len(d)), key=lambda j: (abs(d[j]), j))
    _, side, bj, _ = p.cut(1)
    assert bj == best


# -------------------------------------------------------- brute force (P1) --

def _small_cases(count, max_nc=18, start=1000):
    got, seed = 0, start
    while got < count and seed < start + 50 * count:
        seed += 1
        w = I.random_small(seed, n_max=60, k_max=3)
        a, b = 0, 1
        W = O.total_weight(w["vwgt"])
        Ub = O.budget_base(W, w["k"], w["eps"], w["alpha"])
        p = O.Problem.build(w, a, b, Ub)
        if 1 <= p.nc <= max_nc:
            got += 1
            yield w, p


def test_bruteforce_min_cuts_and_closed_sets():
    checked = mb_optimal = 0
    for w, p in _small_cases(40):
        ex = p.export()
        F = p.maxflow(0)
        masks, cut, bits = BF.cut_values(ex)
        assert F == cut.min()                                        # max flow = min cut
        minimal = cut == F
        in_s, to_t, comp = p.residual_sets()
        inter = np.bitwise_and.reduce(masks[minimal])
        union = np.bitwise_or.reduce(masks[minimal])
        assert inter == BF.mask_of(in_s)                             # smallest source set
        assert union == BF.mask_of(~to_t)                            # largest source set
        af, sf = p.flow()
        closed = BF.closed_masks(ex, af, sf, bits)
        assert np.array_equal(closed, minimal)                       # Picard-Queyranne
        # every sweep step is a minimum cut; the MB choice is one of them
        order, d = p.sweep(0)
        cA = int(w["vwgt"][w["part"] == 0].sum())
        cB = int(w["vwgt"][w["part"] == 1].sum())
        vw = w["vwgt"][ex["gid"]]
        wA, wB = BF.side_weights(ex, vw, cA, cB, bits)
        for j in range(len(order) + 1):
            moved = set(order[:j].tolist())
            src = [(bool(in_s[i]) or (comp[i] >= 0 and comp[i] not in moved)) for i in range(p.nc)]
            mk = BF.mask_of(src)
            assert cut[mk] == F
            assert wA[mk] - wB[mk] == d[j]
        capv, side, bj, br = p.cut(1)
        assert capv == F                                             # duality for the MB cut
        mk = BF.mask_of(side == 0)
        assert cut[mk] == F
        best = np.abs(wA - wB)[minimal].min()
        assert abs(wA[mk] - wB[mk]) >= best                          # heuristic, not exact
        mb_optimal += int(abs(wA[mk] - wB[mk]) == best)
        capv0, side0, _, _ = p.cut(0)
        assert capv0 == F and BF.mask_of(side0 == 0) == inter
        checked += 1
    assert checked >= 30
    assert mb_optimal >= checked // 2


def _random_network(rs, nc):
    """Arbitrary small network in export format: symmetric arc structure, independent capacities."""
    edges = set()
    for _ in range(int(rs.integers(nc, 3 * nc))):
        u, v = rs.integers(0, nc, 2)
        if u != v:
            edges.add((min(u, v), max(u, v)))
    rows = [[] for _ in range(nc)]
    for u, v in sorted(edges):
        rows[u].append((v, int(rs.integers(0, 6))))
        rows[v].append((u, int(rs.integers(0, 6))))
    off = np.zeros(nc + 1, np.int32)
    head, cap = [], []
    for i in range(nc):
        for h, c in rows[i]:
            head.append(h)
            cap.append(c)
        off[i + 1] = len(head)
    border = rs.choice([0, 0, 1, 2], nc).astype(np.int8)
    border[0], border[-1] = 1, 2
    infcap = np.where(border > 0, rs.integers(1, 12, nc), 0).astype(np.int32)
    side0 = (border == 2).astype(np.int8)
    vw = rs.integers(0, 4, nc).astype(np.int32)
    return (off, np.array(head, np.int32), np.array(cap, np.int32), border, infcap, vw, side0)


def test_bruteforce_arbitrary_networks():
    rs = np.random.Generator(np.random.Philox(7))
    for _ in range(60):
        nc = int(rs.integers(2, 15))
        net = _random_network(rs, nc)
        vw, side0 = net[5], net[6]
        cA = int(vw[side0 == 0].sum()) + 3
        cB = int(vw[side0 == 1].sum()) + 5
        ex = dict(gid=np.arange(nc), off=net[0], head=net[1], cap=net[2], border=net[3], infcap=net[4], side0=side0)
        masks, cut, bits = BF.cut_values(ex)
        for method in (0, 1):
            p = O.Problem.from_network(*net, cA, cB)
            F = p.maxflow(method)
            assert F == cut.min()
            in_s, to_t, _ = p.residual_sets()
            assert np.bitwise_and.reduce(masks[cut == F]) == BF.mask_of(in_s)
            af, sf = p.flow()
            assert np.array_equal(BF.closed_masks(ex, af, sf, bits), cut == F)


# ------------------------------------------------ flow validity (P2, P3) ----

def test_flow_conservation_and_capacity():
    for seed in range(200, 230):
        w = I.random_small(seed, n_max=300)
        W = O.total_weight(w["vwgt"])
        p = O.Problem.build(w, 0, 1, O.budget_base(W, w["k"], w["eps"], w["alpha"]))
        F = p.maxflow(0)
        ex = p.export()
        af, sf = p.flow()
        net = np.zeros(p.nc, np.int64)
        for i in range(p.nc):
            for j in range(ex["off"][i], ex["off"][i + 1]):
                assert af[j] <= ex["cap"][j]                        # 0 <= f <= c per direction
                net[i] += af[j]                                     # net outflow on corridor arcs
            if ex["border"][i] == 1:
                assert 0 <= sf[i] < ex["infcap"][i]                 # INF_v never saturated
                net[i] -= sf[i]
            elif ex["border"][i] == 2:
                assert 0 <= sf[i] < ex["infcap"][i]
                net[i] += sf[i]
            else:
                assert sf[i] == 0
        assert np.all(net == 0)                                     # conservation
        assert sf[ex["border"] == 2].sum() == F == sf[ex["border"] == 1].sum()
        for mb in (0, 1):
            assert p.cut(mb)[0] == F                                # duality


# ------------------------------------------------- max-flow invariance (P4) --

def test_partition_independent_of_max_flow():
    differing = 0
    for seed in range(300, 340):
        w = I.random_small(seed, n_max=400)
        W = O.total_weight(w["vwgt"])
        Ub = O.budget_base(W, w["k"], w["eps"], w["alpha"])
        p1, p2 = O.Problem.build(w, 0, 1, Ub), O.Problem.build(w, 0, 1, Ub)
        assert p1.maxflow(0) == p2.maxflow(1)
        differing += int(not np.array_equal(p1.flow()[0], p2.flow()[0]))
        for a, b in zip(p1.residual_sets(), p2.residual_sets()):
            assert np.array_equal(a, b)
        for mb in (0, 1):
            assert np.array_equal(p1.cut(mb, reps=3, seed=seed)[1], p2.cut(mb, reps=3, seed=seed)[1])
    assert differing >= 5     # the two algorithms really produced different flows


# ------------------------------------------- cut property and monotonicity --

def test_cut_property_alpha_one():
    """Section 4.1: at alpha = 1 every minimum cut of G' is balanced in G."""
    for seed in range(400, 440):
        w = I.random_small(seed, n_max=300)
        W = O.total_weight(w["vwgt"])
        Ub = O.budget_base(W, w["k"], w["eps"], 1.0)
        p = O.Problem.build(w, 0, 1, Ub)
        p.maxflow(0)
        cA = int(w["vwgt"][w["part"] == 0].sum())
        cB = int(w["vwgt"][w["part"] == 1].sum())
        order, d = p.sweep(0)
        tot = cA + cB
        for dj in d:
            wA = (tot + dj) // 2
            wB = tot - wA
            assert max(wA, wB) <= max(Ub, cA, cB)


def test_refinement_never_increases_cut():
    for seed in range(500, 560):
        w = I.random_small(seed, n_max=400)
        for mb in (0, 1):
            st, part, res = O.refine_pair(w, 0, 1, opts=O.options(mb=mb))
            assert st == 0
            assert res.cut_after <= res.cut_before
            assert res.cut_after == O.pair_cut(w, part, 0, 1)
            W = O.total_weight(w["vwgt"])
            Lm = O.lmax(W, int(w["vwgt"].max()), w["k"], w["eps"])
            if res.accepted:
                assert max(res.wA_after, res.wB_after) <= Lm
            else:
                assert np.array_equal(part, w["part"])
            # only vertices of the two blocks move, and only between them
            moved = part != w["part"]
            assert np.all(np.isin(w["part"][moved], [0, 1])) and np.all(np.isin(part[moved], [0, 1]))


# --------------------------------------------------------------- corridor --

def test_corridor_is_bfs_prefix():
    """Corridor = longest (distance, id) prefix under the budget, via scipy's BFS."""
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    for seed in range(600, 630):
        w = I.random_small(seed, n_max=400)
        W = O.total_weight(w["vwgt"])
        Ub = O.budget_base(W, w["k"], w["eps"], w["alpha"])
        p = O.Problem.build(w, 0, 1, Ub)
        ex = p.export()
        taken = set(ex["gid"].tolist())
        n, part, vw = w["n"], w["part"], w["vwgt"]
        rows = np.repeat(np.arange(n), np.diff(w["xadj"]))
        cols = w["adjncy"]
        for X, Y in ((0, 1), (1, 0)):
            U = max(0, Ub - int(vw[part == Y].sum()))
            keep = (part[rows] == X) & (part[cols] == X)
            # super source n joined to the boundary of X towards Y
            seeds = np.unique(rows[(part[rows] == X) & (part[cols] == Y)])
            r2 = np.concatenate([rows[keep], np.full(len(seeds), n)])
            c2 = np.concatenate([cols[keep], seeds])
            A = sp.csr_matrix((np.ones(len(r2)), (r2, c2)), shape=(n + 1, n + 1))
            dist = csgraph.shortest_path(A, unweighted=True, indices=n, directed=True)
            reached = [v for v in range(n) if part[v] == X and np.isfinite(dist[v])]
            reached.sort(key=lambda v: (dist[v], v))
            run, expect = 0, []
            for v in reached:
                if run + vw[v] > U:
                    break
                run += vw[v]
                expect.append(v)
            got = sorted(v for v in taken if part[v] == X)
            assert got == sorted(expect)
            dmap = dict(zip(ex["gid"].tolist(), ex["dist"].tolist()))
            assert all(dmap[v] == dist[v] - 1 for v in expect)


# ------------------------------------------------------------- batching --

def test_rounds_are_matchings_covering_the_quotient_graph():
    for seed in range(700, 720):
        w = I.random_small(seed, n_max=400, k_max=8)
        pa, pb, pr, nr = O.rounds(w)
        part, k = w["part"], w["k"]
        adj = set()
        rows = np.repeat(np.arange(w["n"]), np.diff(w["xadj"]))
        for x, y in zip(part[rows], part[w["adjncy"]]):
            if x != y:
                adj.add((min(x, y), max(x, y)))
        assert set(zip(pa.tolist(), pb.tolist())) == adj
        for r in range(nr):
            blocks = np.concatenate([pa[pr == r], pb[pr == r]])
            assert len(blocks) == len(set(blocks.tolist()))          # matching
        deg = np.bincount(np.concatenate([pa, pb]), minlength=k)
        assert nr <= max(1, 2 * deg.max() - 1)


def test_rounds_on_a_path_of_blocks_alternate():
    # blocks in a row (a strip cut into k slabs): the quotient graph is a path
    W, H, k = 40, 3, 5
    xadj, adj, coords = I.grid2d(W, H)
    part = (coords[:, 0] // (W // k)).astype(np.int32)
    w = dict(n=W * H, xadj=xadj, adjncy=adj, part=part, k=k)
    pa, pb, pr, nr = O.rounds(w)
    assert list(zip(pa.tolist(), pb.tolist())) == [(0, 1), (1, 2), (2, 3), (3, 4)]
    assert pr.tolist() == [0, 1, 0, 1] and nr == 2


def test_batch_equals_pairs_in_round_order():
    for seed in range(800, 812):
        w = I.random_small(seed, n_max=400, k_max=6)
        w["mb"] = seed % 2
        st, part_b, res_b, nr = O.refine_batch(w)
        assert st == 0
        pa, pb, pr, _ = O.rounds(w)
        part = w["part"].copy()
        for r in range(nr):
            idx = [i for i in range(len(pa)) if pr[i] == r]
            for i in reversed(idx):              # any order inside a round gives the same result
                st, part, _ = O.refine_pair(w, int(pa[i]), int(pb[i]), part=part)
        assert np.array_equal(part, part_b)


def test_adaptive_iterations_invariants():
    w = I.config(2, scale=1 / 16)
    st, p1, r1 = O.refine_pair(w, opts=O.options(adaptive=0))
    st, pa, ra = O.refine_pair(w, opts=O.options(adaptive=1, max_iters=10, alpha_max=16.0))
    assert ra.iters >= 1 and ra.iters <= 10
    assert ra.cut_after <= r1.cut_after                # later iterations only accept improvements
    st, pa1, ra1 = O.refine_pair(w, opts=O.options(adaptive=1, max_iters=1, alpha_max=16.0))
    assert np.array_equal(pa1, p1)                     # first adaptive iteration = plain iteration
    W = O.total_weight(w["vwgt"])
    assert max(ra.wA_after, ra.wB_after) <= O.lmax(W, 1, 2, w["eps"])
    assert ra.alpha_final in {1.0, 2.0, 4.0, 8.0, 16.0}


def _adaptive_replay(w, a, b, alpha, alpha_max, max_iters, mb):
    """The adaptive loop of Section 4.1 (reading D12) written out over the oracle's
    single-iteration pieces (corridor, max flow, cut; each pinned above): returns the
    final partition, the iterations run and the final alpha."""
    part = np.array(w["part"], np.int32, copy=True)
    vw = np.asarray(w["vwgt"], np.int64)
    W = int(vw.sum())
    Lmax = O.lmax(W, int(vw.max()), w["k"], w["eps"])
    cut = O.pair_cut(w, part, a, b)
    wA, wB = int(vw[part == a].sum()), int(vw[part == b].sum())
    al, iters = alpha, 0
    while iters < max_iters:
        iters += 1
        pb = O.Problem.build(w, a, b, O.budget_base(W, w["k"], w["eps"], al), part=part)
        pb.maxflow()
        _, side, _, _ = pb.cut(mb=mb)
        trial = part.copy()
        trial[pb.export()["gid"]] = np.where(side.astype(bool), b, a)
        ncut = O.pair_cut(w, trial, a, b)
        nA, nB = int(vw[trial == a].sum()), int(vw[trial == b].sum())
        feasible = max(nA, nB) <= Lmax
        if feasible and ncut < cut:
            part, cut, wA, wB = trial, ncut, nA, nB
            al = min(2.0 * al, alpha_max)
            continue
        if feasible:
            if ncut == cut and max(nA, nB) < max(wA, wB):
                part, cut, wA, wB = trial, ncut, nA, nB
            break
        if al == 1.0:
            break
        al = max(al / 2.0, 1.0)
    return part, iters, al


@pytest.mark.parametrize("seed", range(8))
def test_adaptive_loop_replayed(seed):
    """The oracle's adaptive flow iterations against the loop written out here from
    D12 over the oracle's one-iteration pieces: same partition, iterations and alpha."""
    w = I.random_small(5700 + seed, n_max=1500, k_max=3) if seed % 2 else I.config(2, scale=1 / 64)
    pa, pb, _, _ = O.rounds(w)
    a, b = int(pa[0]), int(pb[0])
    mb = seed % 3 == 0
    alpha, amax, iters = (1.0, 16.0, 10) if seed < 4 else (4.0, 8.0, 3)
    exp, it, al = _adaptive_replay(w, a, b, alpha, amax, iters, int(mb))
    st, part, res = O.refine_pair(w, a, b, alpha=alpha,
                                  opts=O.options(mb=int(mb), adaptive=1, max_iters=iters, alpha_max=amax))
    assert st == 0
    assert np.array_equal(part, exp)
    assert (res.iters, res.alpha_final) == (it, al)


def test_sweeps_with_keys_are_valid_orders():
    """Sweeps r >= 1 (splitmix64 keys): each is a permutation of the components whose
    every prefix moved to the sink side leaves a minimum cut (the prefix is closed under
    the residual arcs), checked by brute force; d_j is the weight difference of that cut."""
    checked = 0
    for w, p in _small_cases(30):
        ex = p.export()
        F = p.maxflow(0)
        masks, cut, bits = BF.cut_values(ex)
        in_s, to_t, comp = p.residual_sets()
        cA = int(w["vwgt"][w["part"] == 0].sum())
        cB = int(w["vwgt"][w["part"] == 1].sum())
        vw = w["vwgt"][ex["gid"]]
        wA, wB = BF.side_weights(ex, vw, cA, cB, bits)
        comps = sorted(set(int(c) for c in comp if c >= 0))
        for r in (1, 2, 3):
            order, d = p.sweep(r, seed=17 + r)
            assert sorted(order.tolist()) == comps
            for j in range(len(order) + 1):
                moved = set(order[:j].tolist())
                src = [(bool(in_s[i]) or (comp[i] >= 0 and comp[i] not in moved)) for i in range(p.nc)]
                mk = BF.mask_of(src)
                assert cut[mk] == F
                assert wA[mk] - wB[mk] == d[j]
        checked += 1
    assert checked >= 20
