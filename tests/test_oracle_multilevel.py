"""Pins of the oracle's multilevel V-cycle with a given partition: greedy matching in
expansion*2 order, contraction, projection and refinement on every level (Section 2.1
matching and contraction; Section 2.2 ratings and the weight bound on contracted nodes;
Section 5 global search: no edge between two blocks is matched).

The matching is pinned by its certificate: a set of allowed edges is the greedy
matching in a strict priority order iff an allowed edge belongs to it exactly when no
adjacent edge of the set has a higher priority (induction over the order).  The
priorities are recomputed here exactly with Python integers (splitmix64 written out
from its published definition).  Contraction is checked against S^T A S with the
0/1 membership matrix S (scipy), projection against the cut identity, and the V-cycle
is rebuilt from single matchings, contractions and batch sweeps.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from paper_1012_0006_gb300 import inputs as I

M64 = (1 << 64) - 1


def splitmix64(x):
    z = (x + 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def _edges(w):
    xadj, adj, wg = (np.asarray(w[k]) for k in ("xadj", "adjncy", "adjwgt"))
    src = np.repeat(np.arange(w["n"]), np.diff(xadj))
    m = src < adj
    return src[m], adj[m], wg[m]


def _cut(w, part):
    u, v, wt = _edges(w)
    part = np.asarray(part)
    return int(wt[part[u] != part[v]].sum())


class Prio:
    """Exact priority of an edge: larger expansion*2, then larger hash, then smaller (u, v)."""

    def __init__(self, w, seed_l):
        self.vw = [max(int(c), 1) for c in np.asarray(w["vwgt"])]
        self.seed_l = seed_l

    def key(self, u, v, wt):
        return (wt * wt, self.vw[u] * self.vw[v], splitmix64(self.seed_l ^ (u << 32) ^ v), u, v)

    @staticmethod
    def higher(a, b):
        # rating a[0]/a[1] against b[0]/b[1], exactly
        if a[0] * b[1] != b[0] * a[1]:
            return a[0] * b[1] > b[0] * a[1]
        if a[2] != b[2]:
            return a[2] > b[2]
        return (a[3], a[4]) < (b[3], b[4])


def check_greedy(w, seed_l, mate, part=None):
    part = np.asarray(w["part"] if part is None else part)
    vw = np.asarray(w["vwgt"], np.int64)
    W, k = int(vw.sum()), w["k"]
    pr = Prio(w, seed_l)
    u_, v_, w_ = _edges(w)
    allowed = {}
    for u, v, wt in zip(u_.tolist(), v_.tolist(), w_.tolist()):
        if part[u] == part[v] and 40 * k * vw[u] <= 3 * W and 40 * k * vw[v] <= 3 * W:
            allowed[(u, v)] = pr.key(u, v, wt)
    mate = np.asarray(mate)
    M = set()
    for v in range(w["n"]):
        if mate[v] >= 0:
            assert mate[mate[v]] == v
            e = (min(v, int(mate[v])), max(v, int(mate[v])))
            assert e in allowed, "matched edge not allowed"
            M.add(e)
    inc = {}
    for e in M:
        inc[e[0]] = e
        inc[e[1]] = e
    for e, ke in allowed.items():
        higher_matched = any(f in M and f != e and Prio.higher(allowed[f], ke)
                             for f in (inc.get(e[0]), inc.get(e[1])) if f is not None)
        assert (e in M) == (not higher_matched), e
    return len(M)


@pytest.mark.parametrize("seed", range(12))
def test_matching_is_the_greedy_one(seed):
    w = I.random_small(12000 + seed, n_max=700, k_max=5)
    for seed_l in (0, splitmix64(seed)):
        pairs, mate = O.match(w, seed_l=seed_l)
        assert pairs == check_greedy(w, seed_l, mate)


def test_matching_closed_forms():
    # a path with strictly falling edge weights: greedy takes (0,1), (2,3), ...
    n = 12
    xadj = np.zeros(n + 1, np.int32)
    adj, wgt = [], []
    for v in range(n):
        row = [u for u in (v - 1, v + 1) if 0 <= u < n]
        adj += row
        wgt += [100 - min(v, u) for u in row]
        xadj[v + 1] = len(adj)
    w = dict(n=n, xadj=xadj, adjncy=np.array(adj, np.int32), adjwgt=np.array(wgt, np.int32),
             vwgt=np.ones(n, np.int32), part=np.zeros(n, np.int32), k=1)
    pairs, mate = O.match(w, W=10 ** 6)
    assert pairs == 6 and [int(mate[v]) for v in range(n)] == [v ^ 1 for v in range(n)]
    # a star: equal edge weights, the lightest leaf wins (expansion*2 = omega^2 / (c(u) c(v)))
    leaves = [5, 3, 7, 2, 9]
    n = 1 + len(leaves)
    xadj = np.array([0, len(leaves)] + [len(leaves) + i + 1 for i in range(len(leaves))], np.int32)
    adj = np.array(list(range(1, n)) + [0] * len(leaves), np.int32)
    w = dict(n=n, xadj=xadj, adjncy=adj, adjwgt=np.full(len(adj), 4, np.int32),
             vwgt=np.array([1] + leaves, np.int32), part=np.zeros(n, np.int32), k=1)
    pairs, mate = O.match(w, W=10 ** 6)
    assert pairs == 1 and mate[0] == 1 + leaves.index(2)
    # the same star with the centre above 1.5 W / (20 k): nothing may be matched
    pairs, mate = O.match(w, W=10)
    assert pairs == 0 and (mate == -1).all()


def test_no_edge_between_blocks_is_matched():
    w = I.random_small(12100, n_max=800, k_max=6)
    pairs, mate = O.match(w, seed_l=5)
    part = np.asarray(w["part"])
    m = mate >= 0
    assert (part[m] == part[mate[m]]).all()


@pytest.mark.parametrize("seed", range(8))
def test_contraction_is_the_quotient_graph(seed):
    w = I.random_small(12200 + seed, n_max=900, k_max=5)
    pairs, mate = O.match(w, seed_l=seed)
    cmap, c = O.contract(w, mate)
    n, nc = w["n"], c["n"]
    assert nc == n - pairs
    # S^T A S: coarse edge weights, the matched edges on the diagonal
    xadj = np.asarray(w["xadj"])
    A = sp.csr_matrix((np.asarray(w["adjwgt"], np.int64), np.asarray(w["adjncy"]), xadj), shape=(n, n))
    S = sp.csr_matrix((np.ones(n, np.int64), (np.arange(n), cmap)), shape=(n, nc))
    Q = (S.T @ A @ S).tolil()
    Q.setdiag(0)
    Q = Q.tocsr()
    Q.eliminate_zeros()
    C = sp.csr_matrix((c["adjwgt"].astype(np.int64), c["adjncy"], c["xadj"]), shape=(nc, nc))
    assert (Q != C).nnz == 0
    # rows sorted, no loops, weights summed
    for x in range(nc):
        row = c["adjncy"][c["xadj"][x]:c["xadj"][x + 1]]
        assert (np.diff(row) > 0).all() and x not in row
    assert np.array_equal(c["vwgt"], np.bincount(cmap, weights=np.asarray(w["vwgt"]), minlength=nc).astype(np.int32))
    # coarse ids follow the smaller fine member
    rep = np.full(nc, n, np.int64)
    np.minimum.at(rep, cmap, np.arange(n))
    assert (np.diff(rep) > 0).all()
    # the partition carries over with the same cut (no matched edge crosses blocks)
    part = np.asarray(w["part"])
    cpart = np.empty(nc, np.int32)
    cpart[cmap] = part
    assert (cpart[cmap] == part).all()
    cw = dict(c, k=w["k"])
    assert _cut(cw, cpart) == _cut(w, part)


def _rebuild(w, opts, max_levels, active_outer=0):
    """The V-cycle written out from single matchings, contractions and refinements."""
    k = w["k"]
    W = int(np.asarray(w["vwgt"], np.int64).sum())
    thr = max(60 * k, w["n"] // (60 * k))
    levels, maps = [dict(w, part=np.array(w["part"], np.int32))], []
    while len(levels) < max_levels and levels[-1]["n"] > thr:
        g = levels[-1]
        pairs, mate = O.match(g, seed_l=splitmix64((opts.seed ^ (len(levels) - 1)) & M64), W=W)
        if pairs == 0 or 20 * pairs < g["n"]:
            break
        cmap, c = O.contract(g, mate)
        cp = np.empty(c["n"], np.int32)
        cp[cmap] = g["part"]
        levels.append(dict(c, part=cp, k=k, eps=w["eps"], alpha=w["alpha"]))
        maps.append(cmap)
    cuts = [0] * len(levels)
    part = levels[-1]["part"]
    for l in range(len(levels) - 1, -1, -1):
        g = levels[l]
        if l < len(levels) - 1:
            part = part[maps[l]]
        if active_outer:
            st, part, _, _ = O.refine_active(g, part=part, opts=opts, max_outer=active_outer)
        else:
            st, part, _, _ = O.refine_batch(g, part=part, opts=opts)
        assert st == 0
        cuts[l] = _cut(g, part)
    return [g["n"] for g in levels], cuts, part


@pytest.mark.parametrize("seed", range(6))
def test_vcycle_rebuilt_from_its_steps(seed):
    w = I.random_small(12300 + seed, n_max=2500, k_max=6)
    opts = O.options(mb=seed % 2, seed=seed)
    for max_levels, active in ((64, 0), (3, 0), (64, 2)):
        st, part, r = O.vcycle(w, opts=opts, max_levels=max_levels, active_outer=active)
        assert st == 0
        ns, cuts, want = _rebuild(w, opts, max_levels, active)
        assert r["level_n"] == ns and r["level_cut"] == cuts
        assert np.array_equal(part, want)
        assert r["cut_after"] == _cut(w, part) == cuts[0]
        assert r["cut_before"] == _cut(w, w["part"])
        # refinement never raises the cut, and projection keeps it
        assert all(cuts[l] <= cuts[l + 1] for l in range(len(cuts) - 1))
        assert cuts[-1] <= r["cut_before"]


def _coarsest(w, levels, seed):
    """The coarsest graph of a V-cycle's hierarchy, rebuilt from single steps."""
    W = int(np.asarray(w["vwgt"], np.int64).sum())
    g = dict(w, part=np.array(w["part"], np.int32))
    for l in range(levels - 1):
        _, mate = O.match(g, seed_l=splitmix64(seed ^ l), W=W)
        cmap, c = O.contract(g, mate)
        cp = np.empty(c["n"], np.int32)
        cp[cmap] = g["part"]
        g = dict(c, part=cp, k=w["k"], eps=w["eps"], alpha=w["alpha"])
    return g


def test_vcycle_stops_where_it_should():
    w = I.config(4, scale=1 / 64)   # 65,536 vertices, k = 64: threshold max(3840, 17) vertices
    st, part, r = O.vcycle(w, opts=O.options(mb=1))
    assert st == 0
    ns = r["level_n"]
    assert all(n > 3840 for n in ns[:-1])
    if ns[-1] > 3840 and r["levels"] < 64:   # stalled: the next matching shrinks the level by under 5 %
        g = _coarsest(w, r["levels"], 0)
        pairs, _ = O.match(g, seed_l=splitmix64(r["levels"] - 1), W=int(np.asarray(w["vwgt"]).sum()))
        assert 20 * pairs < ns[-1]
    assert r["cut_after"] < r["cut_before"]


def test_vcycle_option_checks():
    w = I.random_small(12400, n_max=200)
    assert O.vcycle(w, max_levels=0)[0] == 1
    assert O.vcycle(w, max_levels=65)[0] == 1
    assert O.vcycle(w, opts=O.options(mt_alpha=10))[0] == 1            # multi-try needs active scheduling
    assert O.vcycle(w, opts=O.options(mt_alpha=10), active_outer=2)[0] == 0


def test_vcycle_threshold_is_strict():
    # k = 2: contraction runs while the graph has more than max(120, n / 120) vertices
    for nx, ny, want in ((12, 10, 1), (11, 11, 2)):
        w = I.grid2d_halves(nx=nx, ny=ny, swaps=4)
        st, part, r = O.vcycle(w, max_levels=2)
        assert st == 0 and r["levels"] == want and r["level_n"][0] == nx * ny


def _stars(s, leaves):
    """s stars (hub + leaves, hub-leaf weight 2) whose hubs form a ring (weight 1); the
    first half of the stars in block 0.  A matching pairs each hub with one leaf only."""
    size = leaves + 1
    n = s * size
    rows = [[] for _ in range(n)]
    for i in range(s):
        hub = i * size
        for j in range(1, size):
            rows[hub].append((hub + j, 2))
            rows[hub + j].append((hub, 2))
        nxt = ((i + 1) % s) * size
        rows[hub].append((nxt, 1))
        rows[nxt].append((hub, 1))
    xadj = np.zeros(n + 1, np.int32)
    xadj[1:] = np.cumsum([len(r) for r in rows])
    adj = np.array([u for r in rows for u, _ in sorted(r)], np.int32)
    wgt = np.array([c for r in rows for _, c in sorted(r)], np.int32)
    part = (np.arange(n) // size >= s // 2).astype(np.int32)
    return dict(n=n, nnz=len(adj), xadj=xadj, adjncy=adj, adjwgt=wgt, vwgt=np.ones(n, np.int32), part=part, k=2,
                eps=0.03, alpha=1.0, mb=0)


def test_vcycle_stops_when_contraction_stalls():
    # 26 vertices per star: a matching has s pairs, under n / 20: contraction has stalled
    w = _stars(40, 25)
    st, part, r = O.vcycle(w)
    assert st == 0 and r["levels"] == 1 and O.match(w)[0] == 40
    # 15 vertices per star: s pairs >= n / 20 on every level, so contraction goes on
    w = _stars(40, 14)
    st, part, r = O.vcycle(w)
    assert st == 0 and r["levels"] > 5 and r["level_n"][1] == 600 - 40


def _cycle_rebuild(w, kind, d, opts, max_levels=64):
    """The global search cycles of Section 5 written out from single matchings,
    contractions and sweeps, following the pseudocode's recursion."""
    k = w["k"]
    W = int(np.asarray(w["vwgt"], np.int64).sum())
    thr = max(60 * k, w["n"] // (60 * k))
    count = [0] * 64
    stats = dict(coarsenings=0, refinements=0)

    def refine(g, part):
        st, part, _, _ = O.refine_batch(g, part=part, opts=opts)
        assert st == 0
        stats["refinements"] += 1
        return part

    def coarsen(l, g, part):
        if l + 1 >= max_levels or g["n"] <= thr:
            return None
        sl = splitmix64((opts.seed ^ l ^ (count[l] << 32)) & M64)
        count[l] += 1
        stats["coarsenings"] += 1
        pairs, mate = O.match(g, seed_l=sl, part=part, W=W)
        if pairs == 0 or 20 * pairs < g["n"]:
            return None
        cmap, c = O.contract(g, mate)
        cp = np.empty(c["n"], np.int32)
        cp[cmap] = part
        return dict(c, k=k, eps=w["eps"], alpha=w["alpha"]), cmap, cp

    def cyc(l, g, part):
        for trial in (0, 1):
            if trial == 1 and (kind == "V" or l % d or (kind == "F" and count[l] >= 2)):
                break
            r = coarsen(l, g, part)
            if r is None:
                if trial == 0:
                    part = refine(g, part)
                break
            c, cmap, cp = r
            part = refine(g, cyc(l + 1, c, cp)[cmap])
        return part

    part = cyc(0, dict(w), np.array(w["part"], np.int32))
    return part, stats, count


@pytest.mark.parametrize("seed", [15200, 15204, 15213, 15214, 15240])   # 1,600-2,700 vertices
def test_cycles_rebuilt_from_their_steps(seed):
    w = I.random_small(seed, n_max=3000, k_max=5)
    opts = O.options(mb=seed % 2, seed=seed)
    for kind, d in (("V", 2), ("W", 2), ("W", 1), ("F", 2), ("F", 1)):
        st, part, r = O.cycle(w, kind, d=d, opts=opts)
        assert st == 0
        want, stats, count = _cycle_rebuild(w, kind, d, opts)
        assert np.array_equal(part, want), (kind, d)
        assert (r["coarsenings"], r["refinements"]) == (stats["coarsenings"], stats["refinements"])
        assert r["level_coarsenings"] == count[:len(r["level_coarsenings"])]
        assert r["cut_after"] == _cut(w, part) <= r["cut_before"]
    # the V-cycle of the recursion is fro_vcycle
    st, pv, rv = O.vcycle(w, opts=opts)
    st, pc, rc = O.cycle(w, "V", opts=opts)
    assert np.array_equal(pv, pc) and rv["cut_after"] == rc["cut_after"]


def test_cycle_trial_counts():
    # 64x64 grid, k = 2: threshold 120, six contractions of about half each, no stalls
    w = I.grid2d_halves(nx=64, ny=64, swaps=200)
    st, _, rv = O.cycle(w, "V")
    L = rv["depth"]
    assert rv["level_coarsenings"][:L - 1] == [1] * (L - 1)
    st, _, rw = O.cycle(w, "W", d=1)
    # W with d = 1: every call above the coarsest levels coarsens twice, so level l is
    # coarsened 2^(l+1) times (near the bottom some branches end a level earlier)
    top = L - 3
    assert rw["level_coarsenings"][:top] == [2 ** (l + 1) for l in range(top)]
    assert all(c <= 2 ** (l + 1) for l, c in enumerate(rw["level_coarsenings"]))
    st, _, rf = O.cycle(w, "F", d=1)
    # F with d = 1: the second trial happens once per level and level l is reached by
    # l + 1 calls, so it is coarsened l + 2 times
    assert rf["level_coarsenings"][:top] == [l + 2 for l in range(top)]
    assert rw["cut_after"] <= rv["cut_before"] and rf["cut_after"] <= rv["cut_before"]


def test_cycle_option_checks():
    w = I.random_small(15100, n_max=200)
    st, *_ = O.cycle(w, "W", d=0)
    assert st == 1


def _paths_and_isolated(n, p3, p4):
    """p3 paths of three vertices (ids 3i .. 3i+2), one path of four on the ids in p4,
    every other vertex isolated; unit weights.  Block 0 holds the paths, block 1 the
    isolated vertices, so no edge is cut: the quotient graph is empty and every
    refinement leaves the partition as it is, while matchings run inside block 0."""
    rows = [[] for _ in range(n)]

    def edge(u, v):
        rows[u].append(v)
        rows[v].append(u)

    for i in range(p3):
        edge(3 * i, 3 * i + 1)
        edge(3 * i + 1, 3 * i + 2)
    for u, v in zip(p4, p4[1:]):
        edge(u, v)
    xadj = np.zeros(n + 1, np.int32)
    xadj[1:] = np.cumsum([len(r) for r in rows])
    adj = np.array([u for r in rows for u in sorted(r)], np.int32)
    part = np.ones(n, np.int32)
    part[:3 * p3] = 0
    part[list(p4)] = 0
    return dict(n=n, nnz=len(adj), xadj=xadj, adjncy=adj, adjwgt=np.ones(len(adj), np.int32),
                vwgt=np.ones(n, np.int32), part=part, k=2, eps=0.03, alpha=1.0, mb=0)


def _middle_first(p4, sl):
    """Whether the greedy matching takes the middle edge of the path p4 first: its three
    edges have equal expansion*2 ratings, so the larger splitmix64(sl ^ u << 32 ^ v)
    (u < v) decides (ties of the hash are impossible for distinct edges here)."""
    keys = [splitmix64(sl ^ (min(u, v) << 32) ^ max(u, v)) for u, v in zip(p4, p4[1:])]
    return keys[1] > keys[0] and keys[1] > keys[2]


def stall_case(stall_second):
    """n = 200, k = 2 (threshold max(60k, n/(60k)) = 120 < n), 8 three-vertex paths and one
    four-vertex path whose id block is chosen so that the first coarsening of level 0
    (c = 0, seed_l = splitmix64(0 ^ 0 ^ 0 << 32)) matches both end edges of the four-path
    (10 pairs: 20 * 10 = n, not under n, so it goes on), and the second (c = 1) matches its
    middle edge (9 pairs: stalled) if stall_case(True), or both end edges again if False."""
    s0, s1 = splitmix64(0), splitmix64(1 << 32)
    for a in range(24, 196):
        p4 = (a, a + 1, a + 2, a + 3)
        if not _middle_first(p4, s0) and _middle_first(p4, s1) == stall_second:
            return _paths_and_isolated(200, 8, p4)
    raise AssertionError("no placement")


@pytest.mark.parametrize("kind", ["F", "W"])
@pytest.mark.parametrize("d", [1, 2])
def test_cycle_second_coarsening_that_stalls(kind, d):
    """Section 5 cycles where level 0's second coarsening stalls: derived by hand from the
    pseudocode's recursion with max_levels = 2 (level 1 is never coarsened).
      level 0, trial 0: coarsening 1 of level 0 (10 pairs) -> G1 (190 vertices);
        level 1 cannot coarsen: refine G1 (refinement 1); project, refine G0 (2)
      level 0, trial 1 (0 % d == 0; for F fewer than two level-0 coarsenings so far):
        coarsening 2 of level 0 (seed c = 1) stalls at 9 pairs: the trial is skipped,
        nothing more is refined.
    So 2 coarsenings (both of level 0), 2 refinements, depth 2; with a second coarsening
    that does not stall the trial runs: 2 coarsenings, 4 refinements."""
    for stall, refinements in ((True, 2), (False, 4)):
        w = stall_case(stall)
        pairs0, _ = O.match(w, seed_l=splitmix64(0))
        pairs1, _ = O.match(w, seed_l=splitmix64(1 << 32))
        assert (pairs0, pairs1) == (10, 9 if stall else 10)
        st, part, r = O.cycle(w, kind, d=d, max_levels=2)
        assert st == 0
        assert (r["coarsenings"], r["refinements"], r["depth"]) == (2, refinements, 2)
        assert r["level_coarsenings"][:2] == [2, 0] and sum(r["level_coarsenings"]) == 2
        assert np.array_equal(part, w["part"]) and r["cut_after"] == r["cut_before"] == 0
    # the V-cycle never takes a second trial
    st, part, r = O.cycle(stall_case(True), "V", max_levels=2)
    assert (r["coarsenings"], r["refinements"], r["level_coarsenings"][:2]) == (1, 2, [1, 0])
