"""Pins of the oracle's two-way FM with TopGain (Section 2.2; stopping rule of the
Section 6, "Configuring the Algorithm").

The oracle keeps its queues in binary heaps.  The pin replays every run from its
move log with nothing but brute force: at each step it recomputes every gain from
the graph, checks that the moved vertex is the best unmoved boundary vertex of its
block (by gain, then stamp) and that the block follows TopGain (larger top gain;
the seeded bit on a tie; the heavier block while one is overloaded), recomputes the
pair cut and block weights from scratch, and checks the stopping rule and the
rollback to the best prefix.  The stamps and the tie bit come from splitmix64
written out here from its published definition.
"""
import numpy as np
import pytest

import oracle as O
from paper_1012_0006_gb300 import inputs as I

M64 = (1 << 64) - 1


def splitmix64(x):
    z = (x + 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def _pair_state(w, part, a, b):
    xadj, adj, wg, vw = (np.asarray(w[k]) for k in ("xadj", "adjncy", "adjwgt", "vwgt"))
    cut = 0
    for v in range(w["n"]):
        if part[v] != a:
            continue
        for j in range(xadj[v], xadj[v + 1]):
            if part[adj[j]] == b:
                cut += int(wg[j])
    return cut, int(vw[part == a].sum()), int(vw[part == b].sum())


def _gains(w, part, a, b, moved):
    """gain and boundary flag of every unmoved vertex of a and b, from scratch"""
    xadj, adj, wg = (np.asarray(w[k]) for k in ("xadj", "adjncy", "adjwgt"))
    g = {}
    for v in range(w["n"]):
        if moved[v] or part[v] not in (a, b):
            continue
        other = b if part[v] == a else a
        ext = sum(int(wg[j]) for j in range(xadj[v], xadj[v + 1]) if part[adj[j]] == other)
        inn = sum(int(wg[j]) for j in range(xadj[v], xadj[v + 1]) if part[adj[j]] == part[v])
        if ext > 0:
            g[v] = ext - inn
    return g


def replay(w, a, b, permille, seed, Lmax):
    st, out, res, moves = O.fm_pair(w, a, b, permille, seed=seed, Lmax=Lmax)
    assert st == 0
    part = np.array(w["part"], np.int32, copy=True)
    xadj = np.asarray(w["xadj"])
    fs = splitmix64((seed ^ (a << 32) ^ b) & M64)
    stamp = {v: splitmix64(fs ^ v) >> 1 for v in range(w["n"])}
    moved = np.zeros(w["n"], bool)
    cut, wA, wB = _pair_state(w, part, a, b)
    assert res["cut_before"] == cut
    N = int(np.isin(part, (a, b)).sum())
    limit = permille * N // 1000
    rank = lambda c, x, y: (max(0, max(x, y) - Lmax), c, max(x, y))
    best, best_len, idle, t = rank(cut, wA, wB), 0, 0, 0
    hist = [(cut, wA, wB)]
    for i, v in enumerate(moves.tolist()):
        g = _gains(w, part, a, b, moved)
        qa = [u for u in g if part[u] == a]
        qb = [u for u in g if part[u] == b]
        assert qa or qb, "moved with both queues empty"
        top = lambda q: max(q, key=lambda u: (g[u], stamp[u], -u))
        if wA > Lmax or wB > Lmax:
            s = 0 if wA >= wB else 1
            if not (qa, qb)[s]:
                s = 1 - s
        elif not qa:
            s = 1
        elif not qb:
            s = 0
        elif g[top(qa)] != g[top(qb)]:
            s = 0 if g[top(qa)] > g[top(qb)] else 1
        else:
            s = splitmix64((~fs & M64) ^ i) & 1
        assert v == top((qa, qb)[s]), f"move {i}: vertex {v} is not the TopGain choice"
        # apply, with fresh stamps for the neighbours whose gain changed
        part[v] = b if s == 0 else a
        moved[v] = True
        for j in range(xadj[v], xadj[v + 1]):
            u = int(w["adjncy"][j])
            if not moved[u] and part[u] in (a, b):
                stamp[u] = (1 << 63) + int(t) + int(j - xadj[v])
        t += int(xadj[v + 1] - xadj[v])
        cut, wA, wB = _pair_state(w, part, a, b)
        hist.append((cut, wA, wB))
        r = rank(cut, wA, wB)
        if r < best:
            best, best_len, idle = r, i + 1, 0
        else:
            idle += 1
            if idle > limit:
                assert i == len(moves) - 1, "did not stop when the stopping rule fired"
    if len(moves) and idle <= limit:   # ended with empty queues
        assert not _gains(w, part, a, b, moved)
    assert res["kept"] == best_len and res["tried"] == len(moves)
    c, x, y = hist[best_len]
    assert (res["cut_after"], res["wA_after"], res["wB_after"]) == (c, x, y)
    # the output is the start with the kept prefix applied
    exp = np.array(w["part"], np.int32, copy=True)
    for v in moves[:best_len]:
        exp[v] = b if exp[v] == a else a
    assert np.array_equal(out, exp)
    assert _pair_state(w, out, a, b) == (c, x, y)
    return res


def _lmax(w):
    vw = np.asarray(w["vwgt"], np.int64)
    return O.lmax(int(vw.sum()), int(vw.max()), w["k"], w["eps"])


CASES = [(s, pm) for s in range(6) for pm in (0, 50, 300)]


@pytest.mark.parametrize("seed,permille", CASES)
def test_fm_trajectory_is_topgain(seed, permille):
    w = I.random_small(5100 + seed, n_max=120, k_max=4)
    pairs = [(a, b) for a in range(w["k"]) for b in range(a + 1, w["k"])][:3]
    for a, b in pairs:
        res = replay(w, a, b, max(permille, 1), seed * 7 + 1, _lmax(w))
        assert res["cut_after"] <= res["cut_before"] or res["kept"] > 0


def test_fm_overloaded_block_moves_first():
    """A start with block a far above L_max: TopGain empties the overload from a first
    (checked move by move by the replay), and the result is no worse in overload."""
    w = I.random_small(5200, n_max=150, k_max=2)
    part = np.array(w["part"], np.int32)
    xadj = np.asarray(w["xadj"])
    # move most of block 1 into block 0
    ones = np.flatnonzero(part == 1)
    part[ones[: max(1, 3 * len(ones) // 4)]] = 0
    w = dict(w, part=part)
    Lmax = _lmax(w)
    _, wA, wB = _pair_state(w, part, 0, 1)
    assert wA > Lmax
    res = replay(w, 0, 1, 1000, 11, Lmax)
    assert max(res["wA_after"], res["wB_after"]) - Lmax < wA - Lmax


def test_fm_never_worsens_a_feasible_pair():
    for s in range(8):
        w = I.random_small(5300 + s, n_max=200, k_max=3)
        Lmax = _lmax(w)
        st, out, res, _ = O.fm_pair(w, 0, 1, 50, seed=s, Lmax=Lmax)
        cut0, a0, b0 = _pair_state(w, np.asarray(w["part"]), 0, 1)
        if max(a0, b0) <= Lmax:
            assert res["cut_after"] <= cut0 and max(res["wA_after"], res["wB_after"]) <= Lmax
        # only vertices of the two blocks move, and only between them
        p0 = np.asarray(w["part"])
        ch = np.flatnonzero(out != p0)
        assert np.all(np.isin(p0[ch], (0, 1))) and np.all(np.isin(out[ch], (0, 1)))


def test_fm_on_a_grid_bisection_finds_the_straight_cut():
    """64 x 8 grid split at x < 32 with a dent: block a has taken the 4 x 4 square
    x in [32, 36), y in [0, 4).  Each square vertex next to a, and then the rest, has
    a move that keeps the cut from growing until the straight cut is back, and the
    straight cut of weight 8 is the unique minimum among feasible states reached."""
    xadj, adj, coords = I.grid2d(64, 8)
    n = 64 * 8
    part = (coords[:, 0] >= 32).astype(np.int32)
    sq = (coords[:, 0] >= 32) & (coords[:, 0] < 36) & (coords[:, 1] < 4)
    part[sq] = 0
    w = dict(n=n, nnz=len(adj), xadj=xadj, adjncy=adj, adjwgt=np.ones(len(adj), np.int32),
             vwgt=np.ones(n, np.int32), part=part, k=2, eps=0.1, alpha=1.0)
    cut0, _, _ = _pair_state(w, part, 0, 1)
    assert cut0 == 4 + 4 + 4   # 4 rows straight + the dent's top side (4) and right side (4)
    res = replay(w, 0, 1, 100, 5, _lmax(w))
    assert res["cut_after"] == 8


def test_pairwise_step_is_fm_then_flow():
    """With FM on, the oracle's pair refinement is FM followed by the flow step on
    FM's result (and with FM off the two coincide)."""
    for s in range(4):
        w = I.random_small(5400 + s, n_max=300, k_max=3)
        opts_fm = O.options(mb=1, seed=s, fm_permille=50)
        opts = O.options(mb=1, seed=s)
        st, p1, r1 = O.refine_pair(w, 0, 1, opts=opts_fm)
        _, pf, rf, _ = O.fm_pair(w, 0, 1, 50, seed=s)
        st2, p2, r2 = O.refine_pair(w, 0, 1, part=pf, opts=opts)
        r1, r2 = r1.as_dict(), r2.as_dict()
        assert st == st2 == 0 and np.array_equal(p1, p2)
        assert r1["cut_fm"] == rf["cut_after"] == r2["cut_before"] and r1["fm_moves"] == rf["kept"]
        assert r1["cut_after"] == r2["cut_after"] and r1["cut_before"] == rf["cut_before"]


def test_fm_option_range_is_checked():
    w = I.random_small(5500, n_max=100, k_max=3)
    for bad in (-1, 1001):
        st, _, _ = O.refine_pair(w, 0, 1, opts=O.options(fm_permille=bad))
        assert st == 1   # FRO_ERR_INVALID_ARG


@pytest.mark.parametrize("seed", range(12))
def test_fm_full_runs_replayed(seed):
    """permille = 1000: the search only stops when both queues are empty (every boundary
    vertex that can move has moved), on weighted graphs with zero vertex weights among
    them, and the replay still matches move by move."""
    w = I.random_small(5600 + seed, n_max=90, k_max=3)
    res = replay(w, 0, 1, 1000, 1000 + seed, _lmax(w))
    assert res["tried"] >= res["kept"]


def test_fm_empty_boundary_is_a_no_op():
    """Two blocks with no edge between them: no vertex is movable, nothing changes."""
    xadj, adj, coords = I.grid2d(8, 8)
    n = 64
    part = np.zeros(n, np.int32)
    part[coords[:, 0] >= 4] = 2                  # blocks 0 and 2 touch; block 1 holds one far corner
    part[0] = 1
    part[1] = 0
    w = dict(n=n, nnz=len(adj), xadj=xadj, adjncy=adj, adjwgt=np.ones(len(adj), np.int32),
             vwgt=np.ones(n, np.int32), part=part, k=3, eps=0.5, alpha=1.0)
    # block 1 = {0} is adjacent to 1 and 8 (block 0): pair (1, 2) has no cut edge
    st, out, res, moves = O.fm_pair(w, 1, 2, 1000, seed=0)
    assert st == 0 and res["tried"] == 0 and res["kept"] == 0 and np.array_equal(out, part)
