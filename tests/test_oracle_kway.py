"""Pins of the oracle's k-way local search with the KaSPar stopping rule and of its
multi-try FM pass (Section 2.2, k-way local search; Section 4.2, multi-try FM;
Section 6, "Configuring the Algorithm", for alpha = 10 and the global rounds).

The oracle keeps its queue in a binary heap with incremental gain updates.  The
replay below rebuilds every step from the graph alone: the queue is the set of
unmoved vertices of the start set or next to a moved vertex that are boundary
vertices now, each remembering when it was last keyed; at every move it recomputes
all gains and targets from scratch, checks that the moved vertex is the queue's
best by (gain, last keying) after dropping the vertices whose move would exceed
L_max, checks the target (largest connection weight, splitmix64 tie written out
here from its published definition), the recorded gain against the cut recomputed
from scratch, the KaSPar rule in exact rational arithmetic and the rollback to the
first lowest-cut prefix.  Closed forms: constant gains stop after floor(beta/g^2)+1
moves; zero-mean walks never stop; a quadrant partition of a grid with isolated
bumps returns to the straight cut.
"""
import math
from fractions import Fraction

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


def kaspar_exact(p, S1, S2, alpha, beta):
    """p mu^2 > alpha sigma^2 + beta in exact rationals; returns (decision, |margin| small?)."""
    mu = Fraction(S1, p)
    var = Fraction(S2, p) - mu * mu
    lhs = p * mu * mu
    rhs = alpha * var + Fraction(beta)
    near = abs(lhs - rhs) <= Fraction(1, 10 ** 9) * (abs(lhs) + abs(rhs) + 1)
    return lhs > rhs, near


# ------------------------------------------------------------- KaSPar rule --

def test_kaspar_rule_against_exact_arithmetic():
    rs = np.random.default_rng(7)
    checked = 0
    for _ in range(4000):
        p = int(rs.integers(1, 80))
        g = rs.integers(-12, 6, size=p)
        S1, S2 = int(g.sum()), int((g * g).sum())
        alpha = int(rs.choice([0, 1, 3, 10, 50]))
        beta = math.log(int(rs.integers(2, 1 << 24)))
        want, near = kaspar_exact(p, S1, S2, alpha, beta)
        if near:
            continue
        assert O.kaspar_stop(p, S1, S2, alpha, beta) == int(want), (p, S1, S2, alpha, beta)
        checked += 1
    assert checked > 3900


def kaspar_doubles(p, S1, S2, alpha, beta, order="paper"):
    """The rule as both sides take it (a floating-point decision on an integer outcome):
    every step one IEEE double operation rounded to nearest, in this order --
    mu = S1 / p, sigma^2 = S2 / p - mu * mu, lhs = (p * mu) * mu, rhs = alpha * sigma^2 +
    beta.  Python floats are IEEE doubles and round every operation (no fused
    multiply-add).  order="pmm" and "ss" are two other plausible orders of the left
    side, p * (mu * mu) and S1 * S1 / p, used to show the test tells orders apart."""
    pd = float(p)
    mu = float(S1) / pd
    var = float(S2) / pd - mu * mu
    if order == "paper":
        lhs = (pd * mu) * mu
    elif order == "pmm":
        lhs = pd * (mu * mu)
    else:
        lhs = float(S1) * float(S1) / pd
    rhs = float(alpha) * var + beta
    return lhs > rhs


def test_kaspar_rule_ties_by_hand():
    """Constant gains g over p moves: mu = g and sigma^2 = 0 exactly in doubles, so the
    rule is p g^2 > beta with no rounding at all; at beta = p g^2 the strict inequality
    does not stop, one ulp below it does."""
    for p, g in ((4, -3), (7, 2), (25, -1), (3, -5)):
        lhs = float(p * g * g)
        for alpha in (0, 10):
            assert O.kaspar_stop(p, p * g, p * g * g, alpha, lhs) == 0
            assert O.kaspar_stop(p, p * g, p * g * g, alpha, math.nextafter(lhs, -math.inf)) == 1
            assert O.kaspar_stop(p, p * g, p * g * g, alpha, math.nextafter(lhs, math.inf)) == 0


def test_kaspar_rule_within_the_rounding_band():
    """Inputs built to land within a few ulps of the threshold, where exact arithmetic
    and doubles can disagree: the oracle follows the documented double operations on
    every one.  The band is really reached (exact and double decisions differ on some),
    and the other two orders of the left side disagree with the documented one on some,
    so a change of order would fail here."""
    rs = np.random.default_rng(11)
    n_cases = band = other = 0
    for _ in range(3000):
        p = int(rs.integers(2, 200))
        g = rs.integers(-15, 6, size=p)
        S1, S2 = int(g.sum()), int((g * g).sum())
        alpha = int(rs.choice([0, 1, 3, 10, 50]))
        pd = float(p)
        mu = float(S1) / pd
        var = float(S2) / pd - mu * mu
        beta0 = (pd * mu) * mu - float(alpha) * var
        if not beta0 > 0:
            continue
        b = beta0
        for _ in range(3):
            b = math.nextafter(b, -math.inf)
        for _ in range(7):
            want = kaspar_doubles(p, S1, S2, alpha, b)
            assert O.kaspar_stop(p, S1, S2, alpha, b) == int(want), (p, S1, S2, alpha, b)
            band += kaspar_exact(p, S1, S2, alpha, b)[0] != want
            other += any(kaspar_doubles(p, S1, S2, alpha, b, o) != want for o in ("pmm", "ss"))
            n_cases += 1
            b = math.nextafter(b, math.inf)
    assert n_cases > 10000
    assert band > 100 and other > 100


@pytest.mark.parametrize("g", [-1, -2, -3, -5, 4])
@pytest.mark.parametrize("n", [10, 1000, 4194304])
def test_kaspar_constant_gains_closed_form(g, n):
    # sigma^2 = 0: the walk stops at the first p with p g^2 > ln n
    beta = math.log(n)
    first = next(p for p in range(1, 10 ** 4) if O.kaspar_stop(p, p * g, p * g * g, 10, beta))
    assert first == math.floor(beta / (g * g)) + 1


def test_kaspar_zero_mean_never_stops():
    for p in range(2, 400, 2):   # alternating +-3: mu = 0
        assert O.kaspar_stop(p, 0, 9 * p, 10, math.log(1 << 20)) == 0
        assert O.kaspar_stop(p, 0, 9 * p, 0, math.log(2)) == 0


# ------------------------------------------------------- k-way search replay --

def _arrays(w):
    return tuple(np.asarray(w[k]) for k in ("xadj", "adjncy", "adjwgt", "vwgt"))


def _total_cut(w, part):
    xadj, adj, wg, _ = _arrays(w)
    src = np.repeat(np.arange(w["n"]), np.diff(xadj))
    return int(wg[part[src] != part[adj]].sum()) // 2


def _best_move(w, part, u, tseed):
    """(gain, target) of u from scratch, or None if u has no neighbour in another block."""
    u = int(u)
    xadj, adj, wg, _ = _arrays(w)
    conn = {}
    own = 0
    for j in range(xadj[u], xadj[u + 1]):
        P = int(part[adj[j]])
        if P == part[u]:
            own += int(wg[j])
        else:
            conn[P] = conn.get(P, 0) + int(wg[j])
    if not conn:
        return None
    top = max(conn.values())
    ties = [P for P in conn if conn[P] == top]
    t = min(ties, key=lambda P: (splitmix64(tseed ^ (u << 32) ^ P), P))
    return top - own, t


def replay_search(w, init, alpha, tseed, Lmax):
    n, k = w["n"], w["k"]
    xadj, adj, wg, vw = _arrays(w)
    part0 = np.array(w["part"], np.int32)
    st, part_out, bw_out, res, (lv, lt, lg) = O.kway_search(w, init, alpha, tseed=tseed, Lmax=Lmax)
    assert st == 0
    beta = math.log(n)
    part = part0.copy()
    bw = np.bincount(part, weights=vw.astype(np.int64), minlength=k).astype(np.int64)
    moved = np.zeros(n, bool)
    keyed = {}   # vertex -> (step, position) of its last keying
    for pos, v in enumerate(np.asarray(init).tolist()):
        if v not in keyed and _best_move(w, part, v, tseed) is not None:
            keyed[v] = (-1, pos)
    cut0 = cut = _total_cut(w, part)
    cuts = [cut]
    best, p, S1, S2 = cut, 0, 0, 0
    stopped_by_rule = False
    for i, (v, t, g) in enumerate(zip(lv.tolist(), lt.tolist(), lg.tolist())):
        assert not stopped_by_rule, "moved after the KaSPar rule held"
        # pop the queue's best; drop vertices whose move would overload the target
        while True:
            assert keyed, "moved with an empty queue"
            gains = {u: _best_move(w, part, u, tseed) for u in keyed}
            u = max(keyed, key=lambda x: (gains[x][0], keyed[x]))
            gu, tu = gains[u]
            del keyed[u]
            if bw[tu] + vw[u] <= Lmax:
                break
        assert (u, tu, gu) == (v, t, g), f"move {i}"
        assert not moved[v]
        src = part[v]
        part[v] = t
        bw[src] -= vw[v]
        bw[t] += vw[v]
        moved[v] = True
        new_cut = _total_cut(w, part)
        assert new_cut == cut - g, "recorded gain is not the cut change"
        cut = new_cut
        cuts.append(cut)
        for j in range(xadj[v], xadj[v + 1]):
            x = int(adj[j])
            if moved[x]:
                continue
            if _best_move(w, part, x, tseed) is not None:
                keyed[x] = (i, j - xadj[v])
            else:
                keyed.pop(x, None)
        if cut < best:
            best, p, S1, S2 = cut, 0, 0, 0
        else:
            p, S1, S2 = p + 1, S1 + g, S2 + g * g
            want, near = kaspar_exact(p, S1, S2, alpha, beta)
            if not near:
                stopped_by_rule = want
            else:
                stopped_by_rule = bool(res["stop"]) and i == len(lv) - 1
    assert res["stop"] == int(stopped_by_rule)
    if not res["stop"]:
        # the queue ran empty: whatever is left may not move
        for u in keyed:
            gu, tu = _best_move(w, part, u, tseed)
            assert bw[tu] + vw[u] > Lmax
    kept = int(np.argmin(cuts))
    assert res["kept"] == kept and res["tried"] == len(lv)
    assert res["gain"] == cut0 - cuts[kept]
    want_part = part0.copy()
    for v, t in zip(lv[:kept].tolist(), lt[:kept].tolist()):
        want_part[v] = t
    assert np.array_equal(part_out, want_part)
    assert np.array_equal(bw_out, np.bincount(want_part, weights=vw.astype(np.int64), minlength=k))
    return res


def _boundary(w, part):
    xadj, adj, _, _ = _arrays(w)
    src = np.repeat(np.arange(w["n"]), np.diff(xadj))
    return np.unique(src[part[src] != part[adj]])


@pytest.mark.parametrize("seed", range(12))
def test_kway_search_replay(seed):
    w = I.random_small(9100 + seed, n_max=260, k_max=6)
    rs = np.random.default_rng(seed)
    part = np.asarray(w["part"])
    init = rs.permutation(_boundary(w, part)).astype(np.int32)
    W = int(np.asarray(w["vwgt"]).sum())
    tight = O.lmax(W, int(np.max(w["vwgt"])), w["k"], w["eps"])
    for Lmax in (tight, 10 * W):
        for alpha in (0, 10, 10 ** 6):
            tseed = splitmix64(seed * 31 + alpha)
            replay_search(w, init, alpha, tseed, Lmax)


def test_kway_search_small_start_sets_and_tight_balance():
    # a start set of one vertex and its neighbours, as multi-try uses, with L_max at the
    # current heaviest block (many moves refused)
    for seed in range(6):
        w = I.random_small(9300 + seed, n_max=200, k_max=5)
        part = np.asarray(w["part"])
        b = _boundary(w, part)
        xadj, adj, _, vw = _arrays(w)
        heaviest = int(np.bincount(part, weights=vw.astype(np.int64), minlength=w["k"]).max())
        for v in b[:: max(1, len(b) // 5)].tolist():
            init = [v] + [int(u) for u in adj[xadj[v]:xadj[v + 1]] if u in set(b.tolist())]
            replay_search(w, np.asarray(init, np.int32), 10, splitmix64(v), heaviest)


def test_kway_search_argument_checks():
    w = I.random_small(9400, n_max=60)
    st, *_ = O.kway_search(w, np.asarray([w["n"]], np.int32), 10)
    assert st == 1
    st, *_ = O.kway_search(w, np.asarray([0], np.int32), -1)
    assert st == 1


# ------------------------------------------------------- multi-try FM pass --

def multitry_replay(w, pairs, alpha, seed):
    """The multi-try pass as Section 4.2 describes it, written out here with the
    oracle's single k-way search (pinned above) as the search step."""
    n, k = w["n"], w["k"]
    xadj, adj, _, vw = _arrays(w)
    part = np.array(w["part"], np.int32)
    W = int(vw.sum())
    Lmax = O.lmax(W, int(vw.max()), k, w["eps"])
    bw = np.bincount(part, weights=vw.astype(np.int64), minlength=k).astype(np.int64)
    tseed = splitmix64(~seed & M64)

    def boundary(v):
        return bool((part[adj[xadj[v]:xadj[v + 1]]] != part[v]).any())

    todo = []
    for a, b in pairs:
        ms = splitmix64((splitmix64((seed ^ (a << 32) ^ b) & M64) + 1) & M64)
        lst = [v for v in range(n) if part[v] in (a, b)
               and (part[adj[xadj[v]:xadj[v + 1]]] == (b if part[v] == a else a)).any()]
        lst.sort(key=lambda v: (splitmix64(ms ^ v), v))
        todo.append(lst)
    touched = np.zeros(n, np.int32)
    tot = dict(gain=0, searches=0, tried=0, kept=0)
    changed = np.zeros(k, bool)
    sid = 0
    for j in range(max((len(t) for t in todo), default=0)):
        for lst in todo:
            if j >= len(lst):
                continue
            v = lst[j]
            if touched[v] or not boundary(v):
                continue
            init = [v] + [int(u) for u in adj[xadj[v]:xadj[v + 1]] if not touched[u] and boundary(int(u))]
            sid += 1
            before = part.copy()
            st, part, bw, r, _ = O.kway_search(w, np.asarray(init, np.int32), alpha, beta=math.log(n), tseed=tseed,
                                               part=part, blockw=bw, Lmax=Lmax, touched=touched, sid=sid)
            assert st == 0
            tot["gain"] += r["gain"]
            tot["searches"] += 1
            tot["tried"] += r["tried"]
            tot["kept"] += r["kept"]
            d = before != part
            changed[before[d]] = True
            changed[part[d]] = True
    return part, tot, changed


@pytest.mark.parametrize("seed", range(10))
def test_multitry_pass_replay(seed):
    w = I.random_small(9500 + seed, n_max=300, k_max=7)
    pa, pb, pr, nr = O.rounds(w)
    r = seed % max(nr, 1)
    pairs = [(int(a), int(b)) for a, b, c in zip(pa, pb, pr) if c == r]
    for alpha in (1, 10):
        st, part, tot, changed = O.multitry(w, pairs, alpha, seed=seed)
        assert st == 0
        want_part, want_tot, want_changed = multitry_replay(w, pairs, alpha, seed)
        assert np.array_equal(part, want_part)
        assert tot == want_tot
        assert np.array_equal(changed, want_changed)
        assert _total_cut(w, np.asarray(w["part"])) - _total_cut(w, part) == tot["gain"] >= 0
        vw = np.asarray(w["vwgt"], np.int64)
        W = int(vw.sum())
        Lmax = O.lmax(W, int(vw.max()), w["k"], w["eps"])
        before = np.bincount(np.asarray(w["part"]), weights=vw, minlength=w["k"])
        after = np.bincount(part, weights=vw, minlength=w["k"])
        assert (after <= np.maximum(before, Lmax)).all()


def _quadrants_with_bumps(R=16):
    xadj, adj, coords = I.grid2d(R, R)
    n = R * R
    x, y = coords[:, 0].astype(int), coords[:, 1].astype(int)
    h = R // 2
    part = (2 * (y >= h) + (x >= h)).astype(np.int32)
    # isolated single-vertex bumps across the vertical line, two per half, away from the centre
    for yy in (2, 5, h + 2, h + 5):
        v = int(np.flatnonzero((x == h - 1) & (y == yy))[0])
        part[v] = part[v] + 1
    w = dict(name="quadrants", n=n, nnz=len(adj), xadj=xadj, adjncy=adj, adjwgt=np.ones(len(adj), np.int32),
             vwgt=np.ones(n, np.int32), part=part, k=4, eps=0.03)
    return w, 2 * R


def test_quadrant_bumps_return_to_the_straight_cut():
    w, straight = _quadrants_with_bumps()
    assert _total_cut(w, w["part"]) == straight + 2 * 4
    st, part, tot, rounds = O.kway_global(w, alpha=10, init_mode=0, max_rounds=10, seed=3)
    assert st == 0 and _total_cut(w, part) == straight and tot["gain"] == 8
    assert rounds == 2   # one round that improves, one that does not
    # multi-try from the two pairs across the vertical line: a search that queues a bump
    # but rolls back leaves it touched, so no later search of the pass may move it; the
    # pass only guarantees its bookkeeping (cut = start - gain, gains in steps of 2 here)
    st, part, tot, changed = O.multitry(w, [(0, 1), (2, 3)], 10, seed=5)
    assert st == 0 and _total_cut(w, part) == straight + 8 - tot["gain"] and tot["gain"] % 2 == 0
    assert tot["searches"] >= 2


def test_corner_start_set():
    # k = 2: no vertex meets three blocks, so the corner start set is empty
    w = I.grid2d_halves(nx=16, ny=16, swaps=20)
    st, part, tot, rounds = O.kway_global(w, init_mode=1)
    assert st == 0 and rounds == 1 and tot["gain"] == 0 and np.array_equal(part, w["part"])
    # quadrants: only the vertices at the centre meet three blocks; the bumps are not
    # corners, so the corner start set cannot remove them
    w, straight = _quadrants_with_bumps()
    st, part, tot, rounds = O.kway_global(w, init_mode=1, seed=1)
    assert st == 0 and _total_cut(w, part) > straight


def test_kway_global_replays_as_rounds_of_searches():
    w = I.random_small(9700, n_max=300, k_max=6)
    st, part, tot, rounds = O.kway_global(w, alpha=10, init_mode=0, max_rounds=4, seed=11)
    assert st == 0
    # the same rounds from single searches: whole boundary, splitmix64 order of round r
    cur = np.array(w["part"], np.int32)
    gain = 0
    vw = np.asarray(w["vwgt"])
    Lmax = O.lmax(int(vw.sum()), int(vw.max()), w["k"], w["eps"])
    r = 0
    while r < 4:
        rsd = splitmix64(11 ^ r)
        init = sorted(_boundary(w, cur).tolist(), key=lambda v: (splitmix64(rsd ^ v), v))
        _, cur, _, res, _ = O.kway_search(w, np.asarray(init, np.int32), 10, tseed=splitmix64(~11 & M64), part=cur,
                                          Lmax=Lmax)
        gain += res["gain"]
        r += 1
        if res["gain"] == 0:
            break
    assert rounds == r and tot["gain"] == gain and np.array_equal(part, cur)


# --------------------------------------------- inside active block scheduling --

@pytest.mark.parametrize("seed", range(4))
def test_active_scheduling_with_multitry_bookkeeping(seed):
    w = I.random_small(9800 + seed, n_max=300, k_max=6)
    mt = {}
    opts = O.options(mb=1, seed=seed, mt_alpha=10)
    st, part, res, nouter = O.refine_active(w, opts=opts, max_outer=6, mt_out=mt)
    assert st == 0
    pair_gain = sum(r["cut_before"] - r["cut_after"] for r in res)
    assert _total_cut(w, np.asarray(w["part"])) - _total_cut(w, part) == pair_gain + mt["gain"]
    assert mt["searches"] > 0 and mt["gain"] >= 0
    # without the pass: the earlier behaviour
    st0, part0, res0, _ = O.refine_active(w, opts=O.options(mb=1, seed=seed), max_outer=6, mt_out=mt)
    assert st0 == 0 and mt["searches"] == 0


def test_multitry_option_checks():
    w = I.random_small(9900, n_max=80)
    st, *_ = O.refine_active(w, opts=O.options(mt_alpha=-1), max_outer=2)
    assert st == 1
    st, *_ = O.refine_batch(w, opts=O.options(mt_alpha=10))
    assert st == 1
    st, *_ = O.refine_pair(w, opts=O.options(mt_alpha=10))
    assert st == 1
