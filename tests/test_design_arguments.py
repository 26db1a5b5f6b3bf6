"""CPU checks of two arguments the CUDA path rests on, run against the oracle.

1. The multi-try kernel keeps its queue as gain buckets of LIFO stacks with versioned
   entries (a key change pushes a new entry, a pop bumps the version, stale entries are
   skipped).  Emulated here step for step, it must pop exactly what the oracle's binary
   heap keyed by (gain, keying time) pops: same partitions and totals.
2. The multilevel kernels compute the greedy matching with locally dominant rounds (free
   vertices point at their best allowed edge; mutual pointers match).  Emulated here, the
   rounds must end with the oracle's greedy matching.
The emulations recompute every gain from the graph; splitmix64 is written out from its
published definition."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1012_0006_gb300 import inputs as I

M64 = (1 << 64) - 1
G = 1023


def splitmix64(x):
    z = (x + 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def _arrays(w):
    return tuple(np.asarray(w[k]) for k in ("xadj", "adjncy", "adjwgt", "vwgt"))


def _best(w, part, u, tseed):
    xadj, adj, wg, _ = _arrays(w)
    conn, own = {}, 0
    for j in range(xadj[u], xadj[u + 1]):
        P = int(part[adj[j]])
        if P == part[u]:
            own += int(wg[j])
        else:
            conn[P] = conn.get(P, 0) + int(wg[j])
    if not conn:
        return None
    top = max(conn.values())
    t = min((P for P in conn if conn[P] == top), key=lambda P: (splitmix64(tseed ^ (u << 32) ^ P), P))
    return top - own, t


def bucket_pass(w, pairs, alpha, seed):
    """The multi-try pass as the kernel runs it: bucket stacks, versions, lazy deletion."""
    n, k = w["n"], w["k"]
    xadj, adj, wg, vw = _arrays(w)
    part = np.array(w["part"], np.int32)
    Lmax = O.lmax(int(vw.sum()), int(vw.max()), k, w["eps"])
    bw = np.bincount(part, weights=vw.astype(np.int64), minlength=k).astype(np.int64)
    tseed, beta = splitmix64(~seed & M64), math.log(n)
    blk = {}
    for i, (a, b) in enumerate(pairs):
        blk[a] = blk[b] = i
    lists = [[] for _ in pairs]
    for v in range(n):
        x = int(part[v])
        if x not in blk:
            continue
        a, b = pairs[blk[x]]
        other = b if x == a else a
        if (part[adj[xadj[v]:xadj[v + 1]]] == other).any():
            ms = splitmix64((splitmix64((seed ^ (a << 32) ^ b) & M64) + 1) & M64)
            lists[blk[x]].append((splitmix64(ms ^ v), v))
    for lst in lists:
        lst.sort()
    tch, ver, tgt = np.zeros(n, np.int64), np.zeros(n, np.int64), np.zeros(n, np.int64)
    moved = np.zeros(n, bool)
    tot = dict(gain=0, searches=0, tried=0, kept=0)
    sid = 0
    for j in range(max((len(l) for l in lists), default=0)):
        for p in range(len(pairs)):
            if j >= len(lists[p]):
                continue
            v = lists[p][j][1]
            if tch[v] or not (part[adj[xadj[v]:xadj[v + 1]]] != part[v]).any():
                continue
            sid += 1
            top, ent = {}, []

            def push(u, g):
                ver[u] += 1
                ent.append((u, ver[u], top.get(g + G, -1)))
                top[g + G] = len(ent) - 1

            for idx, u in enumerate([v] + [int(x) for x in adj[xadj[v]:xadj[v + 1]]]):
                if idx == 0 or tch[u] == 0:
                    r = _best(w, part, u, tseed)
                    if r is not None:
                        tgt[u], tch[u] = r[1], sid
                        push(u, r[0])
            delta = best = S1 = S2 = 0
            nm = best_len = pc = 0
            log = []
            while True:
                x = -1
                while True:
                    live = [bk for bk, e in top.items() if e >= 0]
                    if not live:
                        break
                    bk = max(live)
                    xv, ev, below = ent[top[bk]]
                    top[bk] = below
                    if ev == ver[xv]:
                        x, g = xv, bk - G
                        ver[xv] += 1
                        break
                if x < 0:
                    break
                to, fr = int(tgt[x]), int(part[x])
                if bw[to] + vw[x] > Lmax:
                    continue
                part[x] = to
                bw[fr] -= vw[x]
                bw[to] += vw[x]
                moved[x] = True
                log.append((x, fr))
                nm += 1
                delta -= g
                for u in adj[xadj[x]:xadj[x + 1]].tolist():
                    if moved[u] or not (tch[u] == 0 or tch[u] == sid):
                        continue
                    r = _best(w, part, u, tseed)
                    if r is None:
                        ver[u] += 1
                    else:
                        tgt[u], tch[u] = r[1], sid
                        push(u, r[0])
                if delta < best:
                    best, best_len, pc, S1, S2 = delta, nm, 0, 0, 0
                else:
                    pc, S1, S2 = pc + 1, S1 + g, S2 + g * g
                    if O.kaspar_stop(pc, S1, S2, alpha, beta):
                        break
            for y, fr in reversed(log[best_len:]):
                bw[part[y]] -= vw[y]
                bw[fr] += vw[y]
                part[y] = fr
            for y, _ in log:
                moved[y] = False
            tot["gain"] -= best
            tot["tried"] += nm
            tot["kept"] += best_len
            tot["searches"] += 1
    return part, tot


@pytest.mark.parametrize("seed", [15200, 15204, 15213, 15214, 15240, 7001, 7004, 7008])
def test_bucket_stacks_pop_in_heap_order(seed):
    w = I.random_small(seed, n_max=3000, k_max=8)
    pa, pb, pr, nr = O.rounds(w)
    pairs = [(int(a), int(b)) for a, b, c in zip(pa, pb, pr) if c == seed % max(nr, 1)]
    alpha = (1, 10, 0, 100)[seed % 4]
    part, tot = bucket_pass(w, pairs, alpha, seed)
    st, pref, tref, _ = O.multitry(w, pairs, alpha, seed=seed)
    assert st == 0 and np.array_equal(part, pref) and tot == tref


def locally_dominant(w, seed_l, W):
    n, k = w["n"], w["k"]
    xadj, adj, wg, vw = _arrays(w)
    part = np.asarray(w["part"])
    ok = [40 * k * int(c) <= 3 * W for c in vw]
    cc = [max(int(c), 1) for c in vw]

    def higher(x, y):   # (w2, cc, h, a, b)
        if x[0] * y[1] != y[0] * x[1]:
            return x[0] * y[1] > y[0] * x[1]
        if x[2] != y[2]:
            return x[2] > y[2]
        return (x[3], x[4]) < (y[3], y[4])

    mate = np.full(n, -1)
    rounds = 0
    while True:
        rounds += 1
        cand = np.full(n, -1)
        for v in range(n):
            if mate[v] != -1 or not ok[v]:
                if mate[v] == -1:
                    mate[v] = -2
                continue
            best = None
            for j in range(xadj[v], xadj[v + 1]):
                u = int(adj[j])
                if mate[u] != -1 or part[u] != part[v] or not ok[u]:
                    continue
                a, b = min(u, v), max(u, v)
                key = (int(wg[j]) ** 2, cc[a] * cc[b], splitmix64(seed_l ^ (a << 32) ^ b), a, b)
                if best is None or higher(key, best[0]):
                    best = (key, u)
            if best is None:
                mate[v] = -2
            else:
                cand[v] = best[1]
        progress = False
        for v in range(n):
            u = cand[v]
            if u > v and cand[u] == v:
                mate[v], mate[u] = u, v
                progress = True
        if not progress:
            break
    mate[mate == -2] = -1
    return mate, rounds


@pytest.mark.parametrize("seed", [15200, 15204, 15213, 15214, 15240, 15246])
def test_locally_dominant_rounds_give_the_greedy_matching(seed):
    w = I.random_small(seed, n_max=3000, k_max=5)
    W = int(np.asarray(w["vwgt"], np.int64).sum())
    for seed_l in (0, splitmix64(seed)):
        mate, rounds = locally_dominant(w, seed_l, W)
        pairs, mref = O.match(w, seed_l=seed_l, W=W)
        assert np.array_equal(mate, mref) and rounds <= w["n"] + 1
