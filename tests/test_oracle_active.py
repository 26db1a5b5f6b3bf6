"""Pins of the oracle's active block scheduling (Section 4.3 and the appendix
pseudocode, pairwise step = flow refinement of Section 4.1).

The schedule is checked against what the pseudocode fixes, recomputed here from
the partitions the run passes through: every outer round refines exactly the
quotient edges of the partition at its start that have an active end, in the
matching order of the rounds; a block is active in the next outer round iff a
refinement of one of its pairs changed the partition; the run ends when no block
is active.  The refinements themselves are pinned by replaying them one by one
with fro_refine_pair (pinned elsewhere), and the first outer round with every
block active is the already pinned one-sweep batch."""
import numpy as np
import pytest

import oracle as O
from paper_1012_0006_gb300 import inputs as I


def _quotient_edges(w, part):
    k = w["k"]
    xadj, adj = np.asarray(w["xadj"]), np.asarray(w["adjncy"])
    src = np.repeat(np.arange(w["n"]), np.diff(xadj))
    pa, pb = part[src], part[adj]
    m = pa < pb
    return sorted(set(zip(pa[m].tolist(), pb[m].tolist())))


def _matching_order(edges):
    """Greedy colouring in lexicographic order (the rounds' rule), then edges by colour."""
    used, col = {}, {}
    for a, b in edges:
        c = 0
        while c in used.get(a, ()) or c in used.get(b, ()):
            c += 1
        used.setdefault(a, set()).add(c)
        used.setdefault(b, set()).add(c)
        col[(a, b)] = c
    return sorted(edges, key=lambda e: (col[e], e))


CASES = [
    ("grid2d-64", lambda: I.config(1), dict(mb=0)),
    ("rgg2d-4096", lambda: I.config(2, scale=1 / 16), dict(mb=1)),
    ("grid3d-32", lambda: I.config(3, scale=1 / 64), dict(mb=1, mb_reps=2, seed=5)),
    ("small-adaptive-a", lambda: I.random_small(4100, n_max=3000, k_max=8),
     dict(mb=1, adaptive=1, max_iters=6, alpha_max=8.0)),
    ("small-adaptive-b", lambda: I.random_small(4101, n_max=3000, k_max=8),
     dict(mb=0, adaptive=1, max_iters=4, alpha_max=4.0)),
    ("small-c", lambda: I.random_small(4102, n_max=3000, k_max=8), dict(mb=1)),
]


@pytest.mark.parametrize("name,make,okw", CASES, ids=[c[0] for c in CASES])
def test_schedule_replay_and_termination(name, make, okw):
    w = make()
    max_outer = 12
    st, final, res, nouter = O.refine_active(w, opts=O.options(**okw), max_outer=max_outer)
    assert st == 0
    part = np.array(w["part"], np.int32)
    active = set(range(w["k"]))
    i = 0
    for outer in range(nouter):
        assert active, "an outer round ran with no active block"
        expect = _matching_order([(a, b) for a, b in _quotient_edges(w, part) if a in active or b in active])
        nxt = set()
        for a, b in expect:
            r = res[i]
            assert (r["a"], r["b"]) == (a, b), (outer, i)
            cut0 = sum(O.pair_cut(w, part, x, y) for x, y in _quotient_edges(w, part))
            st2, part2, rr = O.refine_pair(w, a, b, part=part, opts=O.options(**okw))
            assert st2 == 0
            assert rr.accepted == r["accepted"] and rr.cut_after == r["cut_after"] and rr.iters == r["iters"]
            assert bool(r["accepted"]) == (not np.array_equal(part, part2))
            cut1 = sum(O.pair_cut(w, part2, x, y) for x, y in _quotient_edges(w, part2))
            assert cut1 <= cut0                       # the total cut never grows
            if r["accepted"]:
                nxt |= {a, b}
            part = part2
            i += 1
        active = nxt
    assert i == len(res)
    assert np.array_equal(part, final)
    # ended because no block is active, or at the cap
    assert not active or nouter == max_outer


def test_first_outer_round_is_the_batch():
    for seed in range(5):
        w = I.random_small(4200 + seed, n_max=2500, k_max=8)
        opts = O.options(mb=seed % 2, mb_reps=1 + seed % 2, seed=seed)
        st, p1, r1, nouter = O.refine_active(w, opts=opts, max_outer=1)
        st2, p2, r2, _ = O.refine_batch(w, opts=opts)
        assert st == st2 == 0 and nouter == 1
        assert np.array_equal(p1, p2)
        assert [(r["a"], r["b"], r["round"], r["accepted"], r["cut_after"]) for r in r1] == \
               [(r["a"], r["b"], r["round"], r["accepted"], r["cut_after"]) for r in r2]


@pytest.mark.parametrize("nthreads", [1, 3, 8])
def test_pair_parallel_sweep_is_the_sequential_sweep(nthreads):
    """The pairs of a round are a matching (disjoint blocks), so refining them side
    by side on copies of the round's starting partition must give the sequential
    sweep exactly: same partition, same per-pair results in the same order."""
    cases = [I.random_small(4300 + s, n_max=2500, k_max=8) for s in range(4)] + [I.config(3, scale=1 / 64)]
    for i, w in enumerate(cases):
        opts = O.options(mb=i % 2, mb_reps=1 + i % 2, seed=i, adaptive=i % 3 == 2, max_iters=4,
                         alpha_max=8.0)
        st, p1, r1, nr1 = O.refine_batch(w, opts=opts)
        st2, p2, r2, nr2, done = O.refine_batch_mt(w, nthreads, opts=opts)
        assert st == st2 == 0 and nr1 == nr2 and done == len(r1)
        assert np.array_equal(p1, p2)
        assert r1 == r2


def test_pair_parallel_sweep_stops_after_max_rounds():
    w = I.config(3, scale=1 / 64)
    opts = O.options(mb=1)
    pa, pb, pr, nr = O.rounds(w)
    assert nr >= 2
    st, part, res, nr2, done = O.refine_batch_mt(w, 4, max_rounds=1, opts=opts)
    assert st == 0 and nr2 == nr and done == int((pr == 0).sum())
    assert all(r["round"] == 0 for r in res)
    _, pseq, rseq, _ = O.refine_batch(w, opts=opts)
    assert res == rseq[:done]


def _colours(edges):
    used, col = {}, {}
    for a, b in edges:
        c = 0
        while c in used.get(a, ()) or c in used.get(b, ()):
            c += 1
        used.setdefault(a, set()).add(c)
        used.setdefault(b, set()).add(c)
        col[(a, b)] = c
    return col


@pytest.mark.parametrize("seed", range(4))
def test_schedule_with_multitry_replay(seed):
    """Active scheduling with a multi-try pass after every matching (Section 4.3), rebuilt
    from pinned pieces: fro_refine_pair for each pair of a matching, then fro_multitry on
    the matching's pairs; blocks a kept multi-try move touched become active."""
    w = I.random_small(4400 + seed, n_max=2500, k_max=7)
    okw = dict(mb=seed % 2, seed=seed, fm_permille=(0, 50)[seed % 2])
    mt = {}
    max_outer = 6
    st, final, res, nouter = O.refine_active(w, opts=O.options(mt_alpha=10, **okw), max_outer=max_outer, mt_out=mt)
    assert st == 0
    vw = np.asarray(w["vwgt"])
    Lmax = O.lmax(int(vw.sum()), int(vw.max()), w["k"], w["eps"])
    part = np.array(w["part"], np.int32)
    active = set(range(w["k"]))
    i, gain, searches = 0, 0, 0
    for outer in range(nouter):
        edges = [(a, b) for a, b in _quotient_edges(w, part) if a in active or b in active]
        col = _colours(edges)
        nxt = set()
        for c in sorted(set(col.values())):
            group = sorted(e for e in edges if col[e] == c)
            for a, b in group:
                r = res[i]
                assert (r["a"], r["b"]) == (a, b)
                st2, part, rr = O.refine_pair(w, a, b, part=part, opts=O.options(**okw))
                assert st2 == 0 and rr.cut_after == r["cut_after"]
                if rr.accepted or rr.fm_moves > 0:
                    nxt |= {a, b}
                i += 1
            st3, part, tot, changed = O.multitry(dict(w, part=part), group, 10, seed=seed, Lmax=Lmax)
            assert st3 == 0
            nxt |= set(np.flatnonzero(changed).tolist())
            gain += tot["gain"]
            searches += tot["searches"]
        active = nxt
    assert i == len(res) and np.array_equal(part, final)
    assert (gain, searches) == (mt["gain"], mt["searches"])
    assert not active or nouter == max_outer
