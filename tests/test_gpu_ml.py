"""The multilevel V-cycle on the CUDA path against the oracle: the greedy matching
(locally dominant rounds on the device), the contraction (coarse ids, merged rows,
weights), and whole V-cycles with a sweep or active scheduling on every level.
Integers throughout: bit-exact."""
import numpy as np
import pytest

import oracle as O
from paper_1012_0006_gb300 import inputs as I

pytestmark = pytest.mark.gpu


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


def _W(w):
    return int(np.asarray(w["vwgt"], np.int64).sum())


@pytest.mark.parametrize("seed", range(12))
def test_match_random_small(F, ctx, seed):
    w = I.random_small(14000 + seed, n_max=3000, k_max=6)
    g, part = _dev(F, w)
    for seed_l in (0, 0x9E3779B97F4A7C15 ^ seed):
        pref, mref = O.match(w, seed_l=seed_l)
        st, pairs, mate = ctx.match(g, part, w["k"], _W(w), seed_l)
        assert pairs == pref
        assert np.array_equal(mate.cpu().numpy(), mref)


@pytest.mark.parametrize("cfg,scale", [(1, 1.0), (2, 1 / 16), (4, 1 / 64), (4, 1 / 16)])
def test_match_and_contract_workloads(F, ctx, cfg, scale):
    import torch
    w = I.config(cfg, scale=scale)
    g, part = _dev(F, w)
    pref, mref = O.match(w, seed_l=17)
    st, pairs, mate = ctx.match(g, part, w["k"], _W(w), 17)
    assert pairs == pref and np.array_equal(mate.cpu().numpy(), mref)
    cref_map, cref = O.contract(w, mref)
    st, cmap, c = ctx.contract(g, mate)
    assert np.array_equal(cmap, cref_map)
    for f in ("n", "nnz", "xadj", "adjncy", "adjwgt", "vwgt"):
        assert np.array_equal(np.asarray(c[f]), np.asarray(cref[f])), f


@pytest.mark.parametrize("seed", range(8))
def test_contract_random_small(F, ctx, seed):
    import torch
    w = I.random_small(14100 + seed, n_max=3000, k_max=5)
    g, _ = _dev(F, w)
    _, mref = O.match(w, seed_l=seed)
    cref_map, cref = O.contract(w, mref)
    st, cmap, c = ctx.contract(g, torch.as_tensor(mref).cuda())
    assert np.array_equal(cmap, cref_map)
    for f in ("n", "nnz", "xadj", "adjncy", "adjwgt", "vwgt"):
        assert np.array_equal(np.asarray(c[f]), np.asarray(cref[f])), f


def test_contract_long_row(F, ctx):
    """A coarse row longer than the shared-memory sort (a hub of 3,000 leaves, leaves
    joined in pairs): the selection path builds it."""
    import torch
    leaves = 3000
    n = leaves + 1
    rows = [list(range(1, n))] + [[0] for _ in range(leaves)]
    for i in range(1, n - 1, 2):   # leaf i - leaf i+1
        rows[i].append(i + 1)
        rows[i + 1].append(i)
    xadj = np.zeros(n + 1, np.int32)
    xadj[1:] = np.cumsum([len(r) for r in rows])
    adj = np.concatenate([sorted(r) for r in rows]).astype(np.int32)
    src = np.repeat(np.arange(n), np.diff(xadj))
    w = dict(n=n, xadj=xadj, adjncy=adj, adjwgt=(1 + (src + adj) % 7).astype(np.int32),   # symmetric weights
             vwgt=np.ones(n, np.int32), part=np.zeros(n, np.int32), k=2, eps=0.03)
    mate = np.full(n, -1, np.int32)
    mate[0], mate[1] = 1, 0                       # the hub with leaf 1
    for i in range(3, n - 1, 2):                  # leaves (3,4), (5,6), ...
        mate[i], mate[i + 1] = i + 1, i
    cref_map, cref = O.contract(w, mate)
    g, _ = _dev(F, w)
    st, cmap, c = ctx.contract(g, torch.as_tensor(mate).cuda())
    assert int(np.diff(cref["xadj"]).max()) > 1024
    assert np.array_equal(cmap, cref_map)
    for f in ("n", "nnz", "xadj", "adjncy", "adjwgt", "vwgt"):
        assert np.array_equal(np.asarray(c[f]), np.asarray(cref[f])), f


def _vcycle(F, ctx, w, okw, max_levels=64, active_outer=0):
    st, pref, rref = O.vcycle(w, opts=O.options(**okw), max_levels=max_levels, active_outer=active_outer)
    assert st == 0
    g, part = _dev(F, w)
    st, r = ctx.vcycle(g, part, w["k"], w["eps"], w["alpha"], F.default_options(**okw), max_levels=max_levels,
                       active_outer=active_outer)
    for f in ("levels", "cut_before", "cut_after", "level_n", "level_pairs", "level_cut"):
        assert r[f] == rref[f], f
    assert np.array_equal(part.cpu().numpy(), pref)
    return r


@pytest.mark.parametrize("seed", range(8))
def test_vcycle_random_small(F, ctx, seed):
    w = I.random_small(14200 + seed, n_max=3000, k_max=6)
    okw = dict(mb=seed % 2, seed=seed)
    _vcycle(F, ctx, w, okw)
    _vcycle(F, ctx, w, okw, max_levels=2)


@pytest.mark.parametrize("cfg,scale", [(2, 1 / 16), (4, 1 / 64)])
def test_vcycle_workloads(F, ctx, cfg, scale):
    w = I.config(cfg, scale=scale)
    r = _vcycle(F, ctx, w, dict(mb=1, seed=3))
    assert r["levels"] > 1 and r["cut_after"] < r["cut_before"]


def test_vcycle_active_fm_multitry(F, ctx):
    w = I.random_small(14300, n_max=2500, k_max=6)
    _vcycle(F, ctx, w, dict(mb=1, fm_permille=50, mt_alpha=10, seed=5), active_outer=3)


def test_vcycle_checks(F, ctx):
    w = I.random_small(14400, n_max=300, k_max=4)
    g, part = _dev(F, w)
    before = part.clone()
    for kw in (dict(max_levels=0), dict(max_levels=65)):
        st, _ = ctx.vcycle(g, part, w["k"], w["eps"], w["alpha"], check=False, **kw)
        assert st == F.FR_ERR_INVALID_ARG
    st, _ = ctx.vcycle(g, part, w["k"], w["eps"], w["alpha"], F.default_options(mt_alpha=10), check=False)
    assert st == F.FR_ERR_INVALID_ARG
    assert (part == before).all()


def test_vcycle_stall_rule(F, ctx):
    from tests.test_oracle_multilevel import _stars
    for leaves in (25, 14):
        r = _vcycle(F, ctx, _stars(40, leaves), dict(mb=0))
        assert (r["levels"] == 1) == (leaves == 25)


def _cycle(F, ctx, w, kind, d, okw, active_outer=0, max_levels=64):
    st, pref, rref = O.cycle(w, kind, d=d, opts=O.options(**okw), active_outer=active_outer, max_levels=max_levels)
    assert st == 0
    g, part = _dev(F, w)
    st, r = ctx.cycle(g, part, w["k"], w["eps"], w["alpha"], kind=kind, d=d, opts=F.default_options(**okw),
                      active_outer=active_outer, max_levels=max_levels)
    for f in ("coarsenings", "refinements", "depth", "cut_before", "cut_after", "level_coarsenings"):
        assert r[f] == rref[f], (kind, f)
    assert np.array_equal(part.cpu().numpy(), pref)
    return r


@pytest.mark.parametrize("seed", [15200, 15204, 15213, 15214])   # seeded graphs of 1,600-2,700 vertices
def test_cycles_random_small(F, ctx, seed):
    w = I.random_small(seed, n_max=3000, k_max=5)
    for kind, d in (("V", 2), ("W", 2), ("F", 2), ("F", 1)):
        _cycle(F, ctx, w, kind, d, dict(mb=seed % 2, seed=seed))


def test_cycles_workload(F, ctx):
    w = I.config(4, scale=1 / 64)
    rv = _cycle(F, ctx, w, "V", 2, dict(mb=1, seed=2))
    rf = _cycle(F, ctx, w, "F", 2, dict(mb=1, seed=2))
    assert rf["coarsenings"] > rv["coarsenings"]
    _cycle(F, ctx, I.random_small(15300, n_max=2000, k_max=4), "W", 1, dict(mb=1, fm_permille=50, mt_alpha=10),
           active_outer=2)


def test_cycles_where_a_second_coarsening_stalls(F, ctx):
    """The hand-derived stall case of the oracle's pins (paths and isolated vertices, no
    cut edge, max_levels = 2): the GPU's recursion counts the stalled coarsening and
    skips the trial exactly as the oracle does."""
    from tests.test_oracle_multilevel import stall_case
    for stall, refinements in ((True, 2), (False, 4)):
        w = stall_case(stall)
        for kind, d in (("F", 1), ("W", 2)):
            r = _cycle(F, ctx, w, kind, d, dict(mb=0), max_levels=2)
            assert (r["coarsenings"], r["refinements"]) == (2, refinements)


def test_contract_rejects_a_non_matching(F, ctx):
    import torch
    w = I.random_small(14500, n_max=500, k_max=3)
    g, _ = _dev(F, w)
    n = w["n"]
    for bad in ([1, 2, 0], [0], [n]):   # not pointing back, a self loop, out of range
        mate = np.full(n, -1, np.int32)
        mate[:len(bad)] = bad
        st, _, _ = ctx.contract(g, torch.as_tensor(mate).cuda(), check=False)
        assert st == F.FR_ERR_INVALID_ARG
