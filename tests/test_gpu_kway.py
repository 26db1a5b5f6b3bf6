"""Global k-way refinement rounds (Section 2.2, set up as in Section 6) on the CUDA
path against the oracle: rounds of one k-way search from the whole boundary or the
corner vertices, until a round gains nothing.  Partitions and totals are integers:
bit-exact."""
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


def _rounds(F, ctx, w, init_mode, alpha, max_rounds, seed):
    st, pref, tref, rref = O.kway_global(w, alpha=alpha, init_mode=init_mode, max_rounds=max_rounds, seed=seed)
    assert st == 0
    g, part = _dev(F, w)
    st, tot = ctx.kway_global(g, part, w["k"], w["eps"], init_mode=init_mode, alpha=alpha, max_rounds=max_rounds,
                              seed=seed)
    assert tot["status"] == 0
    assert (tot["gain"], tot["tried"], tot["kept"], tot["searches"]) == \
        (tref["gain"], tref["tried"], tref["kept"], rref)
    assert np.array_equal(part.cpu().numpy(), pref)
    return tref, rref


@pytest.mark.parametrize("seed", range(24))
def test_rounds_random_small(F, ctx, seed):
    w = I.random_small(7600 + seed, n_max=2500, k_max=9)
    _rounds(F, ctx, w, seed % 2, (1, 10, 0, 100)[seed % 4], (1, 3, 10)[seed % 3], seed)


@pytest.mark.parametrize("cfg,scale,init_mode", [(1, 1.0, 0), (1, 1.0, 1), (2, 1 / 16, 0), (3, 1 / 64, 0),
                                                 (4, 1 / 64, 0), (4, 1 / 64, 1), (4, 1 / 16, 0)])
def test_rounds_workloads(F, ctx, cfg, scale, init_mode):
    w = I.config(cfg, scale=scale)
    tref, rounds = _rounds(F, ctx, w, init_mode, 10, 4, 5)
    assert rounds >= 1


def test_rounds_improve_a_perturbed_grid(F, ctx):
    # quadrants of a 64 x 64 grid with vertices swapped across the lines: the rounds
    # must take back cut edges, and the later rounds see the earlier ones' partition
    xadj, adj, coords = I.grid2d(64, 64)
    x, y = coords[:, 0].astype(int), coords[:, 1].astype(int)
    part = (2 * (y >= 32) + (x >= 32)).astype(np.int32)
    rng = np.random.default_rng(3)
    for v in rng.choice(np.flatnonzero((x == 31) | (y == 31)), 40, replace=False):
        part[v] = (part[v] + 1) % 4
    n = 64 * 64
    w = dict(name="quadrants 64x64", n=n, nnz=len(adj), xadj=xadj, adjncy=adj,
             adjwgt=np.ones(len(adj), np.int32), vwgt=np.ones(n, np.int32), part=part, k=4, eps=0.03)
    tref, rounds = _rounds(F, ctx, w, 0, 10, 10, 11)
    assert tref["gain"] > 0


def test_rounds_without_boundary_and_option_checks(F, ctx):
    w = I.random_small(7700, n_max=400, k_max=4)
    w1 = dict(w, part=np.zeros(w["n"], np.int32))   # one block: no start vertex
    g, part = _dev(F, w1)
    st, tot = ctx.kway_global(g, part, w["k"], w["eps"])
    assert st == 0 and (tot["gain"], tot["tried"], tot["kept"], tot["searches"]) == (0, 0, 0, 1)
    assert (part == 0).all()
    g, part = _dev(F, w)
    before = part.clone()
    for kw in (dict(init_mode=2), dict(alpha=-1), dict(max_rounds=0)):
        st, _ = ctx.kway_global(g, part, w["k"], w["eps"], check=False, **kw)
        assert st == F.FR_ERR_INVALID_ARG
    st, _ = ctx.kway_global(g, part, w["k"], 0.0, check=False)
    assert st == F.FR_ERR_INVALID_ARG
    w2 = dict(w, adjwgt=np.full(len(w["adjncy"]), 2000, np.int32))   # gains beyond +-1023
    g2, part2 = _dev(F, w2)
    st, _ = ctx.kway_global(g2, part2, w["k"], w["eps"], check=False)
    assert st == F.FR_ERR_TOO_LARGE
    assert (part == before).all() and (part2 == before).all()


@pytest.mark.parametrize("seed,init_mode", [(1, 0), (2, 0), (3, 1), (4, 1)])
def test_rounds_hub_graph(F, ctx, seed, init_mode):
    # hubs of degree 33-110 with neighbours in up to 16 blocks (serial gain path and its
    # re-summing fallback), in the start set and keyed again as their neighbours move
    from tests.hub_graph import hub_workload
    w = hub_workload(seed, weighted=seed % 2 == 1)
    _rounds(F, ctx, w, init_mode, 10, 6, seed)
