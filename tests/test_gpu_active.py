"""Active block scheduling (fr_refine_active) against the oracle's
fro_refine_active: the same refinements in the same order with the same results,
the same number of outer rounds and the same final partition (all integers, so
bit-exact), with and without adaptive flow iterations."""
import numpy as np
import pytest

import oracle as O
from paper_1012_0006_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FIELDS = ("a", "b", "round", "accepted", "iters", "flow", "cut_before", "cut_after", "wA_before", "wB_before",
          "wA_after", "wB_after", "corridor_n", "corridor_arcs", "alpha_final")


@pytest.fixture(scope="module")
def F(gpu_lib):
    return gpu_lib


@pytest.fixture(scope="module")
def ctx(F):
    c = F.Context(0)
    yield c
    c.close()


def _check(F, ctx, w, okw, max_outer=12, alpha=None):
    import torch
    alpha = w["alpha"] if alpha is None else alpha
    st, pref, rref, nref = O.refine_active(w, alpha=alpha, opts=O.options(**okw), max_outer=max_outer)
    assert st == 0
    g = F.DeviceGraph.from_workload(w)
    part = torch.as_tensor(np.array(w["part"], np.int32)).cuda()
    st, res, summ, nouter = ctx.refine_active(g, part, w["k"], w["eps"], alpha, F.default_options(**okw),
                                              max_outer=max_outer)
    assert nouter == nref
    assert len(res) == len(rref)
    for rg, rc in zip(res, rref):
        for f in FIELDS:
            assert rg[f] == rc[f], (f, rg["a"], rg["b"], rg["round"])
    assert np.array_equal(part.cpu().numpy(), pref)
    assert summ["npairs"] == len(rref) and summ["accepted"] == sum(r["accepted"] for r in rref)
    assert summ["cut_after"] == summ["cut_before"] + sum(r["cut_after"] - r["cut_before"] for r in rref)
    return res, nouter


def test_grid2d_64_plain(F, ctx):
    res, nouter = _check(F, ctx, I.config(1), dict(mb=0))
    assert nouter >= 2


def test_rgg2d_4096_adaptive_mb(F, ctx):
    _check(F, ctx, I.config(2, scale=1 / 16), dict(mb=1, adaptive=1, max_iters=8, alpha_max=16.0), alpha=1.0)


def test_grid3d_32_mb_two_sweeps(F, ctx):
    _check(F, ctx, I.config(3, scale=1 / 64), dict(mb=1, mb_reps=2, seed=5))


def test_rgg3d_small_adaptive(F, ctx):
    _check(F, ctx, I.config(4, scale=1 / 64), dict(mb=1, adaptive=1, max_iters=5, alpha_max=8.0), alpha=1.0)


@pytest.mark.parametrize("seed", range(12))
def test_random_small(F, ctx, seed):
    w = I.random_small(4300 + seed, n_max=3000, k_max=8)
    okw = dict(mb=seed % 2, mb_reps=1 + seed % 3, seed=seed)
    if seed % 3:
        okw.update(adaptive=1, max_iters=2 + seed % 5, alpha_max=float(2 ** (seed % 4)))
    _check(F, ctx, w, okw, max_outer=1 + seed % 6)


def test_invalid_max_outer_leaves_part(F, ctx):
    import torch
    w = I.config(1)
    g = F.DeviceGraph.from_workload(w)
    part = torch.as_tensor(np.array(w["part"], np.int32)).cuda()
    st, _, _, _ = ctx.refine_active(g, part, w["k"], w["eps"], w["alpha"], F.default_options(), max_outer=0,
                                    check=False)
    assert st == 1   # FR_ERR_INVALID_ARG
    assert np.array_equal(part.cpu().numpy(), np.array(w["part"], np.int32))


@pytest.mark.parametrize("name,make,okw", [
    ("rgg2d-4096", lambda: I.config(2, scale=1 / 16), dict(mb=1, adaptive=1, max_iters=8, alpha_max=16.0)),
    ("grid3d-32", lambda: I.config(3, scale=1 / 64), dict(mb=1, adaptive=1, max_iters=5, alpha_max=8.0)),
    ("small", lambda: I.random_small(7100, n_max=2500, k_max=8), dict(mb=0, adaptive=1, max_iters=6, alpha_max=8.0)),
    ("small-fm", lambda: I.random_small(7101, n_max=2500, k_max=8),
     dict(mb=1, adaptive=1, max_iters=6, alpha_max=8.0, fm_permille=50)),
], ids=lambda x: x if isinstance(x, str) else "")
def test_batch_with_adaptive_iterations(F, ctx, name, make, okw):
    """fr_refine_batch with adaptive flow iterations: every pair of a round on its own
    alpha, against the oracle's batch (same pairs, results and partition)."""
    import torch
    w = make()
    st, pref, rref, nr = O.refine_batch(w, alpha=1.0, opts=O.options(**okw))
    assert st == 0
    g = F.DeviceGraph.from_workload(w)
    part = torch.as_tensor(np.array(w["part"], np.int32)).cuda()
    st, res, summ = ctx.refine_batch(g, part, w["k"], w["eps"], 1.0, F.default_options(**okw))
    assert summ["npairs"] == len(rref) and summ["nrounds"] == nr
    for rg, rc in zip(res, rref):
        for f in FIELDS + ("cut_fm", "fm_moves"):
            assert rg[f] == rc[f], (f, rg["a"], rg["b"], rg["round"])
    assert np.array_equal(part.cpu().numpy(), pref)
    if name.startswith("rgg2d"):
        assert any(r["iters"] > 1 for r in rref)   # the adaptive loop did iterate
