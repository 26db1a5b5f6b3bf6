"""Serving (continuous batching): every request's result is the same alone and in
the mix, bit for bit; admission by footprint; a bad request fails alone."""
import numpy as np
import pytest

from paper_1012_0006_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _graphs():
    out = []
    for i, (kind, size) in enumerate([("grid", 24), ("rgg2", 3000), ("rgg3", 4000), ("grid", 40)]):
        if kind == "grid":
            xadj, adj, coords = I.grid2d(size, size)
        else:
            dim = 2 if kind == "rgg2" else 3
            xadj, adj, coords = I.rgg(dim, size, I.rgg_radius(dim, size, 9.0), 900 + i)
        n = len(xadj) - 1
        wgt = I.edge_weights(xadj, adj, 1, 10, 77 + i) if i % 2 else np.ones(len(adj), np.int32)
        out.append(dict(xadj=xadj, adjncy=adj, adjwgt=wgt, vwgt=np.ones(n, np.int32), coords=coords, n=n, seed=i))
    return out


def _requests(graphs, count, seed=5):
    rs = np.random.Generator(np.random.Philox(seed))
    reqs = []
    for t in range(count):
        gi = int(rs.integers(0, len(graphs)))
        g = graphs[gi]
        k = int(rs.choice([2, 4, 8]))
        part = I.rcb(g["coords"], g["vwgt"], k)
        I.noise(g["xadj"], g["adjncy"], g["vwgt"], k, part, max(1, g["n"] // 50), 1000 + t)
        eps = float(rs.choice([0.01, 0.03, 0.05]))
        reqs.append(dict(gi=gi, part=part, k=k, eps=eps, alpha=2.0, tag=t))
    return reqs


def _alone(F, ctx, g, r, opts):
    import torch
    dg = F.DeviceGraph(g["xadj"], g["adjncy"], g["adjwgt"], g["vwgt"])
    part = torch.as_tensor(r["part"]).cuda()
    st, _, summ = ctx.refine_batch(dg, part, r["k"], r["eps"], r["alpha"], opts, results=False)
    return part.cpu().numpy(), summ


def test_results_are_the_same_alone_and_in_the_mix(gpu_lib):
    F = gpu_lib
    graphs = _graphs()
    reqs = _requests(graphs, 24)
    opts = F.default_options(mb=1)
    with F.Server(0, max_inflight=8, opts=opts) as srv:
        ids = [srv.add_graph(g["xadj"], g["adjncy"], g["adjwgt"], g["vwgt"]) for g in graphs]
        for r in reqs:
            srv.submit(ids[r["gi"]], r["part"], r["k"], r["eps"], r["alpha"], r["tag"])
        got = {}
        for _ in reqs:
            resp, part = srv.next(max(g["n"] for g in graphs), timeout_ms=120000)
            got[resp["tag"]] = (resp, part)
        stats = srv.stats()
    assert stats["completed"] == len(reqs) and stats["max_concurrent"] > 1
    with F.Context(0) as ctx:
        for r in reqs:
            g = graphs[r["gi"]]
            resp, part = got[r["tag"]]
            assert resp["status"] == 0
            ref, summ = _alone(F, ctx, g, r, opts)
            assert np.array_equal(part[:g["n"]], ref)
            assert (resp["npairs"], resp["nrounds"], resp["accepted"]) == (summ["npairs"], summ["nrounds"],
                                                                            summ["accepted"])
            assert (resp["cut_before"], resp["cut_after"]) == (summ["cut_before"], summ["cut_after"])


def test_admission_by_footprint_serialises_requests(gpu_lib):
    F = gpu_lib
    graphs = _graphs()[:2]
    reqs = _requests(graphs, 6, seed=9)
    with F.Server(0, max_inflight=8, arena_bytes=1, opts=F.default_options(mb=1)) as srv:
        ids = [srv.add_graph(g["xadj"], g["adjncy"], g["adjwgt"], g["vwgt"]) for g in graphs]
        for r in reqs:
            srv.submit(ids[r["gi"]], r["part"], r["k"], r["eps"], r["alpha"], r["tag"])
        for _ in reqs:
            resp, _ = srv.next(max(g["n"] for g in graphs), timeout_ms=120000)
            assert resp["status"] == 0
        assert srv.stats()["max_concurrent"] == 1      # nothing else fits beside a running request


def test_a_bad_request_fails_alone(gpu_lib):
    F = gpu_lib
    graphs = _graphs()[:2]
    reqs = _requests(graphs, 4, seed=11)
    bad = dict(reqs[1])
    bad["part"] = bad["part"].copy()
    bad["part"][0] = 99                                 # block id >= k: rejected on the device
    bad["tag"] = 100
    with F.Server(0, max_inflight=4, opts=F.default_options(mb=1)) as srv:
        ids = [srv.add_graph(g["xadj"], g["adjncy"], g["adjwgt"], g["vwgt"]) for g in graphs]
        for r in reqs + [bad]:
            srv.submit(ids[r["gi"]], r["part"], r["k"], r["eps"], r["alpha"], r["tag"])
        res = {}
        for _ in range(len(reqs) + 1):
            resp, part = srv.next(max(g["n"] for g in graphs), timeout_ms=120000)
            res[resp["tag"]] = (resp, part)
    assert res[100][0]["status"] == F.FR_ERR_INVALID_ARG
    assert np.array_equal(res[100][1][:graphs[bad["gi"]]["n"]], bad["part"])
    assert all(res[r["tag"]][0]["status"] == 0 for r in reqs)


def test_served_results_match_the_oracle(gpu_lib):
    """A seeded sample of the request mix through the server against the CPU oracle's
    sweep of the same request (partition, pairs, rounds, cuts)."""
    import oracle as O
    F = gpu_lib
    graphs = _graphs()
    reqs = _requests(graphs, 16, seed=11)
    opts = F.default_options(mb=1)
    with F.Server(0, max_inflight=6, opts=opts) as srv:
        ids = [srv.add_graph(g["xadj"], g["adjncy"], g["adjwgt"], g["vwgt"]) for g in graphs]
        for r in reqs:
            srv.submit(ids[r["gi"]], r["part"], r["k"], r["eps"], r["alpha"], r["tag"])
        got = {}
        for _ in reqs:
            resp, part = srv.next(max(g["n"] for g in graphs), timeout_ms=120000)
            got[resp["tag"]] = (resp, part)
    for r in reqs:
        g = graphs[r["gi"]]
        w = dict(n=g["n"], xadj=g["xadj"], adjncy=g["adjncy"], adjwgt=g["adjwgt"], vwgt=g["vwgt"],
                 part=r["part"], k=r["k"], eps=r["eps"], alpha=r["alpha"])
        st, pref, rref, nr = O.refine_batch(w, opts=O.options(mb=1))
        assert st == 0
        resp, part = got[r["tag"]]
        assert resp["status"] == 0
        assert np.array_equal(part[:g["n"]], pref)
        assert (resp["npairs"], resp["nrounds"]) == (len(rref), nr)
        assert resp["cut_after"] - resp["cut_before"] == sum(x["cut_after"] - x["cut_before"] for x in rref)
