"""A seeded graph with hubs, for the k-way searches' high-degree paths: a 2D random
geometric graph plus a few hub vertices joined to random vertices anywhere in it, so that
hubs have degrees above 32 and neighbours in more than eight blocks.  Generic graph
construction only (no arithmetic of the method)."""
import numpy as np

from paper_1012_0006_gb300 import inputs as I


def hub_workload(seed, n=3000, hubs=12, deg_lo=33, deg_hi=110, k=16, weighted=True):
    rs = np.random.Generator(np.random.Philox(seed))
    xadj, adj, coords = I.rgg(2, n, I.rgg_radius(2, n, 7.0), seed * 3 + 1)
    src = np.repeat(np.arange(n), np.diff(xadj))
    us, vs = [src], [adj]
    for h in range(hubs):
        d = int(rs.integers(deg_lo, deg_hi + 1))
        nb = rs.choice(n, size=d, replace=False)
        hv = np.full(d, n + h)
        us += [hv, nb]
        vs += [nb, hv]
    u = np.concatenate(us).astype(np.int64)
    v = np.concatenate(vs).astype(np.int64)
    N = n + hubs
    key = np.unique(u * N + v)
    u, v = key // N, key % N
    xadj2 = np.zeros(N + 1, np.int64)
    np.add.at(xadj2, u + 1, 1)
    xadj2 = np.cumsum(xadj2).astype(np.int32)
    adj2 = v.astype(np.int32)
    if weighted:   # symmetric weights in [1, 8]: a function of the unordered pair
        lo, hi = np.minimum(u, v), np.maximum(u, v)
        adjwgt = (1 + (lo * 1000003 + hi * 7 + seed) % 8).astype(np.int32)
    else:
        adjwgt = np.ones(len(adj2), np.int32)
    vwgt = np.ones(N, np.int32)
    coords2 = np.vstack([coords, rs.uniform(0, 1, size=(hubs, coords.shape[1]))])
    part = I.rcb(coords2, vwgt, k)
    I.noise(xadj2, adj2, vwgt, k, part, N // 20, seed ^ 0x5A)
    return dict(name=f"rgg2d n={n} + {hubs} hubs k={k} seed={seed}", n=N, nnz=len(adj2), xadj=xadj2, adjncy=adj2,
                adjwgt=adjwgt, vwgt=vwgt, part=part, k=k, eps=0.05, alpha=1.0, mb=0)
