"""Seeded synthetic inputs shaped like the paper's instances (Section 6, "Instances").

The paper evaluates on random geometric graphs, Delaunay meshes and FEM graphs
with k in {2..64} and 1-5 % imbalance.  Those files are not available, so the
workloads are generated here: 2D/3D grids stand in for the meshes and 2D/3D
random geometric graphs for the rgg instances.  Partitions come from recursive
coordinate bisection plus seeded boundary noise, standing in for the multilevel
partitioner's projected partition that flow refinement receives.

This module only builds inputs.  It holds none of the refinement arithmetic and is
the one piece of code shared by the CPU oracle's tests and the CUDA path.

Every workload is a plain dict of numpy int32 arrays plus parameters:
    xadj[n+1], adjncy[nnz], adjwgt[nnz], vwgt[n], part[n], k, eps, alpha, ...
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None

SEED_BASE = 0xF10E0000

i32p = ctypes.POINTER(ctypes.c_int32)
f64p = ctypes.POINTER(ctypes.c_double)


def _lib():
    global _LIB
    if _LIB is None:
        path = os.path.join(_HERE, "lib", "libfrgen.so")
        if not os.path.exists(path):
            from . import build as _build
            _build.build_inputs()
        lib = ctypes.CDLL(path)
        lib.frg_grid2d_nnz.restype = ctypes.c_int64
        lib.frg_grid2d_nnz.argtypes = [ctypes.c_int32, ctypes.c_int32]
        lib.frg_grid2d.argtypes = [ctypes.c_int32, ctypes.c_int32, i32p, i32p, f64p]
        lib.frg_grid3d_nnz.restype = ctypes.c_int64
        lib.frg_grid3d_nnz.argtypes = [ctypes.c_int32] * 3
        lib.frg_grid3d.argtypes = [ctypes.c_int32] * 3 + [i32p, i32p, f64p]
        lib.frg_rgg_points.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_uint64, f64p]
        lib.frg_rgg_edges.restype = ctypes.c_int64
        lib.frg_rgg_edges.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, f64p, i32p, i32p]
        lib.frg_uniform_i32.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, i32p]
        lib.frg_edge_weights.argtypes = [ctypes.c_int32, i32p, i32p, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_uint64, i32p]
        lib.frg_rcb.argtypes = [ctypes.c_int32, ctypes.c_int32, f64p, i32p, ctypes.c_int32, ctypes.c_int32, i32p]
        lib.frg_noise.restype = ctypes.c_int64
        lib.frg_noise.argtypes = [ctypes.c_int32, i32p, i32p, i32p, ctypes.c_int32, i32p, ctypes.c_int64,
                                  ctypes.c_uint64]
        _LIB = lib
    return _LIB


def _p(a, t=i32p):
    return a.ctypes.data_as(t)


# ----------------------------------------------------------------- graphs --

def grid2d(nx: int, ny: int):
    """4-neighbour grid, row-major ids; returns (xadj, adjncy, coords[n,2])."""
    lib = _lib()
    n = nx * ny
    nnz = lib.frg_grid2d_nnz(nx, ny)
    xadj = np.empty(n + 1, np.int32)
    adj = np.empty(nnz, np.int32)
    coords = np.empty((n, 2), np.float64)
    lib.frg_grid2d(nx, ny, _p(xadj), _p(adj), _p(coords, f64p))
    return xadj, adj, coords


def grid3d(nx: int, ny: int, nz: int):
    """7-point grid, id = (z*ny + y)*nx + x; returns (xadj, adjncy, coords[n,3])."""
    lib = _lib()
    n = nx * ny * nz
    nnz = lib.frg_grid3d_nnz(nx, ny, nz)
    xadj = np.empty(n + 1, np.int32)
    adj = np.empty(nnz, np.int32)
    coords = np.empty((n, 3), np.float64)
    lib.frg_grid3d(nx, ny, nz, _p(xadj), _p(adj), _p(coords, f64p))
    return xadj, adj, coords


def rgg(dim: int, n: int, r: float, seed: int):
    """Random geometric graph in the unit square/cube: edge iff distance^2 < r^2."""
    lib = _lib()
    coords = np.empty((n, dim), np.float64)
    lib.frg_rgg_points(dim, n, r, seed & 0xFFFFFFFFFFFFFFFF, _p(coords, f64p))
    xadj = np.empty(n + 1, np.int32)
    nnz = lib.frg_rgg_edges(dim, n, r, _p(coords, f64p), _p(xadj), None)
    adj = np.empty(nnz, np.int32)
    lib.frg_rgg_edges(dim, n, r, _p(coords, f64p), _p(xadj), _p(adj))
    return xadj, adj, coords


def rgg_radius(dim: int, n: int, mean_degree: float) -> float:
    """Radius giving the requested expected degree away from the border."""
    if dim == 2:
        return math.sqrt(mean_degree / (math.pi * n))
    return (3.0 * mean_degree / (4.0 * math.pi * n)) ** (1.0 / 3.0)


def uniform_i32(count: int, lo: int, hi: int, seed: int):
    out = np.empty(count, np.int32)
    _lib().frg_uniform_i32(count, lo, hi, seed & 0xFFFFFFFFFFFFFFFF, _p(out))
    return out


def edge_weights(xadj, adjncy, lo: int, hi: int, seed: int):
    out = np.empty(len(adjncy), np.int32)
    _lib().frg_edge_weights(len(xadj) - 1, _p(xadj), _p(adjncy), lo, hi, seed & 0xFFFFFFFFFFFFFFFF, _p(out))
    return out


def rcb(coords, vwgt, k: int, force_axis: int = -1):
    n, dim = coords.shape
    part = np.empty(n, np.int32)
    c = np.ascontiguousarray(coords, np.float64)
    _lib().frg_rcb(n, dim, _p(c, f64p), _p(vwgt), k, force_axis, part.ctypes.data_as(i32p))
    return part


def noise(xadj, adjncy, vwgt, k: int, part, nswaps: int, seed: int) -> int:
    """In-place boundary noise; nswaps < 0 means a fraction in parts per million."""
    return int(_lib().frg_noise(len(xadj) - 1, _p(xadj), _p(adjncy), _p(vwgt), k, _p(part), nswaps,
                                seed & 0xFFFFFFFFFFFFFFFF))


# --------------------------------------------------------------- workloads --

def _workload(name, xadj, adjncy, adjwgt, vwgt, part, k, **params):
    w = dict(name=name, n=len(xadj) - 1, nnz=len(adjncy), xadj=xadj, adjncy=adjncy, adjwgt=adjwgt,
             vwgt=vwgt, part=part, k=k)
    w.update(params)
    return w


def grid2d_halves(nx=64, ny=64, swaps=200, seed=SEED_BASE + 1, eps=0.03, alpha=1.0):
    """64x64 4-neighbour grid split into column halves (block 0 = x < nx/2) with seeded swaps."""
    xadj, adj, coords = grid2d(nx, ny)
    n = nx * ny
    vwgt = np.ones(n, np.int32)
    adjwgt = np.ones(len(adj), np.int32)
    part = (coords[:, 0] >= nx // 2).astype(np.int32)
    applied = noise(xadj, adj, vwgt, 2, part, swaps, seed ^ 0x33)
    return _workload(f"grid2d {nx}x{ny} k=2", xadj, adj, adjwgt, vwgt, part, 2, eps=eps, alpha=alpha,
                     mb=0, adaptive=0, alpha_max=alpha, max_iters=1, swaps=applied, seed=seed)


def rgg2d_bisection(n=65536, mean_degree=8.0, noise_ppm=20000, seed=SEED_BASE + 2, eps=0.03):
    """2D random geometric graph, bisected at the x median, with boundary noise."""
    r = rgg_radius(2, n, mean_degree)
    xadj, adj, coords = rgg(2, n, r, seed)
    vwgt = np.ones(n, np.int32)
    adjwgt = np.ones(len(adj), np.int32)
    part = rcb(coords, vwgt, 2, force_axis=0)
    applied = noise(xadj, adj, vwgt, 2, part, -noise_ppm, seed ^ 0x33)
    return _workload(f"rgg2d n={n} k=2", xadj, adj, adjwgt, vwgt, part, 2, eps=eps, alpha=1.0,
                     mb=0, adaptive=1, alpha_max=16.0, max_iters=10, radius=r, swaps=applied, seed=seed)


def grid3d_rcb(nx=128, ny=128, nz=128, k=16, noise_ppm=10000, seed=SEED_BASE + 3, eps=0.03, alpha=2.0):
    """3D 7-point grid, recursive coordinate bisection into k blocks, 1 % boundary noise."""
    xadj, adj, coords = grid3d(nx, ny, nz)
    n = nx * ny * nz
    vwgt = np.ones(n, np.int32)
    adjwgt = np.ones(len(adj), np.int32)
    part = rcb(coords, vwgt, k)
    applied = noise(xadj, adj, vwgt, k, part, -noise_ppm, seed ^ 0x33)
    return _workload(f"grid3d {nx}x{ny}x{nz} k={k}", xadj, adj, adjwgt, vwgt, part, k, eps=eps,
                     alpha=alpha, mb=1, adaptive=0, alpha_max=alpha, max_iters=1, swaps=applied, seed=seed)


def rgg3d_rcb(n=4194304, mean_degree=12.0, k=64, noise_ppm=10000, seed=SEED_BASE + 4, eps=0.01, alpha=4.0,
              wlo=1, whi=10, clo=1, chi=4):
    """3D random geometric graph, edge weights U[wlo,whi], vertex weights U[clo,chi], RCB + noise."""
    r = rgg_radius(3, n, mean_degree)
    xadj, adj, coords = rgg(3, n, r, seed)
    vwgt = uniform_i32(n, clo, chi, seed ^ 0x22)
    adjwgt = edge_weights(xadj, adj, wlo, whi, seed ^ 0x11)
    part = rcb(coords, vwgt, k)
    applied = noise(xadj, adj, vwgt, k, part, -noise_ppm, seed ^ 0x33)
    return _workload(f"rgg3d n={n} k={k}", xadj, adj, adjwgt, vwgt, part, k, eps=eps, alpha=alpha, mb=1,
                     adaptive=0, alpha_max=alpha, max_iters=1, radius=r, swaps=applied, seed=seed)


def config(i: int, scale: float = 1.0):
    """Workload i in 1..4 at full size (scale=1) or shrunk by `scale` for quick tests."""
    if i == 1:
        return grid2d_halves()
    if i == 2:
        return rgg2d_bisection(n=max(256, int(65536 * scale)))
    if i == 3:
        s = max(8, int(round(128 * scale ** (1.0 / 3.0))))
        s -= s % 4
        return grid3d_rcb(s, s, s)
    if i == 4:
        return rgg3d_rcb(n=max(4096, int(4194304 * scale)))
    raise ValueError(i)


def serving_pool(count=48, seed=SEED_BASE + 5, max_n=1 << 21, min_n=1 << 10):
    """Pool of seeded graphs for the serving mix: 2D grids and 2D/3D random geometric graphs."""
    rs = np.random.Generator(np.random.Philox(seed))
    pool = []
    for g in range(count):
        kind = g % 3
        gseed = seed * 1000 + g
        weighted = bool(rs.integers(0, 2))
        if kind == 0:
            e = int(rs.integers(5, 11))               # 2^10 .. 2^20 vertices
            nx, ny = 1 << e, 1 << e
            while nx * ny > max_n:
                nx //= 2
            xadj, adj, coords = grid2d(nx, ny)
            n = nx * ny
            desc = f"grid2d {nx}x{ny}"
        else:
            dim = 2 if kind == 1 else 3
            e = int(rs.integers(12, 22))
            n = min(1 << e, max_n)
            deg = float(rs.choice([8.0, 10.0, 12.0]))
            xadj, adj, coords = rgg(dim, n, rgg_radius(dim, n, deg), gseed)
            desc = f"rgg{dim}d n={n} deg={deg:g}"
        if n < min_n:
            continue
        vwgt = np.ones(n, np.int32)
        adjwgt = edge_weights(xadj, adj, 1, 10, gseed ^ 0x11) if weighted else np.ones(len(adj), np.int32)
        pool.append(dict(name=desc, n=n, nnz=len(adj), xadj=xadj, adjncy=adj, adjwgt=adjwgt, vwgt=vwgt,
                         coords=coords, seed=gseed))
    return pool


def serving_partition(graph, k: int, noise_ppm=10000):
    part = rcb(graph["coords"], graph["vwgt"], k)
    noise(graph["xadj"], graph["adjncy"], graph["vwgt"], k, part, -noise_ppm, graph["seed"] ^ (0x33 + k))
    return part


def random_small(seed: int, n_max: int = 400, k_max: int = 5):
    """A small seeded workload for parity sweeps: grid or rgg, random weights (zero vertex
    weights allowed), k in [2, k_max], coordinate bisection plus boundary noise."""
    rs = np.random.Generator(np.random.Philox(seed))
    kind = int(rs.integers(0, 3))
    if kind == 0:
        nx = int(rs.integers(3, 24))
        ny = int(rs.integers(2, max(3, min(24, n_max // nx))))
        xadj, adj, coords = grid2d(nx, ny)
        desc = f"grid2d {nx}x{ny}"
    elif kind == 1:
        n = int(rs.integers(16, n_max + 1))
        deg = float(rs.uniform(4.0, 10.0))
        xadj, adj, coords = rgg(2, n, rgg_radius(2, n, deg), seed * 7 + 1)
        desc = f"rgg2d n={n}"
    else:
        s = int(rs.integers(2, 8))
        xadj, adj, coords = grid3d(s, s, max(2, min(8, n_max // (s * s))))
        desc = f"grid3d {s}^2x{len(xadj) // (s * s)}"
    n = len(xadj) - 1
    if rs.integers(0, 2):
        adjwgt = edge_weights(xadj, adj, 1, 10, seed ^ 0x11)
    else:
        adjwgt = np.ones(len(adj), np.int32)
    if rs.integers(0, 2):
        vwgt = uniform_i32(n, 0, 4, seed ^ 0x22)
    else:
        vwgt = np.ones(n, np.int32)
    k = int(rs.integers(2, k_max + 1))
    k = min(k, max(2, n // 4))
    part = rcb(coords, vwgt, k)
    noise(xadj, adj, vwgt, k, part, int(rs.integers(0, max(2, n // 10))), seed ^ 0x33)
    eps = float(rs.choice([0.01, 0.03, 0.05, 0.1, 0.125, 0.25]))
    alpha = float(rs.choice([1.0, 1.0, 2.0, 4.0]))
    mb = int(rs.integers(0, 2))
    return _workload(f"{desc} k={k} seed={seed}", xadj, adj, adjwgt, vwgt, part, k, eps=eps, alpha=alpha, mb=mb,
                     adaptive=0, alpha_max=alpha, max_iters=1, seed=seed, coords=coords)
