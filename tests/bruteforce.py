"""Brute-force enumeration of all s-t cuts of a small corridor network (test helper).

The network is given in the export format shared by the oracle and the CUDA
path: corridor arcs (off, head, cap), border kind per vertex (1: s -> v,
2: v -> t) and the capacity INF_v of that arc.  Bit i of a mask set means
corridor vertex i lies on the source side; s is always on the source side and
t never is.
"""
import numpy as np


def cut_values(ex):
    nc = len(ex["gid"])
    assert nc <= 22
    masks = np.arange(1 << nc, dtype=np.int64)
    bits = [((masks >> i) & 1).astype(bool) for i in range(nc)]
    cut = np.zeros(1 << nc, dtype=np.int64)
    off, head, cap = ex["off"], ex["head"], ex["cap"]
    for i in range(nc):
        for j in range(off[i], off[i + 1]):
            h = head[j]
            cut += cap[j] * (bits[i] & ~bits[h])
        if ex["border"][i] == 1:
            cut += int(ex["infcap"][i]) * (~bits[i])
        elif ex["border"][i] == 2:
            cut += int(ex["infcap"][i]) * bits[i]
    return masks, cut, bits


def closed_masks(ex, arcflow, stflow, bits):
    """Masks (source sides) closed under residual arcs of the given flow."""
    nc = len(ex["gid"])
    ok = np.ones(len(bits[0]), dtype=bool)
    off, head, cap = ex["off"], ex["head"], ex["cap"]
    for i in range(nc):
        for j in range(off[i], off[i + 1]):
            if cap[j] - arcflow[j] > 0:          # residual arc i -> head
                ok &= ~bits[i] | bits[head[j]]
        if ex["border"][i] == 1 and ex["infcap"][i] - stflow[i] > 0:
            ok &= bits[i]                        # residual s -> i
        elif ex["border"][i] == 2 and ex["infcap"][i] - stflow[i] > 0:
            ok &= ~bits[i]                       # residual i -> t
    return ok


def side_weights(ex, vw, cA, cB, mask_bits_source):
    """c(A') for each mask: block a minus its corridor vertices on the sink side plus block b's on the source side."""
    wA = np.full(len(mask_bits_source[0]), cA, dtype=np.int64)
    for i in range(len(ex["gid"])):
        if ex["side0"][i] == 0:
            wA -= int(vw[i]) * (~mask_bits_source[i])
        else:
            wA += int(vw[i]) * mask_bits_source[i]
    return wA, (cA + cB) - wA


def mask_of(sel):
    m = 0
    for i, s in enumerate(sel):
        if s:
            m |= 1 << i
    return m
