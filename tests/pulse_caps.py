"""A host-side way to make a later adaptive flow iteration fail, for the GPU tests.

The pulse cap (fr_options.pulse_cap) bounds the push-relabel pulses of one flow.  A
cap between the pulses of the first iteration (alpha = 1, accepted with a smaller cut,
so the adaptive loop goes on) and those of the second (alpha = 2 on its result) makes
the first succeed and write part, and the second fail with FR_ERR_ITER_LIMIT.  No
fault is involved: the kernels stop at the cap and report it.
"""
import numpy as np


def later_iteration_cap(run, w, kw, runs=3, exact=False):
    """run(part_tensor, alpha, opts_kw) -> fr_pair_result of one non-adaptive call on
    pair (0, 1).  Returns a cap at least a quarter above the first iteration's pulses
    and an eighth below the second's (lock-free pulse counts vary a little between
    runs), or None if the counts do not separate that far or the first iteration would
    not continue the loop.  On the 2D rgg workloads of 16,384 and 32,768 vertices the
    two take 17 and 33 pulses.  exact=True (the level-ordered waves of flow_sched = 1,
    whose counts do not vary): the first iteration's count itself, if the second's is
    larger in every run."""
    import torch
    p0 = torch.as_tensor(np.array(w["part"], np.int32)).cuda()
    first, p1 = [], None
    for _ in range(runs):
        p = p0.clone()
        r = run(p, 1.0, kw)
        if r.status != 0 or not (r.accepted and r.cut_after < r.cut_before):
            return None
        first.append(r.pulses)
        p1 = p
    second = []
    for _ in range(runs):
        p = p1.clone()
        r = run(p, 2.0, kw)
        if r.status != 0:
            return None
        second.append(r.pulses)
    if exact:
        return max(first) if min(second) > max(first) else None
    lo, hi = max(first) * 5 // 4 + 1, min(second) * 7 // 8
    return (lo + hi) // 2 if lo <= hi else None
