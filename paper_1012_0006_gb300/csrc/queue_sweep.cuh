// The queue sweep: every pair of a sweep in one persistent launch of thread-block
// clusters, each pair started as soon as the pairs before it that share one of its
// blocks have committed (internal to libflowref).
#pragma once

#include <cuda_runtime.h>

#include "fr_internal.cuh"

namespace fr {

// Per-cluster workspace: the network, visit list and control block of
// the pair the cluster is working on.  Capacities are the QueueArgs' nu_cap / mu_cap /
// vq_cap.
struct QSlot {
    GraphDev *graph;      // this cluster's copy of the graph descriptor (its own sob)
    int *sob;             // [k] side of each block for the current pair, -1 otherwise
    Ctl *ctl;
    long long *hist;      // [3 * 2 * kHistBins]
    int *cta_cnt;         // [cluster size + 1]
    unsigned int *cbits;  // corridor bitmap over the graph's vertices (zero between pairs)
    unsigned int *sbits;  // one bit per 1,024 vertices: groups with corridor bits (zero between pairs)
    unsigned int *sdbits; // corridor vertices of side b, one bit per vertex (zero between pairs)
    int *vq_v, *vq_s;
    int *gid, *sid, *off, *infc, *fx, *lab, *rflag, *color, *scc, *vc, *fq0, *fq1;
    int *cid, *cpair, *cmin, *indeg, *outoff, *ocur, *plist, *sinkc, *pcur;
    long long *ex, *cw;
    unsigned char *border, *side_out;
    int *head, *rev, *res, *cap, *outs;
    int *indeg_r, *order, *hcomp;
    unsigned long long *hkey;
    long long *sw_absd;
    int *sw_j;
    long long *stat;      // [4]: visited entries, corridor vertices, corridor arcs, pairs, summed
};

struct QueueArgs {
    Work wt;              // options and the sweep's pair arrays (pairs, sides, pacc at pair 0)
    const QSlot *slots;   // [clusters]
    int np;               // pairs of the sweep, in round order
    int *ticket;          // next pair to take (zero before the launch)
    const int *prev;      // [2 np]: the last earlier pair that shares block a (b), or -1
    int *gabort;          // 0, E_MISFIT (run the sweep round by round instead), or an error code
    unsigned long long wait_ns;   // bound of one wait for a dependency (then E_ABORT)
};

cudaError_t launch_queue_sweep(const QueueArgs &q, int cluster, int clusters, cudaStream_t st);
// Clusters of `cluster` CTAs the queue kernel can keep resident at once (0: none).
cudaError_t queue_capacity(int cluster, int *max_clusters);
size_t queue_smem();   // dynamic shared memory of one CTA of the queue kernel
// The candidate list bl[0, *blc) bucketed by block into sorted / start (k + 1 entries);
// lst[v] = part[v] for listed v (the caller sets every entry to -1 first); cnt (k) is
// scratch, app (k) is cleared.  k <= 1024.
cudaError_t launch_qb_build(const int *bl, const int *blc, const int *part, int k, int *cnt, int *start, int *app,
                            int *lst, int *sorted, cudaStream_t st);

}  // namespace fr
