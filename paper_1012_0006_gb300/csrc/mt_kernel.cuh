// Multi-try FM (k-way local searches with the KaSPar stopping rule) after the pairwise
// improvements of a matching: device state and launch.
#pragma once

#include <cuda_runtime.h>

#include "fr_internal.cuh"

namespace fr {

constexpr int kMtGmax = 1023;                 // |gain| bound (max weighted degree)
constexpr int kMtBuckets = 2 * kMtGmax + 2;   // gain buckets of the single queue
constexpr int kMtMaxK = 1024;                 // block weights cached in shared memory
constexpr int kKwChunk = 1024;                // start entries per warp when a round's queue is built

// Totals of one pass.
struct MtRes {
    long long gain;          // cut decrease kept
    int searches, tried, kept;
    int stopped;             // global k-way round: 1 if the KaSPar rule stopped its search
};

// Device state of a multi-try pass over the pairs of one matching of one graph.
// Per-vertex arrays: tch is cleared before every pass (by the launcher); mvd is zero
// between searches; cur is meaningful only for the current search's epoch.
struct MtDev {
    int *tch;                    // [n] search of this pass that queued the vertex, 0 = none
    unsigned long long *cur;     // [n] epoch << 32 | the vertex's latest entry in that search
    unsigned *epoch;             // [1] epoch of the last search run (searches number 1, 2, ...)
    unsigned char *mvd;          // [n] moved by the current search
    int4 *lmv;                   // [n] moves of the current search: {vertex, source, target, weight}
    int *kept;                   // [n] the pass's kept movers (a vertex moves at most once in a pass)
    int *kwtab;                  // global rounds: per chunk of the start set and gain bucket, the
                                 // chunk's last entry, then the last entry before the chunk
                                 // (2 x kwchunks x kMtBuckets), then each bucket's top (kMtBuckets)
    int kwchunks;                // chunks the table holds (ceil(n / kKwChunk) + 1)
    int4 *ent;                   // [2 ecap] bucket stack entries of the current search:
                                 //   {vertex, entry below, live, target}, {block, weight, adjacency range}
    int *bpair;                  // [k] pair of the pass that the block belongs to, -1 none
    int *pa, *pb;                // [P] the pairs, in pass order
    int *cnt, *fil;              // [P] todo list lengths, fill cursors
    long long *off;              // [P + 1] todo list offsets (each padded to a power of two)
    unsigned long long *tkey;    // [scap] todo sort keys
    int *tv;                     // [scap] todo vertices
    long long *bw;               // [k] block weights, accumulated as the pass starts
    unsigned char *chg;          // [k] blocks a kept move left or entered
    MtRes *res;
    long long ecap, scap;
    int np, alpha;
    double beta;                 // ln n
    unsigned long long seed;     // option seed: todo orders and target ties derive from it
};

// Enqueues one multi-try pass over the md.np pairs already in md.pa / md.pb (md.bpair
// set): boundary counts and block weights, todo lists, their sort, and the searches.
// G is the graph as the pairwise step leaves it; the pass updates part, blockw and the
// boundary candidate list.  *nl += kernels launched.
cudaError_t launch_mt(const GraphDev &G, const MtDev &md, Ctl *ctl, int sms, cudaStream_t st, int *nl);

// Enqueues one round of the global k-way refinement (Section 2.2, set up as in
// Section 6): one k-way search from every vertex with at least `need` (1 or 2) blocks
// other than its own around it, in ascending splitmix64(rs ^ v) order; target ties
// use splitmix64(~md.seed).  Updates part and md.bw (recomputed as the round starts);
// md.res receives the round's gain, moves tried and kept, and (stopped) whether the KaSPar
// rule stopped it.  G.bl must be null.  *nl += kernels launched.
cudaError_t launch_kway_round(const GraphDev &G, const MtDev &md, Ctl *ctl, int need, unsigned long long rs,
                              int sms, cudaStream_t st, int *nl);

}  // namespace fr
