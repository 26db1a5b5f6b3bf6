// Two-way FM (TopGain) before the flows of a round's pairs: device state and launch.
#pragma once

#include <cuda_runtime.h>

#include "fr_internal.cuh"

namespace fr {

constexpr int kFmMaxBuckets = 2048;   // gain buckets per block: gains in [-1023, 1023]
constexpr int kFmSortSmem = 4096;     // boundary entries a pair sorts in shared memory

// Result of one pair's FM search (what fr_pair_result reports).
struct FmRes {
    long long cut0, wA0, wB0;   // pair cut and block weights before
    long long cut1, wA1, wB1;   // after the rollback to the best prefix
    int kept, tried;            // moves kept / made
};

// Device state of the FM searches of one round (pairs of one graph).  Per-vertex arrays
// are zero between rounds: every search clears what it touched.
struct FmDev {
    int *in, *ext;              // [n] weight to the vertex's own block / to the pair's other block
    int *ver;                   // [n] queue version: an entry is current iff its version matches
    unsigned char *flags;       // [n] kFmTouched | kFmInQ | kFmMoved
    int *vlist;                 // [n] per pair region: boundary vertices, then vertices touched later
    int *mlog;                  // [n] per pair region: vertices moved, in order
    int *blockn, *blockarcs;    // [k] vertex and arc counts of the blocks (zeroed by fm_offsets)
    long long *voff, *eoff;     // [P], [P + 1] region offsets: vertices (vlist, mlog), stack entries
    int *np, *bcnt;             // [P] pair vertex counts, boundary vertices gathered
    int *ent_v, *ent_ver, *ent_below;   // [ecap] bucket stack entries
    unsigned long long *skey;   // [scap] sort scratch for boundaries beyond shared memory
    int *sbkt, *sv;             // [scap]
    FmRes *res;                 // [P]
    const int *maxwdeg;         // max weighted degree of the graph (from prep): bounds |gain|
    long long ecap, scap;
    int permille;
};

constexpr unsigned char kFmTouched = 1, kFmInQ = 2, kFmMoved = 4;

// Enqueues the FM searches of the round described by w (one graph with k blocks,
// w.npairs pairs): block counts, pair regions, boundary gather, one CTA per pair.
// *nl += kernels launched.
cudaError_t launch_fm(const Work &w, const FmDev &f, int k, int sms, cudaStream_t st, int *nl);
size_t fm_pair_smem();

}  // namespace fr
