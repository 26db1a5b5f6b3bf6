// Multilevel V-cycle with a given partition: matching, contraction and projection
// kernels (the refinement of every level is the batched flow sweep).
#pragma once

#include <cuda_runtime.h>

#include "fr_internal.cuh"

namespace fr {

struct MlGraph {
    const int *xadj, *adjncy, *adjwgt, *vwgt;
    int n, nnz;
};

// One round of the locally dominant matching: every free vertex points at its best
// allowed edge to a free vertex (cand), or is marked dead (mate = -2) if it has none.
cudaError_t launch_ml_point(const MlGraph &g, const int *part, int k, long long W, unsigned long long seed_l, int *mate,
                            int *cand, cudaStream_t st);
// Pairs of vertices pointing at each other are matched; *progress is set if any was.
cudaError_t launch_ml_pair(int n, int *mate, const int *cand, int *progress, cudaStream_t st);
// Dead marks back to -1; *pairs += matched pairs.
cudaError_t launch_ml_finish(int n, int *mate, int *pairs, cudaStream_t st);
// Exclusive prefix sum of in[0..n) into out[0..n], out[n] = total; tmp holds
// (n + 1023) / 1024 + 1 ints.
cudaError_t launch_ml_scan(const int *in, int *out, int n, int *tmp, cudaStream_t st);
// Contraction, step 1: isrep[v] = 1 for the smaller end of a pair and for single vertices.
cudaError_t launch_ml_reps(int n, const int *mate, int *isrep, cudaStream_t st);
// Step 2 (cid = exclusive scan of isrep): cmap, coarse vertex weights, representative
// of every coarse vertex, and an upper bound of every coarse row's length.
cudaError_t launch_ml_cmap(const MlGraph &g, const int *mate, const int *cid, int *cmap, int *cvwgt, int *crep,
                           int *rowcap, cudaStream_t st);
// Step 3: coarse rows (neighbours by coarse id, parallel edges merged, the matched edge
// dropped).  count = true: cdeg[x] = row length; false: the rows at cxadj[x].
cudaError_t launch_ml_rows(const MlGraph &g, int nc, const int *mate, const int *cmap, const int *crep,
                           const int *rowcap, bool count, int *cdeg, const int *cxadj, int *cadj, int *cwgt,
                           cudaStream_t st);
// *bad = 1 unless mate is a matching (entries -1 or in-range partners pointing back).
cudaError_t launch_ml_check(int n, const int *mate, int *bad, cudaStream_t st);
// cpart[cmap[v]] = part[v]  /  part[v] = cpart[cmap[v]].
cudaError_t launch_ml_down(int n, const int *cmap, const int *part, int *cpart, cudaStream_t st);
cudaError_t launch_ml_up(int n, const int *cmap, const int *cpart, int *part, cudaStream_t st);

}  // namespace fr
