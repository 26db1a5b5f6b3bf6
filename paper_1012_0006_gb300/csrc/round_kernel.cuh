// Host-side launchers of the step kernels (internal to libflowref).
#pragma once

#include <cuda_runtime.h>

#include "fr_internal.cuh"

namespace fr {

cudaError_t launch_scan(const Work &w, int g, int n, bool vec, cudaStream_t st);
cudaError_t launch_step(const Work &w, uint32_t phases, int grid, int tpb, cudaStream_t st);
cudaError_t step_max_grid(int tpb, int nsides, int *max_blocks, int *sms);
size_t step_smem_bytes(int nsides);
// cluster_flow.cu: per-pair max flow and reachability on distributed shared memory
cudaError_t launch_cluster_flow(const Work &w, int cluster, int max_clusters, cudaStream_t st);
cudaError_t cluster_flow_capacity(int cluster, int *max_clusters);
size_t cluster_flow_smem();   // dynamic shared memory of one CTA of the cluster kernel

// prep_kernel.cu
struct PrepOut {
    long long W, maxc, totcut;
    int err, err_where;
    int npairs, nrounds;
    int maxw;            // max edge weight
    int maxwdeg;         // max weighted degree
};
// bl, blc, inb (optional, all or none): the boundary candidate list of the sweep
// (GraphDev.bl); inb needs no clearing, prep writes every entry.
cudaError_t launch_prep(const int *xadj, const int *adjncy, const int *adjwgt, const int *vwgt, const int *part,
                        int n, int nnz, int k, long long *blockw, unsigned int *qbits, PrepOut *out,
                        cudaStream_t st, int *bl = nullptr, int *blc = nullptr, int *inb = nullptr);
// The boundary scan over the candidate list of graph g (GraphDev.bl must be set).
cudaError_t launch_scan_list(const Work &w, int g, cudaStream_t st);
cudaError_t launch_check_symmetric(const int *xadj, const int *adjncy, const int *adjwgt, int n, PrepOut *out,
                                   cudaStream_t st);
cudaError_t launch_color(const unsigned int *qbits, int k, int *pair_a, int *pair_b, int *pair_round,
                         int *round_off, int *sob_round, unsigned int *used, PrepOut *out, cudaStream_t st);
cudaError_t launch_fill_pairs(PairDev *pairs, const int *pair_a, const int *pair_b, int np, int g, int mb,
                              long long Ubase, cudaStream_t st);
cudaError_t launch_gather(int *dst, const int *src, const int *idx, int n, cudaStream_t st);

}  // namespace fr
