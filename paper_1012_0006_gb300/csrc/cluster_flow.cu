// Max flow, residual sets and SCCs of each pair inside one thread-block cluster, on
// distributed shared memory (Sanders & Schulz, Section 4.1: the max-flow problem of
// the B-corridor network; Section 4.1.1: residual reachability and the strongly
// connected components that represent all minimum cuts).
//
// The round's persistent kernel builds every pair's corridor network in HBM.  This
// kernel then gives each pair one cluster of C CTAs: the pair's vertices are split
// into C contiguous ranges with about equal arc counts, and every CTA loads its
// range -- labels, excess, s/t-arc flow, CSR offsets, the shared::cluster addresses
// of each arc's head label and reverse residual, residual capacities -- into its
// shared memory.  Push-relabel (lock-free pulses, or waves by levels), the exact
// relabels, the reachability sets and the SCCs then run on shared memory with the
// cluster's hardware barrier (~0.3 us) instead of a grid barrier (~3 us).  No CTA
// reads another's vertex state in these loops: updates travel as remote stores and
// relaxed reductions into the owner's memory, and each arc keeps a copy of its head's
// label that the head publishes.  Results go back to HBM for the DAG and sweep
// phases.  A pair whose network does not fit is left to a second launch with larger
// clusters, then to the grid-wide path (ctl->fallback).
#include <cooperative_groups.h>

#include <climits>

#include "cluster_flow.cuh"
#include "fr_internal.cuh"
#include "round_kernel.cuh"

namespace fr {


template <int TPB>
__global__ void __launch_bounds__(TPB, 1) cluster_flow_kernel(Work w, size_t smem_bytes) {
    extern __shared__ __align__(16) char csmem[];
    if (w.prev_err && __ldcg(w.prev_err)) return;
    if (w.cl_tier == 1 && __ldcg(&w.ctl->cl_left) == 0) return;
    ClusterFlow<TPB> K(w, csmem);
    for (int it = 0;; ++it) {
        // slot grab: CTA 0 takes it, every CTA reads it after the barrier; the two
        // parities keep a slot readable until every CTA has passed the next barrier
        if (K.rank == 0 && threadIdx.x == 0)
            K.hdr->grab[it & 1] = __ldcg(&w.ctl->error) ? INT_MAX : atomicAdd(&w.ctl->cl_next[w.cl_tier], 1);
        K.sync();
        const int j = *(volatile int *)&K.hdr0->grab[it & 1];
        if (j >= w.npairs) break;
        const int p = __ldcg(&w.pacc[j].ord);
        if (w.cl_tier == 1 && __ldcg(&w.pacc[p].status) != 1) continue;
        if (K.rank == 0 && threadIdx.x == 0) w.pacc[p].t0 = globaltimer();
        const bool done = K.solve(p, csmem, smem_bytes);
        if (K.rank == 0 && threadIdx.x == 0) {
            w.pacc[p].t1 = globaltimer();
            if (w.cl_tier == 0) {
                if (!done) {
                    atomicAdd(&w.ctl->fallback, 1);
                    atomicAdd(&w.ctl->cl_left, 1);
                    w.pacc[p].status = 1;
                }
            } else {
                w.pacc[p].status = done ? 2 : 3;
                if (done) atomicAdd(&w.ctl->fallback, -1);
            }
        }
    }
    K.sync();   // no CTA exits while another may still read its shared memory (the last slot)
}

// Dynamic shared memory of the cluster kernel: the opt-in maximum per block minus
// its static shared memory (set once per process).
static int g_cluster_dyn_smem = -1;

static cudaError_t cluster_setup() {
    if (g_cluster_dyn_smem >= 0) return cudaSuccess;
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, cluster_flow_kernel<512>);
    if (e != cudaSuccess) return e;
    const int dyn = optin - (int)fa.sharedSizeBytes - 64;
    e = cudaFuncSetAttribute(cluster_flow_kernel<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(cluster_flow_kernel<512>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    g_cluster_dyn_smem = dyn;
    return cudaSuccess;
}

cudaError_t launch_cluster_flow(const Work &w, int cluster, int max_clusters, cudaStream_t st) {
    const int tpb = 512;
    cudaError_t e0 = cluster_setup();
    if (e0 != cudaSuccess) return e0;
    const size_t smem = (size_t)g_cluster_dyn_smem;
    int nclusters = w.npairs < max_clusters ? w.npairs : max_clusters;
    if (nclusters < 1) nclusters = 1;
    if (cluster < 1 || cluster > kClusterMax) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nclusters * cluster);
    cfg.blockDim = dim3(tpb);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, cluster_flow_kernel<512>, w, smem);
}

size_t cluster_flow_smem() { return g_cluster_dyn_smem > 0 ? (size_t)g_cluster_dyn_smem : 0; }

cudaError_t cluster_flow_capacity(int cluster, int *max_clusters) {
    cudaError_t e = cluster_setup();
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cluster * 64);
    cfg.blockDim = dim3(512);
    cfg.dynamicSmemBytes = (size_t)g_cluster_dyn_smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(max_clusters, cluster_flow_kernel<512>, &cfg);
}

}  // namespace fr
