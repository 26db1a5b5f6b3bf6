// Kernels of one refinement step: the boundary scan and the persistent step
// kernel (Sanders & Schulz, Section 4.1 and 4.1.1).
//
// A step refines a set of block-disjoint pairs (one pair, or one round of a
// matching of the quotient graph).  All pairs' corridors form one union network;
// every phase runs grid-wide over that union, so uneven corridors share the GPU
// instead of each pair waiting for its own launch.
//
//   scan_kernel      full CSR pass: boundary delta_a / delta_b of every pair
//                    (BFS level 0) and the pair cut omega(E_ab); HBM bound
//   step_kernel      cooperative persistent kernel, grid barriers between phases
//     PH_BFS         level-synchronous BFS per side, overflow level picked by a
//                    weighted radix select on vertex ids ((distance, id) order)
//     PH_LID         local ids in (graph, id) order: scan over the vertex range
//     PH_BUILD       corridor CSR with reverse arcs, INF_v border arcs
//     PH_FLOW        push-relabel (lock-free pulses, global relabel by reverse BFS
//                    from t), then excess returned to s: a maximum flow
//     PH_CUT         reachability from s / to t; MB: SCC colouring, DAG, sweeps
//     PH_EVAL        new weights, cut change, cut == flow check, acceptance
//     PH_COMMIT      apply accepted pairs to part, release dist / lid
#include <climits>

#include "fr_internal.cuh"
#include "round_kernel.cuh"
#include "step_kernel.cuh"

namespace fr {

#define FULL 0xffffffffu

// ====================================================================== scan ==

template <int TPB, bool VEC>
__global__ void __launch_bounds__(TPB) scan_kernel(Work w, int g) {
    extern __shared__ long long s_cut[];   // [npairs]
    __shared__ int s_seed[TPB];
    if (w.prev_err && __ldcg(w.prev_err)) {   // an earlier round failed: propagate, do nothing
        if (blockIdx.x == 0 && threadIdx.x == 0) { w.ctl->error = E_ABORT; w.ctl->error_where = 999; }
        return;
    }
    const GraphDev G = w.graphs[g];
    for (int i = threadIdx.x; i < w.npairs; i += TPB) s_cut[i] = 0;
    if (blockIdx.x == 0)
        for (int s = threadIdx.x; s < w.nsides; s += TPB) {
            const PairDev P = w.pairs[s >> 1];
            if (P.g == g) w.sides[s].cw = G.blockw[(s & 1) ? P.b : P.a];
        }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int wslot = threadIdx.x & ~31;
    const long long nw = (long long)gridDim.x * (TPB / 32);
    const long long gw = (long long)blockIdx.x * (TPB / 32) + (threadIdx.x >> 5);
    const int n = G.n, nnz = G.nnz;
    const int *__restrict__ xadj = G.xadj;
    const int *__restrict__ adjncy = G.adjncy;
    const int *__restrict__ part = G.part;
    const int e_end = __ldg(xadj + n);
    for (long long base = gw * 32; base < n; base += nw * 32) {
        const int v = (int)(base + lane);
        const bool valid = v < n;
        const int blk = valid ? __ldg(part + v) : -1;
        const int sd = valid ? side_of(G, blk) : -1;
        if (__ballot_sync(FULL, sd >= 0) == 0) continue;
        int pb = -2;
        if (sd >= 0) {
            const PairDev P = w.pairs[sd >> 1];
            pb = (sd & 1) ? P.a : P.b;
        }
        const int rs = valid ? __ldg(xadj + v) : e_end;
        const int re = valid ? __ldg(xadj + v + 1) : e_end;
        s_seed[threadIdx.x] = 0;
        __syncwarp();
        const int e0 = __shfl_sync(FULL, rs, 0);
        const int e1 = __shfl_sync(FULL, re, 31);
        for (int ea = VEC ? (e0 & ~3) : e0; ea < e1; ea += VEC ? 128 : 32) {
            int u4[4] = {0, 0, 0, 0};
            int q;
            if (VEC) {
                q = ea + 4 * lane;
                if (q + 3 < nnz) {
                    const int4 x = __ldg(reinterpret_cast<const int4 *>(adjncy + q));
                    u4[0] = x.x; u4[1] = x.y; u4[2] = x.z; u4[3] = x.w;
                } else {
#pragma unroll
                    for (int t = 0; t < 4; ++t) u4[t] = (q + t < nnz) ? __ldg(adjncy + q + t) : 0;
                }
            } else {
                q = ea + lane;
                u4[0] = q < e1 ? __ldg(adjncy + q) : 0;
            }
#pragma unroll
            for (int t = 0; t < (VEC ? 4 : 1); ++t) {
                const int e = q + t;
                const bool act = e >= e0 && e < e1;
                int src = 0;   // source row: the last lane whose row starts at or before e
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const int rc = __shfl_sync(FULL, rs, src + step);
                    if (rc <= e) src += step;
                }
                const int sd_s = __shfl_sync(FULL, sd, src);
                const int pb_s = __shfl_sync(FULL, pb, src);
                const int blk_s = __shfl_sync(FULL, blk, src);
                if (act && sd_s >= 0) {
                    const int pu = __ldg(part + u4[t]);
                    if (pu == pb_s) {
                        s_seed[wslot + src] = 1;
                        if (blk_s < pb_s)
                            atomicAdd((unsigned long long *)&s_cut[sd_s >> 1],
                                      (unsigned long long)__ldg(G.adjwgt + e));
                    }
                }
            }
        }
        __syncwarp();
        const bool seed = sd >= 0 && s_seed[threadIdx.x] != 0;
        if (seed) G.dist[v] = 0;
        const int pos = warp_agg_inc(&w.ctl->qcnt[0], seed);
        if (seed) {
            if (pos < w.vq_cap) {
                w.vq_v[pos] = v;
                w.vq_s[pos] = sd;
            } else {
                fail(w.ctl, E_INTERNAL, 1);
            }
        }
        warp_agg_add(seed ? &w.sides[sd].lw[0] : nullptr, seed ? (long long)__ldg(G.vwgt + v) : 0, seed);
        warp_agg_inc(seed ? &w.sides[sd].lc[0] : nullptr, seed);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < w.npairs; i += TPB)
        if (s_cut[i]) atomicAddLL(&w.pacc[i].oldcut, s_cut[i]);
}

// S1 over the boundary candidates (GraphDev.bl): each warp takes 32 listed
// vertices, spreads the adjacency rows of those in the round's blocks over its
// lanes, and a vertex is a seed when it has a neighbour in its pair's other block;
// omega(E_ab) sums the arcs seen from the lower-numbered block.  The list holds
// every vertex with a neighbour in another block, so the seeds and the cut are
// those of the full scan.
template <int TPB>
__global__ void __launch_bounds__(TPB) scan_list_kernel(Work w, int g) {
    extern __shared__ long long s_cut[];   // [npairs]
    __shared__ int s_seed[TPB];
    if (w.prev_err && __ldcg(w.prev_err)) {   // an earlier round failed: propagate, do nothing
        if (blockIdx.x == 0 && threadIdx.x == 0) { w.ctl->error = E_ABORT; w.ctl->error_where = 999; }
        return;
    }
    const GraphDev G = w.graphs[g];
    for (int i = threadIdx.x; i < w.npairs; i += TPB) s_cut[i] = 0;
    if (blockIdx.x == 0)
        for (int s = threadIdx.x; s < w.nsides; s += TPB) {
            const PairDev P = w.pairs[s >> 1];
            if (P.g == g) w.sides[s].cw = G.blockw[(s & 1) ? P.b : P.a];
        }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int wslot = threadIdx.x & ~31;
    const long long nw = (long long)gridDim.x * (TPB / 32);
    const long long gw = (long long)blockIdx.x * (TPB / 32) + (threadIdx.x >> 5);
    const int cnt = __ldcg(G.blc);
    long long n_rows = 0, n_arcs = 0;
    for (long long base = gw * 32; base < cnt; base += nw * 32) {
        const long long li = base + lane;
        int v = 0, blk = -1, sd = -1, pb = -2, rs = 0, deg = 0;
        if (li < cnt) {
            v = __ldcg(G.bl + li);
            blk = __ldg(G.part + v);
            sd = side_of(G, blk);
        }
        if (__ballot_sync(FULL, sd >= 0) == 0) continue;
        if (sd >= 0) {
            const PairDev P = w.pairs[sd >> 1];
            pb = (sd & 1) ? P.a : P.b;
            rs = __ldg(G.xadj + v);
            deg = __ldg(G.xadj + v + 1) - rs;
        }
        int incl = deg;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(FULL, incl, d);
            if (lane >= d) incl += y;
        }
        const int total = __shfl_sync(FULL, incl, 31);
        const int excl = incl - deg;
        n_rows += sd >= 0;
        n_arcs += deg;
        s_seed[threadIdx.x] = 0;
        __syncwarp();
        for (int t0 = 0; t0 < total; t0 += 32) {
            const int t = t0 + lane;
            int src = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1)
                if (__shfl_sync(FULL, incl, src + step - 1) <= t) src += step;
            const int rs_s = __shfl_sync(FULL, rs, src);
            const int ex_s = __shfl_sync(FULL, excl, src);
            const int pb_s = __shfl_sync(FULL, pb, src);
            const int blk_s = __shfl_sync(FULL, blk, src);
            const int sd_s = __shfl_sync(FULL, sd, src);
            if (t < total) {
                const int e = rs_s + (t - ex_s);
                const int u = __ldg(G.adjncy + e);
                if (__ldg(G.part + u) == pb_s) {
                    s_seed[wslot + src] = 1;
                    if (blk_s < pb_s)
                        atomicAdd((unsigned long long *)&s_cut[sd_s >> 1], (unsigned long long)__ldg(G.adjwgt + e));
                }
            }
        }
        __syncwarp();
        const bool seed = sd >= 0 && s_seed[threadIdx.x] != 0;
        if (seed) G.dist[v] = 0;
        const int pos = warp_agg_inc(&w.ctl->qcnt[0], seed);
        if (seed) {
            if (pos < w.vq_cap) {
                w.vq_v[pos] = v;
                w.vq_s[pos] = sd;
            } else {
                fail(w.ctl, E_INTERNAL, 1);
            }
        }
        warp_agg_add(seed ? &w.sides[sd].lw[0] : nullptr, seed ? (long long)__ldg(G.vwgt + v) : 0, seed);
        warp_agg_inc(seed ? &w.sides[sd].lc[0] : nullptr, seed);
    }
    n_rows = block_sum_ll<TPB>(n_rows);
    n_arcs = block_sum_ll<TPB>(n_arcs);
    if (threadIdx.x == 0) {
        if (n_rows) atomicAddLL(&w.ctl->scan_rows, n_rows);
        if (n_arcs) atomicAddLL(&w.ctl->scan_arcs, n_arcs);
        if (blockIdx.x == 0) atomicAddLL(&w.ctl->scan_listed, (long long)cnt);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < w.npairs; i += TPB)
        if (s_cut[i]) atomicAddLL(&w.pacc[i].oldcut, s_cut[i]);
}


template <int TPB>
__global__ void __launch_bounds__(TPB, 1) step_kernel(Work w, uint32_t phases) {
    extern __shared__ __align__(16) int smem[];
    if (threadIdx.x == 0) g_nsync = 0;
    __syncthreads();
    if (w.prev_err && __ldcg(w.prev_err)) return;
    if (__ldcg(&w.ctl->error)) return;   // the scan of this round failed
    StepKernel<TPB> K(w, smem);
    if (phases & PH_BFS) {
        if (!K.bfs()) return;
    } else {
        // later phases need the side decisions in shared memory
        for (int s = threadIdx.x; s < w.nsides; s += TPB) {
            K.s_state[s] = w.sides[s].state;
            K.s_lstar[s] = w.sides[s].lstar;
            K.s_T[s] = w.sides[s].T;
        }
        __syncthreads();
    }
    if (phases & PH_LID) {
        if (!K.lids()) return;
    }
    if (phases & PH_BUILD) {
        if (!K.build()) return;
    }
    if (phases & PH_FLOW) {
        if (!K.maxflow()) return;
    }
    if (phases & PH_CUT) {
        if (!K.reach()) return;
        if (w.any_mb) {
            if (!K.scc()) return;
            if (!K.sweeps()) return;
        }
    }
    if (phases & PH_EVAL) {
        if (!K.eval()) return;
    }
    if (phases & PH_COMMIT) {
        if (!K.commit()) return;
    }
    K.save_indices();
}

size_t step_smem_bytes(int nsides) {
    return (size_t)nsides * (3 * sizeof(long long) + 4 * sizeof(int)) + 16;
}

template <int TPB>
static cudaError_t launch_step_t(const Work &w, uint32_t phases, int grid, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(TPB);
    cfg.dynamicSmemBytes = step_smem_bytes(w.nsides);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = grid > 1 ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, step_kernel<TPB>, w, phases);
}

cudaError_t launch_step(const Work &w, uint32_t phases, int grid, int tpb, cudaStream_t st) {
    switch (tpb) {
        case 256: return launch_step_t<256>(w, phases, grid, st);
        case 512: return launch_step_t<512>(w, phases, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t step_max_grid(int tpb, int nsides, int *max_blocks, int *sms) {
    int dev = 0, nsm = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const size_t sm = step_smem_bytes(nsides);
    if (tpb == 256) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, step_kernel<256>, 256, sm);
    else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, step_kernel<512>, 512, sm);
    if (e != cudaSuccess) return e;
    *max_blocks = per * nsm;
    *sms = nsm;
    return cudaSuccess;
}

cudaError_t launch_scan_list(const Work &w, int g, cudaStream_t st) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const size_t sm = (size_t)w.npairs * sizeof(long long);
    scan_list_kernel<256><<<nsm * 8, 256, sm, st>>>(w, g);
    return cudaGetLastError();
}

cudaError_t launch_scan(const Work &w, int g, int n, bool vec, cudaStream_t st) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int tpb = 256;
    long long warps = ((long long)n + 31) / 32;
    long long blocks = (warps + tpb / 32 - 1) / (tpb / 32);
    long long cap = (long long)nsm * 8;
    int grid = (int)(blocks < cap ? blocks : cap);
    if (grid < 1) grid = 1;
    const size_t sm = (size_t)w.npairs * sizeof(long long);
    if (vec) scan_kernel<256, true><<<grid, tpb, sm, st>>>(w, g);
    else scan_kernel<256, false><<<grid, tpb, sm, st>>>(w, g);
    return cudaGetLastError();
}

}  // namespace fr
