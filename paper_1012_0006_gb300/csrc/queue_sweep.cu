// The queue sweep (Sanders & Schulz, Section 4.1 and 4.1.1 on every pair of a sweep;
// pairs in the order of the quotient graph's matching rounds).
//
// A round-by-round sweep lasts as long as the slowest pair of each round, and every
// round pays for grid barriers between its phases.  Here one persistent launch of
// thread-block clusters takes the pairs of the whole sweep from a counter in round
// order.  A pair (a, b) reads and writes only vertices of blocks a and b (their
// membership, weights, boundary and the cut between them), and a pair of another
// block pair moves vertices only between its own two blocks, so pair j sees exactly
// the partition it would see at the start of its round once the last earlier pair
// touching a and the last one touching b have committed.  A cluster therefore waits
// for those two pairs only (a flag written with release after their commit, read with
// acquire), then runs every phase of the pair with the cluster as the group: boundary
// scan, BFS and select, local ids, network build, max flow / residual sets / SCCs on
// distributed shared memory, DAG sweeps, evaluation and commit.  Results are those of
// the round-by-round sweep bit for bit.  Clusters take pairs in increasing order and
// wait only for smaller ones, which running clusters hold, so the waits end; each wait
// is also bounded in time.  A pair whose corridor outgrows the per-cluster workspace
// stops the sweep with E_MISFIT, and the host runs it again round by round.
#include <cooperative_groups.h>

#include <climits>

#include "cluster_flow.cuh"
#include "queue_sweep.cuh"
#include "step_kernel.cuh"

namespace fr {

namespace {

__device__ __forceinline__ int ld_acquire_i(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_i(int *p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// The per-step part of a control block (counters and triple buffers of one pair);
// the statistics (timers, pulses, arcs scanned, ...) keep adding up over the pairs.
__device__ void reset_step(Ctl *c) {
    c->bar_count = c->bar_gen = 0;
    c->abort = c->error = c->error_where = 0;
    for (int i = 0; i < 3; ++i) c->qcnt[i] = c->fcnt[i] = c->act[i] = c->chg[i] = 0;
    c->fl = c->pl = c->cl = 0;
    c->nu = c->mu = c->ncomp = c->levels = c->vq_total = c->hmax = c->remain = 0;
    c->fallback = 0;
    c->cl_next[0] = c->cl_next[1] = 0;
    c->cl_left = 0;
    c->vmin = INT_MAX;
    c->vmax = -1;
}

}  // namespace

template <int TPB>
__global__ void __launch_bounds__(TPB, 1) queue_kernel(QueueArgs q, size_t smem_bytes) {
    extern __shared__ __align__(16) char csmem[];
    __shared__ Work s_w;
    __shared__ __align__(16) int s_side[32];   // the step phases' per-side state (two sides)
    __shared__ int s_grab[2];
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank(), C = (int)cl.num_blocks();
    const QSlot &S = q.slots[blockIdx.x / C];
    ClusterGrp::init();
    if (threadIdx.x == 0) g_nsync = 0;
    cl.sync();
    for (int it = 0;; ++it) {
        // CTA 0 takes the next pair and waits for its two predecessors
        if (rank == 0 && threadIdx.x == 0) {
            int j = INT_MAX;
            if (*(volatile int *)q.gabort == 0) {
                j = atomicAdd(q.ticket, 1);
                if (j < q.np) {
                    const int pa = q.prev[2 * j], pb = q.prev[2 * j + 1];
                    const unsigned long long t_start = globaltimer();
                    unsigned int spins = 0;
                    while ((pa >= 0 && ld_acquire_i(&q.wt.pacc[pa].done) == 0) ||
                           (pb >= 0 && ld_acquire_i(&q.wt.pacc[pb].done) == 0)) {
                        if (*(volatile int *)q.gabort) { j = INT_MAX; break; }
                        if (++spins > 32) __nanosleep(200);
                        if ((spins & 255) == 0 && globaltimer() - t_start > q.wait_ns) {
                            atomicCAS(q.gabort, 0, (int)E_ABORT);
                            j = INT_MAX;
                            break;
                        }
                    }
                }
            }
            s_grab[it & 1] = j;
        }
        cl.sync();
        const int j = *(volatile int *)cl.map_shared_rank(&s_grab[it & 1], 0);
        if (j >= q.np) break;
        const PairDev P = q.wt.pairs[j];
        if (threadIdx.x == 0) {
            Work w = q.wt;
            w.graphs = S.graph;
            w.pairs = q.wt.pairs + j;
            w.sides = q.wt.sides + 2LL * j;
            w.pacc = q.wt.pacc + j;
            w.ctl = S.ctl;
            w.prev_err = nullptr;
            w.ngraphs = 1; w.npairs = 1; w.nsides = 2;
            w.vq_v = S.vq_v; w.vq_s = S.vq_s; w.cbits = S.cbits; w.sbits = S.sbits; w.sdbits = S.sdbits;
            w.gid = S.gid; w.sid = S.sid; w.off = S.off; w.head = S.head; w.rev = S.rev; w.res = S.res;
            w.cap = S.cap; w.infc = S.infc; w.fx = S.fx; w.lab = S.lab; w.rflag = S.rflag; w.color = S.color;
            w.scc = S.scc; w.vc = S.vc; w.ex = S.ex; w.border = S.border; w.side_out = S.side_out;
            w.fq0 = S.fq0; w.fq1 = S.fq1; w.cta_cnt = S.cta_cnt; w.hist = S.hist;
            w.cw = S.cw; w.cpair = S.cpair; w.cmin = S.cmin; w.cid = S.cid; w.indeg = S.indeg;
            w.outoff = S.outoff; w.outs = S.outs; w.ocur = S.ocur; w.plist = S.plist; w.pcur = S.pcur;
            w.indeg_r = S.indeg_r; w.order = S.order; w.sinkc = S.sinkc; w.hkey = S.hkey; w.hcomp = S.hcomp;
            w.sw_absd = S.sw_absd; w.sw_j = S.sw_j;
            w.cluster_mode = 1;
            w.cl_tier = 0;
            w.list_ids = 1;
            w.gabort = q.gabort;
            s_w = w;
            g_nsync = 0;
        }
        if (rank == 0) {
            if (threadIdx.x == 0) {
                reset_step(S.ctl);
                S.sob[P.a] = 0;
                S.sob[P.b] = 1;
                q.wt.pacc[j].t0 = globaltimer();
            }
            for (int i = threadIdx.x; i < 3 * 2 * kHistBins; i += TPB) S.hist[i] = 0;
        }
        bool ok = ClusterGrp::sync(s_w);
        StepKernel<TPB, ClusterGrp> K(s_w, s_side);
        ok = ok && K.scan_pair();
        ok = ok && K.bfs();
        ok = ok && K.lids();
        ok = ok && K.build();
        if (ok) {
            ClusterFlow<TPB> F(s_w, csmem);
            const bool fit = F.solve(0, csmem, smem_bytes);   // the same answer in every CTA
            if (!fit && rank == 0 && threadIdx.x == 0) fail(S.ctl, E_MISFIT, 310);
            ok = ClusterGrp::sync(s_w);                       // also collects errors of the flow
        }
        ok = ok && K.maxflow();
        if (ok && s_w.any_mb) ok = K.sweeps();
        ok = ok && K.eval();
        ok = ok && K.commit();
        if (!ok) {
            // every CTA left after the same barrier; the control block holds the reason
            if (rank == 0 && threadIdx.x == 0) {
                const int e = *(volatile int *)&S.ctl->error;
                atomicCAS(q.gabort, 0, e ? e : (int)E_ABORT);
            }
            break;
        }
        // publish the commit: every CTA's writes, then the flag with release
        __threadfence();
        cl.sync();
        if (rank == 0 && threadIdx.x == 0) {
            S.sob[P.a] = -1;
            S.sob[P.b] = -1;
            S.stat[0] += S.ctl->vq_total;
            S.stat[1] += S.ctl->nu;
            S.stat[2] += S.ctl->mu;
            S.stat[3] += 1;
            q.wt.pacc[j].t1 = globaltimer();
            __threadfence();
            st_release_i(&q.wt.pacc[j].done, 1);
        }
    }
    cl.sync();   // no CTA exits while another may still read its shared memory
}

// Dynamic shared memory of the queue kernel: the opt-in maximum per block minus its
// static shared memory (set once per process).
static int g_queue_dyn_smem = -1;

static cudaError_t queue_setup() {
    if (g_queue_dyn_smem >= 0) return cudaSuccess;
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, queue_kernel<512>);
    if (e != cudaSuccess) return e;
    const int dyn = optin - (int)fa.sharedSizeBytes - 64;
    e = cudaFuncSetAttribute(queue_kernel<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(queue_kernel<512>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    g_queue_dyn_smem = dyn;
    return cudaSuccess;
}

static cudaLaunchConfig_t queue_config(int cluster, int clusters, cudaLaunchAttribute *attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(clusters * cluster);
    cfg.blockDim = dim3(512);
    cfg.dynamicSmemBytes = (size_t)g_queue_dyn_smem;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

cudaError_t launch_queue_sweep(const QueueArgs &q, int cluster, int clusters, cudaStream_t st) {
    cudaError_t e = queue_setup();
    if (e != cudaSuccess) return e;
    if (cluster < 1 || cluster > kClusterMax || clusters < 1) return cudaErrorInvalidValue;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = queue_config(cluster, clusters, attr);
    cfg.stream = st;
    return cudaLaunchKernelEx(&cfg, queue_kernel<512>, q, (size_t)g_queue_dyn_smem);
}

cudaError_t queue_capacity(int cluster, int *max_clusters) {
    cudaError_t e = queue_setup();
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = queue_config(cluster, 64, attr);
    return cudaOccupancyMaxActiveClusters(max_clusters, queue_kernel<512>, &cfg);
}

size_t queue_smem() { return g_queue_dyn_smem > 0 ? (size_t)g_queue_dyn_smem : 0; }

// The sweep's boundary candidates bucketed by block (counting sort; order inside a
// block does not matter): counts, offsets, placement; every listed vertex records its
// block in lst (the others hold -1, set by the host).
// Per-CTA block histograms in shared memory (k <= 1024), then one global addition per
// (CTA, block): the candidates of a k-way partition hit k counters, and global atomics
// on so few addresses serialise.
__global__ void __launch_bounds__(256) qb_count_kernel(const int *bl, const int *blc, const int *part, int k,
                                                       int *cnt, int *lst) {
    __shared__ int h[1024];
    for (int x = threadIdx.x; x < k; x += blockDim.x) h[x] = 0;
    __syncthreads();
    const int m = *blc;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const int v = bl[i], x = part[v];
        atomicAdd(h + x, 1);
        lst[v] = x;
    }
    __syncthreads();
    for (int x = threadIdx.x; x < k; x += blockDim.x)
        if (h[x]) atomicAdd(cnt + x, h[x]);
}

__global__ void qb_offsets_kernel(int *cnt, int *start, int *app, int k) {
    // one CTA of 1024 threads, k <= 1024: exclusive scan of cnt into start; cnt and app
    // are cleared for the placement pass and the sweep's appends
    __shared__ int s[1024];
    const int t = threadIdx.x;
    int c = t < k ? cnt[t] : 0;
    s[t] = c;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {
        const int y = t >= d ? s[t - d] : 0;
        __syncthreads();
        s[t] += y;
        __syncthreads();
    }
    if (t < k) {
        start[t] = s[t] - c;
        cnt[t] = 0;
        app[t] = 0;
    }
    if (t == 0) start[k] = s[1023];
}

// Each CTA places one contiguous chunk of the list: it counts its chunk per block in
// shared memory, reserves a range of each block's bucket with one global addition, and
// places the entries with shared-memory offsets.  (The order inside a bucket is free:
// the pairs' boundary scans do not depend on it.)
__global__ void __launch_bounds__(256) qb_place_kernel(const int *bl, const int *blc, const int *part, int k,
                                                       int *fill, const int *start, int *sorted) {
    __shared__ int h[1024];
    const int m = *blc;
    const long long per = ((long long)m + gridDim.x - 1) / gridDim.x;
    const long long c0 = per * blockIdx.x, c1 = min((long long)m, c0 + per);
    for (int x = threadIdx.x; x < k; x += blockDim.x) h[x] = 0;
    __syncthreads();
    for (long long i = c0 + threadIdx.x; i < c1; i += blockDim.x) atomicAdd(h + part[bl[i]], 1);
    __syncthreads();
    for (int x = threadIdx.x; x < k; x += blockDim.x) h[x] = h[x] ? start[x] + atomicAdd(fill + x, h[x]) : 0;
    __syncthreads();
    for (long long i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
        const int v = bl[i];
        sorted[atomicAdd(h + part[v], 1)] = v;
    }
}

cudaError_t launch_qb_build(const int *bl, const int *blc, const int *part, int k, int *cnt, int *start, int *app,
                            int *lst, int *sorted, cudaStream_t st) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (k > 1024) return cudaErrorInvalidValue;
    qb_count_kernel<<<nsm * 4, 256, 0, st>>>(bl, blc, part, k, cnt, lst);
    qb_offsets_kernel<<<1, 1024, 0, st>>>(cnt, start, app, k);
    qb_place_kernel<<<nsm * 4, 256, 0, st>>>(bl, blc, part, k, cnt, start, sorted);
    return cudaGetLastError();
}

}  // namespace fr
