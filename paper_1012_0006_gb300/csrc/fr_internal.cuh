// Internal structures and device helpers of libflowref (CUDA path only).
//
// Data layout in HBM for one "step" (one flow iteration over a set of
// block-disjoint pairs, possibly from several graphs):
//   per graph  dist[n], lid[n]      BFS distance / local id, -1 when idle
//   visit list vq_v/vq_s[]          BFS entries (vertex, side), level by level
//   union network, N vertices       corridor vertices of every pair of the step,
//                                   local ids in (graph, global id) order;
//                                   off[N+1], head/rev/res/cap[M] (int32 CSR),
//                                   ex[N] int64 excess, lab[N] labels,
//                                   fx[N] flow on the vertex's s or t arc
//   sides 2p (block a_p) and 2p+1 (block b_p) of pair p
// s and t are not materialised: a border vertex carries the s->v (or v->t) arc
// of capacity INF_v = 1 + weighted degree in fx/infc.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace fr {

constexpr int kMaxSides = 2048;        // pairs per step <= 1024
constexpr int kHistBins = 256;
constexpr int kMaxGraphs = 64;         // graphs per step (serving)
constexpr unsigned int kSpinLimit = 1u << 22;   // barrier polls (a few seconds with backoff)
constexpr unsigned int kBarrierCap = 1u << 21;  // grid barriers per launch before E_ITER (a few seconds)

// Grid barriers passed by this CTA in the current launch (reset by the kernel prologue).
__shared__ unsigned int g_nsync;

enum PhaseBits : uint32_t {
    PH_BFS = 1u << 0,
    PH_LID = 1u << 1,
    PH_BUILD = 1u << 2,
    PH_FLOW = 1u << 3,
    PH_CUT = 1u << 4,
    PH_EVAL = 1u << 5,
    PH_COMMIT = 1u << 6,
    PH_ALL = 0x7fu
};

enum TimerIdx { T_BFS = 0, T_SELECT, T_LID, T_BUILD, T_FLOW1, T_GR, T_FLOW2, T_REACH, T_SCC, T_SWEEP, T_EVAL,
                T_COMMIT,
                // cluster kernel, summed over pairs: member scan and load, flow to t, return to s, reach
                T_CL_LOAD, T_CL_FLOW, T_CL_RETURN, T_CL_REACH, T_CL_SCC, T_CL_MEMBERS, T_CL_RELABEL,
                // FM step, summed over pairs: boundary sort and initial stacks, moves, rollback
                T_FM_SORT, T_FM_MOVES, T_FM_FINISH,
                // queue sweep, summed over pairs: the single pair's boundary scan
                T_QSCAN, T_COUNT };

enum SideCode { SS_EXPAND = 1, SS_SELECT = 2, SS_DONE = 3 };

// E_MISFIT: a pair's corridor outgrew the per-pair workspace of a queue sweep (visit
// list, network or a cluster's shared memory); the sweep is run again round by round.
enum ErrCode { E_OK = 0, E_INVALID = 1, E_ITER = 4, E_TOO_LARGE = 5, E_ABORT = 6, E_INTERNAL = 7, E_MISFIT = 8 };

struct GraphDev {
    const int *xadj, *adjncy, *adjwgt, *vwgt;
    int *part;           // in/out
    int *dist;           // [n]
    int *lid;            // [n]
    const int *sob;      // [k] side of each block in this step, -1 if unpaired
    long long *blockw;   // [k] c(V_i), maintained by the commit phase
    int n, nnz, k, base; // base: offset of this graph in the concatenated vertex range
    long long Lmax;
    int sbase;           // sob values are relative to this graph's first side in the step
    int ebase;           // offset of this graph's CSR entries in the concatenated arc range
    // boundary candidates (optional; NULL: the boundary scan reads every vertex): every
    // vertex with a neighbour in another block is on the list bl[0, *blc), inb[v] = 1
    // marks the listed ones; the commit phase appends moved vertices and their
    // neighbours, so the list stays a superset of the boundary during a sweep
    int *bl, *blc;
    int *inb;
};

// Side of block `blk` of graph Gr in this step, or -1.
__device__ __forceinline__ int side_of(const GraphDev &Gr, int blk) {
    const int s = __ldcg(Gr.sob + blk);   // (a queue sweep rewrites sob per pair: no read-only cache)
    return s < 0 ? -1 : s + Gr.sbase;
}

struct PairDev {
    int g, a, b, mb;
    long long Ubase;     // floor((1 + alpha*eps) W / k), host-evaluated
};

struct SideDev {
    long long cw;        // c(V_block)
    long long U;         // corridor budget of this side
    long long wcum;      // weight of the fully taken levels
    long long lw[3];     // weight of the entries of a level (triple buffer)
    long long rem;       // budget left for the overflow level
    int lc[3];           // entries of a level (triple buffer)
    int state, lstar;    // SideCode; overflow level
    int prefix, T;       // radix select prefix; threshold id (level lstar: id < T taken)
    int nseeds, pad;
};

struct PairAcc {
    long long oldcut;    // omega(E_ab) before
    long long flow;      // max flow value
    long long dcut;      // change of omega(E_ab) on corridor edges
    long long cutin;     // omega of corridor edges cut by the result (= flow)
    long long dwA;       // c(A') - c(A)
    long long d0;        // MB: c(A'_0) - c(B'_0)
    int nc, m;           // corridor vertices and arcs
    int ncomp, cbase;    // MB components and their offset in the pair-ordered list
    int best_j, best_r;
    int accept, feasible;
    int status;          // cluster max flow: 0 solved or pending, 1 left by the first cluster
                         // launch, 2 solved by the second, 3 left to the grid-wide flow
    int ord;             // the pair whose network is the ord-th largest of the round (slot ord)
    unsigned long long t0, t1;   // global timer when a cluster took the pair and finished it
    int done;            // queue sweep: 1 once the pair's commit is visible (release / acquire)
    int pad;
};

struct Ctl {
    unsigned int bar_count, bar_gen;
    int abort, error;
    int error_where, pad0;
    int qcnt[3];         // BFS level entry counts
    int fcnt[3];         // network frontier counts
    int act[3];          // pulse activity
    int chg[3];          // SCC colour changes
    int fl, pl, cl, pad1;// running indices of the triple buffers
    int nu, mu;          // union vertices / arcs
    int ncomp, levels;
    int vq_total, hmax;
    int scc_rounds, remain;
    long long pulses, relabels;
    long long timers[T_COUNT];
    long long arcs_scanned;   // BFS arcs scanned (for the bytes model)
    long long gr_arcs;        // arcs scanned by global relabels
    long long pr_arcs;        // arcs scanned by push-relabel pulses
    long long pushes;         // pushes
    long long barriers;       // grid barriers passed (CTA 0)
    long long cl_syncs;       // cluster barriers, summed over pairs
    long long cl_remote;      // cluster-held arcs whose head is in another CTA's shared memory
    long long scan_listed, scan_rows, scan_arcs;   // boundary-list scan: entries, rows in the round, arcs
    int fallback;             // pairs the cluster kernels left to the grid-wide flow
    int cl_next[2];           // next slot of the size order each cluster launch takes
    int cl_left;              // pairs the first cluster launch left (written by it only)
    int vmin, vmax;           // queue sweep: smallest and largest vertex id on the pair's visit list
    long long gaps;           // gap checks that found a gap (push-relabel), summed
    long long gap_lifted;     // vertices they lifted to hmax
    int gap_top, gap_pos;     // grid-wide gap check: largest label below hmax, smallest empty label
};

// Everything a kernel needs, passed by value.
struct Work {
    GraphDev *graphs;
    PairDev *pairs;
    SideDev *sides;
    PairAcc *pacc;
    Ctl *ctl;
    const int *prev_err;                    // error word of the previous round (NULL for the first)
    int ngraphs, npairs, nsides, total_n;   // total_n = sum of n over graphs
    // visit list
    int *vq_v, *vq_s;
    int vq_cap;
    unsigned int *cbits;         // one bit per vertex of the graphs (base + v): corridor marks, zero between phases
    // union network
    int *gid, *sid, *off, *head, *rev, *res, *cap, *infc, *fx, *lab, *rflag, *color, *scc, *vc;
    long long *ex;
    unsigned char *border, *side_out;
    int nu_cap, mu_cap;
    int *fq0, *fq1;              // frontier queues [nu_cap]
    int *cta_cnt;                // per-CTA counts for scans [grid]
    long long *hist;             // radix histograms [nsides * 256]
    // components (MB)
    long long *cw;               // [nu_cap] component weight
    int *cpair, *cmin, *cid;     // [nu_cap]
    int *indeg, *outoff, *outs, *ocur;  // [nu_cap], [nu_cap+1], [mu_cap], [nu_cap]
    int *plist, *pcur;           // [nu_cap], [npairs]
    int *indeg_r, *order, *sinkc;// [reps*nu_cap], [reps*nu_cap], [nu_cap]
    unsigned long long *hkey;    // heap keys [reps*nu_cap]
    int *hcomp;                  // heap comps [reps*nu_cap]
    long long *sw_absd;          // [npairs*reps]
    int *sw_j;                   // [npairs*reps]
    // options
    int reps, gr_interval, inner, any_mb;
    int passes, cluster_mode;    // lock-free pulse passes per barrier; 1: the cluster kernel ran the flow
    int flow_sched;              // cluster max flow: 1 level-ordered waves, otherwise lock-free pulses
    int cl_tier;                 // cluster launch: 0 every pair, 1 the pairs the first left
    int full_flow;               // 1: return every excess to s (a flow); 0: a maximum preflow
    int narrow;                  // 1: every arc capacity < 2^15 (cluster kernel packs residual and capacity sum)
    int pre_waves;               // cluster pulses: waves by levels before the first pulse
    int gap_interval;            // pulses between gap checks of push-relabel (0: none)
    unsigned long long seed;
    long long pulse_cap;
    int *crank;                  // per graph arc: rank among its row's corridor arcs (NULL: outs holds it)
    int list_ids;                // 1: queue sweep (local ids by visit order, or by id over the window
                                 //    of the visit list's ids), 0: in global id order
    unsigned int *sbits;         // queue sweep: one bit per 1,024 vertex ids (groups holding corridor bits)
    unsigned int *sdbits;        // queue sweep: one bit per vertex, set for corridor vertices of side b
    // queue sweep: the boundary candidates bucketed by block.  Block x's candidates are
    // qb_sorted[qb_start[x] .. qb_start[x + 1]) (the sweep's start) and the first
    // qb_app[x] entries of its region qb_pool[x * qb_cap ..) (appended by commits);
    // qb_lst[v] = the block whose list got v's latest entry (-1: none).  NULL: the
    // graph's global list (GraphDev.bl) serves.
    const int *qb_sorted, *qb_start;
    int *qb_app, *qb_pool, *qb_lst;
    int qb_cap;
    const int *gabort;           // queue sweep: abort flag of the whole sweep (NULL otherwise)
};

// ------------------------------------------------------------ device helpers --

__device__ __forceinline__ int ldcg(const int *p) { return __ldcg(p); }
__device__ __forceinline__ long long ldcg(const long long *p) { return __ldcg(p); }

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned int *p, unsigned int v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ long long atomicAddLL(long long *p, long long v) {
    return (long long)atomicAdd((unsigned long long *)p, (unsigned long long)v);
}

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// splitmix64(x): the first output of a splitmix64 generator seeded with x
// (Steele, Lea & Flood 2014; mixing constants as published by Vigna).
__host__ __device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    unsigned long long z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ void fail(Ctl *ctl, int code, int where) {
    if (atomicCAS(&ctl->error, 0, code) == 0) ctl->error_where = where;
    atomicExch(&ctl->abort, 1);
}

// Grid-wide barrier of a cooperatively launched (co-resident) grid.  Every wait
// is bounded: after kSpinLimit polls the CTA raises the abort flag and returns
// false; every CTA that sees the flag returns false too, so the kernel ends in
// bounded time and the host reports FR_ERR_ABORTED.  A single CTA synchronises
// with __syncthreads only.
__device__ __forceinline__ unsigned int atom_add_acq_rel(unsigned int *p, unsigned int v) {
    unsigned int old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ bool grid_sync(Ctl *ctl) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        if (++g_nsync > kBarrierCap) fail(ctl, E_ITER, 901);
        if (gridDim.x > 1) {
            // The arrival is a release (it covers the block's writes ordered before it
            // by the block barrier), the wait an acquire; the last arrival resets the
            // count before it releases the next generation.
            const unsigned int gen = ld_acquire(&ctl->bar_gen);
            const unsigned int prev = atom_add_acq_rel(&ctl->bar_count, 1u);
            if (prev == gridDim.x - 1) {
                *(volatile unsigned int *)&ctl->bar_count = 0u;
                st_release(&ctl->bar_gen, gen + 1);
            } else {
                unsigned int spins = 0;
                while (ld_acquire(&ctl->bar_gen) == gen) {
                    ++spins;
                    if ((spins & 255) == 0 && *(volatile int *)&ctl->abort) break;
                    if (spins > kSpinLimit) {
                        fail(ctl, E_ABORT, 900);
                        break;
                    }
                    if (spins > 2048) __nanosleep(256);
                }
            }
        } else {
            __threadfence_block();
        }
        if (*(volatile int *)&ctl->abort) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <int TPB>
__device__ __forceinline__ int block_exclusive_scan(int x, int *total) {
    // exclusive prefix over the block; returns this thread's offset
    __shared__ int warp_sums[TPB / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int v = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += y;
    }
    if (lane == 31) warp_sums[wid] = v;
    __syncthreads();
    if (wid == 0) {
        int s = lane < TPB / 32 ? warp_sums[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, d);
            if (lane >= d) s += y;
        }
        if (lane < TPB / 32) warp_sums[lane] = s;
    }
    __syncthreads();
    int excl = v - x + (wid > 0 ? warp_sums[wid - 1] : 0);
    if (total) *total = warp_sums[TPB / 32 - 1];
    __syncthreads();
    return excl;
}

template <int TPB>
__device__ __forceinline__ long long block_sum_ll(long long x) {
    __shared__ long long sums[TPB / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) x += __shfl_down_sync(0xffffffffu, x, d);
    if (lane == 0) sums[wid] = x;
    __syncthreads();
    long long t = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < TPB / 32; ++i) t += sums[i];
    __syncthreads();
    return t;   // valid in thread 0
}

// Add v to *p once per group of lanes that share the same address (warp-aggregated atomics).
__device__ __forceinline__ void warp_agg_add(long long *p, long long v, bool active) {
    const unsigned int mask = __ballot_sync(0xffffffffu, active);
    if (!active) return;
    const unsigned int peers = __match_any_sync(mask, (unsigned long long)p);
    const int leader = __ffs(peers) - 1;
    const int lane = threadIdx.x & 31;
    // reduce v over peers
    long long sum = 0;
    unsigned int m = peers;
    while (m) {
        int l = __ffs(m) - 1;
        m &= m - 1;
        sum += __shfl_sync(peers, v, l);
    }
    if (lane == leader && sum) atomicAddLL(p, sum);
}

__device__ __forceinline__ void warp_agg_add_i(int *p, int v, bool active) {
    const unsigned int mask = __ballot_sync(0xffffffffu, active);
    if (!active) return;
    const unsigned int peers = __match_any_sync(mask, (unsigned long long)p);
    const int leader = __ffs(peers) - 1;
    int sum = 0;
    unsigned int m = peers;
    while (m) {
        const int l = __ffs(m) - 1;
        m &= m - 1;
        sum += __shfl_sync(peers, v, l);
    }
    if ((int)(threadIdx.x & 31) == leader && sum) atomicAdd(p, sum);
}

__device__ __forceinline__ int warp_agg_inc(int *p, bool active) {
    // returns the old value + rank for active lanes (one atomic per distinct address)
    const unsigned int mask = __ballot_sync(0xffffffffu, active);
    int res = 0;
    if (active) {
        const unsigned int peers = __match_any_sync(mask, (unsigned long long)p);
        const int leader = __ffs(peers) - 1;
        const int lane = threadIdx.x & 31;
        int base = 0;
        if (lane == leader) base = atomicAdd(p, __popc(peers));
        base = __shfl_sync(peers, base, leader);
        res = base + __popc(peers & ((1u << lane) - 1u));
    }
    return res;
}

}  // namespace fr
