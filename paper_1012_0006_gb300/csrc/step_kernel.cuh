// The phases of one refinement step (Sanders & Schulz, Section 4.1 and 4.1.1) as a
// struct of device functions over a group of CTAs: the whole grid of the cooperative
// step kernel (GridGrp, grid barriers), or one thread-block cluster of the queue sweep
// (ClusterGrp, hardware cluster barriers).  Every phase strides its work over the
// group's threads and synchronises the group between dependent passes.
#pragma once

#include <climits>
#include <cooperative_groups.h>

#include "fr_internal.cuh"

namespace fr {

#ifndef FULL
#define FULL 0xffffffffu
#endif

// ---------------------------------------------------------------- groups --

// The whole grid of a cooperative launch.
struct GridGrp {
    __device__ static int rank() { return (int)blockIdx.x; }
    __device__ static int count() { return (int)gridDim.x; }
    __device__ static bool sync(const Work &w) { return grid_sync(w.ctl); }
};

// Rotating slots of the cluster barrier's abort vote (CTA 0's copy counts).
__shared__ int g_cvote[3];
__shared__ int g_cvrot;

__device__ __forceinline__ unsigned grp_cta_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned grp_map_rank(unsigned a, int r) {
    unsigned x;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(x) : "r"(a), "r"(r));
    return x;
}

// One thread-block cluster.  A barrier is also a vote: each CTA reports whether it saw
// its pair's error flag or the sweep's abort flag before arriving, and every CTA leaves
// with the OR of the votes, so all CTAs of the cluster take the same exit after the
// same barrier (a cluster barrier cannot time out).  The votes rotate over three slots
// in CTA 0: slot r + 1 was last read before barrier r - 1, so CTA 0 clears it before
// arriving at barrier r.
struct ClusterGrp {
    __device__ static int rank() { return (int)cooperative_groups::this_cluster().block_rank(); }
    __device__ static int count() { return (int)cooperative_groups::this_cluster().num_blocks(); }
    // every CTA calls this once before the first sync
    __device__ static void init() {
        if (threadIdx.x < 3) g_cvote[threadIdx.x] = 0;
        if (threadIdx.x == 0) g_cvrot = 0;
    }
    __device__ static bool sync(const Work &w) {
        __shared__ int s_ok;
        __syncthreads();
        const int rot = g_cvrot;
        const unsigned slot = grp_map_rank(grp_cta_addr(&g_cvote[rot]), 0);
        if (threadIdx.x == 0) {
            ++g_nsync;
            int f = *(volatile int *)&w.ctl->abort;
            if (w.gabort) f |= *(volatile int *)w.gabort;
            if (f) asm volatile("red.shared::cluster.or.b32 [%0], %1;" ::"r"(slot), "r"(1) : "memory");
            if (rank() == 0) g_cvote[(rot + 1) % 3] = 0;
        }
        cooperative_groups::this_cluster().sync();
        if (threadIdx.x == 0) {
            int v;
            asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(slot) : "memory");
            s_ok = v == 0;
            g_cvrot = (rot + 1) % 3;
        }
        __syncthreads();
        return s_ok != 0;
    }
};

// ============================================================ step helpers ==

template <class Grp>
struct GridT {
    long long tid, size, warp, nwarps;
    __device__ GridT(int tpb) {
        tid = (long long)Grp::rank() * tpb + threadIdx.x;
        size = (long long)Grp::count() * tpb;
        warp = tid >> 5;
        nwarps = size >> 5;
    }
};

// Warp-cooperative walk over the arcs of many rows: each warp takes R consecutive
// rows, R = ceil(rows / warps) clamped to [1, 32], so that small frontiers still
// spread over every warp; the warp flattens its rows' arc ranges and visits 32
// arcs per iteration with all lanes converged (appends aggregate per warp).
template <class Grp, class RowF, class ArcF>
__device__ __forceinline__ void warp_rows(long long begin, long long end, const GridT<Grp> &G, RowF row, ArcF arc) {
    const int lane = threadIdx.x & 31;
    long long R = (end - begin + G.nwarps - 1) / G.nwarps;
    R = R < 1 ? 1 : (R > 32 ? 32 : R);
    for (long long b = begin + G.warp * R; b < end; b += G.nwarps * R) {
        const long long idx = b + lane;
        int rs = 0, deg = 0, ctx = 0;
        if (lane < R && idx < end) row(idx, rs, deg, ctx);
        int incl = deg;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(FULL, incl, d);
            if (lane >= d) incl += y;
        }
        const int total = __shfl_sync(FULL, incl, 31);
        const int excl = incl - deg;
        for (int t0 = 0; t0 < total; t0 += 32) {
            const int t = t0 + lane;
            int src = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1)
                if (__shfl_sync(FULL, incl, src + step - 1) <= t) src += step;
            const int rs_s = __shfl_sync(FULL, rs, src);
            const int ex_s = __shfl_sync(FULL, excl, src);
            const int ctx_s = __shfl_sync(FULL, ctx, src);
            const bool valid = t < total;
            arc(valid, rs_s + (t - ex_s), ctx_s);
        }
    }
}

// Append a lane's element to a queue with one atomic per warp.  Returns the slot or -1.
__device__ __forceinline__ int warp_append(int *counter, bool want) {
    const unsigned int m = __ballot_sync(FULL, want);
    if (m == 0) return -1;
    const int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == __ffs(m) - 1) base = atomicAdd(counter, __popc(m));
    base = __shfl_sync(FULL, base, __ffs(m) - 1);
    return want ? base + __popc(m & ((1u << lane) - 1u)) : -1;
}

template <class Grp>
__device__ __forceinline__ void timer_mark(const Work &w, unsigned long long &t0, int idx) {
    if (Grp::rank() == 0 && threadIdx.x == 0) {
        unsigned long long t1 = globaltimer();
        w.ctl->timers[idx] += (long long)(t1 - t0);
        t0 = t1;
    }
}

// Ranks of elements in index order over [0, N): val(x) >= 0 is the element's
// count; emit(x, offset) is called for every x (offset = exclusive prefix).
// Chunked per CTA: count pass, barrier, prefix of CTA totals, write pass.
template <int TPB, class Grp, class ValF, class EmitF>
__device__ bool grid_scan(const Work &w, long long N, ValF val, EmitF emit, long long *total_out) {
    const int gr = Grp::rank(), gn = Grp::count();
    const long long per = ((N + gn - 1) / gn + TPB - 1) / TPB * TPB;
    const long long c0 = per * gr, c1 = min(N, c0 + per);
    long long mine = 0;
    for (long long x = c0 + threadIdx.x; x < c1; x += TPB) mine += val(x);
    long long tot = block_sum_ll<TPB>(mine);
    if (threadIdx.x == 0) w.cta_cnt[gr] = (int)tot;
    if (!Grp::sync(w)) return false;
    long long before = 0, all = 0;
    for (int b = threadIdx.x; b < gn; b += TPB) {
        const long long c = __ldcg(&w.cta_cnt[b]);
        all += c;
        if (b < gr) before += c;
    }
    __shared__ long long s_before, s_all;
    long long bsum = block_sum_ll<TPB>(before);
    long long asum = block_sum_ll<TPB>(all);
    if (threadIdx.x == 0) { s_before = bsum; s_all = asum; }
    __syncthreads();
    long long run = s_before;
    for (long long x0 = c0; x0 < c1; x0 += TPB) {
        const long long x = x0 + threadIdx.x;
        const int v = x < c1 ? val(x) : 0;
        int tile_total;
        const int excl = block_exclusive_scan<TPB>(v, &tile_total);
        if (x < c1) emit(x, run + excl);
        run += tile_total;
    }
    if (total_out) *total_out = s_all;
    return true;
}

// ============================================================== step kernel ==

// Visit-list offsets of the BFS levels of this launch (kLvlCap levels; deeper levels are
// not recorded and the select then scans the whole list).
constexpr int kLvlCap = 64;
__shared__ long long g_lvl[kLvlCap + 2];

template <int TPB, class Grp = GridGrp>
struct StepKernel {
    const Work &w;
    const GridT<Grp> G;
    int fl, pl, cl;   // running indices of the triple-buffered counters (identical in every CTA)
    long long vtotal; // BFS entries in the visit list
    int *s_state, *s_lstar, *s_T;
    long long *s_wcum, *s_rem, *s_lw;
    int *s_lc;

    __device__ StepKernel(const Work &w_, int *smem) : w(w_), G(TPB) {
        const int ns = w.nsides;
        fl = w.ctl->fl;
        pl = w.ctl->pl;
        cl = w.ctl->cl;
        vtotal = w.ctl->vq_total;
        s_wcum = reinterpret_cast<long long *>(smem);
        s_rem = s_wcum + ns;
        s_lw = s_rem + ns;
        s_state = reinterpret_cast<int *>(s_lw + ns);
        s_lstar = s_state + ns;
        s_T = s_lstar + ns;
        s_lc = s_T + ns;
    }

    // U_side = max(0, Ubase - c(other block))
    __device__ long long budget(int s) const {
        const long long U = w.pairs[s >> 1].Ubase - __ldcg(&w.sides[s ^ 1].cw);
        return U < 0 ? 0 : U;
    }

    __device__ void save_indices() const {
        if (G.tid == 0) {
            w.ctl->fl = fl;
            w.ctl->pl = pl;
            w.ctl->cl = cl;
            w.ctl->barriers += g_nsync;
        }
    }

    // the id range of the visit list (queue sweep; the whole warp calls it)
    __device__ __forceinline__ void track_ids(bool got, int v) {
        const int mn = __reduce_min_sync(FULL, got ? v : INT_MAX);
        const int mx = __reduce_max_sync(FULL, got ? v : -1);
        if ((threadIdx.x & 31) == 0 && mx >= 0) {
            atomicMin(&w.ctl->vmin, mn);
            atomicMax(&w.ctl->vmax, mx);
        }
    }

    // ------------------------------------------- boundary of a single pair --
    // S1 for the one pair of this step (a queue sweep runs each pair on its own, as
    // soon as the pairs before it that share a block have committed): the candidates
    // of blocks a and b (the per-block lists, or else the graph's list) are scanned
    // like the round's boundary scan does, a vertex with a neighbour in the other
    // block is a seed (BFS level 0), and omega(E_ab) sums the arcs seen from the
    // lower-numbered block.  A list entry whose vertex has left the block since is
    // skipped by its block test, and the seed mark is taken with a compare-and-swap,
    // so a vertex listed twice counts once.
    __device__ bool scan_pair() {
        unsigned long long t_scan = globaltimer();
        __shared__ int s_seed[TPB];
        __shared__ long long s_rcut[TPB];
        const GraphDev &Gr = w.graphs[0];
        const PairDev P = w.pairs[0];
        if (G.tid == 0) {
            w.sides[0].cw = __ldcg(Gr.blockw + P.a);
            w.sides[1].cw = __ldcg(Gr.blockw + P.b);
        }
        const int lane = threadIdx.x & 31;
        const int wslot = threadIdx.x & ~31;
        // the entries: the graph's list, or four segments (initial and appended
        // candidates of block a, then of block b) laid end to end
        int seg[4] = {0, 0, 0, 0};
        const int *segp[4] = {nullptr, nullptr, nullptr, nullptr};
        int cnt;
        if (w.qb_sorted) {
            const int blks[2] = {P.a, P.b};
            for (int h = 0; h < 2; ++h) {
                const int x = blks[h];
                const int s0 = __ldcg(w.qb_start + x);
                seg[2 * h] = __ldcg(w.qb_start + x + 1) - s0;
                segp[2 * h] = w.qb_sorted + s0;
                seg[2 * h + 1] = min(__ldcg(w.qb_app + x), w.qb_cap);
                segp[2 * h + 1] = w.qb_pool + (long long)x * w.qb_cap;
            }
            cnt = seg[0] + seg[1] + seg[2] + seg[3];
        } else {
            cnt = __ldcg(Gr.blc);
        }
        long long n_rows = 0, n_arcs = 0, cut = 0;
        for (long long base = G.warp * 32; base < cnt; base += G.nwarps * 32) {
            const long long li = base + lane;
            int v = 0, blk = -1, sd = -1, pb = -2, rs = 0, deg = 0;
            if (li < cnt) {
                if (w.qb_sorted) {
                    int q = (int)li, h = 0;
                    while (q >= seg[h]) q -= seg[h++];
                    v = __ldcg(segp[h] + q);
                } else {
                    v = __ldcg(Gr.bl + li);
                }
                if (v >= 0 && v < Gr.n) {
                    blk = __ldcg(Gr.part + v);
                    sd = blk == P.a ? 0 : (blk == P.b ? 1 : -1);
                }
            }
            if (__ballot_sync(FULL, sd >= 0) == 0) continue;
            if (sd >= 0) {
                pb = sd ? P.a : P.b;
                rs = __ldg(Gr.xadj + v);
                deg = __ldg(Gr.xadj + v + 1) - rs;
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
            s_rcut[threadIdx.x] = 0;
            __syncwarp();
            // four chunks of 32 arcs per step, their loads issued together
            for (int t0 = 0; t0 < total; t0 += 128) {
                int e4[4], src4[4], pb4[4], blk4[4], u4[4], pu4[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int t = t0 + 32 * q + lane;
                    int src = 0;
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1)
                        if (__shfl_sync(FULL, incl, src + step - 1) <= t) src += step;
                    const int rs_s = __shfl_sync(FULL, rs, src);
                    const int ex_s = __shfl_sync(FULL, excl, src);
                    pb4[q] = __shfl_sync(FULL, pb, src);
                    blk4[q] = __shfl_sync(FULL, blk, src);
                    src4[q] = src;
                    e4[q] = t < total ? rs_s + (t - ex_s) : -1;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) u4[q] = e4[q] >= 0 ? __ldg(Gr.adjncy + e4[q]) : 0;
#pragma unroll
                for (int q = 0; q < 4; ++q) pu4[q] = e4[q] >= 0 ? __ldcg(Gr.part + u4[q]) : -3;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (e4[q] >= 0 && pu4[q] == pb4[q]) {
                        s_seed[wslot + src4[q]] = 1;
                        if (blk4[q] < pb4[q]) atomicAdd((unsigned long long *)&s_rcut[wslot + src4[q]],
                                                        (unsigned long long)__ldg(Gr.adjwgt + e4[q]));
                    }
                }
            }
            __syncwarp();
            const bool seed = sd >= 0 && s_seed[threadIdx.x] != 0 && atomicCAS(Gr.dist + v, -1, 0) == -1;
            if (seed) cut += s_rcut[threadIdx.x];
            if (w.list_ids) track_ids(seed, v);
            const int pos = warp_agg_inc(&w.ctl->qcnt[0], seed);
            if (seed) {
                if (pos < w.vq_cap) {
                    w.vq_v[pos] = v;
                    w.vq_s[pos] = sd;
                } else {
                    fail(w.ctl, E_MISFIT, 1);
                }
            }
            warp_agg_add(seed ? &w.sides[sd].lw[0] : nullptr, seed ? (long long)__ldg(Gr.vwgt + v) : 0, seed);
            warp_agg_inc(seed ? &w.sides[sd].lc[0] : nullptr, seed);
        }
        n_rows = block_sum_ll<TPB>(n_rows);
        n_arcs = block_sum_ll<TPB>(n_arcs);
        cut = block_sum_ll<TPB>(cut);
        if (threadIdx.x == 0) {
            if (n_rows) atomicAddLL(&w.ctl->scan_rows, n_rows);
            if (n_arcs) atomicAddLL(&w.ctl->scan_arcs, n_arcs);
            if (cut) atomicAddLL(&w.pacc[0].oldcut, cut);
            if (Grp::rank() == 0) atomicAddLL(&w.ctl->scan_listed, (long long)cnt);
        }
        if (!Grp::sync(w)) return false;
        timer_mark<Grp>(w, t_scan, T_QSCAN);
        return true;
    }

    // ---------------------------------------------------------------- BFS --
    __device__ bool bfs() {
        Ctl *ctl = w.ctl;
        const int ns = w.nsides;
        unsigned long long t0 = globaltimer();
        for (int s = threadIdx.x; s < ns; s += TPB) {
            s_state[s] = SS_EXPAND;
            s_lstar[s] = INT_MAX;
            s_wcum[s] = 0;
            s_rem[s] = 0;
            s_T[s] = INT_MAX;
        }
        __syncthreads();
        int level = 0;
        long long base = 0, arcs = 0;
        for (;;) {
            const int cnt = __ldcg(&ctl->qcnt[level % 3]);
            bool any = false;
            for (int s = threadIdx.x; s < ns; s += TPB) {
                SideDev *S = &w.sides[s];
                if (s_state[s] == SS_EXPAND) {
                    const long long U = budget(s);
                    const long long W = __ldcg(&S->lw[level % 3]);
                    const int c = __ldcg(&S->lc[level % 3]);
                    if (c == 0) {
                        s_state[s] = SS_DONE;                 // BFS exhausted its block
                    } else if (s_wcum[s] + W <= U) {
                        s_wcum[s] += W;                       // whole level fits
                        any = true;
                    } else {
                        s_state[s] = SS_SELECT;               // overflow level: take an id prefix
                        s_lstar[s] = level;
                        s_rem[s] = U - s_wcum[s];
                    }
                    if (Grp::rank() == 0) S->U = U;
                }
                if (Grp::rank() == 0) {
                    S->lw[(level + 2) % 3] = 0;
                    S->lc[(level + 2) % 3] = 0;
                }
                s_lw[s] = 0;
                s_lc[s] = 0;
            }
            if (Grp::rank() == 0 && threadIdx.x == 0) ctl->qcnt[(level + 2) % 3] = 0;
            if (threadIdx.x == 0 && level <= kLvlCap) {
                g_lvl[level] = base;
                g_lvl[level + 1] = base + cnt;
            }
            any = __syncthreads_or(any);
            if (!any) {
                vtotal = base + cnt;
                if (Grp::rank() == 0 && threadIdx.x == 0) {
                    ctl->vq_total = (int)vtotal;
                    ctl->levels = level + 1;
                }
                break;
            }
            const long long next_base = base + cnt;
            int *qc = &ctl->qcnt[(level + 1) % 3];
            const int nlev = level + 1;
            warp_rows(
                base, base + cnt, G,
                [&](long long e, int &rs, int &deg, int &ctx) {
                    const int v = w.vq_v[e], s = w.vq_s[e];
                    if (s_state[s] != SS_EXPAND) return;
                    const GraphDev &Gr = w.graphs[w.pairs[s >> 1].g];
                    rs = __ldg(Gr.xadj + v);
                    deg = __ldg(Gr.xadj + v + 1) - rs;
                    ctx = s;
                },
                [&](bool valid, int e, int s) {
                    bool got = false;
                    int u = 0;
                    if (valid) {
                        const PairDev P = w.pairs[s >> 1];
                        const GraphDev &Gr = w.graphs[P.g];
                        const int blk = (s & 1) ? P.b : P.a;
                        u = __ldg(Gr.adjncy + e);
                        if (__ldcg(Gr.part + u) == blk && __ldcg(Gr.dist + u) == -1)
                            got = atomicCAS(Gr.dist + u, -1, nlev) == -1;
                        ++arcs;
                    }
                    const int slot = warp_append(qc, got);
                    if (w.list_ids) track_ids(got, u);
                    if (got) {
                        const long long idx = next_base + slot;
                        if (idx < w.vq_cap) {
                            w.vq_v[idx] = u;
                            w.vq_s[idx] = s;
                        } else {
                            fail(w.ctl, E_MISFIT, 10);
                        }
                        const GraphDev &Gr = w.graphs[w.pairs[s >> 1].g];
                        atomicAdd((unsigned long long *)&s_lw[s], (unsigned long long)__ldg(Gr.vwgt + u));
                        atomicAdd(&s_lc[s], 1);
                    }
                });
            __syncthreads();
            for (int s = threadIdx.x; s < ns; s += TPB) {
                if (s_lw[s]) atomicAddLL(&w.sides[s].lw[nlev % 3], s_lw[s]);
                if (s_lc[s]) atomicAdd(&w.sides[s].lc[nlev % 3], s_lc[s]);
            }
            base = next_base;
            if (!Grp::sync(w)) return false;
            level = nlev;
            if (level > w.total_n + 1) {
                fail(ctl, E_ITER, 11);
                return false;
            }
        }
        if (arcs) atomicAdd((unsigned long long *)&ctl->arcs_scanned, (unsigned long long)arcs);
        timer_mark<Grp>(w, t0, T_BFS);
        return select(t0);
    }

    // Weighted radix select per SELECT side: the overflow vertex v* is the first
    // vertex of level lstar, in id order, at which the running weight exceeds rem;
    // vertices of that level with id < v* are taken.
    __device__ bool select(unsigned long long &t0) {
        Ctl *ctl = w.ctl;
        const int ns = w.nsides;
        bool anysel = false;
        for (int s = threadIdx.x; s < ns; s += TPB) anysel |= s_state[s] == SS_SELECT;
        anysel = __syncthreads_or(anysel);
        const long long total = vtotal;
        if (anysel) {
            // the overflow levels' entries: the visit list is in level order
            int lmin = INT_MAX, lmax = -1;
            for (int s = threadIdx.x; s < ns; s += TPB) {
                s_T[s] = 0;   // prefix being built
                if (s_state[s] == SS_SELECT) { lmin = min(lmin, s_lstar[s]); lmax = max(lmax, s_lstar[s]); }
            }
            lmin = __reduce_min_sync(FULL, lmin);
            lmax = __reduce_max_sync(FULL, lmax);
            __shared__ int s_lmm[2];
            if (threadIdx.x == 0) { s_lmm[0] = INT_MAX; s_lmm[1] = -1; }
            __syncthreads();
            if ((threadIdx.x & 31) == 0) { atomicMin(&s_lmm[0], lmin); atomicMax(&s_lmm[1], lmax); }
            __syncthreads();
            const bool rec = s_lmm[1] < kLvlCap;
            const long long e_lo = rec ? g_lvl[s_lmm[0]] : 0, e_hi = rec ? g_lvl[s_lmm[1] + 1] : total;
            // histograms are triple buffered: pass p fills buffer p % 3 (cleared by the
            // host or during pass p - 2) and clears buffer (p + 1) % 3, last read in pass p - 2
            const long long hsz = (long long)ns * kHistBins;
            // ids are below total_n: the digits above its highest byte are zero for every
            // vertex, and those passes are skipped
            const int first = w.total_n <= (1 << 8) ? 3 : w.total_n <= (1 << 16) ? 2 : w.total_n <= (1 << 24) ? 1 : 0;
            for (int pass = 0; pass < 4 - first; ++pass) {
                const int shift = 24 - 8 * (pass + first);
                long long *hist = w.hist + (pass % 3) * hsz;
                if (pass >= 1) {
                    long long *nxt = w.hist + ((pass + 1) % 3) * hsz;
                    for (long long i = G.tid; i < hsz; i += G.size) nxt[i] = 0;
                }
                for (long long e = e_lo + G.tid; e < e_hi; e += G.size) {
                    const int v = w.vq_v[e], s = w.vq_s[e];
                    if (s_state[s] != SS_SELECT) continue;
                    const GraphDev &Gr = w.graphs[w.pairs[s >> 1].g];
                    if (__ldcg(Gr.dist + v) != s_lstar[s]) continue;
                    if (pass > 0 && ((unsigned)v >> (shift + 8)) != ((unsigned)s_T[s] >> (shift + 8))) continue;
                    const int digit = ((unsigned)v >> shift) & 255;
                    atomicAdd((unsigned long long *)&hist[(long long)s * kHistBins + digit],
                              (unsigned long long)__ldg(Gr.vwgt + v));
                }
                if (!Grp::sync(w)) return false;
                // every CTA picks the same bucket for every side (one warp per side)
                {
                    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
                    for (int s = wid; s < ns; s += TPB / 32) {
                        if (s_state[s] != SS_SELECT) continue;
                        const long long *hs = hist + (long long)s * kHistBins + lane * 8;
                        long long hv[8], lsum = 0;
#pragma unroll
                        for (int u = 0; u < 8; ++u) { hv[u] = __ldcg(hs + u); lsum += hv[u]; }
                        long long incl = lsum;
#pragma unroll
                        for (int dd = 1; dd < 32; dd <<= 1) {
                            const long long y = __shfl_up_sync(FULL, incl, dd);
                            if (lane >= dd) incl += y;
                        }
                        const long long rem = s_rem[s];
                        const unsigned int over = __ballot_sync(FULL, incl > rem);
                        if (over == 0) {   // cannot happen: the level's weight exceeds rem
                            if (lane == 0) fail(ctl, E_INTERNAL, 20);
                            continue;
                        }
                        const int L = __ffs(over) - 1;
                        if (lane == L) {
                            long long acc = incl - lsum;
                            int b = 0;
                            for (; b < 8; ++b) {
                                if (acc + hv[b] > rem) break;
                                acc += hv[b];
                            }
                            s_rem[s] = rem - acc;
                            s_T[s] |= (L * 8 + b) << shift;
                        }
                    }
                }
                __syncthreads();
            }
        }
        if (Grp::rank() == 0) {
            for (int s = threadIdx.x; s < ns; s += TPB) {
                SideDev *S = &w.sides[s];
                S->state = s_state[s];
                S->lstar = s_lstar[s];
                S->T = s_state[s] == SS_SELECT ? s_T[s] : INT_MAX;
                S->wcum = s_wcum[s];
                S->rem = s_rem[s];
            }
        }
        for (int s = threadIdx.x; s < ns; s += TPB)
            if (s_state[s] != SS_SELECT) s_T[s] = INT_MAX;
        __syncthreads();
        timer_mark<Grp>(w, t0, T_SELECT);
        return true;
    }

    __device__ bool in_corridor(const GraphDev &Gr, int v) const {
        const int d = __ldcg(Gr.dist + v);
        if (d < 0) return false;
        const int s = side_of(Gr, __ldcg(Gr.part + v));
        if (s < 0) return false;
        const int ls = s_lstar[s];
        return d < ls || (d == ls && v < s_T[s]);
    }

    __device__ int graph_of(long long x) const {   // last graph whose base <= x
        int lo = 0, hi = w.ngraphs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (w.graphs[mid].base <= x) lo = mid; else hi = mid - 1;
        }
        return lo;
    }

    // -------------------------------------------------------------- local ids --
    // With w.list_ids (the queue sweep: one pair, a cluster): the corridor vertices are
    // numbered in the order of the visit list, by one scan over its entries -- work in
    // the size of the BFS, not of the graph.  Nothing else depends on the numbering:
    // cuts, residual sets and SCCs are sets, an SCC's key is the smallest global id
    // of its members (computed in sweeps), and every edge is counted once by comparing
    // its ends' ids.
    __device__ bool lids_list() {
        unsigned long long t0 = globaltimer();
        const GraphDev &Gr = w.graphs[0];
        long long nu = 0;
        bool ok = grid_scan<TPB, Grp>(
            w, vtotal, [&](long long e) -> int { return in_corridor(Gr, w.vq_v[e]) ? 1 : 0; },
            [&](long long e, long long off) {
                const int v = w.vq_v[e];
                if (!in_corridor(Gr, v)) return;
                if (off < w.nu_cap) {
                    Gr.lid[v] = (int)off;
                    w.gid[off] = v;
                    w.sid[off] = w.vq_s[e];
                } else {
                    fail(w.ctl, E_MISFIT, 31);
                }
            },
            &nu);
        if (!ok) return false;
        if (Grp::rank() == 0 && threadIdx.x == 0) {
            w.ctl->nu = (int)nu;
            w.ctl->hmax = (int)nu + 2;
        }
        if (!Grp::sync(w)) return false;
        timer_mark<Grp>(w, t0, T_LID);
        return true;
    }

    // Local ids in id order for one pair (queue sweep) from a two-level bitmap: a
    // corridor vertex sets its bit in cbits (and in sdbits if it is on side b) and its
    // group's bit (1,024 ids) in sbits; the scan then reads only the words of marked
    // groups in the window [g0, g1).
    __device__ bool lids_window(long long g0, long long g1) {
        unsigned long long t0 = globaltimer();
        const GraphDev &Gr = w.graphs[0];
        for (long long e = G.tid; e < vtotal; e += G.size) {
            const int v = w.vq_v[e];
            if (in_corridor(Gr, v)) {
                atomicOr(&w.cbits[v >> 5], 1u << (v & 31));
                if (w.vq_s[e]) atomicOr(&w.sdbits[v >> 5], 1u << (v & 31));   // side b
                const unsigned gb = 1u << ((v >> 10) & 31);   // (most groups are marked already:
                if (!(__ldcg(&w.sbits[v >> 15]) & gb)) atomicOr(&w.sbits[v >> 15], gb);   // no atomic)
            }
        }
        if (!Grp::sync(w)) return false;
        // a warp per group: lane z reads word z (coalesced); the group's count goes to
        // gcnt, a scan over the groups gives their offsets, and the warp numbers the
        // group's vertices in id order
        auto marked = [&](long long g) { return (__ldcg(&w.sbits[g >> 5]) >> (g & 31)) & 1u; };
        const int lane = threadIdx.x & 31;
        int *gcnt = w.fq0;   // (free until the network exists; the caller checks the size)
        for (long long g = g0 + G.warp; g < g1; g += G.nwarps) {
            int c = 0;
            if (marked(g)) c = __popc(__ldcg(&w.cbits[g * 32 + lane]));
            c = __reduce_add_sync(FULL, c);
            if (lane == 0) gcnt[g - g0] = c;
        }
        if (!Grp::sync(w)) return false;
        long long nu = 0;
        bool ok = grid_scan<TPB, Grp>(
            w, g1 - g0, [&](long long gr) -> int { return __ldcg(&gcnt[gr]); },
            [&](long long gr, long long off) { w.fq1[gr] = (int)off; }, &nu);
        if (!ok) return false;
        if (nu > w.nu_cap && G.tid == 0) fail(w.ctl, E_MISFIT, 32);
        if (!Grp::sync(w)) return false;
        if (nu <= w.nu_cap) {
            for (long long g = g0 + G.warp; g < g1; g += G.nwarps) {
                if (!__ldcg(&gcnt[g - g0])) continue;   // (the same in every lane)
                const long long x = g * 32 + lane;
                unsigned m = __ldcg(&w.cbits[x]);
                const unsigned sd = __ldcg(&w.sdbits[x]);
                int incl = __popc(m);
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const int y = __shfl_up_sync(FULL, incl, d);
                    if (lane >= d) incl += y;
                }
                int off = __ldcg(&w.fq1[g - g0]) + incl - __popc(m);
                if (m) {
                    w.cbits[x] = 0;
                    w.sdbits[x] = 0;
                }
                for (; m; m &= m - 1) {
                    const int bit = __ffs(m) - 1;
                    const int v = (int)((x << 5) + bit);
                    Gr.lid[v] = off;
                    w.gid[off] = v;
                    w.sid[off] = (sd >> bit) & 1;
                    ++off;
                }
            }
        }
        if (Grp::rank() == 0 && threadIdx.x == 0) {
            w.ctl->nu = (int)nu;
            w.ctl->hmax = (int)nu + 2;
        }
        if (!Grp::sync(w)) return false;
        // the group marks of the window, cleared for the next pair (nothing reads them now)
        for (long long s = (g0 >> 5) + G.tid; s <= ((g1 - 1) >> 5); s += G.size) w.sbits[s] = 0;
        timer_mark<Grp>(w, t0, T_LID);
        return true;
    }

    // Union ids in increasing (base + v) order: the corridor vertices, found on the
    // visit list, set their bit in cbits; a scan over the words (popcounts, then
    // the set bits of each word in order) numbers them and clears the words again.
    // The corridor export relies on this order (local ids ascending with global ids).
    __device__ bool lids() {
        // the queue sweep numbers by id when the visit list's id range is narrow (the
        // ids of spatially ordered meshes: neighbours get nearby local ids and mostly
        // the same CTA of the cluster), by visit order otherwise
        if (w.list_ids) {
            const int vmin = __ldcg(&w.ctl->vmin), vmax = __ldcg(&w.ctl->vmax);
            if (vmax < 0 || !w.sbits) return lids_list();
            const long long g0 = vmin >> 10, g1 = (vmax >> 10) + 1;
            if (g1 - g0 > max(4096LL, vtotal) || g1 - g0 > (long long)w.nu_cap) return lids_list();
            return lids_window(g0, g1);
        }
        const long long w0 = 0, w1 = (w.total_n + 31) >> 5;
        unsigned long long t0 = globaltimer();
        for (long long e = G.tid; e < vtotal; e += G.size) {
            const int v = w.vq_v[e], s = w.vq_s[e];
            const GraphDev &Gr = w.graphs[w.pairs[s >> 1].g];
            if (in_corridor(Gr, v)) {
                const long long x = Gr.base + v;
                atomicOr(&w.cbits[x >> 5], 1u << (x & 31));
            }
        }
        if (!Grp::sync(w)) return false;
        long long nu = 0;
        bool ok = grid_scan<TPB, Grp>(
            w, w1 - w0, [&](long long x) -> int { return __popc(__ldcg(&w.cbits[w0 + x])); },
            [&](long long xr, long long off) {
                const long long x = w0 + xr;
                unsigned m = __ldcg(&w.cbits[x]);
                if (!m) return;
                w.cbits[x] = 0;
                for (; m; m &= m - 1) {
                    const long long y = (x << 5) + (__ffs(m) - 1);
                    const GraphDev &Gr = w.graphs[graph_of(y)];
                    const int v = (int)(y - Gr.base);
                    if (off < w.nu_cap) {
                        Gr.lid[v] = (int)off;
                        w.gid[off] = v;
                        w.sid[off] = side_of(Gr, __ldcg(Gr.part + v));
                    } else {
                        fail(w.ctl, E_MISFIT, 30);
                    }
                    ++off;
                }
            },
            &nu);
        if (!ok) return false;
        if (Grp::rank() == 0 && threadIdx.x == 0) {
            w.ctl->nu = (int)nu;
            w.ctl->hmax = (int)nu + 2;
        }
        if (!Grp::sync(w)) return false;
        timer_mark<Grp>(w, t0, T_LID);
        return true;
    }

    // ---------------------------------------------------------- network build --
    __device__ bool build() {
        unsigned long long t0 = globaltimer();
        Ctl *ctl = w.ctl;
        const int nu = __ldcg(&ctl->nu);
        // degree, border, INF_v; crank[e] = rank of arc e among its row's corridor
        // arcs (-1 for other arcs), so that reverse arcs need no re-filtering later
        int *crank = w.crank ? w.crank : w.outs;
        for (long long b0 = G.warp * 32; b0 < nu; b0 += G.nwarps * 32) {
            const long long i = b0 + (threadIdx.x & 31);
            const bool valid = i < nu;
            int cnt = 0, p = 0;
            if (valid) {
                const int v = w.gid[i], s = w.sid[i];
                p = s >> 1;
                const PairDev P = w.pairs[p];
                const GraphDev &Gr = w.graphs[P.g];
                int bor = 0;
                long long wdeg = 0;
                const int j0 = __ldg(Gr.xadj + v), j1 = __ldg(Gr.xadj + v + 1);
                // eight arcs at a time, the loads of each step issued together (the
                // chain arc -> head's block -> head's local id is latency bound)
                for (int jb = j0; jb < j1; jb += 8) {
                    int u[8], c[8], pu[8], lu[8];
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        const int j = min(jb + t, j1 - 1);
                        u[t] = __ldg(Gr.adjncy + j);
                        c[t] = __ldg(Gr.adjwgt + j);
                    }
#pragma unroll
                    for (int t = 0; t < 8; ++t) pu[t] = __ldcg(Gr.part + u[t]);
#pragma unroll
                    for (int t = 0; t < 8; ++t) lu[t] = (pu[t] == P.a || pu[t] == P.b) ? __ldcg(Gr.lid + u[t]) : -1;
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        if (jb + t >= j1) break;
                        wdeg += c[t];
                        int rk = -1;
                        if (pu[t] == P.a || pu[t] == P.b) {
                            if (lu[t] >= 0) rk = cnt++; else bor = 1;
                        }
                        crank[Gr.ebase + jb + t] = rk;
                    }
                }
                w.off[i] = cnt;   // degree for now
                w.border[i] = bor ? ((s & 1) ? 2 : 1) : 0;
                w.infc[i] = (int)(wdeg + 1);
            }
            warp_agg_add_i(valid ? &w.pacc[p].nc : nullptr, 1, valid);
            warp_agg_add_i(valid ? &w.pacc[p].m : nullptr, cnt, valid);
        }
        if (!Grp::sync(w)) return false;
        // offsets: exclusive scan of the degrees (in place via the deg copy in rev)
        for (long long i = G.tid; i < nu; i += G.size) w.rev[i] = w.off[i];
        if (!Grp::sync(w)) return false;
        long long mu = 0;
        bool ok = grid_scan<TPB, Grp>(
            w, nu, [&](long long i) -> int { return __ldcg(&w.rev[i]); },
            [&](long long i, long long off) { w.off[i] = (int)off; }, &mu);
        if (!ok) return false;
        if (mu > w.mu_cap) {
            if (G.tid == 0) fail(ctl, E_MISFIT, 40);
        }
        if (G.tid == 0) {
            w.off[nu] = (int)mu;
            ctl->mu = (int)mu;
        }
        if (!Grp::sync(w)) return false;
        // arcs, reverse arcs, residual = capacity: the corridor arcs of every row,
        // flattened over the lanes of a warp (warp_rows) so that long rows do not hold
        // up one thread and a row's arcs are read together; arc e of row i goes to
        // off[i] + crank[e].  ex[i] collects, for s-border rows, the capacity toward
        // vertices off the s-border.
        for (long long i = G.tid; i < nu; i += G.size) w.ex[i] = 0;
        if (!Grp::sync(w)) return false;
        warp_rows(
            0, nu, G,
            [&](long long i, int &rs, int &deg, int &ctx) {
                const int v = w.gid[i];
                const GraphDev &Gr = w.graphs[w.pairs[w.sid[i] >> 1].g];
                rs = __ldg(Gr.xadj + v);
                deg = __ldg(Gr.xadj + v + 1) - rs;
                ctx = (int)i;
            },
            [&](bool valid, int e, int i) {
                if (!valid) return;
                const GraphDev &Gr = w.graphs[w.pairs[w.sid[i] >> 1].g];
                const int rk = __ldcg(&crank[Gr.ebase + e]);
                if (rk < 0) return;
                const int v = w.gid[i];
                const int u = __ldg(Gr.adjncy + e);
                const int h = __ldcg(Gr.lid + u);
                const int c = __ldg(Gr.adjwgt + e);
                const int j = __ldcg(&w.off[i]) + rk;
                w.head[j] = h;
                w.cap[j] = c;
                w.res[j] = c;
                if (w.border[i] == 1 && __ldcg(&w.border[h]) != 1)   // arcs into other s-border vertices carry
                    atomicAddLL(&w.ex[i], (long long)c);             // nothing s could not send directly
                // the reverse arc: v's position in u's row, then its rank among u's corridor arcs
                const int k0 = __ldg(Gr.xadj + u), k1 = __ldg(Gr.xadj + u + 1);
                int t = -1;
                for (int f = k0; f < k1 && t < 0; f += 8) {
                    int x[8];
#pragma unroll
                    for (int z = 0; z < 8; ++z) x[z] = f + z < k1 ? __ldg(Gr.adjncy + f + z) : -1;
#pragma unroll
                    for (int z = 7; z >= 0; --z)
                        if (x[z] == v) t = f + z;
                }
                const int q = t >= 0 ? __ldcg(&crank[Gr.ebase + t]) : 0;
                if (t < 0) fail(w.ctl, E_INVALID, 41);   // no reverse arc: the CSR is not symmetric
                w.rev[j] = __ldcg(&w.off[h]) + q;
            });
        if (!Grp::sync(w)) return false;
        // Preflow: s -> v carries what v can pass on to vertices outside the s-border,
        // c_out(v) < INF_v.  Some maximum flow sends no more through s -> v (flow
        // s -> v -> u with u on the s-border can go s -> u directly), so the max flow
        // is unchanged and only the excess that is pushed in and then stranded has to
        // move again.
        for (long long i = G.tid; i < nu; i += G.size) {
            const unsigned char bd = w.border[i];
            const long long cout = __ldcg(&w.ex[i]);
            const int fx0 = bd == 1 ? (int)(cout < w.infc[i] ? cout : w.infc[i]) : 0;
            w.fx[i] = fx0;
            w.ex[i] = fx0;
            w.lab[i] = 0;
        }
        // pairs by network size, largest first (ties by index): the order in which
        // the clusters take them
        for (long long i = G.tid; i < w.npairs; i += G.size) {
            const int mi = __ldcg(&w.pacc[i].m);
            int rk = 0;
            for (int q = 0; q < w.npairs; ++q) {
                const int mq = __ldcg(&w.pacc[q].m);
                rk += mq > mi || (mq == mi && q < i);
            }
            w.pacc[rk].ord = (int)i;
        }
        if (!Grp::sync(w)) return false;
        timer_mark<Grp>(w, t0, T_BUILD);
        return true;
    }

    // ------------------------------------------------------------- max flow --

    // Exact distance labels, to t (phase 1) or to s (phase 2): reverse BFS over
    // residual arcs, level by level from the target's border.  Each frontier row is
    // expanded once; warp_rows spreads a level over all warps.  Vertices that cannot
    // reach the target keep hmax (the gap heuristic comes with it).
    __device__ bool global_relabel(int phase2, int hmax, int nu) {
        Ctl *ctl = w.ctl;
        {
            int *cnt = &ctl->fcnt[(fl + 1) % 3];
            int *q = ((fl + 1) & 1) ? w.fq1 : w.fq0;
            for (long long b = G.warp * 32; b < nu; b += G.nwarps * 32) {
                const long long i = b + (threadIdx.x & 31);
                bool src = false;
                if (i < nu) {
                    const unsigned char bd = w.border[i];
                    src = phase2 ? (bd == 1 && __ldcg(&w.fx[i]) > 0) : (bd == 2);
                    w.lab[i] = src ? 1 : hmax;
                }
                const int slot = warp_append(cnt, src);
                if (src) q[slot] = (int)i;
            }
            if (G.tid == 0) ctl->fcnt[(fl + 2) % 3] = 0;
            if (!Grp::sync(w)) return false;
            ++fl;
        }
        long long arcs = 0;
        for (int d = 1;; ++d) {
            const int cur = __ldcg(&ctl->fcnt[fl % 3]);
            if (cur == 0) break;
            const int *q = (fl & 1) ? w.fq1 : w.fq0;
            int *nq = ((fl + 1) & 1) ? w.fq1 : w.fq0;
            int *ncnt = &ctl->fcnt[(fl + 1) % 3];
            warp_rows(
                0, cur, G,
                [&](long long e, int &rs, int &deg, int &ctx) {
                    const int x = q[e];
                    rs = w.off[x];
                    deg = w.off[x + 1] - rs;
                    ctx = x;
                },
                [&](bool valid, int j, int x) {
                    bool got = false;
                    int y = 0;
                    if (valid) {
                        ++arcs;
                        y = w.head[j];
                        const int rv = w.rev[j];
                        const int ly = __ldcg(&w.lab[y]);
                        if (ly == hmax && __ldcg(&w.res[rv]) > 0) got = atomicCAS(&w.lab[y], hmax, d + 1) == hmax;
                    }
                    const int slot = warp_append(ncnt, got);
                    if (got) nq[slot] = y;
                    (void)x;
                });
            if (G.tid == 0) ctl->fcnt[(fl + 2) % 3] = 0;
            if (!Grp::sync(w)) return false;
            ++fl;
            if (d > nu + 2) {
                fail(ctl, E_ITER, 50);
                return false;
            }
        }
        if (G.tid == 0) ctl->relabels += 1;
        if (arcs) atomicAddLL(&ctl->gr_arcs, arcs);
        return true;
    }

    // One pulse of lock-free push-relabel (every active vertex pushes to its
    // lowest residual neighbour or relabels, a few times).  Counts vertices that
    // may be active afterwards.
    __device__ void pulse(int phase2, int hmax, int nu, int *act) {
        int local = 0;
        long long scanned = 0, pushes = 0;
        for (int pass = 0; pass < w.passes; ++pass) {
        const bool last = pass + 1 == w.passes;
        for (long long i = G.tid; i < nu; i += G.size) {
            long long e = __ldcg(&w.ex[i]);
            if (e <= 0) continue;
            int h = __ldcg(&w.lab[i]);
            if (h >= hmax) continue;
            const int j0 = w.off[i], j1 = w.off[i + 1];
            const unsigned char bd = w.border[i];
            for (int it = 0; it < w.inner; ++it) {
                int hmin = INT_MAX, best = -1;
                scanned += j1 - j0;
                for (int j = j0; j < j1; j += 4) {
                    int r[4], hd[4], hh[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        r[u] = j + u < j1 ? __ldcg(&w.res[j + u]) : 0;
                        hd[u] = j + u < j1 ? w.head[j + u] : 0;
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) hh[u] = r[u] > 0 ? __ldcg(&w.lab[hd[u]]) : INT_MAX;
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (hh[u] < hmin) { hmin = hh[u]; best = j + u; }
                }
                if (phase2 ? (bd == 1 && w.fx[i] > 0) : (bd == 2)) { hmin = 0; best = -2; }
                if (best == -1) { h = hmax; w.lab[i] = h; break; }
                if (h > hmin) {
                    long long d;
                    ++pushes;
                    if (best == -2) {
                        if (!phase2) {
                            d = e;                       // v -> t is never saturated
                            w.fx[i] += (int)d;
                        } else {
                            const int f = w.fx[i];
                            d = e < f ? e : f;
                            w.fx[i] = f - (int)d;
                        }
                    } else {
                        const int r = __ldcg(&w.res[best]);
                        d = e < r ? e : r;
                        atomicSub(&w.res[best], (int)d);
                        atomicAdd(&w.res[w.rev[best]], (int)d);
                        atomicAddLL(&w.ex[w.head[best]], d);
                        if (last) ++local;
                    }
                    atomicAddLL(&w.ex[i], -d);
                    e -= d;
                    if (e == 0) break;
                } else {
                    h = hmin + 1;
                    if (h >= hmax) h = hmax;
                    w.lab[i] = h;
                    if (h >= hmax) break;
                }
            }
            if (last && e > 0 && h < hmax) ++local;
        }
        }
        __syncthreads();
        const long long tot = block_sum_ll<TPB>(local);
        const long long tsc = block_sum_ll<TPB>(scanned);
        const long long tpu = block_sum_ll<TPB>(pushes);
        if (threadIdx.x == 0) {
            if (tot) atomicAdd(act, (int)tot);
            if (tsc) atomicAddLL(&w.ctl->pr_arcs, tsc);
            if (tpu) atomicAddLL(&w.ctl->pushes, tpu);
        }
    }

    __device__ bool count_active(int hmax, int nu, bool any_excess, int *out) {
        // counts vertices with excess (any_excess) or active vertices into *out
        int local = 0;
        for (long long i = G.tid; i < nu; i += G.size) {
            const long long e = __ldcg(&w.ex[i]);
            if (e > 0 && (any_excess || __ldcg(&w.lab[i]) < hmax)) ++local;
            if (e < 0) fail(w.ctl, E_INTERNAL, 60);
        }
        __syncthreads();
        const long long tot = block_sum_ll<TPB>(local);
        if (threadIdx.x == 0 && tot) atomicAdd(out, (int)tot);
        return Grp::sync(w);
    }

    __device__ bool flow_phase(int phase2, int hmax, int nu) {
        Ctl *ctl = w.ctl;
        unsigned long long t0 = globaltimer();
        if (!global_relabel(phase2, hmax, nu)) return false;
        timer_mark<Grp>(w, t0, T_GR);
        long long pulses = 0;
        int since_gr = 0;
        for (;;) {
            int *act = &ctl->act[pl % 3];
            if (G.tid == 0) ctl->act[(pl + 1) % 3] = 0;
            pulse(phase2, hmax, nu, act);
            if (!Grp::sync(w)) return false;
            const int a = __ldcg(act);
            ++pl;
            ++pulses;
            ++since_gr;
            if (pulses > w.pulse_cap) {
                fail(ctl, E_ITER, 70);
                return false;
            }
            timer_mark<Grp>(w, t0, phase2 ? T_FLOW2 : T_FLOW1);
            // Nothing moved in the last pass.  Pushes of earlier lock-free passes may
            // have landed after their target was scanned, so count once more behind
            // the barrier; if no vertex with excess is below hmax, an exact global
            // relabel confirms that no excess can reach the target.
            if (a == 0) {
                int *cnt = &ctl->act[pl % 3];
                if (G.tid == 0) ctl->act[(pl + 1) % 3] = 0;
                if (!count_active(hmax, nu, false, cnt)) return false;
                int left = __ldcg(cnt);
                ++pl;
                if (left == 0) {
                    // exact labels decide: the phase ends only if no vertex with
                    // excess can reach the target
                    if (!global_relabel(phase2, hmax, nu)) return false;
                    since_gr = 0;
                    timer_mark<Grp>(w, t0, T_GR);
                    cnt = &ctl->act[pl % 3];
                    if (G.tid == 0) ctl->act[(pl + 1) % 3] = 0;
                    if (!count_active(hmax, nu, false, cnt)) return false;
                    left = __ldcg(cnt);
                    ++pl;
                    if (left == 0) break;
                    continue;
                }
            }
            if (since_gr >= w.gr_interval) {
                if (!global_relabel(phase2, hmax, nu)) return false;
                since_gr = 0;
                timer_mark<Grp>(w, t0, T_GR);
            } else if (w.gap_interval > 0 && since_gr % w.gap_interval == 0) {
                if (!gap_check(hmax, nu)) return false;
            }
        }
        if (G.tid == 0) ctl->pulses += pulses;
        return true;
    }

    // Gap heuristic over the union network (the paper's max-flow solver, HIPR, uses it):
    // with no push in flight, a label h below the largest held label (below hmax) that
    // no vertex holds is held by no vertex of any pair, so no vertex above h reaches its
    // pair's target (a valid labelling never lets a residual arc drop more than one
    // label): they all go to hmax.  The held labels are marked in a bitmap in vc (free
    // during the flow).
    __device__ bool gap_check(int hmax, int nu) {
        Ctl *ctl = w.ctl;
        unsigned *bm = reinterpret_cast<unsigned *>(w.vc);
        const int nwords = (hmax + 31) >> 5;
        if (nwords > w.nu_cap) return true;
        for (long long i = G.tid; i < nwords; i += G.size) bm[i] = 0u;
        if (G.tid == 0) {
            ctl->gap_top = 0;
            ctl->gap_pos = INT_MAX;
        }
        if (!Grp::sync(w)) return false;
        int top = 0;
        for (long long i = G.tid; i < nu; i += G.size) {
            const int h = __ldcg(&w.lab[i]);
            if (h >= 1 && h < hmax) {
                const unsigned b = 1u << (h & 31);
                if (!(__ldcg(&bm[h >> 5]) & b)) atomicOr(&bm[h >> 5], b);
                top = max(top, h);
            }
        }
        top = __reduce_max_sync(FULL, top);
        if ((threadIdx.x & 31) == 0 && top) atomicMax(&ctl->gap_top, top);
        if (!Grp::sync(w)) return false;
        top = __ldcg(&ctl->gap_top);
        int pos = INT_MAX;
        for (long long i = G.tid; i <= (top >> 5); i += G.size) {
            unsigned empty = ~__ldcg(&bm[i]);
            if (i == 0) empty &= ~1u;                                                     // label 0: the target
            if (i == (top >> 5)) empty &= (top & 31) ? ((1u << (top & 31)) - 1u) : 0u;   // below top
            if (empty) pos = min(pos, (int)(i << 5) + __ffs(empty) - 1);
        }
        pos = __reduce_min_sync(FULL, pos);
        if ((threadIdx.x & 31) == 0 && pos != INT_MAX) atomicMin(&ctl->gap_pos, pos);
        if (!Grp::sync(w)) return false;
        const int h0 = __ldcg(&ctl->gap_pos);
        if (h0 == INT_MAX) return true;
        long long lifted = 0;
        for (long long i = G.tid; i < nu; i += G.size) {
            const int h = __ldcg(&w.lab[i]);
            if (h > h0 && h < hmax) {
                w.lab[i] = hmax;
                ++lifted;
            }
        }
        lifted = block_sum_ll<TPB>(lifted);
        if (threadIdx.x == 0 && lifted) atomicAddLL(&ctl->gap_lifted, lifted);
        if (G.tid == 0) atomicAddLL(&ctl->gaps, 1);
        return Grp::sync(w);
    }

    // Maximum preflow (phase 0).  The cut needs no more: with an arc v -> s of
    // capacity e(v) for every vertex v left with excess e(v), the preflow is a flow
    // of the same value, the new arcs enter s and change no cut capacity, so the
    // network has the same minimum cuts and this flow is maximum; its residual
    // graph is the preflow's plus s -> v for each such v.  The residual sets
    // therefore take vertices with excess as reached from s (reach), and phase 1,
    // which returns the excess to s, runs only where a flow is handed out
    // (full_flow).
    __device__ bool maxflow() {
        Ctl *ctl = w.ctl;
        const int nu = __ldcg(&ctl->nu), hmax = __ldcg(&ctl->hmax);
        // pairs already solved in their clusters have no excess that can move, so the
        // grid-wide phases only move the excess of the pairs that did not fit a cluster
        if (!w.cluster_mode || __ldcg(&ctl->fallback) > 0) {
            if (!flow_phase(0, hmax, nu)) return false;
            if (w.full_flow && !flow_phase(1, hmax, nu)) return false;
        }
        unsigned long long t0 = globaltimer();
        if (w.full_flow) {
            // every excess must have returned to s: the result is a flow
            int *cnt = &ctl->act[pl % 3];
            if (G.tid == 0) ctl->act[(pl + 1) % 3] = 0;
            if (!count_active(hmax, nu, true, cnt)) return false;
            if (__ldcg(cnt) != 0 && G.tid == 0) fail(ctl, E_INTERNAL, 80);
            ++pl;
        }
        // flow value per pair: flow into t
        for (long long i = G.tid; i < nu; i += G.size)
            if (w.border[i] == 2) atomicAddLL(&w.pacc[w.sid[i] >> 1].flow, (long long)w.fx[i]);
        if (!Grp::sync(w)) return false;
        timer_mark<Grp>(w, t0, T_FLOW2);
        return true;
    }

    // ---------------------------------------------------------- residual sets --
    // Bit 1: reachable from s (the smallest source set, Ford-Fulkerson labelling),
    // seeded with the s-border and every vertex holding excess (see maxflow);
    // bit 2: reaches t.  Both searches share one frontier queue, entries tagged by
    // the top bit.
    __device__ bool reach() {
        Ctl *ctl = w.ctl;
        unsigned long long t0 = globaltimer();
        const int nu = __ldcg(&ctl->nu);
        if (w.cluster_mode && __ldcg(&ctl->fallback) == 0) return true;   // the clusters wrote the sets
        {
            int *cnt = &ctl->fcnt[(fl + 1) % 3];
            int *q = ((fl + 1) & 1) ? w.fq1 : w.fq0;
            for (long long b = G.warp * 32; b < nu; b += G.nwarps * 32) {
                const long long i = b + (threadIdx.x & 31);
                bool sb = false, tb = false;
                if (i < nu) {
                    const unsigned char bd = w.border[i];
                    sb = bd == 1 || __ldcg(&w.ex[i]) > 0;
                    tb = bd == 2;
                    w.rflag[i] = (sb ? 1 : 0) | (tb ? 2 : 0);
                }
                const int slot = warp_append(cnt, sb || tb);
                if (sb || tb) q[slot] = (int)i | (tb ? (int)0x80000000 : 0);
            }
            if (G.tid == 0) ctl->fcnt[(fl + 2) % 3] = 0;
            if (!Grp::sync(w)) return false;
            ++fl;
        }
        for (int d = 1;; ++d) {
            const int cur = __ldcg(&ctl->fcnt[fl % 3]);
            if (cur == 0) break;
            const int *q = (fl & 1) ? w.fq1 : w.fq0;
            int *nq = ((fl + 1) & 1) ? w.fq1 : w.fq0;
            int *ncnt = &ctl->fcnt[(fl + 1) % 3];
            warp_rows(
                0, cur, G,
                [&](long long e, int &rs, int &deg, int &ctx) {
                    const int ent = q[e];
                    const int x = ent & 0x7fffffff;
                    rs = w.off[x];
                    deg = w.off[x + 1] - rs;
                    ctx = ent;
                },
                [&](bool valid, int j, int ent) {
                    bool got = false;
                    int y = 0;
                    const bool tside = ent < 0;
                    if (valid) {
                        y = w.head[j];
                        const int bit = tside ? 2 : 1;
                        if (!(__ldcg(&w.rflag[y]) & bit) && __ldcg(&w.res[tside ? w.rev[j] : j]) > 0)
                            got = !(atomicOr(&w.rflag[y], bit) & bit);
                    }
                    const int slot = warp_append(ncnt, got);
                    if (got) nq[slot] = y | (tside ? (int)0x80000000 : 0);
                });
            if (G.tid == 0) ctl->fcnt[(fl + 2) % 3] = 0;
            if (!Grp::sync(w)) return false;
            ++fl;
            if (d > nu + 2) {
                fail(ctl, E_ITER, 90);
                return false;
            }
        }
        // s must not reach t (maximality); plain pairs take the smallest source set
        for (long long i = G.tid; i < nu; i += G.size) {
            const int f = __ldcg(&w.rflag[i]);
            if (f == 3) fail(ctl, E_INTERNAL, 91);
            w.side_out[i] = (f & 1) ? 0 : 1;
        }
        if (!Grp::sync(w)) return false;
        timer_mark<Grp>(w, t0, T_REACH);
        return true;
    }

    // ------------------------------------------------------- SCC colouring --
    // SCCs of the residual graph on X = vertices of MB pairs reached from
    // neither s nor t.  Forward min-label propagation gives every vertex the
    // smallest local id that reaches it; a root (label == own id) collects by
    // backward BFS the vertices of its colour that reach it: its SCC.  The label
    // of an SCC is therefore its smallest local id, i.e. its smallest global id.
    __device__ bool scc() {
        Ctl *ctl = w.ctl;
        unsigned long long t0 = globaltimer();
        const int nu = __ldcg(&ctl->nu);
        if (w.cluster_mode && __ldcg(&ctl->fallback) == 0) return true;   // the clusters wrote scc
        for (long long i = G.tid; i < nu; i += G.size) {
            const bool mbp = w.pairs[w.sid[i] >> 1].mb != 0;
            w.scc[i] = (mbp && __ldcg(&w.rflag[i]) == 0) ? -1 : -2;
        }
        if (!Grp::sync(w)) return false;
        int rounds = 0;
        for (;;) {
            // remaining unassigned?
            int *rem = &ctl->chg[cl % 3];
            if (G.tid == 0) ctl->chg[(cl + 1) % 3] = 0;
            int local = 0;
            for (long long i = G.tid; i < nu; i += G.size)
                if (__ldcg(&w.scc[i]) == -1) { w.color[i] = (int)i; ++local; }
            if (local) atomicAdd(rem, local);
            if (!Grp::sync(w)) return false;
            ++cl;
            if (__ldcg(rem) == 0) break;
            ++rounds;
            if (rounds > nu + 1) { fail(ctl, E_ITER, 100); return false; }
            // forward propagation of the minimum label
            for (int it = 0;; ++it) {
                int *chg = &ctl->chg[cl % 3];
                if (G.tid == 0) ctl->chg[(cl + 1) % 3] = 0;
                int changed = 0;
                for (long long i = G.tid; i < nu; i += G.size) {
                    if (__ldcg(&w.scc[i]) != -1) continue;
                    const int c = __ldcg(&w.color[i]);
                    const int j1 = w.off[i + 1];
                    for (int j = w.off[i]; j < j1; ++j) {
                        if (__ldcg(&w.res[j]) <= 0) continue;
                        const int y = w.head[j];
                        if (__ldcg(&w.scc[y]) != -1) continue;
                        if (__ldcg(&w.color[y]) > c && atomicMin(&w.color[y], c) > c) changed = 1;
                    }
                }
                if (changed) atomicAdd(chg, 1);
                if (!Grp::sync(w)) return false;
                ++cl;
                if (__ldcg(chg) == 0) break;
                if (it > nu + 1) { fail(ctl, E_ITER, 101); return false; }
            }
            // roots and backward BFS inside each colour class
            {
                int *cnt = &ctl->fcnt[(fl + 1) % 3];
                int *q = ((fl + 1) & 1) ? w.fq1 : w.fq0;
                for (long long b = G.warp * 32; b < nu; b += G.nwarps * 32) {
                    const long long i = b + (threadIdx.x & 31);
                    bool root = false;
                    if (i < nu) root = __ldcg(&w.scc[i]) == -1 && __ldcg(&w.color[i]) == (int)i;
                    const int slot = warp_append(cnt, root);
                    if (root) { q[slot] = (int)i; w.scc[i] = (int)i; }
                }
                if (G.tid == 0) ctl->fcnt[(fl + 2) % 3] = 0;
                if (!Grp::sync(w)) return false;
                ++fl;
            }
            for (int d = 1;; ++d) {
                const int cur = __ldcg(&ctl->fcnt[fl % 3]);
                if (cur == 0) break;
                const int *q = (fl & 1) ? w.fq1 : w.fq0;
                int *nq = ((fl + 1) & 1) ? w.fq1 : w.fq0;
                int *ncnt = &ctl->fcnt[(fl + 1) % 3];
                warp_rows(
                    0, cur, G,
                    [&](long long e, int &rs, int &deg, int &ctx) {
                        const int x = q[e];
                        rs = w.off[x];
                        deg = w.off[x + 1] - rs;
                        ctx = x;
                    },
                    [&](bool valid, int j, int x) {
                        bool got = false;
                        int y = 0;
                        if (valid) {
                            y = w.head[j];
                            const int cx = __ldcg(&w.color[x]);
                            if (__ldcg(&w.res[w.rev[j]]) > 0 && __ldcg(&w.scc[y]) == -1 &&
                                __ldcg(&w.color[y]) == cx)
                                got = atomicCAS(&w.scc[y], -1, cx) == -1;
                        }
                        const int slot = warp_append(ncnt, got);
                        if (got) nq[slot] = y;
                    });
                if (G.tid == 0) ctl->fcnt[(fl + 2) % 3] = 0;
                if (!Grp::sync(w)) return false;
                ++fl;
                if (d > nu + 2) { fail(ctl, E_ITER, 102); return false; }
            }
        }
        if (G.tid == 0) ctl->scc_rounds += rounds;
        timer_mark<Grp>(w, t0, T_SCC);
        return true;
    }

    // --------------------------------------------------- DAG and sweeps (MB) --
    __device__ bool sweeps() {
        Ctl *ctl = w.ctl;
        unsigned long long t0 = globaltimer();
        const int nu = __ldcg(&ctl->nu);
        const int P = w.npairs, R = w.reps;
        // component ids for roots, in local-id order
        long long ncomp = 0;
        bool ok = grid_scan<TPB, Grp>(
            w, nu, [&](long long i) -> int { return __ldcg(&w.scc[i]) == (int)i ? 1 : 0; },
            [&](long long i, long long off) {
                if (__ldcg(&w.scc[i]) == (int)i) {
                    w.cid[i] = (int)off;
                    w.cpair[off] = w.sid[i] >> 1;
                    w.cmin[off] = INT_MAX;   // the smallest global id of the members (below)
                    w.cw[off] = 0;
                    w.indeg[off] = 0;
                    w.ocur[off] = 0;
                    w.outoff[off] = 0;
                    w.sinkc[off] = 0;
                }
            },
            &ncomp);
        if (!ok) return false;
        if (G.tid == 0) ctl->ncomp = (int)ncomp;
        for (int p = G.tid; p < P; p += G.size) w.pcur[p] = 0;
        if (!Grp::sync(w)) return false;
        // vertex -> component, component weights, d_0 terms
        for (long long b0 = G.warp * 32; b0 < nu; b0 += G.nwarps * 32) {
            const long long i = b0 + (threadIdx.x & 31);
            bool valid = i < nu;
            long long dd = 0;
            int p = 0;
            if (valid) {
                const int sc = __ldcg(&w.scc[i]);
                const int s = w.sid[i];
                p = s >> 1;
                const PairDev Pd = w.pairs[p];
                valid = Pd.mb != 0;
                if (valid) {
                    const GraphDev &Gr = w.graphs[Pd.g];
                    const long long c = __ldg(Gr.vwgt + w.gid[i]);
                    const int f = __ldcg(&w.rflag[i]);
                    // d_0: the source side is every corridor vertex that does not reach t
                    if (!(s & 1) && (f & 2)) dd = -c;
                    if ((s & 1) && !(f & 2)) dd = c;
                    if (sc >= 0) {
                        const int cc = __ldcg(&w.cid[sc]);
                        w.vc[i] = cc;
                        atomicAddLL(&w.cw[cc], c);
                        atomicMin(&w.cmin[cc], w.gid[i]);
                    }
                }
            }
            warp_agg_add(valid ? &w.pacc[p].d0 : nullptr, dd, valid);
        }
        if (!Grp::sync(w)) return false;
        for (long long i = G.tid; i < nu; i += G.size) {
            const int sc = __ldcg(&w.scc[i]);
            if (sc < 0) continue;
            const int cc = __ldcg(&w.vc[i]);
            if (sc == (int)i) atomicAdd(&w.pacc[w.sid[i] >> 1].ncomp, 1);
            const int j1 = w.off[i + 1];
            for (int j = w.off[i]; j < j1; ++j) {
                if (__ldcg(&w.res[j]) <= 0) continue;
                const int y = w.head[j];
                if (__ldcg(&w.scc[y]) < 0) continue;
                const int cy = __ldcg(&w.vc[y]);
                if (cy == cc) continue;
                atomicAdd(&w.outoff[cc], 1);
                atomicAdd(&w.indeg[cy], 1);
            }
        }
        if (!Grp::sync(w)) return false;
        // pair offsets of the component lists (few pairs: one thread)
        if (G.tid == 0) {
            int acc = 0;
            for (int p = 0; p < P; ++p) {
                w.pacc[p].cbase = acc;
                acc += __ldcg(&w.pacc[p].ncomp);
            }
        }
        // out-arc offsets
        for (long long c = G.tid; c < ncomp; c += G.size) w.indeg_r[c] = __ldcg(&w.outoff[c]);
        if (!Grp::sync(w)) return false;
        long long narcs = 0;
        ok = grid_scan<TPB, Grp>(
            w, ncomp, [&](long long c) -> int { return __ldcg(&w.indeg_r[c]); },
            [&](long long c, long long off) { w.outoff[c] = (int)off; }, &narcs);
        if (!ok) return false;
        if (G.tid == 0) w.outoff[ncomp] = (int)narcs;
        // per-pair lists of components
        for (long long c = G.tid; c < ncomp; c += G.size) {
            const int p = w.cpair[c];
            const int slot = atomicAdd(&w.pcur[p], 1);
            w.plist[__ldcg(&w.pacc[p].cbase) + slot] = (int)c;
        }
        if (!Grp::sync(w)) return false;
        for (long long i = G.tid; i < nu; i += G.size) {
            const int sc = __ldcg(&w.scc[i]);
            if (sc < 0) continue;
            const int cc = __ldcg(&w.vc[i]);
            const int j1 = w.off[i + 1];
            for (int j = w.off[i]; j < j1; ++j) {
                if (__ldcg(&w.res[j]) <= 0) continue;
                const int y = w.head[j];
                if (__ldcg(&w.scc[y]) < 0) continue;
                const int cy = __ldcg(&w.vc[y]);
                if (cy == cc) continue;
                w.outs[__ldcg(&w.outoff[cc]) + atomicAdd(&w.ocur[cc], 1)] = cy;
            }
        }
        for (long long x = G.tid; x < (long long)R * ncomp; x += G.size)
            w.indeg_r[x] = __ldcg(&w.indeg[x % ncomp]);
        if (!Grp::sync(w)) return false;
        timer_mark<Grp>(w, t0, T_SCC);

        // Kahn sweeps: one warp per (pair, r); ready components leave a binary
        // heap keyed (key_r, minid); sweep position j moves the j-th component to
        // the sink side and changes c(A') - c(B') by -2 c(component).
        const int lane = threadIdx.x & 31;
        for (long long task = G.warp; task < (long long)P * R; task += G.nwarps) {
            const int p = (int)(task / R), r = (int)(task % R);
            const PairDev Pd = w.pairs[p];
            const int nc = __ldcg(&w.pacc[p].ncomp);
            if (!Pd.mb) continue;
            const int cb = __ldcg(&w.pacc[p].cbase);
            const long long cA = __ldcg(&w.sides[2 * p].cw), cB = __ldcg(&w.sides[2 * p + 1].cw);
            long long d = 2 * (cA + __ldcg(&w.pacc[p].d0)) - (cA + cB);
            long long best = d < 0 ? -d : d;
            int bestj = 0;
            unsigned long long *hk = w.hkey + (long long)r * nu + cb;
            int *hc = w.hcomp + (long long)r * nu + cb;
            int *ord = w.order + (long long)r * nu + cb;
            int *ind = w.indeg_r + (long long)r * ncomp;
            int hn = 0;
            auto key_of = [&](int c) -> unsigned long long {
                return r == 0 ? 0ull : splitmix64(w.seed ^ (unsigned long long)r ^ (unsigned long long)w.cmin[c]);
            };
            auto less = [&](int i1, int i2) -> bool {
                if (hk[i1] != hk[i2]) return hk[i1] < hk[i2];
                return w.cmin[hc[i1]] < w.cmin[hc[i2]];
            };
            auto push = [&](int c) {
                int i = hn++;
                hk[i] = key_of(c);
                hc[i] = c;
                while (i > 0) {
                    const int par = (i - 1) >> 1;
                    if (!less(i, par)) break;
                    const unsigned long long tk = hk[i]; hk[i] = hk[par]; hk[par] = tk;
                    const int tc = hc[i]; hc[i] = hc[par]; hc[par] = tc;
                    i = par;
                }
            };
            auto pop = [&]() -> int {
                const int top = hc[0];
                --hn;
                hk[0] = hk[hn];
                hc[0] = hc[hn];
                int i = 0;
                for (;;) {
                    const int l = 2 * i + 1, rr = l + 1;
                    int m = i;
                    if (l < hn && less(l, m)) m = l;
                    if (rr < hn && less(rr, m)) m = rr;
                    if (m == i) break;
                    const unsigned long long tk = hk[i]; hk[i] = hk[m]; hk[m] = tk;
                    const int tc = hc[i]; hc[i] = hc[m]; hc[m] = tc;
                    i = m;
                }
                return top;
            };
            // initial ready set
            for (int x0 = 0; x0 < nc; x0 += 32) {
                const int x = x0 + lane;
                int c = -1;
                bool ready = false;
                if (x < nc) {
                    c = w.plist[cb + x];
                    ready = __ldcg(&ind[c]) == 0;
                }
                unsigned int m = __ballot_sync(FULL, ready);
                while (m) {
                    const int l = __ffs(m) - 1;
                    m &= m - 1;
                    const int cc = __shfl_sync(FULL, c, l);
                    if (lane == 0) push(cc);
                }
            }
            int done = 0;
            for (;;) {
                int c = -1;
                if (lane == 0 && hn > 0) c = pop();
                c = __shfl_sync(FULL, c, 0);
                if (c < 0) break;
                if (lane == 0) ord[done] = c;
                ++done;
                d -= 2 * __ldcg(&w.cw[c]);
                const long long ad = d < 0 ? -d : d;
                if (ad < best) { best = ad; bestj = done; }
                const int o0 = __ldcg(&w.outoff[c]), o1 = __ldcg(&w.outoff[c + 1]);
                for (int x0 = o0; x0 < o1; x0 += 32) {
                    const int x = x0 + lane;
                    int cy = -1;
                    bool ready = false;
                    if (x < o1) {
                        cy = __ldcg(&w.outs[x]);
                        ready = atomicSub(&ind[cy], 1) == 1;
                    }
                    unsigned int m = __ballot_sync(FULL, ready);
                    while (m) {
                        const int l = __ffs(m) - 1;
                        m &= m - 1;
                        const int cc = __shfl_sync(FULL, cy, l);
                        if (lane == 0) push(cc);
                    }
                }
                hn = __shfl_sync(FULL, hn, 0);
            }
            if (lane == 0) {
                if (done != nc) fail(ctl, E_INTERNAL, 110);
                w.sw_absd[task] = best;
                w.sw_j[task] = bestj;
            }
        }
        if (!Grp::sync(w)) return false;
        // best (|d|, j, r) per pair, then mark the moved components
        for (int p = G.tid; p < P; p += G.size) {
            long long best = LLONG_MAX;
            int bj = 0, br = 0;
            if (w.pairs[p].mb) {
                for (int r = 0; r < R; ++r) {
                    const long long ad = __ldcg(&w.sw_absd[(long long)p * R + r]);
                    const int j = __ldcg(&w.sw_j[(long long)p * R + r]);
                    if (ad < best || (ad == best && j < bj)) { best = ad; bj = j; br = r; }
                }
            }
            w.pacc[p].best_j = bj;
            w.pacc[p].best_r = br;
        }
        if (!Grp::sync(w)) return false;
        for (int p = 0; p < P; ++p) {
            if (!w.pairs[p].mb) continue;
            const int bj = __ldcg(&w.pacc[p].best_j), br = __ldcg(&w.pacc[p].best_r);
            const int cb = __ldcg(&w.pacc[p].cbase);
            const int *ord = w.order + (long long)br * nu + cb;
            for (long long x = G.tid; x < bj; x += G.size) w.sinkc[ord[x]] = 1;
        }
        if (!Grp::sync(w)) return false;
        for (long long i = G.tid; i < nu; i += G.size) {
            const int sc = __ldcg(&w.scc[i]);
            if (sc >= 0) w.side_out[i] = __ldcg(&w.sinkc[__ldcg(&w.vc[i])]) ? 1 : 0;
        }
        if (!Grp::sync(w)) return false;
        timer_mark<Grp>(w, t0, T_SWEEP);
        return true;
    }

    // ------------------------------------------------------------ evaluation --
    __device__ bool eval() {
        Ctl *ctl = w.ctl;
        unsigned long long t0 = globaltimer();
        const int nu = __ldcg(&ctl->nu);
        for (long long b0 = G.warp * 32; b0 < nu; b0 += G.nwarps * 32) {
            const long long i = b0 + (threadIdx.x & 31);
            const bool valid = i < nu;
            long long dwa = 0, dc = 0, cin = 0;
            int p = 0;
            if (valid) {
                const int s = w.sid[i];
                p = s >> 1;
                const int s0 = s & 1, so = w.side_out[i];
                if (so != s0) {
                    const GraphDev &Gr = w.graphs[w.pairs[p].g];
                    const long long c = __ldg(Gr.vwgt + w.gid[i]);
                    dwa = so == 0 ? c : -c;
                }
                const int j1 = w.off[i + 1];
                for (int j = w.off[i]; j < j1; ++j) {
                    const int y = w.head[j];
                    if (y <= i) continue;   // each corridor edge once
                    const int oldc = s0 != (w.sid[y] & 1);
                    const int newc = so != w.side_out[y];
                    dc += (long long)w.cap[j] * (newc - oldc);
                    cin += (long long)w.cap[j] * newc;
                }
            }
            warp_agg_add(valid ? &w.pacc[p].dwA : nullptr, dwa, valid);
            warp_agg_add(valid ? &w.pacc[p].dcut : nullptr, dc, valid);
            warp_agg_add(valid ? &w.pacc[p].cutin : nullptr, cin, valid);
        }
        if (!Grp::sync(w)) return false;
        for (int p = G.tid; p < w.npairs; p += G.size) {
            PairAcc *A = &w.pacc[p];
            const PairDev Pd = w.pairs[p];
            const long long cA = __ldcg(&w.sides[2 * p].cw), cB = __ldcg(&w.sides[2 * p + 1].cw);
            const long long dwA = __ldcg(&A->dwA), dcut = __ldcg(&A->dcut);
            const long long nA = cA + dwA, nB = cB - dwA;
            const long long nmax = nA > nB ? nA : nB, omax = cA > cB ? cA : cB;
            const int feasible = nmax <= w.graphs[Pd.g].Lmax;
            if (__ldcg(&A->cutin) != __ldcg(&A->flow)) fail(ctl, E_INTERNAL, 120 + (p & 7));
            A->feasible = feasible;
            A->accept = feasible && (dcut < 0 || (dcut == 0 && nmax < omax));
        }
        if (!Grp::sync(w)) return false;
        timer_mark<Grp>(w, t0, T_EVAL);
        return true;
    }

    // v onto the candidate list of block x unless its latest entry is there already
    // (queue sweep; only the cluster holding a pair of x appends to x's list)
    __device__ void qb_append(int v, int x) {
        if (__ldcg(w.qb_lst + v) == x || atomicExch(w.qb_lst + v, x) == x) return;
        const int pos = atomicAdd(w.qb_app + x, 1);
        if (pos < w.qb_cap) w.qb_pool[(long long)x * w.qb_cap + pos] = v;
        else fail(w.ctl, E_MISFIT, 320);
    }

    // ---------------------------------------------------------------- commit --
    __device__ bool commit() {
        Ctl *ctl = w.ctl;
        unsigned long long t0 = globaltimer();
        const int nu = __ldcg(&ctl->nu);
        const bool ok = __ldcg(&ctl->error) == 0;
        if (ok) {
            for (int p = G.tid; p < w.npairs; p += G.size) {
                if (!__ldcg(&w.pacc[p].accept)) continue;
                const PairDev Pd = w.pairs[p];
                const long long dwA = __ldcg(&w.pacc[p].dwA);
                atomicAddLL(&w.graphs[Pd.g].blockw[Pd.a], dwA);    // (in L2: a queue sweep's other
                atomicAddLL(&w.graphs[Pd.g].blockw[Pd.b], -dwA);   // clusters read them there)
            }
            for (long long i = G.tid; i < nu; i += G.size) {
                const int s = w.sid[i], p = s >> 1;
                if (!__ldcg(&w.pacc[p].accept)) continue;
                const PairDev Pd = w.pairs[p];
                const int nb = w.side_out[i] ? Pd.b : Pd.a;
                const GraphDev &Gr = w.graphs[Pd.g];
                const int v = w.gid[i];
                Gr.part[v] = nb;
                const int ob = (s & 1) ? Pd.b : Pd.a;
                if (w.qb_pool && nb != ob) {
                    // the same upkeep on the per-block lists: v joins the list of its new
                    // block, its neighbours left in the old block join that block's list
                    qb_append(v, nb);
                    const int j1 = __ldg(Gr.xadj + v + 1);
                    for (int j = __ldg(Gr.xadj + v); j < j1; ++j) {
                        const int x = __ldg(Gr.adjncy + j);
                        if (__ldcg(Gr.part + x) == ob) qb_append(x, ob);
                    }
                } else if (Gr.bl && nb != ob) {
                    // A moved vertex may now be on a boundary, and so may its neighbours
                    // in its old block (the others had it as a foreign neighbour already).
                    if (!__ldcg(Gr.inb + v) && atomicExch(Gr.inb + v, 1) == 0) Gr.bl[atomicAdd(Gr.blc, 1)] = v;
                    const int j1 = __ldg(Gr.xadj + v + 1);
                    for (int j = __ldg(Gr.xadj + v); j < j1; ++j) {
                        const int x = __ldg(Gr.adjncy + j);
                        if (__ldcg(Gr.inb + x)) continue;
                        if (__ldcg(Gr.part + x) == ob && atomicExch(Gr.inb + x, 1) == 0) Gr.bl[atomicAdd(Gr.blc, 1)] = x;
                    }
                }
            }
        }
        for (long long e = G.tid; e < vtotal; e += G.size) {
            const int v = w.vq_v[e], s = w.vq_s[e];
            const GraphDev &Gr = w.graphs[w.pairs[s >> 1].g];
            Gr.dist[v] = -1;
            Gr.lid[v] = -1;
        }
        if (!Grp::sync(w)) return false;
        timer_mark<Grp>(w, t0, T_COMMIT);
        return true;
    }
};

}  // namespace fr
