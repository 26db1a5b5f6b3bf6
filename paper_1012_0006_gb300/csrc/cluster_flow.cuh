// ClusterFlow: max flow, residual sets and SCCs of one pair inside one thread-block
// cluster, on distributed shared memory (Sanders & Schulz, Section 4.1 and 4.1.1).
// Used by the round's cluster kernel (cluster_flow.cu) and by the queue sweep
// (queue_sweep.cu).
#pragma once

#include <cooperative_groups.h>

#include <climits>

#include "fr_internal.cuh"

namespace fr {

namespace cg = cooperative_groups;

#ifndef FULL
#define FULL 0xffffffffu
#endif

constexpr int kClusterMax = 16;
constexpr int kHdrBytes = 1024;

struct ClusterHdr {
    int klo[kClusterMax + 1];   // member ranges of the CTAs (identical in every CTA)
    int cab[kClusterMax + 1];   // first arc (pair-local prefix) of each CTA's range
    int cnt[3];                 // rotating counters (CTA 0's copy is the cluster's)
    int err;                    // cluster error (CTA 0's copy)
    int nvcap, nacap;           // common capacities (identical in every CTA)
    int nv, na;                 // this CTA's vertices and arcs
    int counts[kClusterMax];    // scratch for the member scan (CTA 0's copy)
    int counts2[kClusterMax];   // second scratch (byte prefix of the split)
    int kloc[3][kClusterMax + 1];   // candidate splits (by arcs, by bytes, by vertices; CTA 0's copy)
    int cabc[3][kClusterMax + 1];
    int grab[2];                // slot of the size order taken (CTA 0's copy, by parity)
    long long flow;
};

// Distributed shared memory by explicit address: a shared::cluster address (32 bits) of an
// element of some CTA's shared memory, and plain stores / relaxed reductions to it.  Every
// CTA carves its arrays at the same offsets, so the address of array X at the same index
// is the address of array Y plus a fixed byte offset.
__device__ __forceinline__ unsigned cta_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned map_rank(unsigned a, int rank) {
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ void dsm_st(unsigned a, int v) {
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void dsm_add(unsigned a, int v) {
    asm volatile("red.shared::cluster.add.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void dsm_min(unsigned a, int v) {
    asm volatile("red.shared::cluster.min.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void dsm_max(unsigned a, int v) {
    asm volatile("red.shared::cluster.max.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void dsm_or(unsigned a, int v) {
    asm volatile("red.shared::cluster.or.b32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

template <int TPB>
struct ClusterFlow {
    const Work &w;
    cg::cluster_group cl;
    const int rank, C;
    ClusterHdr *hdr;
    ClusterHdr *hdr0;          // CTA 0's header
    // local arrays
    int *lab, *ex, *fx, *cofs, *gidx, *rfl, *cla, *res, *csum;
    // narrow: every capacity sum csum(a) = c(a) + c(reverse a) is below 2^16, and
    // res[a] holds res(a) | csum(a) << 16 (csum unused); additions to the residual
    // never carry into the upper half because res(a) <= csum(a)
    bool narrow;
    __device__ __forceinline__ int rs(int a) const {
        const int x = *(volatile int *)&res[a];
        return narrow ? (x & 0xFFFF) : x;
    }
    __device__ __forceinline__ int cs(int a) const { return narrow ? (int)((unsigned)res[a] >> 16) : csum[a]; }
    __device__ __forceinline__ void set_rs(int a, int v) { res[a] = narrow ? ((res[a] & ~0xFFFF) | v) : v; }
    // per arc: shared::cluster addresses of the head's label (hadr) and of the reverse
    // arc's residual (radr); other arrays of the same element are a fixed offset away
    unsigned *hadr, *radr;
    unsigned o_ex, o_rfl, o_cla, o_hlab;   // byte offsets: ex/rfl/cla from lab, hlab from res
    int *hlab;                 // per arc: the label of its head as last published by the head
    unsigned char *bord;
    int rot;                   // rotating counter index (identical in every CTA)

    static constexpr int U = 8;   // arcs whose loads are issued together

    // Lowest head label over the residual arcs [a0, a1) (res > 0), and the arc holding
    // it.  Reads only this CTA's memory: the arcs' copies of their head labels.
    __device__ __forceinline__ void lowest(int a0, int a1, int &hmin, int &best) const {
        hmin = INT_MAX;
        best = -1;
        for (int a = a0; a < a1; a += U) {
            int r[U], l[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                r[u] = a + u < a1 ? rs(a + u) : 0;
                l[u] = a + u < a1 ? *(volatile int *)&hlab[a + u] : INT_MAX;
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (r[u] > 0 && l[u] < hmin) { hmin = l[u]; best = a + u; }
        }
    }


    // Runs f(src, gl, G) once on every lane for the flagged vertices among this
    // warp's 32 (flag is the lane's own vertex, base + lane).  Up to eight flagged:
    // group g = lane / 4 takes the g-th of them, src = its lane (-1: none for this
    // group), gl = lane % 4 the lane's place in the group, G = 4, so a vertex's arcs
    // are walked four at a time.  More than eight: each lane takes its own vertex
    // (src = lane or -1, gl = 0, G = 1).  f gets per-vertex values from lane src with
    // __shfl_sync on all lanes before it tests src.
    template <class Fn>
    __device__ __forceinline__ void for_flagged(bool flag, Fn f) const {
        const int lane = threadIdx.x & 31;
        const unsigned m = __ballot_sync(FULL, flag);
        if (!m) return;
        if (__popc(m) > 8) {
            f(flag ? lane : -1, 0, 1);
            return;
        }
        unsigned mm = m;
        for (int i = 0; i < (lane >> 2); ++i) mm &= mm - 1;
        f(mm ? __ffs(mm) - 1 : -1, lane & 3, 4);
    }

    // New label h of local vertex lv: its own word and the copies on the reverse
    // arcs of its arcs (the arcs of which lv is the head), local or in other CTAs.
    // The copies may lag; they never run ahead of the label, and labels only rise
    // between exact relabels, so a lagging copy only makes a push look admissible
    // that is not -- capacities and excesses stay exact, and a phase ends only once
    // exact labels (phase 1) or the residual sets (phase 0) show that no excess can
    // still reach its target.
    __device__ __forceinline__ void set_label(int lv, int h) {
        lab[lv] = h;
        const int a1 = cofs[lv + 1];
        for (int a = cofs[lv]; a < a1; ++a) dsm_st(radr[a] + o_hlab, h);
    }

    __device__ ClusterFlow(const Work &w_, char *smem)
        : w(w_), cl(cg::this_cluster()), rank((int)cg::this_cluster().block_rank()),
          C((int)cg::this_cluster().num_blocks()) {
        hdr = reinterpret_cast<ClusterHdr *>(smem);
        hdr0 = cl.map_shared_rank(hdr, 0);
        rot = 0;
    }

    long long nsync = 0;       // cluster barriers of the current pair (CTA 0, thread 0)

    __device__ void sync() {
        ++nsync;
        cl.sync();
    }

    // Cluster-wide sum of x (one value per thread); every thread gets the total.
    // Each warp adds its sum straight into CTA 0's counter, so one cluster barrier
    // is the only synchronisation.  The counters rotate over three slots: slot
    // rot + 1 was last read before the previous barrier, so CTA 0 may clear it now.
    __device__ int cluster_sum(int x) { return cluster_reduce(x, false); }
    // cluster-wide maximum of non-negative x
    __device__ int cluster_max(int x) { return cluster_reduce(x, true); }

    __device__ int cluster_reduce(int x, bool is_max) {
        x = is_max ? (int)__reduce_max_sync(FULL, (unsigned)x) : (int)__reduce_add_sync(FULL, (unsigned)x);
        int *c = &hdr0->cnt[rot];
        if ((threadIdx.x & 31) == 0 && x) {
            if (is_max) atomicMax(c, x); else atomicAdd(c, x);
        }
        if (rank == 0 && threadIdx.x == 0) hdr->cnt[(rot + 1) % 3] = 0;
        sync();
        const int tot = *(volatile int *)c;
        rot = (rot + 1) % 3;
        return tot;
    }

    __device__ void carve(char *smem, int nvcap, int nacap, bool narrow_) {
        narrow = narrow_;
        char *p = smem + kHdrBytes;
        auto take = [&](size_t bytes) {
            char *r = p;
            p += (bytes + 15) / 16 * 16;
            return r;
        };
        lab = reinterpret_cast<int *>(take(4ull * nvcap));
        ex = reinterpret_cast<int *>(take(4ull * nvcap));
        fx = reinterpret_cast<int *>(take(4ull * nvcap));
        cofs = reinterpret_cast<int *>(take(4ull * (nvcap + 1)));
        gidx = reinterpret_cast<int *>(take(4ull * nvcap));
        rfl = reinterpret_cast<int *>(take(4ull * nvcap));
        cla = reinterpret_cast<int *>(take(4ull * nvcap));
        bord = reinterpret_cast<unsigned char *>(take(nvcap));
        hadr = reinterpret_cast<unsigned *>(take(4ull * nacap));
        radr = reinterpret_cast<unsigned *>(take(4ull * nacap));
        res = reinterpret_cast<int *>(take(4ull * nacap));
        csum = narrow ? nullptr : reinterpret_cast<int *>(take(4ull * nacap));
        hlab = reinterpret_cast<int *>(take(4ull * nacap));
        o_ex = cta_addr(ex) - cta_addr(lab);
        o_rfl = cta_addr(rfl) - cta_addr(lab);
        o_cla = cta_addr(cla) - cta_addr(lab);
        o_hlab = cta_addr(hlab) - cta_addr(res);
    }

    static __host__ __device__ size_t bytes_for(int nvcap, int nacap, bool narrow) {
        auto a = [](size_t b) { return (b + 15) / 16 * 16; };
        return kHdrBytes + 7 * a(4ull * nvcap) + a(4ull * (nvcap + 1)) + a(nvcap) + (narrow ? 4 : 5) * a(4ull * nacap);
    }

    __device__ int owner(int k) const {   // CTA whose range holds member k
        int r = 0;
        while (r + 1 < C && hdr->klo[r + 1] <= k) ++r;
        return r;
    }

    // ------------------------------------------------------------ one pair --
    // Returns false when the pair does not fit (left to the grid-wide path).
    // adds the time since t to timer slot idx (one thread per cluster; sums over clusters)
    __device__ bool mark(unsigned long long &t, int idx) {
        const unsigned long long now = globaltimer();
        if (rank == 0 && threadIdx.x == 0) atomicAddLL(&w.ctl->timers[idx], (long long)(now - t));
        t = now;
        return true;
    }

    __device__ bool solve(int p, char *smem, size_t smem_bytes) {
        unsigned long long t_in = globaltimer();
        nsync = 0;
        const int nu = __ldcg(&w.ctl->nu);
        const int V = __ldcg(&w.pacc[p].nc), A = __ldcg(&w.pacc[p].m);
        if (V == 0) return true;
        // members of pair p in local-id order: pmem = cid, their arc prefix = outoff, plocal = color
        int pbase = 0;
        for (int q = 0; q < p; ++q) pbase += __ldcg(&w.pacc[q].nc);
        int *pmem = w.cid + pbase, *pacs = w.outoff + pbase, *plocal = w.color;
        {
            // every warp takes a contiguous chunk of the CTA's share of the union and
            // reads it 32 entries at a time (coalesced), counting and then placing the
            // pair's members with ballots; one block scan over the warps' counts and one
            // cluster prefix give the positions, so the list stays in local-id order
            const long long per = (nu + C - 1) / C;
            const long long c0 = per * rank, c1 = min((long long)nu, c0 + per);
            const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
            const long long wper = ((max(0LL, c1 - c0) + TPB / 32 - 1) / (TPB / 32) + 31) / 32 * 32;
            const long long w0 = min(c1, c0 + wper * wid), w1 = min(c1, w0 + wper);
            int mine = 0;
            for (long long b = w0; b < w1; b += 32) {
                const long long i = b + lane;
                mine += __popc(__ballot_sync(FULL, i < w1 && (__ldcg(&w.sid[i]) >> 1) == p));
            }
            int tot;
            const int ex0 = block_exclusive_scan<TPB>(lane == 0 ? mine : 0, &tot);
            if (threadIdx.x == 0) hdr0->counts[rank] = tot;
            sync();
            int pos = __shfl_sync(FULL, ex0, 0);
            for (int r = 0; r < rank; ++r) pos += *(volatile int *)&hdr0->counts[r];
            sync();   // counts read before they are reused
            for (long long b = w0; b < w1; b += 32) {
                const long long i = b + lane;
                const bool m = i < w1 && (__ldcg(&w.sid[i]) >> 1) == p;
                const unsigned bal = __ballot_sync(FULL, m);
                if (m) {
                    const int at = pos + __popc(bal & ((1u << lane) - 1u));
                    pmem[at] = (int)i;
                    plocal[i] = at;
                }
                pos += __popc(bal);
            }
        }
        __threadfence();
        sync();
        // arc and shared-memory byte prefixes over members (each CTA a slice of the
        // member list, each thread a contiguous part of it), and three candidate splits
        // into C contiguous ranges: equal arcs (the work of the flow), equal bytes (29
        // per vertex, 16 or 20 per arc) and equal vertices.  Every CTA carves its arrays
        // for the largest range's vertices and arcs, so the first candidate that fits
        // shared memory is taken: the arc split where it fits, the others where the
        // order of the vertices puts many light vertices together.
        const int ab = w.narrow ? 16 : 20;
        {
            const long long Btot = 29LL * V + (long long)ab * A;
            const long long tot3[3] = {(long long)A, Btot, (long long)V};
            const int per = (V + C - 1) / C;
            const int k0 = min(V, per * rank), k1 = min(V, k0 + per);
            const int tper = (k1 - k0 + TPB - 1) / TPB;
            const int s0 = min(k1, k0 + tper * (int)threadIdx.x), s1 = min(k1, s0 + tper);
            int mine = 0;
            for (int k = s0; k < s1; ++k) {
                const int i = __ldcg(&pmem[k]);
                mine += w.off[i + 1] - w.off[i];
            }
            int tot, btot;
            const int e0 = block_exclusive_scan<TPB>(mine, &tot);
            const int b0 = block_exclusive_scan<TPB>(29 * (s1 - s0) + ab * mine, &btot);
            if (threadIdx.x == 0) {
                hdr0->counts[rank] = tot;
                hdr0->counts2[rank] = btot;
            }
            sync();
            int run = e0;
            long long brun = b0;
            for (int r = 0; r < rank; ++r) {
                run += *(volatile int *)&hdr0->counts[r];
                brun += *(volatile int *)&hdr0->counts2[r];
            }
            sync();
            // split points of candidate c: kloc[c][r] = the first member whose prefix
            // reaches tot3[c] * r / C, so the member whose share (prefix, prefix + size]
            // holds that target is the one before it; its thread writes the split and
            // the range's first arc into CTA 0
            if (rank == 0 && threadIdx.x == 0) {
                for (int c = 0; c < 3; ++c) {
                    hdr->kloc[c][0] = 0;
                    hdr->cabc[c][0] = 0;
                    hdr->kloc[c][C] = V;
                    hdr->cabc[c][C] = A;
                    for (int r = 1; r < C; ++r)
                        if (tot3[c] * r / C <= 0) { hdr->kloc[c][r] = 0; hdr->cabc[c][r] = 0; }
                }
            }
            for (int k = s0; k < s1; ++k) {
                const int i = __ldcg(&pmem[k]);
                const int d = w.off[i + 1] - w.off[i];
                const int b = 29 + ab * d;
                pacs[k] = run;
                const long long lo3[3] = {(long long)run, brun, (long long)k};
                const long long sz3[3] = {(long long)d, (long long)b, 1};
                for (int c = 0; c < 3; ++c)
                    for (int r = 1; r < C; ++r) {
                        const long long target = tot3[c] * r / C;
                        if (target > lo3[c] && target <= lo3[c] + sz3[c]) {
                            hdr0->kloc[c][r] = k + 1;
                            hdr0->cabc[c][r] = run + d;
                        }
                    }
                run += d;
                brun += b;
            }
        }
        __threadfence();
        sync();
        if (rank == 0 && threadIdx.x == 0) {
            int pick = 0;
            for (int c = 0; c < 3; ++c) {
                int nvc = 0, nac = 0;
                for (int r = 0; r < C; ++r) {
                    nvc = max(nvc, hdr->kloc[c][r + 1] - hdr->kloc[c][r]);
                    nac = max(nac, hdr->cabc[c][r + 1] - hdr->cabc[c][r]);
                }
                pick = c;
                if (bytes_for(nvc, nac, w.narrow != 0) <= smem_bytes) break;
            }
            for (int r = 0; r <= C; ++r) {
                hdr->klo[r] = hdr->kloc[pick][r];
                hdr->cab[r] = hdr->cabc[pick][r];
            }
        }
        sync();
        // the C ranges, copied from CTA 0 (same in every CTA)
        if (threadIdx.x <= C && rank != 0) {
            hdr->klo[threadIdx.x] = *(volatile int *)&hdr0->klo[threadIdx.x];
            hdr->cab[threadIdx.x] = *(volatile int *)&hdr0->cab[threadIdx.x];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int nvcap = 0, nacap = 0;
            for (int r = 0; r < C; ++r) {
                nvcap = max(nvcap, hdr->klo[r + 1] - hdr->klo[r]);
                nacap = max(nacap, hdr->cab[r + 1] - hdr->cab[r]);
            }
            hdr->nvcap = nvcap;
            hdr->nacap = nacap;
        }
        __syncthreads();
        const int nvcap = hdr->nvcap, nacap = hdr->nacap;
        const bool nar = w.narrow != 0;
        unsigned long long t1 = t_in;
        mark(t1, T_CL_MEMBERS);
        if (bytes_for(nvcap, nacap, nar) > smem_bytes) return false;   // same decision in every CTA
        carve(smem, nvcap, nacap, nar);
        const int klo = hdr->klo[rank], khi = hdr->klo[rank + 1];
        const int nv = khi - klo;
        const int abase = hdr->cab[rank];
        // load this CTA's vertices and arcs
        int nremote = 0;   // arcs whose head another CTA holds
        for (int lv = threadIdx.x; lv < nv; lv += TPB) {
            const int i = __ldcg(&pmem[klo + lv]);
            gidx[lv] = i;
            ex[lv] = (int)__ldcg(&w.ex[i]);
            fx[lv] = __ldcg(&w.fx[i]);
            bord[lv] = w.border[i];
            const int a0 = __ldcg(&pacs[klo + lv]) - abase;
            cofs[lv] = a0;
            const int j0 = w.off[i], j1 = w.off[i + 1];
            // four arcs at a time, their loads issued together (each arc is a chain
            // head -> head's member index -> its arc prefix)
            for (int jb = j0; jb < j1; jb += 4) {
                int h[4], rv[4], r0[4], cj[4], kh[4], oh[4], cr[4], ph[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = min(jb + u, j1 - 1);
                    h[u] = w.head[j];
                    rv[u] = w.rev[j];
                    r0[u] = __ldcg(&w.res[j]);
                    cj[u] = w.cap[j];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    kh[u] = __ldcg(&plocal[h[u]]);
                    oh[u] = w.off[h[u]];
                    cr[u] = w.cap[rv[u]];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) ph[u] = __ldcg(&pacs[kh[u]]);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (jb + u >= j1) break;
                    const int la = a0 + (jb + u - j0);
                    const int rh = owner(kh[u]);
                    nremote += rh != rank;
                    hadr[la] = map_rank(cta_addr(lab + (kh[u] - hdr->klo[rh])), rh);
                    const int ar = ph[u] - hdr->cab[rh] + (rv[u] - oh[u]);
                    radr[la] = map_rank(cta_addr(res + ar), rh);
                    const int c0 = cj[u] + cr[u];   // res(a) + res(reverse of a), fixed
                    if (nar) {
                        res[la] = r0[u] | (c0 << 16);
                    } else {
                        res[la] = r0[u];
                        csum[la] = c0;
                    }
                }
            }
        }
        nremote = (int)__reduce_add_sync(FULL, (unsigned)nremote);
        if ((threadIdx.x & 31) == 0 && nremote) atomicAddLL(&w.ctl->cl_remote, (long long)nremote);
        if (threadIdx.x == 0) {
            hdr->nv = nv;
            const int a1 = khi < V ? __ldcg(&pacs[khi]) : A;
            cofs[nv] = a1 - abase;
            hdr->na = a1 - abase;
            if (rank == 0) { hdr->cnt[0] = hdr->cnt[1] = hdr->cnt[2] = 0; hdr->err = 0; }
        }
        rot = 0;
        sync();
        const int hmax = V + 2;
        mark(t1, T_CL_LOAD);
        // a maximum preflow is enough for the cut (see the grid-wide maxflow); the
        // excess goes back to s only when the flow itself is handed out
        // The pulse phase stops when no excess can move by its labels; whether the
        // preflow is maximum is then read off the residual sets: no vertex reached
        // from s -- the s-border or one holding excess -- may reach t.  If one does
        // (lagging label copies), the phase resumes from exact labels.
        bool ok = true;
        for (int attempt = 0;; ++attempt) {
            ok = w.flow_sched == 1 ? phase_wave(0, nv, hmax) : phase_pulse(0, nv, hmax, false);
            mark(t1, T_CL_FLOW);
            if (ok && w.full_flow) ok = w.flow_sched == 1 ? phase_wave(1, nv, hmax) : phase_pulse(1, nv, hmax, true);
            mark(t1, T_CL_RETURN);
            if (!ok) break;
            reach(nv);
            mark(t1, T_CL_REACH);
            int open = 0;
            for (int lv = threadIdx.x; lv < nv; lv += TPB) open += rfl[lv] == 3;
            if (cluster_sum(open) == 0) break;
            if (attempt >= 16) {   // the same count in every CTA
                if (rank == 0 && threadIdx.x == 0) fail(w.ctl, E_INTERNAL, 304);
                break;
            }
        }
        if (!ok) {
            // cap reached: report, leave the pair's arrays as they were
            if (rank == 0 && threadIdx.x == 0) fail(w.ctl, E_ITER, 300);
            sync();
            return true;
        }
        // write back: residuals, s/t flows, zero excess, reachability and plain sides
        for (int lv = threadIdx.x; lv < nv; lv += TPB) {
            const int i = gidx[lv];
            const int j0 = w.off[i];
            const int a0 = cofs[lv], a1 = cofs[lv + 1];
            for (int a = a0; a < a1; ++a) w.res[j0 + (a - a0)] = rs(a);
            w.fx[i] = fx[lv];
            w.ex[i] = ex[lv];
            w.rflag[i] = rfl[lv];
            w.side_out[i] = (rfl[lv] & 1) ? 0 : 1;
            if (w.full_flow && ex[lv] != 0) fail(w.ctl, E_INTERNAL, 301);
            if (rfl[lv] == 3) fail(w.ctl, E_INTERNAL, 302);
        }
        sync();
        // most balanced cut: SCCs of the residual graph on the vertices reached from
        // neither s nor t (lab, ex, fx are free now)
        int *sc = fx;
        if (w.pairs[p].mb) {
            scc_local(nv, V, sc);
        } else {
            for (int lv = threadIdx.x; lv < nv; lv += TPB) sc[lv] = -2;
        }
        for (int lv = threadIdx.x; lv < nv; lv += TPB) w.scc[gidx[lv]] = sc[lv];
        mark(t1, T_CL_SCC);
        sync();
        if (rank == 0 && threadIdx.x == 0) atomicAddLL(&w.ctl->cl_syncs, nsync);
        return true;
    }

    // SCCs of the residual graph on X = the vertices with rfl == 0, labelled by
    // their smallest union id (the same labels as the grid-wide colouring): in
    // rounds, every unassigned vertex takes the smallest union id that reaches it
    // over unassigned vertices (colour; label correction pushed along residual arcs
    // with an atomic min), a vertex whose colour is its own id is a root, and the
    // vertices of its colour that reach it join it: members claim the tails of
    // their residual in-arcs with an atomic max of their colour, and a vertex
    // joins when the largest claim it received is its own colour (claims from
    // other classes are smaller: whatever reaches a vertex reaches its
    // successors).  sc: -2 outside X, else the root's union id.
    // V, the pair's vertex count, bounds the rounds: the same bound in every CTA, so
    // that every CTA leaves the loop after the same barrier.
    __device__ void scc_local(int nv, int V, int *sc) {
        int *col = lab, *done = ex;
        for (int lv = threadIdx.x; lv < nv; lv += TPB) sc[lv] = rfl[lv] == 0 ? -1 : -2;
        sync();
        long long rounds = 0;
        for (;;) {
            int rem = 0;
            for (int lv = threadIdx.x; lv < nv; lv += TPB) {
                const bool un = sc[lv] == -1;
                col[lv] = un ? gidx[lv] : INT_MAX;
                done[lv] = un ? INT_MAX : 0;   // colour last passed on
                cla[lv] = -1;
                rem += un;
            }
            if (cluster_sum(rem) == 0) break;
            if (++rounds > (long long)V + 1) {
                if (rank == 0 && threadIdx.x == 0) fail(w.ctl, E_ITER, 303);
                break;
            }
            // colours
            const int lane = threadIdx.x & 31;
            for (;;) {
                int nproc = 0;
                for (int k = 0; k < kScans; ++k) {
                    for (int base = threadIdx.x - lane; base < nv; base += TPB) {
                        const int lv = base + lane;
                        int c = 0;
                        bool fl = false;
                        if (lv < nv && sc[lv] == -1) {
                            c = *(volatile int *)&col[lv];
                            fl = c < done[lv];
                            if (fl) done[lv] = c;
                        }
                        nproc += fl;
                        for_flagged(fl, [&](int src, int gl, int G) {
                            const int cu = __shfl_sync(FULL, c, src < 0 ? 0 : src);
                            if (src < 0) return;
                            const int u = base + src, a1 = cofs[u + 1];
                            for (int a = cofs[u] + gl; a < a1; a += G)
                                if (rs(a) > 0) dsm_min(hadr[a], cu);   // col is lab
                        });
                    }
                }
                if (cluster_sum(nproc) == 0) break;
            }
            // roots, then members claim the vertices of their colour that reach them
            for (int lv = threadIdx.x; lv < nv; lv += TPB) {
                done[lv] = sc[lv] == -1 ? 0 : 1;   // 1: nothing to pass on
                if (sc[lv] == -1 && col[lv] == gidx[lv]) sc[lv] = gidx[lv];
            }
            sync();
            for (;;) {
                int nproc = 0;
                for (int k = 0; k < kScans; ++k) {
                    for (int base = threadIdx.x - lane; base < nv; base += TPB) {
                        const int lv = base + lane;
                        int s = -1;
                        bool fl = false;
                        if (lv < nv && !done[lv]) {
                            s = sc[lv];
                            if (s == -1 && *(volatile int *)&cla[lv] == col[lv]) {
                                s = col[lv];
                                sc[lv] = s;
                            }
                            fl = s >= 0;
                            if (fl) done[lv] = 1;
                        }
                        nproc += fl;
                        for_flagged(fl, [&](int src, int gl, int G) {
                            const int su = __shfl_sync(FULL, s, src < 0 ? 0 : src);
                            if (src < 0) return;
                            const int u = base + src, a1 = cofs[u + 1];
                            for (int a = cofs[u] + gl; a < a1; a += G)
                                if (cs(a) > rs(a)) dsm_max(hadr[a] + o_cla, su);
                        });
                    }
                }
                if (cluster_sum(nproc) == 0) break;
            }
        }
        if (rank == 0 && threadIdx.x == 0) atomicAdd(&w.ctl->scc_rounds, (int)rounds);
    }

    static constexpr int kScans = 4;   // local scans between cluster barriers (relabel, reach)
    static constexpr int kMaxSweeps = 1024;   // sweeps of one wave (a bound; a wave ends when one moves nothing)
    static constexpr int kMaxLocalRounds = 4096;   // local rounds of one sweep (a bound)

    // Exact labels: distances over residual arcs to the level-1 vertices, found by
    // label correction pushed outward.  A vertex whose label dropped since it last
    // passed it on lowers the label of each v with a residual arc v -> u to its own
    // + 1 (an atomic min into v's CTA; the residual of v -> u is csum - res of
    // u -> v) and publishes it to the arcs' copies.  Every CTA rescans its own
    // vertices kScans times between cluster barriers, without waiting for the
    // others; a barrier window in which no CTA had a vertex to pass on ends it
    // (every update sent before the window's barrier was seen in it), and the
    // fixed point is the breadth-first distance.  rfl, free during the flow, holds
    // the label each vertex last passed on.  phase 0: distance to t; phase 1:
    // distance to s.  Returns the highest label below hmax if want_top.
    __device__ int relabel(int ph, int nv, int hmax, bool want_top = false) {
        const unsigned long long t_rel = globaltimer();
        for (int lv = threadIdx.x; lv < nv; lv += TPB) {
            const bool src = ph ? (bord[lv] == 1 && fx[lv] > 0) : (bord[lv] == 2);
            lab[lv] = src ? 1 : hmax;
            rfl[lv] = hmax;
        }
        const int na = hdr->na;
        for (int a = threadIdx.x; a < na; a += TPB) hlab[a] = hmax;
        sync();
        long long arcs = 0;   // arcs this thread's vertices passed their labels along
        const int lane = threadIdx.x & 31;
        for (;;) {
            int nproc = 0;
            for (int k = 0; k < kScans; ++k) {
                for (int base = threadIdx.x - lane; base < nv; base += TPB) {
                    const int lv = base + lane;
                    int L = 0;
                    bool fr = false;
                    if (lv < nv) {
                        L = *(volatile int *)&lab[lv];
                        fr = L < rfl[lv];
                        if (fr) {
                            rfl[lv] = L;
                            arcs += cofs[lv + 1] - cofs[lv];
                        }
                    }
                    nproc += fr;
                    for_flagged(fr, [&](int src, int gl, int G) {
                        const int Lu = __shfl_sync(FULL, L, src < 0 ? 0 : src);
                        if (src < 0) return;
                        const int u = base + src, a1 = cofs[u + 1];
                        for (int a = cofs[u] + gl; a < a1; a += G) {
                            dsm_st(radr[a] + o_hlab, Lu);
                            if (cs(a) > rs(a)) dsm_min(hadr[a], Lu + 1);
                        }
                    });
                }
            }
            if (cluster_sum(nproc) == 0) break;
        }
        for (int o = 16; o > 0; o >>= 1) arcs += __shfl_xor_sync(FULL, arcs, o);
        if (lane == 0 && arcs) atomicAddLL(&w.ctl->gr_arcs, arcs);
        int top = 0;
        if (want_top) {
            top = 1;
            for (int lv = threadIdx.x; lv < nv; lv += TPB)
                if (lab[lv] < hmax && lab[lv] > top) top = lab[lv];
            top = cluster_max(top);
        }
        if (rank == 0 && threadIdx.x == 0) atomicAddLL(&w.ctl->timers[T_CL_RELABEL], (long long)(globaltimer() - t_rel));
        return top;
    }

    // One level-synchronous wave (the waves before the pulses): the levels from the
    // top down, each level pushing only along admissible arcs into the level below
    // (level 1 into the target), one cluster barrier per level.  Within a level step
    // a vertex is the only writer of its own excess and of the residuals of its arcs
    // and their reverses, so only the excess of the receiving vertex needs an atomic.
    __device__ void wave_levels_sync(int ph, int nv, int top) {
        for (int L = top; L >= 1; --L) {
            for (int lv = threadIdx.x; lv < nv; lv += TPB) {
                if (lab[lv] != L) continue;
                int e = ex[lv];
                if (e <= 0) continue;
                if (L == 1) {
                    if (!ph) { fx[lv] += e; e = 0; }
                    else if (bord[lv] == 1) { const int d = e < fx[lv] ? e : fx[lv]; fx[lv] -= d; e -= d; }
                } else {
                    const int a1 = cofs[lv + 1];
                    for (int a = cofs[lv]; a < a1 && e > 0; a += U) {
                        int r[U], hr[U], l[U];
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            r[u] = a + u < a1 ? rs(a + u) : 0;
                            hr[u] = a + u < a1 ? (int)hadr[a + u] : 0;
                            l[u] = a + u < a1 ? hlab[a + u] : -1;
                        }
#pragma unroll
                        for (int u = 0; u < U; ++u) l[u] = r[u] > 0 ? l[u] : -1;
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            if (e > 0 && l[u] == L - 1) {
                                const int d = e < r[u] ? e : r[u];
                                set_rs(a + u, r[u] - d);
                                dsm_add(radr[a + u], d);
                                dsm_add((unsigned)hr[u] + o_ex, d);
                                e -= d;
                            }
                        }
                    }
                }
                ex[lv] = e;
            }
            sync();
        }
    }

    // One wave with fixed labels (the waves schedule).  Every vertex holding excess
    // at a level L in [1, top] pushes along its admissible arcs into level L - 1
    // (level 1 into the target).  Each CTA repeats local rounds -- one pass over its vertices, then a
    // CTA barrier -- while a push lands on one of its own vertices; excess sent to
    // another CTA lands there as an atomic addition whenever it lands.  One cluster
    // barrier then ends a sweep, and sweeps repeat until one moves nothing: no
    // excess has an admissible arc with residual capacity any more, and only new
    // labels can move it.  With labels fixed, no two vertices push along an arc and
    // its reverse at once (one of the two pushes would go uphill), so the owner of
    // an arc is the only writer of its residual besides the atomic additions of
    // pushes along the reverse, and every change of an excess is atomic (a vertex
    // pushes at most what it read; others only add).  Every push lowers the sum of
    // excess times label, so the rounds and the sweeps end.
    __device__ void wave_levels(int ph, int nv, int top) {
        const unsigned own_lo = map_rank(cta_addr(lab), rank), own_hi = own_lo + 4u * (unsigned)nv;
        for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
            int moved = 0;
            for (int round = 0; round < kMaxLocalRounds; ++round) {
                int local = 0;
                for (int lv = threadIdx.x; lv < nv; lv += TPB) {
                    const int L = lab[lv];
                    if (L < 1 || L > top) continue;
                    int e = *(volatile int *)&ex[lv];
                    if (e <= 0) continue;
                    int sent = 0;
                    if (L == 1) {
                        if (!ph) { sent = e; fx[lv] += e; }
                        else if (bord[lv] == 1) { sent = e < fx[lv] ? e : fx[lv]; fx[lv] -= sent; }
                    } else {
                        const int a1 = cofs[lv + 1];
                        for (int a = cofs[lv]; a < a1 && e > 0; a += U) {
                            int r[U], l[U];
                            unsigned hr[U];
#pragma unroll
                            for (int u = 0; u < U; ++u) {
                                r[u] = a + u < a1 ? rs(a + u) : 0;
                                hr[u] = a + u < a1 ? hadr[a + u] : 0u;
                                l[u] = a + u < a1 ? hlab[a + u] : -1;
                            }
#pragma unroll
                            for (int u = 0; u < U; ++u) l[u] = r[u] > 0 ? l[u] : -1;
#pragma unroll
                            for (int u = 0; u < U; ++u) {
                                if (e > 0 && l[u] == L - 1) {
                                    const int d = e < r[u] ? e : r[u];
                                    set_rs(a + u, r[u] - d);
                                    dsm_add(radr[a + u], d);
                                    dsm_add(hr[u] + o_ex, d);
                                    e -= d;
                                    sent += d;
                                    local |= hr[u] >= own_lo && hr[u] < own_hi;
                                }
                            }
                        }
                    }
                    if (sent) {
                        atomicSub(&ex[lv], sent);
                        ++moved;
                    }
                }
                if (!__syncthreads_or(local)) break;
            }
            if (cluster_sum(moved) == 0) break;
        }
    }

    // Push-relabel in waves: exact labels, then one wave; repeat until no vertex
    // with excess can reach the target.  Phase 0 sends excess to t, phase 1 returns
    // what is left to s.
    __device__ bool phase_wave(int ph, int nv, int hmax) {
        long long waves = 0;
        for (;;) {
            const int top = relabel(ph, nv, hmax, true);
            int act = 0;
            for (int lv = threadIdx.x; lv < nv; lv += TPB) act += ex[lv] > 0 && lab[lv] < hmax;
            if (cluster_sum(act) == 0) break;
            if (++waves > w.pulse_cap) return false;
            wave_levels(ph, nv, top);
        }
        if (rank == 0 && threadIdx.x == 0) {
            atomicAddLL(&w.ctl->pulses, waves);
            atomicAddLL(&w.ctl->relabels, waves + 1);
        }
        return true;
    }

    // Lock-free pulses (push to the lowest residual neighbour or relabel) until no
    // vertex with excess has a label below hmax; phase 1 returns excess to s.
    // certify: end only after an exact relabel confirms that no excess can move
    // (phase 1; phase 0 is checked by the residual sets instead).
    __device__ bool phase_pulse(int ph, int nv, int hmax, bool certify) {
        {
            // w.pre_waves waves first move the bulk of the excess along shortest paths
            // (labels stay valid: pushes go one level down); the pulses finish
            const int top = relabel(ph, nv, hmax, w.pre_waves > 0);
            for (int k = 0; k < w.pre_waves; ++k) {
                wave_levels_sync(ph, nv, top);
                if (k + 1 < w.pre_waves) relabel(ph, nv, hmax);
            }
        }
        long long pulses = 0, relabels = 1;
        int since = 0;
        for (;;) {
            int act = 0;
            for (int pass = 0; pass < w.passes; ++pass) {
                const bool last = pass + 1 == w.passes;
                for (int lv = threadIdx.x; lv < nv; lv += TPB) {
                    int e = *(volatile int *)&ex[lv];
                    if (e <= 0) continue;
                    int h = lab[lv];
                    if (h >= hmax) continue;
                    const int a0 = cofs[lv], a1 = cofs[lv + 1];
                    const unsigned char bd = bord[lv];
                    for (int it = 0; it < w.inner; ++it) {
                        int hmin, best;
                        lowest(a0, a1, hmin, best);
                        if (ph ? (bd == 1 && fx[lv] > 0) : (bd == 2)) { hmin = 0; best = -2; }
                        if (best == -1) { h = hmax; set_label(lv, h); break; }
                        if (h > hmin) {
                            int d;
                            if (best == -2) {
                                if (!ph) { d = e; fx[lv] += d; }
                                else { d = e < fx[lv] ? e : fx[lv]; fx[lv] -= d; }
                            } else {
                                const int r = rs(best);
                                d = e < r ? e : r;
                                const unsigned hh = hadr[best], rv = radr[best];
                                atomicSub(&res[best], d);
                                dsm_add(rv, d);
                                dsm_add(hh + o_ex, d);
                                if (last) ++act;
                            }
                            atomicSub(&ex[lv], d);
                            e -= d;
                            if (e == 0) break;
                        } else {
                            h = hmin + 1;
                            if (h >= hmax) h = hmax;
                            set_label(lv, h);
                            if (h >= hmax) break;
                        }
                    }
                    if (last && e > 0 && h < hmax) ++act;
                }
            }
            ++pulses;
            ++since;
            const int a = cluster_sum(act);
            if (pulses > w.pulse_cap) return false;
            if (a == 0) {
                // pushes of earlier passes may land after their target was scanned
                int left = 0;
                for (int lv = threadIdx.x; lv < nv; lv += TPB)
                    left += ex[lv] > 0 && lab[lv] < hmax;
                if (cluster_sum(left) == 0) {
                    if (!certify) break;
                    // Nothing can move by the current labels.  Exact labels decide:
                    // the phase ends only if no vertex with excess can reach its
                    // target (the preflow of phase 0 is then maximum; phase 1 has
                    // returned every excess); otherwise they start the next pulse.
                    relabel(ph, nv, hmax);
                    since = 0;
                    ++relabels;
                    left = 0;
                    for (int lv = threadIdx.x; lv < nv; lv += TPB)
                        left += ex[lv] > 0 && lab[lv] < hmax;
                    if (cluster_sum(left) == 0) break;
                    continue;
                }
            }
            if (since >= w.gr_interval) {
                relabel(ph, nv, hmax);
                since = 0;
                ++relabels;
            } else if (w.gap_interval > 0 && since % w.gap_interval == 0) {
                gap(nv, hmax);
            }
        }
        if (rank == 0 && threadIdx.x == 0) {
            atomicAddLL(&w.ctl->pulses, pulses);
            atomicAddLL(&w.ctl->relabels, relabels);
        }
        return true;
    }

    // Gap heuristic (the paper's max-flow solver, HIPR, uses it): between barriers no
    // label moves, and a valid labelling never lets a residual arc drop more than one
    // label, so if no vertex holds some label h below the largest label held (below
    // hmax), no vertex above h can reach the target: all of them go to hmax at once
    // instead of climbing one push at a time until the next exact relabel.  The held
    // labels are marked in a bitmap in CTA 0's claim array (free during the flow).
    // Returns the vertices lifted (cluster-wide).
    __device__ int gap(int nv, int hmax) {
        const int nwords = (hmax + 31) >> 5;
        if (nwords > hdr->nvcap) return 0;   // (tiny ranges: the bitmap does not fit; the same in every CTA)
        unsigned *bm = reinterpret_cast<unsigned *>(cla);
        if (rank == 0)
            for (int i = threadIdx.x; i < nwords; i += TPB) bm[i] = 0u;
        sync();
        const unsigned bm0 = map_rank(cta_addr(bm), 0);
        int top = 0;
        for (int lv = threadIdx.x; lv < nv; lv += TPB) {
            const int h = lab[lv];
            if (h >= 1 && h < hmax) {
                dsm_or(bm0 + 4u * (unsigned)(h >> 5), (int)(1u << (h & 31)));
                top = max(top, h);
            }
        }
        top = cluster_max(top);   // (its barrier also completes the marks)
        // the smallest label in [1, top) that no vertex holds (CTA 0 reads its bitmap)
        int pos = INT_MAX;
        if (rank == 0)
            for (int i = threadIdx.x; i <= (top >> 5); i += TPB) {
                unsigned empty = ~bm[i];
                if (i == 0) empty &= ~1u;                                     // label 0: the target
                if (i == (top >> 5)) empty &= (top & 31) ? ((1u << (top & 31)) - 1u) : 0u;   // below top
                if (empty) pos = min(pos, (i << 5) + __ffs(empty) - 1);
            }
        pos = __reduce_min_sync(FULL, pos);
        const int found = cluster_max(pos == INT_MAX ? 0 : (1 << 30) - pos);
        if (found == 0) return 0;
        const int h0 = (1 << 30) - found;
        int lifted = 0;
        for (int lv = threadIdx.x; lv < nv; lv += TPB) {
            const int h = lab[lv];
            if (h > h0 && h < hmax) {
                set_label(lv, hmax);
                ++lifted;
            }
        }
        lifted = cluster_sum(lifted);
        if (rank == 0 && threadIdx.x == 0) {
            atomicAddLL(&w.ctl->gaps, 1);
            atomicAddLL(&w.ctl->gap_lifted, lifted);
        }
        return lifted;
    }

    // bit 1: reachable from s, seeded with the s-border and with every vertex
    // holding excess (the flow that carries each excess back over a new arc v -> s
    // leaves the residual arc s -> v); bit 2: reaches t.  Frontier pushes: a vertex
    // with a bit not yet passed on sets bit 1 at the heads of its residual arcs and
    // bit 2 at the tails of residual arcs into it (atomic or into the owner's CTA),
    // kScans local scans per cluster barrier as in relabel.  lab, free after the
    // flow, holds the bits already passed on.
    __device__ void reach(int nv) {
        for (int lv = threadIdx.x; lv < nv; lv += TPB) {
            rfl[lv] = (bord[lv] == 1 || ex[lv] > 0 ? 1 : 0) | (bord[lv] == 2 ? 2 : 0);
            lab[lv] = 0;
        }
        sync();
        const int lane = threadIdx.x & 31;
        for (;;) {
            int nproc = 0;
            for (int k = 0; k < kScans; ++k) {
                for (int base = threadIdx.x - lane; base < nv; base += TPB) {
                    const int lv = base + lane;
                    int nw = 0;
                    if (lv < nv) {
                        const int f = *(volatile int *)&rfl[lv], dn = lab[lv];
                        nw = f & ~dn;
                        if (nw) lab[lv] = dn | nw;
                    }
                    nproc += nw != 0;
                    for_flagged(nw != 0, [&](int src, int gl, int G) {
                        const int nwu = __shfl_sync(FULL, nw, src < 0 ? 0 : src);
                        if (src < 0) return;
                        const int u = base + src, a1 = cofs[u + 1];
                        for (int a = cofs[u] + gl; a < a1; a += G) {
                            const int r = rs(a);
                            const int bits = ((nwu & 1) && r > 0 ? 1 : 0) | ((nwu & 2) && cs(a) > r ? 2 : 0);
                            if (bits) dsm_or(hadr[a] + o_rfl, bits);
                        }
                    });
                }
            }
            if (cluster_sum(nproc) == 0) break;
        }
    }
};

}  // namespace fr
