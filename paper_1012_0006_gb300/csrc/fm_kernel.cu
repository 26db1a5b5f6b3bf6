// Two-way FM local search with TopGain on each pair of a round, before the pair's flow
// (Sanders & Schulz, Section 2.2: one priority queue of movable vertices per block,
// keyed by the gain -- the decrease of the pair cut when the vertex changes blocks --,
// every vertex moves at most once, the queues start with the boundary in random order,
// TopGain takes the block whose best vertex has the larger gain and the heavier block
// while one is overloaded, and the moves are rolled back to the best cut found within
// the balance constraint; the setup of Section 6 stops a search once more than a given
// fraction of the pair's vertices moved without an improvement, and runs the FM search
// first and the flow after it).
//
// The keys follow the readings of the CPU oracle: gains and the boundary within
// G[A u B]; order by gain, then by stamp, larger first, where the initial stamps are
// random 63-bit values (splitmix64 of the pair's seed and the vertex id, the random
// initial order) and every later insertion or gain change takes a larger stamp than
// any before, in the adjacency order of the moved vertex; ties of the two top gains
// go by a seeded bit; the best state is the smallest (overload, cut, max block weight).
//
// GPU form.  Pairs of a round are block-disjoint, so one CTA searches one pair on
// vertex-indexed state shared by the round.  Each block's queue is an array of gain
// buckets, each bucket a stack of entries (vertex, version) in global memory with its
// top in shared memory: a gain change pushes a new entry with the vertex's next version
// (its stamp is larger than every earlier one, so a stack stays ordered by stamp) and
// makes the old entry stale; pops skip stale entries.  The initial stacks come from a
// sort of the boundary by (block, gain, stamp).  One warp runs the moves: the top of
// each block's highest non-empty bucket (bitmap in shared memory), the TopGain choice,
// then the moved vertex's arcs 32 at a time -- gain updates, lazy first-touch of a
// neighbour (its weights to both blocks from its adjacency), and the pushes, placed in
// arc order so that every bucket stays ordered.  The rollback, the block weights and
// the boundary candidate list are updated by the whole CTA afterwards.
#include <climits>

#include "fm_kernel.cuh"

namespace fr {

constexpr int kFmTPB = 256;

// ---------------------------------------------------------------- counts ----
// Vertex and arc counts of every paired block.
__global__ void __launch_bounds__(kFmTPB) fm_count_kernel(Work w, FmDev f) {
    const GraphDev G = w.graphs[0];
    extern __shared__ int s_cnt[];   // [2k]
    for (int i = threadIdx.x; i < 2 * G.k; i += blockDim.x) s_cnt[i] = 0;
    __syncthreads();
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < G.n; v += gridDim.x * blockDim.x) {
        const int b = G.part[v];
        if (side_of(G, b) < 0) continue;
        atomicAdd(&s_cnt[b], 1);
        atomicAdd(&s_cnt[G.k + b], __ldg(G.xadj + v + 1) - __ldg(G.xadj + v));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < G.k; i += blockDim.x) {
        if (s_cnt[i]) atomicAdd(f.blockn + i, s_cnt[i]);
        if (s_cnt[G.k + i]) atomicAdd(f.blockarcs + i, s_cnt[G.k + i]);
    }
}

// Region offsets of the pairs (one CTA): vertices (vlist, mlog) by pair vertex counts,
// stack entries by vertex + arc counts (every push is a boundary vertex at the start or
// the update of one arc of a moved vertex).  Clears the block counts for the next round.
__global__ void __launch_bounds__(1024) fm_offsets_kernel(Work w, FmDev f) {
    const GraphDev G = w.graphs[0];
    if (threadIdx.x == 0) {
        long long vo = 0, eo = 0;
        for (int p = 0; p < w.npairs; ++p) {
            const PairDev P = w.pairs[p];
            const int n_p = f.blockn[P.a] + f.blockn[P.b];
            const long long a_p = (long long)f.blockarcs[P.a] + f.blockarcs[P.b];
            f.voff[p] = vo;
            f.eoff[p] = eo;
            f.np[p] = n_p;
            f.bcnt[p] = 0;
            vo += n_p;
            eo += n_p + a_p;
        }
        f.eoff[w.npairs] = eo;
        if (vo > G.n || eo > f.ecap) fail(w.ctl, E_INTERNAL, 700);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < G.k; i += blockDim.x) f.blockn[i] = f.blockarcs[i] = 0;
}

// Weights of every paired vertex to its own block and to the partner block within
// G[A u B] (so that the moves never scan an adjacency for them); vertices with an edge
// to the partner are the boundary and enter their pair's list.
__global__ void __launch_bounds__(kFmTPB) fm_gather_kernel(Work w, FmDev f) {
    if ((w.prev_err && __ldcg(w.prev_err)) || __ldcg(&w.ctl->error)) return;
    const GraphDev G = w.graphs[0];
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < G.n; v += gridDim.x * blockDim.x) {
        const int b = G.part[v];
        const int s = side_of(G, b);
        if (s < 0) continue;
        const PairDev P = w.pairs[s >> 1];
        const int partner = (s & 1) ? P.a : P.b;
        int in = 0, ex = 0;
        const int j1 = __ldg(G.xadj + v + 1);
        for (int j = __ldg(G.xadj + v); j < j1; ++j) {
            const int pu = G.part[__ldg(G.adjncy + j)];
            const int wt = __ldg(G.adjwgt + j);
            if (pu == b) in += wt;
            else if (pu == partner) ex += wt;
        }
        f.in[v] = in;
        f.ext[v] = ex;
        if (ex == 0) continue;
        f.flags[v] = kFmTouched | kFmInQ;
        const int pos = atomicAdd(f.bcnt + (s >> 1), 1);
        f.vlist[f.voff[s >> 1] + pos] = v;
    }
}

// --------------------------------------------------------------- search ----

struct SortRef {   // one sort element: (bucket key, stamp, vertex), ascending by (bk, st, -v)
    unsigned long long *st;
    int *bk, *v;
    __device__ bool less(int i, int j) const {
        if (bk[i] != bk[j]) return bk[i] < bk[j];
        if (st[i] != st[j]) return st[i] < st[j];
        return v[i] > v[j];
    }
    __device__ void swap(int i, int j) const {
        const unsigned long long t = st[i]; st[i] = st[j]; st[j] = t;
        const int b = bk[i]; bk[i] = bk[j]; bk[j] = b;
        const int x = v[i]; v[i] = v[j]; v[j] = x;
    }
};

// Bitonic sort of m (a power of two) elements by the whole CTA.
__device__ void bitonic(const SortRef &r, int m) {
    for (int k = 2; k <= m; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < m; i += blockDim.x) {
                const int l = i ^ j;
                if (l <= i) continue;
                const bool up = (i & k) == 0;
                if (up ? r.less(l, i) : r.less(i, l)) r.swap(i, l);
            }
            __syncthreads();
        }
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

constexpr int kFmWords = kFmMaxBuckets / 32;   // bitmap words per block

struct FmShared {
    int top[2 * kFmMaxBuckets];          // top entry of each (block, bucket) stack, -1 empty
    // where vbits says the top entry is current: its vertex, the entry below it and the
    // vertex's adjacency range (so a move reads no entry and no offsets from memory)
    int topv[2 * kFmMaxBuckets], topb[2 * kFmMaxBuckets];
    int topj0[2 * kFmMaxBuckets], topj1[2 * kFmMaxBuckets];
    unsigned bits[2 * kFmWords];         // non-empty stacks (possibly holding only stale entries)
    unsigned vbits[2 * kFmWords];        // the top entry is known to be current
    long long red[kFmTPB / 32];
    int best_len, tried;
    long long best_cut, best_wA, best_wB;
};

__global__ void __launch_bounds__(kFmTPB, 1) fm_pair_kernel(Work w, FmDev f) {
    extern __shared__ __align__(16) char fm_smem[];
    FmShared &S = *reinterpret_cast<FmShared *>(fm_smem);
    const GraphDev G = w.graphs[0];
    const int p = blockIdx.x;
    const PairDev P = w.pairs[p];
    const int a = P.a, b = P.b;
    const int n_p = f.np[p];
    // the gather ran only without an earlier error; what it marked is cleared on every exit
    const bool gathered = !(w.prev_err && __ldcg(w.prev_err));
    const int B = gathered ? f.bcnt[p] : 0;
    int *vl = f.vlist + f.voff[p];
    int *ml = f.mlog + f.voff[p];
    auto bail = [&]() {
        for (int i = threadIdx.x; i < B; i += blockDim.x) f.flags[vl[i]] = 0;
    };
    if (!gathered || __ldcg(&w.ctl->error)) {
        bail();
        return;
    }
    FmRes *R = f.res + p;
    const long long wA0 = G.blockw[a], wB0 = G.blockw[b];
    if (n_p == 0 || f.permille <= 0) {
        bail();
        if (threadIdx.x == 0) *R = FmRes{0, wA0, wB0, 0, wA0, wB0, 0, 0};
        return;
    }
    const int gmax = __ldcg(f.maxwdeg);   // |gain| <= max weighted degree
    if (2 * gmax + 1 > kFmMaxBuckets) {
        bail();
        if (threadIdx.x == 0) fail(w.ctl, E_TOO_LARGE, 701);
        return;
    }
    const unsigned long long fs = splitmix64(w.seed ^ ((unsigned long long)(unsigned)a << 32) ^ (unsigned)b);
    const long long E = f.eoff[p];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    unsigned long long t_mark = globaltimer();
    auto mark = [&](int idx) {
        const unsigned long long now = globaltimer();
        if (threadIdx.x == 0) atomicAddLL(&w.ctl->timers[idx], (long long)(now - t_mark));
        t_mark = now;
    };
    // 1. sort the boundary by (block, bucket, stamp)
    int m = 1;
    while (m < B) m <<= 1;
    SortRef sr;
    char *sm_sort = fm_smem + sizeof(FmShared);
    if (m <= kFmSortSmem) {
        sr.st = reinterpret_cast<unsigned long long *>(sm_sort);
        sr.bk = reinterpret_cast<int *>(sm_sort + 8ull * kFmSortSmem);
        sr.v = sr.bk + kFmSortSmem;
    } else {
        long long so = 0;   // this pair's scratch: after the larger boundaries of earlier pairs
        for (int q = 0; q < p; ++q) {
            const int bq = f.bcnt[q];
            int mq = 1;
            while (mq < bq) mq <<= 1;
            if (mq > kFmSortSmem) so += mq;
        }
        if (so + m > f.scap) {
            bail();
            if (threadIdx.x == 0) fail(w.ctl, E_INTERNAL, 702);
            return;
        }
        sr.st = f.skey + so;
        sr.bk = f.sbkt + so;
        sr.v = f.sv + so;
    }
    long long c0 = 0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        if (i < B) {
            const int v = vl[i];
            const int side = G.part[v] == a ? 0 : 1;
            const int g = f.ext[v] - f.in[v];
            sr.bk[i] = side * kFmMaxBuckets + g + gmax;
            sr.st[i] = splitmix64(fs ^ (unsigned long long)(unsigned)v) >> 1;
            sr.v[i] = v;
            if (side == 0) c0 += f.ext[v];
        } else {
            sr.bk[i] = INT_MAX;
            sr.st[i] = ~0ull;
            sr.v[i] = -1;
        }
    }
    for (int i = threadIdx.x; i < 2 * kFmMaxBuckets; i += blockDim.x) S.top[i] = -1;
    for (int i = threadIdx.x; i < 2 * kFmWords; i += blockDim.x) S.bits[i] = S.vbits[i] = 0;
    for (int o = 16; o > 0; o >>= 1) c0 += __shfl_down_sync(0xffffffffu, c0, o);
    if (lane == 0) S.red[warp] = c0;
    __syncthreads();
    bitonic(sr, m);
    long long cut0 = 0;
    for (int i = 0; i < kFmTPB / 32; ++i) cut0 += S.red[i];
    // 2. initial stacks: entries in sorted order, each below its predecessor in the bucket
    for (int i = threadIdx.x; i < B; i += blockDim.x) {
        const int bk = sr.bk[i];
        f.ent_v[E + i] = sr.v[i];
        f.ent_ver[E + i] = 0;
        f.ent_below[E + i] = (i > 0 && sr.bk[i - 1] == bk) ? (int)(E + i - 1) : -1;
        if (i + 1 == B || sr.bk[i + 1] != bk) {
            S.top[bk] = (int)(E + i);
            S.topv[bk] = sr.v[i];
            S.topb[bk] = (i > 0 && sr.bk[i - 1] == bk) ? (int)(E + i - 1) : -1;
            S.topj0[bk] = __ldg(G.xadj + sr.v[i]);
            S.topj1[bk] = __ldg(G.xadj + sr.v[i] + 1);
            atomicOr(&S.bits[bk >> 5], 1u << (bk & 31));
            atomicOr(&S.vbits[bk >> 5], 1u << (bk & 31));
        }
    }
    __syncthreads();

    mark(T_FM_SORT);
    // 3. the moves (warp 0).  vbits: the top entry of a stack is known to be current
    // (set by a push or a check, cleared when the top is popped or goes stale), with its
    // vertex, the entry below and the adjacency range cached.  While
    // a move updates its neighbours, lane 0 checks the entry below the popped one, so
    // that the next pop from the same stack usually needs no memory round trip.
    if (warp == 0) {
        const long long Lmax = G.Lmax;
        const long long limit = (long long)f.permille * n_p / 1000;
        long long cut = cut0, wA = wA0, wB = wB0;
        long long bcut = cut, bwA = wA, bwB = wB;
        int nm = 0, best_len = 0, tl = B;   // tl: end of the touched list in vl
        long long idle = 0;
        long long nxt = E + B;
        const long long eend = f.eoff[p + 1];   // entries of this pair: [E, eend)
        bool bad = false;
        for (;;) {
            // top of each block: highest bucket whose top entry is current
            int tb[2];
            for (int s = 0; s < 2; ++s) {
                tb[s] = -1;
                for (;;) {
                    int best = -1;   // lane L looks at the words 2L, 2L + 1, from the top
                    for (int k2 = 1; k2 >= 0; --k2) {
                        const unsigned word = S.bits[s * kFmWords + lane * 2 + k2];
                        if (best < 0 && word) best = (lane * 2 + k2) * 32 + 31 - __clz(word);
                    }
                    const unsigned has = __ballot_sync(0xffffffffu, best >= 0);
                    if (!has) break;
                    const int hb = __shfl_sync(0xffffffffu, best, 31 - __clz(has));
                    const int key = s * kFmMaxBuckets + hb;
                    if ((S.vbits[key >> 5] >> (key & 31)) & 1u) { tb[s] = hb; break; }
                    int ok = 0;
                    if (lane == 0) {
                        const int e = S.top[key];
                        const int v = f.ent_v[e];
                        const int ev = f.ent_ver[e], below = f.ent_below[e];
                        const unsigned char fl = f.flags[v];
                        const int vv = f.ver[v], x0 = __ldg(G.xadj + v), x1 = __ldg(G.xadj + v + 1);
                        ok = (fl & kFmInQ) && !(fl & kFmMoved) && vv == ev;
                        if (ok) {
                            S.topv[key] = v;
                            S.topb[key] = below;
                            S.topj0[key] = x0;
                            S.topj1[key] = x1;
                            S.vbits[key >> 5] |= 1u << (key & 31);
                        } else {
                            S.top[key] = below;
                            if (below < 0) S.bits[key >> 5] &= ~(1u << (key & 31));
                        }
                    }
                    ok = __shfl_sync(0xffffffffu, ok, 0);
                    __syncwarp();
                    if (ok) { tb[s] = hb; break; }
                }
            }
            if (tb[0] < 0 && tb[1] < 0) break;
            int s;
            if (wA > Lmax || wB > Lmax) {
                s = wA >= wB ? 0 : 1;
                if (tb[s] < 0) s = 1 - s;
            } else if (tb[0] < 0) {
                s = 1;
            } else if (tb[1] < 0) {
                s = 0;
            } else if (tb[0] != tb[1]) {
                s = tb[0] > tb[1] ? 0 : 1;
            } else {
                s = (int)(splitmix64(~fs ^ (unsigned long long)nm) & 1);
            }
            const int key = s * kFmMaxBuckets + tb[s];
            const int v = S.topv[key], below = S.topb[key];
            const int j0 = S.topj0[key], j1 = S.topj1[key];
            const int g = tb[s] - gmax;
            const int from = s ? b : a, to = s ? a : b;
            const long long cv = __ldg(G.vwgt + v);
            __syncwarp();
            // pop; the check of the entry below starts now (lane 0)
            int v2 = -1, ev2 = 0, b2 = -1;
            if (lane == 0) {
                S.top[key] = below;
                S.vbits[key >> 5] &= ~(1u << (key & 31));
                if (below < 0) S.bits[key >> 5] &= ~(1u << (key & 31));
                f.flags[v] = kFmTouched | kFmMoved;
                G.part[v] = to;
                ml[nm] = v;
                if (below >= 0) { v2 = f.ent_v[below]; ev2 = f.ent_ver[below]; b2 = f.ent_below[below]; }
            }
            ++nm;
            cut -= g;
            __syncwarp();
            unsigned char fl2 = 0;
            int ver2 = -1, x20 = 0, x21 = 0;
            bool hit2 = false;   // the entry below belongs to a neighbour updated by this move
            // the moved vertex's arcs, 32 at a time in adjacency order
            for (int jb = j0; jb < j1; jb += 32) {
                const int j = jb + lane;
                int u = -1, wt = 0;
                if (j < j1) { u = __ldg(G.adjncy + j); wt = __ldg(G.adjwgt + j); }
                if (jb == j0 && lane == 0 && below >= 0) {   // second half of the check
                    fl2 = f.flags[v2]; ver2 = f.ver[v2];
                    x20 = __ldg(G.xadj + v2); x21 = __ldg(G.xadj + v2 + 1);
                }
                bool act = false;
                int nin = 0, nex = 0, ukey = -1, okey = -1, nver = 0, ux0 = 0, ux1 = 0;
                unsigned char fl = 0;
                if (u >= 0) {
                    // independent loads, issued together
                    const int pu = G.part[u];
                    fl = f.flags[u];
                    const int in0 = f.in[u], ex0 = f.ext[u], ver0 = f.ver[u];
                    ux0 = __ldg(G.xadj + u); ux1 = __ldg(G.xadj + u + 1);
                    if ((pu == a || pu == b) && !(fl & kFmMoved)) {
                        act = true;
                        nin = in0; nex = ex0;
                        if (pu == from) { nin -= wt; nex += wt; }
                        else { nin += wt; nex -= wt; }
                        const int sb = pu == a ? 0 : kFmMaxBuckets;
                        ukey = sb + (nex - nin) + gmax;
                        if (fl & kFmInQ) okey = sb + (ex0 - in0) + gmax;
                        nver = ver0 + 1;
                    }
                }
                const int v2b = __shfl_sync(0xffffffffu, v2, 0);
                hit2 |= __ballot_sync(0xffffffffu, act && u == v2b) != 0;
                // first changes join the touched list (for the cleanup)
                const bool fresh = act && !(fl & kFmTouched);
                const unsigned fm_ = __ballot_sync(0xffffffffu, fresh);
                if (fresh) vl[tl + __popc(fm_ & lanemask_lt())] = u;
                tl += __popc(fm_);
                // u's old entry is stale now.  If it is the known-current top of its stack,
                // take it off: the entry below becomes the top, not yet checked.  (A top known
                // to be current that belongs to another vertex stays current.)  Done before any
                // lane reads a top for a push.
                if (okey >= 0 && ((S.vbits[okey >> 5] >> (okey & 31)) & 1u) && S.topv[okey] == u) {
                    const int nb = S.topb[okey];
                    S.top[okey] = nb;
                    if (nb < 0) atomicAnd(&S.bits[okey >> 5], ~(1u << (okey & 31)));
                    atomicAnd(&S.vbits[okey >> 5], ~(1u << (okey & 31)));
                }
                __syncwarp();
                const bool push = act && nex > 0;
                const unsigned pm = __ballot_sync(0xffffffffu, push);
                if (nxt + __popc(pm) > eend) {   // cannot happen: pushes <= boundary + arcs
                    if (lane == 0) fail(w.ctl, E_INTERNAL, 703);
                    bad = true;
                    break;
                }
                const long long pos = nxt + __popc(pm & lanemask_lt());
                // lanes pushing onto the same stack: the lower lane's entry goes below
                const unsigned grp = __match_any_sync(0xffffffffu, push ? ukey : -1 - lane);
                const unsigned lower = grp & lanemask_lt();
                const long long pos_lower = __shfl_sync(0xffffffffu, pos, lower ? 31 - __clz(lower) : lane);
                int ubelow = -1;
                if (push) ubelow = lower ? (int)pos_lower : S.top[ukey];
                __syncwarp();
                if (act) {
                    f.in[u] = nin;
                    f.ext[u] = nex;
                    f.ver[u] = nver;
                    f.flags[u] = (unsigned char)(kFmTouched | (push ? kFmInQ : 0));
                    if (push) {
                        f.ent_v[pos] = u;
                        f.ent_ver[pos] = nver;
                        f.ent_below[pos] = ubelow;
                        if ((grp & ~lower & ~(1u << lane)) == 0) {   // highest lane of the group
                            S.top[ukey] = (int)pos;
                            S.topv[ukey] = u;
                            S.topb[ukey] = ubelow;
                            S.topj0[ukey] = ux0;
                            S.topj1[ukey] = ux1;
                            atomicOr(&S.bits[ukey >> 5], 1u << (ukey & 31));
                            atomicOr(&S.vbits[ukey >> 5], 1u << (ukey & 31));
                        }
                    }
                }
                nxt += __popc(pm);
                __syncwarp();
            }
            if (bad) break;
            if (s == 0) { wA -= cv; wB += cv; } else { wB -= cv; wA += cv; }   // (its load overlapped the arcs)
            // the entry below the popped one: current, and still the top of its stack?
            if (lane == 0 && below >= 0) {
                if (j0 >= j1) {   // no arcs: the second half of the check did not run
                    fl2 = f.flags[v2]; ver2 = f.ver[v2];
                    x20 = __ldg(G.xadj + v2); x21 = __ldg(G.xadj + v2 + 1);
                }
                if (!hit2 && S.top[key] == below && (fl2 & kFmInQ) && !(fl2 & kFmMoved) && ver2 == ev2) {
                    S.topv[key] = v2;
                    S.topb[key] = b2;
                    S.topj0[key] = x20;
                    S.topj1[key] = x21;
                    S.vbits[key >> 5] |= 1u << (key & 31);
                }
            }
            __syncwarp();
            // best state: smallest (overload, cut, max block weight)
            const long long mx = wA > wB ? wA : wB, bmx = bwA > bwB ? bwA : bwB;
            const long long ov = mx > Lmax ? mx - Lmax : 0, bov = bmx > Lmax ? bmx - Lmax : 0;
            if (ov < bov || (ov == bov && (cut < bcut || (cut == bcut && mx < bmx)))) {
                bcut = cut; bwA = wA; bwB = wB; best_len = nm; idle = 0;
            } else if (++idle > limit) {
                break;
            }
        }
        if (lane == 0) {
            S.best_len = best_len;
            S.tried = nm;
            S.best_cut = bcut;
            S.best_wA = bwA;
            S.best_wB = bwB;
            S.red[0] = tl;
        }
    }
    __syncthreads();
    mark(T_FM_MOVES);
    const int best_len = S.best_len, nm = S.tried, tl = (int)S.red[0];
    // 4. roll back the moves after the best prefix; clear what the search touched
    for (int i = best_len + threadIdx.x; i < nm; i += blockDim.x) {
        const int v = ml[i];
        G.part[v] = G.part[v] == a ? b : a;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < tl; i += blockDim.x) {
        const int v = vl[i];
        f.flags[v] = 0;
        f.ver[v] = 0;
    }
    // 5. block weights and boundary candidates of the kept moves (the moved vertex and
    // its neighbours in its old block, as the commit of a flow does)
    if (threadIdx.x == 0) {
        G.blockw[a] = S.best_wA;
        G.blockw[b] = S.best_wB;
        *R = FmRes{cut0, wA0, wB0, S.best_cut, S.best_wA, S.best_wB, best_len, nm};
    }
    if (G.bl) {
        for (int i = threadIdx.x; i < best_len; i += blockDim.x) {
            const int v = ml[i];
            const int ob = G.part[v] == a ? b : a;
            if (!__ldcg(G.inb + v) && atomicExch(G.inb + v, 1) == 0) G.bl[atomicAdd(G.blc, 1)] = v;
            const int j1 = __ldg(G.xadj + v + 1);
            for (int j = __ldg(G.xadj + v); j < j1; ++j) {
                const int x = __ldg(G.adjncy + j);
                if (__ldcg(G.inb + x)) continue;
                if (G.part[x] == ob && atomicExch(G.inb + x, 1) == 0) G.bl[atomicAdd(G.blc, 1)] = x;
            }
        }
    }
    __syncthreads();
    mark(T_FM_FINISH);
}

size_t fm_pair_smem() {
    return sizeof(FmShared) + (8ull + 4 + 4) * kFmSortSmem;
}

static bool g_fm_setup = false;

cudaError_t launch_fm(const Work &w, const FmDev &f, int k, int sms, cudaStream_t st, int *nl) {
    if (!g_fm_setup) {
        cudaError_t e = cudaFuncSetAttribute(fm_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)fm_pair_smem());
        if (e != cudaSuccess) return e;
        g_fm_setup = true;
    }
    if (w.npairs <= 0) return cudaSuccess;
    const int grid = 4 * (sms > 0 ? sms : 1);
    fm_count_kernel<<<grid, kFmTPB, 2 * sizeof(int) * (size_t)k, st>>>(w, f);
    fm_offsets_kernel<<<1, 1024, 0, st>>>(w, f);
    fm_gather_kernel<<<grid, kFmTPB, 0, st>>>(w, f);
    fm_pair_kernel<<<w.npairs, kFmTPB, fm_pair_smem(), st>>>(w, f);
    *nl += 4;
    return cudaGetLastError();
}

}  // namespace fr
