// Multi-try FM after the pairwise improvements of a matching (Sanders & Schulz,
// Section 4.2, run from active block scheduling as Section 4.3 describes): every
// boundary vertex of a pair goes on the pair's todo list, the list is taken in a
// random order, and each vertex that no earlier search of the pass touched and that
// still lies on the boundary starts a k-way local search from itself and its boundary
// neighbours; no search touches a vertex an earlier search of the pass touched.
//
// The k-way search is the one of Section 2.2: a single queue keyed by the max gain
// g(v) = max_P omega(v, P) - omega(v, own block) over the blocks P next to v; the
// best vertex moves to its best block unless that block would exceed L_max; each
// vertex moves at most once; the search stops when the queue is empty or by the
// KaSPar rule (over the p moves since the last new minimum, with mean mu and variance
// sigma^2 of their gains: p mu^2 > alpha sigma^2 + beta, beta = ln n) and rolls back
// to the first lowest cut.  Readings, as in the CPU oracle: keys order by gain, then
// by the time of the vertex's last keying (later first): the start set in its order,
// then after each move the moved vertex's neighbours in CSR order; target ties go to
// the smaller splitmix64(tseed ^ u << 32 ^ P); a vertex that may not move leaves the
// queue; after a move every unmoved neighbour the search may touch is keyed again if
// it is a boundary vertex and leaves the queue if not; the pairs' todo lists are
// visited round-robin (entry j of every pair in pair order, then entry j + 1).
//
// GPU form.  The searches of a pass are sequential by definition: each sees the
// partition and the touched marks the earlier ones left.  So one warp runs the whole
// pass (all lanes in lockstep; lane 0 pops and moves, the lanes key the moved
// vertex's neighbours 32 at a time, each lane computing its neighbour's connection
// weights from the adjacency in registers).  The queue is an array of gain buckets,
// each a stack of entries in global memory with its top and a non-empty bitmap in
// shared memory; an entry carries what the move needs (vertex, target, block, weight,
// adjacency range) and a live flag: keying pushes a new entry (so each stack stays
// ordered by keying time) and clears the flag of the vertex's previous entry of the same
// search; pops skip dead entries.  The block weights live in shared memory for the pass.
// Grid-wide kernels before it count the pair boundaries and block weights, fill the
// todo lists and sort each (one CTA per pair, bitonic by key).
//
// The same search, without the touched rule and started from the whole boundary (or
// its corner vertices), makes one round of the global k-way refinement (end of file).
#include <climits>

#include "mt_kernel.cuh"

namespace fr {

constexpr int kMtTPB = 256;
constexpr unsigned kFull = 0xffffffffu;

// Pair of the pass that v's block belongs to (and the partner block), if v has a
// neighbour in the partner block; else -1.
__device__ __forceinline__ int mt_pair_of(const GraphDev &G, const MtDev &m, int v, int *partner) {
    const int x = G.part[v];
    const int p = m.bpair[x];
    if (p < 0) return -1;
    const int other = m.pa[p] == x ? m.pb[p] : m.pa[p];
    const int j1 = __ldg(G.xadj + v + 1);
    for (int j = __ldg(G.xadj + v); j < j1; ++j)
        if (G.part[__ldg(G.adjncy + j)] == other) {
            *partner = other;
            return p;
        }
    return -1;
}

__device__ __forceinline__ unsigned long long mt_list_seed(unsigned long long seed, int a, int b) {
    return splitmix64(splitmix64(seed ^ ((unsigned long long)(unsigned)a << 32) ^ (unsigned)b) + 1);
}

// Block weights and the todo list length of every pair.
__global__ void __launch_bounds__(kMtTPB) mt_count_kernel(GraphDev G, MtDev m) {
    extern __shared__ long long s_bw[];   // [k]
    for (int i = threadIdx.x; i < G.k; i += blockDim.x) s_bw[i] = 0;
    __syncthreads();
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < G.n; v += gridDim.x * blockDim.x) {
        const int c = __ldg(G.vwgt + v);
        if (c) atomicAdd(reinterpret_cast<unsigned long long *>(s_bw + G.part[v]), (unsigned long long)c);
        int partner;
        const int p = mt_pair_of(G, m, v, &partner);
        if (p >= 0) atomicAdd(m.cnt + p, 1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < G.k; i += blockDim.x)
        if (s_bw[i]) atomicAdd(reinterpret_cast<unsigned long long *>(m.bw + i), (unsigned long long)s_bw[i]);
}

// Todo list offsets, each list padded to a power of two for its sort.
__global__ void mt_offsets_kernel(MtDev m, Ctl *ctl) {
    if (threadIdx.x != 0) return;
    long long o = 0;
    for (int p = 0; p < m.np; ++p) {
        m.off[p] = o;
        long long q = 1;
        while (q < m.cnt[p]) q <<= 1;
        o += q;
        m.fil[p] = 0;
    }
    m.off[m.np] = o;
    if (o > m.scap) fail(ctl, E_INTERNAL, 801);
}

__global__ void __launch_bounds__(kMtTPB) mt_fill_kernel(GraphDev G, MtDev m, Ctl *ctl) {
    if (__ldcg(&ctl->error)) return;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < G.n; v += gridDim.x * blockDim.x) {
        int partner;
        const int p = mt_pair_of(G, m, v, &partner);
        if (p < 0) continue;
        const int pos = atomicAdd(m.fil + p, 1);
        if (pos >= m.cnt[p]) {   // cannot happen: the count pass saw the same partition
            fail(ctl, E_INTERNAL, 802);
            return;
        }
        const long long i = m.off[p] + pos;
        m.tv[i] = v;
        m.tkey[i] = splitmix64(mt_list_seed(m.seed, m.pa[p], m.pb[p]) ^ (unsigned long long)(unsigned)v);
    }
}

// One CTA per pair: its todo list ascending by (key, vertex), bitonic in global memory.
__global__ void __launch_bounds__(kMtTPB) mt_sort_kernel(MtDev m, Ctl *ctl) {
    if (__ldcg(&ctl->error)) return;
    const int p = blockIdx.x;
    const long long o = m.off[p], len = m.off[p + 1] - o;
    const int c = m.cnt[p];
    unsigned long long *K = m.tkey + o;
    int *V = m.tv + o;
    for (long long i = c + threadIdx.x; i < len; i += blockDim.x) {
        K[i] = ~0ull;
        V[i] = INT_MAX;
    }
    __syncthreads();
    for (long long kk = 2; kk <= len; kk <<= 1)
        for (long long j = kk >> 1; j > 0; j >>= 1) {
            for (long long i = threadIdx.x; i < len; i += blockDim.x) {
                const long long l = i ^ j;
                if (l <= i) continue;
                const unsigned long long ki = K[i], kl = K[l];
                const int vi = V[i], vl = V[l];
                const bool l_less = kl < ki || (kl == ki && vl < vi);
                const bool i_less = ki < kl || (ki == kl && vi < vl);
                if ((i & kk) == 0 ? l_less : i_less) {
                    K[i] = kl; K[l] = ki;
                    V[i] = vl; V[l] = vi;
                }
            }
            __syncthreads();
        }
}

// ---------------------------------------------------------------- the pass ----

// Max gain of u and its target: the adjacent block other than u's own with the largest
// connection weight, ties to the smaller splitmix64(tseed ^ u << 32 ^ P), then the
// smaller P.  False if u has no neighbour outside its block.  Up to 8 blocks around u
// are summed in registers; more fall back to summing each block over the adjacency.
// The arcs are read 16 at a time, their heads' blocks loaded together after them, so
// that a vertex costs two dependent memory round trips per 16 arcs; a vertex of degree
// <= 32 takes the register-only path below.
// (pu, j0, j1: u's block and adjacency range, loaded by the caller)
__device__ bool mt_gain(const GraphDev &G, int u, int pu, int j0, int j1, unsigned long long tseed, int &gain,
                        int &to) {
    constexpr int T = 8;
    int tb[T], tw[T];
#pragma unroll
    for (int s = 0; s < T; ++s) { tb[s] = -1; tw[s] = 0; }
    int own = 0, nt = 0;
    bool over = false;
    auto fold = [&](int P, int w) {
        if (P == pu) { own += w; return; }
        bool hit = false;
#pragma unroll
        for (int s = 0; s < T; ++s)
            if (tb[s] == P) { tw[s] += w; hit = true; }
        if (!hit) {
            if (nt < T) {
#pragma unroll
                for (int s = 0; s < T; ++s)
                    if (s == nt) { tb[s] = P; tw[s] = w; }
                ++nt;
            } else {
                over = true;
            }
        }
    };
    constexpr int C = 16;
    constexpr int CF = 32;
    if (j1 - j0 <= CF) {
        // degree <= 32: the arcs and their heads' blocks in registers, then one pass over
        // them per distinct foreign block (in the order of first appearance), each a set
        // of independent compares; a target's hash only when its weight ties the best
        const int deg = j1 - j0;
        int a[CF], wv[CF], P[CF];
#pragma unroll
        for (int s = 0; s < CF; ++s) {
            a[s] = s < deg ? __ldg(G.adjncy + j0 + s) : 0;
            wv[s] = s < deg ? __ldg(G.adjwgt + j0 + s) : 0;
        }
#pragma unroll
        for (int s = 0; s < CF; ++s) P[s] = s < deg ? G.part[a[s]] : pu;
        unsigned rem = 0;
#pragma unroll
        for (int s = 0; s < CF; ++s) {
            if (P[s] == pu) own += wv[s];
            else rem |= 1u << s;
        }
        if (!rem) return false;
        const unsigned long long hu = tseed ^ ((unsigned long long)(unsigned)u << 32);
        int best = -1, bw = 0;
        unsigned long long bh = 0;
        bool hv = false;
        while (rem) {
            int B = 0;
#pragma unroll
            for (int s = CF - 1; s >= 0; --s)
                if ((rem >> s) & 1u) B = P[s];
            int wB = 0;
            unsigned hit = 0;
#pragma unroll
            for (int s = 0; s < CF; ++s)
                if (((rem >> s) & 1u) && P[s] == B) {
                    wB += wv[s];
                    hit |= 1u << s;
                }
            rem &= ~hit;
            if (best < 0 || wB > bw) {
                best = B;
                bw = wB;
                hv = false;
            } else if (wB == bw) {
                const unsigned long long hB = splitmix64(hu ^ (unsigned)B);
                if (!hv) {
                    bh = splitmix64(hu ^ (unsigned)best);
                    hv = true;
                }
                if (hB < bh || (hB == bh && B < best)) {
                    best = B;
                    bh = hB;
                }
            }
        }
        gain = bw - own;
        to = best;
        return true;
    }
    for (int j = j0; j < j1; j += C) {
        int a[C], wv[C], P[C];
#pragma unroll
        for (int s = 0; s < C; ++s) {
            a[s] = j + s < j1 ? __ldg(G.adjncy + j + s) : -1;
            wv[s] = j + s < j1 ? __ldg(G.adjwgt + j + s) : 0;
        }
#pragma unroll
        for (int s = 0; s < C; ++s) P[s] = a[s] >= 0 ? G.part[a[s]] : -1;
#pragma unroll
        for (int s = 0; s < C; ++s)
            if (a[s] >= 0) fold(P[s], wv[s]);
    }
    if (nt == 0) return false;
    const unsigned long long hu = tseed ^ ((unsigned long long)(unsigned)u << 32);
    int best = -1, bw = 0;
    unsigned long long bh = 0;
    auto consider = [&](int P, int w) {
        const unsigned long long h = splitmix64(hu ^ (unsigned)P);
        if (best < 0 || w > bw || (w == bw && (h < bh || (h == bh && P < best)))) { best = P; bw = w; bh = h; }
    };
    if (!over) {
#pragma unroll
        for (int s = 0; s < T; ++s)
            if (s < nt) consider(tb[s], tw[s]);
    } else {
        for (int j = j0; j < j1; ++j) {
            const int P = G.part[__ldg(G.adjncy + j)];
            if (P == pu) continue;
            bool first = true;
            for (int q = j0; q < j && first; ++q) first = G.part[__ldg(G.adjncy + q)] != P;
            if (!first) continue;
            int wsum = 0;
            for (int q = j; q < j1; ++q)
                if (G.part[__ldg(G.adjncy + q)] == P) wsum += __ldg(G.adjwgt + q);
            consider(P, wsum);
        }
    }
    gain = bw - own;
    to = best;
    return true;
}

__device__ __forceinline__ bool mt_gain(const GraphDev &G, int u, unsigned long long tseed, int &gain, int &to) {
    return mt_gain(G, u, G.part[u], __ldg(G.xadj + u), __ldg(G.xadj + u + 1), tseed, gain, to);
}

// KaSPar rule p mu^2 > alpha sigma^2 + beta (mu, sigma^2: mean and variance of the p
// gains since the last new minimum; S1, S2: their sum and sum of squares), decided as the
// oracle's rounded double operations in its order decide it.  Times p^2 the rule reads
// D = p S1^2 - alpha (p S2 - S1^2) - beta p^2 > 0.  D is first estimated in single
// precision; with M the sum of the four terms' magnitudes, that estimate is within about
// 1.1e-6 M of the exact D (18 roundings of 2^-24), and the double expression within
// about 1e-15 M, so whenever the estimate exceeds 1e-5 M in magnitude all three have the
// same sign.  Only the rest take the double path (FP64 is slow on this part).
__device__ __forceinline__ bool kaspar_stop(int p, long long S1, long long S2, int alpha, double beta) {
    {
        const float pf = (float)p, s1 = (float)S1, s2 = (float)S2, af = (float)alpha, bf = (float)beta;
        const float s11 = s1 * s1;
        const float t1 = pf * s11, t2 = af * (pf * s2), t3 = af * s11, t4 = bf * (pf * pf);
        const float D = ((t1 - t2) + t3) - t4;
        const float M = ((t1 + t2) + t3) + t4;
        if (fabsf(D) > 1e-5f * M) return D > 0.f;
    }
    const double pd = (double)p;
    const double mu = __ddiv_rn((double)S1, pd);
    const double var = __dsub_rn(__ddiv_rn((double)S2, pd), __dmul_rn(mu, mu));
    const double lhs = __dmul_rn(__dmul_rn(pd, mu), mu);
    const double rhs = __dadd_rn(__dmul_rn((double)alpha, var), beta);
    return lhs > rhs;
}

__device__ __forceinline__ unsigned mt_lanemask_lt() {
    unsigned r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

struct MtShared {
    int top[kMtBuckets];               // top entry of each gain bucket, -1 empty
    unsigned bits[kMtBuckets / 32];    // non-empty buckets (possibly holding only dead entries)
    long long bw[kMtMaxK];             // block weights during the pass
};

// A queue entry: two int4, {vertex, entry below it in its bucket, live, target block}
// and {block, weight, adjacency begin, adjacency end} of the vertex, so that a pop is
// one memory round trip.  Keying a vertex again clears `live` in its previous entry of
// the same search (cur[v] = search epoch << 32 | entry).
__device__ __forceinline__ void mt_kill(const MtDev &m, unsigned long long cu, unsigned epoch) {
    if ((unsigned)(cu >> 32) == epoch) reinterpret_cast<int *>(m.ent + 2 * (cu & 0xffffffffull))[2] = 0;
}

// Pushes the lanes' entries (in lane order) onto their buckets: entries go to
// [nxt, nxt + popc(pm)); a lower lane's entry lies below a higher lane's in one bucket.
// Each pushing lane's vertex u gets cur[u] = this entry.
__device__ __forceinline__ void mt_push(MtShared &S, const MtDev &m, unsigned pm, bool push, int bk, int u, int tu,
                                        int pu, int cw, int u0, int u1, unsigned epoch, long long nxt, int lane) {
    const long long pos = nxt + __popc(pm & mt_lanemask_lt());
    const unsigned grp = __match_any_sync(kFull, push ? bk : -1 - lane);
    const unsigned lower = grp & mt_lanemask_lt();
    const long long pos_lower = __shfl_sync(kFull, pos, lower ? 31 - __clz(lower) : lane);
    int below = -1;
    if (push) below = lower ? (int)pos_lower : S.top[bk];
    __syncwarp();
    if (push) {
        m.ent[2 * pos] = make_int4(u, below, 1, tu);
        m.ent[2 * pos + 1] = make_int4(pu, cw, u0, u1);
        m.cur[u] = ((unsigned long long)epoch << 32) | (unsigned long long)pos;
        if ((grp & ~lower & ~(1u << lane)) == 0) {   // highest lane of its bucket
            S.top[bk] = (int)pos;
            atomicOr(&S.bits[bk >> 5], 1u << (bk & 31));
        }
    }
    __syncwarp();
}

// One k-way search (one warp) from the entries already pushed, nxt of them: pop the
// highest live entry, move its vertex unless the target would exceed L_max, key its
// unmoved neighbours again (CSR order), stop by the KaSPar rule or an empty queue.
// touch: the multi-try pass's rule (a vertex another search of the pass queued is
// neither queued nor moved; what this search queues is marked with sid); false: no
// such rule (the global k-way rounds).  Returns the best prefix (best < 0 is the
// largest cut decrease), the moves made and kept, and whether the KaSPar rule stopped
// it; bad on an error.
__device__ __forceinline__ void mt_search(const GraphDev &G, const MtDev &m, MtShared &S, Ctl *ctl, int sid,
                                          bool touch, unsigned epoch, long long &nxt, long long Lmax,
                                          unsigned long long tseed, int lane, bool &bad, long long &best, int &nm,
                                          int &best_len, bool &stopped) {
    long long delta = 0, S1 = 0, S2 = 0;
    int pc = 0;
    best = 0;
    nm = 0;
    best_len = 0;
    stopped = false;
    while (!bad) {
        // pop the highest live entry
        int x = -1, g = 0, xto = 0, xfrom = 0, xc = 0, xy0 = 0, xy1 = 0;
        for (;;) {
            int hb = -1;
            for (int k2 = 1; k2 >= 0; --k2) {
                const unsigned word = S.bits[lane * 2 + k2];
                if (hb < 0 && word) hb = (lane * 2 + k2) * 32 + 31 - __clz(word);
            }
            const unsigned has = __ballot_sync(kFull, hb >= 0);
            if (!has) break;
            const int b = __shfl_sync(kFull, hb, 31 - __clz(has));
            int got = -1, gto = 0, gfrom = 0, gc = 0, gy0 = 0, gy1 = 0;
            if (lane == 0) {
                const int e = S.top[b];
                if (e < 0 || e >= nxt) {   // (never: a set bit has a pushed top entry)
                    S.top[b] = -1;
                    S.bits[b >> 5] &= ~(1u << (b & 31));
                } else {
                    const int4 h = m.ent[2 * e], d = m.ent[2 * e + 1];
                    S.top[b] = h.y;
                    if (h.y < 0) S.bits[b >> 5] &= ~(1u << (b & 31));
                    if (h.z) {   // live: the vertex leaves the queue
                        got = h.x;
                        gto = h.w; gfrom = d.x; gc = d.y; gy0 = d.z; gy1 = d.w;
                    }
                }
            }
            got = __shfl_sync(kFull, got, 0);
            __syncwarp();
            if (got >= 0) {
                x = got;
                g = b - kMtGmax;
                xto = __shfl_sync(kFull, gto, 0);
                xfrom = __shfl_sync(kFull, gfrom, 0);
                xc = __shfl_sync(kFull, gc, 0);
                xy0 = __shfl_sync(kFull, gy0, 0);
                xy1 = __shfl_sync(kFull, gy1, 0);
                break;
            }
        }
        if (x < 0) break;   // the queue is empty
        const int to = xto;
        const int from = xfrom;
        const long long cx = xc;
        if (S.bw[to] + cx > Lmax) continue;   // would overload the target: not moved
        if (lane == 0) {
            G.part[x] = to;
            S.bw[from] -= cx;
            S.bw[to] += cx;
            m.mvd[x] = 1;
            m.lmv[nm] = make_int4(x, from, to, (int)cx);
        }
        ++nm;
        delta -= g;
        __syncwarp();
        // key the neighbours again, 32 at a time in CSR order
        const int y0 = xy0, y1 = xy1;
        for (int jb = y0; jb < y1; jb += 32) {
            const int jj = jb + lane;
            const int u = jj < y1 ? __ldg(G.adjncy + jj) : -1;
            bool elig = false, push = false;
            int gu = 0, tu = -1, pu = 0, cw = 0, u0 = 0, u1 = 0;
            unsigned long long cu = 0;
            if (u >= 0) {
                // u's marks, block, weight, adjacency range and entry, loaded together
                const unsigned char mv = m.mvd[u];
                const int tc = touch ? m.tch[u] : 0;
                pu = G.part[u];
                cw = __ldg(G.vwgt + u);
                u0 = __ldg(G.xadj + u);
                u1 = __ldg(G.xadj + u + 1);
                cu = m.cur[u];
                elig = !mv && (tc == 0 || tc == sid);
                if (elig) push = mt_gain(G, u, pu, u0, u1, tseed, gu, tu);
            }
            const bool range = __all_sync(kFull, !push || (gu >= -kMtGmax && gu <= kMtGmax));
            const unsigned pm = __ballot_sync(kFull, push);
            if (!range || nxt + __popc(pm) > m.ecap) {
                if (lane == 0) fail(ctl, range ? E_INTERNAL : E_TOO_LARGE, 805);
                bad = true;
                break;
            }
            if (elig) mt_kill(m, cu, epoch);   // its old entry (if any) is dead from here on
            if (push && touch) m.tch[u] = sid;
            mt_push(S, m, pm, push, gu + kMtGmax, u, tu, pu, cw, u0, u1, epoch, nxt, lane);
            nxt += __popc(pm);
        }
        if (bad) break;
        if (delta < best) {
            best = delta; best_len = nm; pc = 0; S1 = 0; S2 = 0;
        } else {
            ++pc;
            S1 += g;
            S2 += (long long)g * g;
            if (kaspar_stop(pc, S1, S2, m.alpha, m.beta)) {
                stopped = true;
                break;
            }
        }
    }
    __syncwarp();
}

// After a search: roll back to the first lowest cut and clear the moved marks.  With
// bookkeeping (the multi-try pass), mark the blocks the kept moves left and entered and
// list the kept movers (kbase: the pass's count so far) for the boundary list, which
// mt_bl_kernel fills after the pass.
__device__ __forceinline__ void mt_finish(const GraphDev &G, const MtDev &m, MtShared &S, int nm, int best_len,
                                          int lane, bool keep, int &kbase) {
    for (int i = best_len + lane; i < nm; i += 32) {
        const int4 mv = m.lmv[i];
        G.part[mv.x] = mv.y;
        atomicAdd(reinterpret_cast<unsigned long long *>(&S.bw[mv.z]), (unsigned long long)(-(long long)mv.w));
        atomicAdd(reinterpret_cast<unsigned long long *>(&S.bw[mv.y]), (unsigned long long)(long long)mv.w);
    }
    __syncwarp();
    for (int i = lane; i < nm; i += 32) m.mvd[m.lmv[i].x] = 0;
    if (keep) {
        for (int i = lane; i < best_len; i += 32) {
            const int4 mv = m.lmv[i];
            m.chg[mv.y] = 1;
            m.chg[mv.z] = 1;
            m.kept[kbase + i] = mv.x;
        }
        kbase += best_len;
    }
    __syncwarp();
}

// Keys lane's vertex u for a start set (state loaded here): its gain and target, and,
// if it is a boundary vertex, its entry in the lanes' push.  Returns whether it pushes.
__device__ __forceinline__ bool mt_start_key(const GraphDev &G, const MtDev &m, int u, unsigned long long tseed,
                                             int &g, int &t, int &pu, int &cw, int &u0, int &u1,
                                             unsigned long long &cu) {
    pu = G.part[u];
    cw = __ldg(G.vwgt + u);
    u0 = __ldg(G.xadj + u);
    u1 = __ldg(G.xadj + u + 1);
    cu = m.cur[u];
    return mt_gain(G, u, pu, u0, u1, tseed, g, t);
}

// The whole pass: one warp.
__global__ void __launch_bounds__(32, 1) mt_pass_kernel(GraphDev G, MtDev m, Ctl *ctl) {
    __shared__ MtShared S;
    const int lane = threadIdx.x;
    if (__ldcg(&ctl->error)) return;
    if (G.k > kMtMaxK) {
        if (lane == 0) fail(ctl, E_TOO_LARGE, 803);
        return;
    }
    for (int i = lane; i < G.k; i += 32) S.bw[i] = m.bw[i];
    const unsigned long long tseed = splitmix64(~m.seed);
    const long long Lmax = G.Lmax;
    int maxlen = 0;
    for (int p = 0; p < m.np; ++p) maxlen = max(maxlen, m.cnt[p]);
    long long gain_tot = 0;
    int searches = 0, tried_tot = 0, kept_tot = 0, sid = 0;
    unsigned epoch = *m.epoch;
    int kbase = 0;   // kept movers listed so far (the list is kept_tot long at the end)
    bool bad = false;
    __syncwarp();
    // the todo entries in pass order (entry j of every pair, then j + 1), 32 at a time:
    // the lanes fetch them and their touched marks together; marks only ever go from 0
    // to set during a pass, so an entry seen touched is skipped at once and the others
    // are checked again when their turn comes
    const long long total = (long long)maxlen * m.np;
    for (long long pos = 0; pos < total && !bad; pos += 32) {
        const long long q = pos + lane;
        int cv = -1;
        bool fresh = false;
        if (q < total) {
            const int j = (int)(q / m.np), p = (int)(q - (long long)j * m.np);
            if (j < m.cnt[p]) {
                cv = m.tv[m.off[p] + j];
                fresh = m.tch[cv] == 0;
            }
        }
        unsigned live = __ballot_sync(kFull, fresh);
        while (live && !bad) {
            const int v = __shfl_sync(kFull, cv, __ffs(live) - 1);
            live &= live - 1;
            if (m.tch[v] != 0) continue;
            const int pv = G.part[v];
            const int x0 = __ldg(G.xadj + v), x1 = __ldg(G.xadj + v + 1);
            bool bnd = false;
            for (int jb = x0; jb < x1 && !bnd; jb += 32) {
                const int jj = jb + lane;
                bnd = __any_sync(kFull, jj < x1 && G.part[__ldg(G.adjncy + jj)] != pv);
            }
            if (!bnd) continue;
            ++sid;
            if (++epoch == 0) epoch = 1;
            // ---- one k-way search ----
            for (int i = lane; i < kMtBuckets; i += 32) S.top[i] = -1;
            for (int i = lane; i < kMtBuckets / 32; i += 32) S.bits[i] = 0;
            __syncwarp();
            long long nxt = 0;
            // start set: v, then its neighbours in CSR order that no search of the pass
            // queued and that are boundary vertices (all chosen before any is queued)
            const int deg = x1 - x0;
            for (int base = -1; base < deg && !bad; base += 32) {
                const int i = base + lane;
                int u = -1;
                if (i < 0) u = v;
                else if (i < deg) u = __ldg(G.adjncy + x0 + i);
                int g = 0, t = -1, pu = 0, cw = 0, u0 = 0, u1 = 0;
                unsigned long long cu = 0;
                bool push = false;
                if (u >= 0 && (u == v || m.tch[u] == 0)) push = mt_start_key(G, m, u, tseed, g, t, pu, cw, u0, u1, cu);
                const bool range = __all_sync(kFull, !push || (g >= -kMtGmax && g <= kMtGmax));
                const unsigned pm = __ballot_sync(kFull, push);
                if (!range || nxt + __popc(pm) > m.ecap) {
                    if (lane == 0) fail(ctl, range ? E_INTERNAL : E_TOO_LARGE, 804);
                    bad = true;
                    break;
                }
                if (push) {
                    mt_kill(m, cu, epoch);
                    m.tch[u] = sid;
                }
                mt_push(S, m, pm, push, g + kMtGmax, u, t, pu, cw, u0, u1, epoch, nxt, lane);
                nxt += __popc(pm);
            }
            long long best;
            int nm, best_len;
            bool stopped;
            mt_search(G, m, S, ctl, sid, true, epoch, nxt, Lmax, tseed, lane, bad, best, nm, best_len, stopped);
            mt_finish(G, m, S, nm, best_len, lane, true, kbase);
            gain_tot -= best;
            tried_tot += nm;
            kept_tot += best_len;
            ++searches;
        }
    }
    __syncwarp();
    for (int i = lane; i < G.k; i += 32) {
        m.bw[i] = S.bw[i];
        G.blockw[i] = S.bw[i];
    }
    if (lane == 0) {
        *m.epoch = epoch;
        m.res->gain = gain_tot;
        m.res->searches = searches;
        m.res->tried = tried_tot;
        m.res->kept = kept_tot;
    }
}

// The boundary candidates of the pass's kept moves, as a flow's commit lists them: each
// mover and its neighbours outside its block (one warp per mover).  Taken on the
// partition the pass leaves: a vertex that is a boundary vertex after the pass is a
// mover, a neighbour of one in another block, or was one before the pass (and listed).
__global__ void __launch_bounds__(kMtTPB) mt_bl_kernel(GraphDev G, MtDev m, Ctl *ctl) {
    if (__ldcg(&ctl->error)) return;
    const int nk = m.res->kept;
    const int lane = threadIdx.x & 31;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nk; i += nw) {
        const int y = m.kept[i], t = G.part[y];
        const int a0 = __ldg(G.xadj + y), a1 = __ldg(G.xadj + y + 1);
        // slot a0 - 1 stands for the mover itself
        for (int q = a0 - 1 + lane; q < a1; q += 32) {
            const int z = q < a0 ? y : __ldg(G.adjncy + q);
            if ((q < a0 || G.part[z] != t) && !__ldcg(G.inb + z) && atomicExch(G.inb + z, 1) == 0)
                G.bl[atomicAdd(G.blc, 1)] = z;
        }
    }
}

cudaError_t launch_mt(const GraphDev &G, const MtDev &md, Ctl *ctl, int sms, cudaStream_t st, int *nl) {
    if (md.np <= 0) return cudaSuccess;
    cudaError_t e;
    if ((e = cudaMemsetAsync(md.tch, 0, sizeof(int) * (size_t)G.n, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(md.cnt, 0, sizeof(int) * (size_t)md.np, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(md.bw, 0, sizeof(long long) * (size_t)G.k, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(md.chg, 0, (size_t)G.k, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(md.res, 0, sizeof(MtRes), st)) != cudaSuccess) return e;
    const int grid = 4 * (sms > 0 ? sms : 1);
    mt_count_kernel<<<grid, kMtTPB, sizeof(long long) * (size_t)G.k, st>>>(G, md);
    mt_offsets_kernel<<<1, 32, 0, st>>>(md, ctl);
    mt_fill_kernel<<<grid, kMtTPB, 0, st>>>(G, md, ctl);
    mt_sort_kernel<<<md.np, kMtTPB, 0, st>>>(md, ctl);
    mt_pass_kernel<<<1, 32, 0, st>>>(G, md, ctl);
    *nl += 5;
    if (G.bl) {
        mt_bl_kernel<<<grid, kMtTPB, 0, st>>>(G, md, ctl);
        *nl += 1;
    }
    return cudaGetLastError();
}

// ------------------------------------------------- global k-way rounds ----
// One round of Section 2.2 with the setup of Section 6: a single k-way search started
// from every vertex with at least `need` blocks other than its own around it (1: the
// whole boundary; 2: the corner vertices), in ascending splitmix64(rs ^ v) order.
// Grid-wide: the start set is bucketed by the top bits of its keys (the keys are
// hashes, so the buckets hold a few entries each), each bucket is sorted by one
// thread, and the start vertices' gains and targets are computed side by side; then
// one warp queues them in order and runs the search.  Bucket scratch, in the entry
// array (free until the search): counts, fill cursors and offsets of the nb buckets
// (kw_scratch); the sorted start set: tv, with its packed gains and targets in tkey.

// True if v has at least `need` distinct blocks other than its own among its
// neighbours (need is 1 or 2).
__device__ __forceinline__ bool kw_start(const GraphDev &G, int v, int need) {
    const int pv = G.part[v];
    const int j1 = __ldg(G.xadj + v + 1);
    int first = -1;
    for (int j = __ldg(G.xadj + v); j < j1; ++j) {
        const int P = G.part[__ldg(G.adjncy + j)];
        if (P == pv || P == first) continue;
        if (need == 1 || first >= 0) return true;
        first = P;
    }
    return false;
}

// counts, fill cursors, offsets (nb + 1 each) of the start set's buckets
struct KwScratch {
    int *cnt, *fil, *off;
};
__device__ __forceinline__ KwScratch kw_scratch(const MtDev &m, int nb) {
    int *b = reinterpret_cast<int *>(m.ent);
    return {b, b + (nb + 1), b + 2 * (nb + 1)};
}

__global__ void __launch_bounds__(kMtTPB) kw_count_kernel(GraphDev G, MtDev m, int need, unsigned long long rs,
                                                          int bbits) {
    const KwScratch K = kw_scratch(m, 1 << bbits);
    extern __shared__ long long s_bw[];   // [k]
    for (int i = threadIdx.x; i < G.k; i += blockDim.x) s_bw[i] = 0;
    __syncthreads();
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < G.n; v += gridDim.x * blockDim.x) {
        const int c = __ldg(G.vwgt + v);
        if (c) atomicAdd(reinterpret_cast<unsigned long long *>(s_bw + G.part[v]), (unsigned long long)c);
        if (!kw_start(G, v, need)) continue;
        const unsigned long long key = splitmix64(rs ^ (unsigned long long)(unsigned)v);
        atomicAdd(K.cnt + (int)(key >> (64 - bbits)), 1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < G.k; i += blockDim.x)
        if (s_bw[i]) atomicAdd(reinterpret_cast<unsigned long long *>(m.bw + i), (unsigned long long)s_bw[i]);
}

// Exclusive scan of the bucket counts (one CTA of 1,024 threads); the start set's size
// goes to cnt[0].
__global__ void __launch_bounds__(1024) kw_offsets_kernel(MtDev m, int nb) {
    __shared__ int part_sum[1024];
    const KwScratch K = kw_scratch(m, nb);
    const int t = threadIdx.x;
    const int per = (nb + 1023) / 1024, b0 = min(nb, t * per), b1 = min(nb, b0 + per);
    int s = 0;
    for (int b = b0; b < b1; ++b) s += K.cnt[b];
    part_sum[t] = s;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {
        const int x = t >= d ? part_sum[t - d] : 0;
        __syncthreads();
        part_sum[t] += x;
        __syncthreads();
    }
    int o = part_sum[t] - s;
    for (int b = b0; b < b1; ++b) {
        K.off[b] = o;
        K.fil[b] = 0;
        o += K.cnt[b];
    }
    if (t == 1023) {
        K.off[nb] = part_sum[1023];
        m.cnt[0] = part_sum[1023];
    }
}

__global__ void __launch_bounds__(kMtTPB) kw_place_kernel(GraphDev G, MtDev m, int need, unsigned long long rs,
                                                          int bbits) {
    const KwScratch K = kw_scratch(m, 1 << bbits);
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < G.n; v += gridDim.x * blockDim.x) {
        if (!kw_start(G, v, need)) continue;
        const unsigned long long key = splitmix64(rs ^ (unsigned long long)(unsigned)v);
        const int b = (int)(key >> (64 - bbits));
        const int pos = K.off[b] + atomicAdd(K.fil + b, 1);
        m.tkey[pos] = key;
        m.tv[pos] = v;
    }
}

// Each bucket ascending by (key, vertex), one thread per bucket (insertion sort).
__global__ void __launch_bounds__(kMtTPB) kw_bsort_kernel(MtDev m, int nb) {
    const KwScratch K = kw_scratch(m, nb);
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        const int o0 = K.off[b], o1 = K.off[b + 1];
        for (int i = o0 + 1; i < o1; ++i) {
            const unsigned long long ki = m.tkey[i];
            const int vi = m.tv[i];
            int j = i - 1;
            while (j >= o0 && (m.tkey[j] > ki || (m.tkey[j] == ki && m.tv[j] > vi))) {
                m.tkey[j + 1] = m.tkey[j];
                m.tv[j + 1] = m.tv[j];
                --j;
            }
            m.tkey[j + 1] = ki;
            m.tv[j + 1] = vi;
        }
    }
}

// Gain and target of every start vertex on the round's starting partition, packed as
// (gain + kMtGmax) << 32 | target into tkey; a gain out of range fails the round.
__global__ void __launch_bounds__(kMtTPB) kw_gain_kernel(GraphDev G, MtDev m, Ctl *ctl) {
    const int ns = m.cnt[0];
    const unsigned long long tseed = splitmix64(~m.seed);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += gridDim.x * blockDim.x) {
        int g = 0, t = -1;
        if (!mt_gain(G, m.tv[i], tseed, g, t) || g < -kMtGmax || g > kMtGmax) {
            fail(ctl, E_INTERNAL, 806);
            return;
        }
        m.tkey[i] = ((unsigned long long)(unsigned)(g + kMtGmax) << 32) | (unsigned)t;
    }
}

// The round's queue, built on the grid: the start set pushed in its order makes bucket
// stacks in which an entry lies on the entry of the same bucket before it.  Each warp
// takes a chunk of kKwChunk entries and links them within the chunk (32 at a time, a
// shared-memory table of each bucket's last entry so far); kw_stitch_kernel then finds,
// per chunk and bucket, the last entry of the chunks before it, and kw_fix_kernel links
// each chunk's first entry of a bucket to it.  Entries as mt_push writes them.
constexpr int kKwWarps = 4;   // warps per CTA of kw_stack_kernel (a 2,048-entry table each)

__global__ void __launch_bounds__(32 * kKwWarps) kw_stack_kernel(GraphDev G, MtDev m, Ctl *ctl) {
    __shared__ int s_last[kKwWarps][kMtBuckets];
    if (__ldcg(&ctl->error)) return;   // (a gain out of range left the packed keys unwritten)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int ns = m.cnt[0];
    const int nch = (ns + kKwChunk - 1) / kKwChunk;
    const int chunk = blockIdx.x * kKwWarps + wid;
    if (chunk >= nch || chunk >= m.kwchunks) return;   // (the whole warp leaves together)
    unsigned epoch = *m.epoch + 1;
    if (epoch == 0) epoch = 1;
    int *last = s_last[wid];
    for (int b = lane; b < kMtBuckets; b += 32) last[b] = -1;
    __syncwarp();
    const int c0 = chunk * kKwChunk, c1 = min(ns, c0 + kKwChunk);
    for (int base = c0; base < c1; base += 32) {
        const int i = base + lane;
        const bool valid = i < c1;
        int u = 0, b = 0, t = 0, pu = 0, cw = 0, u0 = 0, u1 = 0;
        if (valid) {
            const unsigned long long pk = m.tkey[i];
            u = m.tv[i];
            b = min((int)(pk >> 32), kMtBuckets - 1);   // (always in range: the gains were checked)
            t = (int)(unsigned)pk;
            pu = G.part[u];
            cw = __ldg(G.vwgt + u);
            u0 = __ldg(G.xadj + u);
            u1 = __ldg(G.xadj + u + 1);
        }
        const unsigned grp = __match_any_sync(kFull, valid ? b : -1 - lane);
        const unsigned lower = grp & mt_lanemask_lt();
        int below = -1;
        if (valid) below = lower ? base + 31 - __clz(lower) : last[b];
        __syncwarp();
        if (valid) {
            m.ent[2LL * i] = make_int4(u, below, 1, t);
            m.ent[2LL * i + 1] = make_int4(pu, cw, u0, u1);
            m.cur[u] = ((unsigned long long)epoch << 32) | (unsigned long long)(unsigned)i;
            if ((grp & ~lower & ~(1u << lane)) == 0) last[b] = i;   // highest lane of its bucket
        }
        __syncwarp();
    }
    int *cl = m.kwtab + (long long)chunk * kMtBuckets;
    for (int b = lane; b < kMtBuckets; b += 32) cl[b] = last[b];
}

// One thread per bucket: over the chunks in order, the last entry before each chunk,
// and the bucket's top after all of them.
__global__ void __launch_bounds__(256) kw_stitch_kernel(MtDev m) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= kMtBuckets) return;
    const int ns = m.cnt[0];
    const int nch = min((ns + kKwChunk - 1) / kKwChunk, m.kwchunks);
    const int *cl = m.kwtab;
    int *prev = m.kwtab + (long long)m.kwchunks * kMtBuckets;
    int carry = -1;
    for (int k = 0; k < nch; ++k) {
        prev[(long long)k * kMtBuckets + b] = carry;
        const int p = cl[(long long)k * kMtBuckets + b];
        if (p >= 0) carry = p;
    }
    m.kwtab[2LL * m.kwchunks * kMtBuckets + b] = carry;
}

__global__ void __launch_bounds__(kMtTPB) kw_fix_kernel(MtDev m, Ctl *ctl) {
    if (__ldcg(&ctl->error)) return;
    const int ns = m.cnt[0];
    const int *prev = m.kwtab + (long long)m.kwchunks * kMtBuckets;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += gridDim.x * blockDim.x) {
        int *below = reinterpret_cast<int *>(m.ent + 2LL * i) + 1;
        if (*below >= 0) continue;
        const int b = min((int)(m.tkey[i] >> 32), kMtBuckets - 1);
        *below = prev[(long long)(i / kKwChunk) * kMtBuckets + b];
    }
}

// The round's search: one warp takes the queue the grid built and searches.
// res: gain kept, tried, kept; stopped = 1 if the KaSPar rule stopped the search.
__global__ void __launch_bounds__(32, 1) kw_search_kernel(GraphDev G, MtDev m, Ctl *ctl) {
    __shared__ MtShared S;
    const int lane = threadIdx.x;
    if (__ldcg(&ctl->error)) return;
    for (int i = lane; i < G.k; i += 32) S.bw[i] = m.bw[i];
    const int *top = m.kwtab + 2LL * m.kwchunks * kMtBuckets;
    for (int i = lane; i < kMtBuckets; i += 32) S.top[i] = top[i];
    for (int w = lane; w < kMtBuckets / 32; w += 32) {
        unsigned word = 0;
        for (int j = 0; j < 32; ++j) word |= (top[w * 32 + j] >= 0 ? 1u : 0u) << j;
        S.bits[w] = word;
    }
    __syncwarp();
    const unsigned long long tseed = splitmix64(~m.seed);
    const int ns = m.cnt[0];
    unsigned epoch = *m.epoch + 1;
    if (epoch == 0) epoch = 1;
    bool bad = false;
    long long nxt = ns;
    long long best = 0;
    int nm = 0, best_len = 0, kbase = 0;
    bool stopped = false;
    mt_search(G, m, S, ctl, 0, false, epoch, nxt, G.Lmax, tseed, lane, bad, best, nm, best_len, stopped);
    mt_finish(G, m, S, nm, best_len, lane, false, kbase);
    for (int i = lane; i < G.k; i += 32) m.bw[i] = S.bw[i];
    if (lane == 0) {
        *m.epoch = epoch;
        m.res->gain = -best;
        m.res->searches = 1;
        m.res->tried = nm;
        m.res->kept = best_len;
        m.res->stopped = stopped ? 1 : 0;
    }
}

cudaError_t launch_kway_round(const GraphDev &G, const MtDev &md, Ctl *ctl, int need, unsigned long long rs,
                              int sms, cudaStream_t st, int *nl) {
    int bbits = 1;
    while (bbits < 16 && (2ll << (bbits + 3)) <= G.n) ++bbits;   // about 8 vertices per bucket
    const int nb = 1 << bbits;
    cudaError_t e;
    if ((e = cudaMemsetAsync(md.ent, 0, sizeof(int) * (size_t)nb, st)) != cudaSuccess) return e;   // bucket counts
    if ((e = cudaMemsetAsync(md.bw, 0, sizeof(long long) * (size_t)G.k, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(md.res, 0, sizeof(MtRes), st)) != cudaSuccess) return e;
    const int grid = 4 * (sms > 0 ? sms : 1);
    kw_count_kernel<<<grid, kMtTPB, sizeof(long long) * (size_t)G.k, st>>>(G, md, need, rs, bbits);
    kw_offsets_kernel<<<1, 1024, 0, st>>>(md, nb);
    kw_place_kernel<<<grid, kMtTPB, 0, st>>>(G, md, need, rs, bbits);
    kw_bsort_kernel<<<(nb + kMtTPB - 1) / kMtTPB, kMtTPB, 0, st>>>(md, nb);
    kw_gain_kernel<<<grid, kMtTPB, 0, st>>>(G, md, ctl);
    // the queue: chunks of the start set linked by warps, stitched per bucket, fixed up
    const int chunks = (G.n + kKwChunk - 1) / kKwChunk;   // >= the start set's chunks
    kw_stack_kernel<<<(chunks + kKwWarps - 1) / kKwWarps, 32 * kKwWarps, 0, st>>>(G, md, ctl);
    kw_stitch_kernel<<<(kMtBuckets + 255) / 256, 256, 0, st>>>(md);
    kw_fix_kernel<<<grid, kMtTPB, 0, st>>>(md, ctl);
    kw_search_kernel<<<1, 32, 0, st>>>(G, md, ctl);
    *nl += 9;
    return cudaGetLastError();
}

}  // namespace fr
