// Two-way FM local search with TopGain on each pair of a round, before the pair's flow
// (Sanders & Schulz, Section 2.2: one priority queue of movable vertices per block,
// keyed by the gain -- the decrease of the pair cut when the vertex changes blocks --,
// every vertex moves at most once, the queues start with the boundary in random order,
// TopGain takes the block whose best vertex has the larger gain and the heavier block
// while one is overloaded, and the moves are rolled back to the best cut found within
// the balance constraint; the setup of Section 5 stops a search once more than a given
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

// Boundary of every pair: weights to the own block and to the partner block within
// G[A u B]; vertices with an edge to the partner enter their pair's list.  Reads the
// boundary candidate list when there is one (a superset of the k-way boundary).
__global__ void __launch_bounds__(kFmTPB) fm_gather_kernel(Work w, FmDev f) {
    if ((w.prev_err && __ldcg(w.prev_err)) || __ldcg(&w.ctl->error)) return;
    const GraphDev G = w.graphs[0];
    const long long cnt = G.bl ? (long long)__ldcg(G.blc) : (long long)G.n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < cnt;
         i += (long long)gridDim.x * blockDim.x) {
        const int v = G.bl ? __ldcg(G.bl + i) : (int)i;
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
        if (ex == 0) continue;
        f.in[v] = in;
        f.ext[v] = ex;
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

struct FmShared {
    int top[2 * kFmMaxBuckets];          // top entry of each (block, bucket) stack, -1 empty
    unsigned bits[2 * kFmMaxBuckets / 32];   // non-empty (or holding stale entries) stacks
    long long red[kFmTPB / 32];
    int best_len, tried;
    long long best_cut, best_wA, best_wB;
};

__global__ void __launch_bounds__(kFmTPB) fm_pair_kernel(Work w, FmDev f) {
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
    for (int i = threadIdx.x; i < 2 * kFmMaxBuckets / 32; i += blockDim.x) S.bits[i] = 0;
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
            atomicOr(&S.bits[bk >> 5], 1u << (bk & 31));
        }
    }
    __syncthreads();

    // 3. the moves (warp 0)
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
            // top entry of each block: highest bucket whose top is current
            int tb[2];
            for (int s = 0; s < 2; ++s) {
                tb[s] = -1;
                for (;;) {
                    // highest set bit among the block's bucket words (kFmMaxBuckets / 32 = 128
                    // words: four per lane)
                    // lane L looks at words 4L..4L+3, from the top
                    int best = -1;
                    for (int k4 = 3; k4 >= 0; --k4) {
                        const unsigned word = S.bits[s * (kFmMaxBuckets / 32) + lane * 4 + k4];
                        if (best < 0 && word) best = (lane * 4 + k4) * 32 + 31 - __clz(word);
                    }
                    const unsigned has = __ballot_sync(0xffffffffu, best >= 0);
                    if (!has) break;
                    const int src = 31 - __clz(has);
                    const int hb = __shfl_sync(0xffffffffu, best, src);
                    const int key = s * kFmMaxBuckets + hb;
                    const int e = S.top[key];
                    int ok = 0;
                    if (lane == 0) {
                        const int v = f.ent_v[e];
                        const unsigned char fl = f.flags[v];
                        ok = (fl & kFmInQ) && !(fl & kFmMoved) && f.ver[v] == f.ent_ver[e];
                        if (!ok) {
                            const int below = f.ent_below[e];
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
            const int e = S.top[key];
            const int v = f.ent_v[e];
            const int g = tb[s] - gmax;
            const int from = s ? b : a, to = s ? a : b;
            __syncwarp();
            if (lane == 0) {
                const int below = f.ent_below[e];
                S.top[key] = below;
                if (below < 0) S.bits[key >> 5] &= ~(1u << (key & 31));
                f.flags[v] = kFmTouched | kFmMoved;
                G.part[v] = to;
                ml[nm] = v;
            }
            ++nm;
            cut -= g;
            const long long cv = __ldg(G.vwgt + v);
            if (s == 0) { wA -= cv; wB += cv; } else { wB -= cv; wA += cv; }
            __syncwarp();
            // the moved vertex's arcs, 32 at a time in adjacency order
            const int j0 = __ldg(G.xadj + v), j1 = __ldg(G.xadj + v + 1);
            for (int jb = j0; jb < j1; jb += 32) {
                const int j = jb + lane;
                bool act = false;
                int u = -1, nin = 0, nex = 0, ukey = -1;
                if (j < j1) {
                    u = __ldg(G.adjncy + j);
                    const int pu = G.part[u];
                    if (pu == a || pu == b) {
                        const unsigned char fl = f.flags[u];
                        if (!(fl & kFmMoved)) {
                            act = true;
                            if (fl & kFmTouched) {
                                const int wt = __ldg(G.adjwgt + j);
                                nin = f.in[u];
                                nex = f.ext[u];
                                if (pu == from) { nin -= wt; nex += wt; }
                                else { nin += wt; nex -= wt; }
                            } else {
                                // first touch: weights from the current blocks (v already moved)
                                const int partner = pu == a ? b : a;
                                const int k1 = __ldg(G.xadj + u + 1);
                                for (int k = __ldg(G.xadj + u); k < k1; ++k) {
                                    const int px = G.part[__ldg(G.adjncy + k)];
                                    const int wt = __ldg(G.adjwgt + k);
                                    if (px == pu) nin += wt;
                                    else if (px == partner) nex += wt;
                                }
                            }
                            ukey = (pu == a ? 0 : kFmMaxBuckets) + (nex - nin) + gmax;
                        }
                    }
                }
                // first touches join the touched list (for the cleanup)
                const bool fresh = act && !(f.flags[u] & kFmTouched);
                const unsigned fm_ = __ballot_sync(0xffffffffu, fresh);
                if (fresh) vl[tl + __popc(fm_ & lanemask_lt())] = u;
                tl += __popc(fm_);
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
                int below = -1;
                if (push) below = lower ? (int)pos_lower : S.top[ukey];
                __syncwarp();
                if (act) {
                    f.in[u] = nin;
                    f.ext[u] = nex;
                    const int nv = f.ver[u] + 1;
                    f.ver[u] = nv;
                    f.flags[u] = (unsigned char)(kFmTouched | (push ? kFmInQ : 0));
                    if (push) {
                        f.ent_v[pos] = u;
                        f.ent_ver[pos] = nv;
                        f.ent_below[pos] = below;
                        if ((grp & ~lower & ~(1u << lane)) == 0) {   // highest lane of the group
                            S.top[ukey] = (int)pos;
                            atomicOr(&S.bits[ukey >> 5], 1u << (ukey & 31));
                        }
                    }
                }
                nxt += __popc(pm);
                __syncwarp();
            }
            if (bad) break;
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
