// Multilevel V-cycle with a given partition (Sanders & Schulz, Sections 2.1, 2.2 and
// 5): edges are rated by expansion*2 = omega(u, v)^2 / (c(u) c(v)), matched inside
// blocks only (the given partition survives every contraction), contracted, and the
// partition is projected back level by level with the flow refinement on each level.
//
// Matching.  The readings (as in the CPU oracle) fix a strict order on the allowed
// edges -- rating, exact in 128-bit integers with c taken as max(c, 1); then the larger
// splitmix64(seed_l ^ min << 32 ^ max); then the smaller (min, max) -- and the matching
// is the greedy one in that order.  The GPU computes it with locally dominant edges: in
// every round each free vertex points at its best allowed edge to a free vertex, and
// two vertices pointing at each other are matched.  The best remaining edge is always
// such a pair, and an edge matched this way is the one greedy takes (every better edge
// at its ends is already gone), so the rounds end with exactly the greedy matching.
// A vertex with no allowed edge to a free vertex is marked dead and skipped.
//
// Contraction.  The smaller end of a pair, or a single vertex, represents a coarse
// vertex; coarse ids follow the representatives' fine ids (an exclusive scan).  A warp
// builds each coarse row: the members' arcs mapped to coarse ids, the matched edge
// dropped, sorted by a bitonic sort in shared memory and merged (parallel edges summed);
// rows longer than the shared buffer are built by selecting the next larger coarse id
// straight from the adjacencies.  A counting pass sizes the rows, a scan places them.
#include <climits>

#include "ml_kernel.cuh"

namespace fr {

constexpr unsigned kMlFull = 0xffffffffu;
constexpr int kMlTPB = 256;
constexpr int kMlRowSmem = 1024;   // entries of a coarse row sorted in shared memory

__device__ __forceinline__ unsigned ml_lanemask_lt() {
    unsigned r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

// ------------------------------------------------------------------ matching ----

struct MlKey {
    unsigned long long w2, cc, h;   // omega^2, max(c(a),1) * max(c(b),1), tie hash
    int a, b;                       // a < b
};

// x before y in the matching order: larger rating w2 / cc, larger hash, smaller (a, b)
__device__ __forceinline__ bool ml_higher(const MlKey &x, const MlKey &y) {
    const unsigned __int128 lx = (unsigned __int128)x.w2 * y.cc;
    const unsigned __int128 ly = (unsigned __int128)y.w2 * x.cc;
    if (lx != ly) return lx > ly;
    if (x.h != y.h) return x.h > y.h;
    if (x.a != y.a) return x.a < y.a;
    return x.b < y.b;
}

__global__ void __launch_bounds__(kMlTPB) ml_point_kernel(MlGraph g, const int *part, int k, long long W,
                                                          unsigned long long seed_l, int *mate, int *cand) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < g.n; v += gridDim.x * blockDim.x) {
        if (mate[v] != -1) { cand[v] = -1; continue; }
        const long long cv = __ldg(g.vwgt + v);
        if (40LL * k * cv > 3 * W) { mate[v] = -2; cand[v] = -1; continue; }
        const int pv = part[v];
        MlKey best;
        int bu = -1;
        const int j1 = __ldg(g.xadj + v + 1);
        for (int j = __ldg(g.xadj + v); j < j1; ++j) {
            const int u = __ldg(g.adjncy + j);
            if (mate[u] != -1 || part[u] != pv) continue;
            const long long cu = __ldg(g.vwgt + u);
            if (40LL * k * cu > 3 * W) continue;
            const unsigned long long wt = (unsigned long long)__ldg(g.adjwgt + j);
            MlKey key;
            key.a = min(u, v);
            key.b = max(u, v);
            key.w2 = wt * wt;
            key.cc = (unsigned long long)(cu > 0 ? cu : 1) * (unsigned long long)(cv > 0 ? cv : 1);
            key.h = splitmix64(seed_l ^ ((unsigned long long)(unsigned)key.a << 32) ^ (unsigned)key.b);
            if (bu < 0 || ml_higher(key, best)) { best = key; bu = u; }
        }
        if (bu < 0) { mate[v] = -2; cand[v] = -1; }   // no allowed edge to a free vertex, now or later
        else cand[v] = bu;
    }
}

__global__ void __launch_bounds__(kMlTPB) ml_pair_kernel(int n, int *mate, const int *cand, int *progress) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const int u = cand[v];
        if (u > v && cand[u] == v) {
            mate[v] = u;
            mate[u] = v;
            *progress = 1;
        }
    }
}

__global__ void __launch_bounds__(kMlTPB) ml_finish_kernel(int n, int *mate, int *pairs) {
    int c = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const int m = mate[v];
        if (m == -2) mate[v] = -1;
        else if (m > v) ++c;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(kMlFull, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(pairs, c);
}

// ---------------------------------------------------------------------- scan ----

// Exclusive scan of x over a block of 256 threads; *total = the block's sum.
__device__ int ml_block_scan(int x, int *s_warp, int *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int y = x;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(kMlFull, y, o);
        if (lane >= o) y += t;
    }
    if (lane == 31) s_warp[warp] = y;
    __syncthreads();
    if (warp == 0) {
        int z = lane < kMlTPB / 32 ? s_warp[lane] : 0;
        for (int o = 1; o < kMlTPB / 32; o <<= 1) {
            const int t = __shfl_up_sync(kMlFull, z, o);
            if (lane >= o) z += t;
        }
        if (lane < kMlTPB / 32) s_warp[lane] = z;
    }
    __syncthreads();
    const int base = warp ? s_warp[warp - 1] : 0;
    *total = s_warp[kMlTPB / 32 - 1];
    __syncthreads();
    return base + y - x;
}

__global__ void __launch_bounds__(kMlTPB) ml_scan_a(const int *in, int *out, int n, int *tmp) {
    __shared__ int s_warp[kMlTPB / 32];
    const long long base = (long long)blockIdx.x * 1024 + threadIdx.x * 4;
    int v[4], sum = 0;
    for (int i = 0; i < 4; ++i) {
        v[i] = base + i < n ? in[base + i] : 0;
        sum += v[i];
    }
    int total;
    int run = ml_block_scan(sum, s_warp, &total);
    for (int i = 0; i < 4; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
    if (threadIdx.x == 0) tmp[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kMlTPB) ml_scan_b(int *tmp, int nb) {
    __shared__ int s_warp[kMlTPB / 32];
    int carry = 0;
    for (int c = 0; c < nb; c += kMlTPB) {
        const int i = c + threadIdx.x;
        const int x = i < nb ? tmp[i] : 0;
        int total;
        const int ex = ml_block_scan(x, s_warp, &total);
        if (i < nb) tmp[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) tmp[nb] = carry;
}

__global__ void __launch_bounds__(kMlTPB) ml_scan_c(int *out, int n, const int *tmp) {
    const long long base = (long long)blockIdx.x * 1024;
    const int add = tmp[blockIdx.x];
    for (int t = threadIdx.x; t < 1024; t += blockDim.x)
        if (base + t < n) out[base + t] += add;
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = tmp[gridDim.x];
}

// --------------------------------------------------------------- contraction ----

__global__ void __launch_bounds__(kMlTPB) ml_reps_kernel(int n, const int *mate, int *isrep) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const int m = mate[v];
        isrep[v] = (m < 0 || v < m) ? 1 : 0;
    }
}

__global__ void __launch_bounds__(kMlTPB) ml_cmap_kernel(MlGraph g, const int *mate, const int *cid, int *cmap,
                                                         int *cvwgt, int *crep, int *rowcap) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < g.n; v += gridDim.x * blockDim.x) {
        const int m = mate[v];
        const int r = (m < 0 || v < m) ? v : m;
        const int x = cid[r];
        cmap[v] = x;
        if (r == v) {
            crep[x] = v;
            int c = __ldg(g.vwgt + v), cap = __ldg(g.xadj + v + 1) - __ldg(g.xadj + v);
            if (m >= 0) {
                c += __ldg(g.vwgt + m);
                cap += __ldg(g.xadj + m + 1) - __ldg(g.xadj + m);
            }
            cvwgt[x] = c;
            rowcap[x] = cap;
        }
    }
}

constexpr int kMlRowWarps = 4;

__global__ void __launch_bounds__(32 * kMlRowWarps) ml_rows_kernel(MlGraph g, int nc, const int *mate,
                                                                   const int *cmap, const int *crep,
                                                                   const int *rowcap, int count, int *cdeg,
                                                                   const int *cxadj, int *cadj, int *cwgt) {
    __shared__ int s_key[kMlRowWarps][kMlRowSmem];
    __shared__ int s_w[kMlRowWarps][kMlRowSmem];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int *K = s_key[wid], *Wt = s_w[wid];
    for (long long xl = (long long)blockIdx.x * kMlRowWarps + wid; xl < nc; xl += (long long)gridDim.x * kMlRowWarps) {
        const int x = (int)xl;
        const int r = crep[x], m = mate[r];
        const int mem[2] = {r, m};
        const int base = count ? 0 : cxadj[x];
        int outn = 0;
        if (rowcap[x] <= kMlRowSmem) {
            int L = 0;
            for (int t = 0; t < 2; ++t) {
                const int v = mem[t];
                if (v < 0) continue;
                const int j0 = __ldg(g.xadj + v), j1 = __ldg(g.xadj + v + 1);
                for (int jb = j0; jb < j1; jb += 32) {
                    const int j = jb + lane;
                    int y = -1, wv = 0;
                    if (j < j1) {
                        y = cmap[__ldg(g.adjncy + j)];
                        wv = __ldg(g.adjwgt + j);
                    }
                    const bool keep = j < j1 && y != x;
                    const unsigned km = __ballot_sync(kMlFull, keep);
                    if (keep) {
                        const int pos = L + __popc(km & ml_lanemask_lt());
                        K[pos] = y;
                        Wt[pos] = wv;
                    }
                    L += __popc(km);
                }
            }
            int P = 1;
            while (P < L) P <<= 1;
            for (int i = L + lane; i < P; i += 32) {
                K[i] = INT_MAX;
                Wt[i] = 0;
            }
            __syncwarp();
            for (int kk = 2; kk <= P; kk <<= 1)
                for (int jj = kk >> 1; jj > 0; jj >>= 1) {
                    for (int i = lane; i < P; i += 32) {
                        const int l = i ^ jj;
                        if (l > i) {
                            const int ki = K[i], kl = K[l];
                            if ((i & kk) == 0 ? kl < ki : ki < kl) {
                                K[i] = kl;
                                K[l] = ki;
                                const int t = Wt[i];
                                Wt[i] = Wt[l];
                                Wt[l] = t;
                            }
                        }
                    }
                    __syncwarp();
                }
            if (lane == 0) {
                int i = 0;
                while (i < L) {
                    const int y = K[i];
                    int s = 0;
                    while (i < L && K[i] == y) s += Wt[i++];
                    if (!count) {
                        cadj[base + outn] = y;
                        cwgt[base + outn] = s;
                    }
                    ++outn;
                }
            }
            __syncwarp();
        } else {
            // a row longer than the shared buffer: next larger coarse id, one at a time
            int last = -1;
            for (;;) {
                int mn = INT_MAX;
                for (int t = 0; t < 2; ++t) {
                    const int v = mem[t];
                    if (v < 0) continue;
                    const int j1 = __ldg(g.xadj + v + 1);
                    for (int j = __ldg(g.xadj + v) + lane; j < j1; j += 32) {
                        const int y = cmap[__ldg(g.adjncy + j)];
                        if (y != x && y > last && y < mn) mn = y;
                    }
                }
                for (int o = 16; o > 0; o >>= 1) mn = min(mn, __shfl_xor_sync(kMlFull, mn, o));
                if (mn == INT_MAX) break;
                int s = 0;
                for (int t = 0; t < 2; ++t) {
                    const int v = mem[t];
                    if (v < 0) continue;
                    const int j1 = __ldg(g.xadj + v + 1);
                    for (int j = __ldg(g.xadj + v) + lane; j < j1; j += 32)
                        if (cmap[__ldg(g.adjncy + j)] == mn) s += __ldg(g.adjwgt + j);
                }
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kMlFull, s, o);
                if (lane == 0 && !count) {
                    cadj[base + outn] = mn;
                    cwgt[base + outn] = s;
                }
                ++outn;
                last = mn;
            }
        }
        if (lane == 0 && count) cdeg[x] = outn;
        __syncwarp();
    }
}

// *bad = 1 unless mate is a matching: every entry -1 or a partner in range that points back.
__global__ void __launch_bounds__(kMlTPB) ml_check_kernel(int n, const int *mate, int *bad) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const int m = mate[v];
        if (m == -1) continue;
        if (m < 0 || m >= n || m == v || mate[m] != v) *bad = 1;
    }
}

__global__ void __launch_bounds__(kMlTPB) ml_down_kernel(int n, const int *cmap, const int *part, int *cpart) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) cpart[cmap[v]] = part[v];
}

__global__ void __launch_bounds__(kMlTPB) ml_up_kernel(int n, const int *cmap, const int *cpart, int *part) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) part[v] = cpart[cmap[v]];
}

// ------------------------------------------------------------------ launchers ----

static int ml_grid(long long n) {
    const long long b = (n + kMlTPB - 1) / kMlTPB;
    return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

cudaError_t launch_ml_point(const MlGraph &g, const int *part, int k, long long W, unsigned long long seed_l, int *mate,
                            int *cand, cudaStream_t st) {
    ml_point_kernel<<<ml_grid(g.n), kMlTPB, 0, st>>>(g, part, k, W, seed_l, mate, cand);
    return cudaGetLastError();
}

cudaError_t launch_ml_pair(int n, int *mate, const int *cand, int *progress, cudaStream_t st) {
    ml_pair_kernel<<<ml_grid(n), kMlTPB, 0, st>>>(n, mate, cand, progress);
    return cudaGetLastError();
}

cudaError_t launch_ml_finish(int n, int *mate, int *pairs, cudaStream_t st) {
    ml_finish_kernel<<<ml_grid(n), kMlTPB, 0, st>>>(n, mate, pairs);
    return cudaGetLastError();
}

cudaError_t launch_ml_scan(const int *in, int *out, int n, int *tmp, cudaStream_t st) {
    if (n <= 0) return cudaMemsetAsync(out, 0, sizeof(int), st);
    const int nb = (int)(((long long)n + 1023) / 1024);
    ml_scan_a<<<nb, kMlTPB, 0, st>>>(in, out, n, tmp);
    ml_scan_b<<<1, kMlTPB, 0, st>>>(tmp, nb);
    ml_scan_c<<<nb, kMlTPB, 0, st>>>(out, n, tmp);
    return cudaGetLastError();
}

cudaError_t launch_ml_reps(int n, const int *mate, int *isrep, cudaStream_t st) {
    ml_reps_kernel<<<ml_grid(n), kMlTPB, 0, st>>>(n, mate, isrep);
    return cudaGetLastError();
}

cudaError_t launch_ml_cmap(const MlGraph &g, const int *mate, const int *cid, int *cmap, int *cvwgt, int *crep,
                           int *rowcap, cudaStream_t st) {
    ml_cmap_kernel<<<ml_grid(g.n), kMlTPB, 0, st>>>(g, mate, cid, cmap, cvwgt, crep, rowcap);
    return cudaGetLastError();
}

cudaError_t launch_ml_rows(const MlGraph &g, int nc, const int *mate, const int *cmap, const int *crep,
                           const int *rowcap, bool count, int *cdeg, const int *cxadj, int *cadj, int *cwgt,
                           cudaStream_t st) {
    if (nc <= 0) return cudaSuccess;
    long long b = ((long long)nc + kMlRowWarps - 1) / kMlRowWarps;
    const int grid = (int)(b > 8192 ? 8192 : b);
    ml_rows_kernel<<<grid, 32 * kMlRowWarps, 0, st>>>(g, nc, mate, cmap, crep, rowcap, count ? 1 : 0, cdeg, cxadj,
                                                       cadj, cwgt);
    return cudaGetLastError();
}

cudaError_t launch_ml_check(int n, const int *mate, int *bad, cudaStream_t st) {
    ml_check_kernel<<<ml_grid(n), kMlTPB, 0, st>>>(n, mate, bad);
    return cudaGetLastError();
}

cudaError_t launch_ml_down(int n, const int *cmap, const int *part, int *cpart, cudaStream_t st) {
    ml_down_kernel<<<ml_grid(n), kMlTPB, 0, st>>>(n, cmap, part, cpart);
    return cudaGetLastError();
}

cudaError_t launch_ml_up(int n, const int *cmap, const int *cpart, int *part, cudaStream_t st) {
    ml_up_kernel<<<ml_grid(n), kMlTPB, 0, st>>>(n, cmap, cpart, part);
    return cudaGetLastError();
}

}  // namespace fr
