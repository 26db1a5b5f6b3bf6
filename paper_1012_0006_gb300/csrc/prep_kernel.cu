// Input checks, block weights and the quotient graph (Sanders & Schulz,
// Section 2.1), and the rounds of block pairs.
//
//   prep_kernel          one pass over the CSR: part in [0, k), c >= 0, omega >= 1,
//                        ids in range, no self loops, weighted degree < 2^30;
//                        c(V_i) per block, c(V), max c(v), total cut, quotient
//                        adjacency bits (i < j)
//   check_sym_kernel     opt-in: the CSR is symmetric with equal weights and simple
//   color_kernel         greedy edge colouring of the quotient graph in
//                        lexicographic (a, b) order, smallest free colour; each
//                        colour is a round of block-disjoint pairs
//   fill_pairs_kernel    pair descriptors of every round
#include <climits>

#include "fr_internal.cuh"
#include "round_kernel.cuh"

namespace fr {

constexpr int kPrepTPB = 256;
constexpr int kSmemQuotientK = 256;   // k up to this keeps the quotient bits in shared memory

__global__ void __launch_bounds__(kPrepTPB)
prep_kernel(const int *__restrict__ xadj, const int *__restrict__ adjncy, const int *__restrict__ adjwgt,
            const int *__restrict__ vwgt, const int *__restrict__ part, int n, int nnz, int k, long long *blockw,
            unsigned int *qbits, PrepOut *out, int *inb) {
    extern __shared__ unsigned int s_dyn[];
    // shared: block weights [k] (long long) when k <= 4096, quotient bits when k <= 256
    const bool smem_w = k <= 4096;
    const bool smem_q = qbits && k <= kSmemQuotientK;
    long long *s_w = reinterpret_cast<long long *>(s_dyn);
    unsigned int *s_q = reinterpret_cast<unsigned int *>(s_w + (smem_w ? k : 0));
    const int qwords = (k * k + 31) / 32;
    if (smem_w)
        for (int i = threadIdx.x; i < k; i += kPrepTPB) s_w[i] = 0;
    if (smem_q)
        for (int i = threadIdx.x; i < qwords; i += kPrepTPB) s_q[i] = 0;
    __syncthreads();
    int err = 0;
    long long W = 0, maxc = 0, cut = 0;
    int maxw = 0, maxwd = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0 && (xadj[0] != 0 || xadj[n] != nnz)) err = E_INVALID;
    for (long long v = (long long)blockIdx.x * kPrepTPB + threadIdx.x; v < n; v += (long long)gridDim.x * kPrepTPB) {
        const int pv = part[v];
        const int c = vwgt[v];
        if (pv < 0 || pv >= k || c < 0) {
            err = E_INVALID;
            continue;
        }
        W += c;
        if (c > maxc) maxc = c;
        if (smem_w) atomicAdd((unsigned long long *)&s_w[pv], (unsigned long long)c);
        else atomicAdd((unsigned long long *)&blockw[pv], (unsigned long long)c);
        const int r0 = xadj[v], r1 = xadj[v + 1];
        if (r0 > r1 || r1 > nnz || r0 < 0) {
            err = E_INVALID;
            continue;
        }
        long long wdeg = 0;
        bool bnd = false;
        for (int j = r0; j < r1; ++j) {
            const int u = adjncy[j];
            const int om = adjwgt[j];
            if (u < 0 || u >= n || u == v || om < 1) {
                err = E_INVALID;
                break;
            }
            wdeg += om;
            if (om > maxw) maxw = om;
            const int pu = part[u];
            bnd |= pu != pv;
            if (pu > pv && pu < k) {
                cut += om;
                const int bit = pv * k + pu;
                if (smem_q) atomicOr(&s_q[bit >> 5], 1u << (bit & 31));
                else if (qbits && !(qbits[bit >> 5] & (1u << (bit & 31)))) atomicOr(&qbits[bit >> 5], 1u << (bit & 31));
            }
        }
        if (wdeg >= (1LL << 30) && err == 0) err = E_TOO_LARGE;
        else if (wdeg > maxwd) maxwd = (int)wdeg;
        if (inb) inb[v] = bnd ? 1 : 0;
    }
    __syncthreads();
    if (smem_w)
        for (int i = threadIdx.x; i < k; i += kPrepTPB)
            if (s_w[i]) atomicAdd((unsigned long long *)&blockw[i], (unsigned long long)s_w[i]);
    if (smem_q)
        for (int i = threadIdx.x; i < qwords; i += kPrepTPB)
            if (s_q[i]) atomicOr(&qbits[i], s_q[i]);
    const long long bW = block_sum_ll<kPrepTPB>(W);
    const long long bC = block_sum_ll<kPrepTPB>(cut);
    __shared__ long long s_max;
    __shared__ int s_err, s_maxw, s_maxwd;
    if (threadIdx.x == 0) { s_max = 0; s_err = 0; s_maxw = 0; s_maxwd = 0; }
    __syncthreads();
    if (maxc) atomicMax((unsigned long long *)&s_max, (unsigned long long)maxc);
    if (maxw) atomicMax(&s_maxw, maxw);
    if (maxwd) atomicMax(&s_maxwd, maxwd);
    if (err) atomicMax(&s_err, err);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (bW) atomicAdd((unsigned long long *)&out->W, (unsigned long long)bW);
        if (bC) atomicAdd((unsigned long long *)&out->totcut, (unsigned long long)bC);
        if (s_max) atomicMax((unsigned long long *)&out->maxc, (unsigned long long)s_max);
        if (s_maxw) atomicMax(&out->maxw, s_maxw);
        if (s_maxwd) atomicMax(&out->maxwdeg, s_maxwd);
        if (s_err) atomicMax(&out->err, s_err);
    }
}

__global__ void __launch_bounds__(kPrepTPB)
check_sym_kernel(const int *__restrict__ xadj, const int *__restrict__ adjncy, const int *__restrict__ adjwgt,
                 int n, PrepOut *out) {
    int err = 0;
    for (long long v = (long long)blockIdx.x * kPrepTPB + threadIdx.x; v < n; v += (long long)gridDim.x * kPrepTPB) {
        const int r0 = xadj[v], r1 = xadj[v + 1];
        for (int j = r0; j < r1 && !err; ++j) {
            const int u = adjncy[j];
            for (int q = r0; q < j; ++q)
                if (adjncy[q] == u) err = E_INVALID;            // parallel edge
            int found = 0;
            for (int q = xadj[u]; q < xadj[u + 1]; ++q)
                if (adjncy[q] == (int)v) { found = adjwgt[q] == adjwgt[j] ? 1 : -1; break; }
            if (found != 1) err = E_INVALID;                    // missing or unequal reverse
        }
    }
    if (err) atomicMax(&out->err, err);
}

// Greedy edge colouring, one thread (k is small: the quotient graph has k vertices).
__global__ void color_kernel(const unsigned int *qbits, int k, int *pair_a, int *pair_b, int *pair_round,
                             int *round_off, int *sob_round, unsigned int *used, PrepOut *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int ncol = 2 * k;
    const int cw = (ncol + 31) / 32;
    for (long long i = 0; i < (long long)k * cw; ++i) used[i] = 0;
    int np = 0, nr = 0;
    for (int a = 0; a < k; ++a)
        for (int b = a + 1; b < k; ++b) {
            const int bit = a * k + b;
            if (!(qbits[bit >> 5] & (1u << (bit & 31)))) continue;
            int c = 0;
            for (int wi = 0; wi < cw; ++wi) {
                const unsigned int freebits = ~(used[(long long)a * cw + wi] | used[(long long)b * cw + wi]);
                if (freebits) { c = wi * 32 + __ffs(freebits) - 1; break; }
            }
            used[(long long)a * cw + (c >> 5)] |= 1u << (c & 31);
            used[(long long)b * cw + (c >> 5)] |= 1u << (c & 31);
            pair_round[np] = c;
            pair_a[np] = a;
            pair_b[np] = b;
            ++np;
            if (c + 1 > nr) nr = c + 1;
        }
    // stable counting sort by round: (round, a, b) order
    for (int r = 0; r <= nr; ++r) round_off[r] = 0;
    for (int i = 0; i < np; ++i) round_off[pair_round[i] + 1]++;
    for (int r = 0; r < nr; ++r) round_off[r + 1] += round_off[r];
    // sort through the tail of pair_round's storage is not possible in place; use sob_round as scratch
    int *tmp = sob_round;   // needs 2*np ints; sob_round has nr*k >= 2*np entries
    int *cur = pair_round;  // reuse: after reading rounds into tmp order
    for (int i = 0; i < np; ++i) {
        tmp[2 * i] = pair_a[i] * k + pair_b[i];
        tmp[2 * i + 1] = pair_round[i];
    }
    for (int r = 0; r < nr; ++r) cur[r] = round_off[r];
    for (int i = 0; i < np; ++i) {
        const int r = tmp[2 * i + 1];
        const int pos = cur[r]++;
        // pair_a / pair_b are overwritten after all reads of tmp: store packed for now
        tmp[2 * i + 1] = pos;
    }
    for (int i = 0; i < np; ++i) {
        const int pos = tmp[2 * i + 1];
        pair_a[pos] = tmp[2 * i] / k;
        pair_b[pos] = tmp[2 * i] % k;
    }
    for (int r = 0; r < nr; ++r)
        for (int pos = round_off[r]; pos < round_off[r + 1]; ++pos) pair_round[pos] = r;
    for (long long i = 0; i < (long long)nr * k; ++i) sob_round[i] = -1;
    for (int r = 0; r < nr; ++r)
        for (int pos = round_off[r]; pos < round_off[r + 1]; ++pos) {
            const int lp = pos - round_off[r];
            sob_round[(long long)r * k + pair_a[pos]] = 2 * lp;
            sob_round[(long long)r * k + pair_b[pos]] = 2 * lp + 1;
        }
    out->npairs = np;
    out->nrounds = nr;
}

__global__ void fill_pairs_kernel(PairDev *pairs, const int *pair_a, const int *pair_b, int np, int g, int mb,
                                  long long Ubase) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
        PairDev p;
        p.g = g;
        p.a = pair_a[i];
        p.b = pair_b[i];
        p.mb = mb;
        p.Ubase = Ubase;
        pairs[i] = p;
    }
}

static int grid_for(long long n, int tpb) {
    int dev = 0, nsm = 132;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    long long b = (n + tpb - 1) / tpb;
    long long cap = (long long)nsm * 8;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

// The marked vertices in increasing order per warp of 32 (one atomic per warp).
__global__ void __launch_bounds__(kPrepTPB) compact_kernel(const int *inb, int n, int *bl, int *blc) {
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * (kPrepTPB / 32);
    for (long long b = ((long long)blockIdx.x * (kPrepTPB / 32) + (threadIdx.x >> 5)) * 32; b < n; b += nw * 32) {
        const long long v = b + lane;
        const bool f = v < n && inb[v];
        const unsigned m = __ballot_sync(0xffffffffu, f);
        if (!m) continue;
        int base = 0;
        if (lane == 0) base = atomicAdd(blc, __popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (f) bl[base + __popc(m & ((1u << lane) - 1u))] = (int)v;
    }
}

cudaError_t launch_prep(const int *xadj, const int *adjncy, const int *adjwgt, const int *vwgt, const int *part,
                        int n, int nnz, int k, long long *blockw, unsigned int *qbits, PrepOut *out,
                        cudaStream_t st, int *bl, int *blc, int *inb) {
    size_t sm = 0;
    if (k <= 4096) sm += sizeof(long long) * k;
    if (qbits && k <= kSmemQuotientK) sm += sizeof(unsigned int) * ((k * k + 31) / 32);
    prep_kernel<<<grid_for(n, kPrepTPB), kPrepTPB, sm, st>>>(xadj, adjncy, adjwgt, vwgt, part, n, nnz, k, blockw,
                                                            qbits, out, bl ? inb : nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !bl) return e;
    e = cudaMemsetAsync(blc, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    compact_kernel<<<grid_for(n, kPrepTPB), kPrepTPB, 0, st>>>(inb, n, bl, blc);
    return cudaGetLastError();
}

cudaError_t launch_check_symmetric(const int *xadj, const int *adjncy, const int *adjwgt, int n, PrepOut *out,
                                   cudaStream_t st) {
    check_sym_kernel<<<grid_for(n, kPrepTPB), kPrepTPB, 0, st>>>(xadj, adjncy, adjwgt, n, out);
    return cudaGetLastError();
}

// The same colouring for k <= kColorSmallK in one CTA's shared memory: each row of the
// quotient bitmap lists its edges (a, b > a) in parallel and a scan over the rows gives
// the lexicographic edge list; one thread colours the edges in that order (the greedy
// rule is sequential) and sorts them by round, stably; the threads write the outputs.
// Identical results to color_kernel.
constexpr int kColorSmallK = 90;
constexpr int kColorMaxEdges = kColorSmallK * (kColorSmallK - 1) / 2;
constexpr int kColorWords = (2 * kColorSmallK + 31) / 32;

__global__ void __launch_bounds__(256) color_small_kernel(const unsigned int *qbits, int k, int *pair_a, int *pair_b,
                                                         int *pair_round, int *round_off, int *sob_round,
                                                         PrepOut *out) {
    __shared__ int s_edge[kColorMaxEdges];   // a << 16 | b, lexicographic; then in round order
    __shared__ short s_col[kColorMaxEdges];
    __shared__ unsigned s_used[kColorSmallK * kColorWords];
    __shared__ int s_rowc[kColorSmallK + 1];
    __shared__ int s_off[2 * kColorSmallK + 2];
    __shared__ int s_np, s_nr;
    const int t = threadIdx.x;
    const int cw = (2 * k + 31) / 32;
    for (int i = t; i < k * cw; i += blockDim.x) s_used[i] = 0;
    // row a: its edges (a, b), b > a
    for (int a2 = t; a2 < k; a2 += blockDim.x) {
        int c = 0;
        for (int b2 = a2 + 1; b2 < k; ++b2) {
            const int bit = a2 * k + b2;
            c += (qbits[bit >> 5] >> (bit & 31)) & 1u;
        }
        s_rowc[a2] = c;
    }
    __syncthreads();
    if (t == 0) {
        int o = 0;
        for (int a2 = 0; a2 < k; ++a2) {
            const int c = s_rowc[a2];
            s_rowc[a2] = o;
            o += c;
        }
        s_rowc[k] = o;
        s_np = o;
    }
    __syncthreads();
    for (int a2 = t; a2 < k; a2 += blockDim.x) {
        int o = s_rowc[a2];
        for (int b2 = a2 + 1; b2 < k; ++b2) {
            const int bit = a2 * k + b2;
            if ((qbits[bit >> 5] >> (bit & 31)) & 1u) s_edge[o++] = (a2 << 16) | b2;
        }
    }
    __syncthreads();
    const int np = s_np;
    if (t == 0) {
        // greedy: the smallest colour free at both ends
        int nr = 0;
        for (int e = 0; e < np; ++e) {
            const int a2 = s_edge[e] >> 16, b2 = s_edge[e] & 0xFFFF;
            int c = 0;
            for (int wi = 0; wi < cw; ++wi) {
                const unsigned freebits = ~(s_used[a2 * cw + wi] | s_used[b2 * cw + wi]);
                if (freebits) { c = wi * 32 + __ffs(freebits) - 1; break; }
            }
            s_used[a2 * cw + (c >> 5)] |= 1u << (c & 31);
            s_used[b2 * cw + (c >> 5)] |= 1u << (c & 31);
            s_col[e] = (short)c;
            if (c + 1 > nr) nr = c + 1;
        }
        s_nr = nr;
        // round offsets (stable counting sort by round keeps the lexicographic order)
        for (int r = 0; r <= nr; ++r) s_off[r] = 0;
        for (int e = 0; e < np; ++e) s_off[s_col[e] + 1]++;
        for (int r = 0; r < nr; ++r) s_off[r + 1] += s_off[r];
    }
    __syncthreads();
    const int nr = s_nr;
    for (int r = t; r <= nr; r += blockDim.x) round_off[r] = s_off[r];
    for (long long i = t; i < (long long)nr * k; i += blockDim.x) sob_round[i] = -1;
    __syncthreads();
    // positions: round offset + rank among the earlier edges of the same round, one
    // thread per edge (np <= 4005: a quadratic count is cheap here)
    for (int e = t; e < np; e += blockDim.x) {
        const int c = s_col[e];
        int rk = 0;
        for (int q = 0; q < e; ++q) rk += s_col[q] == c;
        const int pos = s_off[c] + rk;
        const int a2 = s_edge[e] >> 16, b2 = s_edge[e] & 0xFFFF;
        pair_a[pos] = a2;
        pair_b[pos] = b2;
        pair_round[pos] = c;
        sob_round[(long long)c * k + a2] = 2 * rk;
        sob_round[(long long)c * k + b2] = 2 * rk + 1;
    }
    if (t == 0) {
        out->npairs = np;
        out->nrounds = nr;
    }
}

cudaError_t launch_color(const unsigned int *qbits, int k, int *pair_a, int *pair_b, int *pair_round,
                         int *round_off, int *sob_round, unsigned int *used, PrepOut *out, cudaStream_t st) {
    if (k <= kColorSmallK)
        color_small_kernel<<<1, 256, 0, st>>>(qbits, k, pair_a, pair_b, pair_round, round_off, sob_round, out);
    else
        color_kernel<<<1, 32, 0, st>>>(qbits, k, pair_a, pair_b, pair_round, round_off, sob_round, used, out);
    return cudaGetLastError();
}

cudaError_t launch_fill_pairs(PairDev *pairs, const int *pair_a, const int *pair_b, int np, int g, int mb,
                              long long Ubase, cudaStream_t st) {
    fill_pairs_kernel<<<grid_for(np, 128), 128, 0, st>>>(pairs, pair_a, pair_b, np, g, mb, Ubase);
    return cudaGetLastError();
}

}  // namespace fr

namespace fr {

__global__ void gather_kernel(int *dst, const int *src, const int *idx, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = src[idx[i]];
}

cudaError_t launch_gather(int *dst, const int *src, const int *idx, int n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    gather_kernel<<<grid_for(n, 256), 256, 0, st>>>(dst, src, idx, n);
    return cudaGetLastError();
}

}  // namespace fr
