// fr_refine_pair_noalloc: the single-pair refinement of fr_refine_pair for
// callers that cannot allocate device memory (see include/flowref.h).  All
// scratch lives in one file-scope __device__ array; this file never calls
// cudaMalloc, cudaFree, cudaHostAlloc or any allocating library routine.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "api_internal.h"

using namespace fr;

namespace {

constexpr int kNaMaxN = FR_NOALLOC_MAX_N;
constexpr int kNaMaxNNZ = FR_NOALLOC_MAX_NNZ;
constexpr int kNaMaxK = FR_NOALLOC_MAX_K;
constexpr int kNaMaxReps = FR_NOALLOC_MAX_REPS;
constexpr int kNaMaxGrid = 4096;

constexpr size_t al(size_t b) { return (b + 255) / 256 * 256; }

// Bytes of every carved array, in carving order (must match carve_all below).
constexpr size_t kNaBytes =
    5 * al(4ull * kNaMaxN) +                                  // dist lid vq_v vq_s part0
    al(4ull * (kNaMaxN / 32 + 2)) +                           // cbits
    21 * al(4ull * (kNaMaxN + 1)) +                           // union vertex arrays
    2 * al(8ull * kNaMaxN) + 2 * al(1ull * kNaMaxN) +         // ex cw / border side_out
    5 * al(4ull * kNaMaxNNZ) +                                // head rev res cap outs
    3 * al(4ull * kNaMaxReps * kNaMaxN) + al(8ull * kNaMaxReps * kNaMaxN) +   // sweeps
    al(4ull * (kNaMaxGrid + 1)) +                             // cta_cnt
    al(8ull * kNaMaxK) + al(4ull * kNaMaxK) +                 // blockw sob
    al(sizeof(PrepOut)) + al(sizeof(GraphDev)) + al(sizeof(PairDev)) + al(2 * sizeof(SideDev)) +
    al(sizeof(PairAcc)) + al(sizeof(Ctl)) + al(8ull * 3 * 2 * kHistBins) + al(4) +
    al(8ull * kNaMaxReps) + al(4ull * kNaMaxReps);

// The scratch.  A GPU that loads the library holds it until the process exits.
__device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

struct Scratch {
    int *dist, *lid, *vq_v, *vq_s;
    int *part0;   // part as the call found it (restored on error)
    unsigned int *cbits;
    int *gid, *sid, *off, *infc, *fx, *lab, *rflag, *color, *scc, *vc, *fq0, *fq1, *spare;
    int *cpair, *cmin, *cid, *indeg, *outoff, *ocur, *plist, *sinkc;
    long long *ex, *cw;
    unsigned char *border, *side_out;
    int *head, *rev, *res, *cap, *outs;
    int *indeg_r, *order, *hcomp;
    unsigned long long *hkey;
    int *cta_cnt;
    long long *blockw;
    int *sob;
    PrepOut *prep;
    GraphDev *graph;
    PairDev *pair;
    SideDev *sides;
    PairAcc *pacc;
    Ctl *ctl;
    long long *hist;
    int *pcur;
    long long *sw_absd;
    int *sw_j;
};

template <class T>
T *take(char *&p, size_t count) {
    T *r = reinterpret_cast<T *>(p);
    p += al(sizeof(T) * count);
    return r;
}

void carve_all(char *p, Scratch &s) {
    const size_t N = kNaMaxN, N1 = kNaMaxN + 1, M = kNaMaxNNZ, R = kNaMaxReps;
    s.dist = take<int>(p, N); s.lid = take<int>(p, N); s.vq_v = take<int>(p, N); s.vq_s = take<int>(p, N);
    s.part0 = take<int>(p, N);
    s.cbits = take<unsigned int>(p, N / 32 + 2);
    int **v21[21] = {&s.gid, &s.sid, &s.off, &s.infc, &s.fx, &s.lab, &s.rflag, &s.color, &s.scc, &s.vc, &s.fq0,
                     &s.fq1, &s.spare, &s.cpair, &s.cmin, &s.cid, &s.indeg, &s.outoff, &s.ocur, &s.plist, &s.sinkc};
    for (auto a : v21) *a = take<int>(p, N1);
    s.ex = take<long long>(p, N); s.cw = take<long long>(p, N);
    s.border = take<unsigned char>(p, N); s.side_out = take<unsigned char>(p, N);
    s.head = take<int>(p, M); s.rev = take<int>(p, M); s.res = take<int>(p, M); s.cap = take<int>(p, M);
    s.outs = take<int>(p, M);
    s.indeg_r = take<int>(p, R * N); s.order = take<int>(p, R * N); s.hcomp = take<int>(p, R * N);
    s.hkey = take<unsigned long long>(p, R * N);
    s.cta_cnt = take<int>(p, kNaMaxGrid + 1);
    s.blockw = take<long long>(p, kNaMaxK);
    s.sob = take<int>(p, kNaMaxK);
    s.prep = take<PrepOut>(p, 1);
    s.graph = take<GraphDev>(p, 1);
    s.pair = take<PairDev>(p, 1);
    s.sides = take<SideDev>(p, 2);
    s.pacc = take<PairAcc>(p, 1);
    s.ctl = take<Ctl>(p, 1);
    s.hist = take<long long>(p, 3 * 2 * kHistBins);
    s.pcur = take<int>(p, 1);
    s.sw_absd = take<long long>(p, R);
    s.sw_j = take<int>(p, R);
}

// Device address of the scratch on the current device.  It is looked up on every call
// (a host-side table lookup): an address kept from an earlier call could belong to a
// context that no longer exists (after cudaDeviceReset the module is loaded again and
// the array may sit elsewhere).
cudaError_t scratch_address(void **out) {
    void *ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = ptr;
    return cudaSuccess;
}

struct NaIter {
    long long flow, oldcut, newcut, cA, cB, nA, nB;
    int nc, m, accept, feasible, ncomp;
    Ctl ctl;
};

}  // namespace

#define NA_CK(call)                                   \
    do {                                              \
        if ((call) != cudaSuccess) return FR_ERR_CUDA; \
    } while (0)

static fr_status na_iteration(const Scratch &S, const fr_graph *g, int32_t *part, int32_t k, int32_t a, int32_t b,
                              long long Ubase, long long Lmax, const fr_options &opt, cudaStream_t st, NaIter *o) {
    GraphDev gd;
    memset(&gd, 0, sizeof(gd));
    gd.xadj = g->xadj; gd.adjncy = g->adjncy; gd.adjwgt = g->adjwgt; gd.vwgt = g->vwgt;
    gd.part = part; gd.dist = S.dist; gd.lid = S.lid; gd.sob = S.sob; gd.blockw = S.blockw;
    gd.n = g->n; gd.nnz = g->nnz; gd.k = k; gd.base = 0; gd.Lmax = Lmax;
    PairDev pd;
    pd.g = 0; pd.a = a; pd.b = b; pd.mb = opt.mb ? 1 : 0; pd.Ubase = Ubase;
    const int sides01[2] = {0, 1};
    // scratch keeps the previous call's contents: everything a step expects cleared is cleared here
    NA_CK(cudaMemcpyAsync(S.graph, &gd, sizeof(gd), cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemcpyAsync(S.pair, &pd, sizeof(pd), cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemsetAsync(S.sob, 0xFF, sizeof(int) * k, st));
    NA_CK(cudaMemcpyAsync(S.sob + a, &sides01[0], sizeof(int), cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemcpyAsync(S.sob + b, &sides01[1], sizeof(int), cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemsetAsync(S.ctl, 0, sizeof(Ctl), st));
    NA_CK(cudaMemsetAsync(S.sides, 0, 2 * sizeof(SideDev), st));
    NA_CK(cudaMemsetAsync(S.pacc, 0, sizeof(PairAcc), st));
    NA_CK(cudaMemsetAsync(S.hist, 0, sizeof(long long) * 3 * 2 * kHistBins, st));
    NA_CK(cudaStreamSynchronize(st));   // the host sources above live on this stack frame
    Work w;
    memset(&w, 0, sizeof(w));
    w.graphs = S.graph; w.pairs = S.pair; w.sides = S.sides; w.pacc = S.pacc; w.ctl = S.ctl;
    w.prev_err = nullptr;
    w.ngraphs = 1; w.npairs = 1; w.nsides = 2; w.total_n = g->n;
    w.vq_v = S.vq_v; w.vq_s = S.vq_s; w.vq_cap = kNaMaxN; w.cbits = S.cbits;
    w.gid = S.gid; w.sid = S.sid; w.off = S.off; w.head = S.head; w.rev = S.rev; w.res = S.res; w.cap = S.cap;
    w.infc = S.infc; w.fx = S.fx; w.lab = S.lab; w.rflag = S.rflag; w.color = S.color; w.scc = S.scc;
    w.vc = S.vc; w.ex = S.ex; w.border = S.border; w.side_out = S.side_out;
    w.nu_cap = kNaMaxN; w.mu_cap = kNaMaxNNZ;
    w.fq0 = S.fq0; w.fq1 = S.fq1; w.cta_cnt = S.cta_cnt; w.hist = S.hist;
    w.cw = S.cw; w.cpair = S.cpair; w.cmin = S.cmin; w.cid = S.cid; w.indeg = S.indeg; w.outoff = S.outoff;
    w.outs = S.outs; w.ocur = S.ocur; w.plist = S.plist; w.pcur = S.pcur; w.indeg_r = S.indeg_r;
    w.order = S.order; w.sinkc = S.sinkc; w.hkey = S.hkey; w.hcomp = S.hcomp;
    w.sw_absd = S.sw_absd; w.sw_j = S.sw_j;
    w.reps = opt.mb_reps > 0 ? opt.mb_reps : 1;
    w.gr_interval = opt.gr_interval > 0 ? opt.gr_interval : 16;
    w.inner = opt.inner_ops > 0 ? opt.inner_ops : 2;
    w.passes = opt.pulse_passes > 0 ? opt.pulse_passes : 2;
    w.any_mb = opt.mb ? 1 : 0;
    w.seed = opt.seed;
    w.pulse_cap = opt.pulse_cap > 0 ? opt.pulse_cap : (1LL << 20);
    w.gap_interval = gap_interval_of(&opt);
    const int tpb = opt.block_threads == 256 ? 256 : 512;
    int maxb = 1, sms = 1;
    if (step_max_grid(tpb, 2, &maxb, &sms) != cudaSuccess) return FR_ERR_CUDA;
    long long want = opt.grid_blocks > 0 ? opt.grid_blocks : (2 * Ubase + 2LL * tpb - 1) / (2LL * tpb);
    want = std::max(1LL, std::min<long long>(want, std::min(sms, kNaMaxGrid)));
    const int grid = (int)std::min<long long>(want, maxb);
    NA_CK(launch_scan(w, 0, g->n, (reinterpret_cast<uintptr_t>(g->adjncy) & 15) == 0, st));
    NA_CK(launch_step(w, PH_ALL, grid, tpb, st));
    PairAcc A;
    SideDev Sd[2];
    NA_CK(cudaMemcpyAsync(&A, S.pacc, sizeof(A), cudaMemcpyDeviceToHost, st));
    NA_CK(cudaMemcpyAsync(Sd, S.sides, sizeof(Sd), cudaMemcpyDeviceToHost, st));
    NA_CK(cudaMemcpyAsync(&o->ctl, S.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
    if (o->ctl.error) {
        switch (o->ctl.error) {
            case E_INVALID: return FR_ERR_INVALID_ARG;
            case E_ITER: return FR_ERR_ITER_LIMIT;
            case E_TOO_LARGE: return FR_ERR_TOO_LARGE;
            case E_ABORT: return FR_ERR_ABORTED;
            default: return FR_ERR_INTERNAL;
        }
    }
    o->flow = A.flow;
    o->oldcut = A.oldcut;
    o->newcut = A.oldcut + A.dcut;
    o->cA = Sd[0].cw; o->cB = Sd[1].cw;
    o->nA = Sd[0].cw + A.dwA; o->nB = Sd[1].cw - A.dwA;
    o->nc = A.nc; o->m = A.m; o->accept = A.accept; o->feasible = A.feasible; o->ncomp = A.ncomp;
    return FR_OK;
}

extern "C" fr_status fr_refine_pair_noalloc(const fr_graph *g, int32_t *part, int32_t k, int32_t a, int32_t b,
                                            double eps, double alpha, const fr_options *opt_in,
                                            fr_pair_result *res, void *stream) {
    fr_options opt;
    if (opt_in) opt = *opt_in; else fr_default_options(&opt);
    if (res) memset(res, 0, sizeof(*res));
    // the same checks as fr_refine_pair's (no context, so no message), plus no FM or
    // multi-try step: those need the context's workspace
    const char *why = nullptr;
    fr_status st = validate_params(eps, alpha, &opt, &why);
    if (st == FR_OK &&
        (!g || !part || g->n < 1 || g->nnz < 0 || !g->xadj || !g->vwgt || (g->nnz > 0 && (!g->adjncy || !g->adjwgt)) ||
         k < 2 || k > kMaxK || a < 0 || b < 0 || a >= k || b >= k || a == b || opt.fm_permille != 0 ||
         opt.mt_alpha != 0))
        st = FR_ERR_INVALID_ARG;
    else if (g->n > kNaMaxN || g->nnz > kNaMaxNNZ || k > kNaMaxK || opt.mb_reps > kNaMaxReps)
        st = FR_ERR_TOO_LARGE;   // beyond the fixed scratch: use fr_refine_pair
    if (st != FR_OK) {
        if (res) res->status = st;
        return st;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    void *base = nullptr;
    if (scratch_address(&base) != cudaSuccess) {
        cudaGetLastError();
        if (res) res->status = FR_ERR_CUDA;
        return FR_ERR_CUDA;
    }
    Scratch S;
    carve_all(reinterpret_cast<char *>(base), S);
    // idle state of the BFS marks, then validation and weights
    PrepOut po;
    memset(&po, 0, sizeof(po));
    if (cudaMemsetAsync(S.dist, 0xFF, sizeof(int) * g->n, s) != cudaSuccess ||
        cudaMemsetAsync(S.lid, 0xFF, sizeof(int) * g->n, s) != cudaSuccess ||
        cudaMemsetAsync(S.cbits, 0, sizeof(unsigned int) * (g->n / 32 + 2), s) != cudaSuccess ||
        cudaMemsetAsync(S.prep, 0, sizeof(PrepOut), s) != cudaSuccess ||
        cudaMemsetAsync(S.blockw, 0, sizeof(long long) * k, s) != cudaSuccess ||
        cudaMemcpyAsync(S.part0, part, sizeof(int) * g->n, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        launch_prep(g->xadj, g->adjncy, g->adjwgt, g->vwgt, part, g->n, g->nnz, k, S.blockw, nullptr, S.prep, s) !=
            cudaSuccess ||
        (opt.checked && launch_check_symmetric(g->xadj, g->adjncy, g->adjwgt, g->n, S.prep, s) != cudaSuccess) ||
        cudaMemcpyAsync(&po, S.prep, sizeof(PrepOut), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        if (res) res->status = FR_ERR_CUDA;
        return FR_ERR_CUDA;
    }
    if (po.err) {
        st = po.err == E_TOO_LARGE ? FR_ERR_TOO_LARGE : FR_ERR_INVALID_ARG;
        if (res) res->status = st;
        return st;
    }
    const long long W = po.W, Lmax = host_lmax(W, po.maxc, k, eps);
    const int adaptive = opt.adaptive ? 1 : 0;
    const int max_iters = adaptive ? (opt.max_iters > 0 ? opt.max_iters : 10) : 1;
    const double alpha_max = adaptive ? opt.alpha_max : alpha;
    double al = alpha;
    int iters = 0, accepted = 0;
    NaIter o;
    memset(&o, 0, sizeof(o));
    long long cut0 = -1, wA0 = 0, wB0 = 0, cut = 0, wA = 0, wB = 0;
    Ctl last;   // counters of the last iteration that succeeded
    memset(&last, 0, sizeof(last));
    int ncomp = 0;
    while (iters < max_iters) {
        ++iters;
        st = na_iteration(S, g, part, k, a, b, host_budget_base(W, k, eps, al), Lmax, opt, s, &o);
        if (st != FR_OK) {
            // a failed step may stop before releasing its BFS marks; the next call clears them
            break;
        }
        last = o.ctl;
        ncomp = o.ncomp;
        if (cut0 < 0) { cut0 = o.oldcut; wA0 = o.cA; wB0 = o.cB; }
        cut = o.oldcut; wA = o.cA; wB = o.cB;
        if (o.accept) { cut = o.newcut; wA = o.nA; wB = o.nB; accepted = 1; }
        if (o.feasible && o.newcut < o.oldcut) {
            if (!adaptive) break;
            al = 2.0 * al < alpha_max ? 2.0 * al : alpha_max;
            continue;
        }
        if (o.feasible) break;
        if (!adaptive || al == 1.0) break;
        al = al / 2.0 > 1.0 ? al / 2.0 : 1.0;
    }
    if (st != FR_OK) {
        // an earlier iteration may have been applied before a later one failed: put part back
        if (cudaMemcpyAsync(part, S.part0, sizeof(int) * g->n, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            cudaGetLastError();
            st = FR_ERR_CUDA;
        }
        accepted = 0;
        cut = cut0 < 0 ? 0 : cut0; wA = wA0; wB = wB0;
    }
    if (res) {
        res->status = st;
        res->a = a; res->b = b;
        res->iters = iters;
        res->alpha_final = al;
        res->flow = o.flow;
        res->cut_before = cut0 < 0 ? 0 : cut0;
        res->wA_before = wA0; res->wB_before = wB0;
        res->cut_after = cut; res->wA_after = wA; res->wB_after = wB;
        res->corridor_n = o.nc; res->corridor_arcs = o.m;
        res->accepted = accepted;
        res->pulses = last.pulses; res->relabels = last.relabels;
        res->bfs_levels = last.levels; res->scc_rounds = last.scc_rounds; res->ncomp = ncomp;
    }
    return st;
}
