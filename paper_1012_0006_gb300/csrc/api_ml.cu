// C ABI, part 5: the multilevel V-cycle with a given partition (Sanders & Schulz,
// Section 2.1 matching and contraction, Section 2.2 the expansion*2 rating and the
// weight bound on contracted nodes, Section 5 the given partition kept through the
// hierarchy): fr_match, fr_contract and fr_vcycle.  The refinement of every level is the
// batched flow sweep (fr_refine_batch) or active block scheduling (fr_refine_active).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <vector>

#include "api_internal.h"
#include "ml_kernel.cuh"

using namespace fr;

#define CK(call)                                                 \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

namespace {

// Device allocations of one call, freed together.
struct DevPool {
    std::vector<void *> ptrs;
    ~DevPool() {
        for (void *p : ptrs) cudaFree(p);
    }
    template <typename T>
    T *get(long long count) {
        void *p = nullptr;
        if (cudaMalloc(&p, sizeof(T) * (size_t)std::max(1LL, count)) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        ptrs.push_back(p);
        return reinterpret_cast<T *>(p);
    }
};

// Scratch of the matching and contraction kernels for graphs up to n vertices.
struct MlScratch {
    int *cand, *isrep, *cid, *crep, *rowcap, *cdeg, *tmp, *flags;
    bool make(DevPool &pool, int n) {
        cand = pool.get<int>(n);
        isrep = pool.get<int>(n);
        cid = pool.get<int>((long long)n + 1);
        crep = pool.get<int>(n);
        rowcap = pool.get<int>(n);
        cdeg = pool.get<int>(n);
        tmp = pool.get<int>(((long long)n + 1023) / 1024 + 2);
        flags = pool.get<int>(2);
        return cand && isrep && cid && crep && rowcap && cdeg && tmp && flags;
    }
};

MlGraph ml_view(const fr_graph *g) {
    MlGraph m;
    m.xadj = g->xadj; m.adjncy = g->adjncy; m.adjwgt = g->adjwgt; m.vwgt = g->vwgt;
    m.n = g->n; m.nnz = g->nnz;
    return m;
}

// Locally dominant rounds until no pair forms; *pairs = matched pairs.
fr_status match_level(fr_ctx *ctx, const fr_graph *g, const int32_t *part, int k, long long W,
                      unsigned long long seed_l, int *mate, MlScratch &s, int *pairs) {
    const MlGraph mg = ml_view(g);
    int *h = reinterpret_cast<int *>(ctx->h_stage + 8192);
    CK(cudaMemsetAsync(mate, 0xff, sizeof(int) * (size_t)g->n, ctx->stream));
    for (int round = 0;; ++round) {
        if (round > g->n) {   // cannot happen: every round matches the best remaining edge
            ctx_error(ctx, "matching did not settle");
            return FR_ERR_INTERNAL;
        }
        CK(launch_ml_point(mg, part, k, W, seed_l, mate, s.cand, ctx->stream));
        CK(cudaMemsetAsync(s.flags, 0, sizeof(int), ctx->stream));
        CK(launch_ml_pair(g->n, mate, s.cand, s.flags, ctx->stream));
        CK(cudaMemcpyAsync(h, s.flags, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        if (!h[0]) break;
    }
    CK(cudaMemsetAsync(s.flags + 1, 0, sizeof(int), ctx->stream));
    CK(launch_ml_finish(g->n, mate, s.flags + 1, ctx->stream));
    CK(cudaMemcpyAsync(h, s.flags + 1, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    *pairs = h[0];
    return FR_OK;
}

// The coarse graph of a matching into caller arrays (room for n + 1, nnz, nnz, n);
// the row arrays are allocated by `alloc` once their size is known when cadj is NULL.
template <typename Alloc>
fr_status contract_level(fr_ctx *ctx, const fr_graph *g, const int *mate, int *cmap, MlScratch &s, int *cxadj,
                         int **cadj, int **cwgt, int *cvwgt, int *cn, int *cnnz, Alloc alloc) {
    const MlGraph mg = ml_view(g);
    int *h = reinterpret_cast<int *>(ctx->h_stage + 8192);
    CK(launch_ml_reps(g->n, mate, s.isrep, ctx->stream));
    CK(launch_ml_scan(s.isrep, s.cid, g->n, s.tmp, ctx->stream));
    CK(cudaMemcpyAsync(h, s.cid + g->n, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const int nc = h[0];
    CK(launch_ml_cmap(mg, mate, s.cid, cmap, cvwgt, s.crep, s.rowcap, ctx->stream));
    CK(launch_ml_rows(mg, nc, mate, cmap, s.crep, s.rowcap, true, s.cdeg, nullptr, nullptr, nullptr, ctx->stream));
    CK(launch_ml_scan(s.cdeg, cxadj, nc, s.tmp, ctx->stream));
    CK(cudaMemcpyAsync(h, cxadj + nc, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const int nnz = h[0];
    if (nnz > g->nnz) {   // cannot happen: contraction never adds arcs
        ctx_error(ctx, "contraction produced %d arcs from %d", nnz, g->nnz);
        return FR_ERR_INTERNAL;
    }
    if (!*cadj) {
        *cadj = alloc(nnz);
        *cwgt = alloc(nnz);
        if (!*cadj || !*cwgt) {
            ctx_error(ctx, "cudaMalloc for a coarse graph failed");
            return FR_ERR_OOM;
        }
    }
    CK(launch_ml_rows(mg, nc, mate, cmap, s.crep, s.rowcap, false, nullptr, cxadj, *cadj, *cwgt, ctx->stream));
    *cn = nc;
    *cnnz = nnz;
    return FR_OK;
}

double ms_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

extern "C" fr_status fr_match(fr_ctx *ctx, const fr_graph *g, const int32_t *part, int32_t k, int64_t W,
                              uint64_t seed_l, int32_t *mate, int32_t *pairs) {
    if (!ctx) return FR_ERR_INVALID_ARG;
    fr_status st = check_graph(ctx, g, part, k);
    if (st == FR_OK && (!mate || W < 0)) {
        ctx_error(ctx, "fr_match: mate needed, W >= 0");
        st = FR_ERR_INVALID_ARG;
    }
    if (st != FR_OK) return st;
    CK(cudaSetDevice(ctx->device));
    DevPool pool;
    MlScratch s;
    if (!s.make(pool, g->n)) {
        ctx_error(ctx, "cudaMalloc for the matching scratch failed");
        return FR_ERR_OOM;
    }
    int p = 0;
    st = match_level(ctx, g, part, k, W, seed_l, mate, s, &p);
    if (pairs) *pairs = p;
    return st;
}

extern "C" fr_status fr_contract(fr_ctx *ctx, const fr_graph *g, const int32_t *mate, int32_t *cmap, int32_t *cn,
                                 int32_t *cnnz, int32_t *cxadj, int32_t *cadjncy, int32_t *cadjwgt, int32_t *cvwgt) {
    if (!ctx) return FR_ERR_INVALID_ARG;
    if (!g || g->n < 1 || !g->xadj || !mate || !cmap || !cxadj || !cadjncy || !cadjwgt || !cvwgt || !cn || !cnnz) {
        ctx_error(ctx, "fr_contract: missing argument");
        return FR_ERR_INVALID_ARG;
    }
    CK(cudaSetDevice(ctx->device));
    DevPool pool;
    MlScratch s;
    if (!s.make(pool, g->n)) {
        ctx_error(ctx, "cudaMalloc for the contraction scratch failed");
        return FR_ERR_OOM;
    }
    // a caller's matching is checked first: the contraction indexes by it
    int *h = reinterpret_cast<int *>(ctx->h_stage + 8192);
    CK(cudaMemsetAsync(s.flags, 0, sizeof(int), ctx->stream));
    CK(launch_ml_check(g->n, mate, s.flags, ctx->stream));
    CK(cudaMemcpyAsync(h, s.flags, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (h[0]) {
        ctx_error(ctx, "fr_contract: mate is not a matching (entries must be -1 or partners pointing back)");
        return FR_ERR_INVALID_ARG;
    }
    int *adj = cadjncy, *wgt = cadjwgt;
    return contract_level(ctx, g, mate, cmap, s, cxadj, &adj, &wgt, cvwgt, cn, cnnz,
                          [](int) -> int * { return nullptr; });
}

extern "C" fr_status fr_vcycle(fr_ctx *ctx, const fr_graph *g, int32_t *part, int32_t k, double eps, double alpha,
                               const fr_options *opt_in, int32_t max_levels, int32_t active_outer,
                               fr_vcycle_result *out) {
    if (!ctx) return FR_ERR_INVALID_ARG;
    fr_options opt;
    if (opt_in) opt = *opt_in; else fr_default_options(&opt);
    if (out) memset(out, 0, sizeof(*out));
    fr_status st = check_graph(ctx, g, part, k);
    if (st == FR_OK) st = check_params(ctx, eps, alpha, &opt);
    if (st == FR_OK && (max_levels < 1 || max_levels > FR_MAX_LEVELS || active_outer < 0 ||
                        (opt.mt_alpha != 0 && active_outer == 0))) {
        ctx_error(ctx, "fr_vcycle: max_levels in [1, %d], active_outer >= 0, mt_alpha only with active_outer",
                  FR_MAX_LEVELS);
        st = FR_ERR_INVALID_ARG;
    }
    if (st != FR_OK) { if (out) out->status = st; return st; }
    CK(cudaSetDevice(ctx->device));
    release_corridor(ctx);
    st = ensure_base(ctx, g->n, g->nnz, k, opt.mb_reps);
    PrepOut po;
    if (st == FR_OK) st = run_prep(ctx, g, part, k, false, opt.checked != 0, &po);
    if (st != FR_OK) { if (out) out->status = st; return st; }
    const auto t0 = std::chrono::steady_clock::now();
    DevPool pool;
    MlScratch s;
    int *backup = pool.get<int>(g->n);
    int *mate = pool.get<int>(g->n);
    if (!backup || !mate || !s.make(pool, g->n)) {
        ctx_error(ctx, "cudaMalloc for the V-cycle scratch failed");
        if (out) out->status = FR_ERR_OOM;
        return FR_ERR_OOM;
    }
    CK(cudaMemcpyAsync(backup, part, sizeof(int) * (size_t)g->n, cudaMemcpyDeviceToDevice, ctx->stream));
    struct Level {
        fr_graph g;
        int *part;
        int *cmap;   // fine vertex -> vertex of the next coarser level
    };
    std::vector<Level> lv;
    lv.push_back({*g, part, nullptr});
    const long long W = po.W;
    const long long thr = std::max(60LL * k, (long long)g->n / (60LL * k));
    // contraction
    while ((int)lv.size() < max_levels && lv.back().g.n > thr && st == FR_OK) {
        Level &f = lv.back();
        const int l = (int)lv.size() - 1;
        int pairs = 0;
        st = match_level(ctx, &f.g, f.part, k, W, splitmix64(opt.seed ^ (unsigned long long)l), mate, s, &pairs);
        if (st != FR_OK || pairs == 0 || 20LL * pairs < f.g.n) break;   // stalled: under 5 %
        const int n_f = f.g.n;
        const int nc_bound = n_f - pairs;
        int *cmap = pool.get<int>(n_f);
        int *cxadj = pool.get<int>((long long)nc_bound + 1);
        int *cvwgt = pool.get<int>(nc_bound);
        int *cpart = pool.get<int>(nc_bound);
        if (!cmap || !cxadj || !cvwgt || !cpart) {
            ctx_error(ctx, "cudaMalloc for a coarse graph failed");
            st = FR_ERR_OOM;
            break;
        }
        int *cadj = nullptr, *cwgt = nullptr, cn = 0, cnnz = 0;
        st = contract_level(ctx, &f.g, mate, cmap, s, cxadj, &cadj, &cwgt, cvwgt, &cn, &cnnz,
                            [&](int cnt) { return pool.get<int>(cnt); });
        if (st != FR_OK) break;
        if (cn != nc_bound) {
            ctx_error(ctx, "contraction gave %d vertices, expected %d", cn, nc_bound);
            st = FR_ERR_INTERNAL;
            break;
        }
        const fr_graph fg = f.g;
        int *fpart = f.part;
        f.cmap = cmap;
        CK(launch_ml_down(fg.n, cmap, fpart, cpart, ctx->stream));
        fr_graph cg;
        cg.n = cn; cg.nnz = cnnz; cg.xadj = cxadj; cg.adjncy = cadj; cg.adjwgt = cwgt; cg.vwgt = cvwgt;
        lv.push_back({cg, cpart, nullptr});
    }
    const double coarsen_ms = ms_since(t0);
    const auto t1 = std::chrono::steady_clock::now();
    const int L = (int)lv.size();
    std::vector<int> lpairs(L, 0);
    std::vector<long long> lcut(L, 0);
    // refinement from the coarsest level up
    for (int l = L - 1; l >= 0 && st == FR_OK; --l) {
        if (l < L - 1) {
            cudaError_t e = launch_ml_up(lv[l].g.n, lv[l].cmap, lv[l + 1].part, lv[l].part, ctx->stream);
            if (e != cudaSuccess) { st = cuda_fail(ctx, e, "launch_ml_up"); break; }
        }
        fr_batch_result summ;
        // coarse graphs live only during this call: their sweeps launch directly instead
        // of being captured into the context's graph cache
        const bool graphs = ctx->use_graphs;
        if (l > 0) ctx->use_graphs = false;
        if (active_outer > 0)
            st = fr_refine_active(ctx, &lv[l].g, lv[l].part, k, eps, alpha, &opt, active_outer, 0, nullptr, &summ,
                                  nullptr);
        else
            st = fr_refine_batch(ctx, &lv[l].g, lv[l].part, k, eps, alpha, &opt, 0, nullptr, &summ);
        ctx->use_graphs = graphs;
        if (st != FR_OK) break;
        lpairs[l] = summ.npairs;
        lcut[l] = summ.cut_after;
    }
    cudaStreamSynchronize(ctx->stream);
    const double refine_ms = ms_since(t1);
    if (st != FR_OK) {
        cudaMemcpyAsync(part, backup, sizeof(int) * (size_t)g->n, cudaMemcpyDeviceToDevice, ctx->stream);
        cudaStreamSynchronize(ctx->stream);
        if (out) out->status = st;
        return st;
    }
    if (out) {
        out->levels = L;
        out->status = FR_OK;
        out->cut_before = po.totcut;
        out->cut_after = lcut[0];
        for (int l = 0; l < L; ++l) {
            out->level_n[l] = lv[l].g.n;
            out->level_pairs[l] = lpairs[l];
            out->level_cut[l] = lcut[l];
        }
        out->coarsen_ms = coarsen_ms;
        out->refine_ms = refine_ms;
    }
    return FR_OK;
}

// ------------------------------------------------------- W- and F-cycles ----

namespace {

struct CycleRun {
    fr_ctx *ctx;
    int k, type, d, max_levels, active_outer;
    double eps, alpha;
    fr_options opt;
    long long W, thr;
    int count[FR_MAX_LEVELS];
    fr_cycle_result *out;
    fr_status st;
    MlScratch *s;
    int *mate;
};

void cycle_refine(CycleRun &R, int l, const fr_graph &g, int *part) {
    if (R.st != FR_OK) return;
    fr_batch_result summ;
    fr_graph gg = g;
    // coarse graphs live only while their branch runs: their sweeps launch directly
    const bool graphs = R.ctx->use_graphs;
    if (l > 0) R.ctx->use_graphs = false;
    if (R.active_outer > 0)
        R.st = fr_refine_active(R.ctx, &gg, part, R.k, R.eps, R.alpha, &R.opt, R.active_outer, 0, nullptr, &summ,
                                nullptr);
    else
        R.st = fr_refine_batch(R.ctx, &gg, part, R.k, R.eps, R.alpha, &R.opt, 0, nullptr, &summ);
    R.ctx->use_graphs = graphs;
    R.out->refinements += 1;
}

// One coarsening of (g, part) at level l into pool memory; false if it stalled (or failed).
bool cycle_coarsen(CycleRun &R, int l, const fr_graph &g, const int *part, DevPool &pool, fr_graph &cg, int *&cmap,
                   int *&cpart) {
    fr_ctx *ctx = R.ctx;
    if (l + 1 >= R.max_levels || g.n <= R.thr) return false;
    const unsigned long long sl =
        splitmix64(R.opt.seed ^ (unsigned long long)l ^ ((unsigned long long)(unsigned)R.count[l] << 32));
    R.count[l] += 1;
    R.out->coarsenings += 1;
    int pairs = 0;
    R.st = match_level(ctx, &g, part, R.k, R.W, sl, R.mate, *R.s, &pairs);
    if (R.st != FR_OK || pairs == 0 || 20LL * pairs < g.n) return false;
    const int nc_bound = g.n - pairs;
    cmap = pool.get<int>(g.n);
    int *cxadj = pool.get<int>((long long)nc_bound + 1);
    int *cvwgt = pool.get<int>(nc_bound);
    cpart = pool.get<int>(nc_bound);
    if (!cmap || !cxadj || !cvwgt || !cpart) {
        ctx_error(ctx, "cudaMalloc for a coarse graph failed");
        R.st = FR_ERR_OOM;
        return false;
    }
    int *cadj = nullptr, *cwgt = nullptr, cn = 0, cnnz = 0;
    R.st = contract_level(ctx, &g, R.mate, cmap, *R.s, cxadj, &cadj, &cwgt, cvwgt, &cn, &cnnz,
                          [&](int cnt) { return pool.get<int>(cnt); });
    if (R.st != FR_OK) return false;
    if (cn != nc_bound) {
        ctx_error(ctx, "contraction gave %d vertices, expected %d", cn, nc_bound);
        R.st = FR_ERR_INTERNAL;
        return false;
    }
    cudaError_t e = launch_ml_down(g.n, cmap, part, cpart, ctx->stream);
    if (e != cudaSuccess) {
        R.st = cuda_fail(ctx, e, "launch_ml_down");
        return false;
    }
    cg.n = cn; cg.nnz = cnnz; cg.xadj = cxadj; cg.adjncy = cadj; cg.adjwgt = cwgt; cg.vwgt = cvwgt;
    return true;
}

void cycle_run(CycleRun &R, int l, const fr_graph &g, int *part) {
    if (R.st != FR_OK) return;
    R.out->depth = std::max(R.out->depth, l + 1);
    for (int trial = 0; trial < 2; ++trial) {
        if (trial == 1 && (R.type == 0 || l % R.d != 0 || (R.type == 2 && R.count[l] >= 2))) break;
        DevPool pool;   // this trial's coarse graph, freed when the trial ends
        fr_graph cg;
        int *cmap = nullptr, *cpart = nullptr;
        if (!cycle_coarsen(R, l, g, part, pool, cg, cmap, cpart)) {
            if (R.st == FR_OK && trial == 0) cycle_refine(R, l, g, part);   // the coarsest graph of this branch
            break;
        }
        cycle_run(R, l + 1, cg, cpart);
        if (R.st != FR_OK) return;
        cudaError_t e = launch_ml_up(g.n, cmap, cpart, part, R.ctx->stream);
        if (e != cudaSuccess) {
            R.st = cuda_fail(R.ctx, e, "launch_ml_up");
            return;
        }
        cycle_refine(R, l, g, part);
        cudaStreamSynchronize(R.ctx->stream);   // the pool is freed next
    }
}

}  // namespace

extern "C" fr_status fr_cycle(fr_ctx *ctx, const fr_graph *g, int32_t *part, int32_t k, double eps, double alpha,
                              const fr_options *opt_in, int32_t type, int32_t d, int32_t max_levels,
                              int32_t active_outer, fr_cycle_result *out) {
    if (!ctx) return FR_ERR_INVALID_ARG;
    fr_options opt;
    if (opt_in) opt = *opt_in; else fr_default_options(&opt);
    fr_cycle_result local;
    fr_cycle_result *o = out ? out : &local;
    memset(o, 0, sizeof(*o));
    fr_status st = check_graph(ctx, g, part, k);
    if (st == FR_OK) st = check_params(ctx, eps, alpha, &opt);
    if (st == FR_OK && (type < 0 || type > 2 || d < 1 || max_levels < 1 || max_levels > FR_MAX_LEVELS ||
                        active_outer < 0 || (opt.mt_alpha != 0 && active_outer == 0))) {
        ctx_error(ctx, "fr_cycle: type 0-2, d >= 1, max_levels in [1, %d], active_outer >= 0, mt_alpha only with "
                  "active_outer", FR_MAX_LEVELS);
        st = FR_ERR_INVALID_ARG;
    }
    if (st != FR_OK) { o->status = st; return st; }
    CK(cudaSetDevice(ctx->device));
    release_corridor(ctx);
    st = ensure_base(ctx, g->n, g->nnz, k, opt.mb_reps);
    PrepOut po;
    if (st == FR_OK) st = run_prep(ctx, g, part, k, false, opt.checked != 0, &po);
    if (st != FR_OK) { o->status = st; return st; }
    const auto t0 = std::chrono::steady_clock::now();
    DevPool pool;
    MlScratch s;
    int *backup = pool.get<int>(g->n);
    int *mate = pool.get<int>(g->n);
    if (!backup || !mate || !s.make(pool, g->n)) {
        ctx_error(ctx, "cudaMalloc for the cycle scratch failed");
        o->status = FR_ERR_OOM;
        return FR_ERR_OOM;
    }
    CK(cudaMemcpyAsync(backup, part, sizeof(int) * (size_t)g->n, cudaMemcpyDeviceToDevice, ctx->stream));
    CycleRun R;
    memset(&R, 0, sizeof(R));
    R.ctx = ctx; R.k = k; R.type = type; R.d = d; R.max_levels = max_levels; R.active_outer = active_outer;
    R.eps = eps; R.alpha = alpha; R.opt = opt; R.W = po.W;
    R.thr = std::max(60LL * k, (long long)g->n / (60LL * k));
    R.out = o; R.st = FR_OK; R.s = &s; R.mate = mate;
    cycle_run(R, 0, *g, part);
    cudaStreamSynchronize(ctx->stream);
    st = R.st;
    if (st != FR_OK) {
        cudaMemcpyAsync(part, backup, sizeof(int) * (size_t)g->n, cudaMemcpyDeviceToDevice, ctx->stream);
        cudaStreamSynchronize(ctx->stream);
        o->status = st;
        return st;
    }
    PrepOut pa;
    st = run_prep(ctx, g, part, k, false, false, &pa);
    if (st != FR_OK) { o->status = st; return st; }
    o->status = FR_OK;
    o->cut_before = po.totcut;
    o->cut_after = pa.totcut;
    for (int l = 0; l < FR_MAX_LEVELS; ++l) o->level_coarsenings[l] = R.count[l];
    o->ms = ms_since(t0);
    return FR_OK;
}
