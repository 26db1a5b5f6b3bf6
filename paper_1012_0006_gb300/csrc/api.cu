// C ABI of libflowref (include/flowref.h): context, workspace, host orchestration.
//
// Host code here only validates arguments, evaluates the two double expressions
// of the balance bounds (Section 2.1 / 4.1, without FMA contraction), sizes the
// device workspace and launches kernels; every step of the refinement runs in
// the kernels of round_kernel.cu and prep_kernel.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "api_internal.h"
#include "flowref.h"

using namespace fr;

// ------------------------------------------------------------------ helpers --

void ctx_error(fr_ctx *ctx, const char *fmt, ...) {
    if (!ctx) return;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
    va_end(ap);
}

fr_status cuda_fail(fr_ctx *ctx, cudaError_t e, const char *what) {
    ctx_error(ctx, "%s: %s", what, cudaGetErrorString(e));
    return FR_ERR_CUDA;
}

#define CK(call)                                               \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

// floor((1 + alpha*eps) * W / k), evaluated step by step in double precision.
long long host_budget_base(long long W, int k, double eps, double alpha) {
    double ae = alpha * eps;
    double t = 1.0 + ae;
    t = t * (double)W;
    t = t / (double)k;
    return (long long)std::floor(t);
}

// L_max = floor((1 + eps) * W / k) + max_v c(v)
long long host_lmax(long long W, long long maxc, int k, double eps) {
    double t = 1.0 + eps;
    t = t * (double)W;
    t = t / (double)k;
    return (long long)std::floor(t) + maxc;
}

static fr_status map_err(int e) {
    switch (e) {
        case E_OK: return FR_OK;
        case E_INVALID: return FR_ERR_INVALID_ARG;
        case E_ITER: return FR_ERR_ITER_LIMIT;
        case E_TOO_LARGE: return FR_ERR_TOO_LARGE;
        case E_ABORT: return FR_ERR_ABORTED;
        default: return FR_ERR_INTERNAL;
    }
}

fr_status status_from_ctl(fr_ctx *ctx, const Ctl &c, const char *where) {
    if (c.error == 0) return FR_OK;
    ctx_error(ctx, "%s: device reported error %d at check %d", where, c.error, c.error_where);
    return map_err(c.error);
}

// ---------------------------------------------------------------- workspace --

template <class T>
static T *carve(char *&p, size_t count) {
    size_t bytes = ((sizeof(T) * count + 255) / 256) * 256;
    T *r = reinterpret_cast<T *>(p);
    p += bytes;
    return r;
}

static size_t base_bytes(long long n, long long nnz, int k, int reps, int grid) {
    const long long nu = n, mu = nnz;
    size_t b = 0;
    auto add = [&](size_t elem, long long cnt) { b += ((elem * (size_t)cnt + 255) / 256) * 256; };
    add(4, n); add(4, n);                                   // dist, lid
    add(4, n); add(4, n);                                   // vq_v, vq_s
    add(4, n / 32 + 2);                                     // cbits
    add(4, n); add(4, n); add(4, 1);                        // bl, inb, blc
    for (int i = 0; i < 13; ++i) add(4, nu + 1);            // gid sid off infc fx lab rflag color scc vc fq0 fq1 ...
    add(8, nu); add(1, nu); add(1, nu);                     // ex border side_out
    for (int i = 0; i < 4; ++i) add(4, mu);                 // head rev res cap
    add(4, grid + 1);                                       // cta_cnt
    add(8, nu);                                             // cw
    for (int i = 0; i < 9; ++i) add(4, nu + 1);             // cpair cmin cid indeg outoff ocur plist sinkc part_backup(n)
    add(4, mu);                                             // outs
    add(8, k);                                              // blockw
    add(4, ((long long)k * k + 31) / 32);                   // qbits
    add(4, (long long)k * ((2 * k + 31) / 32));             // used
    add(4, (long long)2 * k * k);                           // sob_round (2k rounds max)
    add(4, (long long)k * (k - 1) / 2 + 1); add(4, (long long)k * (k - 1) / 2 + 1);  // pair_a pair_b
    add(4, (long long)k * (k - 1) / 2 + 1);                 // pair_round
    add(4, 2 * k + 2);                                      // round_off
    add(sizeof(PrepOut), 1);
    add(4, k);                                              // sob of a single pair
    add(4, 4);                                              // flags
    return b;
}

static size_t pair_bytes(long long P, int R, int reps) {
    size_t b = 0;
    auto add = [&](size_t elem, long long cnt) { b += ((elem * (size_t)cnt + 255) / 256) * 256; };
    add(sizeof(GraphDev), R);
    add(sizeof(PairDev), P);
    add(sizeof(SideDev), 2 * P);
    add(sizeof(PairAcc), P);
    add(sizeof(Ctl), R);
    add(8, 3LL * 2 * P * kHistBins);
    add(4, P);
    (void)reps;
    return b;
}

// Arrays whose size grows with the number of sweeps R (they hold no state between
// steps, so they can be reallocated without touching a live corridor).
static size_t reps_bytes(long long nu, long long P, int reps) {
    size_t b = 0;
    auto add = [&](size_t elem, long long cnt) { b += ((elem * (size_t)cnt + 255) / 256) * 256; };
    add(4, (long long)reps * nu); add(4, (long long)reps * nu); add(4, (long long)reps * nu);  // indeg_r order hcomp
    add(8, (long long)reps * nu);                           // hkey
    add(8, P * reps);                                       // sw_absd
    add(4, P * reps);                                       // sw_j
    return b;
}

fr_status ensure_reps(fr_ctx *ctx, int reps) {
    if (reps < 1) reps = 1;
    const long long nu = ctx->n_cap;
    const long long P = std::max(ctx->pairs_cap, 1);
    if (ctx->reps_mem && reps <= ctx->reps_cap && nu <= ctx->reps_nu && P <= ctx->reps_P) return FR_OK;
    const int rr = std::max(reps, ctx->reps_cap);
    const size_t bytes = reps_bytes(nu, P, rr);
    if (ctx->arena_limit && bytes + ctx->base_bytes + ctx->pair_bytes > ctx->arena_limit) {
        ctx_error(ctx, "sweep workspace exceeds the arena bound");
        return FR_ERR_OOM;
    }
    destroy_graph_cache(ctx);   // captured sweeps hold pointers into the old workspace
    if (ctx->reps_mem) cudaFree(ctx->reps_mem);
    ctx->reps_mem = nullptr;
    ctx->reps_bytes = 0;
    if (cudaMalloc(&ctx->reps_mem, bytes) != cudaSuccess) {
        cudaGetLastError();
        ctx_error(ctx, "cudaMalloc(%zu) for sweep state failed", bytes);
        return FR_ERR_OOM;
    }
    ctx->reps_bytes = bytes;
    ctx->reps_cap = rr;
    ctx->reps_nu = nu;
    ctx->reps_P = P;
    char *p = reinterpret_cast<char *>(ctx->reps_mem);
    ctx->indeg_r = carve<int>(p, (long long)rr * nu);
    ctx->order = carve<int>(p, (long long)rr * nu);
    ctx->hcomp = carve<int>(p, (long long)rr * nu);
    ctx->hkey = carve<unsigned long long>(p, (long long)rr * nu);
    ctx->sw_absd = carve<long long>(p, P * rr);
    ctx->sw_j = carve<int>(p, P * rr);
    return FR_OK;
}

static void free_base(fr_ctx *ctx) {
    if (ctx->base_mem) cudaFree(ctx->base_mem);
    ctx->base_mem = nullptr;
    ctx->base_bytes = 0;
    ctx->n_cap = ctx->nnz_cap = ctx->k_cap = ctx->reps_cap = 0;
}

static void free_pairs(fr_ctx *ctx) {
    if (ctx->pair_mem) cudaFree(ctx->pair_mem);
    ctx->pair_mem = nullptr;
    ctx->pair_bytes = 0;
    ctx->pairs_cap = ctx->rounds_cap = 0;
}

fr_status ensure_base(fr_ctx *ctx, int n, int nnz, int k, int reps) {
    if (reps < 1) reps = 1;
    if (ctx->base_mem && n <= ctx->n_cap && nnz <= ctx->nnz_cap && k <= ctx->k_cap)
        return ensure_reps(ctx, reps);
    const int nn = std::max(n, ctx->n_cap), mm = std::max(nnz, ctx->nnz_cap);
    const int kk = std::max(k, ctx->k_cap), rr = reps;
    const int grid = ctx->max_coop + 1;
    const size_t bytes = base_bytes(nn, mm, kk, rr, grid);
    if (ctx->arena_limit && bytes + ctx->pair_bytes > ctx->arena_limit) {
        ctx_error(ctx, "workspace of %zu bytes exceeds the arena bound %zu", bytes + ctx->pair_bytes, ctx->arena_limit);
        return FR_ERR_OOM;
    }
    free_base(ctx);
    cudaError_t e = cudaMalloc(&ctx->base_mem, bytes);
    if (e != cudaSuccess) {
        ctx->base_mem = nullptr;
        cudaGetLastError();
        ctx_error(ctx, "cudaMalloc(%zu) for the workspace failed: %s", bytes, cudaGetErrorString(e));
        return FR_ERR_OOM;
    }
    ctx->base_bytes = bytes;
    ctx->n_cap = nn; ctx->nnz_cap = mm; ctx->k_cap = kk;
    char *p = reinterpret_cast<char *>(ctx->base_mem);
    const long long nu = nn, mu = mm;
    ctx->dist = carve<int>(p, nn); ctx->lid = carve<int>(p, nn);
    ctx->vq_v = carve<int>(p, nn); ctx->vq_s = carve<int>(p, nn);
    ctx->cbits = carve<unsigned int>(p, nn / 32 + 2);
    ctx->bl = carve<int>(p, nn); ctx->inb = carve<int>(p, nn); ctx->blc = carve<int>(p, 1);
    ctx->gid = carve<int>(p, nu + 1); ctx->sid = carve<int>(p, nu + 1); ctx->off = carve<int>(p, nu + 1);
    ctx->infc = carve<int>(p, nu + 1); ctx->fx = carve<int>(p, nu + 1); ctx->lab = carve<int>(p, nu + 1);
    ctx->rflag = carve<int>(p, nu + 1); ctx->color = carve<int>(p, nu + 1); ctx->scc = carve<int>(p, nu + 1);
    ctx->vc = carve<int>(p, nu + 1); ctx->fq0 = carve<int>(p, nu + 1); ctx->fq1 = carve<int>(p, nu + 1);
    ctx->spare = carve<int>(p, nu + 1);
    ctx->ex = carve<long long>(p, nu); ctx->border = carve<unsigned char>(p, nu);
    ctx->side_out = carve<unsigned char>(p, nu);
    ctx->head = carve<int>(p, mu); ctx->rev = carve<int>(p, mu); ctx->res = carve<int>(p, mu);
    ctx->cap = carve<int>(p, mu);
    ctx->cta_cnt = carve<int>(p, grid + 1);
    ctx->cw = carve<long long>(p, nu);
    ctx->cpair = carve<int>(p, nu + 1); ctx->cmin = carve<int>(p, nu + 1); ctx->cid = carve<int>(p, nu + 1);
    ctx->indeg = carve<int>(p, nu + 1); ctx->outoff = carve<int>(p, nu + 1); ctx->ocur = carve<int>(p, nu + 1);
    ctx->plist = carve<int>(p, nu + 1); ctx->sinkc = carve<int>(p, nu + 1); ctx->part_backup = carve<int>(p, nu + 1);
    ctx->outs = carve<int>(p, mu);
    ctx->blockw = carve<long long>(p, kk);
    ctx->qbits = carve<unsigned int>(p, ((long long)kk * kk + 31) / 32);
    ctx->used = carve<unsigned int>(p, (long long)kk * ((2 * kk + 31) / 32));
    ctx->sob_round = carve<int>(p, (long long)2 * kk * kk);
    ctx->pair_a = carve<int>(p, (long long)kk * (kk - 1) / 2 + 1);
    ctx->pair_b = carve<int>(p, (long long)kk * (kk - 1) / 2 + 1);
    ctx->pair_round = carve<int>(p, (long long)kk * (kk - 1) / 2 + 1);
    ctx->round_off = carve<int>(p, 2 * kk + 2);
    ctx->prep = carve<PrepOut>(p, 1);
    ctx->sob1 = carve<int>(p, kk);
    ctx->flags = carve<int>(p, 4);
    // idle state: dist = lid = -1
    CK(cudaMemsetAsync(ctx->dist, 0xFF, sizeof(int) * (size_t)nn, ctx->stream));
    CK(cudaMemsetAsync(ctx->lid, 0xFF, sizeof(int) * (size_t)nn, ctx->stream));
    CK(cudaMemsetAsync(ctx->cbits, 0, sizeof(unsigned int) * (size_t)(nn / 32 + 2), ctx->stream));
    destroy_graph_cache(ctx);   // captured sweeps hold pointers into the old workspace
    return ensure_reps(ctx, rr);
}

fr_status ensure_fm(fr_ctx *ctx, int n, int nnz, int k, int P) {
    if (ctx->fm_mem && n <= ctx->fm_n && nnz <= ctx->fm_nnz && k <= ctx->fm_k && P <= ctx->fm_p) return FR_OK;
    const long long nn = std::max(n, ctx->fm_n), mm = std::max(nnz, ctx->fm_nnz);
    const int kk = std::max(k, ctx->fm_k), pp = std::max(P, ctx->fm_p);
    const long long ecap = nn + mm, scap = 2 * nn;
    size_t b = 0;
    auto add = [&](size_t elem, long long cnt) { b += ((elem * (size_t)cnt + 255) / 256) * 256; };
    add(4, nn); add(4, nn); add(4, nn); add(1, nn);         // in ext ver flags
    add(4, nn); add(4, nn);                                 // vlist mlog
    add(4, kk); add(4, kk);                                 // blockn blockarcs
    add(8, pp); add(8, pp + 1); add(4, pp); add(4, pp);     // voff eoff np bcnt
    add(4, ecap); add(4, ecap); add(4, ecap);               // ent_v ent_ver ent_below
    add(8, scap); add(4, scap); add(4, scap);               // skey sbkt sv
    add(sizeof(FmRes), pp);                                 // res
    if (ctx->arena_limit && b + ctx->base_bytes + ctx->pair_bytes > ctx->arena_limit) {
        ctx_error(ctx, "FM workspace of %zu bytes exceeds the arena bound", b);
        return FR_ERR_OOM;
    }
    free_fm(ctx);
    if (cudaMalloc(&ctx->fm_mem, b) != cudaSuccess) {
        ctx->fm_mem = nullptr;
        cudaGetLastError();
        ctx_error(ctx, "cudaMalloc(%zu) for the FM workspace failed", b);
        return FR_ERR_OOM;
    }
    ctx->fm_bytes = b;
    ctx->fm_n = (int)nn; ctx->fm_nnz = (int)mm; ctx->fm_k = kk; ctx->fm_p = pp;
    char *p = reinterpret_cast<char *>(ctx->fm_mem);
    FmDev &f = ctx->fm;
    f.in = carve<int>(p, nn); f.ext = carve<int>(p, nn); f.ver = carve<int>(p, nn);
    f.flags = carve<unsigned char>(p, nn);
    f.vlist = carve<int>(p, nn); f.mlog = carve<int>(p, nn);
    f.blockn = carve<int>(p, kk); f.blockarcs = carve<int>(p, kk);
    f.voff = carve<long long>(p, pp); f.eoff = carve<long long>(p, pp + 1);
    f.np = carve<int>(p, pp); f.bcnt = carve<int>(p, pp);
    f.ent_v = carve<int>(p, ecap); f.ent_ver = carve<int>(p, ecap); f.ent_below = carve<int>(p, ecap);
    f.skey = carve<unsigned long long>(p, scap); f.sbkt = carve<int>(p, scap); f.sv = carve<int>(p, scap);
    f.res = carve<FmRes>(p, pp);
    f.ecap = ecap; f.scap = scap;
    // per-vertex state is zero between searches; block counts start at zero
    CK(cudaMemsetAsync(f.ver, 0, sizeof(int) * (size_t)nn, ctx->stream));
    CK(cudaMemsetAsync(f.flags, 0, (size_t)nn, ctx->stream));
    CK(cudaMemsetAsync(f.blockn, 0, sizeof(int) * (size_t)kk, ctx->stream));
    CK(cudaMemsetAsync(f.blockarcs, 0, sizeof(int) * (size_t)kk, ctx->stream));
    destroy_graph_cache(ctx);   // captured sweeps hold pointers into the old workspace
    return FR_OK;
}

void free_fm(fr_ctx *ctx) {
    if (ctx->fm_mem) cudaFree(ctx->fm_mem);
    ctx->fm_mem = nullptr;
    ctx->fm_bytes = 0;
    ctx->fm_n = ctx->fm_nnz = ctx->fm_k = ctx->fm_p = 0;
    ctx->fm = FmDev{};
}

FmDev fm_view(fr_ctx *ctx, int p0, const fr_options *opt) {
    FmDev f = ctx->fm;
    f.res = ctx->fm.res + p0;
    f.maxwdeg = &ctx->prep->maxwdeg;
    f.permille = opt ? opt->fm_permille : 0;
    return f;
}

fr_status ensure_pairs(fr_ctx *ctx, int P, int R, int reps) {
    if (reps < 1) reps = 1;
    if (ctx->pair_mem && P <= ctx->pairs_cap && R <= ctx->rounds_cap) return ensure_reps(ctx, reps);
    const int pp = std::max(P, ctx->pairs_cap), rr = std::max(R, ctx->rounds_cap);
    const int rp = reps;
    const size_t bytes = pair_bytes(pp, rr, rp);
    if (ctx->arena_limit && bytes + ctx->base_bytes > ctx->arena_limit) {
        ctx_error(ctx, "pair workspace of %zu bytes exceeds the arena bound", bytes);
        return FR_ERR_OOM;
    }
    free_pairs(ctx);
    cudaError_t e = cudaMalloc(&ctx->pair_mem, bytes);
    if (e != cudaSuccess) {
        ctx->pair_mem = nullptr;
        cudaGetLastError();
        ctx_error(ctx, "cudaMalloc(%zu) for pair state failed", bytes);
        return FR_ERR_OOM;
    }
    ctx->pair_bytes = bytes;
    ctx->pairs_cap = pp; ctx->rounds_cap = rr;
    char *p = reinterpret_cast<char *>(ctx->pair_mem);
    ctx->graphs = carve<GraphDev>(p, rr);
    ctx->pairs = carve<PairDev>(p, pp);
    ctx->sides = carve<SideDev>(p, 2LL * pp);
    ctx->pacc = carve<PairAcc>(p, pp);
    ctx->ctl = carve<Ctl>(p, rr);
    ctx->hist = carve<long long>(p, 3LL * 2 * pp * kHistBins);
    ctx->pcur = carve<int>(p, pp);
    destroy_graph_cache(ctx);   // captured sweeps hold pointers into the old workspace
    return ensure_reps(ctx, rp);
}

// Work descriptor of round r (pairs [p0, p0 + P) of the pair arrays).
Work make_work(fr_ctx *ctx, int r, int p0, int P, int n, const fr_options *opt) {
    Work w;
    memset(&w, 0, sizeof(w));
    w.graphs = ctx->graphs + r;
    w.pairs = ctx->pairs + p0;
    w.sides = ctx->sides + 2LL * p0;
    w.pacc = ctx->pacc + p0;
    w.ctl = ctx->ctl + r;
    w.prev_err = r > 0 ? &ctx->ctl[r - 1].error : nullptr;
    w.ngraphs = 1;
    w.npairs = P;
    w.nsides = 2 * P;
    w.total_n = n;
    w.vq_v = ctx->vq_v; w.vq_s = ctx->vq_s; w.vq_cap = ctx->n_cap; w.cbits = ctx->cbits;
    w.gid = ctx->gid; w.sid = ctx->sid; w.off = ctx->off; w.head = ctx->head; w.rev = ctx->rev; w.res = ctx->res;
    w.cap = ctx->cap; w.infc = ctx->infc; w.fx = ctx->fx; w.lab = ctx->lab; w.rflag = ctx->rflag;
    w.color = ctx->color; w.scc = ctx->scc; w.vc = ctx->vc; w.ex = ctx->ex; w.border = ctx->border;
    w.side_out = ctx->side_out;
    w.nu_cap = ctx->n_cap; w.mu_cap = ctx->nnz_cap;
    w.fq0 = ctx->fq0; w.fq1 = ctx->fq1; w.cta_cnt = ctx->cta_cnt;
    w.hist = ctx->hist + 3LL * 2 * p0 * kHistBins;
    w.cw = ctx->cw; w.cpair = ctx->cpair; w.cmin = ctx->cmin; w.cid = ctx->cid; w.indeg = ctx->indeg;
    w.outoff = ctx->outoff; w.outs = ctx->outs; w.ocur = ctx->ocur; w.plist = ctx->plist; w.pcur = ctx->pcur + p0;
    w.indeg_r = ctx->indeg_r; w.order = ctx->order; w.sinkc = ctx->sinkc; w.hkey = ctx->hkey; w.hcomp = ctx->hcomp;
    const int reps = opt && opt->mb_reps > 0 ? opt->mb_reps : 1;
    w.sw_absd = ctx->sw_absd + (long long)p0 * reps;
    w.sw_j = ctx->sw_j + (long long)p0 * reps;
    w.reps = reps;
    w.gr_interval = opt && opt->gr_interval > 0 ? opt->gr_interval : ctx->tune_gr;
    w.inner = opt && opt->inner_ops > 0 ? opt->inner_ops : ctx->tune_inner;
    w.passes = opt && opt->pulse_passes > 0 ? opt->pulse_passes : ctx->tune_passes;
    w.flow_sched = opt && opt->flow_sched ? opt->flow_sched : ctx->tune_sched;
    w.any_mb = opt && opt->mb ? 1 : 0;
    w.seed = opt ? opt->seed : 0;
    w.pulse_cap = opt && opt->pulse_cap > 0 ? opt->pulse_cap : (1LL << 20);
    w.narrow = ctx->narrow_ok;
    w.pre_waves = opt && opt->pre_waves ? (opt->pre_waves < 0 ? 0 : opt->pre_waves) : ctx->tune_prewaves;
    w.gap_interval = gap_interval_of(opt);
    return w;
}

int gap_interval_of(const fr_options *opt) {
    if (!opt || opt->gap_interval == 0) return 8;
    return opt->gap_interval < 0 ? 0 : opt->gap_interval;
}

int choose_tpb(fr_ctx *ctx, const fr_options *opt) {
    int t = opt && opt->block_threads ? opt->block_threads : ctx->tune_tpb;
    return t == 256 ? 256 : 512;
}

// Grid of the persistent kernel: the tuned/requested CTA count, bounded by
// co-residency; small corridors get fewer CTAs (cheaper barriers).
int choose_grid(fr_ctx *ctx, const fr_options *opt, int tpb, int nsides, long long est_vertices) {
    int maxb = 0, sms = 0;
    if (step_max_grid(tpb, nsides, &maxb, &sms) != cudaSuccess || maxb < 1) maxb = 1;
    int want;
    if (opt && opt->grid_blocks > 0) want = opt->grid_blocks;
    else if (ctx->tune_grid > 0) want = ctx->tune_grid;
    else {
        long long per = (long long)tpb * 2;
        long long b = (est_vertices + per - 1) / per;
        if (b < 1) b = 1;
        want = (int)std::min<long long>(b, sms);
    }
    return std::max(1, std::min(want, maxb));
}

// ---------------------------------------------------------------- context --

extern "C" int32_t fr_struct_size(int32_t which) {
    switch (which) {
    case 0: return (int32_t)sizeof(fr_graph);
    case 1: return (int32_t)sizeof(fr_options);
    case 2: return (int32_t)sizeof(fr_pair_result);
    case 3: return (int32_t)sizeof(fr_batch_result);
    case 4: return (int32_t)sizeof(fr_profile_info);
    case 5: return (int32_t)sizeof(fr_server_config);
    case 6: return (int32_t)sizeof(fr_request);
    case 7: return (int32_t)sizeof(fr_response);
    case 8: return (int32_t)sizeof(fr_mt_result);
    case 9: return (int32_t)sizeof(fr_vcycle_result);
    case 10: return (int32_t)sizeof(fr_cycle_result);
    default: return -1;
    }
}

extern "C" void fr_default_options(fr_options *opt) {
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->mb = 0;
    opt->mb_reps = 1;
    opt->adaptive = 0;
    opt->max_iters = 10;
    opt->alpha_max = 1.0;
    opt->seed = 0;
    opt->pulse_cap = 1LL << 20;
}

extern "C" fr_status fr_create(fr_ctx **out, int32_t device, size_t arena_bytes, void *stream) {
    if (!out) return FR_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= device || device < 0) {
        cudaGetLastError();
        return FR_ERR_CUDA;
    }
    fr_ctx *ctx = new fr_ctx();
    ctx->device = device;
    ctx->arena_limit = arena_bytes;
    if (cudaSetDevice(device) != cudaSuccess) { delete ctx; return FR_ERR_CUDA; }
    if (stream) {
        ctx->stream = reinterpret_cast<cudaStream_t>(stream);
        ctx->own_stream = false;
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) { delete ctx; return FR_ERR_CUDA; }
        ctx->own_stream = true;
    }
    int maxb = 0, sms = 0;
    if (step_max_grid(512, 64, &maxb, &sms) != cudaSuccess) { delete ctx; return FR_ERR_CUDA; }
    ctx->sms = sms;
    ctx->max_coop = std::max(maxb, 1) * 4;
    for (int t = 0; t < fr_ctx::kNumClusterSizes; ++t) {
        int mc = 0;
        if (cluster_flow_capacity(fr_ctx::kClusterSizes[t], &mc) != cudaSuccess) {
            cudaGetLastError();
            mc = 0;
        }
        ctx->cl_cap[t] = mc;
        ctx->max_clusters = std::max(ctx->max_clusters, mc);
        int qc = 0;
        if (queue_capacity(fr_ctx::kClusterSizes[t], &qc) != cudaSuccess) {
            cudaGetLastError();
            qc = 0;
        }
        ctx->q_cap[t] = qc;
    }
    cudaEventCreate(&ctx->ev0);
    cudaEventCreate(&ctx->ev1);
    if (cudaHostAlloc(&ctx->h_stage, kHostStage, cudaHostAllocDefault) != cudaSuccess) {
        delete ctx;
        return FR_ERR_CUDA;
    }
    *out = ctx;
    return FR_OK;
}

extern "C" fr_status fr_destroy(fr_ctx *ctx) {
    if (!ctx) return FR_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    destroy_graph_cache(ctx);
    free_base(ctx);
    free_pairs(ctx);
    free_fm(ctx);
    free_mt(ctx);
    free_queue(ctx);
    if (ctx->reps_mem) cudaFree(ctx->reps_mem);
    if (ctx->hg_mem) cudaFree(ctx->hg_mem);
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    cudaEventDestroy(ctx->ev0);
    cudaEventDestroy(ctx->ev1);
    for (auto e : ctx->pev) cudaEventDestroy(e);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return FR_OK;
}

extern "C" const char *fr_last_error(const fr_ctx *ctx) { return ctx ? ctx->err : "no context"; }

extern "C" const char *fr_status_string(fr_status st) {
    switch (st) {
        case FR_OK: return "ok";
        case FR_ERR_INVALID_ARG: return "invalid argument";
        case FR_ERR_CUDA: return "CUDA error";
        case FR_ERR_OOM: return "out of device memory / arena";
        case FR_ERR_ITER_LIMIT: return "device iteration limit reached";
        case FR_ERR_TOO_LARGE: return "problem too large";
        case FR_ERR_ABORTED: return "aborted";
        case FR_ERR_INTERNAL: return "internal consistency check failed";
    }
    return "unknown status";
}

extern "C" size_t fr_workspace_bytes(const fr_ctx *ctx) {
    return ctx ? ctx->base_bytes + ctx->pair_bytes + ctx->reps_bytes : 0;
}

// ---------------------------------------------------------- argument checks --

fr_status check_graph(fr_ctx *ctx, const fr_graph *g, const int32_t *part, int32_t k) {
    if (!g || !part) { ctx_error(ctx, "graph or part is NULL"); return FR_ERR_INVALID_ARG; }
    if (g->n < 1 || g->nnz < 0 || !g->xadj || !g->vwgt || (g->nnz > 0 && (!g->adjncy || !g->adjwgt))) {
        ctx_error(ctx, "graph arrays or sizes are invalid (n=%d nnz=%d)", g->n, g->nnz);
        return FR_ERR_INVALID_ARG;
    }
    if (k < 2 || k > kMaxK) { ctx_error(ctx, "k=%d outside [2, %d]", k, kMaxK); return FR_ERR_INVALID_ARG; }
    return FR_OK;
}

fr_status validate_params(double eps, double alpha, const fr_options *opt, const char **why) {
    *why = nullptr;
    if (!(eps > 0.0) || !std::isfinite(eps)) *why = "epsilon must be > 0";
    else if (!(alpha >= 1.0) || !std::isfinite(alpha)) *why = "alpha must be >= 1";
    else if (opt) {
        if (opt->mb_reps < 0 || opt->max_iters < 0 || opt->pulse_cap < 0) *why = "negative option";
        else if (opt->adaptive && !(opt->alpha_max >= 1.0)) *why = "alpha_max must be >= 1";
        else if (opt->block_threads && opt->block_threads != 256 && opt->block_threads != 512)
            *why = "block_threads must be 256 or 512";
        else if (opt->mb_reps > 64) *why = "mb_reps > 64";
        else if (opt->pre_waves < -1 || opt->pre_waves > 4) *why = "pre_waves must be in [-1, 4]";
        else if (opt->fm_permille < 0 || opt->fm_permille > 1000) *why = "fm_permille must be in [0, 1000]";
        else if (opt->mt_alpha < 0) *why = "mt_alpha must be >= 0";
        else if (opt->sweep_sched < 0 || opt->sweep_sched > 1) *why = "sweep_sched must be 0 or 1";
        else if (opt->gap_interval < -1) *why = "gap_interval must be >= -1";
        else if (opt->cluster_ctas != 0) {
            bool known = false;
            for (int t = 0; t < fr_ctx::kNumClusterSizes; ++t) known |= opt->cluster_ctas == fr_ctx::kClusterSizes[t];
            if (!known) *why = "cluster_ctas must be 0, 4, 6, 8, 12 or 16";
        }
    }
    return *why ? FR_ERR_INVALID_ARG : FR_OK;
}

fr_status check_params(fr_ctx *ctx, double eps, double alpha, const fr_options *opt) {
    const char *why = nullptr;
    const fr_status st = validate_params(eps, alpha, opt, &why);
    if (st != FR_OK) ctx_error(ctx, "%s", why);
    return st;
}

// Validation pass + W, max c, block weights (and the quotient graph when qbits).
fr_status run_prep(fr_ctx *ctx, const fr_graph *g, const int32_t *part, int32_t k, bool quotient, bool checked,
                   PrepOut *host_out) {
    CK(cudaMemsetAsync(ctx->prep, 0, sizeof(PrepOut), ctx->stream));
    CK(cudaMemsetAsync(ctx->blockw, 0, sizeof(long long) * k, ctx->stream));
    if (quotient) CK(cudaMemsetAsync(ctx->qbits, 0, sizeof(unsigned int) * (((size_t)k * k + 31) / 32), ctx->stream));
    CK(launch_prep(g->xadj, g->adjncy, g->adjwgt, g->vwgt, part, g->n, g->nnz, k, ctx->blockw,
                   quotient ? ctx->qbits : nullptr, ctx->prep, ctx->stream, ctx->bl, ctx->blc, ctx->inb));
    if (checked) CK(launch_check_symmetric(g->xadj, g->adjncy, g->adjwgt, g->n, ctx->prep, ctx->stream));
    if (quotient)
        CK(launch_color(ctx->qbits, k, ctx->pair_a, ctx->pair_b, ctx->pair_round, ctx->round_off, ctx->sob_round,
                        ctx->used, ctx->prep, ctx->stream));
    PrepOut *h = reinterpret_cast<PrepOut *>(ctx->h_stage);
    CK(cudaMemcpyAsync(h, ctx->prep, sizeof(PrepOut), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    *host_out = *h;
    ctx->narrow_ok = h->maxw < (1 << 15) ? 1 : 0;
    if (h->err) {
        ctx_error(ctx, h->err == E_TOO_LARGE ? "weighted degree >= 2^30" :
                       "graph or partition violates the input conventions (ids, weights, part range, symmetry)");
        return map_err(h->err);
    }
    return FR_OK;
}

// Step state of one pair on graph g (round slot 0): descriptors + cleared counters.
fr_status setup_single(fr_ctx *ctx, const fr_graph *g, int32_t *part, int32_t k, int32_t a, int32_t b,
                       long long Ubase, long long Lmax, int mb) {
    GraphDev gd;
    memset(&gd, 0, sizeof(gd));
    gd.xadj = g->xadj; gd.adjncy = g->adjncy; gd.adjwgt = g->adjwgt; gd.vwgt = g->vwgt;
    gd.part = part; gd.dist = ctx->dist; gd.lid = ctx->lid; gd.sob = ctx->sob1; gd.blockw = ctx->blockw;
    gd.n = g->n; gd.nnz = g->nnz; gd.k = k; gd.base = 0; gd.Lmax = Lmax;
    gd.bl = ctx->bl; gd.blc = ctx->blc; gd.inb = ctx->inb;
    PairDev pd;
    pd.g = 0; pd.a = a; pd.b = b; pd.mb = mb; pd.Ubase = Ubase;
    char *h = ctx->h_stage + 1024;   // staging after the PrepOut slot
    memcpy(h, &gd, sizeof(gd));
    memcpy(h + 256, &pd, sizeof(pd));
    int *hs = reinterpret_cast<int *>(h + 512);
    hs[0] = 0;
    hs[1] = 1;
    CK(cudaMemcpyAsync(ctx->graphs, h, sizeof(gd), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->pairs, h + 256, sizeof(pd), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemsetAsync(ctx->sob1, 0xFF, sizeof(int) * k, ctx->stream));
    CK(cudaMemcpyAsync(ctx->sob1 + a, hs, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->sob1 + b, hs + 1, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemsetAsync(ctx->ctl, 0, sizeof(Ctl), ctx->stream));
    CK(cudaMemsetAsync(ctx->sides, 0, 2 * sizeof(SideDev), ctx->stream));
    CK(cudaMemsetAsync(ctx->pacc, 0, sizeof(PairAcc), ctx->stream));
    CK(cudaMemsetAsync(ctx->hist, 0, sizeof(long long) * 3 * 2 * kHistBins, ctx->stream));
    // h_stage is pinned, so the copies run asynchronously: its bytes [1024, 1544) must stay
    // as written until they ran.  Every caller synchronises the stream (reading its results
    // back) before anything writes there again, so no synchronisation is needed here.
    return FR_OK;
}

// Clears dist / lid after a failed step (the kernel may have stopped before its cleanup).
fr_status reset_idle(fr_ctx *ctx) {
    CK(cudaMemsetAsync(ctx->dist, 0xFF, sizeof(int) * (size_t)ctx->n_cap, ctx->stream));
    CK(cudaMemsetAsync(ctx->lid, 0xFF, sizeof(int) * (size_t)ctx->n_cap, ctx->stream));
    CK(cudaMemsetAsync(ctx->cbits, 0, sizeof(unsigned int) * (size_t)(ctx->n_cap / 32 + 2), ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return FR_OK;
}

// Cluster launches of one round's max flows: tier 0 with the smallest cluster that
// holds the estimated largest network (or opt->cluster_ctas), then, if tier 0 was
// smaller than the largest size, tier 1 with the largest clusters for the pairs that
// did not fit (it returns at once when there are none).  Smaller clusters let more
// pairs of a round run at once.  Returns the launches enqueued in *nl.
cudaError_t launch_clusters(fr_ctx *ctx, Work &w, long long est_pair_vertices, double avg_degree, int force,
                            cudaStream_t st, int *nl) {
    *nl = 0;
    const int T = fr_ctx::kNumClusterSizes;
    // shared memory a pair needs: ~29 B per vertex and 16 B per arc (20 B when
    // capacities do not pack into 16 bits), plus a little for an uneven split; a CTA
    // has cluster_flow_smem() bytes
    const double need = 1.05 * (double)est_pair_vertices * (29.0 + (w.narrow ? 16.0 : 20.0) * avg_degree);
    const double per_cta = 0.95 * (double)cluster_flow_smem();
    // Among the sizes that hold the estimate, the one with the least expected time:
    // waves of resident clusters times the relative time of one pair, measured on
    // 3D rgg / grid pairs (a pair's time falls slowly with more CTAs: its steps are
    // bound by barriers and latency).  Many pairs favour small clusters, few pairs
    // large ones.
    static const double kRelTime[fr_ctx::kNumClusterSizes] = {1.25, 1.05, 1.0, 0.85, 0.74};
    int t0 = -1, tmax = -1;
    double best = 0;
    const int P = std::max(1, w.npairs);
    for (int t = 0; t < T; ++t) {
        if (ctx->cl_cap[t] <= 0) continue;
        tmax = t;
        const int c = fr_ctx::kClusterSizes[t];
        if (force) {
            if (force == c && t0 < 0) t0 = t;
            continue;
        }
        if (need > per_cta * c) continue;
        const double cost = (double)((P + ctx->cl_cap[t] - 1) / ctx->cl_cap[t]) * kRelTime[t];
        if (t0 < 0 || cost < best) { t0 = t; best = cost; }
    }
    if (t0 < 0) t0 = tmax;   // nothing fits the estimate (or the forced size is unavailable)
    if (t0 < 0) return cudaErrorInvalidValue;
    w.cl_tier = 0;
    cudaError_t e = launch_cluster_flow(w, fr_ctx::kClusterSizes[t0], ctx->cl_cap[t0], st);
    if (e != cudaSuccess) return e;
    ++*nl;
    if (t0 < tmax) {
        w.cl_tier = 1;
        e = launch_cluster_flow(w, fr_ctx::kClusterSizes[tmax], ctx->cl_cap[tmax], st);
        w.cl_tier = 0;
        if (e != cudaSuccess) return e;
        ++*nl;
    }
    return cudaSuccess;
}

cudaError_t launch_round(fr_ctx *ctx, Work &w, int grid, int tpb, cudaStream_t st, cudaEvent_t *ev,
                         long long est_pair_vertices, double avg_degree, int cluster_ctas) {
    // ev (optional): 6 events bracketing step 1, the cluster kernels and step 2
    if (ctx->max_clusters <= 0) {
        w.cluster_mode = 0;
        if (ev) cudaEventRecord(ev[0], st);
        cudaError_t e = launch_step(w, PH_ALL, grid, tpb, st);
        if (ev) {
            cudaEventRecord(ev[1], st);
            for (int i = 2; i < 6; ++i) cudaEventRecord(ev[i], st);
        }
        ctx->round_launches = 1;
        return e;
    }
    w.cluster_mode = 1;
    if (ev) cudaEventRecord(ev[0], st);
    cudaError_t e = launch_step(w, PH_BFS | PH_LID | PH_BUILD, grid, tpb, st);
    if (ev) cudaEventRecord(ev[1], st);
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[2], st);
    int nl = 0;
    e = launch_clusters(ctx, w, est_pair_vertices, avg_degree, cluster_ctas, st, &nl);
    if (ev) cudaEventRecord(ev[3], st);
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[4], st);
    e = launch_step(w, PH_FLOW | PH_CUT | PH_EVAL | PH_COMMIT, grid, tpb, st);
    if (ev) cudaEventRecord(ev[5], st);
    ctx->round_launches = 2 + nl;
    return e;
}

// ------------------------------------------------------------ one pair ------

struct IterOut {
    long long flow, oldcut, newcut, cA, cB, nA, nB;
    int nc, m, accept, feasible;
    Ctl ctl;
};

static fr_status run_pair_iteration(fr_ctx *ctx, const fr_graph *g, int32_t *part, int32_t k, int32_t a, int32_t b,
                                    long long Ubase, long long Lmax, long long W, const fr_options *opt,
                                    IterOut *o) {
    const int mb = opt && opt->mb ? 1 : 0;
    fr_status st = setup_single(ctx, g, part, k, a, b, Ubase, Lmax, mb);
    if (st != FR_OK) return st;
    Work w = make_work(ctx, 0, 0, 1, g->n, opt);
    const int tpb = choose_tpb(ctx, opt);
    // corridor estimate: two sides of about (Ubase - W/k) weight each
    const double avgc = std::max(1.0, (double)W / g->n);
    const long long est = std::max<long long>(1, (long long)(2.0 * std::max(0LL, Ubase - W / k) / avgc));
    const int grid = choose_grid(ctx, opt, tpb, 2, est);
    CK(launch_scan_list(w, 0, ctx->stream));
    CK(launch_round(ctx, w, grid, tpb, ctx->stream, nullptr, est, (double)g->nnz / g->n,
                    opt && opt->cluster_ctas ? opt->cluster_ctas : ctx->tune_ctas));
    char *h = ctx->h_stage + 2048;
    CK(cudaMemcpyAsync(h, ctx->pacc, sizeof(PairAcc), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(h + 512, ctx->sides, 2 * sizeof(SideDev), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(h + 1024, ctx->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const PairAcc &A = *reinterpret_cast<PairAcc *>(h);
    const SideDev *S = reinterpret_cast<SideDev *>(h + 512);
    o->ctl = *reinterpret_cast<Ctl *>(h + 1024);
    st = status_from_ctl(ctx, o->ctl, "fr_refine_pair");
    if (st != FR_OK) {
        reset_idle(ctx);
        return st;
    }
    o->flow = A.flow;
    o->oldcut = A.oldcut;
    o->newcut = A.oldcut + A.dcut;
    o->cA = S[0].cw;
    o->cB = S[1].cw;
    o->nA = S[0].cw + A.dwA;
    o->nB = S[1].cw - A.dwA;
    o->nc = A.nc;
    o->m = A.m;
    o->accept = A.accept;
    o->feasible = A.feasible;
    return FR_OK;
}

extern "C" fr_status fr_refine_pair(fr_ctx *ctx, const fr_graph *g, int32_t *part, int32_t k, int32_t a,
                                    int32_t b, double eps, double alpha, const fr_options *opt_in,
                                    fr_pair_result *res) {
    if (!ctx) return FR_ERR_INVALID_ARG;
    fr_options opt;
    if (opt_in) opt = *opt_in; else fr_default_options(&opt);
    if (res) memset(res, 0, sizeof(*res));
    fr_status st = check_graph(ctx, g, part, k);
    if (st == FR_OK) st = check_params(ctx, eps, alpha, &opt);
    if (st == FR_OK && opt.mt_alpha != 0) { ctx_error(ctx, "mt_alpha: fr_refine_active only"); st = FR_ERR_INVALID_ARG; }
    if (st == FR_OK && (a < 0 || b < 0 || a >= k || b >= k || a == b)) {
        ctx_error(ctx, "pair (%d, %d) invalid for k=%d", a, b, k);
        st = FR_ERR_INVALID_ARG;
    }
    if (st != FR_OK) { if (res) res->status = st; return st; }
    CK(cudaSetDevice(ctx->device));
    release_corridor(ctx);
    st = ensure_base(ctx, g->n, g->nnz, k, opt.mb_reps);
    if (st == FR_OK) st = ensure_pairs(ctx, 1, 1, opt.mb_reps);
    PrepOut po;
    if (st == FR_OK) st = run_prep(ctx, g, part, k, false, opt.checked != 0, &po);
    if (st != FR_OK) { if (res) res->status = st; return st; }
    // part as it came: the FM step or an accepted iteration may write it before a later
    // step fails, and an error must leave it unchanged
    CK(cudaMemcpyAsync(ctx->part_backup, part, sizeof(int) * (size_t)g->n, cudaMemcpyDeviceToDevice, ctx->stream));
    const long long W = po.W;
    const long long Lmax = host_lmax(W, po.maxc, k, eps);
    const int adaptive = opt.adaptive ? 1 : 0;
    const int max_iters = adaptive ? (opt.max_iters > 0 ? opt.max_iters : 10) : 1;
    const double alpha_max = adaptive ? opt.alpha_max : alpha;
    double al = alpha;
    int iters = 0, accepted = 0;
    IterOut o;
    memset(&o, 0, sizeof(o));
    long long cut_before = -1, wA0 = 0, wB0 = 0, cur_cut = 0, cur_A = 0, cur_B = 0;
    long long pulses = 0, relabels = 0;
    int levels = 0, sccr = 0;
    // pairwise improvement: the FM step first (once), then the flow iterations on its result
    FmRes fres;
    memset(&fres, 0, sizeof(fres));
    const bool fm_on = opt.fm_permille > 0;
    if (fm_on) {
        st = ensure_fm(ctx, g->n, g->nnz, k, 1);
        if (st == FR_OK) st = setup_single(ctx, g, part, k, a, b, host_budget_base(W, k, eps, al), Lmax, opt.mb ? 1 : 0);
        if (st == FR_OK) {
            Work w = make_work(ctx, 0, 0, 1, g->n, &opt);
            int nf = 0;
            CK(launch_fm(w, fm_view(ctx, 0, &opt), k, ctx->sms, ctx->stream, &nf));
            Ctl c;
            CK(cudaMemcpyAsync(ctx->h_stage + 2048, ctx->fm.res, sizeof(FmRes), cudaMemcpyDeviceToHost, ctx->stream));
            CK(cudaMemcpyAsync(ctx->h_stage + 4096, ctx->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
            memcpy(&fres, ctx->h_stage + 2048, sizeof(FmRes));
            memcpy(&c, ctx->h_stage + 4096, sizeof(Ctl));
            st = status_from_ctl(ctx, c, "fr_refine_pair (FM)");
        }
        if (st != FR_OK) {
            cudaMemcpyAsync(part, ctx->part_backup, sizeof(int) * (size_t)g->n, cudaMemcpyDeviceToDevice, ctx->stream);
            cudaStreamSynchronize(ctx->stream);
            if (res) res->status = st;
            return st;
        }
    }
    while (iters < max_iters) {
        ++iters;
        st = run_pair_iteration(ctx, g, part, k, a, b, host_budget_base(W, k, eps, al), Lmax, W, &opt, &o);
        if (st != FR_OK) break;
        if (cut_before < 0) { cut_before = o.oldcut; wA0 = o.cA; wB0 = o.cB; }
        cur_cut = o.oldcut; cur_A = o.cA; cur_B = o.cB;
        pulses = o.ctl.pulses; relabels = o.ctl.relabels; levels = o.ctl.levels; sccr = o.ctl.scc_rounds;
        if (o.accept) { cur_cut = o.newcut; cur_A = o.nA; cur_B = o.nB; accepted = 1; }
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
        // a later iteration failed after an earlier one was applied: undo everything
        cudaError_t e = cudaMemcpyAsync(part, ctx->part_backup, sizeof(int) * (size_t)g->n, cudaMemcpyDeviceToDevice,
                                        ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) st = cuda_fail(ctx, e, "restoring part");
        accepted = 0;
        cur_cut = cut_before < 0 ? 0 : cut_before; cur_A = wA0; cur_B = wB0;
    }
    if (res) {
        res->status = st;
        res->a = a; res->b = b; res->round = 0;
        res->iters = iters;
        res->alpha_final = al;
        res->flow = o.flow;
        res->cut_before = cut_before < 0 ? 0 : cut_before;
        res->wA_before = wA0; res->wB_before = wB0;
        res->cut_fm = res->cut_before;
        if (fm_on) {
            res->cut_before = fres.cut0;
            res->wA_before = fres.wA0; res->wB_before = fres.wB0;
            res->cut_fm = fres.cut1;
            res->fm_moves = fres.kept;
        }
        res->cut_after = cur_cut; res->wA_after = cur_A; res->wB_after = cur_B;
        res->corridor_n = o.nc; res->corridor_arcs = o.m;
        res->accepted = accepted;
        res->pulses = pulses; res->relabels = relabels; res->bfs_levels = levels; res->scc_rounds = sccr;
    }
    return st;
}
