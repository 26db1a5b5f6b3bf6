// C ABI, part 4: multi-try FM passes (Sanders & Schulz, Section 4.2; k-way local
// search with the KaSPar stopping rule of Section 2.2): the workspace, one pass over
// the pairs of a matching (used by fr_refine_active after each matching), the
// stand-alone entry point fr_multitry, and the global k-way rounds (fr_kway_global).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>

#include "api_internal.h"

using namespace fr;

#define CK(call)                                                 \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

namespace {

template <typename T>
T *carve_mt(char *&p, long long count) {
    T *r = reinterpret_cast<T *>(p);
    p += ((sizeof(T) * (size_t)count + 255) / 256) * 256;
    return r;
}

}  // namespace

fr_status ensure_mt(fr_ctx *ctx, int n, int nnz, int k, int P) {
    if (ctx->mt_mem && n <= ctx->mt_n && nnz <= ctx->mt_nnz && k <= ctx->mt_k && P <= ctx->mt_p) return FR_OK;
    const long long nn = std::max(n, ctx->mt_n), mm = std::max(nnz, ctx->mt_nnz);
    const int kk = std::max(k, ctx->mt_k), pp = std::max(P, ctx->mt_p);
    // queue entries of one search: its start set (<= max degree + 1) plus one per arc of
    // a moved vertex; todo lists: each padded to a power of two (< 2 x its length, 1 if empty)
    const long long ecap = nn + mm + 64, scap = 2 * nn + pp;
    if (ecap > INT_MAX) {
        ctx_error(ctx, "multi-try: n + nnz exceeds the entry index range");
        return FR_ERR_TOO_LARGE;
    }
    size_t b = 0;
    auto add = [&](size_t elem, long long cnt) { b += ((elem * (size_t)cnt + 255) / 256) * 256; };
    add(4, nn); add(8, nn); add(4, 1); add(1, nn);      // tch cur epoch mvd
    add(16, nn); add(4, nn);                            // lmv kept
    const long long kwch = (nn + kKwChunk - 1) / kKwChunk + 1;
    add(4, (2 * kwch + 1) * kMtBuckets);                // kwtab
    add(32, ecap);                                      // ent (two int4 per entry)
    add(4, kk);                                         // bpair
    add(4, pp); add(4, pp); add(4, pp); add(4, pp);     // pa pb cnt fil
    add(8, pp + 1);                                     // off
    add(8, scap); add(4, scap);                         // tkey tv
    add(8, kk); add(1, kk);                             // bw chg
    add(sizeof(MtRes), 1);                              // res
    if (ctx->arena_limit && b + ctx->base_bytes + ctx->pair_bytes + ctx->fm_bytes > ctx->arena_limit) {
        ctx_error(ctx, "multi-try workspace of %zu bytes exceeds the arena bound", b);
        return FR_ERR_OOM;
    }
    free_mt(ctx);
    if (cudaMalloc(&ctx->mt_mem, b) != cudaSuccess) {
        ctx->mt_mem = nullptr;
        cudaGetLastError();
        ctx_error(ctx, "cudaMalloc(%zu) for the multi-try workspace failed", b);
        return FR_ERR_OOM;
    }
    ctx->mt_bytes = b;
    ctx->mt_n = (int)nn; ctx->mt_nnz = (int)mm; ctx->mt_k = kk; ctx->mt_p = pp;
    char *p = reinterpret_cast<char *>(ctx->mt_mem);
    MtDev &m = ctx->mt;
    m.tch = carve_mt<int>(p, nn); m.cur = carve_mt<unsigned long long>(p, nn); m.epoch = carve_mt<unsigned>(p, 1);
    m.mvd = carve_mt<unsigned char>(p, nn);
    m.lmv = carve_mt<int4>(p, nn); m.kept = carve_mt<int>(p, nn);
    m.kwtab = carve_mt<int>(p, (2 * kwch + 1) * kMtBuckets);
    m.kwchunks = (int)kwch;
    m.ent = carve_mt<int4>(p, 2 * ecap);
    m.bpair = carve_mt<int>(p, kk);
    m.pa = carve_mt<int>(p, pp); m.pb = carve_mt<int>(p, pp); m.cnt = carve_mt<int>(p, pp); m.fil = carve_mt<int>(p, pp);
    m.off = carve_mt<long long>(p, pp + 1);
    m.tkey = carve_mt<unsigned long long>(p, scap); m.tv = carve_mt<int>(p, scap);
    m.bw = carve_mt<long long>(p, kk); m.chg = carve_mt<unsigned char>(p, kk);
    m.res = carve_mt<MtRes>(p, 1);
    m.ecap = ecap; m.scap = scap;
    // versions start at zero; the moved marks are zero between searches
    CK(cudaMemsetAsync(m.cur, 0, sizeof(unsigned long long) * (size_t)nn, ctx->stream));
    CK(cudaMemsetAsync(m.epoch, 0, sizeof(unsigned), ctx->stream));
    CK(cudaMemsetAsync(m.mvd, 0, (size_t)nn, ctx->stream));
    return FR_OK;
}

void free_mt(fr_ctx *ctx) {
    if (ctx->mt_mem) cudaFree(ctx->mt_mem);
    ctx->mt_mem = nullptr;
    ctx->mt_bytes = 0;
    ctx->mt_n = ctx->mt_nnz = ctx->mt_k = ctx->mt_p = 0;
    ctx->mt = MtDev{};
}

fr_status run_mt_pass(fr_ctx *ctx, const fr_graph *g, int32_t *part, int32_t k, const int32_t *pa, const int32_t *pb,
                      int np, long long Lmax, int alpha, unsigned long long seed, bool bl_on, MtRes *out,
                      int8_t *changed) {
    memset(out, 0, sizeof(*out));
    if (np <= 0) return FR_OK;
    if (k > kMtMaxK) {
        ctx_error(ctx, "multi-try: k = %d exceeds %d", k, kMtMaxK);
        return FR_ERR_TOO_LARGE;
    }
    fr_status st = ensure_mt(ctx, g->n, g->nnz, k, np);
    if (st == FR_OK && !ctx->ctl) st = ensure_pairs(ctx, 1, 1, 1);   // the control block lives there
    if (st != FR_OK) return st;
    MtDev md = ctx->mt;
    // staging: pairs and the block -> pair map
    int *h = reinterpret_cast<int *>(ctx->h_stage + 4096);
    if (4096 + sizeof(int) * (size_t)(2 * np + k) > kHostStage / 2) {
        ctx_error(ctx, "multi-try: %d pairs / k = %d exceed the staging buffer", np, k);
        return FR_ERR_TOO_LARGE;
    }
    int *hb = h + 2 * np;
    for (int x = 0; x < k; ++x) hb[x] = -1;
    for (int i = 0; i < np; ++i) {
        if (pa[i] < 0 || pb[i] < 0 || pa[i] >= k || pb[i] >= k || pa[i] == pb[i] || hb[pa[i]] >= 0 ||
            hb[pb[i]] >= 0) {
            ctx_error(ctx, "multi-try: pairs must be valid and block-disjoint");
            return FR_ERR_INVALID_ARG;
        }
        h[i] = pa[i];
        h[np + i] = pb[i];
        hb[pa[i]] = hb[pb[i]] = i;
    }
    CK(cudaMemcpyAsync(md.pa, h, sizeof(int) * (size_t)np, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(md.pb, h + np, sizeof(int) * (size_t)np, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(md.bpair, hb, sizeof(int) * (size_t)k, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemsetAsync(ctx->ctl, 0, sizeof(Ctl), ctx->stream));
    md.np = np;
    md.alpha = alpha;
    md.beta = std::log((double)g->n);
    md.seed = seed;
    GraphDev G;
    memset(&G, 0, sizeof(G));
    G.xadj = g->xadj; G.adjncy = g->adjncy; G.adjwgt = g->adjwgt; G.vwgt = g->vwgt;
    G.part = part; G.blockw = ctx->blockw;
    G.n = g->n; G.nnz = g->nnz; G.k = k; G.Lmax = Lmax;
    if (bl_on) { G.bl = ctx->bl; G.blc = ctx->blc; G.inb = ctx->inb; }
    int nl = 0;
    CK(launch_mt(G, md, ctx->ctl, ctx->sms, ctx->stream, &nl));
    ctx->last_launches += nl;
    char *o = ctx->h_stage + kHostStage / 2;
    Ctl *hc = reinterpret_cast<Ctl *>(o);
    MtRes *hr = reinterpret_cast<MtRes *>(o + 1024);
    unsigned char *hchg = reinterpret_cast<unsigned char *>(o + 2048);
    CK(cudaMemcpyAsync(hc, ctx->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(hr, md.res, sizeof(MtRes), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(hchg, md.chg, (size_t)k, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    st = status_from_ctl(ctx, *hc, "multi-try pass");
    if (st != FR_OK) {
        reset_idle(ctx);
        return st;
    }
    *out = *hr;
    if (changed)
        for (int x = 0; x < k; ++x) changed[x] = hchg[x] ? 1 : 0;
    return FR_OK;
}

extern "C" fr_status fr_multitry(fr_ctx *ctx, const fr_graph *g, int32_t *part, int32_t k, double eps, int32_t np,
                                 const int32_t *pa, const int32_t *pb, int32_t alpha, uint64_t seed,
                                 fr_mt_result *out, int8_t *changed) {
    if (!ctx) return FR_ERR_INVALID_ARG;
    if (out) memset(out, 0, sizeof(*out));
    fr_status st = check_graph(ctx, g, part, k);
    if (st == FR_OK && (!(eps > 0.0) || !std::isfinite(eps) || alpha < 0 || np < 0 || (np > 0 && (!pa || !pb)))) {
        ctx_error(ctx, "fr_multitry: eps > 0, alpha >= 0 and np pairs needed");
        st = FR_ERR_INVALID_ARG;
    }
    if (st != FR_OK) { if (out) out->status = st; return st; }
    CK(cudaSetDevice(ctx->device));
    release_corridor(ctx);
    ctx->last_launches = 0;
    st = ensure_base(ctx, g->n, g->nnz, k, 1);
    PrepOut po;
    if (st == FR_OK) st = run_prep(ctx, g, part, k, false, false, &po);
    if (st == FR_OK && po.maxwdeg > kMtGmax) {
        ctx_error(ctx, "multi-try: max weighted degree %d exceeds %d", po.maxwdeg, kMtGmax);
        st = FR_ERR_TOO_LARGE;
    }
    if (st != FR_OK) { if (out) out->status = st; return st; }
    CK(cudaMemcpyAsync(ctx->part_backup, part, sizeof(int) * (size_t)g->n, cudaMemcpyDeviceToDevice, ctx->stream));
    MtRes r;
    st = run_mt_pass(ctx, g, part, k, pa, pb, np, host_lmax(po.W, po.maxc, k, eps), alpha, seed, true, &r, changed);
    if (st != FR_OK) {
        cudaMemcpyAsync(part, ctx->part_backup, sizeof(int) * (size_t)g->n, cudaMemcpyDeviceToDevice, ctx->stream);
        cudaStreamSynchronize(ctx->stream);
        if (out) out->status = st;
        return st;
    }
    if (out) {
        out->gain = r.gain;
        out->searches = r.searches;
        out->tried = r.tried;
        out->kept = r.kept;
        out->status = FR_OK;
    }
    return FR_OK;
}

extern "C" fr_status fr_kway_global(fr_ctx *ctx, const fr_graph *g, int32_t *part, int32_t k, double eps,
                                    int32_t init_mode, int32_t alpha, int32_t max_rounds, uint64_t seed,
                                    fr_mt_result *out) {
    if (!ctx) return FR_ERR_INVALID_ARG;
    if (out) memset(out, 0, sizeof(*out));
    fr_status st = check_graph(ctx, g, part, k);
    if (st == FR_OK && (!(eps > 0.0) || !std::isfinite(eps) || alpha < 0 || max_rounds < 1 ||
                        (init_mode != 0 && init_mode != 1))) {
        ctx_error(ctx, "fr_kway_global: eps > 0, alpha >= 0, max_rounds >= 1 and init_mode 0 or 1 needed");
        st = FR_ERR_INVALID_ARG;
    }
    if (st == FR_OK && k > kMtMaxK) {
        ctx_error(ctx, "k-way rounds: k = %d exceeds %d", k, kMtMaxK);
        st = FR_ERR_TOO_LARGE;
    }
    if (st != FR_OK) { if (out) out->status = st; return st; }
    CK(cudaSetDevice(ctx->device));
    release_corridor(ctx);
    ctx->last_launches = 0;
    st = ensure_base(ctx, g->n, g->nnz, k, 1);
    PrepOut po;
    if (st == FR_OK) st = run_prep(ctx, g, part, k, false, false, &po);
    if (st == FR_OK && po.maxwdeg > kMtGmax) {
        ctx_error(ctx, "k-way rounds: max weighted degree %d exceeds %d", po.maxwdeg, kMtGmax);
        st = FR_ERR_TOO_LARGE;
    }
    if (st == FR_OK) st = ensure_mt(ctx, g->n, g->nnz, k, 1);
    if (st == FR_OK && !ctx->ctl) st = ensure_pairs(ctx, 1, 1, 1);   // the control block lives there
    if (st != FR_OK) { if (out) out->status = st; return st; }
    CK(cudaMemcpyAsync(ctx->part_backup, part, sizeof(int) * (size_t)g->n, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemsetAsync(ctx->ctl, 0, sizeof(Ctl), ctx->stream));
    MtDev md = ctx->mt;
    md.np = 0;
    md.alpha = alpha;
    md.beta = std::log((double)g->n);
    md.seed = seed;
    GraphDev G;
    memset(&G, 0, sizeof(G));
    G.xadj = g->xadj; G.adjncy = g->adjncy; G.adjwgt = g->adjwgt; G.vwgt = g->vwgt;
    G.part = part; G.blockw = ctx->blockw;
    G.n = g->n; G.nnz = g->nnz; G.k = k; G.Lmax = host_lmax(po.W, po.maxc, k, eps);
    char *o = ctx->h_stage + kHostStage / 2;
    Ctl *hc = reinterpret_cast<Ctl *>(o);
    MtRes *hr = reinterpret_cast<MtRes *>(o + 1024);
    fr_mt_result tot;
    memset(&tot, 0, sizeof(tot));
    for (int r = 0; r < max_rounds; ++r) {
        int nl = 0;
        const unsigned long long rs = splitmix64(seed ^ (unsigned long long)(unsigned)r);
        cudaError_t e = launch_kway_round(G, md, ctx->ctl, init_mode == 1 ? 2 : 1, rs, ctx->sms, ctx->stream, &nl);
        ctx->last_launches += nl;
        if (e == cudaSuccess) e = cudaMemcpyAsync(hc, ctx->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hr, md.res, sizeof(MtRes), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        st = e == cudaSuccess ? status_from_ctl(ctx, *hc, "k-way round") : cuda_fail(ctx, e, "k-way round");
        if (st != FR_OK) {
            reset_idle(ctx);
            cudaMemcpyAsync(part, ctx->part_backup, sizeof(int) * (size_t)g->n, cudaMemcpyDeviceToDevice,
                            ctx->stream);
            cudaStreamSynchronize(ctx->stream);
            if (out) out->status = st;
            return st;
        }
        tot.gain += hr->gain;
        tot.tried += hr->tried;
        tot.kept += hr->kept;
        tot.searches = r + 1;
        if (hr->gain <= 0) break;
    }
    if (out) {
        *out = tot;
        out->status = FR_OK;
    }
    return FR_OK;
}
