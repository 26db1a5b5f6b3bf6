// C ABI, part 2: the corridor / max-flow / cut steps on one pair, the batched
// sweep over the rounds of the quotient graph, its host-buffer form, and the
// launch-shape autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <vector>

#include "api_internal.h"

using namespace fr;

#define CK(call)                                                 \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

// ------------------------------------------------------------ corridor handle --

static fr_status cleanup_launch(fr_ctx *ctx) {
    // releases dist / lid of the live corridor (commit phase with nothing accepted)
    fr_options opt;
    fr_default_options(&opt);
    Work w = make_work(ctx, 0, 0, 1, ctx->live ? ctx->live->g.n : 0, &opt);
    CK(cudaMemsetAsync(&ctx->pacc[0].accept, 0, sizeof(int), ctx->stream));
    CK(launch_step(w, PH_COMMIT, 1, 256, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return FR_OK;
}

void release_corridor(fr_ctx *ctx) {
    if (ctx->dirty && ctx->live) {
        if (cleanup_launch(ctx) != FR_OK) reset_idle(ctx);
    }
    ctx->dirty = false;
    ctx->live = nullptr;
    ++ctx->gen;
}

void destroy_graph_cache(fr_ctx *ctx) {
    for (auto &e : ctx->gcache)
        if (e.exec) cudaGraphExecDestroy(e.exec);
    ctx->gcache.clear();
}

static fr_status check_handle(fr_ctx *ctx, const fr_corridor *c, int stage_min) {
    if (!ctx || !c || c->ctx != ctx || c->gen != ctx->gen || ctx->live != c) {
        if (ctx) ctx_error(ctx, "stale or foreign corridor handle");
        return FR_ERR_INVALID_ARG;
    }
    if (c->stage < stage_min) {
        ctx_error(ctx, "corridor step called out of order");
        return FR_ERR_INVALID_ARG;
    }
    return FR_OK;
}

static fr_status read_step(fr_ctx *ctx, PairAcc *A, SideDev *S, Ctl *C) {
    char *h = ctx->h_stage + 4096;
    CK(cudaMemcpyAsync(h, ctx->pacc, sizeof(PairAcc), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(h + 512, ctx->sides, 2 * sizeof(SideDev), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(h + 1024, ctx->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (A) *A = *reinterpret_cast<PairAcc *>(h);
    if (S) memcpy(S, h + 512, 2 * sizeof(SideDev));
    if (C) *C = *reinterpret_cast<Ctl *>(h + 1024);
    return FR_OK;
}

extern "C" fr_status fr_build_corridor(fr_ctx *ctx, const fr_graph *g, const int32_t *part, int32_t k, int32_t a,
                                       int32_t b, double eps, double alpha, fr_corridor **out) {
    if (!ctx || !out) return FR_ERR_INVALID_ARG;
    *out = nullptr;
    fr_status st = check_graph(ctx, g, part, k);
    if (st == FR_OK) st = check_params(ctx, eps, alpha, nullptr);
    if (st == FR_OK && (a < 0 || b < 0 || a >= k || b >= k || a == b)) {
        ctx_error(ctx, "pair (%d, %d) invalid for k=%d", a, b, k);
        st = FR_ERR_INVALID_ARG;
    }
    if (st != FR_OK) return st;
    CK(cudaSetDevice(ctx->device));
    release_corridor(ctx);
    if ((st = ensure_base(ctx, g->n, g->nnz, k, 1)) != FR_OK) return st;
    if ((st = ensure_pairs(ctx, 1, 1, 1)) != FR_OK) return st;
    PrepOut po;
    if ((st = run_prep(ctx, g, part, k, false, false, &po)) != FR_OK) return st;
    const long long Ubase = host_budget_base(po.W, k, eps, alpha);
    const long long Lmax = host_lmax(po.W, po.maxc, k, eps);
    int32_t *mpart = const_cast<int32_t *>(part);
    if ((st = setup_single(ctx, g, mpart, k, a, b, Ubase, Lmax, 0)) != FR_OK) return st;
    fr_options opt;
    fr_default_options(&opt);
    Work w = make_work(ctx, 0, 0, 1, g->n, &opt);
    const int tpb = choose_tpb(ctx, &opt);
    const int grid = choose_grid(ctx, &opt, tpb, 2, std::max<long long>(1, 2 * Ubase));
    CK(launch_scan_list(w, 0, ctx->stream));
    CK(launch_step(w, PH_BFS | PH_LID | PH_BUILD, grid, tpb, ctx->stream));
    PairAcc A;
    Ctl C;
    if ((st = read_step(ctx, &A, nullptr, &C)) != FR_OK) return st;
    ctx->dirty = true;
    if ((st = status_from_ctl(ctx, C, "fr_build_corridor")) != FR_OK) {
        reset_idle(ctx);
        ctx->dirty = false;
        return st;
    }
    fr_corridor *c = new fr_corridor();
    c->ctx = ctx;
    c->gen = ctx->gen;
    c->nc = A.nc;
    c->m = A.m;
    c->k = k; c->a = a; c->b = b;
    c->stage = 1;
    c->part = mpart;
    c->g = *g;
    c->Ubase = Ubase;
    c->Lmax = Lmax;
    ctx->live = c;
    *out = c;
    return FR_OK;
}

extern "C" fr_status fr_corridor_info(const fr_corridor *c, int32_t *nc, int32_t *m) {
    if (!c) return FR_ERR_INVALID_ARG;
    if (nc) *nc = c->nc;
    if (m) *m = c->m;
    return FR_OK;
}

extern "C" fr_status fr_corridor_export(fr_ctx *ctx, const fr_corridor *c, int32_t *gid, int32_t *off,
                                        int32_t *head, int32_t *cap, int8_t *border, int32_t *infcap, int8_t *side0,
                                        int32_t *dist) {
    fr_status st = check_handle(ctx, c, 1);
    if (st != FR_OK) return st;
    if (c->stage >= 3 && dist) {
        ctx_error(ctx, "BFS distances are released by fr_extract_cut");
        return FR_ERR_INVALID_ARG;
    }
    const int nc = c->nc, m = c->m;
    if (gid) CK(cudaMemcpyAsync(gid, ctx->gid, sizeof(int) * nc, cudaMemcpyDeviceToHost, ctx->stream));
    if (off) CK(cudaMemcpyAsync(off, ctx->off, sizeof(int) * (nc + 1), cudaMemcpyDeviceToHost, ctx->stream));
    if (head) CK(cudaMemcpyAsync(head, ctx->head, sizeof(int) * m, cudaMemcpyDeviceToHost, ctx->stream));
    if (cap) CK(cudaMemcpyAsync(cap, ctx->cap, sizeof(int) * m, cudaMemcpyDeviceToHost, ctx->stream));
    std::vector<unsigned char> bd(nc);
    std::vector<int> inf(nc), sid(nc);
    CK(cudaMemcpyAsync(bd.data(), ctx->border, nc, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(inf.data(), ctx->infc, sizeof(int) * nc, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(sid.data(), ctx->sid, sizeof(int) * nc, cudaMemcpyDeviceToHost, ctx->stream));
    if (dist) {
        CK(launch_gather(ctx->spare, ctx->dist, ctx->gid, nc, ctx->stream));
        CK(cudaMemcpyAsync(dist, ctx->spare, sizeof(int) * nc, cudaMemcpyDeviceToHost, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < nc; ++i) {
        if (border) border[i] = (int8_t)bd[i];
        if (infcap) infcap[i] = bd[i] ? inf[i] : 0;
        if (side0) side0[i] = (int8_t)(sid[i] & 1);
    }
    return FR_OK;
}

extern "C" fr_status fr_maxflow(fr_ctx *ctx, fr_corridor *c, int64_t *flow_out) {
    fr_status st = check_handle(ctx, c, 1);
    if (st != FR_OK) return st;
    if (c->stage != 1) {
        ctx_error(ctx, "fr_maxflow runs once per corridor");
        return FR_ERR_INVALID_ARG;
    }
    fr_options opt;
    fr_default_options(&opt);
    Work w = make_work(ctx, 0, 0, 1, c->g.n, &opt);
    w.full_flow = 1;   // fr_corridor_flow hands out the arc flows
    const int tpb = choose_tpb(ctx, &opt);
    const int grid = choose_grid(ctx, &opt, tpb, 2, std::max(1, c->nc));
    if (ctx->max_clusters > 0) {
        w.cluster_mode = 1;
        int nl = 0;
        CK(launch_clusters(ctx, w, c->nc, (double)c->m / std::max(1, c->nc), 0, ctx->stream, &nl));
    }
    CK(launch_step(w, PH_FLOW, grid, tpb, ctx->stream));
    PairAcc A;
    Ctl C;
    if ((st = read_step(ctx, &A, nullptr, &C)) != FR_OK) return st;
    if ((st = status_from_ctl(ctx, C, "fr_maxflow")) != FR_OK) return st;
    c->stage = 2;
    if (flow_out) *flow_out = A.flow;
    return FR_OK;
}

extern "C" fr_status fr_corridor_flow(fr_ctx *ctx, const fr_corridor *c, int64_t *arcflow, int64_t *stflow) {
    fr_status st = check_handle(ctx, c, 2);
    if (st != FR_OK) return st;
    const int nc = c->nc, m = c->m;
    std::vector<int> capv(m), resv(m), fxv(nc);
    std::vector<unsigned char> bd(nc);
    CK(cudaMemcpyAsync(capv.data(), ctx->cap, sizeof(int) * m, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(resv.data(), ctx->res, sizeof(int) * m, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(fxv.data(), ctx->fx, sizeof(int) * nc, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(bd.data(), ctx->border, nc, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (arcflow)
        for (int j = 0; j < m; ++j) arcflow[j] = (int64_t)capv[j] - resv[j];
    if (stflow)
        for (int i = 0; i < nc; ++i) stflow[i] = bd[i] ? fxv[i] : 0;
    return FR_OK;
}

extern "C" fr_status fr_extract_cut(fr_ctx *ctx, fr_corridor *c, int32_t most_balanced, int32_t mb_reps,
                                    uint64_t seed, int32_t *part, fr_pair_result *res) {
    fr_status st = check_handle(ctx, c, 2);
    if (st != FR_OK) return st;
    if (c->stage != 2 || part != c->part || mb_reps < 0 || mb_reps > 64) {
        ctx_error(ctx, "fr_extract_cut needs the flow of this corridor, its own part array and 0 <= mb_reps <= 64");
        return FR_ERR_INVALID_ARG;
    }
    fr_options opt;
    fr_default_options(&opt);
    opt.mb = most_balanced ? 1 : 0;
    opt.mb_reps = mb_reps > 0 ? mb_reps : 1;
    opt.seed = seed;
    if ((st = ensure_reps(ctx, opt.mb_reps)) != FR_OK) return st;   // sweep arrays hold no corridor state
    int mbv = opt.mb;
    int *h = reinterpret_cast<int *>(ctx->h_stage + 8192);
    h[0] = mbv;
    CK(cudaMemcpyAsync(&ctx->pairs[0].mb, h, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    Work w = make_work(ctx, 0, 0, 1, c->g.n, &opt);
    // the cut kind is chosen only now: the residual sets and SCCs are computed here,
    // grid-wide, from the flow fr_maxflow left
    w.cluster_mode = 0;
    w.full_flow = 1;
    const int tpb = choose_tpb(ctx, &opt);
    const int grid = choose_grid(ctx, &opt, tpb, 2, std::max(1, c->nc));
    CK(launch_step(w, PH_CUT | PH_EVAL | PH_COMMIT, grid, tpb, ctx->stream));
    PairAcc A;
    SideDev S[2];
    Ctl C;
    if ((st = read_step(ctx, &A, S, &C)) != FR_OK) return st;
    ctx->dirty = false;
    c->stage = 3;
    st = status_from_ctl(ctx, C, "fr_extract_cut");
    if (st != FR_OK) reset_idle(ctx);
    if (res) {
        memset(res, 0, sizeof(*res));
        res->status = st;
        res->a = c->a; res->b = c->b;
        res->flow = A.flow;
        res->cut_before = A.oldcut;
        res->wA_before = S[0].cw; res->wB_before = S[1].cw;
        res->accepted = st == FR_OK ? A.accept : 0;
        res->cut_after = A.oldcut + (res->accepted ? A.dcut : 0);
        res->wA_after = S[0].cw + (res->accepted ? A.dwA : 0);
        res->wB_after = S[1].cw - (res->accepted ? A.dwA : 0);
        res->corridor_n = A.nc; res->corridor_arcs = A.m;
        res->iters = 1;
        res->alpha_final = 0.0;
        res->ncomp = A.ncomp;
        res->scc_rounds = C.scc_rounds;
    }
    return st;
}

extern "C" fr_status fr_corridor_sets(fr_ctx *ctx, const fr_corridor *c, int8_t *in_s, int8_t *to_t, int32_t *comp,
                                      int8_t *side) {
    fr_status st = check_handle(ctx, c, 3);
    if (st != FR_OK) return st;
    const int nc = c->nc;
    std::vector<int> rf(nc), sc(nc), gid(nc);
    std::vector<unsigned char> so(nc);
    CK(cudaMemcpyAsync(rf.data(), ctx->rflag, sizeof(int) * nc, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(sc.data(), ctx->scc, sizeof(int) * nc, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(gid.data(), ctx->gid, sizeof(int) * nc, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(so.data(), ctx->side_out, nc, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    int32_t mbflag = 0;
    CK(cudaMemcpy(&mbflag, &ctx->pairs[0].mb, sizeof(int), cudaMemcpyDeviceToHost));
    for (int i = 0; i < nc; ++i) {
        if (in_s) in_s[i] = (int8_t)(rf[i] & 1);
        if (to_t) to_t[i] = (int8_t)((rf[i] >> 1) & 1);
        if (comp) comp[i] = (mbflag && rf[i] == 0 && sc[i] >= 0) ? gid[sc[i]] : -1;
        if (side) side[i] = (int8_t)so[i];
    }
    return FR_OK;
}

extern "C" fr_status fr_corridor_free(fr_ctx *ctx, fr_corridor *c) {
    if (!ctx || !c) return FR_ERR_INVALID_ARG;
    if (ctx->live == c) release_corridor(ctx);
    delete c;
    return FR_OK;
}

// ---------------------------------------------------------------- rounds --

extern "C" fr_status fr_rounds(fr_ctx *ctx, const fr_graph *g, const int32_t *part, int32_t k, int32_t cap,
                               int32_t *pair_a, int32_t *pair_b, int32_t *pair_round, int32_t *npairs,
                               int32_t *nrounds) {
    if (!ctx) return FR_ERR_INVALID_ARG;
    fr_status st = check_graph(ctx, g, part, k);
    if (st != FR_OK) return st;
    CK(cudaSetDevice(ctx->device));
    release_corridor(ctx);
    if ((st = ensure_base(ctx, g->n, g->nnz, k, 1)) != FR_OK) return st;
    PrepOut po;
    if ((st = run_prep(ctx, g, part, k, true, false, &po)) != FR_OK) return st;
    const int c = std::min(cap, po.npairs);
    if (c > 0) {
        if (pair_a) CK(cudaMemcpyAsync(pair_a, ctx->pair_a, sizeof(int) * c, cudaMemcpyDeviceToHost, ctx->stream));
        if (pair_b) CK(cudaMemcpyAsync(pair_b, ctx->pair_b, sizeof(int) * c, cudaMemcpyDeviceToHost, ctx->stream));
        if (pair_round)
            CK(cudaMemcpyAsync(pair_round, ctx->pair_round, sizeof(int) * c, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    if (npairs) *npairs = po.npairs;
    if (nrounds) *nrounds = po.nrounds;
    return FR_OK;
}

// ---------------------------------------------------------------- batch --

// Enqueues a whole sweep: pair descriptors, cleared per-round state, then per
// round the boundary scan and the persistent step kernel.
static fr_status enqueue_sweep(fr_ctx *ctx, const fr_graph *g, const BatchPlan &pl, const fr_options *opt) {
    const int np = pl.np, nr = pl.nr;
    CK(launch_fill_pairs(ctx->pairs, ctx->pair_a, ctx->pair_b, np, 0, opt->mb ? 1 : 0, pl.Ubase, ctx->stream));
    CK(cudaMemsetAsync(ctx->ctl, 0, sizeof(Ctl) * nr, ctx->stream));
    CK(cudaMemsetAsync(ctx->sides, 0, sizeof(SideDev) * 2 * np, ctx->stream));
    CK(cudaMemsetAsync(ctx->pacc, 0, sizeof(PairAcc) * np, ctx->stream));
    CK(cudaMemsetAsync(ctx->hist, 0, sizeof(long long) * 3 * 2 * (size_t)np * kHistBins, ctx->stream));
    long long nl = 3;   // prep, colouring, pair fill
    for (int r = 0; r < nr; ++r) {
        const int P = pl.off[r + 1] - pl.off[r];
        Work w = make_work(ctx, r, pl.off[r], P, g->n, opt);
        if (opt->fm_permille > 0) {   // pairwise improvement: FM first, then the flow
            int nf = 0;
            CK(launch_fm(w, fm_view(ctx, pl.off[r], opt), pl.k, ctx->sms, ctx->stream, &nf));
            nl += nf;
        }
        CK(launch_scan_list(w, 0, ctx->stream));
        CK(launch_round(ctx, w, pl.grid[r], pl.tpb, ctx->stream, nullptr, pl.est_max[r], pl.avg_degree,
                        opt->cluster_ctas ? opt->cluster_ctas : ctx->tune_ctas));
        nl += 1 + ctx->round_launches;
    }
    ctx->sweep_launches = nl;
    return FR_OK;
}

// Same launches as enqueue_sweep, each bracketed by CUDA events (profiling mode).
static fr_status enqueue_sweep_profiled(fr_ctx *ctx, const fr_graph *g, const BatchPlan &pl, const fr_options *opt) {
    const int np = pl.np, nr = pl.nr;
    while ((int)ctx->pev.size() < 8 * nr) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        ctx->pev.push_back(e);
    }
    CK(launch_fill_pairs(ctx->pairs, ctx->pair_a, ctx->pair_b, np, 0, opt->mb ? 1 : 0, pl.Ubase, ctx->stream));
    CK(cudaMemsetAsync(ctx->ctl, 0, sizeof(Ctl) * nr, ctx->stream));
    CK(cudaMemsetAsync(ctx->sides, 0, sizeof(SideDev) * 2 * np, ctx->stream));
    CK(cudaMemsetAsync(ctx->pacc, 0, sizeof(PairAcc) * np, ctx->stream));
    CK(cudaMemsetAsync(ctx->hist, 0, sizeof(long long) * 3 * 2 * (size_t)np * kHistBins, ctx->stream));
    long long nl = 3;
    for (int r = 0; r < nr; ++r) {
        const int P = pl.off[r + 1] - pl.off[r];
        Work w = make_work(ctx, r, pl.off[r], P, g->n, opt);
        if (opt->fm_permille > 0) {   // (not bracketed: the profile's phases are the flow path's)
            int nf = 0;
            CK(launch_fm(w, fm_view(ctx, pl.off[r], opt), pl.k, ctx->sms, ctx->stream, &nf));
            nl += nf;
        }
        CK(cudaEventRecord(ctx->pev[8 * r], ctx->stream));
        CK(launch_scan_list(w, 0, ctx->stream));
        CK(cudaEventRecord(ctx->pev[8 * r + 1], ctx->stream));
        CK(launch_round(ctx, w, pl.grid[r], pl.tpb, ctx->stream, &ctx->pev[8 * r + 2], pl.est_max[r],
                        pl.avg_degree, opt->cluster_ctas ? opt->cluster_ctas : ctx->tune_ctas));
        nl += 1 + ctx->round_launches;
    }
    ctx->sweep_launches = nl;
    return FR_OK;
}

static fr_status run_sweep(fr_ctx *ctx, const fr_graph *g, int32_t *part, const BatchPlan &pl,
                           const fr_options *opt, float *ms) {
    // per-round graph descriptors (sob of round r) go up before the launches
    std::vector<GraphDev> gds(pl.nr);
    for (int r = 0; r < pl.nr; ++r) {
        GraphDev &gd = gds[r];
        memset(&gd, 0, sizeof(gd));
        gd.xadj = g->xadj; gd.adjncy = g->adjncy; gd.adjwgt = g->adjwgt; gd.vwgt = g->vwgt;
        gd.part = part; gd.dist = ctx->dist; gd.lid = ctx->lid;
        gd.sob = ctx->sob_round + (long long)r * pl.k;
        gd.blockw = ctx->blockw;
        gd.n = g->n; gd.nnz = g->nnz; gd.k = pl.k; gd.base = 0; gd.Lmax = pl.Lmax;
        gd.bl = ctx->bl; gd.blc = ctx->blc; gd.inb = ctx->inb;
    }
    memcpy(ctx->h_stage + 16384, gds.data(), sizeof(GraphDev) * pl.nr);
    CK(cudaMemcpyAsync(ctx->graphs, ctx->h_stage + 16384, sizeof(GraphDev) * pl.nr, cudaMemcpyHostToDevice,
                       ctx->stream));
    CK(cudaMemcpyAsync(ctx->part_backup, part, sizeof(int) * (size_t)g->n, cudaMemcpyDeviceToDevice, ctx->stream));
    // key of the captured sweep
    std::vector<long long> key = {(long long)(uintptr_t)g->xadj, (long long)(uintptr_t)part, g->n, g->nnz,
                                  pl.np, pl.nr, pl.tpb, pl.Ubase, opt->mb, opt->mb_reps, (long long)opt->seed,
                                  opt->gr_interval, opt->inner_ops, opt->pulse_cap, (long long)(uintptr_t)ctx->base_mem,
                                  (long long)(uintptr_t)ctx->pair_mem, ctx->tune_gr, ctx->tune_inner,
                                  opt->pulse_passes, ctx->tune_passes, (long long)(uintptr_t)ctx->reps_mem,
                                  opt->flow_sched, opt->cluster_ctas, ctx->tune_ctas, ctx->tune_sched,
                                  ctx->narrow_ok, opt->pre_waves, ctx->tune_prewaves, opt->fm_permille,
                                  opt->gap_interval,
                                  (long long)(uintptr_t)ctx->fm_mem};
    for (int r = 0; r <= pl.nr; ++r) key.push_back(pl.off[r]);
    for (int r = 0; r < pl.nr; ++r) key.push_back(pl.grid[r]);
    cudaGraphExec_t exec = nullptr;
    long long exec_launches = 0;
    if (ctx->profiling) {
        CK(cudaEventRecord(ctx->ev0, ctx->stream));
        fr_status st = enqueue_sweep_profiled(ctx, g, pl, opt);
        if (st != FR_OK) return st;
        CK(cudaEventRecord(ctx->ev1, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        CK(cudaEventElapsedTime(ms, ctx->ev0, ctx->ev1));
        double sc = 0, stp = 0, clu = 0;
        ctx->round_ms.assign(4 * (size_t)pl.nr, 0.f);
        for (int r = 0; r < pl.nr; ++r) {
            float a = 0, b1 = 0, c = 0, b2 = 0;
            CK(cudaEventElapsedTime(&a, ctx->pev[8 * r], ctx->pev[8 * r + 1]));
            CK(cudaEventElapsedTime(&b1, ctx->pev[8 * r + 2], ctx->pev[8 * r + 3]));
            CK(cudaEventElapsedTime(&c, ctx->pev[8 * r + 4], ctx->pev[8 * r + 5]));
            CK(cudaEventElapsedTime(&b2, ctx->pev[8 * r + 6], ctx->pev[8 * r + 7]));
            sc += a;
            stp += b1 + b2;
            clu += c;
            float *rm = &ctx->round_ms[4 * (size_t)r];
            rm[0] = a; rm[1] = b1; rm[2] = c; rm[3] = b2;
        }
        ctx->prof.scan_ms = sc;
        ctx->prof.step_ms = stp;
        ctx->prof.cluster_ms = clu;
        ctx->last_launches = ctx->sweep_launches;
        std::vector<PairAcc> A(pl.np);
        CK(cudaMemcpyAsync(A.data(), ctx->pacc, sizeof(PairAcc) * pl.np, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        ctx->pair_ms.assign(3 * (size_t)pl.np, 0.f);
        for (int r = 0; r < pl.nr; ++r) {
            unsigned long long first = ~0ull;
            for (int i = pl.off[r]; i < pl.off[r + 1]; ++i)
                if (A[i].t1 && A[i].t0 < first) first = A[i].t0;
            for (int i = pl.off[r]; i < pl.off[r + 1]; ++i) {
                float *pm = &ctx->pair_ms[3 * (size_t)i];
                pm[0] = (float)r;
                pm[1] = A[i].t1 ? (float)((A[i].t0 - first) * 1e-6) : -1.f;
                pm[2] = A[i].t1 ? (float)((A[i].t1 - first) * 1e-6) : -1.f;
            }
        }
        return FR_OK;
    }
    ctx->prof.scan_ms = ctx->prof.step_ms = ctx->prof.cluster_ms = 0;
    ctx->round_ms.clear();
    ctx->pair_ms.clear();
    if (ctx->use_graphs) {
        for (auto &e : ctx->gcache)
            if (e.key == key) { exec = e.exec; exec_launches = e.launches; break; }
        if (!exec) {
            cudaGraph_t graph = nullptr;
            CK(cudaStreamSynchronize(ctx->stream));
            cudaError_t e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
            fr_status st = FR_OK;
            if (e == cudaSuccess) {
                st = enqueue_sweep(ctx, g, pl, opt);
                cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &graph);
                if (st == FR_OK && e2 == cudaSuccess && graph) {
                    e2 = cudaGraphInstantiate(&exec, graph, 0);
                    cudaGraphDestroy(graph);
                    if (e2 != cudaSuccess) exec = nullptr;
                } else if (graph) {
                    cudaGraphDestroy(graph);
                }
            }
            cudaGetLastError();
            if (exec) {
                if (ctx->gcache.size() >= 16) {
                    cudaGraphExecDestroy(ctx->gcache.front().exec);
                    ctx->gcache.erase(ctx->gcache.begin());
                }
                exec_launches = ctx->sweep_launches;
                ctx->gcache.push_back({key, exec, exec_launches});
            } else {
                ctx->use_graphs = false;   // capture unsupported here: launch directly from now on
            }
        }
    }
    CK(cudaEventRecord(ctx->ev0, ctx->stream));
    if (exec) {
        CK(cudaGraphLaunch(exec, ctx->stream));
    } else {
        fr_status st = enqueue_sweep(ctx, g, pl, opt);
        if (st != FR_OK) return st;
    }
    CK(cudaEventRecord(ctx->ev1, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaEventElapsedTime(ms, ctx->ev0, ctx->ev1));
    // prep + colour + fill + per round the scan, the steps and the cluster launches
    ctx->last_launches = exec ? exec_launches : ctx->sweep_launches;
    return FR_OK;
}

// Plans a sweep: prep + quotient rounds, budgets, per-round grid sizes.
static fr_status plan_sweep(fr_ctx *ctx, const fr_graph *g, const int32_t *part, int32_t k, double eps, double alpha,
                            const fr_options *opt, BatchPlan *pl) {
    fr_status st = ensure_base(ctx, g->n, g->nnz, k, opt->mb_reps);
    if (st != FR_OK) return st;
    PrepOut po;
    if ((st = run_prep(ctx, g, part, k, true, opt->checked != 0, &po)) != FR_OK) return st;
    pl->np = po.npairs;
    pl->nr = po.nrounds;
    pl->k = k;
    pl->totcut = po.totcut;
    pl->Ubase = host_budget_base(po.W, k, eps, alpha);
    pl->Lmax = host_lmax(po.W, po.maxc, k, eps);
    pl->tpb = choose_tpb(ctx, opt);
    if (pl->np == 0) return FR_OK;
    if ((st = ensure_pairs(ctx, pl->np, pl->nr, opt->mb_reps)) != FR_OK) return st;
    // round offsets, pair lists and block weights for the grid estimate
    std::vector<int> &pa = pl->pa, &pb = pl->pb;
    pa.assign(pl->np, 0);
    pb.assign(pl->np, 0);
    std::vector<long long> bw(k);
    pl->off.assign(pl->nr + 1, 0);
    CK(cudaMemcpyAsync(pl->off.data(), ctx->round_off, sizeof(int) * (pl->nr + 1), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(pa.data(), ctx->pair_a, sizeof(int) * pl->np, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(pb.data(), ctx->pair_b, sizeof(int) * pl->np, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(bw.data(), ctx->blockw, sizeof(long long) * k, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const double avgc = std::max(1.0, (double)po.W / (double)g->n);
    pl->grid.assign(pl->nr, 1);
    pl->est_max.assign(pl->nr, 0);
    pl->avg_degree = (double)g->nnz / g->n;
    for (int r = 0; r < pl->nr; ++r) {
        long long est = 0;
        for (int i = pl->off[r]; i < pl->off[r + 1]; ++i) {
            const long long e1 = std::max(0LL, pl->Ubase - bw[pb[i]]) + std::max(0LL, pl->Ubase - bw[pa[i]]);
            est += e1;
            pl->est_max[r] = std::max(pl->est_max[r], (long long)(e1 / avgc));
        }
        pl->grid[r] = choose_grid(ctx, opt, pl->tpb, 2 * (pl->off[r + 1] - pl->off[r]),
                                  std::max<long long>(1, (long long)(est / avgc)));
    }
    return FR_OK;
}

static fr_status batch_core(fr_ctx *ctx, const fr_graph *g, int32_t *part, int32_t k, double eps, double alpha,
                            const fr_options *opt, int32_t cap, fr_pair_result *results, fr_batch_result *summary) {
    BatchPlan pl;
    fr_status st = plan_sweep(ctx, g, part, k, eps, alpha, opt, &pl);
    if (st != FR_OK) return st;
    fr_batch_result sum;
    memset(&sum, 0, sizeof(sum));
    sum.npairs = pl.np;
    sum.nrounds = pl.nr;
    sum.cut_before = sum.cut_after = pl.totcut;
    if (pl.np == 0) {
        if (summary) *summary = sum;
        return FR_OK;
    }
    if (opt->fm_permille > 0 && (st = ensure_fm(ctx, g->n, g->nnz, k, pl.np)) != FR_OK) return st;
    float ms = 0.f;
    std::vector<Ctl> C;
    bool queued = false;
    const int qt = queue_size_for(ctx, pl, opt);
    if (qt >= 0) {
        // every pair in one launch, each as soon as its predecessors on its blocks committed
        if ((st = run_queue_sweep(ctx, g, part, pl, opt, qt, &ms, &queued, &C)) != FR_OK) {
            sum.status = st;
            if (summary) *summary = sum;
            return st;
        }
        // a pair outgrew its cluster: part is restored; plan again and go round by round
        if (!queued && (st = plan_sweep(ctx, g, part, k, eps, alpha, opt, &pl)) != FR_OK) return st;
    }
    ctx->last_queue = queued;
    if (!queued) {
        if ((st = run_sweep(ctx, g, part, pl, opt, &ms)) != FR_OK) return st;
        C.assign(pl.nr, Ctl());
        CK(cudaMemcpyAsync(C.data(), ctx->ctl, sizeof(Ctl) * pl.nr, cudaMemcpyDeviceToHost, ctx->stream));
    }
    std::vector<PairAcc> A(pl.np);
    std::vector<SideDev> S(2 * pl.np);
    const std::vector<int> &pa = pl.pa, &pb = pl.pb;
    std::vector<FmRes> FR(opt->fm_permille > 0 ? pl.np : 0);
    if (!FR.empty())
        CK(cudaMemcpyAsync(FR.data(), ctx->fm.res, sizeof(FmRes) * pl.np, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(A.data(), ctx->pacc, sizeof(PairAcc) * pl.np, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(S.data(), ctx->sides, sizeof(SideDev) * 2 * pl.np, cudaMemcpyDeviceToHost, ctx->stream));
    std::vector<long long> qst(queued ? 4 * ctx->last_queue_clusters : 0);
    if (!qst.empty())
        CK(cudaMemcpyAsync(qst.data(), ctx->q_stats, sizeof(long long) * qst.size(), cudaMemcpyDeviceToHost,
                           ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    fr_status bad = FR_OK;
    for (size_t r = 0; r < C.size() && bad == FR_OK; ++r) bad = status_from_ctl(ctx, C[r], "fr_refine_batch");
    if (bad != FR_OK) {
        // leave part exactly as it was
        CK(cudaMemcpyAsync(part, ctx->part_backup, sizeof(int) * (size_t)g->n, cudaMemcpyDeviceToDevice, ctx->stream));
        reset_idle(ctx);
        sum.status = bad;
        if (summary) *summary = sum;
        return bad;
    }
    long long flow_ns = 0;
    for (size_t r = 0; r < C.size(); ++r)
        flow_ns += C[r].timers[T_FLOW1] + C[r].timers[T_GR] + C[r].timers[T_FLOW2] + C[r].timers[T_CL_FLOW] +
                   C[r].timers[T_CL_RETURN];
    {
        fr_profile_info &P = ctx->prof;
        const double sc = P.scan_ms, stp = P.step_ms, clu = P.cluster_ms;
        memset(&P, 0, sizeof(P));
        P.scan_ms = sc;
        P.step_ms = stp;
        P.cluster_ms = clu;
        P.nrounds = pl.nr;
        P.launches = (int32_t)ctx->last_launches;
        for (int t = 0; t < fr_ctx::kNumClusterSizes && t < 5; ++t) {
            P.cluster_sizes[t] = fr_ctx::kClusterSizes[t];
            P.cluster_max_active[t] = ctx->cl_cap[t];
        }
        P.n = g->n;
        P.nnz = g->nnz;
        for (size_t r = 0; r < C.size(); ++r) {
            for (int t = 0; t < T_COUNT && t < 12; ++t) P.phase_ms[t] += C[r].timers[t] * 1e-6;
            if (!queued) {   // (per step; the queue sweep sums them per cluster below)
                P.bfs_visited += C[r].vq_total;
                P.corridor_n += C[r].nu;
                P.corridor_arcs += C[r].mu;
            }
            P.bfs_arcs += C[r].arcs_scanned;
            P.pulses += C[r].pulses;
            P.relabels += C[r].relabels;
            P.gr_arcs += C[r].gr_arcs;
            P.pr_arcs += C[r].pr_arcs;
            P.pushes += C[r].pushes;
            P.scc_rounds += C[r].scc_rounds;
            P.barriers += C[r].barriers;
            for (int t = 0; t < 7; ++t) P.cluster_phase_ms[t] += C[r].timers[T_CL_LOAD + t] * 1e-6;
            P.cluster_syncs += C[r].cl_syncs;
            P.cluster_remote_arcs += C[r].cl_remote;
            P.scan_listed += C[r].scan_listed;
            P.scan_rows += C[r].scan_rows;
            P.scan_arcs += C[r].scan_arcs;
            P.fallback_pairs += C[r].fallback;
            for (int t = 0; t < 3; ++t) P.fm_ms[t] += C[r].timers[T_FM_SORT + t] * 1e-6;
            P.queue_scan_ms += C[r].timers[T_QSCAN] * 1e-6;
            P.gaps += C[r].gaps;
            P.gap_lifted += C[r].gap_lifted;
        }
        for (size_t i = 0; i + 3 < qst.size(); i += 4) {
            P.bfs_visited += qst[i];
            P.corridor_n += qst[i + 1];
            P.corridor_arcs += qst[i + 2];
        }
        P.queue = queued ? 1 : 0;
        P.queue_ctas = queued ? ctx->last_queue_ctas : 0;
        P.queue_clusters = queued ? ctx->last_queue_clusters : 0;
        P.queue_fallbacks = ctx->queue_fallbacks;
    }
    for (int r = 0; r < pl.nr; ++r)
        for (int i = pl.off[r]; i < pl.off[r + 1]; ++i) {
            const PairAcc &a = A[i];
            const int acc = a.accept;
            sum.accepted += acc;
            sum.cut_after += acc ? a.dcut : 0;
            if (!FR.empty()) sum.cut_after += FR[i].cut1 - FR[i].cut0;
            sum.corridor_arcs += a.m;
            if (results && i < cap) {
                fr_pair_result &R = results[i];
                memset(&R, 0, sizeof(R));
                R.a = pa[i]; R.b = pb[i]; R.round = r;
                R.flow = a.flow;
                R.cut_before = a.oldcut;
                R.cut_after = a.oldcut + (acc ? a.dcut : 0);
                R.wA_before = S[2 * i].cw; R.wB_before = S[2 * i + 1].cw;
                R.wA_after = S[2 * i].cw + (acc ? a.dwA : 0);
                R.wB_after = S[2 * i + 1].cw - (acc ? a.dwA : 0);
                R.corridor_n = a.nc; R.corridor_arcs = a.m;
                R.accepted = acc;
                R.iters = 1;
                R.alpha_final = alpha;
                R.status = FR_OK;
                if (!queued) {   // step-wide counters of the pair's round (the queue keeps none per pair)
                    R.pulses = C[r].pulses; R.relabels = C[r].relabels;
                    R.bfs_levels = C[r].levels; R.scc_rounds = C[r].scc_rounds;
                }
                R.ncomp = a.ncomp;
                R.cut_fm = a.oldcut;
                if (!FR.empty()) {   // before = before the FM step
                    R.cut_before = FR[i].cut0;
                    R.wA_before = FR[i].wA0;
                    R.wB_before = FR[i].wB0;
                    R.fm_moves = FR[i].kept;
                }
            }
        }
    sum.device_ns = (long long)(ms * 1e6);
    sum.flow_ns = flow_ns;
    if (summary) *summary = sum;
    return FR_OK;
}

extern "C" fr_status fr_refine_batch(fr_ctx *ctx, const fr_graph *g, int32_t *part, int32_t k, double eps,
                                     double alpha, const fr_options *opt_in, int32_t cap, fr_pair_result *results,
                                     fr_batch_result *summary) {
    if (!ctx) return FR_ERR_INVALID_ARG;
    fr_options opt;
    if (opt_in) opt = *opt_in; else fr_default_options(&opt);
    if (opt.mb_reps < 1) opt.mb_reps = 1;
    if (summary) memset(summary, 0, sizeof(*summary));
    fr_status st = check_graph(ctx, g, part, k);
    if (st == FR_OK) st = check_params(ctx, eps, alpha, &opt);
    if (st == FR_OK && opt.mt_alpha != 0) { ctx_error(ctx, "mt_alpha: fr_refine_active only"); st = FR_ERR_INVALID_ARG; }
    if (st == FR_OK && cap > 0 && !results) { ctx_error(ctx, "results is NULL"); st = FR_ERR_INVALID_ARG; }
    if (st != FR_OK) { if (summary) summary->status = st; return st; }
    if (opt.adaptive) {
        // adaptive flow iterations (Section 4.1) per pair: the rounds' pairs iterate
        // together, each on its own alpha, launch sequence by launch sequence -- the
        // first outer round of active block scheduling, where every block is active
        return fr_refine_active(ctx, g, part, k, eps, alpha, &opt, 1, cap, results, summary, nullptr);
    }
    CK(cudaSetDevice(ctx->device));
    release_corridor(ctx);
    st = batch_core(ctx, g, part, k, eps, alpha, &opt, cap, results, summary);
    if (summary) summary->status = st;
    return st;
}

extern "C" fr_status fr_refine_batch_host(fr_ctx *ctx, int32_t n, int32_t nnz, const int32_t *xadj_host,
                                          const int32_t *adjncy_host, const int32_t *adjwgt_host,
                                          const int32_t *vwgt_host, int32_t *part_host, int32_t k, double eps,
                                          double alpha, const fr_options *opt, int32_t cap, fr_pair_result *results,
                                          fr_batch_result *summary) {
    if (!ctx) return FR_ERR_INVALID_ARG;
    if (n < 1 || nnz < 0 || !xadj_host || !vwgt_host || !part_host || (nnz > 0 && (!adjncy_host || !adjwgt_host))) {
        ctx_error(ctx, "host graph arrays invalid");
        return FR_ERR_INVALID_ARG;
    }
    CK(cudaSetDevice(ctx->device));
    const size_t need = sizeof(int) * ((size_t)(n + 1) + 2 * (size_t)nnz + 2 * (size_t)n) + 4 * 256;
    if (need > ctx->hg_bytes) {
        if (ctx->hg_mem) cudaFree(ctx->hg_mem);
        ctx->hg_mem = nullptr;
        ctx->hg_bytes = 0;
        if (cudaMalloc(&ctx->hg_mem, need) != cudaSuccess) {
            cudaGetLastError();
            ctx_error(ctx, "cudaMalloc for the host graph copy failed");
            return FR_ERR_OOM;
        }
        ctx->hg_bytes = need;
    }
    char *p = reinterpret_cast<char *>(ctx->hg_mem);
    auto take = [&](size_t cnt) {
        int *r = reinterpret_cast<int *>(p);
        p += ((sizeof(int) * cnt + 255) / 256) * 256;
        return r;
    };
    int *dx = take(n + 1), *da = take(nnz), *dw = take(nnz), *dv = take(n), *dp = take(n);
    CK(cudaMemcpyAsync(dx, xadj_host, sizeof(int) * (size_t)(n + 1), cudaMemcpyHostToDevice, ctx->stream));
    if (nnz) {
        CK(cudaMemcpyAsync(da, adjncy_host, sizeof(int) * (size_t)nnz, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(dw, adjwgt_host, sizeof(int) * (size_t)nnz, cudaMemcpyHostToDevice, ctx->stream));
    }
    CK(cudaMemcpyAsync(dv, vwgt_host, sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(dp, part_host, sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, ctx->stream));
    fr_graph g = {n, nnz, dx, da, dw, dv};
    fr_status st = fr_refine_batch(ctx, &g, dp, k, eps, alpha, opt, cap, results, summary);
    CK(cudaMemcpyAsync(part_host, dp, sizeof(int) * (size_t)n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return st;
}

// ------------------------------------------------------------- autotuner --

extern "C" fr_status fr_autotune(fr_ctx *ctx, const fr_graph *g, const int32_t *part, int32_t k, double eps,
                                 double alpha, const fr_options *opt_in, int32_t trials, fr_options *best,
                                 double *best_ms) {
    if (!ctx) return FR_ERR_INVALID_ARG;
    fr_options base;
    if (opt_in) base = *opt_in; else fr_default_options(&base);
    if (base.mb_reps < 1) base.mb_reps = 1;
    fr_status st = check_graph(ctx, g, part, k);
    if (st == FR_OK) st = check_params(ctx, eps, alpha, &base);
    if (st == FR_OK && base.mt_alpha != 0) { ctx_error(ctx, "mt_alpha: fr_refine_active only"); st = FR_ERR_INVALID_ARG; }
    if (st != FR_OK) return st;
    if (trials < 1) trials = 1;
    CK(cudaSetDevice(ctx->device));
    release_corridor(ctx);
    int32_t *scratch = nullptr;
    if (cudaMalloc(&scratch, sizeof(int) * (size_t)g->n) != cudaSuccess) {
        cudaGetLastError();
        return FR_ERR_OOM;
    }
    std::vector<int> ref, cur(g->n);
    auto time_shape = [&](const fr_options &o, double *ms_out) -> fr_status {
        double bestv = 1e30;
        for (int t = 0; t < trials + 1; ++t) {   // first run warms up (and captures)
            if (cudaMemcpyAsync(scratch, part, sizeof(int) * (size_t)g->n, cudaMemcpyDeviceToDevice, ctx->stream) !=
                cudaSuccess)
                return FR_ERR_CUDA;
            fr_batch_result sum;
            fr_status s2 = batch_core(ctx, g, scratch, k, eps, alpha, &o, 0, nullptr, &sum);
            if (s2 != FR_OK) return s2;
            if (t > 0) bestv = std::min(bestv, sum.device_ns * 1e-6);
        }
        if (cudaMemcpy(cur.data(), scratch, sizeof(int) * (size_t)g->n, cudaMemcpyDeviceToHost) != cudaSuccess)
            return FR_ERR_CUDA;
        if (ref.empty()) ref = cur;
        else if (ref != cur) {
            ctx_error(ctx, "launch shapes gave different partitions");
            return FR_ERR_INTERNAL;
        }
        *ms_out = bestv;
        return FR_OK;
    };
    fr_options cand = base;
    cand.block_threads = base.block_threads ? base.block_threads : 512;
    cand.gr_interval = base.gr_interval ? base.gr_interval : ctx->tune_gr;
    cand.inner_ops = base.inner_ops ? base.inner_ops : ctx->tune_inner;
    cand.pulse_passes = base.pulse_passes ? base.pulse_passes : ctx->tune_passes;
    cand.grid_blocks = base.grid_blocks;
    double bms = 0;
    st = time_shape(cand, &bms);
    const int sms = ctx->sms > 0 ? ctx->sms : 1;
    // coordinate descent over the launch shape
    const std::vector<int> grids = {0, sms / 8, sms / 4, sms / 2, sms, 2 * sms};
    const std::vector<int> tpbs = {256, 512};
    const std::vector<int> grs = {2, 4, 8, 16, 32};
    const std::vector<int> inners = {1, 2, 4, 8};
    const std::vector<int> passes = {1, 2, 4, 8};
    std::vector<int> ctas = {0};
    for (int t = 0; t < fr_ctx::kNumClusterSizes; ++t)
        if (ctx->cl_cap[t] > 0) ctas.push_back(fr_ctx::kClusterSizes[t]);
    cand.cluster_ctas = base.cluster_ctas ? base.cluster_ctas : ctx->tune_ctas;
    cand.flow_sched = base.flow_sched ? base.flow_sched : (ctx->tune_sched ? ctx->tune_sched : 2);
    const std::vector<int> scheds = {2, 1};
    const std::vector<int> prewaves = {-1, 1, 2};
    cand.pre_waves = base.pre_waves ? base.pre_waves : (ctx->tune_prewaves ? ctx->tune_prewaves : -1);
    for (int sweep = 0; sweep < 2 && st == FR_OK; ++sweep) {
        for (int dim = 0; dim < 8 && st == FR_OK; ++dim) {
            const std::vector<int> &vals = dim == 0   ? tpbs
                                           : dim == 1 ? grids
                                           : dim == 2 ? grs
                                           : dim == 3 ? inners
                                           : dim == 4 ? passes
                                           : dim == 5 ? ctas
                                           : dim == 6 ? scheds
                                                      : prewaves;
            for (int v : vals) {
                fr_options o = cand;
                if (dim == 0) o.block_threads = v;
                if (dim == 1) { if (v < 0) continue; o.grid_blocks = v; }
                if (dim == 2) o.gr_interval = v;
                if (dim == 3) o.inner_ops = v;
                if (dim == 4) o.pulse_passes = v;
                if (dim == 5) o.cluster_ctas = v;
                if (dim == 6) o.flow_sched = v;
                if (dim == 7) o.pre_waves = v;
                if (memcmp(&o, &cand, sizeof(o)) == 0) continue;
                double ms = 0;
                st = time_shape(o, &ms);
                if (st != FR_OK) break;
                if (ms < bms * 0.98) { bms = ms; cand = o; }
            }
        }
    }
    cudaFree(scratch);
    if (st != FR_OK) return st;
    ctx->tune_tpb = cand.block_threads;
    ctx->tune_grid = cand.grid_blocks;
    ctx->tune_gr = cand.gr_interval;
    ctx->tune_inner = cand.inner_ops;
    ctx->tune_passes = cand.pulse_passes;
    ctx->tune_ctas = cand.cluster_ctas;
    ctx->tune_sched = cand.flow_sched;
    ctx->tune_prewaves = cand.pre_waves > 0 ? cand.pre_waves : 0;
    if (best) *best = cand;
    if (best_ms) *best_ms = bms;
    return FR_OK;
}

extern "C" int64_t fr_last_launch_count(const fr_ctx *ctx) { return ctx ? ctx->last_launches : 0; }

extern "C" fr_status fr_set_profiling(fr_ctx *ctx, int32_t on) {
    if (!ctx) return FR_ERR_INVALID_ARG;
    ctx->profiling = on != 0;
    return FR_OK;
}

extern "C" fr_status fr_profile_last(const fr_ctx *ctx, fr_profile_info *info) {
    if (!ctx || !info) return FR_ERR_INVALID_ARG;
    *info = ctx->prof;
    return FR_OK;
}

extern "C" int32_t fr_profile_pairs(const fr_ctx *ctx, float *ms, int32_t cap) {
    if (!ctx || (cap > 0 && !ms)) return -1;
    const int np = (int)(ctx->pair_ms.size() / 3);
    for (int i = 0; i < 3 * std::min(np, (int)std::max(cap, 0)); ++i) ms[i] = ctx->pair_ms[i];
    return np;
}

extern "C" int32_t fr_profile_rounds(const fr_ctx *ctx, float *ms, int32_t cap) {
    if (!ctx || (cap > 0 && !ms)) return -1;
    const int nr = (int)(ctx->round_ms.size() / 4);
    for (int i = 0; i < 4 * std::min(nr, (int)std::max(cap, 0)); ++i) ms[i] = ctx->round_ms[i];
    return nr;
}
