// C ABI, host side of the queue sweep (queue_sweep.cu): per-cluster workspaces, the
// choice of cluster size, the launch (captured as a CUDA graph like the round-by-round
// sweep) and the fallback to the round-by-round sweep when a pair outgrows a cluster.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "api_internal.h"

using namespace fr;

#define CK(call)                                                 \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

namespace {

// relative time of one pair on clusters of 4, 6, 8, 12, 16 CTAs (measured on 3D rgg and
// grid pairs; the same table as the round-by-round cluster launches)
constexpr double kRelTime[fr_ctx::kNumClusterSizes] = {1.25, 1.05, 1.0, 0.85, 0.74};
// host staging offsets (the first megabytes of h_stage belong to the other paths)
constexpr size_t kStageGraphs = 4u << 20;
constexpr size_t kStagePrev = (4u << 20) + (64u << 10);
constexpr unsigned long long kWaitNs = 10ull * 1000 * 1000 * 1000;   // one dependency wait, at most 10 s

size_t al256(size_t b) { return (b + 255) / 256 * 256; }

struct QCaps {
    long long nu, mu, vq, words, swords;
};

// Per-pair capacities of a cluster of `ctas` CTAs: a network that fits its shared
// memory has at most dyn / 29 vertices and dyn / 16 arcs per CTA.
QCaps caps_for(int ctas, int n) {
    const long long dyn = (long long)queue_smem();
    QCaps c;
    c.nu = (long long)ctas * dyn / 28 + 64;
    c.mu = (long long)ctas * dyn / 16 + 64;
    c.vq = std::min<long long>(n, std::max<long long>(4 * c.nu, 1 << 16));
    c.words = n / 32 + 2;
    c.swords = n / 32768 + 2;
    return c;
}

size_t slot_bytes(const QCaps &c, int ctas, int k, int reps) {
    size_t b = 0;
    auto add = [&](size_t elem, long long cnt) { b += al256(elem * (size_t)cnt); };
    add(4, k);                                      // sob
    add(8, 3LL * 2 * kHistBins);                    // hist
    add(4, ctas + 1);                               // cta_cnt
    add(4, c.words);                                // cbits
    add(4, c.words);                                // sdbits
    add(4, c.swords);                               // sbits
    add(4, c.vq); add(4, c.vq);                     // vq_v vq_s
    for (int i = 0; i < 21; ++i) add(4, c.nu + 1);  // gid .. sinkc, pcur
    add(8, c.nu); add(8, c.nu);                     // ex cw
    add(1, c.nu); add(1, c.nu);                     // border side_out
    for (int i = 0; i < 5; ++i) add(4, c.mu);       // head rev res cap outs
    for (int i = 0; i < 3; ++i) add(4, (long long)reps * c.nu);   // indeg_r order hcomp
    add(8, (long long)reps * c.nu);                 // hkey
    add(8, reps); add(4, reps);                     // sw_absd sw_j
    return b;
}

template <class T>
T *take(char *&p, long long count) {
    T *r = reinterpret_cast<T *>(p);
    p += al256(sizeof(T) * (size_t)count);
    return r;
}

fr_status ensure_queue(fr_ctx *ctx, int ctas, int clusters, int n, int nnz, int k, int reps, int np) {
    if (ctx->q_mem && ctas == ctx->q_ctas && clusters <= ctx->q_clusters && n <= ctx->q_n && nnz <= ctx->q_nnz &&
        k <= ctx->q_k && reps <= ctx->q_reps && np <= ctx->q_np)
        return FR_OK;
    const int nn = std::max(n, ctx->q_ctas == ctas ? ctx->q_n : 0);
    const int mm = std::max(nnz, ctx->q_ctas == ctas ? ctx->q_nnz : 0);
    const int kk = std::max(k, ctx->q_ctas == ctas ? ctx->q_k : 0);
    const int rr = std::max(reps, ctx->q_ctas == ctas ? ctx->q_reps : 1);
    const int pp = std::max(np, ctx->q_ctas == ctas ? ctx->q_np : 0);
    const int cc = std::max(clusters, ctx->q_ctas == ctas ? ctx->q_clusters : 0);
    const QCaps c = caps_for(ctas, nn);
    const size_t per = slot_bytes(c, ctas, kk, rr);
    // per-block candidate lists: the sweep's candidates bucketed, and a region per block
    // for the commits' appends (a sweep that fills one runs again round by round)
    const long long qcap = std::max<long long>(4096, 8LL * ((nn + kk - 1) / kk));
    size_t bytes = al256(4) + al256(4) + al256(8ull * pp) + al256(4ull * mm) + al256(sizeof(QSlot) * cc) +
                   al256(sizeof(GraphDev) * cc) + al256(sizeof(fr_ctx::QCtl) * cc) + al256(32ull * cc) + per * cc +
                   al256(4ull * nn) + al256(4ull * (kk + 1)) + 2 * al256(4ull * kk) + al256(4ull * kk * qcap) +
                   al256(4ull * nn);
    if (ctx->arena_limit && bytes + ctx->base_bytes + ctx->pair_bytes + ctx->reps_bytes > ctx->arena_limit) {
        ctx_error(ctx, "queue sweep workspace exceeds the arena bound");
        return FR_ERR_OOM;
    }
    free_queue(ctx);
    if (cudaMalloc(&ctx->q_mem, bytes) != cudaSuccess) {
        cudaGetLastError();
        ctx->q_mem = nullptr;
        ctx_error(ctx, "cudaMalloc(%zu) for the queue sweep failed", bytes);
        return FR_ERR_OOM;
    }
    ctx->q_bytes = bytes;
    ctx->q_ctas = ctas; ctx->q_clusters = cc; ctx->q_n = nn; ctx->q_nnz = mm; ctx->q_k = kk; ctx->q_reps = rr;
    ctx->q_np = pp;
    ctx->q_nu = c.nu; ctx->q_mu = c.mu; ctx->q_vq = c.vq;
    char *p = reinterpret_cast<char *>(ctx->q_mem);
    ctx->q_ticket = take<int>(p, 1);
    ctx->q_gabort = take<int>(p, 1);
    ctx->q_prev = take<int>(p, 2LL * pp);
    ctx->q_crank = take<int>(p, mm);
    ctx->q_slots = take<QSlot>(p, cc);
    ctx->qb_sorted = take<int>(p, nn);
    ctx->qb_start = take<int>(p, kk + 1);
    ctx->qb_cnt = take<int>(p, kk);
    ctx->qb_app = take<int>(p, kk);
    ctx->qb_pool = take<int>(p, (long long)kk * qcap);
    ctx->qb_lst = take<int>(p, nn);
    ctx->qb_cap = (int)qcap;
    ctx->q_graphs = take<GraphDev>(p, cc);
    ctx->q_ctls = take<fr_ctx::QCtl>(p, cc);
    ctx->q_stats = take<long long>(p, 4LL * cc);
    ctx->q_host.assign(cc, QSlot());
    for (int i = 0; i < cc; ++i) {
        QSlot &S = ctx->q_host[i];
        S.graph = ctx->q_graphs + i;
        S.sob = take<int>(p, kk);
        S.ctl = &ctx->q_ctls[i].c;
        S.hist = take<long long>(p, 3LL * 2 * kHistBins);
        S.cta_cnt = take<int>(p, ctas + 1);
        S.cbits = take<unsigned int>(p, c.words);
        S.sdbits = take<unsigned int>(p, c.words);
        S.sbits = take<unsigned int>(p, c.swords);
        S.vq_v = take<int>(p, c.vq); S.vq_s = take<int>(p, c.vq);
        int **v21[21] = {&S.gid, &S.sid, &S.off, &S.infc, &S.fx, &S.lab, &S.rflag, &S.color, &S.scc, &S.vc,
                         &S.fq0, &S.fq1, &S.cid, &S.cpair, &S.cmin, &S.indeg, &S.outoff, &S.ocur, &S.plist,
                         &S.sinkc, &S.pcur};
        for (auto a : v21) *a = take<int>(p, c.nu + 1);
        S.ex = take<long long>(p, c.nu); S.cw = take<long long>(p, c.nu);
        S.border = take<unsigned char>(p, c.nu); S.side_out = take<unsigned char>(p, c.nu);
        S.head = take<int>(p, c.mu); S.rev = take<int>(p, c.mu); S.res = take<int>(p, c.mu);
        S.cap = take<int>(p, c.mu); S.outs = take<int>(p, c.mu);
        S.indeg_r = take<int>(p, (long long)rr * c.nu); S.order = take<int>(p, (long long)rr * c.nu);
        S.hcomp = take<int>(p, (long long)rr * c.nu);
        S.hkey = take<unsigned long long>(p, (long long)rr * c.nu);
        S.sw_absd = take<long long>(p, rr); S.sw_j = take<int>(p, rr);
        S.stat = ctx->q_stats + 4LL * i;
        // idle state: no block paired, no corridor bit set
        CK(cudaMemsetAsync(S.sob, 0xFF, sizeof(int) * (size_t)kk, ctx->stream));
        CK(cudaMemsetAsync(S.cbits, 0, sizeof(unsigned int) * (size_t)c.words, ctx->stream));
        CK(cudaMemsetAsync(S.sdbits, 0, sizeof(unsigned int) * (size_t)c.words, ctx->stream));
        CK(cudaMemsetAsync(S.sbits, 0, sizeof(unsigned int) * (size_t)c.swords, ctx->stream));
    }
    CK(cudaMemcpyAsync(ctx->q_slots, ctx->q_host.data(), sizeof(QSlot) * cc, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    destroy_graph_cache(ctx);   // captured sweeps hold pointers into the old workspace
    return FR_OK;
}

// After a failed or abandoned queue sweep: BFS marks, corridor bits and block sides idle.
fr_status reset_queue_idle(fr_ctx *ctx) {
    fr_status st = reset_idle(ctx);
    if (st != FR_OK) return st;
    const QCaps c = caps_for(ctx->q_ctas, ctx->q_n);
    for (const QSlot &S : ctx->q_host) {
        CK(cudaMemsetAsync(S.sob, 0xFF, sizeof(int) * (size_t)ctx->q_k, ctx->stream));
        CK(cudaMemsetAsync(S.cbits, 0, sizeof(unsigned int) * (size_t)c.words, ctx->stream));
        CK(cudaMemsetAsync(S.sdbits, 0, sizeof(unsigned int) * (size_t)c.words, ctx->stream));
        CK(cudaMemsetAsync(S.sbits, 0, sizeof(unsigned int) * (size_t)c.swords, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return FR_OK;
}

}  // namespace

void free_queue(fr_ctx *ctx) {
    if (ctx->q_mem) cudaFree(ctx->q_mem);
    ctx->q_mem = nullptr;
    ctx->q_bytes = 0;
    ctx->q_ctas = ctx->q_clusters = ctx->q_n = ctx->q_nnz = ctx->q_k = ctx->q_reps = ctx->q_np = 0;
    ctx->q_host.clear();
    ctx->q_slots = nullptr;
    ctx->q_graphs = nullptr;
    ctx->q_ctls = nullptr;
    ctx->q_stats = nullptr;
}

int queue_size_for(fr_ctx *ctx, const BatchPlan &pl, const fr_options *opt) {
    if (opt->fm_permille > 0 || opt->sweep_sched == 1 || pl.np == 0) return -1;
    if (2LL * pl.np * (long long)sizeof(int) > (long long)(kHostStage - kStagePrev)) return -1;
    const size_t dyn = queue_smem();
    if (dyn == 0) return -1;
    long long est = 0;
    for (long long e : pl.est_max) est = std::max(est, e);
    const double need = 1.05 * (double)est * (29.0 + (ctx->narrow_ok ? 16.0 : 20.0) * pl.avg_degree);
    const double per_cta = 0.95 * (double)dyn;
    const int force = opt->cluster_ctas ? opt->cluster_ctas : ctx->tune_ctas;
    int best = -1;
    double bestv = 0;
    for (int t = 0; t < fr_ctx::kNumClusterSizes; ++t) {
        if (ctx->q_cap[t] <= 0) continue;
        const int c = fr_ctx::kClusterSizes[t];
        if (force) {
            if (force == c) return t;
            continue;
        }
        if (need > per_cta * c) continue;
        // pairs in flight at once over the time of one pair
        const double v = (double)std::min(ctx->q_cap[t], pl.np) / kRelTime[t];
        if (best < 0 || v > bestv) { best = t; bestv = v; }
    }
    return best;
}

fr_status run_queue_sweep(fr_ctx *ctx, const fr_graph *g, int32_t *part, const BatchPlan &pl, const fr_options *opt,
                          int t, float *ms, bool *ran, std::vector<Ctl> *ctls) {
    *ran = false;
    const int ctas = fr_ctx::kClusterSizes[t];
    // resident clusters, or fewer when opt->grid_blocks bounds the CTAs
    int clusters = std::max(1, std::min(ctx->q_cap[t], pl.np));
    if (opt->grid_blocks > 0) clusters = std::max(1, std::min(clusters, opt->grid_blocks / ctas));
    const int reps = opt->mb_reps > 0 ? opt->mb_reps : 1;
    fr_status st = ensure_queue(ctx, ctas, clusters, g->n, g->nnz, pl.k, reps, pl.np);
    if (st != FR_OK) return st;
    // per-cluster graph descriptors (each with its own sob) and each pair's predecessors
    GraphDev *hg = reinterpret_cast<GraphDev *>(ctx->h_stage + kStageGraphs);
    for (int i = 0; i < clusters; ++i) {
        GraphDev &gd = hg[i];
        memset(&gd, 0, sizeof(gd));
        gd.xadj = g->xadj; gd.adjncy = g->adjncy; gd.adjwgt = g->adjwgt; gd.vwgt = g->vwgt;
        gd.part = part; gd.dist = ctx->dist; gd.lid = ctx->lid;
        gd.sob = ctx->q_host[i].sob;
        gd.blockw = ctx->blockw;
        gd.n = g->n; gd.nnz = g->nnz; gd.k = pl.k; gd.base = 0; gd.Lmax = pl.Lmax;
        gd.bl = ctx->bl; gd.blc = ctx->blc; gd.inb = ctx->inb;
    }
    int *hp = reinterpret_cast<int *>(ctx->h_stage + kStagePrev);
    {
        std::vector<int> last(pl.k, -1);
        for (int j = 0; j < pl.np; ++j) {
            hp[2 * j] = last[pl.pa[j]];
            hp[2 * j + 1] = last[pl.pb[j]];
            last[pl.pa[j]] = last[pl.pb[j]] = j;
        }
    }
    CK(cudaMemcpyAsync(ctx->q_graphs, hg, sizeof(GraphDev) * (size_t)clusters, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->q_prev, hp, sizeof(int) * 2 * (size_t)pl.np, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->part_backup, part, sizeof(int) * (size_t)g->n, cudaMemcpyDeviceToDevice, ctx->stream));

    QueueArgs q;
    memset(&q, 0, sizeof(q));
    q.wt = make_work(ctx, 0, 0, pl.np, g->n, opt);
    q.wt.vq_cap = (int)ctx->q_vq;
    q.wt.nu_cap = (int)ctx->q_nu;
    q.wt.mu_cap = (int)ctx->q_mu;
    q.wt.crank = ctx->q_crank;
    q.wt.total_n = g->n;
    q.wt.qb_sorted = ctx->qb_sorted;
    q.wt.qb_start = ctx->qb_start;
    q.wt.qb_app = ctx->qb_app;
    q.wt.qb_pool = ctx->qb_pool;
    q.wt.qb_lst = ctx->qb_lst;
    q.wt.qb_cap = ctx->qb_cap;
    q.slots = ctx->q_slots;
    q.np = pl.np;
    q.ticket = ctx->q_ticket;
    q.prev = ctx->q_prev;
    q.gabort = ctx->q_gabort;
    q.wait_ns = kWaitNs;

    auto enqueue = [&]() -> fr_status {
        CK(launch_fill_pairs(ctx->pairs, ctx->pair_a, ctx->pair_b, pl.np, 0, opt->mb ? 1 : 0, pl.Ubase, ctx->stream));
        CK(cudaMemsetAsync(ctx->sides, 0, sizeof(SideDev) * 2 * (size_t)pl.np, ctx->stream));
        CK(cudaMemsetAsync(ctx->pacc, 0, sizeof(PairAcc) * (size_t)pl.np, ctx->stream));
        CK(cudaMemsetAsync(ctx->q_ticket, 0, sizeof(int), ctx->stream));
        CK(cudaMemsetAsync(ctx->q_gabort, 0, sizeof(int), ctx->stream));
        CK(cudaMemsetAsync(ctx->q_ctls, 0, sizeof(fr_ctx::QCtl) * (size_t)clusters, ctx->stream));
        CK(cudaMemsetAsync(ctx->q_stats, 0, 4 * sizeof(long long) * (size_t)clusters, ctx->stream));
        CK(cudaMemsetAsync(ctx->qb_lst, 0xFF, sizeof(int) * (size_t)g->n, ctx->stream));
        CK(cudaMemsetAsync(ctx->qb_cnt, 0, sizeof(int) * (size_t)pl.k, ctx->stream));
        CK(launch_qb_build(ctx->bl, ctx->blc, part, pl.k, ctx->qb_cnt, ctx->qb_start, ctx->qb_app, ctx->qb_lst,
                           ctx->qb_sorted, ctx->stream));
        if (ctx->profiling) CK(cudaEventRecord(ctx->pev[0], ctx->stream));
        CK(launch_queue_sweep(q, ctas, clusters, ctx->stream));
        if (ctx->profiling) CK(cudaEventRecord(ctx->pev[1], ctx->stream));
        return FR_OK;
    };
    while (ctx->profiling && ctx->pev.size() < 2) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        ctx->pev.push_back(e);
    }
    // launches of the sweep: prep, compaction, colouring, pair fill, the three list
    // kernels, the queue kernel
    const long long launches = 8;
    std::vector<long long> key = {-7, (long long)(uintptr_t)g->xadj, (long long)(uintptr_t)part, g->n, g->nnz,
                                  pl.np, pl.Ubase, opt->mb, reps, (long long)opt->seed, opt->gr_interval,
                                  opt->inner_ops, opt->pulse_cap, (long long)(uintptr_t)ctx->base_mem,
                                  (long long)(uintptr_t)ctx->pair_mem, (long long)(uintptr_t)ctx->q_mem,
                                  ctx->tune_gr, ctx->tune_inner, opt->pulse_passes, ctx->tune_passes,
                                  opt->flow_sched, ctx->tune_sched, ctx->narrow_ok, opt->pre_waves,
                                  ctx->tune_prewaves, ctas, clusters, pl.Lmax, opt->gap_interval};
    ctx->prof.scan_ms = ctx->prof.step_ms = ctx->prof.cluster_ms = 0;
    ctx->round_ms.clear();
    ctx->pair_ms.clear();
    cudaGraphExec_t exec = nullptr;
    if (ctx->use_graphs && !ctx->profiling) {
        for (auto &e : ctx->gcache)
            if (e.key == key) { exec = e.exec; break; }
        if (!exec) {
            cudaGraph_t graph = nullptr;
            CK(cudaStreamSynchronize(ctx->stream));
            cudaError_t e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
            fr_status est = FR_OK;
            if (e == cudaSuccess) {
                est = enqueue();
                cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &graph);
                if (est == FR_OK && e2 == cudaSuccess && graph) {
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
                ctx->gcache.push_back({key, exec, launches});
            } else {
                ctx->use_graphs = false;
            }
        }
    }
    CK(cudaEventRecord(ctx->ev0, ctx->stream));
    if (exec) {
        CK(cudaGraphLaunch(exec, ctx->stream));
    } else {
        if ((st = enqueue()) != FR_OK) return st;
    }
    CK(cudaEventRecord(ctx->ev1, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaEventElapsedTime(ms, ctx->ev0, ctx->ev1));
    ctx->sweep_launches = launches;
    ctx->last_launches = launches;
    int gab = 0;
    CK(cudaMemcpyAsync(&gab, ctx->q_gabort, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    std::vector<fr_ctx::QCtl> qc(clusters);
    CK(cudaMemcpyAsync(qc.data(), ctx->q_ctls, sizeof(fr_ctx::QCtl) * (size_t)clusters, cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctls->resize(clusters);
    for (int i = 0; i < clusters; ++i) (*ctls)[i] = qc[i].c;
    ctx->last_queue_ctas = ctas;
    ctx->last_queue_clusters = clusters;
    if (gab != 0) {
        // leave part exactly as it was, and the workspace idle
        CK(cudaMemcpyAsync(part, ctx->part_backup, sizeof(int) * (size_t)g->n, cudaMemcpyDeviceToDevice, ctx->stream));
        if ((st = reset_queue_idle(ctx)) != FR_OK) return st;
        if (gab == E_MISFIT) {
            ++ctx->queue_fallbacks;
            int where = 0;
            for (const Ctl &x : *ctls)
                if (x.error == E_MISFIT) { where = x.error_where; break; }
            ctx_error(ctx, "queue sweep: a pair outgrew its cluster's workspace (check %d); ran round by round",
                      where);
            return FR_OK;   // *ran = false: the caller runs the sweep round by round
        }
        Ctl c;
        memset(&c, 0, sizeof(c));
        c.error = gab;
        for (const Ctl &x : *ctls)
            if (x.error) { c = x; break; }
        return status_from_ctl(ctx, c, "fr_refine_batch (queue sweep)");
    }
    if (ctx->profiling) {
        // the queue kernel alone; the setup launches before it (pair fill, clears, lists)
        float qk = 0.f, pre = 0.f;
        CK(cudaEventElapsedTime(&pre, ctx->ev0, ctx->pev[0]));
        CK(cudaEventElapsedTime(&qk, ctx->pev[0], ctx->pev[1]));
        ctx->prof.cluster_ms = qk;
        ctx->prof.scan_ms = pre;
        std::vector<PairAcc> A(pl.np);
        CK(cudaMemcpyAsync(A.data(), ctx->pacc, sizeof(PairAcc) * pl.np, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        unsigned long long first = ~0ull;
        for (int i = 0; i < pl.np; ++i)
            if (A[i].t1 && A[i].t0 < first) first = A[i].t0;
        ctx->pair_ms.assign(3 * (size_t)pl.np, 0.f);
        int r = 0;
        for (int i = 0; i < pl.np; ++i) {
            while (r + 1 < pl.nr && i >= pl.off[r + 1]) ++r;
            float *pm = &ctx->pair_ms[3 * (size_t)i];
            pm[0] = (float)r;
            pm[1] = A[i].t1 ? (float)((A[i].t0 - first) * 1e-6) : -1.f;
            pm[2] = A[i].t1 ? (float)((A[i].t1 - first) * 1e-6) : -1.f;
        }
    }
    *ran = true;
    return FR_OK;
}
