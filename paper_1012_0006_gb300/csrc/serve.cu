// Serving loop: continuous batching of refinement requests (fr_server_* in flowref.h).
//
// A request is one sweep of matching rounds (as fr_refine_batch) on a graph that
// is resident on the device.  A host thread drives the device in steps: each step
// is ONE persistent launch over the current round of every in-flight request --
// several graphs in one union network, every pair of every request refined side by
// side -- after which every request advances by one round.  Requests that arrive
// while others run are admitted between steps, as soon as an in-flight slot and
// enough arena bytes are free, so their work joins the next launch.  Pairs of
// different requests never interact, so a request's result does not depend on
// what it was batched with.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "api_internal.h"

using namespace fr;
using Clock = std::chrono::steady_clock;

namespace {

struct SGraph {
    int n = 0, nnz = 0;
    int *xadj = nullptr, *adjncy = nullptr, *adjwgt = nullptr, *vwgt = nullptr;
};

struct Req {
    fr_request r;
    std::vector<int32_t> part0;     // submitted partition (host)
    Clock::time_point t_submit, t_admit;
    // device state owned by the request (stream-ordered allocations)
    void *mem = nullptr;
    size_t bytes = 0;
    int *part = nullptr, *sob_round = nullptr, *pair_a = nullptr, *pair_b = nullptr, *pair_round = nullptr,
        *round_off = nullptr;
    unsigned int *qbits = nullptr, *used = nullptr;
    long long *blockw = nullptr;
    PrepOut *prep = nullptr;
    int n = 0, nnz = 0, k = 0;
    int npairs = 0, nrounds = 0, round = 0;
    std::vector<int> off;
    long long Ubase = 0, Lmax = 0, totcut = 0, dcut = 0, W = 0;
    int accepted = 0, maxw = 0;
    fr_status status = FR_OK;
};

struct Done {
    fr_response resp;
    std::vector<int32_t> part;
};

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// Device bytes a request holds while in flight: its own arrays plus its share of
// the union workspace (about 24 words per vertex, 5 per arc).
size_t request_footprint(int n, int nnz, int k) {
    const size_t own = align256(4ull * n) + align256(8ull * k) + align256(4ull * ((size_t)k * k + 31) / 32) +
                       align256(4ull * k * ((2 * k + 31) / 32)) + align256(8ull * k * k) +
                       3 * align256(4ull * ((size_t)k * (k - 1) / 2 + 1)) + align256(4ull * (2 * k + 2)) +
                       align256(sizeof(PrepOut));
    const size_t share = 112ull * n + 20ull * nnz;
    return own + share;
}

}  // namespace

struct fr_server {
    fr_server_config cfg;
    fr_ctx *ctx = nullptr;          // union workspace, stream, staging
    std::vector<SGraph> graphs;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> pending;
    std::vector<Req *> inflight;
    std::deque<Done> done;
    std::thread th;
    bool stop = false;
    size_t bytes_in_use = 0;
    long long steps = 0, admitted = 0, completed = 0;
    int max_concurrent = 0;
    // step descriptors
    GraphDev *d_graphs = nullptr;
    int graphs_cap = 0;
};

static void free_req_device(fr_server *S, Req *q) {
    if (q->mem) cudaFreeAsync(q->mem, S->ctx->stream);
    q->mem = nullptr;
}

// Admission: device state, upload of the partition, validation and rounds.
static fr_status admit(fr_server *S, Req *q) {
    fr_ctx *ctx = S->ctx;
    const SGraph &G = S->graphs[q->r.graph_id];
    const int n = G.n, k = q->k;
    q->n = n;
    q->nnz = G.nnz;
    size_t b = 0;
    auto sz = [&](size_t bytes) { size_t o = b; b += align256(bytes); return o; };
    const size_t o_part = sz(4ull * n), o_bw = sz(8ull * k), o_q = sz(4ull * (((size_t)k * k + 31) / 32)),
                 o_used = sz(4ull * k * ((2 * k + 31) / 32)), o_sob = sz(8ull * k * k),
                 o_pa = sz(4ull * ((size_t)k * (k - 1) / 2 + 1)), o_pb = sz(4ull * ((size_t)k * (k - 1) / 2 + 1)),
                 o_pr = sz(4ull * ((size_t)k * (k - 1) / 2 + 1)), o_ro = sz(4ull * (2 * k + 2)),
                 o_prep = sz(sizeof(PrepOut));
    if (cudaMallocAsync(&q->mem, b, ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        q->mem = nullptr;
        return FR_ERR_OOM;
    }
    q->bytes = b;
    char *m = reinterpret_cast<char *>(q->mem);
    q->part = reinterpret_cast<int *>(m + o_part);
    q->blockw = reinterpret_cast<long long *>(m + o_bw);
    q->qbits = reinterpret_cast<unsigned int *>(m + o_q);
    q->used = reinterpret_cast<unsigned int *>(m + o_used);
    q->sob_round = reinterpret_cast<int *>(m + o_sob);
    q->pair_a = reinterpret_cast<int *>(m + o_pa);
    q->pair_b = reinterpret_cast<int *>(m + o_pb);
    q->pair_round = reinterpret_cast<int *>(m + o_pr);
    q->round_off = reinterpret_cast<int *>(m + o_ro);
    q->prep = reinterpret_cast<PrepOut *>(m + o_prep);
    cudaStream_t st = ctx->stream;
    if (cudaMemcpyAsync(q->part, q->part0.data(), 4ull * n, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(q->prep, 0, sizeof(PrepOut), st) != cudaSuccess ||
        cudaMemsetAsync(q->blockw, 0, 8ull * k, st) != cudaSuccess ||
        cudaMemsetAsync(q->qbits, 0, 4ull * (((size_t)k * k + 31) / 32), st) != cudaSuccess ||
        launch_prep(G.xadj, G.adjncy, G.adjwgt, G.vwgt, q->part, n, G.nnz, k, q->blockw, q->qbits, q->prep, st) !=
            cudaSuccess ||
        launch_color(q->qbits, k, q->pair_a, q->pair_b, q->pair_round, q->round_off, q->sob_round, q->used, q->prep,
                     st) != cudaSuccess)
        return FR_ERR_CUDA;
    PrepOut po;
    if (cudaMemcpyAsync(&po, q->prep, sizeof(po), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return FR_ERR_CUDA;
    if (po.err) return po.err == E_TOO_LARGE ? FR_ERR_TOO_LARGE : FR_ERR_INVALID_ARG;
    q->npairs = po.npairs;
    q->nrounds = po.nrounds;
    q->totcut = po.totcut;
    q->W = po.W;
    q->maxw = po.maxw;
    q->Ubase = host_budget_base(po.W, k, q->r.eps, q->r.alpha);
    q->Lmax = host_lmax(po.W, po.maxc, k, q->r.eps);
    q->off.assign(q->nrounds + 1, 0);
    if (q->nrounds > 0 &&
        (cudaMemcpyAsync(q->off.data(), q->round_off, sizeof(int) * (q->nrounds + 1), cudaMemcpyDeviceToHost, st) !=
             cudaSuccess ||
         cudaStreamSynchronize(st) != cudaSuccess))
        return FR_ERR_CUDA;
    return FR_OK;
}

static void finish(fr_server *S, Req *q) {
    Done d;
    memset(&d.resp, 0, sizeof(d.resp));
    d.resp.tag = q->r.tag;
    d.resp.status = q->status;
    d.resp.npairs = q->npairs;
    d.resp.nrounds = q->nrounds;
    d.resp.accepted = q->accepted;
    d.resp.cut_before = q->totcut;
    d.resp.cut_after = q->totcut + q->dcut;
    d.part.resize(q->n);
    bool copied = false;
    if (q->status == FR_OK && q->part) {
        copied = cudaMemcpyAsync(d.part.data(), q->part, 4ull * q->n, cudaMemcpyDeviceToHost, S->ctx->stream) ==
                     cudaSuccess &&
                 cudaStreamSynchronize(S->ctx->stream) == cudaSuccess;
    }
    if (!copied) {                 // failed requests return their partition unchanged
        d.part = q->part0;
        d.resp.cut_after = d.resp.cut_before;
        if (q->status == FR_OK) d.resp.status = FR_ERR_CUDA;
    }
    auto now = Clock::now();
    d.resp.latency_ms = std::chrono::duration<double, std::milli>(now - q->t_submit).count();
    d.resp.queue_ms = std::chrono::duration<double, std::milli>(q->t_admit - q->t_submit).count();
    free_req_device(S, q);
    std::lock_guard<std::mutex> lk(S->mu);
    S->bytes_in_use -= request_footprint(q->n, q->nnz, q->k);
    S->done.push_back(std::move(d));
    ++S->completed;
    S->cv_done.notify_all();
    delete q;
}

// One device step: the current round of every in-flight request in one launch.
static fr_status run_step(fr_server *S, std::vector<Req *> &act) {
    fr_ctx *ctx = S->ctx;
    cudaStream_t st = ctx->stream;
    long long totn = 0, totm = 0;
    int P = 0, kmax = 2;
    std::vector<int> pbase(act.size());
    for (size_t i = 0; i < act.size(); ++i) {
        Req *q = act[i];
        totn += q->n;
        totm += q->nnz;
        pbase[i] = P;
        P += q->off[q->round + 1] - q->off[q->round];
        kmax = std::max(kmax, q->k);
    }
    if (totn > INT32_MAX || totm > INT32_MAX) return FR_ERR_TOO_LARGE;
    const int reps = S->cfg.opt.mb_reps > 0 ? S->cfg.opt.mb_reps : 1;
    fr_status s = ensure_base(ctx, (int)totn, (int)totm, kmax, reps);
    if (s == FR_OK) s = ensure_pairs(ctx, P, 1, reps);
    if (s != FR_OK) return s;
    if ((int)act.size() > S->graphs_cap) {
        if (S->d_graphs) cudaFreeAsync(S->d_graphs, st);
        S->graphs_cap = std::max<int>((int)act.size(), 2 * S->graphs_cap);
        if (cudaMallocAsync(&S->d_graphs, sizeof(GraphDev) * S->graphs_cap, st) != cudaSuccess) return FR_ERR_OOM;
    }
    std::vector<GraphDev> gds(act.size());
    long long base = 0, ebase = 0;
    for (size_t i = 0; i < act.size(); ++i) {
        Req *q = act[i];
        const SGraph &G = S->graphs[q->r.graph_id];
        GraphDev &gd = gds[i];
        memset(&gd, 0, sizeof(gd));
        gd.xadj = G.xadj; gd.adjncy = G.adjncy; gd.adjwgt = G.adjwgt; gd.vwgt = G.vwgt;
        gd.part = q->part;
        gd.dist = ctx->dist + base;
        gd.lid = ctx->lid + base;
        gd.sob = q->sob_round + (long long)q->round * q->k;
        gd.blockw = q->blockw;
        gd.n = q->n; gd.nnz = q->nnz; gd.k = q->k; gd.base = (int)base; gd.Lmax = q->Lmax;
        gd.sbase = 2 * pbase[i];
        gd.ebase = (int)ebase;
        base += q->n;
        ebase += q->nnz;
    }
    memcpy(ctx->h_stage + 65536, gds.data(), sizeof(GraphDev) * gds.size());
    if (cudaMemcpyAsync(S->d_graphs, ctx->h_stage + 65536, sizeof(GraphDev) * gds.size(), cudaMemcpyHostToDevice,
                        st) != cudaSuccess)
        return FR_ERR_CUDA;
    const fr_options &opt = S->cfg.opt;
    for (size_t i = 0; i < act.size(); ++i) {
        Req *q = act[i];
        const int np = q->off[q->round + 1] - q->off[q->round];
        if (launch_fill_pairs(ctx->pairs + pbase[i], q->pair_a + q->off[q->round], q->pair_b + q->off[q->round], np,
                              (int)i, opt.mb ? 1 : 0, q->Ubase, st) != cudaSuccess)
            return FR_ERR_CUDA;
    }
    if (cudaMemsetAsync(ctx->ctl, 0, sizeof(Ctl), st) != cudaSuccess ||
        cudaMemsetAsync(ctx->sides, 0, sizeof(SideDev) * 2 * P, st) != cudaSuccess ||
        cudaMemsetAsync(ctx->pacc, 0, sizeof(PairAcc) * P, st) != cudaSuccess ||
        cudaMemsetAsync(ctx->hist, 0, sizeof(long long) * 3 * 2 * (size_t)P * kHistBins, st) != cudaSuccess)
        return FR_ERR_CUDA;
    Work w = make_work(ctx, 0, 0, P, (int)totn, &opt);
    w.narrow = 1;
    for (const Req *q : act) w.narrow &= q->maxw < (1 << 15) ? 1 : 0;
    w.graphs = S->d_graphs;
    w.ngraphs = (int)act.size();
    w.prev_err = nullptr;
    for (size_t i = 0; i < act.size(); ++i) {
        const bool vec = (reinterpret_cast<uintptr_t>(gds[i].adjncy) & 15) == 0;
        if (launch_scan(w, (int)i, act[i]->n, vec, st) != cudaSuccess) return FR_ERR_CUDA;
    }
    long long est = 0;
    for (size_t i = 0; i < act.size(); ++i)
        est += 2LL * (act[i]->off[act[i]->round + 1] - act[i]->off[act[i]->round]) *
               std::max<long long>(1, act[i]->Ubase / std::max(1, act[i]->k));
    const int tpb = choose_tpb(ctx, &opt);
    const int grid = choose_grid(ctx, &opt, tpb, 2 * P, std::max<long long>(1, est));
    long long emax = 0;   // corridor vertices of the largest pair: two sides of (Ubase - W/k) weight
    for (size_t i = 0; i < act.size(); ++i) {
        const Req *q = act[i];
        const double avgc = std::max(1.0, (double)q->W / q->n);
        const long long side = std::max(0LL, q->Ubase - q->W / q->k);
        emax = std::max(emax, (long long)(2.0 * side / avgc));
    }
    if (launch_round(ctx, w, grid, tpb, st, nullptr, emax, (double)totm / std::max(1LL, totn), opt.cluster_ctas) !=
        cudaSuccess)
        return FR_ERR_CUDA;
    std::vector<PairAcc> A(P);
    Ctl C;
    if (cudaMemcpyAsync(A.data(), ctx->pacc, sizeof(PairAcc) * P, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&C, ctx->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return FR_ERR_CUDA;
    if (C.error) {
        reset_idle(ctx);
        return status_from_ctl(ctx, C, "serving step");
    }
    for (size_t i = 0; i < act.size(); ++i) {
        Req *q = act[i];
        const int np = q->off[q->round + 1] - q->off[q->round];
        for (int j = 0; j < np; ++j) {
            const PairAcc &a = A[pbase[i] + j];
            if (a.accept) {
                q->accepted += 1;
                q->dcut += a.dcut;
            }
        }
        q->round += 1;
    }
    return FR_OK;
}

static void server_loop(fr_server *S) {
    cudaSetDevice(S->cfg.device);
    for (;;) {
        std::vector<Req *> admit_now;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->inflight.empty())
                S->cv_work.wait(lk, [&] { return S->stop || !S->pending.empty(); });
            if (S->stop && S->pending.empty() && S->inflight.empty()) return;
            while (!S->pending.empty() && (int)(S->inflight.size() + admit_now.size()) < S->cfg.max_inflight) {
                Req *q = S->pending.front();
                const size_t f = request_footprint(S->graphs[q->r.graph_id].n, S->graphs[q->r.graph_id].nnz, q->k);
                const bool fits = S->cfg.arena_bytes == 0 || S->bytes_in_use + f <= S->cfg.arena_bytes;
                const bool alone = S->inflight.empty() && admit_now.empty();
                if (!fits && !alone) break;   // wait until in-flight requests free memory
                S->pending.pop_front();
                S->bytes_in_use += f;
                admit_now.push_back(q);
            }
        }
        for (Req *q : admit_now) {
            q->t_admit = Clock::now();
            q->status = admit(S, q);
            if (q->status != FR_OK || q->nrounds == 0) {
                finish(S, q);
                continue;
            }
            std::lock_guard<std::mutex> lk(S->mu);
            S->inflight.push_back(q);
            ++S->admitted;
            S->max_concurrent = std::max<int>(S->max_concurrent, (int)S->inflight.size());
        }
        std::vector<Req *> act;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            act = S->inflight;
        }
        if (act.empty()) continue;
        fr_status st = run_step(S, act);
        ++S->steps;
        std::vector<Req *> keep;
        for (Req *q : act) {
            if (st != FR_OK) q->status = st;
            if (st != FR_OK || q->round >= q->nrounds) finish(S, q);
            else keep.push_back(q);
        }
        std::lock_guard<std::mutex> lk(S->mu);
        S->inflight = keep;
    }
}

extern "C" fr_status fr_server_create(fr_server **out, const fr_server_config *cfg) {
    if (!out || !cfg || cfg->max_inflight < 1 || cfg->opt.fm_permille != 0 || cfg->opt.mt_alpha != 0) return FR_ERR_INVALID_ARG;
    *out = nullptr;
    fr_server *S = new fr_server();
    S->cfg = *cfg;
    if (S->cfg.opt.mb_reps < 1) S->cfg.opt.mb_reps = 1;
    fr_status st = fr_create(&S->ctx, cfg->device, 0, nullptr);
    if (st != FR_OK) {
        delete S;
        return st;
    }
    S->th = std::thread(server_loop, S);
    *out = S;
    return FR_OK;
}

extern "C" fr_status fr_server_add_graph(fr_server *S, int32_t n, int32_t nnz, const int32_t *xadj,
                                         const int32_t *adjncy, const int32_t *adjwgt, const int32_t *vwgt,
                                         int32_t *graph_id) {
    if (!S || n < 1 || nnz < 0 || !xadj || !vwgt || (nnz > 0 && (!adjncy || !adjwgt)) || !graph_id)
        return FR_ERR_INVALID_ARG;
    cudaSetDevice(S->cfg.device);
    SGraph G;
    G.n = n;
    G.nnz = nnz;
    const size_t bx = align256(4ull * (n + 1)), ba = align256(4ull * std::max(nnz, 1)), bv = align256(4ull * n);
    char *m = nullptr;
    if (cudaMalloc(&m, bx + 2 * ba + bv) != cudaSuccess) {
        cudaGetLastError();
        return FR_ERR_OOM;
    }
    G.xadj = reinterpret_cast<int *>(m);
    G.adjncy = reinterpret_cast<int *>(m + bx);
    G.adjwgt = reinterpret_cast<int *>(m + bx + ba);
    G.vwgt = reinterpret_cast<int *>(m + bx + 2 * ba);
    if (cudaMemcpy(G.xadj, xadj, 4ull * (n + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
        (nnz && cudaMemcpy(G.adjncy, adjncy, 4ull * nnz, cudaMemcpyHostToDevice) != cudaSuccess) ||
        (nnz && cudaMemcpy(G.adjwgt, adjwgt, 4ull * nnz, cudaMemcpyHostToDevice) != cudaSuccess) ||
        cudaMemcpy(G.vwgt, vwgt, 4ull * n, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(m);
        return FR_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    S->graphs.push_back(G);
    *graph_id = (int32_t)S->graphs.size() - 1;
    return FR_OK;
}

extern "C" fr_status fr_server_submit(fr_server *S, const fr_request *req) {
    if (!S || !req || !req->part_host) return FR_ERR_INVALID_ARG;
    Req *q = new Req();
    q->r = *req;
    q->k = req->k;
    q->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (req->graph_id < 0 || req->graph_id >= (int)S->graphs.size() || req->k < 2 || req->k > kMaxK ||
            !(req->eps > 0.0) || !(req->alpha >= 1.0)) {
            delete q;
            return FR_ERR_INVALID_ARG;
        }
        const int n = S->graphs[req->graph_id].n;
        q->part0.assign(req->part_host, req->part_host + n);
        S->pending.push_back(q);
    }
    S->cv_work.notify_one();
    return FR_OK;
}

extern "C" fr_status fr_server_next(fr_server *S, fr_response *resp, int32_t *part_out, int32_t part_cap,
                                    int32_t timeout_ms) {
    if (!S || !resp) return FR_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto ready = [&] { return !S->done.empty(); };
    if (timeout_ms < 0) S->cv_done.wait(lk, ready);
    else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) return FR_ERR_ABORTED;
    Done d = std::move(S->done.front());
    S->done.pop_front();
    lk.unlock();
    *resp = d.resp;
    if (part_out && part_cap >= (int32_t)d.part.size()) memcpy(part_out, d.part.data(), 4 * d.part.size());
    return FR_OK;
}

extern "C" fr_status fr_server_stats(fr_server *S, int64_t *steps, int64_t *admitted, int64_t *completed,
                                     int32_t *max_concurrent) {
    if (!S) return FR_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    if (steps) *steps = S->steps;
    if (admitted) *admitted = S->admitted;
    if (completed) *completed = S->completed;
    if (max_concurrent) *max_concurrent = S->max_concurrent;
    return FR_OK;
}

extern "C" fr_status fr_server_destroy(fr_server *S) {
    if (!S) return FR_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->th.joinable()) S->th.join();
    cudaSetDevice(S->cfg.device);
    for (Req *q : S->pending) delete q;
    for (auto &G : S->graphs) cudaFree(G.xadj);
    if (S->d_graphs) cudaFreeAsync(S->d_graphs, S->ctx->stream);
    cudaStreamSynchronize(S->ctx->stream);
    fr_destroy(S->ctx);
    delete S;
    return FR_OK;
}
