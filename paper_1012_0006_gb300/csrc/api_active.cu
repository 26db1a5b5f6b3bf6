// C ABI, part 3: active block scheduling (Sanders & Schulz, Section 4.3 and the
// appendix pseudocode of active block scheduling) with the flow refinement of
// Section 4.1 as the pairwise step, and adaptive flow iterations per pair.
//
// Every block starts active.  An outer round takes the quotient edges (a, b) of the
// current partition with a or b active, marks every block inactive, colours the
// edges into matchings (lexicographic order, smallest colour free at both ends, as
// for the sweep's rounds) and refines the pairs matching by matching; a pair whose
// refinement changed the partition marks a and b active.  The run ends when no
// block is active or after max_outer outer rounds.  With mt_alpha > 0 a multi-try FM
// pass (Section 4.2) over the matching's pairs follows their pairwise steps, and every
// block one of its kept moves left or entered becomes active.  Inside a matching every
// pair runs its own adaptive loop; the pairs still iterating go through the round kernels
// together, each with its own corridor budget, so a step is one launch sequence for
// all of them (the pairs are block-disjoint, so their iterations do not interact).
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

struct StepPair {
    int a, b;
    long long Ubase;
};

struct StepOut {
    long long flow, oldcut, newcut, cA, cB, nA, nB;
    int nc, m, accept, feasible;
    long long pulses, relabels;
    FmRes fm;   // the FM step before this iteration (fm_first)
};

// One flow iteration of block-disjoint pairs, each with its budget base: scan, step,
// cluster and step kernels over their union network.  Accepted pairs are applied
// to part (and the device block weights) by the commit phase.  fm_first: the FM step
// of every pair runs first (the pairwise improvement is FM, then the flows).
fr_status run_pairs_step(fr_ctx *ctx, const fr_graph *g, int32_t *part, int32_t k, const std::vector<StepPair> &ps,
                         long long Lmax, long long W, const fr_options *opt, bool fm_first,
                         std::vector<StepOut> &out) {
    const int P = (int)ps.size();
    const int reps = opt->mb_reps > 0 ? opt->mb_reps : 1;
    fr_status st = ensure_pairs(ctx, P, 1, reps);
    if (st != FR_OK) return st;
    // staging in the pinned buffer: graph descriptor, pair descriptors, block -> side
    char *h = ctx->h_stage + 4096;
    GraphDev gd;
    memset(&gd, 0, sizeof(gd));
    gd.xadj = g->xadj; gd.adjncy = g->adjncy; gd.adjwgt = g->adjwgt; gd.vwgt = g->vwgt;
    gd.part = part; gd.dist = ctx->dist; gd.lid = ctx->lid; gd.sob = ctx->sob1; gd.blockw = ctx->blockw;
    gd.n = g->n; gd.nnz = g->nnz; gd.k = k; gd.base = 0; gd.Lmax = Lmax;
    gd.bl = ctx->bl; gd.blc = ctx->blc; gd.inb = ctx->inb;
    memcpy(h, &gd, sizeof(gd));
    PairDev *hp = reinterpret_cast<PairDev *>(h + 1024);
    int *hs = reinterpret_cast<int *>(hp + P);
    if ((size_t)((char *)(hs + k) - ctx->h_stage) > kHostStage) {
        ctx_error(ctx, "active scheduling: %d pairs / k = %d exceed the staging buffer", P, k);
        return FR_ERR_TOO_LARGE;
    }
    for (int x = 0; x < k; ++x) hs[x] = -1;
    for (int i = 0; i < P; ++i) {
        hp[i].g = 0; hp[i].a = ps[i].a; hp[i].b = ps[i].b; hp[i].mb = opt->mb ? 1 : 0; hp[i].Ubase = ps[i].Ubase;
        hs[ps[i].a] = 2 * i;
        hs[ps[i].b] = 2 * i + 1;
    }
    CK(cudaMemcpyAsync(ctx->graphs, h, sizeof(gd), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->pairs, hp, sizeof(PairDev) * P, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->sob1, hs, sizeof(int) * k, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemsetAsync(ctx->ctl, 0, sizeof(Ctl), ctx->stream));
    CK(cudaMemsetAsync(ctx->sides, 0, sizeof(SideDev) * 2 * P, ctx->stream));
    CK(cudaMemsetAsync(ctx->pacc, 0, sizeof(PairAcc) * P, ctx->stream));
    CK(cudaMemsetAsync(ctx->hist, 0, sizeof(long long) * 3 * 2 * (size_t)P * kHistBins, ctx->stream));
    Work w = make_work(ctx, 0, 0, P, g->n, opt);
    const int tpb = choose_tpb(ctx, opt);
    const double avgc = std::max(1.0, (double)W / g->n);
    long long est = 0, emax = 0;
    for (const StepPair &p : ps) {
        const long long e1 = (long long)(2.0 * (double)std::max(0LL, p.Ubase - W / k) / avgc);
        est += e1;
        emax = std::max(emax, e1);
    }
    const int grid = choose_grid(ctx, opt, tpb, 2 * P, std::max(1LL, est));
    if (fm_first) {
        int nf = 0;
        CK(launch_fm(w, fm_view(ctx, 0, opt), k, ctx->sms, ctx->stream, &nf));
    }
    CK(launch_scan_list(w, 0, ctx->stream));
    CK(launch_round(ctx, w, grid, tpb, ctx->stream, nullptr, emax, (double)g->nnz / g->n,
                    opt->cluster_ctas ? opt->cluster_ctas : ctx->tune_ctas));
    PairAcc *ha = reinterpret_cast<PairAcc *>(ctx->h_stage + (kHostStage / 2));
    SideDev *hsd = reinterpret_cast<SideDev *>(ha + P);
    Ctl *hc = reinterpret_cast<Ctl *>(hsd + 2 * P);
    FmRes *hf = reinterpret_cast<FmRes *>(hc + 1);
    if ((size_t)((char *)(hf + P) - ctx->h_stage) > kHostStage) {
        ctx_error(ctx, "active scheduling: %d pairs exceed the staging buffer", P);
        return FR_ERR_TOO_LARGE;
    }
    if (fm_first) CK(cudaMemcpyAsync(hf, ctx->fm.res, sizeof(FmRes) * P, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(ha, ctx->pacc, sizeof(PairAcc) * P, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(hsd, ctx->sides, sizeof(SideDev) * 2 * P, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(hc, ctx->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    st = status_from_ctl(ctx, *hc, "fr_refine_active");
    if (st != FR_OK) {
        reset_idle(ctx);
        return st;
    }
    out.resize(P);
    for (int i = 0; i < P; ++i) {
        StepOut &o = out[i];
        o.flow = ha[i].flow;
        o.oldcut = ha[i].oldcut;
        o.newcut = ha[i].oldcut + ha[i].dcut;
        o.cA = hsd[2 * i].cw;
        o.cB = hsd[2 * i + 1].cw;
        o.nA = o.cA + ha[i].dwA;
        o.nB = o.cB - ha[i].dwA;
        o.nc = ha[i].nc;
        o.m = ha[i].m;
        o.accept = ha[i].accept;
        o.feasible = ha[i].feasible;
        o.pulses = hc->pulses;
        o.relabels = hc->relabels;
        if (fm_first) o.fm = hf[i];
        else memset(&o.fm, 0, sizeof(o.fm));
    }
    return FR_OK;
}

struct PairRun {
    int a, b;
    double al;
    int iters, accepted, running, fm_moves;
    long long cut_before, wA0, wB0, cut_fm, cur_cut, cur_A, cur_B, flow;
    int nc, m;
    long long pulses, relabels;
};

}  // namespace

extern "C" fr_status fr_refine_active(fr_ctx *ctx, const fr_graph *g, int32_t *part, int32_t k, double eps,
                                      double alpha, const fr_options *opt_in, int32_t max_outer, int32_t cap,
                                      fr_pair_result *results, fr_batch_result *summary, int32_t *nouter) {
    if (!ctx) return FR_ERR_INVALID_ARG;
    fr_options opt;
    if (opt_in) opt = *opt_in; else fr_default_options(&opt);
    if (summary) memset(summary, 0, sizeof(*summary));
    if (nouter) *nouter = 0;
    fr_status st = check_graph(ctx, g, part, k);
    if (st == FR_OK) st = check_params(ctx, eps, alpha, &opt);
    if (st == FR_OK && (max_outer < 1 || cap < 0 || (cap > 0 && !results))) {
        ctx_error(ctx, "max_outer must be >= 1 and results must hold cap entries");
        st = FR_ERR_INVALID_ARG;
    }
    if (st != FR_OK) { if (summary) summary->status = st; return st; }
    CK(cudaSetDevice(ctx->device));
    release_corridor(ctx);
    st = ensure_base(ctx, g->n, g->nnz, k, opt.mb_reps);
    if (st == FR_OK && opt.fm_permille > 0) st = ensure_fm(ctx, g->n, g->nnz, k, k / 2 + 1);
    if (st == FR_OK && opt.mt_alpha > 0) st = ensure_mt(ctx, g->n, g->nnz, k, k / 2 + 1);
    if (st != FR_OK) { if (summary) summary->status = st; return st; }
    CK(cudaMemcpyAsync(ctx->part_backup, part, sizeof(int) * (size_t)g->n, cudaMemcpyDeviceToDevice, ctx->stream));
    const int adaptive = opt.adaptive ? 1 : 0;
    const int max_iters = adaptive ? (opt.max_iters > 0 ? opt.max_iters : 10) : 1;
    const double alpha_max = adaptive ? opt.alpha_max : alpha;
    cudaEvent_t e0 = ctx->ev0, e1 = ctx->ev1;
    CK(cudaEventRecord(e0, ctx->stream));
    std::vector<char> active(k, 1);
    std::vector<unsigned int> qb(((size_t)k * k + 31) / 32);
    long long W = 0, Lmax = 0, cut0 = 0, dcut_total = 0, corridor_arcs = 0;
    int out_n = 0, rounds_total = 0, accepted_total = 0, outer = 0;
    MtRes mt_tot;
    memset(&mt_tot, 0, sizeof(mt_tot));
    std::vector<int8_t> changed(k);
    for (; outer < max_outer && st == FR_OK; ++outer) {
        if (std::find(active.begin(), active.end(), 1) == active.end()) break;
        PrepOut po;
        st = run_prep(ctx, g, part, k, true, outer == 0 && opt.checked != 0, &po);
        if (st != FR_OK) break;
        if (outer == 0) {
            W = po.W;
            Lmax = host_lmax(W, po.maxc, k, eps);
            cut0 = po.totcut;
            if (opt.mt_alpha > 0 && po.maxwdeg > kMtGmax) {
                ctx_error(ctx, "multi-try: max weighted degree %d exceeds %d", po.maxwdeg, kMtGmax);
                st = FR_ERR_TOO_LARGE;
                break;
            }
        }
        CK(cudaMemcpy(qb.data(), ctx->qbits, sizeof(unsigned int) * qb.size(), cudaMemcpyDeviceToHost));
        // the quotient edges with an active end, coloured into matchings
        std::vector<int> pa, pb, pr;
        std::vector<std::vector<char>> used(k);
        int nr = 0;
        for (int a = 0; a < k; ++a)
            for (int b = a + 1; b < k; ++b) {
                const size_t bit = (size_t)a * k + b;
                if (!((qb[bit >> 5] >> (bit & 31)) & 1u) || !(active[a] || active[b])) continue;
                int c = 0;
                while ((c < (int)used[a].size() && used[a][c]) || (c < (int)used[b].size() && used[b][c])) ++c;
                for (int x : {a, b}) {
                    if ((int)used[x].size() <= c) used[x].resize(c + 1, 0);
                    used[x][c] = 1;
                }
                pa.push_back(a); pb.push_back(b); pr.push_back(c);
                nr = std::max(nr, c + 1);
            }
        std::fill(active.begin(), active.end(), 0);
        for (int r = 0; r < nr && st == FR_OK; ++r) {
            std::vector<PairRun> run;
            for (size_t i = 0; i < pa.size(); ++i) {
                if (pr[i] != r) continue;
                PairRun q;
                memset(&q, 0, sizeof(q));
                q.a = pa[i]; q.b = pb[i]; q.al = alpha; q.running = 1; q.cut_before = -1;
                run.push_back(q);
            }
            // FM first (once), then adaptive flow iterations (Section 4.1), every pair on
            // its own alpha
            for (bool first = true;; first = false) {
                std::vector<StepPair> ps;
                std::vector<int> idx;
                for (size_t i = 0; i < run.size(); ++i)
                    if (run[i].running) {
                        ps.push_back({run[i].a, run[i].b, host_budget_base(W, k, eps, run[i].al)});
                        idx.push_back((int)i);
                    }
                if (ps.empty()) break;
                std::vector<StepOut> outs;
                const bool fm_first = first && opt.fm_permille > 0;
                st = run_pairs_step(ctx, g, part, k, ps, Lmax, W, &opt, fm_first, outs);
                if (st != FR_OK) break;
                for (size_t j = 0; j < ps.size(); ++j) {
                    PairRun &q = run[idx[j]];
                    const StepOut &o = outs[j];
                    ++q.iters;
                    if (q.cut_before < 0) {
                        q.cut_before = o.oldcut; q.wA0 = o.cA; q.wB0 = o.cB; q.cut_fm = o.oldcut;
                        if (fm_first) {
                            q.cut_before = o.fm.cut0; q.wA0 = o.fm.wA0; q.wB0 = o.fm.wB0;
                            q.fm_moves = o.fm.kept;
                        }
                    }
                    q.cur_cut = o.oldcut; q.cur_A = o.cA; q.cur_B = o.cB;
                    q.flow = o.flow; q.nc = o.nc; q.m = o.m; q.pulses = o.pulses; q.relabels = o.relabels;
                    corridor_arcs += o.m;
                    if (o.accept) { q.cur_cut = o.newcut; q.cur_A = o.nA; q.cur_B = o.nB; q.accepted = 1; }
                    bool go;
                    if (o.feasible && o.newcut < o.oldcut) {
                        go = adaptive != 0;
                        if (go) q.al = 2.0 * q.al < alpha_max ? 2.0 * q.al : alpha_max;
                    } else if (o.feasible) {
                        go = false;
                    } else {
                        go = adaptive && q.al != 1.0;
                        if (go) q.al = q.al / 2.0 > 1.0 ? q.al / 2.0 : 1.0;
                    }
                    q.running = go && q.iters < max_iters;
                }
            }
            if (st != FR_OK) break;
            if (opt.mt_alpha > 0) {
                // the multi-try pass from the boundaries of the matching's pairs
                std::vector<int32_t> ma, mb;
                for (const PairRun &q : run) { ma.push_back(q.a); mb.push_back(q.b); }
                MtRes m;
                st = run_mt_pass(ctx, g, part, k, ma.data(), mb.data(), (int)ma.size(), Lmax, opt.mt_alpha, opt.seed,
                                 true, &m, changed.data());
                if (st != FR_OK) break;
                for (int x = 0; x < k; ++x)
                    if (changed[x]) active[x] = 1;
                mt_tot.gain += m.gain;
                mt_tot.searches += m.searches;
                mt_tot.tried += m.tried;
                mt_tot.kept += m.kept;
            }
            for (const PairRun &q : run) {
                if (q.accepted || q.fm_moves > 0) active[q.a] = active[q.b] = 1;   // partition changed
                accepted_total += q.accepted;
                dcut_total += q.cur_cut - q.cut_before;
                if (out_n < cap) {
                    fr_pair_result &res = results[out_n];
                    memset(&res, 0, sizeof(res));
                    res.status = FR_OK;
                    res.a = q.a; res.b = q.b; res.round = rounds_total + r;
                    res.iters = q.iters;
                    res.alpha_final = q.al;
                    res.flow = q.flow;
                    res.cut_before = q.cut_before;
                    res.wA_before = q.wA0; res.wB_before = q.wB0;
                    res.cut_after = q.cur_cut; res.wA_after = q.cur_A; res.wB_after = q.cur_B;
                    res.corridor_n = q.nc; res.corridor_arcs = q.m;
                    res.accepted = q.accepted;
                    res.pulses = q.pulses; res.relabels = q.relabels;
                    res.cut_fm = q.cut_fm; res.fm_moves = q.fm_moves;
                }
                ++out_n;
            }
        }
        rounds_total += nr;
    }
    if (st != FR_OK) {
        // leave part exactly as it was
        cudaMemcpyAsync(part, ctx->part_backup, sizeof(int) * (size_t)g->n, cudaMemcpyDeviceToDevice, ctx->stream);
        cudaStreamSynchronize(ctx->stream);
        if (summary) summary->status = st;
        return st;
    }
    CK(cudaEventRecord(e1, ctx->stream));
    CK(cudaEventSynchronize(e1));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    if (summary) {
        summary->npairs = out_n;
        summary->nrounds = rounds_total;
        summary->accepted = accepted_total;
        summary->status = FR_OK;
        summary->cut_before = cut0;
        summary->cut_after = cut0 + dcut_total - mt_tot.gain;
        summary->mt_gain = mt_tot.gain;
        summary->mt_searches = mt_tot.searches;
        summary->mt_tried = mt_tot.tried;
        summary->mt_kept = mt_tot.kept;
        summary->corridor_arcs = corridor_arcs;
        summary->device_ns = (int64_t)((double)ms * 1e6);
    }
    if (nouter) *nouter = outer;
    return FR_OK;
}
