// Context and host-side helpers shared by the C-ABI translation units.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "flowref.h"
#include "fr_internal.cuh"
#include "round_kernel.cuh"
#include "fm_kernel.cuh"
#include "mt_kernel.cuh"
#include "queue_sweep.cuh"

constexpr int kMaxK = 1024;                 // blocks per partition (quotient graph in device bitmaps)
constexpr size_t kHostStage = 8u << 20;     // pinned staging for small host<->device copies

struct GraphCacheEntry {
    std::vector<long long> key;
    cudaGraphExec_t exec = nullptr;
    long long launches = 0;   // kernels in the captured sweep
};

struct fr_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t arena_limit = 0;
    char err[512] = {0};
    int sms = 0, max_coop = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    char *h_stage = nullptr;
    // launch shape (fr_autotune writes these)
    int tune_tpb = 512, tune_grid = 0, tune_gr = 16, tune_inner = 2, tune_passes = 2;
    int tune_ctas = 0;   // first cluster size (0: by the estimated corridor size)
    int tune_sched = 0;  // cluster max-flow schedule (fr_options.flow_sched)
    int tune_prewaves = 0;   // waves before the first pulse (fr_options.pre_waves)
    int narrow_ok = 0;   // the last prep found every edge weight < 2^15 (packed residuals in clusters)
    // per-pair max flow in thread-block clusters of kClusterSizes[t] CTAs: how many of
    // each can be resident (all 0: grid-wide path only); max_clusters = the largest
    static constexpr int kNumClusterSizes = 5;
    static constexpr int kClusterSizes[kNumClusterSizes] = {4, 6, 8, 12, 16};
    int cl_cap[kNumClusterSizes] = {0, 0, 0, 0, 0};
    int max_clusters = 0;
    int round_launches = 0;   // kernels the last launch_round enqueued
    // graph-size workspace
    void *base_mem = nullptr;
    size_t base_bytes = 0;
    int n_cap = 0, nnz_cap = 0, k_cap = 0, reps_cap = 0;
    int *dist = nullptr, *lid = nullptr, *vq_v = nullptr, *vq_s = nullptr;
    unsigned int *cbits = nullptr;
    int *bl = nullptr, *blc = nullptr, *inb = nullptr;   // boundary candidates of the current sweep
    int *gid = nullptr, *sid = nullptr, *off = nullptr, *infc = nullptr, *fx = nullptr, *lab = nullptr;
    int *rflag = nullptr, *color = nullptr, *scc = nullptr, *vc = nullptr, *fq0 = nullptr, *fq1 = nullptr;
    int *spare = nullptr;
    long long *ex = nullptr;
    unsigned char *border = nullptr, *side_out = nullptr;
    int *head = nullptr, *rev = nullptr, *res = nullptr, *cap = nullptr;
    int *cta_cnt = nullptr;
    long long *cw = nullptr;
    int *cpair = nullptr, *cmin = nullptr, *cid = nullptr, *indeg = nullptr, *outoff = nullptr, *ocur = nullptr;
    int *plist = nullptr, *sinkc = nullptr, *part_backup = nullptr, *outs = nullptr;
    int *indeg_r = nullptr, *order = nullptr, *hcomp = nullptr;
    unsigned long long *hkey = nullptr;
    long long *blockw = nullptr;
    unsigned int *qbits = nullptr, *used = nullptr;
    int *sob_round = nullptr, *pair_a = nullptr, *pair_b = nullptr, *pair_round = nullptr, *round_off = nullptr;
    fr::PrepOut *prep = nullptr;
    int *sob1 = nullptr, *flags = nullptr;
    // pair-count workspace
    void *pair_mem = nullptr;
    size_t pair_bytes = 0;
    int pairs_cap = 0, rounds_cap = 0;
    // sweep-count workspace
    void *reps_mem = nullptr;
    size_t reps_bytes = 0;
    long long reps_nu = 0, reps_P = 0;
    fr::GraphDev *graphs = nullptr;
    fr::PairDev *pairs = nullptr;
    fr::SideDev *sides = nullptr;
    fr::PairAcc *pacc = nullptr;
    fr::Ctl *ctl = nullptr;
    long long *hist = nullptr;
    int *pcur = nullptr;
    long long *sw_absd = nullptr;
    int *sw_j = nullptr;
    // corridor handle state
    unsigned long long gen = 0;
    fr_corridor *live = nullptr;
    bool dirty = false;
    // device copies of host graphs (fr_refine_batch_host)
    void *hg_mem = nullptr;
    size_t hg_bytes = 0;
    int *hg_xadj = nullptr, *hg_adjncy = nullptr, *hg_adjwgt = nullptr, *hg_vwgt = nullptr, *hg_part = nullptr;
    // two-way FM state (allocated on the first call with fm_permille > 0)
    void *fm_mem = nullptr;
    size_t fm_bytes = 0;
    int fm_n = 0, fm_nnz = 0, fm_k = 0, fm_p = 0;
    fr::FmDev fm = {};
    // multi-try FM state (allocated on the first call with mt_alpha > 0)
    void *mt_mem = nullptr;
    size_t mt_bytes = 0;
    int mt_n = 0, mt_nnz = 0, mt_k = 0, mt_p = 0;
    fr::MtDev mt = {};
    // captured CUDA graphs of batch sweeps
    std::vector<GraphCacheEntry> gcache;
    bool use_graphs = true;
    long long last_launches = 0;   // kernels launched by the last call
    long long sweep_launches = 0;  // kernels the last enqueued sweep holds
    // profiling: direct launches with an event pair around each kernel
    bool profiling = false;
    std::vector<cudaEvent_t> pev;
    fr_profile_info prof = {};
    std::vector<float> round_ms;   // per round: scan, step 1, cluster kernels, step 2 (profiling)
    std::vector<float> pair_ms;    // per pair: round, cluster start and end after the round's first start
    // queue sweep (every pair of a sweep in one launch of clusters, see queue_sweep.cu):
    // resident clusters of the queue kernel per cluster size, and the per-cluster
    // workspaces of the last size used (allocated on first use)
    int q_cap[kNumClusterSizes] = {0, 0, 0, 0, 0};
    void *q_mem = nullptr;
    size_t q_bytes = 0;
    int q_ctas = 0, q_clusters = 0, q_n = 0, q_nnz = 0, q_k = 0, q_reps = 0, q_np = 0;
    long long q_nu = 0, q_mu = 0, q_vq = 0;
    fr::QSlot *q_slots = nullptr;              // device array [q_clusters]
    std::vector<fr::QSlot> q_host;             // the same descriptors on the host
    // the slots' graph descriptors, control blocks and counters, each array contiguous so
    // that a sweep sets and reads them with one copy apiece
    fr::GraphDev *q_graphs = nullptr;
    struct alignas(256) QCtl { fr::Ctl c; };   // one control block per 256 bytes: no line shared by two clusters
    QCtl *q_ctls = nullptr;
    long long *q_stats = nullptr;              // [4 q_clusters]
    int *q_ticket = nullptr, *q_gabort = nullptr, *q_prev = nullptr, *q_crank = nullptr;
    int *qb_sorted = nullptr, *qb_start = nullptr, *qb_cnt = nullptr, *qb_app = nullptr, *qb_pool = nullptr,
        *qb_lst = nullptr;
    int qb_cap = 0;
    bool last_queue = false;                   // the last fr_refine_batch ran as a queue sweep
    int last_queue_ctas = 0, last_queue_clusters = 0, queue_fallbacks = 0;
};

struct fr_corridor {
    fr_ctx *ctx;
    unsigned long long gen;
    int nc, m, k, a, b, stage;
    int32_t *part;
    fr_graph g;
    long long Ubase, Lmax;
};

// A planned sweep: pairs in round order (pa, pb), rounds, budgets, launch shapes.
struct BatchPlan {
    int np, nr;
    std::vector<int> off;      // round offsets
    std::vector<int> grid;     // persistent-kernel CTAs per round
    int tpb, k;
    long long Ubase, Lmax, totcut;
    std::vector<long long> est_max;   // estimated corridor vertices of each round's largest pair
    double avg_degree = 12.0;
    std::vector<int> pa, pb;   // the pairs in round order
};

void ctx_error(fr_ctx *ctx, const char *fmt, ...);
fr_status cuda_fail(fr_ctx *ctx, cudaError_t e, const char *what);
long long host_budget_base(long long W, int k, double eps, double alpha);
long long host_lmax(long long W, long long maxc, int k, double eps);
fr_status status_from_ctl(fr_ctx *ctx, const fr::Ctl &c, const char *where);
fr_status ensure_base(fr_ctx *ctx, int n, int nnz, int k, int reps);
fr_status ensure_pairs(fr_ctx *ctx, int P, int R, int reps);
fr_status ensure_reps(fr_ctx *ctx, int reps);
fr::Work make_work(fr_ctx *ctx, int r, int p0, int P, int n, const fr_options *opt);
int choose_tpb(fr_ctx *ctx, const fr_options *opt);
// Pulses between gap checks of push-relabel (fr_options.gap_interval: 0 -> 8, -1 -> none).
int gap_interval_of(const fr_options *opt);
int choose_grid(fr_ctx *ctx, const fr_options *opt, int tpb, int nsides, long long est_vertices);
fr_status check_graph(fr_ctx *ctx, const fr_graph *g, const int32_t *part, int32_t k);
// Checks of eps, alpha and the options that need no context; *why names the first failure.
fr_status validate_params(double eps, double alpha, const fr_options *opt, const char **why);
fr_status check_params(fr_ctx *ctx, double eps, double alpha, const fr_options *opt);
fr_status run_prep(fr_ctx *ctx, const fr_graph *g, const int32_t *part, int32_t k, bool quotient, bool checked,
                   fr::PrepOut *host_out);
fr_status setup_single(fr_ctx *ctx, const fr_graph *g, int32_t *part, int32_t k, int32_t a, int32_t b,
                       long long Ubase, long long Lmax, int mb);
fr_status reset_idle(fr_ctx *ctx);
// FM workspace for graphs up to n vertices / nnz arcs, k blocks and P pairs per call.
fr_status ensure_fm(fr_ctx *ctx, int n, int nnz, int k, int P);
void free_fm(fr_ctx *ctx);
// Multi-try workspace for graphs up to n vertices / nnz arcs, k blocks, P pairs per pass.
fr_status ensure_mt(fr_ctx *ctx, int n, int nnz, int k, int P);
void free_mt(fr_ctx *ctx);
// One multi-try pass over the pairs (pa[i], pb[i]) on part (a DEVICE array of g's
// vertices) with block weight bound Lmax; ctx->blockw and the boundary candidate list
// (if bl_on) are kept current.  changed (HOST, k entries, optional) receives the
// blocks a kept move left or entered.
fr_status run_mt_pass(fr_ctx *ctx, const fr_graph *g, int32_t *part, int32_t k, const int32_t *pa, const int32_t *pb,
                      int np, long long Lmax, int alpha, unsigned long long seed, bool bl_on, fr::MtRes *out,
                      int8_t *changed);
// The FM state of the pairs [p0, ...) of a call (results at res + p0).
fr::FmDev fm_view(fr_ctx *ctx, int p0, const fr_options *opt);
// Launches of one flow iteration over the pairs of w after the boundary scan:
// step (BFS, ids, build) -> cluster max flow -> step (rest), or one step kernel.
// est_pair_vertices: estimated corridor size of the largest pair (chooses the cluster size);
// cluster_ctas: 4, 8 or 16 forces the first cluster size, 0 chooses it.
cudaError_t launch_round(fr_ctx *ctx, fr::Work &w, int grid, int tpb, cudaStream_t st, cudaEvent_t *ev,
                         long long est_pair_vertices = 0, double avg_degree = 12.0, int cluster_ctas = 0);
cudaError_t launch_clusters(fr_ctx *ctx, fr::Work &w, long long est_pair_vertices, double avg_degree, int force,
                            cudaStream_t st, int *nl);
void release_corridor(fr_ctx *ctx);
void free_queue(fr_ctx *ctx);
// Index into fr_ctx::kClusterSizes of the queue sweep's cluster size for plan pl, or -1
// when the queue does not apply (FM step, no cluster capacity, estimate beyond 16 CTAs).
int queue_size_for(fr_ctx *ctx, const BatchPlan &pl, const fr_options *opt);
// Runs the sweep of plan pl as one queue launch with clusters of kClusterSizes[t] CTAs.
// On success *ran = true and ctls holds one control block per cluster (statistics); if
// a pair outgrew the per-cluster workspace, part and the idle state are restored and
// *ran = false (the caller plans the sweep again and runs it round by round).  Other
// device errors restore part and return the error.
fr_status run_queue_sweep(fr_ctx *ctx, const fr_graph *g, int32_t *part, const BatchPlan &pl, const fr_options *opt,
                          int t, float *ms, bool *ran, std::vector<fr::Ctl> *ctls);
void destroy_graph_cache(fr_ctx *ctx);
