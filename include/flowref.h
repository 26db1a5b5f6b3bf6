/*
 * flowref.h -- C ABI of the GB300 flow-refinement library (libflowref.so).
 *
 * The library improves a k-way partition of an undirected graph by max-flow /
 * min-cut computations on block pairs (Sanders & Schulz, "Engineering
 * Multilevel Graph Partitioning Algorithms", Section 4.1 "Using Max-Flow
 * Min-Cut Computations for Local Improvement" and Section 4.1.1 "Most Balanced
 * Minimum Cuts").  All compute runs in hand-written CUDA kernels for sm_103a;
 * there is no CPU fallback.  If the device or the kernels are unavailable the
 * calls fail with FR_ERR_CUDA.
 *
 * Conventions shared by every entry point
 *   - Graph (Section 2.1): G = (V, E, c, omega), CSR with n vertices and nnz =
 *     2|E| directed entries.  omega(e) >= 1, c(v) >= 0, int32.  The CSR must be
 *     symmetric (v in row u iff u in row v, equal weights), simple and without
 *     self loops; the sum of omega around any vertex must stay below 2^30.
 *   - part[v] in [0, k) is the block of v.  All graph arrays and part are
 *     DEVICE pointers owned by the caller unless the name says _host.
 *   - Blocks are balanced when c(V_i) <= L_max = floor((1 + eps) c(V) / k) +
 *     max_v c(v) (Section 2.1, integer form).
 *   - The corridor of pair (a, b) uses eps' = alpha * eps (Section 4.1): side a
 *     may take weight U_a = max(0, floor((1 + alpha*eps) c(V) / k) - c(V_b)),
 *     side b likewise.  The double expression is evaluated on the host without
 *     fused multiply-adds.
 *   - Calls are ordered on the context's stream and synchronise before
 *     returning (results are in host structs on return).
 *   - part is written only when a pair's new cut is accepted; on any error it is
 *     left unchanged.  Errors are reported by status and fr_last_error().
 *   - A context is not thread safe; use one context per host thread.
 */
#ifndef FLOWREF_H
#define FLOWREF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum fr_status {
    FR_OK = 0,
    FR_ERR_INVALID_ARG = 1,  /* an argument violates the conventions above */
    FR_ERR_CUDA = 2,         /* CUDA runtime error or no usable device */
    FR_ERR_OOM = 3,          /* the context's arena cannot hold the workspace */
    FR_ERR_ITER_LIMIT = 4,   /* a device loop hit its cap (pulses, levels, SCC rounds) */
    FR_ERR_TOO_LARGE = 5,    /* nnz >= 2^31 or weighted degree >= 2^30 */
    FR_ERR_ABORTED = 6,      /* device-side barrier wait timed out or abort flag set */
    FR_ERR_INTERNAL = 7      /* a device-side consistency check failed (e.g. cut != flow) */
} fr_status;

typedef struct fr_ctx fr_ctx;
typedef struct fr_corridor fr_corridor;

/* CSR graph, DEVICE pointers, caller-owned.  vwgt = c, adjwgt = omega. */
typedef struct fr_graph {
    int32_t n;
    int32_t nnz;
    const int32_t *xadj;    /* [n+1], xadj[0] = 0, non-decreasing, xadj[n] = nnz */
    const int32_t *adjncy;  /* [nnz] neighbour ids */
    const int32_t *adjwgt;  /* [nnz] omega >= 1 */
    const int32_t *vwgt;    /* [n]   c >= 0 */
} fr_graph;

typedef struct fr_options {
    int32_t mb;            /* 1: most balanced minimum cut (Section 4.1.1); 0: smallest source set */
    int32_t mb_reps;       /* R >= 1 topological sweeps; sweep r >= 1 keys components by splitmix64(seed ^ r ^ minid) */
    int32_t adaptive;      /* 1: adaptive flow iterations (Section 4.1) in fr_refine_pair, fr_refine_batch
                              (each round's pairs iterate together, every pair on its own alpha;
                              launched round by round, no graph replay) and fr_refine_active */
    int32_t max_iters;     /* iteration cap of the adaptive loop (default 10) */
    double alpha_max;      /* alpha' >= 1, the upper bound of alpha */
    uint64_t seed;         /* sweep keys for r >= 1 */
    int64_t pulse_cap;     /* push-relabel pulse cap per flow (0: default 1<<20) */
    int32_t checked;       /* 1: verify CSR symmetry and weights on the device first */
    int32_t block_threads; /* launch shape; 0 = tuned default (see fr_autotune) */
    int32_t grid_blocks;   /* CTAs of the persistent kernel; 0 = tuned default (a queue sweep: at most
                              this many CTAs in clusters; 0 = every cluster that fits at once) */
    int32_t gr_interval;   /* pulses between global relabels; 0 = tuned default */
    int32_t inner_ops;     /* push/relabel operations per vertex per pulse; 0 = default */
    int32_t pulse_passes;  /* lock-free pulse passes between grid barriers; 0 = default */
    int32_t flow_sched;    /* per-pair cluster max flow: 1 level-ordered waves, 2 lock-free pulses;
                              0 = tuned default (pulses unless fr_autotune chose waves) */
    int32_t cluster_ctas;  /* CTAs of the first per-pair cluster launch (4, 6, 8, 12 or 16); 0 = by the
                              estimated corridor size.  Pairs that do not fit go to 16-CTA
                              clusters, then to the grid-wide flow; results do not depend on it */
    int32_t pre_waves;     /* cluster pulses: level-ordered waves before the first pulse (0-2);
                              -1 = none, 0 = tuned default */
    int32_t fm_permille;   /* > 0: two-way FM with TopGain (Section 2.2) on each pair before its
                              flow, stopped once more than fm_permille / 1000 of the pair's
                              vertices moved without an improvement (50 = the 5 % of the
                              paper's setup); 0 = no FM.  fr_refine_pair, fr_refine_batch and
                              fr_refine_active; needs a simple graph and every gain within
                              +-1023 (max weighted degree of the graph), else FR_ERR_TOO_LARGE */
    int32_t mt_alpha;      /* > 0: fr_refine_active runs a multi-try FM pass (Section 4.2) after
                              the pairwise improvements of every matching, its k-way searches
                              stopped by the KaSPar rule p mu^2 > mt_alpha sigma^2 + ln n
                              (Section 2.2; 10 in the paper's setup); blocks a kept move left or
                              entered become active.  0: none.  Other entry points need 0;
                              needs k <= 1024 and every gain within +-1023 */
    int32_t sweep_sched;   /* fr_refine_batch: 0 = a queue sweep where it applies -- every pair of
                              the sweep in one launch of thread-block clusters, a pair started as
                              soon as the earlier pairs that share one of its blocks committed
                              (the same results as round by round; not with the FM step, and a
                              sweep whose corridor outgrows a cluster runs round by round);
                              1 = round by round (one launch sequence per matching) */
    int32_t gap_interval;  /* push-relabel: every gap_interval pulses between exact relabels, the gap
                              heuristic (a label no vertex holds cuts every vertex above it off the
                              target: they go to the top label at once); 0 = every 8 pulses,
                              -1 = off.  Results do not depend on it */
} fr_options;

/* Outcome of one pair refinement.  cut_* are omega(E_ab); wA/wB are c(V_a), c(V_b);
 * *_before is the state before the pair's FM step (if any) and flow, *_after the final one. */
typedef struct fr_pair_result {
    int64_t flow;           /* value of the maximum s-t flow of the last iteration */
    int64_t cut_before, cut_after;
    int64_t wA_before, wB_before, wA_after, wB_after;
    int32_t corridor_n;     /* corridor vertices of the last iteration */
    int32_t corridor_arcs;  /* arcs between corridor vertices (both directions) */
    int32_t accepted;       /* 1 if a flow's cut was applied */
    int32_t iters;          /* flow iterations run */
    double alpha_final;     /* alpha after the adaptive loop */
    int32_t status;         /* fr_status of this pair */
    int32_t a, b, round;    /* the pair and its round (batch) */
    int64_t pulses;         /* push-relabel pulses of the pair's last flow (step-wide) */
    int64_t relabels;       /* global relabels (step-wide) */
    int32_t bfs_levels;     /* corridor BFS levels (step-wide) */
    int32_t scc_rounds;     /* SCC colouring rounds (step-wide) */
    int32_t ncomp;          /* SCCs outside the S and T sets (MB only) */
    int32_t fm_moves;       /* moves the FM step kept (fm_permille > 0) */
    int64_t cut_fm;         /* omega(E_ab) after the FM step (= cut_before without FM) */
} fr_pair_result;

typedef struct fr_batch_result {
    int32_t npairs;         /* quotient-graph edges = pairs refined */
    int32_t nrounds;        /* matchings (launches of the persistent kernel) */
    int32_t accepted;       /* pairs whose cut was applied */
    int32_t status;
    int64_t cut_before;     /* total cut sum_{i<j} omega(E_ij) before and after */
    int64_t cut_after;
    int64_t corridor_arcs;  /* sum of corridor arcs over all pairs */
    int64_t device_ns;      /* device time of the rounds (CUDA events) */
    int64_t flow_ns;        /* device time spent in the max-flow phase (in-kernel timers) */
    int64_t mt_gain;        /* fr_refine_active with mt_alpha > 0: cut decrease of the multi-try
                               passes (included in cut_after) */
    int32_t mt_searches;    /* k-way searches they started */
    int32_t mt_tried;       /* moves they made */
    int32_t mt_kept;        /* moves kept after the rollbacks */
    int32_t pad0;
} fr_batch_result;

/* One multilevel V-cycle (fr_vcycle). */
#define FR_MAX_LEVELS 64
typedef struct fr_vcycle_result {
    int32_t levels;                       /* graphs in the hierarchy, the input included */
    int32_t status;
    int64_t cut_before, cut_after;        /* total cut of the input and the output partition */
    int32_t level_n[FR_MAX_LEVELS];       /* vertices of each level (0 = the input) */
    int32_t level_pairs[FR_MAX_LEVELS];   /* pair refinements run on each level */
    int64_t level_cut[FR_MAX_LEVELS];     /* total cut after the level's refinement */
    double coarsen_ms;                    /* matching and contraction, all levels (host clock, synchronised) */
    double refine_ms;                     /* projection and refinement, all levels */
} fr_vcycle_result;

/* One global search cycle (fr_cycle). */
typedef struct fr_cycle_result {
    int32_t coarsenings;                        /* matchings computed (stalled ones included) */
    int32_t refinements;                        /* refinement sweeps run */
    int32_t depth;                              /* levels of the deepest branch */
    int32_t status;
    int64_t cut_before, cut_after;
    int32_t level_coarsenings[FR_MAX_LEVELS];   /* coarsenings of level-l graphs */
    double ms;                                  /* host clock around the call (synchronised) */
} fr_cycle_result;

/* Totals of one multi-try FM pass (fr_multitry) or of global k-way rounds
 * (fr_kway_global, where searches counts the rounds). */
typedef struct fr_mt_result {
    int64_t gain;           /* cut decrease kept */
    int32_t searches;       /* k-way searches started */
    int32_t tried;          /* moves made */
    int32_t kept;           /* moves kept after the rollbacks */
    int32_t status;
} fr_mt_result;

/* ---- context ------------------------------------------------------------ */

/* Fills the defaults: mb 0, mb_reps 1, adaptive 0, max_iters 10, alpha_max 1,
 * seed 0, pulse_cap 1<<20, checked 0, launch shape 0 (tuned). */
void fr_default_options(fr_options *opt);

/* sizeof of the structs of this header, for bindings to check their layouts:
 * which = 0 fr_graph, 1 fr_options, 2 fr_pair_result, 3 fr_batch_result,
 * 4 fr_profile_info, 5 fr_server_config, 6 fr_request, 7 fr_response,
 * 8 fr_mt_result, 9 fr_vcycle_result, 10 fr_cycle_result; -1 for
 * any other value.  Needs no device. */
int32_t fr_struct_size(int32_t which);

/* Creates a context on `device` using `stream` (a cudaStream_t; NULL = a new
 * non-blocking stream owned by the context).  arena_bytes bounds the device
 * workspace (0 = no bound); exceeding it returns FR_ERR_OOM. */
fr_status fr_create(fr_ctx **ctx, int32_t device, size_t arena_bytes, void *stream);
fr_status fr_destroy(fr_ctx *ctx);
/* Message of the last failing call on this context (static storage in ctx). */
const char *fr_last_error(const fr_ctx *ctx);
const char *fr_status_string(fr_status st);
/* Bytes of device workspace the context holds now. */
size_t fr_workspace_bytes(const fr_ctx *ctx);

/* ---- the three steps of Section 4.1 on one pair --------------------------- */

/* Corridor of pair (a, b) (Section 4.1): two BFS inside blocks a and b from
 * their boundary towards the other block, vertices taken in (distance, id)
 * order while the side's weight stays <= U_side; then the network G' = G[B] +
 * s + t, s -> border of side a, border of side b -> t with capacity INF_v = 1 +
 * sum of omega at v, border taken with respect to G[V_a u V_b].
 * The corridor lives in the context's workspace: building another corridor or
 * calling another refinement on the same context invalidates the handle (later
 * use returns FR_ERR_INVALID_ARG).  Free with fr_corridor_free. */
fr_status fr_build_corridor(fr_ctx *ctx, const fr_graph *g, const int32_t *part, int32_t k, int32_t a,
                            int32_t b, double eps, double alpha, fr_corridor **out);
fr_status fr_corridor_info(const fr_corridor *c, int32_t *corridor_n, int32_t *corridor_arcs);
/* Copies the network to HOST buffers in a canonical layout: gid[nc] ascending
 * global ids (local id = position), off[nc+1]/head[m]/cap[m] arcs between corridor
 * vertices in CSR order of the graph, border[nc] (0 none, 1 s->v, 2 v->t),
 * infcap[nc] (INF_v for border vertices, else 0), side0[nc] (0 = block a),
 * dist[nc] (BFS distance inside the vertex's block).  Any pointer may be NULL. */
fr_status fr_corridor_export(fr_ctx *ctx, const fr_corridor *c, int32_t *gid, int32_t *off, int32_t *head,
                             int32_t *cap, int8_t *border, int32_t *infcap, int8_t *side0, int32_t *dist);
/* Maximum s-t flow of the corridor network (Section 4.1): push-relabel with
 * global relabels, then excess returned to s so that the result is a flow,
 * not a preflow.  *flow_out receives its value. */
fr_status fr_maxflow(fr_ctx *ctx, fr_corridor *c, int64_t *flow_out);
/* Flow on each corridor arc (net, antisymmetric; m entries) and on the s/t arc
 * of each corridor vertex (nc entries), HOST buffers. */
fr_status fr_corridor_flow(fr_ctx *ctx, const fr_corridor *c, int64_t *arcflow, int64_t *stflow);
/* Minimum cut from the residual graph and its application to part.
 * most_balanced = 0: the smallest source set (vertices reachable from s; the
 * Ford-Fulkerson labelling cut).  most_balanced = 1: SCCs of the residual graph
 * outside the sets reachable from s / reaching t, mb_reps deterministic
 * topological sweeps, the cut with the smallest |c(A') - c(B')| (Section 4.1.1).
 * Corridor vertices on the source side go to block a, the others to block b;
 * the result is applied to part (DEVICE, in/out) only if it is accepted:
 * max(c(A'), c(B')) <= L_max and (cut decreases, or cut equal and
 * max(c(A'), c(B')) decreases).  res receives the outcome. */
fr_status fr_extract_cut(fr_ctx *ctx, fr_corridor *c, int32_t most_balanced, int32_t mb_reps, uint64_t seed,
                         int32_t *part, fr_pair_result *res);
/* After fr_extract_cut: residual sets and output side per corridor vertex (HOST
 * buffers): in_s reachable from s, to_t reaches t, comp = min global id of the
 * vertex's residual SCC (vertices in neither set, else -1), side 0 = source. */
fr_status fr_corridor_sets(fr_ctx *ctx, const fr_corridor *c, int8_t *in_s, int8_t *to_t, int32_t *comp,
                           int8_t *side);
fr_status fr_corridor_free(fr_ctx *ctx, fr_corridor *c);

/* ---- whole refinements ------------------------------------------------------ */

/* Corridor + max flow + cut + acceptance for pair (a, b) in one persistent launch
 * per flow iteration.  With opt->adaptive the iterations follow Section 4.1:
 * accepted smaller cut -> alpha = min(2 alpha, alpha') and repeat; feasible cut
 * that is not smaller -> apply if better balanced and stop; infeasible -> stop at
 * alpha = 1, else alpha = max(alpha / 2, 1) and repeat; at most max_iters. */
fr_status fr_refine_pair(fr_ctx *ctx, const fr_graph *g, int32_t *part, int32_t k, int32_t a, int32_t b,
                         double eps, double alpha, const fr_options *opt, fr_pair_result *res);

/* All block pairs that are adjacent in the quotient graph of part (Section 2.1),
 * scheduled as rounds of block-disjoint pairs: greedy colouring of the quotient
 * edges in lexicographic (a, b) order, smallest free colour.  Each round runs as
 * one persistent launch over the union of its pairs' flow networks; the rounds are
 * replayed from a captured CUDA graph.  One flow iteration per pair at the given
 * alpha.  results (HOST, capacity cap) receives the pairs in round order, then
 * (a, b) order.  Equivalent to fr_refine_pair over the pairs in that order. */
fr_status fr_refine_batch(fr_ctx *ctx, const fr_graph *g, int32_t *part, int32_t k, double eps, double alpha,
                          const fr_options *opt, int32_t cap, fr_pair_result *results, fr_batch_result *summary);

/* Active block scheduling (Section 4.3 and the appendix pseudocode of active block
 * scheduling) with the flow refinement of Section 4.1 as the pairwise step, preceded
 * by the two-way FM search when opt->fm_permille > 0, and with a multi-try FM pass
 * (fr_multitry) over each matching's pairs after their pairwise steps when
 * opt->mt_alpha > 0 (every block a kept multi-try move left or entered becomes
 * active; summary->mt_* receive its totals).  Every block starts active; an outer round takes the quotient edges (a, b) of the
 * current partition with a or b active, marks every block inactive, colours the
 * edges into matchings (lexicographic order, smallest colour free at both ends) and
 * refines the pairs matching by matching, each with adaptive flow iterations
 * (Section 4.1) when opt->adaptive; a pair whose refinement changed part marks a and
 * b active.  Stops when no block is active or after max_outer (>= 1) outer rounds.
 * part: DEVICE, updated in place, unchanged on error.  results (HOST, cap entries,
 * may be NULL if cap = 0): one entry per pair refinement in processing order, round =
 * the matching's index counted over all outer rounds.  summary (HOST, optional):
 * npairs = refinements, nrounds = matchings, accepted, total cut before/after.
 * *nouter (HOST, optional): outer rounds run. */
fr_status fr_refine_active(fr_ctx *ctx, const fr_graph *g, int32_t *part, int32_t k, double eps, double alpha,
                           const fr_options *opt, int32_t max_outer, int32_t cap, fr_pair_result *results,
                           fr_batch_result *summary, int32_t *nouter);

/* One multi-try FM pass (Section 4.2) over the np block-disjoint pairs (pa[i], pb[i])
 * (HOST arrays, pair order), as fr_refine_active runs it after a matching: each pair's
 * vertices with a neighbour in the other block of the pair form its todo list, in the
 * order of splitmix64(splitmix64(splitmix64(seed ^ a << 32 ^ b) + 1) ^ v); the lists
 * are visited round-robin (entry j of every pair, then entry j + 1); a listed vertex
 * that no earlier search of the pass queued and that still has a neighbour in another
 * block starts a k-way local search (Section 2.2) from itself and its unqueued boundary
 * neighbours (CSR order).  A search keeps one queue keyed by max gain (ties: the later
 * keying first), moves the best vertex to its best adjacent block (ties: smaller
 * splitmix64(splitmix64(~seed) ^ v << 32 ^ P), then smaller P) unless that block would
 * exceed L_max = floor((1 + eps) c(V) / k) + max c(v), moves each vertex at most once,
 * keys the unmoved neighbours of a moved vertex again, queues no vertex another search
 * of the pass queued, stops when the queue is empty or p mu^2 > alpha sigma^2 + ln n
 * over the gains of the p moves since the last new minimum cut (KaSPar), and rolls
 * back to the first lowest cut.  part: DEVICE, updated in place (unchanged on error).
 * changed (HOST, k entries, optional): 1 for every block a kept move left or entered.
 * Needs alpha >= 0, k <= 1024 and every gain within +-1023 (FR_ERR_TOO_LARGE). */
fr_status fr_multitry(fr_ctx *ctx, const fr_graph *g, int32_t *part, int32_t k, double eps, int32_t np,
                      const int32_t *pa, const int32_t *pb, int32_t alpha, uint64_t seed, fr_mt_result *out,
                      int8_t *changed);

/* Global k-way refinement (Section 2.2, configured as Section 6 describes): rounds of
 * one k-way local search each (the search of fr_multitry without its touched rule),
 * started from every vertex with a neighbour in another block (init_mode 0) or only
 * from the corner vertices, whose neighbours lie in at least two blocks other than
 * their own (init_mode 1), queued in ascending splitmix64(splitmix64(seed ^ r) ^ v)
 * order in round r = 0, 1, ...; target ties go to the smaller
 * splitmix64(splitmix64(~seed) ^ v << 32 ^ P), then the smaller P.  The rounds end
 * after the first one that gains nothing or after max_rounds (>= 1).  part: DEVICE,
 * updated in place (unchanged on error).  out (HOST, optional): gain, tried and kept
 * summed over the rounds; searches = rounds run.  Needs eps > 0, alpha >= 0,
 * k <= 1024 and every gain within +-1023 (FR_ERR_TOO_LARGE). */
fr_status fr_kway_global(fr_ctx *ctx, const fr_graph *g, int32_t *part, int32_t k, double eps, int32_t init_mode,
                         int32_t alpha, int32_t max_rounds, uint64_t seed, fr_mt_result *out);

/* ---- multilevel V-cycle with a given partition (Sections 2.1, 2.2, 5) ---- */
/* These calls allocate their scratch and the coarse graphs with cudaMalloc for the length
 * of the call (about twice the input graph for a V-cycle, the current branch for W- and
 * F-cycles), outside the context's arena bound; FR_ERR_OOM if an allocation fails. */

/* Greedy matching of one level: the edges inside one block of part whose ends both weigh
 * at most 1.5 W / (20 k) (40 k c(v) <= 3 W), ordered by expansion*2 = omega^2 / (c(u) c(v))
 * (exact, c taken as max(c, 1)), then by the larger splitmix64(seed_l ^ min << 32 ^ max),
 * then by the smaller (min, max); an edge joins when both ends are free.  Computed on the
 * device with locally dominant edges (the same matching).  mate: DEVICE, n entries,
 * receives the partner or -1.  *pairs (HOST): matched pairs. */
fr_status fr_match(fr_ctx *ctx, const fr_graph *g, const int32_t *part, int32_t k, int64_t W, uint64_t seed_l,
                   int32_t *mate, int32_t *pairs);

/* Contraction of a matching (Section 2.1): the smaller end of a pair, or a single vertex,
 * represents a coarse vertex, numbered in the order of those fine ids; c(x) is the sum of
 * its members; rows list the coarse neighbours by increasing id, parallel edges merged
 * with summed weights, the matched edge dropped.  All arrays DEVICE: cmap[n]; coarse
 * xadj / adjncy / adjwgt / vwgt with room for n + 1, nnz, nnz and n entries.  *cn, *cnnz
 * (HOST): coarse sizes.  FR_ERR_INVALID_ARG unless every mate entry is -1 or a partner
 * u != v in range with mate[u] = v (checked on the device first). */
fr_status fr_contract(fr_ctx *ctx, const fr_graph *g, const int32_t *mate, int32_t *cmap, int32_t *cn, int32_t *cnnz,
                      int32_t *cxadj, int32_t *cadjncy, int32_t *cadjwgt, int32_t *cvwgt);

/* One V-cycle with the given partition (Section 5: no edge between two blocks is matched,
 * so part is the coarsest level's partition): contract with fr_match (seed_l =
 * splitmix64(opt->seed ^ level)) and fr_contract while the graph has more than
 * max(60 k, n / (60 k)) vertices, the matching holds at least n_level / 20 pairs (a
 * level that would shrink by less than 5 % has stalled) and fewer than max_levels
 * (<= FR_MAX_LEVELS) levels exist; then from the coarsest level up, project the partition
 * and refine it with one fr_refine_batch sweep, or fr_refine_active with active_outer
 * outer rounds (each level with its own L_max).  part: DEVICE, updated in place,
 * unchanged on error.  out (HOST, optional): the hierarchy's sizes and the cut per
 * level.  opt->mt_alpha needs active_outer > 0. */
fr_status fr_vcycle(fr_ctx *ctx, const fr_graph *g, int32_t *part, int32_t k, double eps, double alpha,
                    const fr_options *opt, int32_t max_levels, int32_t active_outer, fr_vcycle_result *out);

/* A global search cycle with the given partition (Section 5 and its pseudocode):
 * type 0 V-cycle (the result of fr_vcycle), 1 W-cycle, 2 F-cycle, level split parameter
 * d >= 1 (the paper's default is 2).  A cycle on a graph coarsens it (as fr_vcycle does),
 * runs a cycle on the coarse graph, projects and refines; on levels l with l % d == 0 it
 * then coarsens the refined graph again and repeats (a second trial) -- for F-cycles only
 * while fewer than two coarsenings of level-l graphs were made in the run.  A graph that
 * cannot be coarsened is refined and ends its branch.  The c-th coarsening of a level-l
 * graph in the run uses seed_l = splitmix64(opt->seed ^ l ^ c << 32).  Every coarse
 * graph lives only while its branch runs.  part: DEVICE, updated in place, unchanged on
 * error. */
fr_status fr_cycle(fr_ctx *ctx, const fr_graph *g, int32_t *part, int32_t k, double eps, double alpha,
                   const fr_options *opt, int32_t type, int32_t d, int32_t max_levels, int32_t active_outer,
                   fr_cycle_result *out);

/* Same as fr_refine_batch for a graph and partition in HOST memory: uploads the
 * arrays, refines, and copies part back (the end-to-end form; graph buffers are
 * reused across calls of the same size). */
fr_status fr_refine_batch_host(fr_ctx *ctx, int32_t n, int32_t nnz, const int32_t *xadj_host,
                               const int32_t *adjncy_host, const int32_t *adjwgt_host, const int32_t *vwgt_host,
                               int32_t *part_host, int32_t k, double eps, double alpha, const fr_options *opt,
                               int32_t cap, fr_pair_result *results, fr_batch_result *summary);

/* Rounds of the quotient graph of part (HOST outputs, capacity cap): pair_a <
 * pair_b in lexicographic order and the round of each.  Returns counts. */
fr_status fr_rounds(fr_ctx *ctx, const fr_graph *g, const int32_t *part, int32_t k, int32_t cap, int32_t *pair_a,
                    int32_t *pair_b, int32_t *pair_round, int32_t *npairs, int32_t *nrounds);

/* ---- measurement --------------------------------------------------------------- */

/* Per-kernel timing and the work counters behind the bytes model of a sweep. */
typedef struct fr_profile_info {
    int32_t nrounds;          /* rounds of the last fr_refine_batch */
    int32_t launches;         /* kernels launched by it */
    double scan_ms;           /* boundary-scan kernels, CUDA events around each launch (profiling on) */
    double step_ms;           /* persistent step kernels, CUDA events around each launch (profiling on) */
    double cluster_ms;        /* per-pair cluster max-flow kernels, CUDA events (profiling on) */
    double phase_ms[12];      /* in-kernel timers: bfs, select, lid, build, flow, relabel, return,
                                 reach, scc, sweep, eval, commit (summed over rounds) */
    int64_t n, nnz;           /* graph scanned by each boundary-scan launch */
    int64_t bfs_visited;      /* BFS entries */
    int64_t bfs_arcs;         /* arcs scanned by the corridor BFS */
    int64_t corridor_n;       /* corridor vertices, all pairs */
    int64_t corridor_arcs;    /* corridor arcs, all pairs */
    int64_t pulses;           /* push-relabel pulses, summed over rounds */
    int64_t relabels;         /* global relabels */
    int64_t gr_arcs;          /* arcs scanned by global relabels */
    int64_t pr_arcs;          /* arcs scanned by push-relabel pulses */
    int64_t pushes;           /* pushes */
    int64_t scc_rounds;       /* SCC colouring rounds */
    int64_t barriers;         /* grid barriers passed by the persistent kernels */
    double cluster_phase_ms[7]; /* cluster kernel timers summed over pairs: network load into
                                   shared memory, flow to t, return of excess to s, residual
                                   reachability, residual SCCs (most balanced cuts), member scan
                                   and split (before the load), and the exact relabels (part
                                   of the flow and return times) */
    int64_t cluster_syncs;    /* cluster barriers, summed over pairs */
    int64_t cluster_remote_arcs; /* arcs held in a cluster whose head another CTA holds (DSMEM) */
    int64_t fallback_pairs;   /* pairs left to the grid-wide flow */
    int64_t scan_listed;      /* boundary-scan list entries read, summed over rounds */
    int64_t scan_rows;        /* of them, vertices of the rounds' blocks (rows scanned) */
    int64_t scan_arcs;        /* arcs of those rows */
    double fm_ms[3];          /* FM step (fm_permille > 0), summed over pairs: boundary sort and
                                 initial stacks, the moves, rollback and bookkeeping */
    int32_t cluster_sizes[5]; /* CTAs per cluster the library can launch (4, 6, 8, 12, 16) */
    int32_t cluster_max_active[5]; /* clusters of each size resident at once on this GPU */
    int32_t queue;            /* 1: the last fr_refine_batch ran as a queue sweep (fr_options.sweep_sched);
                                 cluster_ms is then the whole sweep's device time */
    int32_t queue_ctas;       /* CTAs per cluster of that queue sweep */
    int32_t queue_clusters;   /* clusters it launched */
    int32_t queue_fallbacks;  /* queue sweeps of this context that a pair outgrew (run round by round) */
    double queue_scan_ms;     /* queue sweep: the pairs' boundary scans, summed over pairs (in-kernel timers) */
    int64_t gaps;             /* gap checks of push-relabel that found a gap */
    int64_t gap_lifted;       /* vertices they lifted to the top label */
} fr_profile_info;

/* on = 1: fr_refine_batch launches its kernels directly (no graph replay) with
 * CUDA events around each one, for fr_profile_last; on = 0: graph replay. */
fr_status fr_set_profiling(fr_ctx *ctx, int32_t on);
fr_status fr_profile_last(const fr_ctx *ctx, fr_profile_info *info);
/* Per-round times of the last profiled fr_refine_batch (CUDA events around each
 * launch): ms[4r .. 4r+3] = boundary scan, step 1 (BFS, ids, build), cluster
 * max-flow kernels, step 2 (flow accounting, cut, evaluation, commit) of round r,
 * in milliseconds, for the first min(rounds, cap) rounds.  ms: host array of
 * 4 * cap floats, owned by the caller.  Returns the number of rounds profiled
 * (0 if the last call ran without profiling), -1 for a null ctx (or null ms with
 * cap > 0). */
int32_t fr_profile_rounds(const fr_ctx *ctx, float *ms, int32_t cap);
/* Per pair of the last profiled fr_refine_batch, in the order of its results:
 * ms[3i] = round, ms[3i+1], ms[3i+2] = when a thread-block cluster took pair i and
 * when it finished it (max flow, residual sets and SCCs), in milliseconds after the
 * first pair of the same round was taken (device global timer); -1 for a pair no
 * cluster solved (empty network, or left to the grid-wide flow).  ms: host array
 * of 3 * cap floats, owned by the caller.  Returns the number of pairs profiled
 * (0 if the last call ran without profiling), -1 for a null ctx (or null ms with
 * cap > 0). */
int32_t fr_profile_pairs(const fr_ctx *ctx, float *ms, int32_t cap);

/* ---- launch-shape autotuner -------------------------------------------------- */

/* Times fr_refine_batch on a copy of part for a set of launch shapes
 * (block_threads, grid_blocks, gr_interval, inner_ops, pulse_passes, cluster_ctas,
 * flow_sched, pre_waves; coordinate descent, two sweeps) and writes the fastest into
 * *best.  Results are
 * identical for every shape; only time differs.  The choice is also cached in the
 * context and used when opt fields are 0. */
fr_status fr_autotune(fr_ctx *ctx, const fr_graph *g, const int32_t *part, int32_t k, double eps, double alpha,
                      const fr_options *opt, int32_t trials, fr_options *best, double *best_ms);

/* ---- refinement without device allocation ------------------------------------ */

/* Size limits of fr_refine_pair_noalloc (its scratch is fixed at build time). */
#define FR_NOALLOC_MAX_N 65536       /* vertices */
#define FR_NOALLOC_MAX_NNZ 524288    /* directed CSR entries (2|E|) */
#define FR_NOALLOC_MAX_K 256         /* blocks */
#define FR_NOALLOC_MAX_REPS 4        /* most-balanced sweeps */

/* Same refinement as fr_refine_pair (same arguments and results), for callers
 * that cannot allocate device memory: a process whose device memory belongs to
 * another allocator (a framework's caching allocator or a quota-managed
 * service), or a latency-critical loop that must not stall on cudaMalloc /
 * cudaFree or risk an allocation failure halfway through.  No paper
 * counterpart: this is a deployment variant, not part of the method.
 *
 * It needs no fr_ctx and never calls cudaMalloc, cudaFree or any other
 * allocating routine.  Its workspace is one static device array of about 23 MB
 * that every GPU which loads libflowref.so holds until the process exits.  Every
 * call looks up that array's device address on the current device (a host-side
 * lookup, so a context created again after cudaDeviceReset is followed); the
 * first call on a device also loads the library's kernels there, so make it
 * before any stream capture on that device.
 * Work is queued on `stream` (a cudaStream_t, NULL = the legacy default stream)
 * and the call returns when it is done.  part is left unchanged on any error: the
 * array keeps a copy of it, written back if an iteration fails after an earlier
 * one was applied.
 *
 * Limits: n <= FR_NOALLOC_MAX_N, nnz <= FR_NOALLOC_MAX_NNZ, k <=
 * FR_NOALLOC_MAX_K, mb_reps <= FR_NOALLOC_MAX_REPS; larger problems return
 * FR_ERR_TOO_LARGE without touching part (use fr_refine_pair for them).
 * Options are checked as fr_refine_pair checks them; opt->fm_permille and
 * opt->mt_alpha must be 0 (FR_ERR_INVALID_ARG otherwise).
 * Every call uses the same array, which keeps the previous call's contents;
 * each call clears what it needs before use.  Two calls whose work overlaps on
 * the GPU (concurrent streams or host threads, on the same device) race on the
 * array and corrupt each other: serialise them. */
fr_status fr_refine_pair_noalloc(const fr_graph *g, int32_t *part, int32_t k, int32_t a, int32_t b, double eps,
                                 double alpha, const fr_options *opt, fr_pair_result *res, void *stream);

/* ---- serving: continuous batching of refinement requests ------------------- */

typedef struct fr_server fr_server;

typedef struct fr_server_config {
    int32_t device;
    int32_t max_inflight;    /* requests resident on the device at once */
    size_t arena_bytes;      /* device bytes for request workspaces (admission bound) */
    fr_options opt;          /* options applied to every request (fm_permille must be 0) */
} fr_server_config;

typedef struct fr_request {
    int32_t graph_id;        /* from fr_server_add_graph */
    int32_t k;
    double eps, alpha;
    const int32_t *part_host;/* initial partition, HOST, copied at submit */
    uint64_t tag;            /* caller's id, returned with the result */
} fr_request;

typedef struct fr_response {
    uint64_t tag;
    int32_t status, npairs, nrounds, accepted;
    int64_t cut_before, cut_after;
    double latency_ms;       /* submit -> completion, host clock */
    double queue_ms;         /* submit -> admission */
} fr_response;

fr_status fr_server_create(fr_server **srv, const fr_server_config *cfg);
/* Copies a graph (HOST arrays) to the device once; requests refer to it by id. */
fr_status fr_server_add_graph(fr_server *srv, int32_t n, int32_t nnz, const int32_t *xadj, const int32_t *adjncy,
                              const int32_t *adjwgt, const int32_t *vwgt, int32_t *graph_id);
/* Queues a request (non-blocking).  Requests are admitted when a slot and enough
 * arena bytes are free; admitted requests advance one round per device step, so
 * requests that arrive while others run join the next step. */
fr_status fr_server_submit(fr_server *srv, const fr_request *req);
/* Blocks until one result is available (timeout_ms < 0: wait forever) and copies
 * the refined partition into part_out (HOST, may be NULL). */
fr_status fr_server_next(fr_server *srv, fr_response *resp, int32_t *part_out, int32_t part_cap,
                         int32_t timeout_ms);
fr_status fr_server_stats(fr_server *srv, int64_t *steps, int64_t *admitted, int64_t *completed,
                          int32_t *max_concurrent);
fr_status fr_server_destroy(fr_server *srv);

#ifdef __cplusplus
}
#endif
#endif /* FLOWREF_H */
