/*
 * fro.h -- CPU oracle for flow-based refinement of a block pair.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The product path
 * (libflowref.so and its binding) never calls, links or reads anything here, and
 * the two share no code: no headers, no helpers, no tables.
 *
 * Sources (Sanders & Schulz, "Engineering Multilevel Graph Partitioning
 * Algorithms"):
 *   Section 2.1   graph G = (V, E, c, omega), blocks, L_max, cut objective
 *   Section 4.1   boundary, corridor by two bounded BFS, B-corridor network
 *                 G' = G[B] + s + t with infinite s/t arcs, max flow, adaptive
 *                 flow iterations (eps' = alpha * eps)
 *   Section 4.1.1 Picard-Queyranne closed sets, smallest source set from
 *                 Ford-Fulkerson labelling, SCC contraction of the residual
 *                 graph, removal of S/T components, topological sweeps
 *   Section 2.2   two-way FM with TopGain; k-way local search with one queue and
 *                 the KaSPar stopping rule p mu^2 > alpha sigma^2 + beta
 *   Section 4.2   multi-try FM (k-way searches from single boundary vertices)
 *   Section 4.3   active block scheduling
 *
 * Readings where the paper is silent or ambiguous are fixed as follows and are
 * shared with the CUDA path only as a written specification:
 *   budget     U_side = max(0, floor((1 + alpha*eps) * W / k) - c(other block)),
 *              evaluated as that double expression without FMA contraction;
 *              L_max = floor((1 + eps) * W / k) + max_v c(v)
 *   corridor   reached vertices ordered by (BFS distance, vertex id); the longest
 *              prefix whose weight stays <= U is taken (no skipping)
 *   border     w.r.t. G[A u B]: a corridor vertex with a neighbour in A u B
 *              outside the corridor; A-side border <- s, B-side border -> t
 *   infinity   INF_v = 1 + sum of omega over all edges at v
 *   plain cut  the smallest source set (vertices reachable from s in the
 *              residual graph of a maximum flow)
 *   MB cut     sweeps r = 0..R-1 of Kahn's algorithm over the SCC DAG of the
 *              vertices neither reachable from s nor reaching t; ready set is a
 *              min-heap on key_0 = min vertex id, key_r = (splitmix64(seed ^ r ^
 *              minid), minid); step j moves the first j components to the sink
 *              side; the (j, r) minimising |c(A') - c(B')| wins, ties to smaller
 *              j, then smaller r
 *   accept     max(c(A'), c(B')) <= L_max and (cut decreases, or cut equal and
 *              max(c(A'), c(B')) decreases)
 *   adaptive   feasible & smaller: apply, alpha = min(2 alpha, alpha');
 *              feasible & equal: apply if better balanced, stop;
 *              infeasible: stop if alpha == 1 else alpha = max(alpha/2, 1)
 *   FM         gains and boundary within G[A u B]; a block's queue holds its
 *              unmoved vertices with an edge to the other block, keyed by (gain,
 *              stamp), larger first: initial stamps are random 63-bit values in
 *              the role of the random initial order, each later insertion or
 *              gain change takes a larger stamp (one per adjacency position of the
 *              moved vertex, in CSR order); TopGain: larger top gain, a seeded
 *              random bit on equal top gains, the heavier block while either
 *              block exceeds L_max; best state = smallest (overload, cut, max
 *              block weight); stop after more than permille/1000 of the pair's
 *              vertices moved since the last best, or when both queues are empty
 *   pairwise   with FM on: FM first, then the flow iterations on its result
 *   k-way      one queue keyed by (max gain, stamp), larger first, stamps in the
 *              order of insertions and key changes (start set in its order, then
 *              per move the moved vertex's neighbours in CSR order); target = the
 *              adjacent block of largest connection weight, ties to the smaller
 *              splitmix64(tseed ^ u << 32 ^ P); a vertex whose target would exceed
 *              L_max leaves the queue unmoved; after a move every unmoved neighbour
 *              is keyed again (boundary) or leaves the queue (not boundary); stop by
 *              the KaSPar rule after each move that is not a new minimum, or an
 *              empty queue; roll back to the first lowest-cut prefix
 *   multilevel greedy matching in expansion*2 order (exact, c as max(c, 1); ties
 *              by a seeded splitmix64 key) inside blocks, ends at most 1.5 W/(20k);
 *              coarse ids in the order of the pairs' smaller fine ids; contract
 *              while n > max(60k, n0/(60k)) and a matching holds >= n/20 pairs;
 *              refine every level with its own L_max
 *   cycles     W: a second trial (a new coarsening of the refined graph) on every
 *              level l % d == 0; F: also only while fewer than two coarsenings of
 *              that level were made; the c-th coarsening of a level uses seed_l =
 *              splitmix64(seed ^ l ^ c << 32); every graph is refined after each trial
 *   multi-try  per pair of a matching, the vertices with a neighbour in the other
 *              block, in splitmix64 order, visited round-robin over the pairs; a
 *              vertex no search of the pass queued that is still a boundary vertex
 *              starts a search from itself and its untouched boundary neighbours;
 *              no vertex is queued by two searches of one pass; beta = ln n
 *
 * Parity unpinned: the order of the sweeps r >= 1 (their splitmix64 keys) is
 * checked only for what any valid order must satisfy (a topological order of the
 * component DAG, every step a minimum cut); the quality of the most balanced cut
 * against the true optimum is bounded by brute force, not fixed.  (KaSPar decisions
 * within a few ulps of the threshold are pinned to the documented double operations
 * and the hand-derived ties of constant gains; the F-cycle's stalled second
 * coarsening to a hand-derived recursion.)
 *   batch      greedy edge colouring of the quotient graph in lexicographic
 *              (a, b) order (smallest free colour); each colour is a round of
 *              block-disjoint pairs; rounds in colour order, pairs of a round
 *              see the partition as it stands at the start of the round
 */
#ifndef FRO_H
#define FRO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { FRO_OK = 0, FRO_ERR_INVALID_ARG = 1, FRO_ERR_TOO_LARGE = 5 };

typedef struct fro_options {
    int32_t mb;          /* 1: most balanced minimum cut, 0: smallest source set */
    int32_t mb_reps;     /* R >= 1 sweeps */
    int32_t adaptive;    /* adaptive flow iterations */
    int32_t max_iters;   /* iteration cap of the adaptive loop (>= 1) */
    double alpha_max;    /* alpha' */
    uint64_t seed;       /* sweep keys for r >= 1, FM keys */
    int32_t fm_permille; /* > 0: two-way FM before the flows, stopped after more than
                            fm_permille / 1000 of the pair's vertices moved without an
                            improvement; 0: no FM */
    int32_t mt_alpha;    /* > 0: multi-try FM pass (KaSPar alpha) after each matching of
                            fro_refine_active; 0: none (other entry points need 0) */
} fro_options;

typedef struct fro_pair_result {
    int64_t flow, cut_before, cut_after, wA_before, wB_before, wA_after, wB_after;
    int32_t corridor_n, corridor_arcs, accepted, iters;
    double alpha_final;
    int32_t status, a, b, round;
    int64_t cut_fm;      /* pair cut after the FM step (= cut_before without FM) */
    int32_t fm_moves;    /* FM moves kept */
    int32_t pad0;
} fro_pair_result;

/* Result of one two-way FM search. */
typedef struct fro_fm_result {
    int64_t cut_before, cut_after, wA_after, wB_after;
    int32_t tried;       /* moves made before the stopping rule */
    int32_t kept;        /* moves kept after the rollback (a prefix) */
} fro_fm_result;

/* Result of one k-way search (or the sum over several). */
typedef struct fro_kway_result {
    int64_t gain;        /* cut decrease kept (>= 0) */
    int32_t tried;       /* moves made before the stop */
    int32_t kept;        /* moves kept after the rollback (a prefix) */
    int32_t stop;        /* 1: the KaSPar rule stopped the (last) search; 0: empty queue */
    int32_t pad0;
} fro_kway_result;

/* Totals of multi-try passes. */
typedef struct fro_mt_result {
    int64_t gain;        /* cut decrease kept */
    int32_t searches;    /* k-way searches started */
    int32_t tried, kept; /* moves made / kept */
    int32_t pad0;
} fro_mt_result;

/* Multilevel V-cycle with a given partition (fro_vcycle). */
#define FRO_MAX_LEVELS 64
typedef struct fro_vcycle_result {
    int32_t levels;                      /* graphs in the hierarchy, the input included */
    int32_t pad0;
    int64_t cut_before, cut_after;       /* total cut of the input and the output partition */
    int32_t level_n[FRO_MAX_LEVELS];     /* vertices of each level (0 = the input) */
    int32_t level_pairs[FRO_MAX_LEVELS]; /* pair refinements run on each level */
    int64_t level_cut[FRO_MAX_LEVELS];   /* total cut after the level's refinement */
} fro_vcycle_result;

/* W-, F- (and V-) cycles with a given partition (fro_cycle). */
typedef struct fro_cycle_result {
    int32_t coarsenings;                       /* matchings computed (stalled ones included) */
    int32_t refinements;                       /* refinement sweeps run */
    int32_t depth;                             /* levels of the deepest branch */
    int32_t pad0;
    int64_t cut_before, cut_after;
    int32_t level_coarsenings[FRO_MAX_LEVELS]; /* coarsenings of level-l graphs */
} fro_cycle_result;

/* Input checks of Section 2.1 (omega > 0, c >= 0, symmetric simple CSR, 0 <= part < k). */
int32_t fro_validate(int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt,
                     const int32_t *vwgt, const int32_t *part, int32_t k);

/* W = c(V), max_v c(v), L_max and the per-call budget base floor((1+alpha*eps) W/k). */
int64_t fro_total_weight(int32_t n, const int32_t *vwgt);
int64_t fro_max_weight(int32_t n, const int32_t *vwgt);
int64_t fro_lmax(int64_t W, int64_t maxc, int32_t k, double eps);
int64_t fro_budget_base(int64_t W, int32_t k, double eps, double alpha);

/* ---- one flow problem: corridor + network + max flow + cuts ------------- */
typedef struct fro_problem fro_problem;

/* Corridor of pair (a, b) under budget base Ubase (Section 4.1). */
fro_problem *fro_build(int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt,
                       const int32_t *vwgt, const int32_t *part, int32_t a, int32_t b, int64_t Ubase);
/* A problem given directly as a network in the export format (for pins on arbitrary networks). */
fro_problem *fro_from_network(int32_t nc, const int32_t *off, const int32_t *head, const int32_t *cap,
                              const int8_t *border, const int32_t *infcap, const int32_t *vw,
                              const int8_t *side0, int64_t cA, int64_t cB);
void fro_free(fro_problem *p);

int32_t fro_nc(const fro_problem *p);   /* corridor vertices */
int32_t fro_m(const fro_problem *p);    /* corridor arcs (both directions of each edge) */
/* Export format: gid[nc] ascending; off[nc+1]; head/cap[m] (corridor arcs in CSR order);
 * border[nc] 0 none, 1 s -> v, 2 v -> t; infcap[nc] INF_v of border vertices (0 otherwise);
 * side0[nc] 0 = block a, 1 = block b; dist[nc] BFS distance inside its block. */
void fro_export(const fro_problem *p, int32_t *gid, int32_t *off, int32_t *head, int32_t *cap,
                int8_t *border, int32_t *infcap, int8_t *side0, int32_t *dist);

/* Max flow: method 0 = Dinic, 1 = Edmonds-Karp scanning arcs in reverse order. */
int64_t fro_maxflow(fro_problem *p, int32_t method);
/* Flow on corridor arcs (m) and on the s/t arc of each corridor vertex (nc). */
void fro_flow(const fro_problem *p, int64_t *arcflow, int64_t *stflow);
/* Residual sets after the max flow: in_s (reachable from s), to_t (reaches t),
 * comp (min gid of the vertex's residual SCC for vertices in neither, else -1). */
void fro_residual_sets(fro_problem *p, int8_t *in_s, int8_t *to_t, int32_t *comp);
/* Sweep r: writes component labels in sweep order and d[j] = c(A'_j) - c(B'_j) for
 * j = 0..ncomp; returns ncomp. */
int32_t fro_sweep(fro_problem *p, int32_t r, uint64_t seed, int32_t *order, int64_t *d);
/* Output sides (0 = source/A, 1 = sink/B) of the plain or MB cut; returns the cut
 * capacity in G' (must equal the flow). */
int64_t fro_cut(fro_problem *p, int32_t mb, int32_t reps, uint64_t seed, int8_t *side, int32_t *best_j,
                int32_t *best_r);

/* ---- full method --------------------------------------------------------- */
int32_t fro_refine_pair(int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt,
                        const int32_t *vwgt, int32_t *part, int32_t k, int32_t a, int32_t b, double eps,
                        double alpha, const fro_options *opt, fro_pair_result *res);

/* Two-way FM with TopGain on pair (a, b) (Section 2.2; stopping rule of Section 6):
 * moves vertices of a and b between the two blocks of part, then rolls back to the
 * best prefix.  moves (optional, moves_cap entries) receives every vertex moved, in
 * order, before the rollback.  FM keys: seed' = splitmix64(seed ^ a << 32 ^ b);
 * initial stamp of v = splitmix64(seed' ^ v) >> 1; the block tie at move i takes
 * b iff splitmix64(~seed' ^ i) is odd. */
int32_t fro_fm_pair(int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt,
                    const int32_t *vwgt, int32_t *part, int32_t a, int32_t b, int64_t Lmax, int32_t permille,
                    uint64_t seed, fro_fm_result *out, int32_t *moves, int32_t moves_cap);
uint64_t fro_fm_seed(uint64_t seed, int32_t a, int32_t b);

/* KaSPar stopping rule (Section 2.2): 1 iff p mu^2 > alpha sigma^2 + beta with
 * mu = S1/p, sigma^2 = S2/p - mu^2 (S1, S2: sum of the p gains and of their
 * squares), evaluated as the double expression (p*mu)*mu > alpha*sigma^2 + beta. */
int32_t fro_kaspar_stop(int32_t p, int64_t S1, int64_t S2, int32_t alpha, double beta);

/* One k-way local search (Section 2.2) from init[0..ninit) in that order, on part and
 * the block weights blockw[k] (both updated to the kept prefix).  touched (may be
 * NULL): multi-try marks, see fro_multitry; id >= 1 marks this search.  tseed keys
 * the target ties.  The logs (optional, log_cap entries) receive every move in
 * order before the rollback: vertex, target block, gain. */
int32_t fro_kway_search(int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt,
                        const int32_t *vwgt, int32_t *part, int32_t k, int64_t *blockw, int64_t Lmax,
                        const int32_t *init, int32_t ninit, int32_t *touched, int32_t id, int32_t alpha,
                        double beta, uint64_t tseed, fro_kway_result *out, int32_t *log_v, int32_t *log_to,
                        int64_t *log_gain, int32_t log_cap);

/* One multi-try FM pass (Section 4.2) over the pairs (pa[i], pb[i]) of a matching;
 * changed[k] (optional) marks every block a kept move left or entered. */
int32_t fro_multitry(int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt,
                     const int32_t *vwgt, int32_t *part, int32_t k, int64_t Lmax, int32_t np, const int32_t *pa,
                     const int32_t *pb, int32_t alpha, uint64_t seed, fro_mt_result *out, int8_t *changed);
uint64_t fro_mt_seed(uint64_t seed, int32_t a, int32_t b);

/* Global k-way refinement (Section 2.2, setup of Section 6): rounds of one k-way
 * search from the whole boundary (init_mode 0) or the corner vertices (1) until a
 * round finds no improvement or max_rounds ran. */
int32_t fro_kway_global(int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt,
                        const int32_t *vwgt, int32_t *part, int32_t k, double eps, int32_t init_mode,
                        int32_t alpha, int32_t max_rounds, uint64_t seed, fro_kway_result *out, int32_t *rounds);

/* Quotient graph rounds: pair list (a < b, lexicographic) with the colour of each pair. */
int32_t fro_rounds(int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *part, int32_t k,
                   int32_t cap, int32_t *pair_a, int32_t *pair_b, int32_t *pair_round, int32_t *nrounds);

/* One sweep over all rounds; per-pair results in round order, then (a, b) order. */
int32_t fro_refine_batch(int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt,
                         const int32_t *vwgt, int32_t *part, int32_t k, double eps, double alpha,
                         const fro_options *opt, int32_t cap, fro_pair_result *res, int32_t *npairs,
                         int32_t *nrounds);

/* The same sweep stopped after max_pairs pairs (a bounded sample for timing; all if < 0). */
int32_t fro_refine_batch_sample(int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt,
                                const int32_t *vwgt, int32_t *part, int32_t k, double eps, double alpha,
                                const fro_options *opt, int32_t max_pairs, int32_t *done);

/* The sweep of fro_refine_batch with the pairs of each round refined on up to
 * nthreads threads (pair-parallel CPU baseline; identical results, same order),
 * stopped after max_rounds rounds (all if < 0).  done = pairs refined. */
int32_t fro_refine_batch_mt(int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt,
                            const int32_t *vwgt, int32_t *part, int32_t k, double eps, double alpha,
                            const fro_options *opt, int32_t nthreads, int32_t max_rounds, int32_t cap,
                            fro_pair_result *res, int32_t *npairs, int32_t *nrounds, int32_t *done);

/* Active block scheduling with flow refinement of each scheduled pair (adaptive
 * flow iterations if opt->adaptive): outer rounds over the quotient edges with an
 * active end until no block is active or max_outer rounds ran.  Per-pair results in
 * processing order (round = matching index counted over all outer rounds).  With
 * opt->mt_alpha > 0 a multi-try pass follows each matching; mt (optional) receives
 * the totals of those passes. */
int32_t fro_refine_active(int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt,
                          const int32_t *vwgt, int32_t *part, int32_t k, double eps, double alpha,
                          const fro_options *opt, int32_t max_outer, int32_t cap, fro_pair_result *res,
                          int32_t *npairs, int32_t *nouter, fro_mt_result *mt);

/* Greedy matching of one level (Sections 2.2 and 5): edges inside one block whose ends
 * weigh at most 1.5 W / (20 k), ordered by expansion*2 (exact; c taken as max(c, 1)),
 * then by splitmix64(seed_l ^ min << 32 ^ max) (larger first), then by (min, max);
 * mate[v] = partner or -1.  Returns the matched pairs. */
int32_t fro_match(int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt, const int32_t *vwgt,
                  const int32_t *part, int32_t k, int64_t W, uint64_t seed_l, int32_t *mate);
/* Contraction of a matching (Section 2.1): coarse vertex of a pair or single vertex
 * numbered by its smaller fine id; rows sorted by coarse id, parallel edges merged.
 * cmap[n]; the coarse arrays need room for n + 1, nnz, nnz, n entries.  Returns nnz. */
int32_t fro_contract(int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt,
                     const int32_t *vwgt, const int32_t *mate, int32_t *cmap, int32_t *cn, int32_t *cxadj,
                     int32_t *cadjncy, int32_t *cadjwgt, int32_t *cvwgt);
/* One V-cycle with the given partition (Section 5): contract level by level with
 * fro_match (seed_l = splitmix64(opt->seed ^ level)) while the graph has more than
 * max(60 k, n / (60 k)) vertices, the matching holds at least n_level / 20 pairs and
 * fewer than max_levels levels exist; then from the coarsest level up, project and refine with one
 * fro_refine_batch sweep (or fro_refine_active with active_outer outer rounds). */
int32_t fro_vcycle(int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt,
                   const int32_t *vwgt, int32_t *part, int32_t k, double eps, double alpha, const fro_options *opt,
                   int32_t max_levels, int32_t active_outer, fro_vcycle_result *out);

/* A global search cycle with the given partition (Section 5): type 0 V-cycle (the same
 * result as fro_vcycle), 1 W-cycle, 2 F-cycle, level split parameter d >= 1.  The c-th
 * coarsening of a level-l graph uses seed_l = splitmix64(opt->seed ^ l ^ c << 32). */
int32_t fro_cycle(int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt, const int32_t *vwgt,
                  int32_t *part, int32_t k, double eps, double alpha, const fro_options *opt, int32_t type, int32_t d,
                  int32_t max_levels, int32_t active_outer, fro_cycle_result *out);

/* Pair cut omega(E_ab) of the current partition. */
int64_t fro_pair_cut(int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt,
                     const int32_t *part, int32_t a, int32_t b);

/* splitmix64(x): first output of a splitmix64 generator seeded with x. */
uint64_t fro_splitmix64(uint64_t x);

#ifdef __cplusplus
}
#endif
#endif
