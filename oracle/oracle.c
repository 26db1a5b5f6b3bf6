/*
 * CPU oracle for flow-based refinement of a block pair -- TEST INFRASTRUCTURE.
 *
 * Plain, deliberately unoptimised C; each pair is refined on one thread (the
 * pair-parallel sweep at the end only runs the pairs of a round side by side).
 * Each step follows the
 * paper's description in the paper's order (Sanders & Schulz, Section 4.1 and
 * 4.1.1); the readings of points the paper leaves open are listed in fro.h.
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg use it.
 * It shares no code with the CUDA path.
 */
#include "fro.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define XALLOC(T, n) ((T *)calloc((size_t)((n) > 0 ? (n) : 1), sizeof(T)))

uint64_t fro_splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* ------------------------------------------------ Section 2.1: the problem -- */

int32_t fro_validate(int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt,
                     const int32_t *vwgt, const int32_t *part, int32_t k) {
    if (n < 1 || k < 2 || !xadj || !adjncy || !adjwgt || !vwgt || !part) return FRO_ERR_INVALID_ARG;
    if (xadj[0] != 0) return FRO_ERR_INVALID_ARG;
    for (int32_t v = 0; v < n; ++v)
        if (xadj[v + 1] < xadj[v]) return FRO_ERR_INVALID_ARG;
    for (int32_t v = 0; v < n; ++v) {
        if (vwgt[v] < 0) return FRO_ERR_INVALID_ARG;           /* c >= 0 */
        if (part[v] < 0 || part[v] >= k) return FRO_ERR_INVALID_ARG;
        int64_t wdeg = 0;
        for (int32_t j = xadj[v]; j < xadj[v + 1]; ++j) {
            int32_t u = adjncy[j];
            if (u < 0 || u >= n || u == v) return FRO_ERR_INVALID_ARG;
            if (adjwgt[j] < 1) return FRO_ERR_INVALID_ARG;      /* omega > 0 */
            wdeg += adjwgt[j];
            /* simple graph: u appears once in v's row */
            for (int32_t q = xadj[v]; q < j; ++q)
                if (adjncy[q] == u) return FRO_ERR_INVALID_ARG;
            /* undirected: v appears in u's row with the same weight */
            int found = 0;
            for (int32_t q = xadj[u]; q < xadj[u + 1]; ++q)
                if (adjncy[q] == v) { found = adjwgt[q] == adjwgt[j] ? 1 : -1; break; }
            if (found != 1) return FRO_ERR_INVALID_ARG;
        }
        if (wdeg >= (1LL << 30)) return FRO_ERR_TOO_LARGE;
    }
    return FRO_OK;
}

int64_t fro_total_weight(int32_t n, const int32_t *vwgt) {
    int64_t w = 0;
    for (int32_t v = 0; v < n; ++v) w += vwgt[v];
    return w;
}

int64_t fro_max_weight(int32_t n, const int32_t *vwgt) {
    int64_t w = 0;
    for (int32_t v = 0; v < n; ++v) if (vwgt[v] > w) w = vwgt[v];
    return w;
}

/* L_max = (1 + eps) c(V)/k + max_v c(v), integerised: block weights are integers. */
int64_t fro_lmax(int64_t W, int64_t maxc, int32_t k, double eps) {
    double t = 1.0 + eps;
    t = t * (double)W;
    t = t / (double)k;
    return (int64_t)floor(t) + maxc;
}

/* Corridor budget base: (1 + eps') c(V)/k with eps' = alpha * eps. */
int64_t fro_budget_base(int64_t W, int32_t k, double eps, double alpha) {
    double ae = alpha * eps;
    double t = 1.0 + ae;
    t = t * (double)W;
    t = t / (double)k;
    return (int64_t)floor(t);
}

int64_t fro_pair_cut(int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt,
                     const int32_t *part, int32_t a, int32_t b) {
    int64_t cut = 0;
    for (int32_t v = 0; v < n; ++v) {
        if (part[v] != a) continue;
        for (int32_t j = xadj[v]; j < xadj[v + 1]; ++j)
            if (part[adjncy[j]] == b) cut += adjwgt[j];
    }
    return cut;
}

/* --------------------------------------------------- the flow problem ----- */

struct fro_problem {
    /* corridor and its network in the export format */
    int32_t nc, m;
    int32_t *gid, *off, *head, *cap, *infcap, *dist;
    int8_t *border, *side0;
    int64_t *vw;
    int64_t cA, cB;
    /* explicit network on N = nc + 2 vertices: s = nc, t = nc + 1 */
    int32_t N, M;
    int32_t *noff, *nhead, *nrev;
    int64_t *ncap, *nres;
    int64_t flow;
    int ok;
    /* residual structure */
    int8_t *in_s, *to_t;
    int32_t *comp;   /* SCC label (min gid) of vertices in neither set, else -1 */
    int sets_done;
};

void fro_free(fro_problem *p) {
    if (!p) return;
    free(p->gid); free(p->off); free(p->head); free(p->cap); free(p->infcap); free(p->dist);
    free(p->border); free(p->side0); free(p->vw);
    free(p->noff); free(p->nhead); free(p->nrev); free(p->ncap); free(p->nres);
    free(p->in_s); free(p->to_t); free(p->comp);
    free(p);
}

int32_t fro_nc(const fro_problem *p) { return p->nc; }
int32_t fro_m(const fro_problem *p) { return p->m; }

void fro_export(const fro_problem *p, int32_t *gid, int32_t *off, int32_t *head, int32_t *cap,
                int8_t *border, int32_t *infcap, int8_t *side0, int32_t *dist) {
    if (gid) memcpy(gid, p->gid, sizeof(int32_t) * (size_t)p->nc);
    if (off) memcpy(off, p->off, sizeof(int32_t) * (size_t)(p->nc + 1));
    if (head) memcpy(head, p->head, sizeof(int32_t) * (size_t)p->m);
    if (cap) memcpy(cap, p->cap, sizeof(int32_t) * (size_t)p->m);
    if (border) memcpy(border, p->border, (size_t)p->nc);
    if (infcap) memcpy(infcap, p->infcap, sizeof(int32_t) * (size_t)p->nc);
    if (side0) memcpy(side0, p->side0, (size_t)p->nc);
    if (dist) memcpy(dist, p->dist, sizeof(int32_t) * (size_t)p->nc);
}

/* Explicit network: corridor arcs of vertex i in export order, then its s/t arc;
 * s's arcs to s-border vertices and t's arcs to t-border vertices, ascending. */
static int build_network(fro_problem *p) {
    int32_t nc = p->nc, N = nc + 2, s = nc, t = nc + 1;
    p->N = N;
    p->noff = XALLOC(int32_t, N + 1);
    int32_t *deg = XALLOC(int32_t, N);
    for (int32_t i = 0; i < nc; ++i) {
        deg[i] = p->off[i + 1] - p->off[i] + (p->border[i] ? 1 : 0);
        if (p->border[i] == 1) deg[s]++;
        if (p->border[i] == 2) deg[t]++;
    }
    for (int32_t v = 0; v < N; ++v) p->noff[v + 1] = p->noff[v] + deg[v];
    int32_t M = p->noff[N];
    p->M = M;
    p->nhead = XALLOC(int32_t, M);
    p->nrev = XALLOC(int32_t, M);
    p->ncap = XALLOC(int64_t, M);
    p->nres = XALLOC(int64_t, M);
    int32_t *pos = XALLOC(int32_t, N);
    for (int32_t v = 0; v < N; ++v) pos[v] = p->noff[v];
    int32_t *stpos = XALLOC(int32_t, nc);   /* position of i's s/t arc */
    for (int32_t i = 0; i < nc; ++i) {
        for (int32_t j = p->off[i]; j < p->off[i + 1]; ++j) {
            int32_t a = pos[i]++;
            p->nhead[a] = p->head[j];
            p->ncap[a] = p->cap[j];
        }
        if (p->border[i] == 1) {          /* reverse of s -> i, capacity 0 */
            int32_t a = pos[i]++;
            p->nhead[a] = s; p->ncap[a] = 0; stpos[i] = a;
        } else if (p->border[i] == 2) {   /* i -> t, "infinite" capacity */
            int32_t a = pos[i]++;
            p->nhead[a] = t; p->ncap[a] = p->infcap[i]; stpos[i] = a;
        }
    }
    for (int32_t i = 0; i < nc; ++i) {
        if (p->border[i] == 1) {
            int32_t a = pos[s]++;
            p->nhead[a] = i; p->ncap[a] = p->infcap[i];
            p->nrev[a] = stpos[i]; p->nrev[stpos[i]] = a;
        } else if (p->border[i] == 2) {
            int32_t a = pos[t]++;
            p->nhead[a] = i; p->ncap[a] = 0;
            p->nrev[a] = stpos[i]; p->nrev[stpos[i]] = a;
        }
    }
    /* reverse of a corridor arc i -> h: the q-th arc h -> i, where q counts earlier i -> h arcs */
    int ok = 1;
    for (int32_t i = 0; i < nc && ok; ++i) {
        int32_t base = p->noff[i];
        int32_t ncorr = p->off[i + 1] - p->off[i];
        for (int32_t x = 0; x < ncorr; ++x) {
            int32_t h = p->nhead[base + x];
            int32_t q = 0;
            for (int32_t y = 0; y < x; ++y) if (p->nhead[base + y] == h) ++q;
            int32_t found = -1;
            int32_t hn = p->off[h + 1] - p->off[h];
            for (int32_t y = 0; y < hn; ++y)
                if (p->nhead[p->noff[h] + y] == i) { if (q == 0) { found = p->noff[h] + y; break; } --q; }
            if (found < 0) { ok = 0; break; }
            p->nrev[base + x] = found;
        }
    }
    for (int32_t a = 0; a < M; ++a) p->nres[a] = p->ncap[a];
    free(deg); free(pos); free(stpos);
    return ok;
}

/* Corridor side (Section 4.1): BFS inside block X from the vertices of X with a
 * neighbour in Y; reached vertices in (distance, id) order; longest prefix of
 * weight <= U.  Writes dist (n-sized, -1 = not taken). */
typedef struct { int32_t d, v; } dv_pair;

static int cmp_dv(const void *pa, const void *pb) {
    const dv_pair *a = (const dv_pair *)pa, *b = (const dv_pair *)pb;
    if (a->d != b->d) return a->d < b->d ? -1 : 1;
    return (a->v > b->v) - (a->v < b->v);
}

static void corridor_side(int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *vwgt,
                          const int32_t *part, int32_t X, int32_t Y, int64_t U, int32_t *taken_dist) {
    int32_t *dist = XALLOC(int32_t, n);
    int32_t *queue = XALLOC(int32_t, n);
    int32_t qh = 0, qt = 0;
    for (int32_t v = 0; v < n; ++v) dist[v] = -1;
    for (int32_t v = 0; v < n; ++v) {            /* boundary delta_X towards Y */
        if (part[v] != X) continue;
        for (int32_t j = xadj[v]; j < xadj[v + 1]; ++j)
            if (part[adjncy[j]] == Y) { dist[v] = 0; queue[qt++] = v; break; }
    }
    while (qh < qt) {                             /* expand only inside block X */
        int32_t v = queue[qh++];
        for (int32_t j = xadj[v]; j < xadj[v + 1]; ++j) {
            int32_t u = adjncy[j];
            if (part[u] == X && dist[u] < 0) { dist[u] = dist[v] + 1; queue[qt++] = u; }
        }
    }
    dv_pair *order = XALLOC(dv_pair, qt);
    for (int32_t i = 0; i < qt; ++i) { order[i].d = dist[queue[i]]; order[i].v = queue[i]; }
    qsort(order, (size_t)qt, sizeof(dv_pair), cmp_dv);
    int64_t run = 0;
    for (int32_t i = 0; i < qt; ++i) {            /* stop at the first vertex that would exceed */
        int32_t v = order[i].v;
        if (run + vwgt[v] > U) break;
        run += vwgt[v];
        taken_dist[v] = order[i].d;
    }
    free(order); free(queue); free(dist);
}

fro_problem *fro_build(int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt,
                       const int32_t *vwgt, const int32_t *part, int32_t a, int32_t b, int64_t Ubase) {
    fro_problem *p = XALLOC(fro_problem, 1);
    int64_t cA = 0, cB = 0;
    for (int32_t v = 0; v < n; ++v) {
        if (part[v] == a) cA += vwgt[v];
        else if (part[v] == b) cB += vwgt[v];
    }
    p->cA = cA; p->cB = cB;
    int64_t UA = Ubase - cB, UB = Ubase - cA;
    if (UA < 0) UA = 0;
    if (UB < 0) UB = 0;
    int32_t *tdist = XALLOC(int32_t, n);
    for (int32_t v = 0; v < n; ++v) tdist[v] = -1;
    corridor_side(n, xadj, adjncy, vwgt, part, a, b, UA, tdist);
    corridor_side(n, xadj, adjncy, vwgt, part, b, a, UB, tdist);
    /* local ids in ascending global id */
    int32_t *lid = XALLOC(int32_t, n);
    int32_t nc = 0;
    for (int32_t v = 0; v < n; ++v) lid[v] = tdist[v] >= 0 ? nc++ : -1;
    p->nc = nc;
    p->gid = XALLOC(int32_t, nc);
    p->dist = XALLOC(int32_t, nc);
    p->side0 = XALLOC(int8_t, nc);
    p->border = XALLOC(int8_t, nc);
    p->infcap = XALLOC(int32_t, nc);
    p->vw = XALLOC(int64_t, nc);
    p->off = XALLOC(int32_t, nc + 1);
    for (int32_t v = 0; v < n; ++v)
        if (lid[v] >= 0) {
            int32_t i = lid[v];
            p->gid[i] = v; p->dist[i] = tdist[v]; p->side0[i] = part[v] == b; p->vw[i] = vwgt[v];
        }
    /* G' = G[B] plus s, t (Section 4.1); border w.r.t. G[A u B] */
    int32_t m = 0;
    for (int32_t i = 0; i < nc; ++i) {
        int32_t v = p->gid[i];
        int64_t wdeg = 0;
        int border = 0;
        for (int32_t j = xadj[v]; j < xadj[v + 1]; ++j) {
            int32_t u = adjncy[j];
            wdeg += adjwgt[j];
            if (part[u] != a && part[u] != b) continue;
            if (lid[u] >= 0) ++m; else border = 1;
        }
        p->off[i + 1] = m;
        if (border) {
            p->border[i] = p->side0[i] ? 2 : 1;
            p->infcap[i] = (int32_t)(wdeg + 1);
        }
    }
    p->m = m;
    p->head = XALLOC(int32_t, m);
    p->cap = XALLOC(int32_t, m);
    int32_t e = 0;
    for (int32_t i = 0; i < nc; ++i) {
        int32_t v = p->gid[i];
        for (int32_t j = xadj[v]; j < xadj[v + 1]; ++j) {
            int32_t u = adjncy[j];
            if ((part[u] == a || part[u] == b) && lid[u] >= 0) { p->head[e] = lid[u]; p->cap[e] = adjwgt[j]; ++e; }
        }
    }
    free(lid); free(tdist);
    p->ok = build_network(p);
    return p;
}

fro_problem *fro_from_network(int32_t nc, const int32_t *off, const int32_t *head, const int32_t *cap,
                              const int8_t *border, const int32_t *infcap, const int32_t *vw,
                              const int8_t *side0, int64_t cA, int64_t cB) {
    fro_problem *p = XALLOC(fro_problem, 1);
    p->nc = nc; p->m = off[nc]; p->cA = cA; p->cB = cB;
    p->gid = XALLOC(int32_t, nc); p->dist = XALLOC(int32_t, nc);
    p->off = XALLOC(int32_t, nc + 1); p->head = XALLOC(int32_t, p->m); p->cap = XALLOC(int32_t, p->m);
    p->border = XALLOC(int8_t, nc); p->infcap = XALLOC(int32_t, nc); p->side0 = XALLOC(int8_t, nc);
    p->vw = XALLOC(int64_t, nc);
    for (int32_t i = 0; i < nc; ++i) {
        p->gid[i] = i; p->border[i] = border[i]; p->infcap[i] = infcap[i];
        p->side0[i] = side0[i]; p->vw[i] = vw[i];
    }
    memcpy(p->off, off, sizeof(int32_t) * (size_t)(nc + 1));
    memcpy(p->head, head, sizeof(int32_t) * (size_t)p->m);
    memcpy(p->cap, cap, sizeof(int32_t) * (size_t)p->m);
    p->ok = build_network(p);
    return p;
}

/* ------------------------------------------------------------ max flow ---- */

/* Dinic: BFS level graph from s, then blocking flow by DFS with current-arc pointers. */
static int64_t maxflow_dinic(fro_problem *p) {
    int32_t N = p->N, s = p->nc, t = p->nc + 1;
    int32_t *level = XALLOC(int32_t, N), *queue = XALLOC(int32_t, N), *it = XALLOC(int32_t, N);
    int32_t *stack = XALLOC(int32_t, N + 1);   /* arcs of the current path */
    int64_t flow = 0;
    for (;;) {
        for (int32_t v = 0; v < N; ++v) level[v] = -1;
        int32_t qh = 0, qt = 0;
        level[s] = 0; queue[qt++] = s;
        while (qh < qt) {
            int32_t v = queue[qh++];
            for (int32_t a = p->noff[v]; a < p->noff[v + 1]; ++a) {
                int32_t u = p->nhead[a];
                if (p->nres[a] > 0 && level[u] < 0) { level[u] = level[v] + 1; queue[qt++] = u; }
            }
        }
        if (level[t] < 0) break;
        for (int32_t v = 0; v < N; ++v) it[v] = p->noff[v];
        int32_t depth = 0, v = s;
        for (;;) {
            if (v == t) {
                int64_t aug = INT64_MAX;
                for (int32_t d = 0; d < depth; ++d) if (p->nres[stack[d]] < aug) aug = p->nres[stack[d]];
                for (int32_t d = 0; d < depth; ++d) {
                    p->nres[stack[d]] -= aug;
                    p->nres[p->nrev[stack[d]]] += aug;
                }
                flow += aug;
                depth = 0; v = s;
                continue;
            }
            int advanced = 0;
            for (; it[v] < p->noff[v + 1]; ++it[v]) {
                int32_t a = it[v], u = p->nhead[a];
                if (p->nres[a] > 0 && level[u] == level[v] + 1) {
                    stack[depth++] = a; v = u; advanced = 1;
                    break;
                }
            }
            if (advanced) continue;
            if (v == s) break;                      /* blocking flow complete */
            level[v] = -1;                          /* dead end: retreat */
            int32_t a = stack[--depth];
            v = p->nhead[p->nrev[a]];
            ++it[v];
        }
    }
    free(level); free(queue); free(it); free(stack);
    return flow;
}

/* Edmonds-Karp with arcs scanned last to first: a second, independent max flow. */
static int64_t maxflow_ek_reverse(fro_problem *p) {
    int32_t N = p->N, s = p->nc, t = p->nc + 1;
    int32_t *parent = XALLOC(int32_t, N), *queue = XALLOC(int32_t, N);
    int64_t flow = 0;
    for (;;) {
        for (int32_t v = 0; v < N; ++v) parent[v] = -2;
        parent[s] = -1;
        int32_t qh = 0, qt = 0;
        queue[qt++] = s;
        while (qh < qt && parent[t] == -2) {
            int32_t v = queue[qh++];
            for (int32_t a = p->noff[v + 1] - 1; a >= p->noff[v]; --a) {
                int32_t u = p->nhead[a];
                if (p->nres[a] > 0 && parent[u] == -2) { parent[u] = a; queue[qt++] = u; }
            }
        }
        if (parent[t] == -2) break;
        int64_t aug = INT64_MAX;
        for (int32_t v = t; v != s; v = p->nhead[p->nrev[parent[v]]])
            if (p->nres[parent[v]] < aug) aug = p->nres[parent[v]];
        for (int32_t v = t; v != s; v = p->nhead[p->nrev[parent[v]]]) {
            p->nres[parent[v]] -= aug;
            p->nres[p->nrev[parent[v]]] += aug;
        }
        flow += aug;
    }
    free(parent); free(queue);
    return flow;
}

int64_t fro_maxflow(fro_problem *p, int32_t method) {
    if (!p->ok) return -1;
    for (int32_t a = 0; a < p->M; ++a) p->nres[a] = p->ncap[a];
    p->flow = method == 1 ? maxflow_ek_reverse(p) : maxflow_dinic(p);
    p->sets_done = 0;
    return p->flow;
}

void fro_flow(const fro_problem *p, int64_t *arcflow, int64_t *stflow) {
    for (int32_t i = 0; i < p->nc; ++i) {
        int32_t ncorr = p->off[i + 1] - p->off[i];
        for (int32_t x = 0; x < ncorr; ++x) {
            int32_t a = p->noff[i] + x;
            if (arcflow) arcflow[p->off[i] + x] = p->ncap[a] - p->nres[a];
        }
        if (stflow) {
            stflow[i] = 0;
            if (p->border[i]) {
                int32_t a = p->noff[i + 1] - 1;     /* i's s/t arc */
                stflow[i] = p->border[i] == 1 ? p->nres[a] /* flow on s -> i */ : p->ncap[a] - p->nres[a];
            }
        }
    }
}

/* ----------------------------------------- residual structure (4.1.1) ----- */

/* Tarjan's SCC algorithm, iterative, on the residual graph (arcs with res > 0). */
static void tarjan(const fro_problem *p, int32_t *scc) {
    int32_t N = p->N;
    int32_t *index = XALLOC(int32_t, N), *low = XALLOC(int32_t, N), *stk = XALLOC(int32_t, N);
    int32_t *cs_v = XALLOC(int32_t, N), *cs_a = XALLOC(int32_t, N);
    int8_t *on = XALLOC(int8_t, N);
    for (int32_t v = 0; v < N; ++v) { index[v] = -1; scc[v] = -1; }
    int32_t counter = 0, sp = 0, nscc = 0;
    for (int32_t root = 0; root < N; ++root) {
        if (index[root] >= 0) continue;
        int32_t csp = 0;
        cs_v[csp] = root; cs_a[csp] = p->noff[root]; ++csp;
        index[root] = low[root] = counter++; stk[sp++] = root; on[root] = 1;
        while (csp > 0) {
            int32_t v = cs_v[csp - 1];
            if (cs_a[csp - 1] < p->noff[v + 1]) {
                int32_t a = cs_a[csp - 1]++;
                if (p->nres[a] <= 0) continue;
                int32_t u = p->nhead[a];
                if (index[u] < 0) {
                    index[u] = low[u] = counter++; stk[sp++] = u; on[u] = 1;
                    cs_v[csp] = u; cs_a[csp] = p->noff[u]; ++csp;
                } else if (on[u] && index[u] < low[v]) {
                    low[v] = index[u];
                }
            } else {
                if (low[v] == index[v]) {
                    int32_t w;
                    do { w = stk[--sp]; on[w] = 0; scc[w] = nscc; } while (w != v);
                    ++nscc;
                }
                --csp;
                if (csp > 0) {
                    int32_t parent = cs_v[csp - 1];
                    if (low[v] < low[parent]) low[parent] = low[v];
                }
            }
        }
    }
    free(index); free(low); free(stk); free(cs_v); free(cs_a); free(on);
}

static void compute_sets(fro_problem *p) {
    if (p->sets_done) return;
    int32_t N = p->N, s = p->nc, t = p->nc + 1, nc = p->nc;
    free(p->in_s); free(p->to_t); free(p->comp);
    p->in_s = XALLOC(int8_t, N); p->to_t = XALLOC(int8_t, N); p->comp = XALLOC(int32_t, N);
    int32_t *queue = XALLOC(int32_t, N);
    /* vertices reachable from s (Ford-Fulkerson labelling) */
    int32_t qh = 0, qt = 0;
    p->in_s[s] = 1; queue[qt++] = s;
    while (qh < qt) {
        int32_t v = queue[qh++];
        for (int32_t a = p->noff[v]; a < p->noff[v + 1]; ++a)
            if (p->nres[a] > 0 && !p->in_s[p->nhead[a]]) { p->in_s[p->nhead[a]] = 1; queue[qt++] = p->nhead[a]; }
    }
    /* vertices that reach t: walk residual arcs backwards */
    qh = qt = 0;
    p->to_t[t] = 1; queue[qt++] = t;
    while (qh < qt) {
        int32_t v = queue[qh++];
        for (int32_t a = p->noff[v]; a < p->noff[v + 1]; ++a) {
            int32_t u = p->nhead[a];
            if (p->nres[p->nrev[a]] > 0 && !p->to_t[u]) { p->to_t[u] = 1; queue[qt++] = u; }
        }
    }
    /* SCCs of the residual graph, labelled by the minimum global id of their members */
    int32_t *scc = XALLOC(int32_t, N);
    tarjan(p, scc);
    int32_t *minid = XALLOC(int32_t, N);
    for (int32_t v = 0; v < N; ++v) minid[v] = INT32_MAX;
    for (int32_t v = 0; v < nc; ++v) if (p->gid[v] < minid[scc[v]]) minid[scc[v]] = p->gid[v];
    for (int32_t v = 0; v < N; ++v)
        p->comp[v] = (v < nc && !p->in_s[v] && !p->to_t[v]) ? minid[scc[v]] : -1;
    free(scc); free(minid); free(queue);
    p->sets_done = 1;
}

void fro_residual_sets(fro_problem *p, int8_t *in_s, int8_t *to_t, int32_t *comp) {
    compute_sets(p);
    for (int32_t i = 0; i < p->nc; ++i) {
        if (in_s) in_s[i] = p->in_s[i];
        if (to_t) to_t[i] = p->to_t[i];
        if (comp) comp[i] = p->comp[i];
    }
}

/* ---------------------------------------------- topological sweeps ------- */

typedef struct { uint64_t k1; int32_t minid; int32_t c; } heap_item;

static int item_less(const heap_item *x, const heap_item *y) {
    if (x->k1 != y->k1) return x->k1 < y->k1;
    return x->minid < y->minid;
}

static void heap_push(heap_item *h, int32_t *hn, heap_item it) {
    int32_t i = (*hn)++;
    h[i] = it;
    while (i > 0) {
        int32_t par = (i - 1) / 2;
        if (!item_less(&h[i], &h[par])) break;
        heap_item tmp = h[i]; h[i] = h[par]; h[par] = tmp;
        i = par;
    }
}

static heap_item heap_pop(heap_item *h, int32_t *hn) {
    heap_item top = h[0];
    h[0] = h[--(*hn)];
    int32_t i = 0;
    for (;;) {
        int32_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < *hn && item_less(&h[l], &h[m])) m = l;
        if (r < *hn && item_less(&h[r], &h[m])) m = r;
        if (m == i) break;
        heap_item tmp = h[i]; h[i] = h[m]; h[m] = tmp;
        i = m;
    }
    return top;
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Sweep r over the DAG of residual SCCs outside the S and T sets (Section 4.1.1):
 * Kahn's algorithm in residual arc direction (a component is ready once all of its
 * residual predecessors are on the sink side); ready components leave a min-heap
 * by key.  order[j] = label of the j-th component moved to the sink side;
 * d[j] = c(A'_j) - c(B'_j) after j moves.  Returns the number of components. */
int32_t fro_sweep(fro_problem *p, int32_t r, uint64_t seed, int32_t *order, int64_t *d) {
    compute_sets(p);
    int32_t nc = p->nc;
    int32_t *labels = XALLOC(int32_t, nc);
    int32_t nl = 0;
    for (int32_t i = 0; i < nc; ++i) if (p->comp[i] >= 0) labels[nl++] = p->comp[i];
    qsort(labels, (size_t)nl, sizeof(int32_t), cmp_i32);
    int32_t ncomp = 0;
    for (int32_t i = 0; i < nl; ++i) if (i == 0 || labels[i] != labels[i - 1]) labels[ncomp++] = labels[i];
    /* component index of each vertex via binary search over the sorted labels */
    int32_t *cidx = XALLOC(int32_t, nc);
    int64_t *cw = XALLOC(int64_t, ncomp);
    for (int32_t i = 0; i < nc; ++i) {
        cidx[i] = -1;
        if (p->comp[i] < 0) continue;
        int32_t lo = 0, hi = ncomp - 1;
        while (lo < hi) { int32_t mid = (lo + hi) / 2; if (labels[mid] < p->comp[i]) lo = mid + 1; else hi = mid; }
        cidx[i] = lo;
        cw[lo] += p->vw[i];
    }
    /* DAG arcs between components (with multiplicity) */
    int32_t *indeg = XALLOC(int32_t, ncomp), *outdeg = XALLOC(int32_t, ncomp + 1);
    for (int32_t i = 0; i < nc; ++i) {
        if (cidx[i] < 0) continue;
        for (int32_t a = p->noff[i]; a < p->noff[i + 1]; ++a) {
            int32_t u = p->nhead[a];
            if (p->nres[a] <= 0 || u >= nc || cidx[u] < 0 || cidx[u] == cidx[i]) continue;
            indeg[cidx[u]]++; outdeg[cidx[i] + 1]++;
        }
    }
    for (int32_t c = 0; c < ncomp; ++c) outdeg[c + 1] += outdeg[c];
    int32_t *outs = XALLOC(int32_t, outdeg[ncomp]);
    int32_t *fill = XALLOC(int32_t, ncomp);
    for (int32_t i = 0; i < nc; ++i) {
        if (cidx[i] < 0) continue;
        for (int32_t a = p->noff[i]; a < p->noff[i + 1]; ++a) {
            int32_t u = p->nhead[a];
            if (p->nres[a] <= 0 || u >= nc || cidx[u] < 0 || cidx[u] == cidx[i]) continue;
            outs[outdeg[cidx[i]] + fill[cidx[i]]++] = cidx[u];
        }
    }
    /* d_0: source side = everything that does not reach t */
    int64_t cA0 = p->cA;
    for (int32_t i = 0; i < nc; ++i) {
        if (!p->side0[i] && p->to_t[i]) cA0 -= p->vw[i];
        if (p->side0[i] && !p->to_t[i]) cA0 += p->vw[i];
    }
    int64_t total = p->cA + p->cB;
    d[0] = cA0 - (total - cA0);
    heap_item *heap = XALLOC(heap_item, ncomp);
    int32_t hn = 0, done = 0;
    for (int32_t c = 0; c < ncomp; ++c)
        if (indeg[c] == 0) {
            heap_item it = { r == 0 ? 0 : fro_splitmix64(seed ^ (uint64_t)r ^ (uint64_t)labels[c]), labels[c], c };
            heap_push(heap, &hn, it);
        }
    while (hn > 0) {
        heap_item top = heap_pop(heap, &hn);
        order[done] = top.minid;
        d[done + 1] = d[done] - 2 * cw[top.c];
        ++done;
        for (int32_t e = outdeg[top.c]; e < outdeg[top.c + 1]; ++e) {
            int32_t c = outs[e];
            if (--indeg[c] == 0) {
                heap_item it = { r == 0 ? 0 : fro_splitmix64(seed ^ (uint64_t)r ^ (uint64_t)labels[c]), labels[c], c };
                heap_push(heap, &hn, it);
            }
        }
    }
    free(labels); free(cidx); free(cw); free(indeg); free(outdeg); free(outs); free(fill); free(heap);
    return done == ncomp ? ncomp : -1;
}

static int64_t abs64(int64_t x) { return x < 0 ? -x : x; }

int64_t fro_cut(fro_problem *p, int32_t mb, int32_t reps, uint64_t seed, int8_t *side, int32_t *best_j,
                int32_t *best_r) {
    compute_sets(p);
    int32_t nc = p->nc, N = p->N;
    int8_t *src = XALLOC(int8_t, N);
    for (int32_t v = 0; v < N; ++v) src[v] = p->in_s[v];     /* smallest source set */
    int32_t bj = -1, br = -1;
    if (mb) {
        int32_t *order = XALLOC(int32_t, nc + 1), *best_order = XALLOC(int32_t, nc + 1);
        int64_t *d = XALLOC(int64_t, nc + 2);
        int64_t best = INT64_MAX;
        int32_t ncomp = 0;
        for (int32_t r = 0; r < (reps < 1 ? 1 : reps); ++r) {
            ncomp = fro_sweep(p, r, seed, order, d);
            if (ncomp < 0) break;
            for (int32_t j = 0; j <= ncomp; ++j) {
                int64_t ad = abs64(d[j]);
                if (ad < best || (ad == best && j < bj)) {
                    best = ad; bj = j; br = r;
                    memcpy(best_order, order, sizeof(int32_t) * (size_t)ncomp);
                }
            }
        }
        if (ncomp >= 0) {
            /* source side = complement of (T set u first bj components of sweep br) */
            for (int32_t i = 0; i < nc; ++i) {
                if (p->comp[i] < 0) continue;
                int moved = 0;
                for (int32_t j = 0; j < bj; ++j) if (best_order[j] == p->comp[i]) { moved = 1; break; }
                src[i] = !moved;
            }
        }
        free(order); free(best_order); free(d);
    }
    int64_t capv = 0;
    for (int32_t v = 0; v < N; ++v) {
        if (!src[v]) continue;
        for (int32_t a = p->noff[v]; a < p->noff[v + 1]; ++a)
            if (!src[p->nhead[a]]) capv += p->ncap[a];
    }
    if (side) for (int32_t i = 0; i < nc; ++i) side[i] = src[i] ? 0 : 1;
    if (best_j) *best_j = bj;
    if (best_r) *best_r = br;
    free(src);
    return capv;
}

/* ------------------------------------------ two-way FM, TopGain (2.2) ---- */

/* Section 2.2 (two-way local search as in KaPPa): one priority queue of movable
 * vertices per block, keyed by the gain (the decrease of the pair cut when the
 * vertex moves to the other block); each vertex moves at most once; the queues
 * start with the boundary vertices in random order; TopGain takes the block whose
 * best vertex has the larger gain (random tie), but the heavier block while a block
 * is overloaded; after the stopping rule the moves are rolled back to the best cut
 * found within the balance constraint.  Section 6 (setup) gives the stopping rule:
 * stop once more than a fraction of the pair's vertices moved without an
 * improvement.  Readings (also in the header): gains and the boundary are taken
 * within G[A u B]; a queue holds the unmoved vertices of its block with an edge to
 * the other block; keys order by gain, then by stamp (larger first: the initial
 * stamps are random 63-bit values, every later insertion or gain change takes a
 * larger stamp than any before, one per adjacency position of the moved vertex);
 * "best" is the smallest (overload, cut, max block weight). */

typedef struct { int64_t gain; uint64_t stamp; int32_t v; } fm_key;

static int fm_better(const fm_key *x, const fm_key *y) {
    if (x->gain != y->gain) return x->gain > y->gain;
    if (x->stamp != y->stamp) return x->stamp > y->stamp;
    return x->v < y->v;
}

typedef struct { fm_key *h; int32_t n; int32_t *pos; } fm_heap;   /* max-heap, pos[v] = index or -1 */

static void fm_swap(fm_heap *q, int32_t i, int32_t j) {
    fm_key t = q->h[i]; q->h[i] = q->h[j]; q->h[j] = t;
    q->pos[q->h[i].v] = i; q->pos[q->h[j].v] = j;
}
static void fm_up(fm_heap *q, int32_t i) {
    while (i > 0 && fm_better(&q->h[i], &q->h[(i - 1) / 2])) { fm_swap(q, i, (i - 1) / 2); i = (i - 1) / 2; }
}
static void fm_down(fm_heap *q, int32_t i) {
    for (;;) {
        int32_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < q->n && fm_better(&q->h[l], &q->h[m])) m = l;
        if (r < q->n && fm_better(&q->h[r], &q->h[m])) m = r;
        if (m == i) return;
        fm_swap(q, i, m);
        i = m;
    }
}
static void fm_set(fm_heap *q, fm_key k) {   /* insert, or replace the key of k.v */
    int32_t i = q->pos[k.v];
    if (i < 0) { i = q->n++; q->h[i] = k; q->pos[k.v] = i; }
    else q->h[i] = k;
    fm_up(q, i);
    fm_down(q, q->pos[k.v]);
}
static void fm_remove(fm_heap *q, int32_t v) {
    int32_t i = q->pos[v];
    if (i < 0) return;
    int32_t last = --q->n;
    if (i != last) {
        fm_swap(q, i, last);
        q->pos[v] = -1;
        fm_up(q, i);
        fm_down(q, i);
    } else {
        q->pos[v] = -1;
    }
}

uint64_t fro_fm_seed(uint64_t seed, int32_t a, int32_t b) {
    return fro_splitmix64(seed ^ ((uint64_t)(uint32_t)a << 32) ^ (uint64_t)(uint32_t)b);
}

int32_t fro_fm_pair(int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt,
                    const int32_t *vwgt, int32_t *part, int32_t a, int32_t b, int64_t Lmax, int32_t permille,
                    uint64_t seed, fro_fm_result *out, int32_t *moves, int32_t moves_cap) {
    memset(out, 0, sizeof(*out));
    if (permille <= 0) return FRO_OK;
    const uint64_t fs = fro_fm_seed(seed, a, b);
    int64_t *in = XALLOC(int64_t, n), *ext = XALLOC(int64_t, n);
    int8_t *moved = XALLOC(int8_t, n);
    int32_t *log = XALLOC(int32_t, n);
    fm_heap q[2];
    for (int s = 0; s < 2; ++s) {
        q[s].h = XALLOC(fm_key, n);
        q[s].n = 0;
        q[s].pos = XALLOC(int32_t, n);
        for (int32_t v = 0; v < n; ++v) q[s].pos[v] = -1;
    }
    int64_t N = 0, wA = 0, wB = 0, cut = 0;
    for (int32_t v = 0; v < n; ++v) {
        if (part[v] != a && part[v] != b) continue;
        ++N;
        if (part[v] == a) wA += vwgt[v]; else wB += vwgt[v];
        for (int32_t j = xadj[v]; j < xadj[v + 1]; ++j) {
            const int32_t u = adjncy[j];
            if (part[u] == part[v]) in[v] += adjwgt[j];
            else if (part[u] == a || part[u] == b) { ext[v] += adjwgt[j]; if (v < u) cut += adjwgt[j]; }
        }
    }
    /* initial queues: the boundary vertices, stamps random (63 bits) */
    for (int32_t v = 0; v < n; ++v) {
        if ((part[v] != a && part[v] != b) || ext[v] == 0) continue;
        fm_key k = { ext[v] - in[v], fro_splitmix64(fs ^ (uint64_t)(uint32_t)v) >> 1, v };
        fm_set(&q[part[v] == a ? 0 : 1], k);
    }
    const int64_t limit = (int64_t)permille * N / 1000;
    uint64_t t = 0;   /* stamps handed out after the start: (1 << 63) + t */
    int64_t best_cut = cut, best_wA = wA, best_wB = wB;
    int32_t nm = 0, best_len = 0;
    int64_t idle = 0;
    out->cut_before = cut;
    for (;;) {
        if (q[0].n == 0 && q[1].n == 0) break;
        int s;
        if (wA > Lmax || wB > Lmax) {
            s = wA >= wB ? 0 : 1;                     /* the heavier block while one is overloaded */
            if (q[s].n == 0) s = 1 - s;
        } else if (q[0].n == 0) {
            s = 1;
        } else if (q[1].n == 0) {
            s = 0;
        } else if (q[0].h[0].gain != q[1].h[0].gain) {
            s = q[0].h[0].gain > q[1].h[0].gain ? 0 : 1;
        } else {
            s = (int)(fro_splitmix64(~fs ^ (uint64_t)nm) & 1);   /* random tie of the top gains */
        }
        const int32_t v = q[s].h[0].v;
        const int64_t g = q[s].h[0].gain;
        fm_remove(&q[s], v);
        const int32_t from = s ? b : a, to = s ? a : b;
        part[v] = to;
        moved[v] = 1;
        log[nm++] = v;
        cut -= g;
        if (s == 0) { wA -= vwgt[v]; wB += vwgt[v]; } else { wB -= vwgt[v]; wA += vwgt[v]; }
        for (int32_t j = xadj[v]; j < xadj[v + 1]; ++j) {
            const int32_t u = adjncy[j];
            if (moved[u] || (part[u] != a && part[u] != b)) continue;
            if (part[u] == from) { in[u] -= adjwgt[j]; ext[u] += adjwgt[j]; }
            else { in[u] += adjwgt[j]; ext[u] -= adjwgt[j]; }
            fm_heap *qu = &q[part[u] == a ? 0 : 1];
            if (ext[u] > 0) {
                fm_key k = { ext[u] - in[u], (1ULL << 63) + t + (uint64_t)(j - xadj[v]), u };
                fm_set(qu, k);
            } else {
                fm_remove(qu, u);
            }
        }
        t += (uint64_t)(xadj[v + 1] - xadj[v]);
        /* best: smallest (overload, cut, max block weight) */
        const int64_t mx = wA > wB ? wA : wB, bmx = best_wA > best_wB ? best_wA : best_wB;
        const int64_t ov = mx > Lmax ? mx - Lmax : 0, bov = bmx > Lmax ? bmx - Lmax : 0;
        if (ov < bov || (ov == bov && (cut < best_cut || (cut == best_cut && mx < bmx)))) {
            best_cut = cut; best_wA = wA; best_wB = wB; best_len = nm; idle = 0;
        } else if (++idle > limit) {
            break;
        }
    }
    for (int32_t i = 0; i < nm && i < moves_cap; ++i) moves[i] = log[i];
    for (int32_t i = nm - 1; i >= best_len; --i) part[log[i]] = part[log[i]] == a ? b : a;   /* roll back */
    out->tried = nm;
    out->kept = best_len;
    out->cut_after = best_cut;
    out->wA_after = best_wA;
    out->wB_after = best_wB;
    for (int s = 0; s < 2; ++s) { free(q[s].h); free(q[s].pos); }
    free(in); free(ext); free(moved); free(log);
    return FRO_OK;
}

/* ------------------------------------- refinement of one pair (4.1) ------ */

static int bad_fm(const fro_options *opt) { return opt && (opt->fm_permille < 0 || opt->fm_permille > 1000); }
/* multi-try FM runs in active block scheduling only; elsewhere mt_alpha must be 0 */
static int bad_mt(const fro_options *opt) { return opt && opt->mt_alpha != 0; }

static int32_t check_pair_args(int32_t k, int32_t a, int32_t b, double eps, double alpha, const fro_options *opt) {
    if (k < 2 || a < 0 || b < 0 || a >= k || b >= k || a == b) return FRO_ERR_INVALID_ARG;
    if (!(eps > 0.0) || !(alpha >= 1.0)) return FRO_ERR_INVALID_ARG;
    if (opt && (opt->mb_reps < 0 || opt->max_iters < 0 || (opt->adaptive && !(opt->alpha_max >= 1.0)) ||
                opt->fm_permille < 0 || opt->fm_permille > 1000 || opt->mt_alpha != 0))
        return FRO_ERR_INVALID_ARG;
    return FRO_OK;
}

static int32_t refine_pair_core(int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt,
                                const int32_t *vwgt, int32_t *part, int32_t k, int32_t a, int32_t b, double eps,
                                double alpha, const fro_options *opt, int64_t W, int64_t Lmax,
                                fro_pair_result *res) {
    int32_t mb = opt ? opt->mb : 0, reps = opt && opt->mb_reps > 0 ? opt->mb_reps : 1;
    int32_t adaptive = opt ? opt->adaptive : 0;
    int32_t max_iters = adaptive ? (opt && opt->max_iters > 0 ? opt->max_iters : 10) : 1;
    double alpha_max = adaptive ? opt->alpha_max : alpha;
    uint64_t seed = opt ? opt->seed : 0;
    memset(res, 0, sizeof(*res));
    res->a = a; res->b = b;
    int64_t cut = fro_pair_cut(n, xadj, adjncy, adjwgt, part, a, b);
    int64_t wA = 0, wB = 0;
    for (int32_t v = 0; v < n; ++v) { if (part[v] == a) wA += vwgt[v]; else if (part[v] == b) wB += vwgt[v]; }
    res->cut_before = cut; res->wA_before = wA; res->wB_before = wB;
    if (opt && opt->fm_permille > 0) {
        /* pairwise improvement: FM first, then the flows on its result (Section 6 setup) */
        fro_fm_result fr;
        fro_fm_pair(n, xadj, adjncy, adjwgt, vwgt, part, a, b, Lmax, opt->fm_permille, seed, &fr, NULL, 0);
        cut = fr.cut_after; wA = fr.wA_after; wB = fr.wB_after;
        res->fm_moves = fr.kept;
    }
    res->cut_fm = cut;
    int32_t *trial = XALLOC(int32_t, n);
    double al = alpha;
    int32_t iters = 0;
    while (iters < max_iters) {
        ++iters;
        fro_problem *p = fro_build(n, xadj, adjncy, adjwgt, vwgt, part, a, b, fro_budget_base(W, k, eps, al));
        int64_t F = fro_maxflow(p, 0);
        int8_t *side = XALLOC(int8_t, p->nc);
        fro_cut(p, mb, reps, seed, side, NULL, NULL);
        memcpy(trial, part, sizeof(int32_t) * (size_t)n);
        for (int32_t i = 0; i < p->nc; ++i) trial[p->gid[i]] = side[i] ? b : a;
        res->flow = F; res->corridor_n = p->nc; res->corridor_arcs = p->m;
        free(side);
        fro_free(p);
        int64_t ncut = fro_pair_cut(n, xadj, adjncy, adjwgt, trial, a, b);
        int64_t nA = 0, nB = 0;
        for (int32_t v = 0; v < n; ++v) { if (trial[v] == a) nA += vwgt[v]; else if (trial[v] == b) nB += vwgt[v]; }
        int64_t nmax = nA > nB ? nA : nB, omax = wA > wB ? wA : wB;
        int feasible = nmax <= Lmax;
        if (feasible && ncut < cut) {
            memcpy(part, trial, sizeof(int32_t) * (size_t)n);
            cut = ncut; wA = nA; wB = nB; res->accepted = 1;
            if (!adaptive) break;
            al = 2.0 * al < alpha_max ? 2.0 * al : alpha_max;
            continue;
        }
        if (feasible) {
            if (ncut == cut && nmax < omax) {
                memcpy(part, trial, sizeof(int32_t) * (size_t)n);
                cut = ncut; wA = nA; wB = nB; res->accepted = 1;
            }
            break;
        }
        if (!adaptive || al == 1.0) break;
        al = al / 2.0 > 1.0 ? al / 2.0 : 1.0;
    }
    res->iters = iters;
    res->alpha_final = al;
    res->cut_after = cut; res->wA_after = wA; res->wB_after = wB;
    res->status = FRO_OK;
    free(trial);
    return FRO_OK;
}

int32_t fro_refine_pair(int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt,
                        const int32_t *vwgt, int32_t *part, int32_t k, int32_t a, int32_t b, double eps,
                        double alpha, const fro_options *opt, fro_pair_result *res) {
    int32_t st = fro_validate(n, xadj, adjncy, adjwgt, vwgt, part, k);
    if (st == FRO_OK) st = check_pair_args(k, a, b, eps, alpha, opt);
    if (st != FRO_OK) { if (res) { memset(res, 0, sizeof(*res)); res->status = st; } return st; }
    int64_t W = fro_total_weight(n, vwgt);
    int64_t Lmax = fro_lmax(W, fro_max_weight(n, vwgt), k, eps);
    return refine_pair_core(n, xadj, adjncy, adjwgt, vwgt, part, k, a, b, eps, alpha, opt, W, Lmax, res);
}

/* --------------------------------------------- rounds of block pairs ------ */

int32_t fro_rounds(int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *part, int32_t k,
                   int32_t cap, int32_t *pair_a, int32_t *pair_b, int32_t *pair_round, int32_t *nrounds) {
    /* quotient graph: an edge wherever two blocks are adjacent */
    int8_t *adj = XALLOC(int8_t, (int64_t)k * k);
    for (int32_t v = 0; v < n; ++v)
        for (int32_t j = xadj[v]; j < xadj[v + 1]; ++j) {
            int32_t x = part[v], y = part[adjncy[j]];
            if (x != y) adj[(int64_t)x * k + y] = 1;
        }
    int32_t ncol = 2 * k;
    int8_t *used = XALLOC(int8_t, (int64_t)k * ncol);
    int32_t np = 0, nr = 0;
    for (int32_t a = 0; a < k; ++a)
        for (int32_t b = a + 1; b < k; ++b) {
            if (!adj[(int64_t)a * k + b]) continue;
            int32_t c = 0;
            while (used[(int64_t)a * ncol + c] || used[(int64_t)b * ncol + c]) ++c;
            used[(int64_t)a * ncol + c] = used[(int64_t)b * ncol + c] = 1;
            if (np < cap) { pair_a[np] = a; pair_b[np] = b; pair_round[np] = c; }
            ++np;
            if (c + 1 > nr) nr = c + 1;
        }
    free(adj); free(used);
    if (nrounds) *nrounds = nr;
    return np;
}

int32_t fro_refine_batch(int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt,
                         const int32_t *vwgt, int32_t *part, int32_t k, double eps, double alpha,
                         const fro_options *opt, int32_t cap, fro_pair_result *res, int32_t *npairs,
                         int32_t *nrounds) {
    int32_t st = fro_validate(n, xadj, adjncy, adjwgt, vwgt, part, k);
    if (st == FRO_OK && (!(eps > 0.0) || !(alpha >= 1.0) || bad_fm(opt) || bad_mt(opt))) st = FRO_ERR_INVALID_ARG;
    if (st != FRO_OK) return st;
    int64_t W = fro_total_weight(n, vwgt);
    int64_t Lmax = fro_lmax(W, fro_max_weight(n, vwgt), k, eps);
    int32_t maxp = k * (k - 1) / 2;
    int32_t *pa = XALLOC(int32_t, maxp), *pb = XALLOC(int32_t, maxp), *pr = XALLOC(int32_t, maxp);
    int32_t nr = 0;
    int32_t np = fro_rounds(n, xadj, adjncy, part, k, maxp, pa, pb, pr, &nr);
    int32_t out = 0;
    for (int32_t r = 0; r < nr; ++r)
        for (int32_t i = 0; i < np; ++i) {
            if (pr[i] != r) continue;
            fro_pair_result tmp;
            refine_pair_core(n, xadj, adjncy, adjwgt, vwgt, part, k, pa[i], pb[i], eps, alpha, opt, W, Lmax, &tmp);
            tmp.round = r;
            if (out < cap) res[out] = tmp;
            ++out;
        }
    free(pa); free(pb); free(pr);
    if (npairs) *npairs = np;
    if (nrounds) *nrounds = nr;
    return FRO_OK;
}

int32_t fro_refine_batch_sample(int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt,
                                const int32_t *vwgt, int32_t *part, int32_t k, double eps, double alpha,
                                const fro_options *opt, int32_t max_pairs, int32_t *done) {
    int32_t st = fro_validate(n, xadj, adjncy, adjwgt, vwgt, part, k);
    if (st == FRO_OK && (!(eps > 0.0) || !(alpha >= 1.0) || bad_fm(opt) || bad_mt(opt))) st = FRO_ERR_INVALID_ARG;
    if (st != FRO_OK) return st;
    int64_t W = fro_total_weight(n, vwgt);
    int64_t Lmax = fro_lmax(W, fro_max_weight(n, vwgt), k, eps);
    int32_t maxp = k * (k - 1) / 2;
    int32_t *pa = XALLOC(int32_t, maxp), *pb = XALLOC(int32_t, maxp), *pr = XALLOC(int32_t, maxp);
    int32_t nr = 0;
    int32_t np = fro_rounds(n, xadj, adjncy, part, k, maxp, pa, pb, pr, &nr);
    int32_t cnt = 0;
    for (int32_t r = 0; r < nr; ++r)
        for (int32_t i = 0; i < np; ++i) {
            if (pr[i] != r || (max_pairs >= 0 && cnt >= max_pairs)) continue;
            fro_pair_result tmp;
            refine_pair_core(n, xadj, adjncy, adjwgt, vwgt, part, k, pa[i], pb[i], eps, alpha, opt, W, Lmax, &tmp);
            ++cnt;
        }
    free(pa); free(pb); free(pr);
    if (done) *done = cnt;
    return FRO_OK;
}

/* ---------------------- k-way local search (2.2) and multi-try FM (4.2) ---- */

/* Section 2.2 (k-way local search): a single priority queue P over the vertices
 * of a start set S, keyed by the max gain g(v) = max_P g_P(v) over the blocks P
 * that v is adjacent to (g_P(v) = omega(v, P) - omega(v, own block)); the search
 * takes the vertex of highest gain again and again and moves it to its best block
 * unless that block would exceed L_max; each vertex moves at most once; it stops
 * when P is empty or when the KaSPar rule finds a further improvement unlikely,
 * and rolls back to the lowest cut it saw.  Section 4.2 (multi-try FM) starts such
 * searches from single boundary vertices of a block pair.  Readings (also in
 * fro.h) are given where each is used. */

/* KaSPar stopping rule (Osipov & Sanders, as adopted in Section 2.2): over the p
 * moves since the cut last reached a new minimum, with mean mu and population
 * variance sigma^2 of their gains, stop once p mu^2 > alpha sigma^2 + beta.  Each
 * operation is one rounded double operation, in this order (no contraction). */
static int kaspar_stop(int32_t p, int64_t S1, int64_t S2, int32_t alpha, double beta) {
    const double pd = (double)p;
    const double mu = (double)S1 / pd;
    const double var = (double)S2 / pd - mu * mu;
    const double lhs = (pd * mu) * mu;
    const double rhs = (double)alpha * var + beta;
    return lhs > rhs;
}

int32_t fro_kaspar_stop(int32_t p, int64_t S1, int64_t S2, int32_t alpha, double beta) {
    return p > 0 ? kaspar_stop(p, S1, S2, alpha, beta) : 0;
}

typedef struct {
    fm_heap q;          /* keys (gain, stamp, v), larger first */
    int32_t *tgt;       /* [n] target block of the vertex's current key */
    int8_t *moved;      /* [n] moved by the current search */
    int64_t *acc;       /* [k] connection weights of the vertex being keyed (zero between uses) */
    int32_t *blk;       /* [k] blocks with acc != 0 */
    int32_t *lv, *lfrom, *lto;   /* [n] moves of the current search: vertex, source, target */
    int64_t *lg;        /* [n] gain of each move */
} kway_ctx;

static void kway_ctx_init(kway_ctx *C, int32_t n, int32_t k) {
    C->q.h = XALLOC(fm_key, n);
    C->q.n = 0;
    C->q.pos = XALLOC(int32_t, n);
    for (int32_t v = 0; v < n; ++v) C->q.pos[v] = -1;
    C->tgt = XALLOC(int32_t, n);
    C->moved = XALLOC(int8_t, n);
    C->acc = XALLOC(int64_t, k);
    C->blk = XALLOC(int32_t, k);
    C->lv = XALLOC(int32_t, n);
    C->lfrom = XALLOC(int32_t, n);
    C->lto = XALLOC(int32_t, n);
    C->lg = XALLOC(int64_t, n);
}

static void kway_ctx_free(kway_ctx *C) {
    free(C->q.h); free(C->q.pos); free(C->tgt); free(C->moved); free(C->acc); free(C->blk);
    free(C->lv); free(C->lfrom); free(C->lto); free(C->lg);
}

/* Max gain of u and its target block.  Target: the adjacent block other than u's
 * own with the largest connection weight; equal weights go to the smaller
 * splitmix64(tseed ^ u << 32 ^ P), then to the smaller P (the random tie).
 * Returns 0 when u has no neighbour outside its block (not a boundary vertex). */
static int kway_gain(const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt, const int32_t *part,
                     int32_t u, uint64_t tseed, kway_ctx *C, int64_t *gain, int32_t *to) {
    int32_t nb = 0;
    int64_t own = 0;
    for (int32_t j = xadj[u]; j < xadj[u + 1]; ++j) {
        const int32_t P = part[adjncy[j]];
        if (P == part[u]) { own += adjwgt[j]; continue; }
        if (C->acc[P] == 0) C->blk[nb++] = P;
        C->acc[P] += adjwgt[j];
    }
    if (nb == 0) return 0;
    int32_t best = -1;
    int64_t bw = 0;
    uint64_t bh = 0;
    for (int32_t i = 0; i < nb; ++i) {
        const int32_t P = C->blk[i];
        const int64_t w = C->acc[P];
        const uint64_t h = fro_splitmix64(tseed ^ ((uint64_t)(uint32_t)u << 32) ^ (uint64_t)(uint32_t)P);
        if (best < 0 || w > bw || (w == bw && (h < bh || (h == bh && P < best)))) { best = P; bw = w; bh = h; }
        C->acc[P] = 0;
    }
    *gain = bw - own;
    *to = best;
    return 1;
}

static int kway_boundary(const int32_t *xadj, const int32_t *adjncy, const int32_t *part, int32_t u) {
    for (int32_t j = xadj[u]; j < xadj[u + 1]; ++j)
        if (part[adjncy[j]] != part[u]) return 1;
    return 0;
}

/* One k-way search from the start set init[0..ninit) (in that order).  Readings:
 *   key      (gain, stamp), larger first; a stamp is taken per insertion or key
 *            change, in the order they happen: the start set in its order, then
 *            after each move the moved vertex's neighbours in CSR order
 *   balance  v moves to its target P only if c(P) + c(v) <= L_max; otherwise it
 *            leaves the queue unmoved (a later move of a neighbour keys it again)
 *   update   after a move every unmoved neighbour the search may touch is keyed
 *            again if it is a boundary vertex (queued if it was not) and leaves the
 *            queue if it is not
 *   stop     the KaSPar rule after every move that does not reach a new minimum
 *            cut (p, S1, S2 restart at each new minimum), or an empty queue
 *   rollback to the first prefix with the lowest cut (the empty prefix included)
 *   touched  (multi-try) touched[v] = id of the search of the current pass that
 *            queued v, 0 if none; a vertex queued by another search is neither
 *            queued nor moved by this one.  touched = NULL: no such restriction. */
static void kway_run(kway_ctx *C, const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt,
                     const int32_t *vwgt, int32_t *part, int64_t *blockw, int64_t Lmax, const int32_t *init,
                     int32_t ninit, int32_t *touched, int32_t id, int32_t alpha, double beta, uint64_t tseed,
                     fro_kway_result *out) {
    uint64_t stamp = 0;
    for (int32_t i = 0; i < ninit; ++i) {
        const int32_t v = init[i];
        if (C->q.pos[v] >= 0 || (touched && touched[v] != 0 && touched[v] != id)) continue;
        int64_t g;
        int32_t to;
        if (!kway_gain(xadj, adjncy, adjwgt, part, v, tseed, C, &g, &to)) continue;
        fm_key key = { g, stamp++, v };
        C->tgt[v] = to;
        fm_set(&C->q, key);
        if (touched) touched[v] = id;
    }
    int64_t delta = 0, best = 0, S1 = 0, S2 = 0;
    int32_t nm = 0, best_len = 0, p = 0, stop = 0;
    while (C->q.n > 0) {
        const fm_key top = C->q.h[0];
        const int32_t v = top.v, to = C->tgt[v], from = part[v];
        fm_remove(&C->q, v);
        if (blockw[to] + vwgt[v] > Lmax) continue;   /* would overload the target: not moved */
        part[v] = to;
        blockw[from] -= vwgt[v];
        blockw[to] += vwgt[v];
        C->moved[v] = 1;
        C->lv[nm] = v; C->lfrom[nm] = from; C->lto[nm] = to; C->lg[nm] = top.gain;
        ++nm;
        delta -= top.gain;
        for (int32_t j = xadj[v]; j < xadj[v + 1]; ++j) {
            const int32_t u = adjncy[j];
            if (C->moved[u] || (touched && touched[u] != 0 && touched[u] != id)) continue;
            int64_t g;
            int32_t t2;
            if (kway_gain(xadj, adjncy, adjwgt, part, u, tseed, C, &g, &t2)) {
                fm_key key = { g, stamp++, u };
                C->tgt[u] = t2;
                fm_set(&C->q, key);
                if (touched) touched[u] = id;
            } else {
                fm_remove(&C->q, u);
            }
        }
        if (delta < best) {
            best = delta; best_len = nm; p = 0; S1 = 0; S2 = 0;
        } else {
            ++p;
            S1 += top.gain;
            S2 += top.gain * top.gain;
            if (kaspar_stop(p, S1, S2, alpha, beta)) { stop = 1; break; }
        }
    }
    for (int32_t i = nm - 1; i >= best_len; --i) {   /* roll back */
        const int32_t v = C->lv[i], to = part[v];
        part[v] = C->lfrom[i];
        blockw[to] -= vwgt[v];
        blockw[C->lfrom[i]] += vwgt[v];
    }
    for (int32_t i = 0; i < nm; ++i) C->moved[C->lv[i]] = 0;
    for (int32_t i = 0; i < C->q.n; ++i) C->q.pos[C->q.h[i].v] = -1;
    C->q.n = 0;
    out->gain = -best;
    out->tried = nm;
    out->kept = best_len;
    out->stop = stop;
}

int32_t fro_kway_search(int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt,
                        const int32_t *vwgt, int32_t *part, int32_t k, int64_t *blockw, int64_t Lmax,
                        const int32_t *init, int32_t ninit, int32_t *touched, int32_t id, int32_t alpha,
                        double beta, uint64_t tseed, fro_kway_result *out, int32_t *log_v, int32_t *log_to,
                        int64_t *log_gain, int32_t log_cap) {
    memset(out, 0, sizeof(*out));
    if (n < 1 || k < 2 || ninit < 0 || alpha < 0 || (touched && id < 1)) return FRO_ERR_INVALID_ARG;
    for (int32_t i = 0; i < ninit; ++i)
        if (init[i] < 0 || init[i] >= n) return FRO_ERR_INVALID_ARG;
    kway_ctx C;
    kway_ctx_init(&C, n, k);
    kway_run(&C, xadj, adjncy, adjwgt, vwgt, part, blockw, Lmax, init, ninit, touched, id, alpha, beta, tseed, out);
    for (int32_t i = 0; i < out->tried && i < log_cap; ++i) {
        if (log_v) log_v[i] = C.lv[i];
        if (log_to) log_to[i] = C.lto[i];
        if (log_gain) log_gain[i] = C.lg[i];
    }
    kway_ctx_free(&C);
    return FRO_OK;
}

/* Seeds of the multi-try pass: the todo list of pair (a, b) is ordered by
 * splitmix64(fro_mt_seed(seed, a, b) ^ v); target ties use splitmix64(~seed). */
uint64_t fro_mt_seed(uint64_t seed, int32_t a, int32_t b) { return fro_splitmix64(fro_fm_seed(seed, a, b) + 1); }

typedef struct { uint64_t key; int32_t v; } todo_item;

static int cmp_todo(const void *pa, const void *pb) {
    const todo_item *x = (const todo_item *)pa, *y = (const todo_item *)pb;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->v > y->v) - (x->v < y->v);
}

/* Section 4.2 (multi-try FM) for the pairs (pa[i], pb[i]), i < np, of one matching,
 * run after their pairwise improvements (Section 4.3).  Readings (also in fro.h):
 *   todo     pair (a, b): its vertices with a neighbour in the other block, as the
 *            pass starts, in a random order (ascending splitmix64 keys); the pairs'
 *            lists are visited round-robin: entry 0 of every pair in pair order,
 *            then entry 1, and so on (the pairs' improvements ran side by side)
 *   search   a todo vertex starts a k-way search if no search of this pass has
 *            queued it and it still has a neighbour in another block; the start
 *            set is that vertex, then its neighbours (CSR order) that are boundary
 *            vertices no search of the pass has queued
 *   touched  a vertex queued by one search of the pass is never queued by another
 *   beta     ln n, the natural logarithm of the graph's vertex count
 * changed[x] (k entries, may be NULL) is set to 1 for the source and target block
 * of every kept move. */
int32_t fro_multitry(int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt,
                     const int32_t *vwgt, int32_t *part, int32_t k, int64_t Lmax, int32_t np, const int32_t *pa,
                     const int32_t *pb, int32_t alpha, uint64_t seed, fro_mt_result *out, int8_t *changed) {
    memset(out, 0, sizeof(*out));
    if (np < 0 || alpha < 0) return FRO_ERR_INVALID_ARG;
    for (int32_t i = 0; i < np; ++i)
        if (pa[i] < 0 || pb[i] < 0 || pa[i] >= k || pb[i] >= k || pa[i] == pb[i]) return FRO_ERR_INVALID_ARG;
    const double beta = log((double)n);
    const uint64_t tseed = fro_splitmix64(~seed);
    int64_t *blockw = XALLOC(int64_t, k);
    for (int32_t v = 0; v < n; ++v) blockw[part[v]] += vwgt[v];
    /* the todo lists, fixed as the pass starts */
    todo_item **todo = XALLOC(todo_item *, np);
    int32_t *len = XALLOC(int32_t, np), maxlen = 0;
    for (int32_t i = 0; i < np; ++i) {
        const int32_t a = pa[i], b = pb[i];
        const uint64_t ms = fro_mt_seed(seed, a, b);
        todo[i] = XALLOC(todo_item, n);
        for (int32_t v = 0; v < n; ++v) {
            if (part[v] != a && part[v] != b) continue;
            const int32_t other = part[v] == a ? b : a;
            for (int32_t j = xadj[v]; j < xadj[v + 1]; ++j)
                if (part[adjncy[j]] == other) {
                    todo[i][len[i]].key = fro_splitmix64(ms ^ (uint64_t)(uint32_t)v);
                    todo[i][len[i]].v = v;
                    ++len[i];
                    break;
                }
        }
        qsort(todo[i], (size_t)len[i], sizeof(todo_item), cmp_todo);
        if (len[i] > maxlen) maxlen = len[i];
    }
    kway_ctx C;
    kway_ctx_init(&C, n, k);
    int32_t *touched = XALLOC(int32_t, n);
    int32_t *init = XALLOC(int32_t, n);
    int32_t id = 0;
    for (int32_t j = 0; j < maxlen; ++j)
        for (int32_t i = 0; i < np; ++i) {
            if (j >= len[i]) continue;
            const int32_t v = todo[i][j].v;
            if (touched[v] || !kway_boundary(xadj, adjncy, part, v)) continue;
            int32_t ni = 0;
            init[ni++] = v;
            for (int32_t q = xadj[v]; q < xadj[v + 1]; ++q) {
                const int32_t u = adjncy[q];
                if (!touched[u] && kway_boundary(xadj, adjncy, part, u)) init[ni++] = u;
            }
            fro_kway_result r;
            kway_run(&C, xadj, adjncy, adjwgt, vwgt, part, blockw, Lmax, init, ni, touched, ++id, alpha, beta,
                     tseed, &r);
            out->searches += 1;
            out->gain += r.gain;
            out->tried += r.tried;
            out->kept += r.kept;
            if (changed)
                for (int32_t q = 0; q < r.kept; ++q) changed[C.lfrom[q]] = changed[C.lto[q]] = 1;
        }
    for (int32_t i = 0; i < np; ++i) free(todo[i]);
    free(todo); free(len); free(touched); free(init); free(blockw);
    kway_ctx_free(&C);
    return FRO_OK;
}

/* Section 2.2 with the setup of Section 6 ("Configuring the Algorithm"): rounds of
 * one k-way search each, started from the complete partition boundary (init_mode 0)
 * or from the corner vertices only (init_mode 1: vertices whose neighbourhood,
 * with themselves, meets at least three blocks), in a random order (ascending
 * splitmix64(splitmix64(seed ^ r) ^ v) in round r); the rounds stop after the first
 * round without an improvement, or after max_rounds.  Sums of all rounds in out;
 * *rounds = rounds run. */
int32_t fro_kway_global(int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt,
                        const int32_t *vwgt, int32_t *part, int32_t k, double eps, int32_t init_mode,
                        int32_t alpha, int32_t max_rounds, uint64_t seed, fro_kway_result *out, int32_t *rounds) {
    memset(out, 0, sizeof(*out));
    if (rounds) *rounds = 0;
    int32_t st = fro_validate(n, xadj, adjncy, adjwgt, vwgt, part, k);
    if (st == FRO_OK && (!(eps > 0.0) || alpha < 0 || max_rounds < 1 || (init_mode != 0 && init_mode != 1)))
        st = FRO_ERR_INVALID_ARG;
    if (st != FRO_OK) return st;
    const int64_t Lmax = fro_lmax(fro_total_weight(n, vwgt), fro_max_weight(n, vwgt), k, eps);
    const double beta = log((double)n);
    const uint64_t tseed = fro_splitmix64(~seed);
    int64_t *blockw = XALLOC(int64_t, k);
    for (int32_t v = 0; v < n; ++v) blockw[part[v]] += vwgt[v];
    todo_item *S = XALLOC(todo_item, n);
    int32_t *init = XALLOC(int32_t, n);
    int8_t *seen = XALLOC(int8_t, k);
    kway_ctx C;
    kway_ctx_init(&C, n, k);
    int32_t r = 0;
    for (; r < max_rounds; ++r) {
        const uint64_t rs = fro_splitmix64(seed ^ (uint64_t)(uint32_t)r);
        int32_t ns = 0;
        for (int32_t v = 0; v < n; ++v) {
            int32_t nb = 0;   /* blocks other than v's own around v */
            for (int32_t j = xadj[v]; j < xadj[v + 1]; ++j) {
                const int32_t P = part[adjncy[j]];
                if (P != part[v] && !seen[P]) { seen[P] = 1; ++nb; }
            }
            for (int32_t j = xadj[v]; j < xadj[v + 1]; ++j) seen[part[adjncy[j]]] = 0;
            if (nb >= (init_mode == 1 ? 2 : 1)) { S[ns].key = fro_splitmix64(rs ^ (uint64_t)(uint32_t)v); S[ns].v = v; ++ns; }
        }
        qsort(S, (size_t)ns, sizeof(todo_item), cmp_todo);
        for (int32_t i = 0; i < ns; ++i) init[i] = S[i].v;
        fro_kway_result rr;
        kway_run(&C, xadj, adjncy, adjwgt, vwgt, part, blockw, Lmax, init, ns, NULL, 0, alpha, beta, tseed, &rr);
        out->gain += rr.gain;
        out->tried += rr.tried;
        out->kept += rr.kept;
        out->stop = rr.stop;
        if (rr.gain <= 0) { ++r; break; }
    }
    if (rounds) *rounds = r;
    free(blockw); free(S); free(init); free(seen);
    kway_ctx_free(&C);
    return FRO_OK;
}

/* --------------------------------------- active block scheduling --------- */

/* Section 4.3 (scheduling quotient graph refinement) and the appendix pseudocode
 * of active block scheduling, with the pairwise improvement restricted to the flow
 * refinement of Section 4.1, preceded by the two-way FM search when fm_permille
 * is set; with mt_alpha set, a multi-try FM pass (Section 4.2) started from the
 * boundaries of a matching's pairs follows the pairwise improvements of that
 * matching, and every block a kept multi-try move left or entered becomes active.  Every block starts active.  An outer round
 * takes the quotient edges (a, b) of the current partition with a or b active,
 * marks every block inactive, and refines those pairs; a pair whose refinement
 * changed the partition marks a and b active again.  The outer rounds end when no
 * block is active, or after max_outer of them.  Inside an outer round the pairs
 * are coloured into matchings exactly as in fro_rounds (lexicographic order,
 * smallest colour free at both ends) and refined matching by matching. */
int32_t fro_refine_active(int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt,
                          const int32_t *vwgt, int32_t *part, int32_t k, double eps, double alpha,
                          const fro_options *opt, int32_t max_outer, int32_t cap, fro_pair_result *res,
                          int32_t *npairs, int32_t *nouter, fro_mt_result *mt) {
    int32_t st = fro_validate(n, xadj, adjncy, adjwgt, vwgt, part, k);
    if (st == FRO_OK && (!(eps > 0.0) || !(alpha >= 1.0) || max_outer < 1 || bad_fm(opt) || (opt && opt->mt_alpha < 0)))
        st = FRO_ERR_INVALID_ARG;
    if (st != FRO_OK) return st;
    int64_t W = fro_total_weight(n, vwgt);
    int64_t Lmax = fro_lmax(W, fro_max_weight(n, vwgt), k, eps);
    int8_t *active = XALLOC(int8_t, k);
    int8_t *adj = XALLOC(int8_t, (int64_t)k * k);
    int32_t ncol = 2 * k;
    int8_t *used = XALLOC(int8_t, (int64_t)k * ncol);
    int32_t maxp = k * (k - 1) / 2;
    int32_t *pa = XALLOC(int32_t, maxp), *pb = XALLOC(int32_t, maxp), *pr = XALLOC(int32_t, maxp);
    for (int32_t x = 0; x < k; ++x) active[x] = 1;
    const int32_t mt_alpha = opt ? opt->mt_alpha : 0;
    const uint64_t seed = opt ? opt->seed : 0;
    int32_t *ma = XALLOC(int32_t, maxp), *mb_ = XALLOC(int32_t, maxp);
    int8_t *changed = XALLOC(int8_t, k);
    if (mt) memset(mt, 0, sizeof(*mt));
    int32_t out = 0, outer = 0, round_base = 0;
    for (; outer < max_outer; ++outer) {
        int32_t any = 0;
        for (int32_t x = 0; x < k; ++x) any |= active[x];
        if (!any) break;
        /* quotient graph of the current partition */
        memset(adj, 0, (size_t)k * k);
        for (int32_t v = 0; v < n; ++v)
            for (int32_t j = xadj[v]; j < xadj[v + 1]; ++j) {
                int32_t x = part[v], y = part[adjncy[j]];
                if (x != y) adj[(int64_t)x * k + y] = 1;
            }
        /* the edges with an active end, coloured into matchings */
        memset(used, 0, (size_t)k * ncol);
        int32_t np = 0, nr = 0;
        for (int32_t a = 0; a < k; ++a)
            for (int32_t b = a + 1; b < k; ++b) {
                if (!adj[(int64_t)a * k + b] || !(active[a] || active[b])) continue;
                int32_t c = 0;
                while (used[(int64_t)a * ncol + c] || used[(int64_t)b * ncol + c]) ++c;
                used[(int64_t)a * ncol + c] = used[(int64_t)b * ncol + c] = 1;
                pa[np] = a; pb[np] = b; pr[np] = c;
                ++np;
                if (c + 1 > nr) nr = c + 1;
            }
        for (int32_t x = 0; x < k; ++x) active[x] = 0;
        for (int32_t r = 0; r < nr; ++r) {
            for (int32_t i = 0; i < np; ++i) {
                if (pr[i] != r) continue;
                fro_pair_result tmp;
                refine_pair_core(n, xadj, adjncy, adjwgt, vwgt, part, k, pa[i], pb[i], eps, alpha, opt, W, Lmax,
                                 &tmp);
                tmp.round = round_base + r;
                if (tmp.accepted || tmp.fm_moves > 0) active[pa[i]] = active[pb[i]] = 1;   /* partition changed */
                if (out < cap) res[out] = tmp;
                ++out;
            }
            if (mt_alpha > 0) {
                /* after the pairwise improvements of the matching: one multi-try pass
                 * started from the boundaries of its pairs; every block a kept move
                 * left or entered becomes active */
                int32_t nm = 0;
                for (int32_t i = 0; i < np; ++i)
                    if (pr[i] == r) { ma[nm] = pa[i]; mb_[nm] = pb[i]; ++nm; }
                memset(changed, 0, (size_t)k);
                fro_mt_result m;
                fro_multitry(n, xadj, adjncy, adjwgt, vwgt, part, k, Lmax, nm, ma, mb_, mt_alpha, seed, &m, changed);
                for (int32_t x = 0; x < k; ++x) if (changed[x]) active[x] = 1;
                if (mt) {
                    mt->gain += m.gain; mt->searches += m.searches; mt->tried += m.tried; mt->kept += m.kept;
                }
            }
        }
        round_base += nr;
    }
    free(active); free(adj); free(used); free(pa); free(pb); free(pr); free(ma); free(mb_); free(changed);
    if (npairs) *npairs = out;
    if (nouter) *nouter = outer;
    return FRO_OK;
}

/* ------------------------------------- pair-parallel sweep (CPU baseline) */

/* The pairs of one round form a matching of the quotient graph, so they touch
 * disjoint blocks: the refinement of (a, b) reads only which vertices lie in a
 * and b (corridor, pair cut, block weights) and moves vertices between a and b
 * only.  Running them on several threads, each on its own copy of the
 * partition as it stood when the round began, and taking from each copy the
 * vertices that were in its two blocks, gives exactly the sequential sweep.
 * This is the pair-parallel CPU baseline; the per-pair arithmetic is the
 * sequential oracle's (refine_pair_core). */

typedef struct {
    int32_t n;
    const int32_t *xadj, *adjncy, *adjwgt, *vwgt;
    int32_t k;
    double eps, alpha;
    const fro_options *opt;
    int64_t W, Lmax;
    const int32_t *snap;     /* partition at the start of the round */
    int32_t *part;           /* merged result */
    const int32_t *idx;      /* pair indices of this round */
    const int32_t *pa, *pb;
    int32_t cnt, next, round;
    fro_pair_result *tmp;    /* one per pair of the round */
    pthread_mutex_t mu;
} mt_round;

static void *mt_worker(void *arg) {
    mt_round *R = (mt_round *)arg;
    int32_t *buf = XALLOC(int32_t, R->n);
    for (;;) {
        pthread_mutex_lock(&R->mu);
        int32_t i = R->next++;
        pthread_mutex_unlock(&R->mu);
        if (i >= R->cnt) break;
        int32_t a = R->pa[R->idx[i]], b = R->pb[R->idx[i]];
        memcpy(buf, R->snap, sizeof(int32_t) * (size_t)R->n);
        refine_pair_core(R->n, R->xadj, R->adjncy, R->adjwgt, R->vwgt, buf, R->k, a, b, R->eps, R->alpha, R->opt,
                         R->W, R->Lmax, &R->tmp[i]);
        R->tmp[i].round = R->round;
        for (int32_t v = 0; v < R->n; ++v)
            if (R->snap[v] == a || R->snap[v] == b) R->part[v] = buf[v];
    }
    free(buf);
    return NULL;
}

int32_t fro_refine_batch_mt(int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt,
                            const int32_t *vwgt, int32_t *part, int32_t k, double eps, double alpha,
                            const fro_options *opt, int32_t nthreads, int32_t max_rounds, int32_t cap,
                            fro_pair_result *res, int32_t *npairs, int32_t *nrounds, int32_t *done) {
    int32_t st = fro_validate(n, xadj, adjncy, adjwgt, vwgt, part, k);
    if (st == FRO_OK && (!(eps > 0.0) || !(alpha >= 1.0) || nthreads < 1 || bad_fm(opt) || bad_mt(opt))) st = FRO_ERR_INVALID_ARG;
    if (st != FRO_OK) return st;
    int64_t W = fro_total_weight(n, vwgt);
    int64_t Lmax = fro_lmax(W, fro_max_weight(n, vwgt), k, eps);
    int32_t maxp = k * (k - 1) / 2;
    int32_t *pa = XALLOC(int32_t, maxp), *pb = XALLOC(int32_t, maxp), *pr = XALLOC(int32_t, maxp);
    int32_t *idx = XALLOC(int32_t, maxp);
    fro_pair_result *tmp = XALLOC(fro_pair_result, maxp);
    int32_t *snap = XALLOC(int32_t, n);
    pthread_t *th = XALLOC(pthread_t, nthreads);
    int32_t nr = 0;
    int32_t np = fro_rounds(n, xadj, adjncy, part, k, maxp, pa, pb, pr, &nr);
    int32_t out = 0, last = max_rounds >= 0 && max_rounds < nr ? max_rounds : nr;
    for (int32_t r = 0; r < last; ++r) {
        int32_t cnt = 0;
        for (int32_t i = 0; i < np; ++i)
            if (pr[i] == r) idx[cnt++] = i;
        memcpy(snap, part, sizeof(int32_t) * (size_t)n);
        mt_round R = {n, xadj, adjncy, adjwgt, vwgt, k, eps, alpha, opt, W, Lmax, snap, part, idx, pa, pb,
                      cnt, 0, r, tmp};
        pthread_mutex_init(&R.mu, NULL);
        int32_t nt = nthreads < cnt ? nthreads : cnt, started = 0;
        for (int32_t t = 0; t < nt; ++t)
            if (pthread_create(&th[t], NULL, mt_worker, &R) == 0) ++started;
        if (started == 0) mt_worker(&R);   /* no thread could start: run the round here */
        for (int32_t t = 0; t < started; ++t) pthread_join(th[t], NULL);
        pthread_mutex_destroy(&R.mu);
        for (int32_t i = 0; i < cnt; ++i) {
            if (out < cap) res[out] = tmp[i];
            ++out;
        }
    }
    free(pa); free(pb); free(pr); free(idx); free(tmp); free(snap); free(th);
    if (npairs) *npairs = np;
    if (nrounds) *nrounds = nr;
    if (done) *done = out;
    return FRO_OK;
}

/* ------------------------------------- multilevel V-cycle (2.1, 2.2, 5) ---- */

/* Section 2.1 defines matching, contraction (c(x) = c(u) + c(v), parallel edges
 * merged with summed weights) and the three phases; Section 2.2 rates edges with
 * expansion*2(u, v) = omega(u, v)^2 / (c(u) c(v)), matches to maximise the rated
 * weight and keeps nodes heavier than 1.5 n / (20 k) out of contractions; Section
 * 5 (global search) reuses a given partition: edges between two blocks are never
 * matched, so the partition is the coarsest graph's initial partition and every
 * level refines it.  Readings (also in fro.h):
 *   rating   expansion*2 with c replaced by max(c, 1) (zero vertex weights are
 *            allowed here); compared exactly as omega1^2 c2(u) c2(v) against
 *            omega2^2 c1(u) c1(v) in 128-bit integers
 *   order    edges by rating, larger first; equal ratings by the larger
 *            splitmix64(seed_l ^ min(u, v) << 32 ^ max(u, v)) (random tie
 *            breaking), then by the smaller (min, max) pair; seed_l =
 *            splitmix64(seed ^ level)
 *   matching the greedy matching in that order (an edge joins if both ends are
 *            still free) over the edges inside one block whose ends both weigh at
 *            most 1.5 W / (20 k) (W = c(V) of the input, n in the paper's unit-weight
 *            setting), i.e. 40 k c(v) <= 3 W.  GPA is replaced by greedy matching:
 *            both are 1/2-approximations of the maximum rated matching, and greedy
 *            has an exact parallel form (locally dominant edges)
 *   ids      the coarse vertex of a matched pair or a single vertex is numbered in
 *            the order of its smaller fine id; coarse rows list their neighbours
 *            in increasing coarse id, parallel edges merged, the matched edge gone
 *   levels   contract while the graph has more than max(60 k, n / (60 k)) vertices,
 *            the level's matching holds at least n_level / 20 pairs (contraction
 *            that shrinks a level by less than 5 % has stalled: the weight bound
 *            keeps the heavy vertices single), and fewer than max_levels levels
 *            exist
 *   refine   on the coarsest level, then after each projection (part(v) =
 *            part(coarse vertex of v)), one sweep of fro_refine_batch, or
 *            fro_refine_active when active_outer > 0, with L_max of that level's
 *            graph */

typedef struct {
    int32_t n, nnz;
    int32_t *xadj, *adjncy, *adjwgt, *vwgt;
} ml_graph;

static void ml_free(ml_graph *g) {
    free(g->xadj); free(g->adjncy); free(g->adjwgt); free(g->vwgt);
}

typedef struct { int32_t u, v, w; uint64_t h; int64_t cu, cv; } ml_edge;

/* 1 if edge x comes before edge y in the matching order */
static int ml_before(const ml_edge *x, const ml_edge *y) {
    const unsigned __int128 lx = (unsigned __int128)((uint64_t)x->w * (uint64_t)x->w) * (uint64_t)y->cu * (uint64_t)y->cv;
    const unsigned __int128 ly = (unsigned __int128)((uint64_t)y->w * (uint64_t)y->w) * (uint64_t)x->cu * (uint64_t)x->cv;
    if (lx != ly) return lx > ly;
    if (x->h != y->h) return x->h > y->h;
    if (x->u != y->u) return x->u < y->u;
    return x->v < y->v;
}

static int ml_cmp(const void *a, const void *b) {
    const ml_edge *x = (const ml_edge *)a, *y = (const ml_edge *)b;
    if (ml_before(x, y)) return -1;
    if (ml_before(y, x)) return 1;
    return 0;
}

/* Greedy matching of one level (mate[v] = partner or -1). */
static int32_t ml_match(const int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt,
                        const int32_t *vwgt, const int32_t *part, int32_t k, int64_t W, uint64_t seed_l,
                        int32_t *mate) {
    int64_t m = 0;
    for (int32_t v = 0; v < n; ++v) mate[v] = -1;
    for (int32_t v = 0; v < n; ++v)
        for (int32_t j = xadj[v]; j < xadj[v + 1]; ++j) if (v < adjncy[j]) ++m;
    ml_edge *E = XALLOC(ml_edge, m);
    int64_t ne = 0;
    for (int32_t v = 0; v < n; ++v)
        for (int32_t j = xadj[v]; j < xadj[v + 1]; ++j) {
            const int32_t u = adjncy[j];
            if (v >= u || part[v] != part[u]) continue;
            if (40LL * k * vwgt[v] > 3 * W || 40LL * k * vwgt[u] > 3 * W) continue;
            ml_edge e;
            e.u = v; e.v = u; e.w = adjwgt[j];
            e.h = fro_splitmix64(seed_l ^ ((uint64_t)(uint32_t)v << 32) ^ (uint64_t)(uint32_t)u);
            e.cu = vwgt[v] > 0 ? vwgt[v] : 1;
            e.cv = vwgt[u] > 0 ? vwgt[u] : 1;
            E[ne++] = e;
        }
    qsort(E, (size_t)ne, sizeof(ml_edge), ml_cmp);
    int32_t pairs = 0;
    for (int64_t i = 0; i < ne; ++i)
        if (mate[E[i].u] < 0 && mate[E[i].v] < 0) {
            mate[E[i].u] = E[i].v;
            mate[E[i].v] = E[i].u;
            ++pairs;
        }
    free(E);
    return pairs;
}

static int cmp_pair_i32(const void *a, const void *b) {
    const int32_t *x = (const int32_t *)a, *y = (const int32_t *)b;
    return (x[0] > y[0]) - (x[0] < y[0]);
}

/* Contraction of a matching: coarse graph and cmap[v] = coarse vertex of v. */
static void ml_contract(const ml_graph *g, const int32_t *mate, ml_graph *c, int32_t *cmap) {
    int32_t nc = 0;
    for (int32_t v = 0; v < g->n; ++v)
        if (mate[v] < 0 || v < mate[v]) cmap[v] = nc++;
    for (int32_t v = 0; v < g->n; ++v)
        if (mate[v] >= 0 && v > mate[v]) cmap[v] = cmap[mate[v]];
    int32_t *first = XALLOC(int32_t, nc);   /* smaller member of each coarse vertex */
    for (int32_t v = g->n - 1; v >= 0; --v) first[cmap[v]] = v;
    c->n = nc;
    c->xadj = XALLOC(int32_t, nc + 1);
    c->vwgt = XALLOC(int32_t, nc);
    int64_t *acc = XALLOC(int64_t, nc);
    int32_t *row = XALLOC(int32_t, 2 * (size_t)(g->nnz > 0 ? g->nnz : 1));
    int32_t *adj = XALLOC(int32_t, g->nnz), *wgt = XALLOC(int32_t, g->nnz);
    int32_t cnt = 0;
    for (int32_t x = 0; x < nc; ++x) {
        c->xadj[x] = cnt;
        const int32_t mem[2] = { first[x], mate[first[x]] };
        int32_t nr = 0;
        for (int t = 0; t < 2; ++t) {
            const int32_t v = mem[t];
            if (v < 0) continue;
            c->vwgt[x] += g->vwgt[v];
            for (int32_t j = g->xadj[v]; j < g->xadj[v + 1]; ++j) {
                const int32_t y = cmap[g->adjncy[j]];
                if (y == x) continue;   /* the matched edge */
                if (acc[y] == 0) { row[2 * nr] = y; row[2 * nr + 1] = 0; ++nr; }
                acc[y] += g->adjwgt[j];
            }
        }
        qsort(row, (size_t)nr, 2 * sizeof(int32_t), cmp_pair_i32);
        for (int32_t i = 0; i < nr; ++i) {
            const int32_t y = row[2 * i];
            adj[cnt] = y;
            wgt[cnt] = (int32_t)acc[y];
            acc[y] = 0;
            ++cnt;
        }
    }
    c->xadj[nc] = cnt;
    c->nnz = cnt;
    c->adjncy = adj;
    c->adjwgt = wgt;
    free(first); free(acc); free(row);
}

int32_t fro_match(int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt, const int32_t *vwgt,
                  const int32_t *part, int32_t k, int64_t W, uint64_t seed_l, int32_t *mate) {
    if (n < 1 || k < 1 || W < 0) return -1;
    return ml_match(n, xadj, adjncy, adjwgt, vwgt, part, k, W, seed_l, mate);
}

int32_t fro_contract(int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt,
                     const int32_t *vwgt, const int32_t *mate, int32_t *cmap, int32_t *cn, int32_t *cxadj,
                     int32_t *cadjncy, int32_t *cadjwgt, int32_t *cvwgt) {
    ml_graph g = { n, xadj[n], (int32_t *)xadj, (int32_t *)adjncy, (int32_t *)adjwgt, (int32_t *)vwgt };
    ml_graph c;
    ml_contract(&g, mate, &c, cmap);
    *cn = c.n;
    memcpy(cxadj, c.xadj, sizeof(int32_t) * (size_t)(c.n + 1));
    memcpy(cadjncy, c.adjncy, sizeof(int32_t) * (size_t)c.nnz);
    memcpy(cadjwgt, c.adjwgt, sizeof(int32_t) * (size_t)c.nnz);
    memcpy(cvwgt, c.vwgt, sizeof(int32_t) * (size_t)c.n);
    int32_t nnz = c.nnz;
    ml_free(&c);
    return nnz;
}

int32_t fro_vcycle(int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt,
                   const int32_t *vwgt, int32_t *part, int32_t k, double eps, double alpha, const fro_options *opt,
                   int32_t max_levels, int32_t active_outer, fro_vcycle_result *out) {
    memset(out, 0, sizeof(*out));
    int32_t st = fro_validate(n, xadj, adjncy, adjwgt, vwgt, part, k);
    if (st == FRO_OK && (!(eps > 0.0) || !(alpha >= 1.0) || max_levels < 1 || max_levels > FRO_MAX_LEVELS ||
                         active_outer < 0 || bad_fm(opt) || (opt && opt->mt_alpha < 0) ||
                         (bad_mt(opt) && active_outer == 0)))
        st = FRO_ERR_INVALID_ARG;
    if (st != FRO_OK) return st;
    const uint64_t seed = opt ? opt->seed : 0;
    const int64_t W = fro_total_weight(n, vwgt);
    int64_t thr = 60LL * k;
    if ((int64_t)n / (60LL * k) > thr) thr = (int64_t)n / (60LL * k);
    ml_graph G[FRO_MAX_LEVELS];
    int32_t *cmap[FRO_MAX_LEVELS];
    int32_t *P[FRO_MAX_LEVELS];
    G[0].n = n; G[0].nnz = xadj[n];
    G[0].xadj = (int32_t *)xadj; G[0].adjncy = (int32_t *)adjncy; G[0].adjwgt = (int32_t *)adjwgt;
    G[0].vwgt = (int32_t *)vwgt;
    P[0] = XALLOC(int32_t, n);
    memcpy(P[0], part, sizeof(int32_t) * (size_t)n);
    int32_t L = 1;
    out->cut_before = 0;
    for (int32_t v = 0; v < n; ++v)
        for (int32_t j = xadj[v]; j < xadj[v + 1]; ++j)
            if (v < adjncy[j] && part[v] != part[adjncy[j]]) out->cut_before += adjwgt[j];
    /* contraction */
    while (L < max_levels && G[L - 1].n > thr) {
        const ml_graph *g = &G[L - 1];
        int32_t *mate = XALLOC(int32_t, g->n);
        const int32_t pairs = ml_match(g->n, g->xadj, g->adjncy, g->adjwgt, g->vwgt, P[L - 1], k, W,
                                       fro_splitmix64(seed ^ (uint64_t)(L - 1)), mate);
        if (pairs == 0 || 20LL * pairs < g->n) { free(mate); break; }   /* stalled: under 5 % */
        cmap[L - 1] = XALLOC(int32_t, g->n);
        ml_contract(g, mate, &G[L], cmap[L - 1]);
        P[L] = XALLOC(int32_t, G[L].n);
        for (int32_t v = 0; v < g->n; ++v) P[L][cmap[L - 1][v]] = P[L - 1][v];
        free(mate);
        ++L;
    }
    out->levels = L;
    for (int32_t l = 0; l < L; ++l) out->level_n[l] = G[l].n;
    /* refinement from the coarsest level up */
    const int32_t cap = k * (k - 1) / 2 * (active_outer > 0 ? active_outer : 1);
    fro_pair_result *res = XALLOC(fro_pair_result, cap > 0 ? cap : 1);
    for (int32_t l = L - 1; l >= 0 && st == FRO_OK; --l) {
        if (l < L - 1)
            for (int32_t v = 0; v < G[l].n; ++v) P[l][v] = P[l + 1][cmap[l][v]];
        int32_t np_ = 0, nr_ = 0;
        if (active_outer > 0)
            st = fro_refine_active(G[l].n, G[l].xadj, G[l].adjncy, G[l].adjwgt, G[l].vwgt, P[l], k, eps, alpha, opt,
                                   active_outer, cap, res, &np_, &nr_, NULL);
        else
            st = fro_refine_batch(G[l].n, G[l].xadj, G[l].adjncy, G[l].adjwgt, G[l].vwgt, P[l], k, eps, alpha, opt,
                                  cap, res, &np_, &nr_);
        out->level_pairs[l] = np_;
        int64_t cut = 0;
        for (int32_t v = 0; v < G[l].n; ++v)
            for (int32_t j = G[l].xadj[v]; j < G[l].xadj[v + 1]; ++j)
                if (v < G[l].adjncy[j] && P[l][v] != P[l][G[l].adjncy[j]]) cut += G[l].adjwgt[j];
        out->level_cut[l] = cut;
    }
    if (st == FRO_OK) {
        memcpy(part, P[0], sizeof(int32_t) * (size_t)n);
        out->cut_after = out->level_cut[0];
    }
    for (int32_t l = 0; l < L; ++l) free(P[l]);
    for (int32_t l = 1; l < L; ++l) ml_free(&G[l]);
    for (int32_t l = 0; l + 1 < L; ++l) free(cmap[l]);
    free(res);
    return st;
}

/* W- and F-cycles (Section 5, the global search pseudocode): a cycle on graph G
 * coarsens G, runs a cycle on the coarse graph, projects and refines G; on levels that
 * allow an independent trial it then coarsens G again (with a new seed, respecting the
 * partition it has now), runs a second cycle on that graph, projects and refines G once
 * more.  Readings (also in fro.h):
 *   coarsest a graph that cannot be coarsened (at most max(60 k, n / (60 k)) vertices,
 *            the level cap reached, or a stalled matching as in fro_vcycle) is refined
 *            and ends the recursion; a V-cycle is the cycle without second trials
 *   trials   W-cycle: a second trial on every level l with l % d == 0 (the level split
 *            parameter); F-cycle: also only while fewer than two coarsenings of level-l
 *            graphs have been made in the whole run; a second coarsening that stalls
 *            skips the trial
 *   seeds    the c-th coarsening of a level-l graph in the run (c = 0, 1, ...) uses
 *            seed_l = splitmix64(seed ^ l ^ c << 32) (c = 0 gives fro_vcycle's seeds)
 *   refine   one fro_refine_batch sweep, or fro_refine_active with active_outer rounds */

typedef struct {
    int32_t k, type, d, max_levels, active_outer;
    double eps, alpha;
    const fro_options *opt;
    int64_t W, thr;
    int32_t count[FRO_MAX_LEVELS];   /* coarsenings made per level */
    fro_cycle_result *out;
    int32_t st;
} ml_run;

static void ml_refine(ml_run *R, const ml_graph *g, int32_t *P) {
    if (R->st != FRO_OK) return;
    const int32_t cap = R->k * (R->k - 1) / 2 * (R->active_outer > 0 ? R->active_outer : 1);
    fro_pair_result *res = XALLOC(fro_pair_result, cap > 0 ? cap : 1);
    int32_t a = 0, b = 0;
    if (R->active_outer > 0)
        R->st = fro_refine_active(g->n, g->xadj, g->adjncy, g->adjwgt, g->vwgt, P, R->k, R->eps, R->alpha, R->opt,
                                  R->active_outer, cap, res, &a, &b, NULL);
    else
        R->st = fro_refine_batch(g->n, g->xadj, g->adjncy, g->adjwgt, g->vwgt, P, R->k, R->eps, R->alpha, R->opt,
                                 cap, res, &a, &b);
    R->out->refinements += 1;
    free(res);
}

/* One coarsening of (g, P) at level l; returns 0 if it stalled. */
static int ml_coarsen(ml_run *R, int32_t l, const ml_graph *g, const int32_t *P, ml_graph *c, int32_t **cmap,
                      int32_t **cP) {
    if (l + 1 >= R->max_levels || g->n <= R->thr) return 0;
    const uint64_t seed = R->opt ? R->opt->seed : 0;
    const uint64_t sl = fro_splitmix64(seed ^ (uint64_t)l ^ ((uint64_t)(uint32_t)R->count[l] << 32));
    R->count[l] += 1;
    R->out->coarsenings += 1;
    int32_t *mate = XALLOC(int32_t, g->n);
    const int32_t pairs = ml_match(g->n, g->xadj, g->adjncy, g->adjwgt, g->vwgt, P, R->k, R->W, sl, mate);
    if (pairs == 0 || 20LL * pairs < g->n) { free(mate); return 0; }
    *cmap = XALLOC(int32_t, g->n);
    ml_contract(g, mate, c, *cmap);
    *cP = XALLOC(int32_t, c->n);
    for (int32_t v = 0; v < g->n; ++v) (*cP)[(*cmap)[v]] = P[v];
    free(mate);
    return 1;
}

static void ml_cycle(ml_run *R, int32_t l, const ml_graph *g, int32_t *P) {
    if (R->st != FRO_OK) return;
    if (l + 1 > R->out->depth) R->out->depth = l + 1;
    for (int32_t trial = 0; trial < 2; ++trial) {
        if (trial == 1) {
            if (l % R->d != 0 || R->type == 0) break;
            if (R->type == 2 && R->count[l] >= 2) break;
        }
        ml_graph c;
        int32_t *cmap = NULL, *cP = NULL;
        if (!ml_coarsen(R, l, g, P, &c, &cmap, &cP)) {
            if (trial == 0) ml_refine(R, g, P);   /* the coarsest graph of this branch */
            break;
        }
        ml_cycle(R, l + 1, &c, cP);
        for (int32_t v = 0; v < g->n; ++v) P[v] = cP[cmap[v]];
        ml_refine(R, g, P);
        ml_free(&c);
        free(cmap); free(cP);
    }
}

int32_t fro_cycle(int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *adjwgt, const int32_t *vwgt,
                  int32_t *part, int32_t k, double eps, double alpha, const fro_options *opt, int32_t type, int32_t d,
                  int32_t max_levels, int32_t active_outer, fro_cycle_result *out) {
    memset(out, 0, sizeof(*out));
    int32_t st = fro_validate(n, xadj, adjncy, adjwgt, vwgt, part, k);
    if (st == FRO_OK && (!(eps > 0.0) || !(alpha >= 1.0) || type < 0 || type > 2 || d < 1 || max_levels < 1 ||
                         max_levels > FRO_MAX_LEVELS || active_outer < 0 || bad_fm(opt) ||
                         (opt && opt->mt_alpha < 0) || (bad_mt(opt) && active_outer == 0)))
        st = FRO_ERR_INVALID_ARG;
    if (st != FRO_OK) return st;
    ml_run R;
    memset(&R, 0, sizeof(R));
    R.k = k; R.type = type; R.d = d; R.max_levels = max_levels; R.active_outer = active_outer;
    R.eps = eps; R.alpha = alpha; R.opt = opt; R.out = out; R.st = FRO_OK;
    R.W = fro_total_weight(n, vwgt);
    R.thr = 60LL * k;
    if ((int64_t)n / (60LL * k) > R.thr) R.thr = (int64_t)n / (60LL * k);
    ml_graph g = { n, xadj[n], (int32_t *)xadj, (int32_t *)adjncy, (int32_t *)adjwgt, (int32_t *)vwgt };
    int32_t *P = XALLOC(int32_t, n);
    memcpy(P, part, sizeof(int32_t) * (size_t)n);
    for (int32_t v = 0; v < n; ++v)
        for (int32_t j = xadj[v]; j < xadj[v + 1]; ++j)
            if (v < adjncy[j] && part[v] != part[adjncy[j]]) out->cut_before += adjwgt[j];
    ml_cycle(&R, 0, &g, P);
    if (R.st == FRO_OK) {
        memcpy(part, P, sizeof(int32_t) * (size_t)n);
        for (int32_t v = 0; v < n; ++v)
            for (int32_t j = xadj[v]; j < xadj[v + 1]; ++j)
                if (v < adjncy[j] && part[v] != part[adjncy[j]]) out->cut_after += adjwgt[j];
        for (int32_t l = 0; l < FRO_MAX_LEVELS; ++l) out->level_coarsenings[l] = R.count[l];
    }
    free(P);
    return R.st;
}
