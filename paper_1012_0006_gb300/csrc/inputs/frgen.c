/*
 * Seeded synthetic input generators: meshes, random geometric graphs, weights,
 * coordinate-bisection partitions and boundary noise.
 *
 * The paper evaluates on random geometric graphs (points in the unit square,
 * edges below a distance threshold), Delaunay meshes and FEM graphs, with k in
 * {2..64} and an imbalance of 1-5 % (Section 6, "Instances").  Those datasets are
 * not available here, so these generators produce inputs with the same shape:
 * 2D/3D grids (FEM-like meshes) and 2D/3D random geometric graphs.
 *
 * This module is shared by the tests, the benchmark and the serving driver.  It
 * contains none of the refinement method's arithmetic: no corridor, no flow, no
 * balance bound of the method.  Both the CPU oracle and the CUDA path only ever
 * see the arrays it writes.
 *
 * Random numbers: splitmix64 (Steele, Lea, Flood 2014; constants as published
 * by Vigna) used as a stream: state += 0x9E3779B97F4A7C15, output = mix(state).
 * Doubles take the top 53 bits.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

static uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static uint64_t sm64_next(uint64_t *state) {
    *state += 0x9E3779B97F4A7C15ULL;
    return sm64_mix(*state);
}

static double sm64_unit(uint64_t *state) {
    return (double)(sm64_next(state) >> 11) * (1.0 / 9007199254740992.0);
}

/* ---------------------------------------------------------------- grids -- */

/* 2D 4-neighbour grid, row-major ids (id = y*nx + x); neighbours in ascending id. */
int64_t frg_grid2d_nnz(int32_t nx, int32_t ny) {
    return 2LL * (nx - 1) * ny + 2LL * nx * (ny - 1);
}

void frg_grid2d(int32_t nx, int32_t ny, int32_t *xadj, int32_t *adjncy, double *coords) {
    int64_t e = 0;
    for (int32_t y = 0; y < ny; ++y)
        for (int32_t x = 0; x < nx; ++x) {
            int32_t v = y * nx + x;
            xadj[v] = (int32_t)e;
            if (y > 0) adjncy[e++] = v - nx;
            if (x > 0) adjncy[e++] = v - 1;
            if (x + 1 < nx) adjncy[e++] = v + 1;
            if (y + 1 < ny) adjncy[e++] = v + nx;
            if (coords) { coords[2 * (int64_t)v] = x; coords[2 * (int64_t)v + 1] = y; }
        }
    xadj[(int64_t)nx * ny] = (int32_t)e;
}

/* 3D 7-point grid, id = (z*ny + y)*nx + x; neighbours in ascending id. */
int64_t frg_grid3d_nnz(int32_t nx, int32_t ny, int32_t nz) {
    return 2LL * ((int64_t)(nx - 1) * ny * nz + (int64_t)nx * (ny - 1) * nz + (int64_t)nx * ny * (nz - 1));
}

void frg_grid3d(int32_t nx, int32_t ny, int32_t nz, int32_t *xadj, int32_t *adjncy, double *coords) {
    int64_t e = 0;
    int64_t plane = (int64_t)nx * ny;
    for (int32_t z = 0; z < nz; ++z)
        for (int32_t y = 0; y < ny; ++y)
            for (int32_t x = 0; x < nx; ++x) {
                int64_t v = z * plane + (int64_t)y * nx + x;
                xadj[v] = (int32_t)e;
                if (z > 0) adjncy[e++] = (int32_t)(v - plane);
                if (y > 0) adjncy[e++] = (int32_t)(v - nx);
                if (x > 0) adjncy[e++] = (int32_t)(v - 1);
                if (x + 1 < nx) adjncy[e++] = (int32_t)(v + 1);
                if (y + 1 < ny) adjncy[e++] = (int32_t)(v + nx);
                if (z + 1 < nz) adjncy[e++] = (int32_t)(v + plane);
                if (coords) {
                    coords[3 * v] = x; coords[3 * v + 1] = y; coords[3 * v + 2] = z;
                }
            }
    xadj[(int64_t)nx * ny * nz] = (int32_t)e;
}

/* ------------------------------------------------ random geometric graphs -- */

/*
 * Points uniform in the unit square (dim=2) or cube (dim=3), drawn in generation
 * order from one splitmix64 stream.  Vertex ids follow the row-major order of an
 * r-sized cell grid (x fastest), ties by generation index, so that ids have the
 * spatial locality of a mesh numbering.  coords_out receives the points in id order.
 */
static int32_t rgg_cells(double r) {
    double g = floor(1.0 / r);
    if (g < 1.0) g = 1.0;
    if (g > 1024.0) g = 1024.0;
    return (int32_t)g;
}

static int64_t rgg_cell_of(int dim, int32_t G, const double *p) {
    int64_t c = 0;
    for (int d = dim - 1; d >= 0; --d) {
        int64_t q = (int64_t)(p[d] * G);
        if (q >= G) q = G - 1;
        if (q < 0) q = 0;
        c = c * G + q;
    }
    return c;
}

void frg_rgg_points(int32_t dim, int32_t n, double r, uint64_t seed, double *coords_out) {
    int32_t G = rgg_cells(r);
    int64_t ncell = 1;
    for (int d = 0; d < dim; ++d) ncell *= G;
    double *raw = (double *)malloc(sizeof(double) * (size_t)n * dim);
    int64_t *cell = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t *cnt = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
    uint64_t st = seed;
    for (int32_t i = 0; i < n; ++i) {
        for (int d = 0; d < dim; ++d) raw[(int64_t)i * dim + d] = sm64_unit(&st);
        cell[i] = rgg_cell_of(dim, G, raw + (int64_t)i * dim);
        cnt[cell[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell; ++c) cnt[c + 1] += cnt[c];
    for (int32_t i = 0; i < n; ++i) {   /* stable counting sort by cell */
        int64_t pos = cnt[cell[i]]++;
        for (int d = 0; d < dim; ++d) coords_out[pos * dim + d] = raw[(int64_t)i * dim + d];
    }
    free(raw); free(cell); free(cnt);
}

/*
 * Edges join points whose squared distance is strictly below r^2.  Called with
 * adjncy == NULL it only fills xadj and returns nnz; called again with adjncy it
 * fills the rows.  Rows come out in ascending neighbour id because cells are
 * visited in ascending cell index and ids follow cell order.
 */
int64_t frg_rgg_edges(int32_t dim, int32_t n, double r, const double *coords,
                      int32_t *xadj, int32_t *adjncy) {
    int32_t G = rgg_cells(r);
    int64_t ncell = 1;
    for (int d = 0; d < dim; ++d) ncell *= G;
    int64_t *start = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
    for (int32_t i = 0; i < n; ++i) start[rgg_cell_of(dim, G, coords + (int64_t)i * dim) + 1]++;
    for (int64_t c = 0; c < ncell; ++c) start[c + 1] += start[c];
    double r2 = r * r;
    int64_t e = 0;
    for (int32_t i = 0; i < n; ++i) {
        const double *p = coords + (int64_t)i * dim;
        int64_t ci[3] = {0, 0, 0};
        for (int d = 0; d < dim; ++d) {
            int64_t q = (int64_t)(p[d] * G);
            if (q >= G) q = G - 1;
            ci[d] = q;
        }
        xadj[i] = (int32_t)e;
        int dzlo = dim == 3 ? -1 : 0, dzhi = dim == 3 ? 1 : 0;
        for (int dz = dzlo; dz <= dzhi; ++dz) {
            int64_t cz = ci[2] + dz;
            if (cz < 0 || cz >= G) continue;
            for (int dy = -1; dy <= 1; ++dy) {
                int64_t cy = ci[1] + dy;
                if (cy < 0 || cy >= G) continue;
                for (int dx = -1; dx <= 1; ++dx) {
                    int64_t cx = ci[0] + dx;
                    if (cx < 0 || cx >= G) continue;
                    int64_t c = (dim == 3 ? (cz * G + cy) * G + cx : cy * G + cx);
                    for (int64_t j = start[c]; j < start[c + 1]; ++j) {
                        if (j == i) continue;
                        const double *q = coords + j * dim;
                        double s = 0.0;
                        for (int d = 0; d < dim; ++d) { double t = p[d] - q[d]; s += t * t; }
                        if (s < r2) {
                            if (adjncy) adjncy[e] = (int32_t)j;
                            ++e;
                        }
                    }
                }
            }
        }
    }
    xadj[n] = (int32_t)e;
    free(start);
    return e;
}

/* ---------------------------------------------------------------- weights -- */

/* Uniform integers in [lo, hi] from one stream (value = lo + draw mod range). */
void frg_uniform_i32(int64_t count, int32_t lo, int32_t hi, uint64_t seed, int32_t *out) {
    uint64_t st = seed;
    uint64_t range = (uint64_t)((int64_t)hi - lo + 1);
    for (int64_t i = 0; i < count; ++i) out[i] = (int32_t)(lo + (int64_t)(sm64_next(&st) % range));
}

/* Symmetric edge weights in [lo, hi]: a hash of the unordered endpoint pair. */
void frg_edge_weights(int32_t n, const int32_t *xadj, const int32_t *adjncy, int32_t lo, int32_t hi,
                      uint64_t seed, int32_t *adjwgt) {
    uint64_t range = (uint64_t)((int64_t)hi - lo + 1);
    for (int32_t v = 0; v < n; ++v)
        for (int32_t j = xadj[v]; j < xadj[v + 1]; ++j) {
            uint64_t u = (uint64_t)adjncy[j];
            uint64_t a = (uint64_t)v < u ? (uint64_t)v : u;
            uint64_t b = (uint64_t)v < u ? u : (uint64_t)v;
            uint64_t h = sm64_mix(seed ^ sm64_mix((a << 32) | b) ^ 0x9E3779B97F4A7C15ULL);
            adjwgt[j] = (int32_t)(lo + (int64_t)(h % range));
        }
}

/* ------------------------------------------- recursive coordinate bisection -- */

typedef struct { double key; int32_t id; } keyed;

static const double *g_sort_coords;
static int g_sort_dim, g_sort_axis;

static int cmp_axis(const void *pa, const void *pb) {
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    double ka = g_sort_coords[(int64_t)a * g_sort_dim + g_sort_axis];
    double kb = g_sort_coords[(int64_t)b * g_sort_dim + g_sort_axis];
    if (ka < kb) return -1;
    if (ka > kb) return 1;
    return (a > b) - (a < b);
}

/*
 * Split ids[0..cnt) into k blocks numbered b0..b0+k-1.  The axis is the longest
 * bounding-box extent (ties: x before y before z) unless force_axis >= 0 at the
 * top level.  The set is sorted by (coordinate, id) and split at the first prefix
 * whose weight reaches total * kl / k, with kl = k/2 blocks on the low side.
 */
static void rcb_rec(int32_t *ids, int64_t cnt, int dim, const double *coords, const int32_t *vwgt,
                    int32_t k, int32_t b0, int force_axis, int32_t *part) {
    if (k <= 1 || cnt == 0) {
        for (int64_t i = 0; i < cnt; ++i) part[ids[i]] = b0;
        return;
    }
    int axis = force_axis;
    if (axis < 0) {
        double best = -1.0;
        for (int d = 0; d < dim; ++d) {
            double lo = INFINITY, hi = -INFINITY;
            for (int64_t i = 0; i < cnt; ++i) {
                double c = coords[(int64_t)ids[i] * dim + d];
                if (c < lo) lo = c;
                if (c > hi) hi = c;
            }
            if (hi - lo > best) { best = hi - lo; axis = d; }
        }
    }
    g_sort_coords = coords; g_sort_dim = dim; g_sort_axis = axis;
    qsort(ids, (size_t)cnt, sizeof(int32_t), cmp_axis);
    int32_t kl = k / 2;
    int64_t total = 0;
    for (int64_t i = 0; i < cnt; ++i) total += vwgt ? vwgt[ids[i]] : 1;
    /* target = total*kl/k, compared exactly in integers: prefix*k >= total*kl */
    int64_t acc = 0, split = cnt;
    for (int64_t i = 0; i < cnt; ++i) {
        acc += vwgt ? vwgt[ids[i]] : 1;
        if (acc * k >= total * kl) { split = i + 1; break; }
    }
    rcb_rec(ids, split, dim, coords, vwgt, kl, b0, -1, part);
    rcb_rec(ids + split, cnt - split, dim, coords, vwgt, k - kl, b0 + kl, -1, part);
}

void frg_rcb(int32_t n, int32_t dim, const double *coords, const int32_t *vwgt, int32_t k,
             int32_t force_axis, int32_t *part) {
    int32_t *ids = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int32_t i = 0; i < n; ++i) ids[i] = i;
    rcb_rec(ids, n, dim, coords, vwgt, k, 0, force_axis, part);
    free(ids);
}

/* ------------------------------------------------------- boundary noise -- */

/*
 * Boundary noise: candidates are the vertices that, before any swap, have a
 * neighbour in another block (ascending id).  Each of nswaps draws picks a
 * candidate v uniformly; if v still has neighbours in other blocks, one of them
 * (u, uniform) is chosen and the labels of u and v are exchanged.  A swap is
 * skipped when it would lift a block above the heaviest block weight present
 * before the noise, so the noise never makes the partition less balanced than
 * its starting point.  If nswaps < 0, the count is round(-nswaps/1e6 * |cand|),
 * i.e. a fraction of the boundary given in parts per million.  Returns the
 * number of swaps applied.
 */
int64_t frg_noise(int32_t n, const int32_t *xadj, const int32_t *adjncy, const int32_t *vwgt,
                  int32_t k, int32_t *part, int64_t nswaps, uint64_t seed) {
    int64_t *bw = (int64_t *)calloc((size_t)k, sizeof(int64_t));
    int64_t bmax = 0;
    for (int32_t v = 0; v < n; ++v) bw[part[v]] += vwgt ? vwgt[v] : 1;
    for (int32_t b = 0; b < k; ++b) if (bw[b] > bmax) bmax = bw[b];
    int32_t *cand = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t nc = 0;
    for (int32_t v = 0; v < n; ++v)
        for (int32_t j = xadj[v]; j < xadj[v + 1]; ++j)
            if (part[adjncy[j]] != part[v]) { cand[nc++] = v; break; }
    if (nswaps < 0) nswaps = (int64_t)llround((double)(-nswaps) * 1e-6 * (double)nc);
    uint64_t st = seed;
    int64_t applied = 0;
    int32_t *other = (int32_t *)malloc(sizeof(int32_t) * 4096);
    for (int64_t s = 0; s < nswaps && nc > 0; ++s) {
        int32_t v = cand[sm64_next(&st) % (uint64_t)nc];
        int64_t no = 0;
        for (int32_t j = xadj[v]; j < xadj[v + 1] && no < 4096; ++j)
            if (part[adjncy[j]] != part[v]) other[no++] = adjncy[j];
        uint64_t pick = sm64_next(&st);
        if (no == 0) continue;
        int32_t u = other[pick % (uint64_t)no];
        int32_t pv = part[v], pu = part[u];
        int64_t cv = vwgt ? vwgt[v] : 1, cu = vwgt ? vwgt[u] : 1;
        if (bw[pv] - cv + cu > bmax || bw[pu] - cu + cv > bmax) continue;
        bw[pv] += cu - cv; bw[pu] += cv - cu;
        part[v] = pu; part[u] = pv;
        ++applied;
    }
    free(other); free(cand); free(bw);
    return applied;
}
