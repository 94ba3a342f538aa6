/*
 * Plain CPU DBSCAN oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this library. The product path (the CUDA library) shares no code,
 * header, table or helper with it.
 *
 * What it computes is the DBSCAN clustering as the paper defines it (Sec. 2.1):
 *   N_eps(x)   = { y in X : dist(x, y) <= eps }        (x is in its own N_eps)
 *   core(x)   <=> |N_eps(x)| >= minPts
 *   clusters   = connected components of the graph on the core points whose
 *                edges join core points within eps of each other
 *   border(x) <=> x is not core but lies within eps of a core point; it may
 *                belong to the cluster of any such core point (Sec. 2.1; the
 *                paper notes implementations differ in which one they pick)
 *   noise      = the remaining points
 * For DBSCAN* (Sec. 2.1, last paragraph) border points are noise.
 *
 * Distance test. The paper uses the Euclidean distance and leaves the
 * rounding open; this oracle fixes it as the fp32 squared form with no fused
 * multiply-add, in this order:
 *   dk = fl(x_k - y_k);  s = fl(d0*d0);  s = fl(s + fl(dk*dk)) for k = 1..d-1
 *   adjacent  <=>  s <= fl(eps*eps)
 * This file must be compiled with -ffp-contract=off (no contraction) and
 * without fast-math; FLT_EVAL_METHOD must be 0 (checked below).
 *
 * Labels are canonical: a cluster is labelled by the smallest input index of
 * its core points; noise is -1. A border point gets the smallest label among
 * the clusters it may join (the full valid set is available through
 * oracle_border_sets()).
 *
 * Method. A uniform grid whose cell side is at least the largest coordinate
 * gap of any pair that passes the test serves only as a candidate filter:
 * every candidate in the 3^d surrounding cells is decided by the exact test
 * above. Counting stops once minPts neighbours are seen, which the paper
 * notes is enough to decide core status (Sec. 3.2). Connected components use
 * a sequential union-find with union by smaller index.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#if !defined(FLT_EVAL_METHOD) || FLT_EVAL_METHOD != 0
#error "the oracle needs FLT_EVAL_METHOD == 0 (plain fp32 evaluation)"
#endif

#define ORACLE_MAX_DIM 8

/* ---- the distance test --------------------------------------------------- */

static int adjacent(const float* a, const float* b, int d, float e2)
{
    float t = a[0] - b[0];
    float s = t * t;
    for (int k = 1; k < d; ++k) {
        float u = a[k] - b[k];
        float v = u * u;
        s = s + v;
    }
    return s <= e2;
}

int oracle_adjacent(const float* a, const float* b, int d, float eps)
{
    float e2 = eps * eps;
    return adjacent(a, b, d, e2);
}

float oracle_dist2(const float* a, const float* b, int d)
{
    float t = a[0] - b[0];
    float s = t * t;
    for (int k = 1; k < d; ++k) {
        float u = a[k] - b[k];
        float v = u * u;
        s = s + v;
    }
    return s;
}

/* ---- candidate grid ------------------------------------------------------ */

typedef struct {
    int d;
    int64_t n;
    int64_t* cc;      /* cell coordinates, n x d */
    int64_t* order;   /* point indices sorted by cell (lexicographic), then index */
    int64_t ncells;
    int64_t* cstart;  /* ncells + 1 offsets into order */
} grid_t;

static int cmp_cell(const int64_t* cc, int d, int64_t a, int64_t b)
{
    for (int k = 0; k < d; ++k) {
        int64_t x = cc[a * d + k], y = cc[b * d + k];
        if (x != y) return x < y ? -1 : 1;
    }
    return (a < b) ? -1 : (a > b);
}

/* bottom-up merge sort of point indices by cell */
static void sort_by_cell(int64_t* a, int64_t n, const int64_t* cc, int d)
{
    int64_t* tmp = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    for (int64_t w = 1; w < n; w *= 2) {
        for (int64_t lo = 0; lo < n; lo += 2 * w) {
            int64_t mid = lo + w < n ? lo + w : n;
            int64_t hi = lo + 2 * w < n ? lo + 2 * w : n;
            int64_t i = lo, j = mid, k = lo;
            while (i < mid && j < hi) tmp[k++] = (cmp_cell(cc, d, a[i], a[j]) <= 0) ? a[i++] : a[j++];
            while (i < mid) tmp[k++] = a[i++];
            while (j < hi) tmp[k++] = a[j++];
        }
        memcpy(a, tmp, (size_t)n * sizeof(int64_t));
    }
    free(tmp);
}

static int grid_build(grid_t* g, const float* X, int64_t n, int d, float eps)
{
    double lo[ORACLE_MAX_DIM], hi[ORACLE_MAX_DIM];
    g->d = d;
    g->n = n;
    for (int k = 0; k < d; ++k) { lo[k] = INFINITY; hi[k] = -INFINITY; }
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < d; ++k) {
            double v = X[i * d + k];
            if (v < lo[k]) lo[k] = v;
            if (v > hi[k]) hi[k] = v;
        }
    /* Any pair that passes the fp32 test has |x_k - y_k| < max(eps, 2^-60)
     * * (1 + 2^-22) on every axis (rounding of the differences, squares and
     * of eps*eps is at most a few ulps; below 2^-60 a squared gap is still a
     * normal fp32 number larger than any eps^2 that small). The 2^-10 margin
     * covers that and the fp64 rounding of the cell coordinates below. */
    double h = (eps > 0x1p-60f ? (double)eps : 0x1p-60) * (1.0 + 0x1p-10);
    for (int k = 0; k < d; ++k) {
        double ext = hi[k] - lo[k];
        if (ext / h > 0x1p30) h = ext * 0x1p-30; /* coarser cells stay correct */
    }
    g->cc = (int64_t*)malloc((size_t)n * d * sizeof(int64_t));
    g->order = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    g->cstart = (int64_t*)malloc((size_t)(n + 1) * sizeof(int64_t));
    if (!g->cc || !g->order || !g->cstart) return -1;
    for (int64_t i = 0; i < n; ++i) {
        g->order[i] = i;
        for (int k = 0; k < d; ++k)
            g->cc[i * d + k] = (int64_t)floor(((double)X[i * d + k] - lo[k]) / h);
    }
    sort_by_cell(g->order, n, g->cc, d);
    int64_t c = 0;
    for (int64_t s = 0; s < n; ++s) {
        int same = 0;
        if (s > 0) {
            same = 1;
            for (int k = 0; k < d; ++k)
                if (g->cc[g->order[s - 1] * d + k] != g->cc[g->order[s] * d + k]) { same = 0; break; }
        }
        if (!same) g->cstart[c++] = s;
    }
    g->cstart[c] = n;
    g->ncells = c;
    return 0;
}

static void grid_free(grid_t* g)
{
    free(g->cc);
    free(g->order);
    free(g->cstart);
}

/* index of the cell with coordinates key[0..d-1], or -1 */
static int64_t grid_find(const grid_t* g, const int64_t* key)
{
    int64_t a = 0, b = g->ncells;
    while (a < b) {
        int64_t m = a + (b - a) / 2;
        const int64_t* cm = g->cc + g->order[g->cstart[m]] * g->d;
        int c = 0;
        for (int k = 0; k < g->d; ++k)
            if (cm[k] != key[k]) { c = cm[k] < key[k] ? -1 : 1; break; }
        if (c == 0) return m;
        if (c < 0) a = m + 1; else b = m;
    }
    return -1;
}

/* The cells (by index) within one step of cell c on every axis, c included;
 * returns their number (at most 3^d). */
static int neighbor_cells(const grid_t* g, int64_t c, int64_t* out)
{
    const int d = g->d;
    const int64_t* base = g->cc + g->order[g->cstart[c]] * d;
    int64_t key[ORACLE_MAX_DIM];
    int off[ORACLE_MAX_DIM];
    int m = 0;
    for (int k = 0; k < d; ++k) off[k] = -1;
    for (;;) {
        for (int k = 0; k < d; ++k) key[k] = base[k] + off[k];
        int64_t f = grid_find(g, key);
        if (f >= 0) out[m++] = f;
        int k = 0;
        while (k < d && off[k] == 1) { off[k] = -1; ++k; }
        if (k == d) break;
        off[k] += 1;
    }
    return m;
}

/* Calls visit(ctx, i, j) for every point i (cell by cell) and every j with
 * adjacent(x_i, x_j); the scan of point i stops early when visit returns
 * nonzero. Only points with want[i] != 0 are scanned (want may be NULL). */
typedef int (*visit_fn)(void* ctx, int64_t i, int64_t j);

static void for_each_pair(const grid_t* g, const float* X, float e2, const uint8_t* want, visit_fn visit, void* ctx)
{
    const int d = g->d;
    int64_t* nb = (int64_t*)malloc(sizeof(int64_t) * 6561); /* 3^8 */
    for (int64_t c = 0; c < g->ncells; ++c) {
        int m = -1;
        for (int64_t s = g->cstart[c]; s < g->cstart[c + 1]; ++s) {
            int64_t i = g->order[s];
            if (want && !want[i]) continue;
            if (m < 0) m = neighbor_cells(g, c, nb);
            int stop = 0;
            for (int t = 0; t < m && !stop; ++t) {
                for (int64_t r = g->cstart[nb[t]]; r < g->cstart[nb[t] + 1]; ++r) {
                    int64_t j = g->order[r];
                    if (adjacent(X + i * d, X + j * d, d, e2) && visit(ctx, i, j)) { stop = 1; break; }
                }
            }
        }
    }
    free(nb);
}

/* ---- union-find (sequential; root = smallest index of the set) ----------- */

static int64_t uf_find(int32_t* p, int64_t x)
{
    int64_t r = x;
    while (p[r] != r) r = p[r];
    while (p[x] != r) { int64_t nx = p[x]; p[x] = (int32_t)r; x = nx; }
    return r;
}

static void uf_union(int32_t* p, int64_t a, int64_t b)
{
    a = uf_find(p, a);
    b = uf_find(p, b);
    if (a == b) return;
    if (a < b) p[b] = (int32_t)a; else p[a] = (int32_t)b;
}

/* ---- visitors ------------------------------------------------------------- */

typedef struct { int32_t* count; int32_t cap; } count_ctx;

static int visit_count(void* c, int64_t i, int64_t j)
{
    (void)j;
    count_ctx* cc = (count_ctx*)c;
    cc->count[i] += 1;
    return cc->count[i] >= cc->cap;
}

typedef struct { int32_t* parent; const uint8_t* core; } union_ctx;

static int visit_union(void* c, int64_t i, int64_t j)
{
    union_ctx* u = (union_ctx*)c;
    if (j > i && u->core[j]) uf_union(u->parent, i, j);
    return 0;
}

typedef struct { const uint8_t* core; int32_t* labels; } minlabel_ctx;

/* labels[i] of a non-core point holds the best label so far (INT32_MAX if none) */
static int visit_minlabel(void* c, int64_t i, int64_t j)
{
    minlabel_ctx* b = (minlabel_ctx*)c;
    if (b->core[j] && b->labels[j] < b->labels[i]) b->labels[i] = b->labels[j];
    return 0;
}

typedef struct { int64_t i; int32_t l; } rec_t;
typedef struct { const uint8_t* core; const int32_t* labels; rec_t* rec; int64_t k, cap; } pairs_ctx;

static int visit_collect(void* c, int64_t i, int64_t j)
{
    pairs_ctx* p = (pairs_ctx*)c;
    if (!p->core[j]) return 0;
    if (p->k == p->cap) {
        p->cap = p->cap ? 2 * p->cap : 1024;
        p->rec = (rec_t*)realloc(p->rec, (size_t)p->cap * sizeof(rec_t));
    }
    p->rec[p->k].i = i;
    p->rec[p->k].l = p->labels[j];
    p->k += 1;
    return 0;
}

static int cmp_rec(const void* a, const void* b)
{
    const rec_t* x = (const rec_t*)a;
    const rec_t* y = (const rec_t*)b;
    if (x->i != y->i) return x->i < y->i ? -1 : 1;
    return (x->l > y->l) - (x->l < y->l);
}

static int check_args(const float* X, int64_t n, int d, float eps)
{
    if (n < 0 || d < 1 || d > ORACLE_MAX_DIM) return -1;
    if (n > 0 && !X) return -1;
    if (!(eps > 0.0f) || isinf(eps)) return -1;
    if (n >= ((int64_t)1 << 31) - 1) return -1;
    for (int64_t i = 0; i < n * d; ++i)
        if (!isfinite(X[i])) return -2;
    return 0;
}

/* ---- public entry points ---------------------------------------------------- */

/*
 * Full DBSCAN (mode 0) or DBSCAN* (mode 1) clustering.
 * X: n x d row-major fp32. labels: n int32 out (canonical, -1 = noise).
 * core: n bytes out (1 = core point). Returns 0, -1 (bad argument) or
 * -2 (non-finite coordinate).
 */
int oracle_dbscan(const float* X, int64_t n, int d, float eps, int min_pts, int mode,
                  int32_t* labels, uint8_t* core)
{
    int rc = check_args(X, n, d, eps);
    if (rc) return rc;
    if (min_pts < 1 || (mode != 0 && mode != 1)) return -1;
    if (n == 0) return 0;
    const float e2 = eps * eps;
    grid_t g;
    if (grid_build(&g, X, n, d, eps)) return -1;

    /* core points: |N_eps(x)| >= minPts, counting x itself */
    int32_t* count = (int32_t*)calloc((size_t)n, sizeof(int32_t));
    count_ctx cnt = {count, min_pts};
    for_each_pair(&g, X, e2, NULL, visit_count, &cnt);
    for (int64_t i = 0; i < n; ++i) core[i] = (uint8_t)(count[i] >= min_pts);
    free(count);

    /* clusters: connected components of the core graph */
    int32_t* parent = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    for (int64_t i = 0; i < n; ++i) parent[i] = (int32_t)i;
    union_ctx u = {parent, core};
    for_each_pair(&g, X, e2, core, visit_union, &u);
    for (int64_t i = 0; i < n; ++i)
        labels[i] = core[i] ? (int32_t)uf_find(parent, i) : -1;

    /* border points join the cluster with the smallest label among the
     * clusters of their core neighbours (DBSCAN); noise in DBSCAN*. The
     * visitor reads labels of core points only, which are final here. */
    if (mode == 0) {
        uint8_t* noncore = (uint8_t*)calloc((size_t)n, 1);
        for (int64_t i = 0; i < n; ++i) {
            noncore[i] = (uint8_t)!core[i];
            if (!core[i]) labels[i] = INT32_MAX;
        }
        minlabel_ctx b = {core, labels};
        for_each_pair(&g, X, e2, noncore, visit_minlabel, &b);
        for (int64_t i = 0; i < n; ++i)
            if (!core[i] && labels[i] == INT32_MAX) labels[i] = -1;
        free(noncore);
    }
    free(parent);
    grid_free(&g);
    return 0;
}

/*
 * For every non-core point, the sorted set of labels of the clusters it may
 * join (labels of its core neighbours, given core flags and canonical labels
 * of core points as produced by oracle_dbscan). CSR output: offsets has n+1
 * entries; sets receives up to cap labels. Returns the total number of labels
 * (call once with cap = 0 to size the buffer), or a negative error.
 */
int64_t oracle_border_sets(const float* X, int64_t n, int d, float eps, const uint8_t* core,
                           const int32_t* labels, int64_t* offsets, int32_t* sets, int64_t cap)
{
    int rc = check_args(X, n, d, eps);
    if (rc) return rc;
    if (n == 0) { if (offsets) offsets[0] = 0; return 0; }
    const float e2 = eps * eps;
    grid_t g;
    if (grid_build(&g, X, n, d, eps)) return -1;
    /* pass 1: for every non-core point, the labels of its core neighbours
     * (with repeats) in per-point lists; pass 2: sort and deduplicate */
    uint8_t* noncore = (uint8_t*)calloc((size_t)n, 1);
    for (int64_t i = 0; i < n; ++i) noncore[i] = (uint8_t)!core[i];
    pairs_ctx pc = {core, labels, NULL, 0, 0};
    for_each_pair(&g, X, e2, noncore, visit_collect, &pc);
    /* sort (point, label) records */
    qsort(pc.rec, (size_t)pc.k, sizeof(rec_t), cmp_rec);
    int64_t total = 0, r = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (offsets) offsets[i] = total;
        int32_t last = INT32_MIN;
        while (r < pc.k && pc.rec[r].i == i) {
            if (pc.rec[r].l != last) {
                if (sets && total < cap) sets[total] = pc.rec[r].l;
                total += 1;
                last = pc.rec[r].l;
            }
            ++r;
        }
    }
    free(pc.rec);
    free(noncore);
    if (offsets) offsets[n] = total;
    grid_free(&g);
    return total;
}

/*
 * Brute force over all n points: the indices j with adjacent(x_q, x_j)
 * (x_q included), in increasing order. Writes up to cap of them to out and
 * returns their total number, or a negative error.
 */
int64_t oracle_point_neighbors(const float* X, int64_t n, int d, float eps, int64_t q, int64_t* out, int64_t cap)
{
    if (n < 0 || d < 1 || d > ORACLE_MAX_DIM || q < 0 || q >= n) return -1;
    if (!(eps > 0.0f) || isinf(eps)) return -1;
    const float e2 = eps * eps;
    int64_t k = 0;
    for (int64_t j = 0; j < n; ++j) {
        if (adjacent(X + q * d, X + j * d, d, e2)) {
            if (out && k < cap) out[k] = j;
            k += 1;
        }
    }
    return k;
}
