/*
 * Oracle: random geometric graph RGG(n, r) in the unit square / cube, Sec. 5.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The procedure, step by step:
 *  1. Coordinates are 32-bit fixed point: the integer x stands for x 2^-32.
 *     The radius becomes R = floor(r 2^32) (0 <= r <= 1/2), and {u, v} is an
 *     edge iff u != v and sum_k (x_k(u) - x_k(v))^2 <= R^2, in exact integer
 *     arithmetic.
 *  2. The grid (Sec. 5): G = 2^g cells per dimension, cell side 2^(32-g)
 *     lattice units.  g is the largest value with side >= R (so that every
 *     neighbour lies in one of the 3^d adjacent cells), at most n cells
 *     (side >= n^(-1/d)), and g <= 15 (d = 2) or 10 (d = 3).
 *  3. Vertex counts per cell (Sec. 5, "Parallelization"): the cube is split
 *     recursively into its 2^d subcubes; every split of a cube is done as d
 *     halvings, one per dimension (last dimension first), each drawing the
 *     count of the lower half as Binomial(c, 1/2) from the stream of its tree
 *     node (heap index h, tag 7).  This is a binary tree over the Morton
 *     index z of the cells (bit d*b + k of z = bit b of the cell coordinate
 *     along dimension k).  Binomial(c, 1/2) is the number of ones among c
 *     fair bits for c <= 1024, else the binomial variate of Sec. 2.2.
 *  4. Vertex ids: cells in row-major order (dimension 0 fastest), the points
 *     of a cell in draw order.
 *  5. Point j of the cell with coordinates (c_0 .. c_{d-1}) and Morton index
 *     z draws the Philox block with counter (j, lo32 z, hi32 z, 8): word k
 *     gives x_k = c_k 2^(32-g) + (w_k >> g), uniform over the cell's lattice
 *     points.
 *  6. Edges of vertex u (Sec. 5): compare u with every point of the cells
 *     adjacent to its own (its own included); emitted in both directions,
 *     sorted by (u, v).
 */
#include <stdlib.h>
#include <string.h>

#include "or_internal.h"

#define OR_TAG_RGG_TREE 7u
#define OR_TAG_RGG_POINT 8u
#define OR_RGG_FAIR_BITS_MAX 1024u

static int rgg_g_max(int dim) { return dim == 2 ? 15 : 10; }

static int rgg_check(int dim, uint64_t n, double r, uint64_t *R)
{
    if (dim != 2 && dim != 3) return 1;
    if (!(r >= 0.0 && r <= 0.5)) return 1;  /* also rejects NaN */
    if (n > 0xffffffffull) return 2;
    *R = (uint64_t)(r * 4294967296.0);      /* exact scaling, truncated = floor */
    return 0;
}

int or_rgg_grid_level(int dim, uint64_t n, double r, int *g_out)
{
    uint64_t R;
    int rc = rgg_check(dim, n, r, &R);
    if (rc) return rc;
    int g = 0;
    while (g < rgg_g_max(dim)) {
        const int h = g + 1;
        if (((uint64_t)1 << (32 - h)) < R) break;      /* cell side below R */
        if (((uint64_t)1 << (dim * h)) > n) break;     /* more cells than points */
        g = h;
    }
    *g_out = g;
    return 0;
}

/* Morton index of the cell with coordinates c[0..dim) on a 2^g grid. */
static uint64_t morton(const uint64_t *c, int dim, int g)
{
    uint64_t z = 0;
    for (int b = 0; b < g; ++b)
        for (int k = 0; k < dim; ++k)
            z |= ((c[k] >> b) & 1u) << (dim * b + k);
    return z;
}

/* Row-major cell index -> coordinates. */
static void cell_coords(uint64_t q, int dim, int g, uint64_t *c)
{
    const uint64_t G = (uint64_t)1 << g;
    for (int k = 0; k < dim; ++k) {
        c[k] = q % G;
        q /= G;
    }
}

/* Binomial(c, 1/2) of tree node h (step 3). */
static int half_split(uint64_t c, uint64_t seed, uint64_t h, uint64_t *x)
{
    if (c == 0) {
        *x = 0;
        return 0;
    }
    or_stream s = or_stream_make(seed, h, OR_TAG_RGG_TREE);
    if (c <= OR_RGG_FAIR_BITS_MAX) {
        uint64_t ones = 0, left = c;
        while (left > 0) {
            uint64_t w = or_next_u64(&s);
            if (left < 64) w &= ((uint64_t)1 << left) - 1;
            ones += (uint64_t)__builtin_popcountll(w);
            left = left < 64 ? 0 : left - 64;
        }
        *x = ones;
        return 0;
    }
    return or_binom_s(c, 0.5, &s, x);
}

/* Depth-first over the tree: node h at `level` holds c points; the leaves
 * (level D) are the cells, leaf h = 2^D + z. */
static int split_node(uint64_t h, int level, int D, uint64_t c, uint64_t seed, uint64_t *cnt_z)
{
    if (level == D) {
        cnt_z[h - ((uint64_t)1 << D)] = c;
        return 0;
    }
    uint64_t x;
    int rc = half_split(c, seed, h, &x);
    if (rc) return rc;
    rc = split_node(2 * h, level + 1, D, x, seed, cnt_z);
    if (rc) return rc;
    return split_node(2 * h + 1, level + 1, D, c - x, seed, cnt_z);
}

int or_rgg_cell_counts(int dim, uint64_t n, double r, uint64_t seed, uint64_t *cnt)
{
    int g;
    int rc = or_rgg_grid_level(dim, n, r, &g);
    if (rc) return rc;
    const int D = dim * g;
    const uint64_t cells = (uint64_t)1 << D;
    uint64_t *cnt_z = (uint64_t *)malloc(cells * sizeof(uint64_t));
    if (!cnt_z) return 6;
    rc = split_node(1, 0, D, n, seed, cnt_z);
    if (rc == 0) {
        uint64_t c[3];
        for (uint64_t q = 0; q < cells; ++q) {
            cell_coords(q, dim, g, c);
            cnt[q] = cnt_z[morton(c, dim, g)];
        }
    }
    free(cnt_z);
    return rc;
}

/* The point set: coordinates (n x dim, row-major) and the first id of every
 * cell (start[cells + 1]). */
typedef struct {
    int dim, g;
    uint64_t n, R, cells;
    uint64_t *start;
    uint32_t *x;
} rgg_points;

static void rgg_free(rgg_points *P)
{
    free(P->start);
    free(P->x);
}

static int rgg_make(int dim, uint64_t n, double r, uint64_t seed, rgg_points *P)
{
    memset(P, 0, sizeof(*P));
    int rc = rgg_check(dim, n, r, &P->R);
    if (rc) return rc;
    rc = or_rgg_grid_level(dim, n, r, &P->g);
    if (rc) return rc;
    P->dim = dim;
    P->n = n;
    P->cells = (uint64_t)1 << (dim * P->g);
    uint64_t *cnt = (uint64_t *)malloc(P->cells * sizeof(uint64_t));
    P->start = (uint64_t *)malloc((P->cells + 1) * sizeof(uint64_t));
    P->x = (uint32_t *)malloc((n ? n : 1) * (uint64_t)dim * sizeof(uint32_t));
    if (!cnt || !P->start || !P->x) {
        free(cnt);
        rgg_free(P);
        return 6;
    }
    rc = or_rgg_cell_counts(dim, n, r, seed, cnt);
    if (rc) {
        free(cnt);
        rgg_free(P);
        return rc;
    }
    uint64_t acc = 0;
    for (uint64_t q = 0; q < P->cells; ++q) {
        P->start[q] = acc;
        acc += cnt[q];
    }
    P->start[P->cells] = acc;
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    const int sh = 32 - P->g;
    for (uint64_t q = 0; q < P->cells; ++q) {
        uint64_t c[3];
        cell_coords(q, dim, P->g, c);
        const uint64_t z = morton(c, dim, P->g);
        for (uint64_t j = 0; j < cnt[q]; ++j) {
            const uint32_t ctr[4] = {(uint32_t)j, (uint32_t)z, (uint32_t)(z >> 32),
                                     OR_TAG_RGG_POINT};
            uint32_t w[4];
            or_philox4x32_10(ctr, key, w);
            const uint64_t id = P->start[q] + j;
            for (int k = 0; k < dim; ++k)
                P->x[id * dim + k] = (uint32_t)((c[k] << sh) | (w[k] >> P->g));
        }
    }
    free(cnt);
    return 0;
}

int or_rgg_points(int dim, uint64_t n, double r, uint64_t seed, uint32_t *coords)
{
    rgg_points P;
    int rc = rgg_make(dim, n, r, seed, &P);
    if (rc) return rc;
    memcpy(coords, P.x, n * (uint64_t)dim * sizeof(uint32_t));
    rgg_free(&P);
    return 0;
}

/* step 1's predicate */
static int within(const rgg_points *P, uint64_t u, uint64_t v)
{
    uint64_t s = 0;
    for (int k = 0; k < P->dim; ++k) {
        const uint64_t a = P->x[u * P->dim + k], b = P->x[v * P->dim + k];
        const uint64_t d = a > b ? a - b : b - a;
        if (d > P->R) return 0;
        s += d * d;  /* d <= R <= 2^31: at most 3 * 2^62 */
    }
    return s <= P->R * P->R;
}

/* Step 6 for vertex u: calls emit(v) for its neighbours in increasing order. */
typedef void (*emit_fn)(void *ctx, uint64_t u, uint64_t v);

static void rgg_row(const rgg_points *P, uint64_t u, emit_fn emit, void *ctx)
{
    const int g = P->g, sh = 32 - g;
    const int64_t G = (int64_t)1 << g;
    int64_t c[3] = {0, 0, 0};
    for (int k = 0; k < P->dim; ++k) c[k] = (int64_t)((uint64_t)P->x[u * P->dim + k] >> sh);
    /* the 3^d adjacent cells in row-major order: last dimension outermost */
    const int64_t d2lo = P->dim == 3 ? -1 : 0, d2hi = P->dim == 3 ? 1 : 0;
    for (int64_t e2 = d2lo; e2 <= d2hi; ++e2) {
        const int64_t c2 = c[2] + e2;
        if (c2 < 0 || c2 >= G) continue;
        for (int64_t e1 = -1; e1 <= 1; ++e1) {
            const int64_t c1 = c[1] + e1;
            if (c1 < 0 || c1 >= G) continue;
            for (int64_t e0 = -1; e0 <= 1; ++e0) {
                const int64_t c0 = c[0] + e0;
                if (c0 < 0 || c0 >= G) continue;
                const uint64_t q = (uint64_t)c0 + (uint64_t)G * ((uint64_t)c1 + (uint64_t)G * (uint64_t)c2);
                for (uint64_t v = P->start[q]; v < P->start[q + 1]; ++v)
                    if (v != u && within(P, u, v)) emit(ctx, u, v);
            }
        }
    }
}

typedef struct {
    uint64_t *u, *v, cap, count;
} list_ctx;

static void emit_list(void *p, uint64_t u, uint64_t v)
{
    list_ctx *L = (list_ctx *)p;
    if (L->count < L->cap) {
        L->u[L->count] = u;
        L->v[L->count] = v;
    }
    ++L->count;
}

int or_rgg_rows(int dim, uint64_t n, double r, uint64_t seed, uint64_t u_lo, uint64_t u_hi,
                uint64_t *u, uint64_t *v, uint64_t cap, uint64_t *count)
{
    rgg_points P;
    int rc = rgg_make(dim, n, r, seed, &P);
    if (rc) return rc;
    if (u_hi > n || u_lo > u_hi) {
        rgg_free(&P);
        return 1;
    }
    list_ctx L = {u, v, cap, 0};
    for (uint64_t a = u_lo; a < u_hi; ++a) rgg_row(&P, a, emit_list, &L);
    rgg_free(&P);
    *count = L.count;
    return L.count > cap ? 3 : 0;
}

int or_rgg(int dim, uint64_t n, double r, uint64_t seed, uint64_t *u, uint64_t *v, uint64_t cap,
           uint64_t *count)
{
    return or_rgg_rows(dim, n, r, seed, 0, n, u, v, cap, count);
}

/* SplitMix64 finaliser (Steele, Lea, Flood 2014), the edge digest's mixer. */
static uint64_t mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

typedef struct {
    uint64_t entries, digest, deg;
} digest_ctx;

static void emit_digest(void *p, uint64_t u, uint64_t v)
{
    digest_ctx *D = (digest_ctx *)p;
    ++D->entries;
    ++D->deg;
    D->digest += mix(u ^ ((v << 32) | (v >> 32)));
}

int or_rgg_digest(int dim, uint64_t n, double r, uint64_t seed, uint64_t *entries,
                  uint64_t *digest, uint64_t hist[65])
{
    rgg_points P;
    int rc = rgg_make(dim, n, r, seed, &P);
    if (rc) return rc;
    digest_ctx D = {0, 0, 0};
    for (int b = 0; b < 65; ++b) hist[b] = 0;
    for (uint64_t a = 0; a < n; ++a) {
        D.deg = 0;
        rgg_row(&P, a, emit_digest, &D);
        ++hist[D.deg < 64 ? D.deg : 64];
    }
    rgg_free(&P);
    *entries = D.entries;
    *digest = D.digest;
    return 0;
}
