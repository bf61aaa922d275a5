/*
 * Oracle: Erdos-Renyi generators (test infrastructure; see oracle.h).
 *
 * Directed G(n,m)   -- Sec. 4.1: P row chunks, chunk counts from a binary
 *                      split tree of hypergeometric variates (Sec. 2.2).
 * Undirected G(n,m) -- Sec. 4.2: triangular P x P chunk matrix, quadrant
 *                      recursion with split l = ceil(P/2); each off-diagonal
 *                      chunk is shared by two PEs and drawn from one seed.
 * G(n,p)            -- Sec. 4.3 with the geometric skips of Batagelj and
 *                      Brandes (Sec. 3.1): chunk streams keyed by chunk id.
 *
 * Inside a chunk the sample count is refined by a tile tree (the recursion
 * of Sec. 2.2 continued below the chunk) until a leaf holds about k_leaf
 * samples, which are then drawn without replacement by Floyd's algorithm
 * (Bentley and Floyd 1987; the sequential base case of Sec. 2.2).
 * Edges are produced chunk by chunk and sorted at the end.
 */
#include <stdlib.h>
#include <string.h>
#include "or_internal.h"

#define TAG_CHUNK_TREE 1u
#define TAG_QUAD 2u
#define TAG_TILE 3u
#define TAG_LEAF 4u
#define TAG_GNP 5u
#define TAG_GNP_COUNT 6u

/* ---------------- growable edge buffer ---------------- */

typedef struct {
    uint64_t u, v;
} edge;

typedef struct {
    edge *e;
    uint64_t n, cap;
    int oom;
} edge_buf;

static void eb_push(edge_buf *b, uint64_t u, uint64_t v)
{
    if (b->n == b->cap) {
        uint64_t nc = b->cap ? b->cap * 2 : 1024;
        edge *ne = (edge *)realloc(b->e, nc * sizeof(edge));
        if (!ne) {
            b->oom = 1;
            return;
        }
        b->e = ne;
        b->cap = nc;
    }
    b->e[b->n].u = u;
    b->e[b->n].v = v;
    b->n++;
}

static int edge_cmp(const void *a, const void *b)
{
    const edge *x = (const edge *)a, *y = (const edge *)b;
    if (x->u != y->u)
        return x->u < y->u ? -1 : 1;
    if (x->v != y->v)
        return x->v < y->v ? -1 : 1;
    return 0;
}

static int u64_cmp(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* Chunk boundary r_c = floor(c n / P)  ("sections of size roughly n/P", Sec. 4.2). */
static uint64_t row_bound(uint64_t n, uint32_t P, uint64_t c)
{
    return (uint64_t)(((u128)c * n) / P);
}

/* ---------------- Floyd leaf sampler ---------------- */

/* Lemire's bounded integer in [0, range): x*range as 128 bits, keep the high
 * word; reject when the low word falls below (2^64 - range) mod range.
 * Draw i takes u64 #i of the leaf stream; retry r >= 1 takes u64 #i of the
 * stream with tag TAG_LEAF | r << 8. */
static uint64_t leaf_draw(uint64_t seed, uint64_t node, uint64_t i, uint64_t range)
{
    uint64_t x = or_stream_u64(seed, node, TAG_LEAF, i);
    u128 prod = (u128)x * range;
    uint64_t lo = (uint64_t)prod;
    if (lo < range) {
        uint64_t thr = (0 - range) % range;
        uint32_t r = 1;
        while (lo < thr) {
            x = or_stream_u64(seed, node, TAG_LEAF | (r << 8), i);
            r++;
            prod = (u128)x * range;
            lo = (uint64_t)prod;
        }
    }
    return (uint64_t)(prod >> 64);
}

/* open-addressing set of u64 values */
typedef struct {
    uint64_t *slot;
    uint8_t *used;
    uint64_t mask;
} u64_set;

static int set_init(u64_set *s, uint64_t k)
{
    uint64_t cap = 16;
    while (cap < 2 * k + 2)
        cap <<= 1;
    s->slot = (uint64_t *)malloc(cap * sizeof(uint64_t));
    s->used = (uint8_t *)calloc(cap, 1);
    s->mask = cap - 1;
    return (s->slot && s->used) ? 0 : 1;
}

static void set_free(u64_set *s)
{
    free(s->slot);
    free(s->used);
}

/* returns 1 if x was inserted, 0 if already present */
static int set_insert(u64_set *s, uint64_t x)
{
    uint64_t h = (x * 0x9E3779B97F4A7C15ULL) >> 7;
    for (uint64_t i = h & s->mask;; i = (i + 1) & s->mask) {
        if (!s->used[i]) {
            s->used[i] = 1;
            s->slot[i] = x;
            return 1;
        }
        if (s->slot[i] == x)
            return 0;
    }
}

/* Floyd: for i = 0..k-1 with j = L-k+i, draw t uniform in [0, j]; insert t
 * unless present, else insert j.  Result: a uniform k-subset of [0, L). */
static int floyd_leaf(uint64_t L, uint64_t k, uint64_t seed, uint64_t node, uint64_t *out)
{
    if (k > L)
        return 1;
    if (k == 0)
        return 0;
    u64_set set;
    if (set_init(&set, k))
        return 1;
    uint64_t nout = 0;
    for (uint64_t i = 0; i < k; i++) {
        uint64_t j = L - k + i;
        uint64_t t = leaf_draw(seed, node, i, j + 1);
        if (set_insert(&set, t))
            out[nout++] = t;
        else {
            set_insert(&set, j);
            out[nout++] = j;
        }
    }
    set_free(&set);
    qsort(out, k, sizeof(uint64_t), u64_cmp);
    return 0;
}

int or_floyd_leaf(uint64_t L, uint64_t k, uint64_t seed, uint64_t node, uint64_t *out)
{
    return floyd_leaf(L, k, seed, node, out);
}

/* ---------------- tile tree inside one chunk ---------------- */

/* Depth d of the tile tree, one value for all chunks of an instance: the
 * smallest d with E <= k_leaf 2^d, where E = m (U_nom / N) is the expected
 * sample count of a chunk of the nominal (largest possible) universe U_nom.
 * It depends only on (n, m, P), not on sampled counts. */
static int tile_depth_e(double E, u128 Unom, uint32_t k_leaf, int *d_out)
{
    int d = 0;
    for (;;) {
        if (E <= (double)k_leaf * (double)((uint64_t)1 << d))
            break;
        if (((u128)2 << d) > Unom)
            break;
        if (d == OR_D_MAX)
            return 2;
        d++;
    }
    *d_out = d;
    return 0;
}

static int tile_depth(uint64_t m, u128 Unom, u128 Ntot, uint32_t k_leaf, int *d_out)
{
    double E = (double)m * (or_dbl128(Unom) / or_dbl128(Ntot));
    return tile_depth_e(E, Unom, k_leaf, d_out);
}

typedef struct {
    uint64_t seed;
    uint64_t chunk;  /* chunk id used in the node names */
    uint64_t Uc;     /* chunk universe */
    int d;           /* tile depth */
    uint64_t W;      /* tile width ceil(Uc / 2^d) */
    uint32_t k_max;
    uint64_t *offs;  /* output: sorted offsets */
    uint64_t noffs;
} tile_ctx;

/* Left end of node (level, j): min(j W 2^(d-level), Uc), for levels below d
 * with the floor of j W / 2^(level-d). */
static uint64_t node_bound(const tile_ctx *c, int level, u128 j)
{
    u128 x = j * (u128)c->W;
    if (level <= c->d)
        x <<= (c->d - level);
    else
        x >>= (level - c->d);
    return x < (u128)c->Uc ? (uint64_t)x : c->Uc;
}

static int tile_node(tile_ctx *c, int level, uint64_t j, uint64_t k)
{
    uint64_t lo = node_bound(c, level, j);
    uint64_t hi = node_bound(c, level, (u128)j + 1);
    uint64_t L = hi - lo;
    if (k > L)
        return 6;
    int split = level < c->d || (k > c->k_max && L >= 2);
    uint64_t heap = ((uint64_t)1 << level) + j;
    if (split) {
        if (level + 1 > OR_LEVEL_MAX)
            return 6;
        uint64_t mid = node_bound(c, level + 1, (u128)2 * j + 1);
        or_stream s = or_stream_make(c->seed, (c->chunk << 32) | heap, TAG_TILE);
        uint64_t X;
        int rc = or_hyper_s((u128)L, (u128)(mid - lo), k, &s, &X);
        if (rc)
            return rc;
        rc = tile_node(c, level + 1, 2 * j, X);
        if (rc)
            return rc;
        return tile_node(c, level + 1, 2 * j + 1, k - X);
    }
    if (k == 0)
        return 0;
    int rc = floyd_leaf(L, k, c->seed, (c->chunk << 32) | heap, c->offs + c->noffs);
    if (rc)
        return rc;
    for (uint64_t i = 0; i < k; i++)
        c->offs[c->noffs + i] += lo;
    c->noffs += k;
    return 0;
}

/* All k_c sorted offsets of one chunk with tile depth d. */
static int chunk_offsets(uint64_t seed, uint64_t chunk, uint64_t Uc, int d, uint32_t k_max,
                         uint64_t kc, uint64_t *offs)
{
    tile_ctx c;
    int rc;
    c.seed = seed;
    c.chunk = chunk;
    c.Uc = Uc;
    c.d = d;
    c.W = (uint64_t)(((u128)Uc + (((u128)1 << c.d) - 1)) >> c.d);
    c.k_max = k_max;
    c.offs = offs;
    c.noffs = 0;
    if (kc > Uc)
        return 1;
    rc = tile_node(&c, 0, 0, kc);
    if (rc)
        return rc;
    return c.noffs == kc ? 0 : 6;
}

/* ---------------- directed G(n,m), Sec. 4.1 ---------------- */

static int check_directed(uint64_t n, uint64_t m, uint32_t P)
{
    if (n == 0 || P == 0 || (uint64_t)P > n)
        return 1;
    u128 N = (u128)n * (n - 1);
    if ((u128)m > N)
        return 1;
    if (m > OR_M_MAX)
        return 2;
    /* the largest chunk universe must fit in 64 bits */
    uint64_t rows_max = (uint64_t)(((u128)n + P - 1) / P);
    if ((u128)rows_max * (n - 1) >> 64)
        return 2;
    return 0;
}

/* Chunk range [a,b) with heap index h receives mc samples; split at
 * s = a + ceil((b-a)/2) (l = ceil(P/2), Sec. 4.2) by a hypergeometric draw
 * over the row universes of the two halves. */
static int chunk_tree(uint64_t n, uint64_t seed, uint32_t P, uint64_t h, uint32_t a, uint32_t b,
                      uint64_t mc, uint64_t *cnt)
{
    if (b - a == 1) {
        cnt[a] = mc;
        return 0;
    }
    uint32_t s = a + (b - a + 1) / 2;
    u128 N = (u128)(row_bound(n, P, b) - row_bound(n, P, a)) * (n - 1);
    u128 NL = (u128)(row_bound(n, P, s) - row_bound(n, P, a)) * (n - 1);
    or_stream st = or_stream_make(seed, h, TAG_CHUNK_TREE);
    uint64_t X;
    int rc = or_hyper_s(N, NL, mc, &st, &X);
    if (rc)
        return rc;
    rc = chunk_tree(n, seed, P, 2 * h, a, s, X, cnt);
    if (rc)
        return rc;
    return chunk_tree(n, seed, P, 2 * h + 1, s, b, mc - X, cnt);
}

int or_gnm_directed_chunk_counts(uint64_t n, uint64_t m, uint64_t seed, uint32_t P, uint64_t *cnt)
{
    int rc = check_directed(n, m, P);
    if (rc)
        return rc;
    return chunk_tree(n, seed, P, 1, 0, P, m, cnt);
}

int or_gnm_directed_chunk(uint64_t n, uint64_t m, uint64_t seed, uint32_t P, uint32_t k_leaf,
                          uint32_t k_max, uint32_t c, uint64_t k_c, uint64_t *u, uint64_t *v)
{
    int rc = check_directed(n, m, P);
    if (rc)
        return rc;
    if (c >= P || k_leaf < 2 || k_max < k_leaf)
        return 1;
    u128 Ntot = (u128)n * (n - 1);
    u128 Unom = (((u128)n + P - 1) / P) * (n - 1);
    int d;
    rc = tile_depth(m, Unom, Ntot, k_leaf, &d);
    if (rc)
        return rc;
    uint64_t r0 = row_bound(n, P, c), r1 = row_bound(n, P, (uint64_t)c + 1);
    uint64_t Uc = (r1 - r0) * (n - 1);
    uint64_t *offs = (uint64_t *)malloc((k_c ? k_c : 1) * sizeof(uint64_t));
    if (!offs)
        return 1;
    rc = chunk_offsets(seed, c, Uc, d, k_max, k_c, offs);
    if (!rc) {
        /* offset -> (u, v): row u = r0 + off / (n-1), column w = off mod (n-1)
         * with the diagonal skipped (no self-loops, Sec. 2). */
        for (uint64_t i = 0; i < k_c; i++) {
            uint64_t uu = r0 + offs[i] / (n - 1);
            uint64_t w = offs[i] % (n - 1);
            u[i] = uu;
            v[i] = w + (w >= uu ? 1 : 0);
        }
    }
    free(offs);
    return rc;
}

int or_gnm_directed(uint64_t n, uint64_t m, uint64_t seed, uint32_t P, uint32_t k_leaf,
                    uint32_t k_max, uint64_t *u, uint64_t *v)
{
    int rc = check_directed(n, m, P);
    if (rc)
        return rc;
    uint64_t *cnt = (uint64_t *)malloc((uint64_t)P * sizeof(uint64_t));
    if (!cnt)
        return 1;
    rc = chunk_tree(n, seed, P, 1, 0, P, m, cnt);
    uint64_t pos = 0;
    for (uint32_t c = 0; !rc && c < P; c++) {
        rc = or_gnm_directed_chunk(n, m, seed, P, k_leaf, k_max, c, cnt[c], u + pos, v + pos);
        pos += cnt[c];
    }
    free(cnt);
    if (rc)
        return rc;
    /* sort the whole list by (u, v) */
    edge *e = (edge *)malloc((m ? m : 1) * sizeof(edge));
    if (!e)
        return 1;
    for (uint64_t i = 0; i < m; i++) {
        e[i].u = u[i];
        e[i].v = v[i];
    }
    qsort(e, m, sizeof(edge), edge_cmp);
    for (uint64_t i = 0; i < m; i++) {
        u[i] = e[i].u;
        v[i] = e[i].v;
    }
    free(e);
    return 0;
}

/* ---------------- undirected G(n,m), Sec. 4.2 ---------------- */

typedef struct {
    uint64_t n, seed;
    uint32_t P;
    uint64_t *cnt; /* P x P */
} quad_ctx;

static u128 tri_pairs(u128 S) { return S == 0 ? 0 : S * (S - 1) / 2; }

static uint64_t quad_node_id(uint32_t a, uint32_t b, uint32_t c, uint32_t d)
{
    return (uint64_t)a | ((uint64_t)(b - 1) << 16) | ((uint64_t)c << 32) | ((uint64_t)(d - 1) << 48);
}

static int quad_rect(quad_ctx *q, uint32_t a, uint32_t b, uint32_t c, uint32_t d, uint64_t mc);

/* Triangle of blocks [a,b): quadrants T1 = tri[a,a+l), R = rows [a+l,b) x
 * cols [a,a+l), T2 = tri[a+l,b), l = ceil((b-a)/2); two sequential
 * conditional hypergeometric draws give the counts of T1 and R. */
static int quad_tri(quad_ctx *q, uint32_t a, uint32_t b, uint64_t mc)
{
    if (b - a == 1) {
        q->cnt[(uint64_t)a * q->P + a] = mc;
        return 0;
    }
    uint32_t l = (b - a + 1) / 2;
    uint64_t ra = row_bound(q->n, q->P, a), rm = row_bound(q->n, q->P, a + l),
             rb = row_bound(q->n, q->P, b);
    u128 S1 = rm - ra, S2 = rb - rm;
    u128 T1 = tri_pairs(S1), R = S2 * S1, T2 = tri_pairs(S2);
    u128 N = T1 + R + T2;
    or_stream st = or_stream_make(q->seed, quad_node_id(a, b, a, b), TAG_QUAD);
    uint64_t X1, X2;
    int rc = or_hyper_s(N, T1, mc, &st, &X1);
    if (rc)
        return rc;
    rc = or_hyper_s(N - T1, R, mc - X1, &st, &X2);
    if (rc)
        return rc;
    rc = quad_tri(q, a, a + l, X1);
    if (rc)
        return rc;
    rc = quad_rect(q, a + l, b, a, a + l, X2);
    if (rc)
        return rc;
    return quad_tri(q, a + l, b, mc - X1 - X2);
}

/* Rectangle rows [a,b) x cols [c,d): each dimension with more than one block
 * is halved at ceil; the (up to four) parts are taken in row-major order and
 * all but the last get sequential conditional hypergeometric counts. */
static int quad_rect(quad_ctx *q, uint32_t a, uint32_t b, uint32_t c, uint32_t d, uint64_t mc)
{
    if (b - a == 1 && d - c == 1) {
        q->cnt[(uint64_t)a * q->P + c] = mc;
        return 0;
    }
    uint32_t rlo[2], rhi[2], clo[2], chi[2];
    int nr = 1, nc = 1;
    rlo[0] = a; rhi[0] = b;
    if (b - a >= 2) {
        uint32_t s = a + (b - a + 1) / 2;
        rhi[0] = s; rlo[1] = s; rhi[1] = b; nr = 2;
    }
    clo[0] = c; chi[0] = d;
    if (d - c >= 2) {
        uint32_t s = c + (d - c + 1) / 2;
        chi[0] = s; clo[1] = s; chi[1] = d; nc = 2;
    }
    u128 size[4];
    uint32_t pa[4], pb[4], pc[4], pd[4];
    int np = 0;
    for (int i = 0; i < nr; i++)
        for (int j = 0; j < nc; j++) {
            pa[np] = rlo[i]; pb[np] = rhi[i]; pc[np] = clo[j]; pd[np] = chi[j];
            size[np] = (u128)(row_bound(q->n, q->P, rhi[i]) - row_bound(q->n, q->P, rlo[i])) *
                       (row_bound(q->n, q->P, chi[j]) - row_bound(q->n, q->P, clo[j]));
            np++;
        }
    u128 N = 0;
    for (int i = 0; i < np; i++)
        N += size[i];
    or_stream st = or_stream_make(q->seed, quad_node_id(a, b, c, d), TAG_QUAD);
    uint64_t part[4];
    uint64_t rem = mc;
    for (int i = 0; i < np - 1; i++) {
        int rc = or_hyper_s(N, size[i], rem, &st, &part[i]);
        if (rc)
            return rc;
        N -= size[i];
        rem -= part[i];
    }
    part[np - 1] = rem;
    for (int i = 0; i < np; i++) {
        int rc = quad_rect(q, pa[i], pb[i], pc[i], pd[i], part[i]);
        if (rc)
            return rc;
    }
    return 0;
}

static int check_undirected(uint64_t n, uint64_t m, uint32_t P)
{
    if (n == 0 || P == 0 || (uint64_t)P > n || P > 65536)
        return 1;
    u128 N = tri_pairs(n);
    if ((u128)m > N)
        return 1;
    if (m > OR_M_MAX)
        return 2;
    uint64_t rows_max = (uint64_t)(((u128)n + P - 1) / P);
    if (((u128)rows_max * rows_max) >> 64)
        return 2;
    return 0;
}

int or_gnm_undirected_chunk_counts(uint64_t n, uint64_t m, uint64_t seed, uint32_t P, uint64_t *cnt)
{
    int rc = check_undirected(n, m, P);
    if (rc)
        return rc;
    memset(cnt, 0, (uint64_t)P * P * sizeof(uint64_t));
    quad_ctx q = {n, seed, P, cnt};
    return quad_tri(&q, 0, P, m);
}

/* Universe size of chunk (i, j), j <= i. */
static uint64_t und_chunk_universe(uint64_t n, uint32_t P, uint32_t i, uint32_t j)
{
    uint64_t si = row_bound(n, P, (uint64_t)i + 1) - row_bound(n, P, i);
    if (i == j)
        return (uint64_t)tri_pairs(si);
    uint64_t sj = row_bound(n, P, (uint64_t)j + 1) - row_bound(n, P, j);
    return si * sj;
}

/* In-chunk offset -> pair (u > v).  Rectangle: row-major.  Triangle:
 * off = w(w-1)/2 + x with 0 <= x < w; w found by binary search. */
static void und_map(uint64_t n, uint32_t P, uint32_t i, uint32_t j, uint64_t off, uint64_t *u,
                    uint64_t *v)
{
    uint64_t ri = row_bound(n, P, i);
    if (i != j) {
        uint64_t rj = row_bound(n, P, j);
        uint64_t sj = row_bound(n, P, (uint64_t)j + 1) - rj;
        *u = ri + off / sj;
        *v = rj + off % sj;
        return;
    }
    uint64_t lo = 1, hi = row_bound(n, P, (uint64_t)i + 1) - ri; /* w in [1, s_i) */
    while (hi - lo > 1) {
        uint64_t mid = lo + (hi - lo) / 2;
        if ((u128)mid * (mid - 1) / 2 <= (u128)off)
            lo = mid;
        else
            hi = mid;
    }
    *u = ri + lo;
    *v = ri + (off - (uint64_t)((u128)lo * (lo - 1) / 2));
}

static int finish_sorted(edge_buf *b, uint64_t *u, uint64_t *v, uint64_t cap, uint64_t *count)
{
    if (b->oom)
        return 1;
    qsort(b->e, b->n, sizeof(edge), edge_cmp);
    if (count)
        *count = b->n;
    if (b->n > cap)
        return 3;
    for (uint64_t i = 0; i < b->n; i++) {
        u[i] = b->e[i].u;
        v[i] = b->e[i].v;
    }
    return 0;
}

int or_gnm_undirected(uint64_t n, uint64_t m, uint64_t seed, uint32_t P, uint32_t k_leaf,
                      uint32_t k_max, uint64_t *u, uint64_t *v)
{
    int rc = check_undirected(n, m, P);
    if (rc)
        return rc;
    if (k_leaf < 2 || k_max < k_leaf)
        return 1;
    uint64_t *cnt = (uint64_t *)malloc((uint64_t)P * P * sizeof(uint64_t));
    if (!cnt)
        return 1;
    rc = or_gnm_undirected_chunk_counts(n, m, seed, P, cnt);
    u128 Ntot = tri_pairs(n);
    u128 rmax = ((u128)n + P - 1) / P;
    int d = 0;
    if (!rc)
        rc = tile_depth(m, rmax * rmax, Ntot, k_leaf, &d);
    edge_buf b = {0, 0, 0, 0};
    for (uint32_t i = 0; !rc && i < P; i++)
        for (uint32_t j = 0; !rc && j <= i; j++) {
            uint64_t kc = cnt[(uint64_t)i * P + j];
            uint64_t Uc = und_chunk_universe(n, P, i, j);
            uint64_t *offs = (uint64_t *)malloc((kc ? kc : 1) * sizeof(uint64_t));
            if (!offs) {
                rc = 1;
                break;
            }
            rc = chunk_offsets(seed, (uint64_t)i * P + j, Uc, d, k_max, kc, offs);
            for (uint64_t t = 0; !rc && t < kc; t++) {
                uint64_t uu, vv;
                und_map(n, P, i, j, offs[t], &uu, &vv);
                eb_push(&b, uu, vv);
                eb_push(&b, vv, uu);
            }
            free(offs);
        }
    free(cnt);
    if (!rc)
        rc = finish_sorted(&b, u, v, 2 * m, NULL);
    free(b.e);
    return rc;
}

/* Rows of the row blocks [b0, b1) of the undirected graph, both directions,
 * sorted by (u, v): the entries (u, v) of the chunks (i, j <= i) of those row
 * blocks, and the mirrored entries (v, u) of the chunks (i >= j, j) of those
 * column blocks -- the chunks a PE of Sec. 4.2 regenerates from their shared
 * seeds.  Concatenated over all blocks this is or_gnm_undirected's list. */
int or_gnm_undirected_rows(uint64_t n, uint64_t m, uint64_t seed, uint32_t P, uint32_t k_leaf,
                           uint32_t k_max, uint32_t b0, uint32_t b1, uint64_t *u, uint64_t *v,
                           uint64_t cap, uint64_t *count)
{
    int rc = check_undirected(n, m, P);
    if (rc)
        return rc;
    if (k_leaf < 2 || k_max < k_leaf || b0 >= b1 || b1 > P)
        return 1;
    uint64_t *cnt = (uint64_t *)malloc((uint64_t)P * P * sizeof(uint64_t));
    if (!cnt)
        return 1;
    rc = or_gnm_undirected_chunk_counts(n, m, seed, P, cnt);
    u128 rmax = ((u128)n + P - 1) / P;
    int d = 0;
    if (!rc)
        rc = tile_depth(m, rmax * rmax, tri_pairs(n), k_leaf, &d);
    uint64_t lo = row_bound(n, P, b0), hi = row_bound(n, P, b1);
    edge_buf b = {0, 0, 0, 0};
    for (uint32_t i = 0; !rc && i < P; i++)
        for (uint32_t j = 0; !rc && j <= i; j++) {
            if (!((i >= b0 && i < b1) || (j >= b0 && j < b1)))
                continue;
            uint64_t kc = cnt[(uint64_t)i * P + j];
            uint64_t *offs = (uint64_t *)malloc((kc ? kc : 1) * sizeof(uint64_t));
            if (!offs) {
                rc = 1;
                break;
            }
            rc = chunk_offsets(seed, (uint64_t)i * P + j, und_chunk_universe(n, P, i, j), d, k_max,
                               kc, offs);
            for (uint64_t t = 0; !rc && t < kc; t++) {
                uint64_t uu, vv;
                und_map(n, P, i, j, offs[t], &uu, &vv);
                if (uu >= lo && uu < hi)
                    eb_push(&b, uu, vv);
                if (vv >= lo && vv < hi)
                    eb_push(&b, vv, uu);
            }
            free(offs);
        }
    free(cnt);
    if (!rc)
        rc = finish_sorted(&b, u, v, cap, count);
    free(b.e);
    return rc;
}

/* ---------------- G(n,p), Sec. 4.3 ---------------- */

/* Tile length T = the largest power of two <= max(1, k_leaf / p), capped at 2^62. */
static uint64_t gnp_tile_len(double p, uint32_t k_leaf)
{
    double q = (double)k_leaf / p;
    if (!(q >= 2.0))
        return 1;
    uint64_t T = 1;
    while (T < ((uint64_t)1 << 62) && (double)(T * 2) <= q)
        T *= 2;
    return T;
}

/* growable array of u64 offsets */
typedef struct {
    uint64_t *a;
    uint64_t n, cap;
    int oom;
} u64_buf;

static void ub_push(u64_buf *b, uint64_t x)
{
    if (b->n == b->cap) {
        uint64_t nc = b->cap ? b->cap * 2 : 1024;
        uint64_t *na = (uint64_t *)realloc(b->a, nc * sizeof(uint64_t));
        if (!na) {
            b->oom = 1;
            return;
        }
        b->a = na;
        b->cap = nc;
    }
    b->a[b->n++] = x;
}

/* Geometric skips in one tile [lo, hi): the next candidate x is kept after
 * g = floor(ln U * (1 / ln(1-p))) rejected candidates, U uniform in (0,1]. */
static void gnp_tile(uint64_t seed, uint64_t node, uint64_t lo, uint64_t hi, double inv_lq,
                     u64_buf *out)
{
    or_stream s = or_stream_make(seed, node, TAG_GNP);
    uint64_t x = lo;
    for (;;) {
        double U = or_u01_open0(or_next_u64(&s));
        double g = __builtin_floor(or_log(U) * inv_lq);
        if (g >= (double)(hi - x))
            break;
        x += (uint64_t)g;
        ub_push(out, x);
        x += 1;
        if (x >= hi)
            break;
    }
}

/* Offsets of one G(n,p) chunk (all pairs when p = 1). */
static int gnp_chunk(uint64_t seed, uint64_t chunk, uint64_t Uc, double p, uint32_t k_leaf,
                     double inv_lq, uint64_t **offs, uint64_t *k)
{
    *k = 0;
    *offs = NULL;
    if (p <= 0.0 || Uc == 0)
        return 0;
    u64_buf b = {0, 0, 0, 0};
    if (p >= 1.0) {
        for (uint64_t i = 0; i < Uc; i++)
            ub_push(&b, i);
    } else {
        uint64_t T = gnp_tile_len(p, k_leaf);
        uint64_t ntiles = Uc / T + (Uc % T ? 1 : 0);
        if (ntiles > ((uint64_t)1 << 32))
            return 2;
        for (uint64_t t = 0; t < ntiles && !b.oom; t++) {
            uint64_t lo = t * T, hi = (Uc - lo > T) ? lo + T : Uc;
            gnp_tile(seed, (chunk << 32) | t, lo, hi, inv_lq, &b);
        }
    }
    if (b.oom) {
        free(b.a);
        return 1;
    }
    *offs = b.a;
    *k = b.n;
    return 0;
}

int or_gnp(int undirected, uint64_t n, double p, uint64_t seed, uint32_t P, uint32_t k_leaf,
           uint64_t *u, uint64_t *v, uint64_t cap, uint64_t *count)
{
    if (!(p >= 0.0 && p <= 1.0) || k_leaf < 2)
        return 1;
    int rc = undirected ? check_undirected(n, 0, P) : check_directed(n, 0, P);
    if (rc)
        return rc;
    double inv_lq = (p > 0.0 && p < 1.0) ? 1.0 / or_log1m(p) : 0.0;
    edge_buf b = {0, 0, 0, 0};
    if (!undirected) {
        for (uint32_t c = 0; !rc && c < P; c++) {
            uint64_t r0 = row_bound(n, P, c), r1 = row_bound(n, P, (uint64_t)c + 1);
            uint64_t Uc = (r1 - r0) * (n - 1);
            uint64_t *offs = NULL, k = 0;
            rc = gnp_chunk(seed, c, Uc, p, k_leaf, inv_lq, &offs, &k);
            for (uint64_t i = 0; !rc && i < k; i++) {
                uint64_t uu = r0 + offs[i] / (n - 1), w = offs[i] % (n - 1);
                eb_push(&b, uu, w + (w >= uu ? 1 : 0));
            }
            free(offs);
        }
    } else {
        for (uint32_t i = 0; !rc && i < P; i++)
            for (uint32_t j = 0; !rc && j <= i; j++) {
                uint64_t Uc = und_chunk_universe(n, P, i, j);
                uint64_t *offs = NULL, k = 0;
                rc = gnp_chunk(seed, (uint64_t)i * P + j, Uc, p, k_leaf, inv_lq, &offs, &k);
                for (uint64_t t = 0; !rc && t < k; t++) {
                    uint64_t uu, vv;
                    und_map(n, P, i, j, offs[t], &uu, &vv);
                    eb_push(&b, uu, vv);
                    eb_push(&b, vv, uu);
                }
                free(offs);
            }
    }
    if (!rc)
        rc = finish_sorted(&b, u, v, cap, count);
    free(b.e);
    return rc;
}

/* ---------------- G(n,p) by binomial chunk counts, Sec. 4.3 ---------------- */

/* Sec. 4.3: the sample count of every chunk is a binomial variate drawn from
 * a stream keyed by the chunk id, so that every PE needing the count draws
 * the same value; the chunk is then sampled exactly like a G(n,m) chunk
 * (tile tree + Floyd), with one tile depth per instance from the expected
 * count p U_nom of the nominal chunk.  Chunks: directed c = 0..P-1 (stream id
 * c); undirected (i, j), j <= i, in the order k = i(i+1)/2 + j (stream id
 * i P + j).  Chunk universes are limited to 2^53 pairs. */
static int gnp_binomial_check(int undirected, uint64_t n, double p, uint32_t P)
{
    if (!(p >= 0.0 && p <= 1.0))
        return 1;
    int rc = undirected ? check_undirected(n, 0, P) : check_directed(n, 0, P);
    if (rc)
        return rc;
    u128 rmax = ((u128)n + P - 1) / P;
    u128 Unom = undirected ? rmax * rmax : rmax * (n - 1);
    return Unom > (u128)OR_BINOM_N_MAX ? 2 : 0;
}

int or_gnp_binomial_counts(int undirected, uint64_t n, double p, uint64_t seed, uint32_t P,
                           uint64_t *cnt)
{
    int rc = gnp_binomial_check(undirected, n, p, P);
    if (rc)
        return rc;
    uint64_t k = 0;
    for (uint32_t i = 0; !rc && i < P; i++) {
        if (!undirected) {
            uint64_t Uc = (row_bound(n, P, (uint64_t)i + 1) - row_bound(n, P, i)) * (n - 1);
            or_stream s = or_stream_make(seed, i, TAG_GNP_COUNT);
            rc = or_binom_big(Uc, p, &s, &cnt[i]);
            continue;
        }
        for (uint32_t j = 0; !rc && j <= i; j++, k++) {
            or_stream s = or_stream_make(seed, (uint64_t)i * P + j, TAG_GNP_COUNT);
            rc = or_binom_big(und_chunk_universe(n, P, i, j), p, &s, &cnt[k]);
        }
    }
    return rc;
}

int or_gnp_binomial(int undirected, uint64_t n, double p, uint64_t seed, uint32_t P,
                    uint32_t k_leaf, uint32_t k_max, uint64_t *u, uint64_t *v, uint64_t cap,
                    uint64_t *count)
{
    if (k_leaf < 2 || k_max < k_leaf)
        return 1;
    int rc = gnp_binomial_check(undirected, n, p, P);
    if (rc)
        return rc;
    uint64_t C = undirected ? (uint64_t)P * (P + 1) / 2 : P;
    uint64_t *cnt = (uint64_t *)malloc(C * sizeof(uint64_t));
    if (!cnt)
        return 1;
    rc = or_gnp_binomial_counts(undirected, n, p, seed, P, cnt);
    u128 rmax = ((u128)n + P - 1) / P;
    u128 Unom = undirected ? rmax * rmax : rmax * (n - 1);
    int d = 0;
    if (!rc)
        rc = tile_depth_e(p * or_dbl128(Unom), Unom, k_leaf, &d);
    edge_buf b = {0, 0, 0, 0};
    uint64_t k = 0;
    for (uint32_t i = 0; !rc && i < P; i++)
        for (uint32_t j = 0; !rc && j <= (undirected ? i : 0); j++, k++) {
            uint64_t kc = cnt[k];
            uint64_t cid = undirected ? (uint64_t)i * P + j : i;
            uint64_t r0 = row_bound(n, P, i);
            uint64_t Uc = undirected ? und_chunk_universe(n, P, i, j)
                                     : (row_bound(n, P, (uint64_t)i + 1) - r0) * (n - 1);
            uint64_t *offs = (uint64_t *)malloc((kc ? kc : 1) * sizeof(uint64_t));
            if (!offs) {
                rc = 1;
                break;
            }
            rc = chunk_offsets(seed, cid, Uc, d, k_max, kc, offs);
            for (uint64_t t = 0; !rc && t < kc; t++) {
                if (undirected) {
                    uint64_t uu, vv;
                    und_map(n, P, i, j, offs[t], &uu, &vv);
                    eb_push(&b, uu, vv);
                    eb_push(&b, vv, uu);
                } else {
                    uint64_t uu = r0 + offs[t] / (n - 1), w = offs[t] % (n - 1);
                    eb_push(&b, uu, w + (w >= uu ? 1 : 0));
                }
            }
            free(offs);
        }
    free(cnt);
    if (!rc)
        rc = finish_sorted(&b, u, v, cap, count);
    free(b.e);
    return rc;
}

/* ---------------- digests ---------------- */

/* SplitMix64 output finaliser (Steele, Lea, Flood, OOPSLA 2014). */
static uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* sum over edges of mix64(u xor rotl(v, 32)) mod 2^64: independent of order */
uint64_t or_edge_checksum(const uint64_t *u, const uint64_t *v, uint64_t count)
{
    uint64_t sum = 0;
    for (uint64_t i = 0; i < count; i++) {
        uint64_t rv = (v[i] << 32) | (v[i] >> 32);
        sum += mix64(u[i] ^ rv);
    }
    return sum;
}

int or_outdegree_hist(const uint64_t *u, uint64_t count, uint64_t row_lo, uint64_t row_hi,
                      uint64_t hist[65])
{
    for (int i = 0; i < 65; i++)
        hist[i] = 0;
    uint64_t i = 0;
    uint64_t seen_rows = 0;
    while (i < count) {
        uint64_t x = u[i], j = i;
        if (x < row_lo || x >= row_hi)
            return 1;
        while (j < count && u[j] == x)
            j++;
        uint64_t d = j - i;
        hist[d < 64 ? d : 64]++;
        seen_rows++;
        i = j;
    }
    hist[0] += (row_hi - row_lo) - seen_rows;
    return 0;
}
