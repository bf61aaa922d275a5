/*
 * Oracle for the communication-free Erdos-Renyi generators of
 * "Communication-free Massively Distributed Graph Generation"
 * (Funke, Lamm, Meyer, Penschuck, Sanders, Schulz, Strash, von Looz).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, single-threaded C
 * restatement of the sampling procedure (Sec. 2.2 divide-and-conquer
 * sampling, Sec. 4.1 directed G(n,m), Sec. 4.2 undirected G(n,m),
 * Sec. 4.3 G(n,p)).  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header or
 * table with the CUDA library; both implement the same written procedure
 * independently, so equal outputs are evidence that both follow it.
 *
 * Integer widths: universe sizes can exceed 2^64 (n(n-1) with n = 2^36), so
 * 128-bit quantities are passed as (lo, hi) pairs of uint64.
 *
 * Return codes: 0 = ok, 1 = bad argument, 2 = out of the supported range,
 * 3 = output buffer too small (the required size is still reported),
 * 6 = internal limit reached (rejection loop cap; never expected).
 */
#ifndef KG_ORACLE_H
#define KG_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- building blocks, exported for the pin tests ---- */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
uint64_t or_stream_u64(uint64_t seed, uint64_t node, uint32_t tag, uint64_t index);
double or_log(double x);
double or_log1m(double p);
double or_exp(double x);
double or_lnfact(double k);
double or_lnfact_diff(double a, double d);
double or_u128_to_double(uint64_t lo, uint64_t hi);

/* One variate drawn from the stream (seed, node, tag), starting at u64 #0. */
int or_hypergeometric(uint64_t N_lo, uint64_t N_hi, uint64_t K_lo, uint64_t K_hi,
                      uint64_t t, uint64_t seed, uint64_t node, uint32_t tag,
                      uint64_t *x);
int or_binomial(uint64_t n, double p, uint64_t seed, uint64_t node, uint32_t tag,
                uint64_t *x);
/* Leaf sampler: k distinct sorted offsets in [0, L) (Floyd's algorithm). */
int or_floyd_leaf(uint64_t L, uint64_t k, uint64_t seed, uint64_t node, uint64_t *out);

/* ---- directed G(n,m), Sec. 4.1 ---- */
int or_gnm_directed_chunk_counts(uint64_t n, uint64_t m, uint64_t seed, uint32_t P,
                                 uint64_t *cnt);
int or_gnm_directed_chunk(uint64_t n, uint64_t m, uint64_t seed, uint32_t P,
                          uint32_t k_leaf, uint32_t k_max, uint32_t c, uint64_t k_c,
                          uint64_t *u, uint64_t *v);
int or_gnm_directed(uint64_t n, uint64_t m, uint64_t seed, uint32_t P,
                    uint32_t k_leaf, uint32_t k_max, uint64_t *u, uint64_t *v);

/* ---- undirected G(n,m), Sec. 4.2 (writes 2m entries, both directions) ---- */
int or_gnm_undirected_chunk_counts(uint64_t n, uint64_t m, uint64_t seed, uint32_t P,
                                   uint64_t *cnt /* P*P, row-major, j<=i used */);
int or_gnm_undirected(uint64_t n, uint64_t m, uint64_t seed, uint32_t P,
                      uint32_t k_leaf, uint32_t k_max, uint64_t *u, uint64_t *v);

/* the rows of row blocks [b0, b1) of the same undirected graph (both directions),
 * from the chunks of those row and column blocks (Sec. 4.2); *count = entries */
int or_gnm_undirected_rows(uint64_t n, uint64_t m, uint64_t seed, uint32_t P, uint32_t k_leaf,
                           uint32_t k_max, uint32_t b0, uint32_t b1, uint64_t *u, uint64_t *v,
                           uint64_t cap, uint64_t *count);

/* ---- G(n,p), Sec. 4.3 (geometric skips); *count = number of entries ---- */
int or_gnp(int undirected, uint64_t n, double p, uint64_t seed, uint32_t P,
           uint32_t k_leaf, uint64_t *u, uint64_t *v, uint64_t cap, uint64_t *count);

/* ---- G(n,p) by binomial chunk counts + the G(n,m) sampler, Sec. 4.3 ---- */
/* cnt: P (directed) or P(P+1)/2 (undirected, order k = i(i+1)/2 + j) counts */
int or_gnp_binomial_counts(int undirected, uint64_t n, double p, uint64_t seed, uint32_t P,
                           uint64_t *cnt);
int or_gnp_binomial(int undirected, uint64_t n, double p, uint64_t seed, uint32_t P,
                    uint32_t k_leaf, uint32_t k_max, uint64_t *u, uint64_t *v, uint64_t cap,
                    uint64_t *count);

/* ---- random geometric graph RGG(n, r), d = 2 or 3, Sec. 5 (see or_rgg.c) ---- */
/* g: the grid has 2^g cells per dimension */
int or_rgg_grid_level(int dim, uint64_t n, double r, int *g);
/* points per cell, cells in row-major order (dimension 0 fastest), 2^(dim g) entries */
int or_rgg_cell_counts(int dim, uint64_t n, double r, uint64_t seed, uint64_t *cnt);
/* fixed-point coordinates (x 2^-32), n x dim, vertex-major */
int or_rgg_points(int dim, uint64_t n, double r, uint64_t seed, uint32_t *coords);
/* all entries (both directions), sorted by (u, v); *count = entries */
int or_rgg(int dim, uint64_t n, double r, uint64_t seed, uint64_t *u, uint64_t *v, uint64_t cap,
           uint64_t *count);
/* the rows of vertices [u_lo, u_hi) */
int or_rgg_rows(int dim, uint64_t n, double r, uint64_t seed, uint64_t u_lo, uint64_t u_hi,
                uint64_t *u, uint64_t *v, uint64_t cap, uint64_t *count);
/* entry count, digest (as or_edge_checksum) and degree histogram, without storing edges */
int or_rgg_digest(int dim, uint64_t n, double r, uint64_t seed, uint64_t *entries,
                  uint64_t *digest, uint64_t hist[65]);

/* ---- order-independent edge-list digest ---- */
uint64_t or_edge_checksum(const uint64_t *u, const uint64_t *v, uint64_t count);
/* out-degree histogram over vertices [row_lo, row_hi): hist[d] for d<64, hist[64] for d>=64.
 * The edge list must be sorted by u and lie inside the row range. */
int or_outdegree_hist(const uint64_t *u, uint64_t count, uint64_t row_lo, uint64_t row_hi,
                      uint64_t hist[65]);

#ifdef __cplusplus
}
#endif
#endif
