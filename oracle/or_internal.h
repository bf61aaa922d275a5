/* Oracle internals (test infrastructure; see oracle.h). */
#ifndef KG_OR_INTERNAL_H
#define KG_OR_INTERNAL_H
#include <stdint.h>
#include "oracle.h"

typedef unsigned __int128 u128;

/* A node's random word stream: Philox4x32-10 keyed by the global seed,
 * counter = (block, lo32(node), hi32(node), tag).  This replaces the paper's
 * "hash of (seed, subtree id) seeds a PRNG" (Sec. 2.2) by a counter-based
 * generator, so every node draws the same numbers wherever it is evaluated. */
typedef struct {
    uint64_t seed;
    uint64_t node;
    uint32_t tag;
    uint64_t next; /* index of the next u64 to hand out */
} or_stream;

or_stream or_stream_make(uint64_t seed, uint64_t node, uint32_t tag);
uint64_t or_next_u64(or_stream *s);
double or_u01_open0(uint64_t x);   /* ((x>>11)+1) * 2^-53, in (0,1] */
double or_u01_open1(uint64_t x);   /* (x>>11) * 2^-53, in [0,1) */
double or_dbl128(u128 x);          /* round-to-nearest-even conversion */

/* variates: all consume the stream in order */
int or_hyper_s(u128 N, u128 K, uint64_t t, or_stream *s, uint64_t *x);
int or_binom_s(uint64_t n, double p, or_stream *s, uint64_t *x);
int or_binom_big(uint64_t n, double p, or_stream *s, uint64_t *x);

/* limits of the procedure */
#define OR_M_MAX ((uint64_t)1 << 44)  /* largest m (and binomial n) accepted */
#define OR_BINOM_N_MAX ((uint64_t)1 << 53) /* largest binomial n for G(n,p) chunk counts */
#define OR_D_MAX 24                     /* largest tile-tree depth */
#define OR_LEVEL_MAX 31                 /* tile heap index must stay below 2^32 */
#define OR_REJECT_CAP 1000000           /* rejection/restart loop cap */

#endif
