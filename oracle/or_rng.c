/*
 * Oracle: pseudorandomisation (test infrastructure; see oracle.h).
 *
 * Sec. 2.2 of the paper derives, for every subtree of the sampling recursion,
 * a seed from (global seed, subtree id) and feeds it to a PRNG, so that all
 * PEs that visit the subtree draw identical variates.  Here the same property
 * comes from the counter-based generator Philox4x32-10 (Salmon, Moraes, Dror,
 * Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC 2011): the key is
 * the global seed and the counter names (node, tag, block).
 */
#include "or_internal.h"

/* Philox4x32 constants as published by Salmon et al. (SC 2011). */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

/* Ten rounds of the Philox4x32 S-P network.  In every round the words 0 and 2
 * are multiplied by M0 and M1; the high halves are mixed with the key and
 * the other two words, the low halves pass through; the key is bumped by the
 * Weyl constants between rounds. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        uint64_t p0 = (uint64_t)PHILOX_M0 * x0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

or_stream or_stream_make(uint64_t seed, uint64_t node, uint32_t tag)
{
    or_stream s;
    s.seed = seed;
    s.node = node;
    s.tag = tag;
    s.next = 0;
    return s;
}

/* u64 number `index` of a stream: block index>>1 of Philox, first or second
 * half (words w0,w1 or w2,w3), each half read as (wA << 32) | wB. */
uint64_t or_stream_u64(uint64_t seed, uint64_t node, uint32_t tag, uint64_t index)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)(index >> 1), (uint32_t)node, (uint32_t)(node >> 32), tag};
    uint32_t w[4];
    or_philox4x32_10(ctr, key, w);
    if ((index & 1) == 0)
        return ((uint64_t)w[0] << 32) | w[1];
    return ((uint64_t)w[2] << 32) | w[3];
}

uint64_t or_next_u64(or_stream *s)
{
    uint64_t x = or_stream_u64(s->seed, s->node, s->tag, s->next);
    s->next++;
    return x;
}

/* 2^-53 as an exact double */
#define TWO_M53 (1.0 / 9007199254740992.0)

double or_u01_open0(uint64_t x) { return (double)((x >> 11) + 1) * TWO_M53; }
double or_u01_open1(uint64_t x) { return (double)(x >> 11) * TWO_M53; }

/* Correctly rounded (nearest-even) conversion; the C conversion of an
 * unsigned __int128 rounds to nearest under the default rounding mode. */
double or_dbl128(u128 x) { return (double)x; }

double or_u128_to_double(uint64_t lo, uint64_t hi)
{
    return or_dbl128(((u128)hi << 64) | lo);
}
