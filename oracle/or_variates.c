/*
 * Oracle: non-uniform variates (test infrastructure; see oracle.h).
 *
 * Sec. 2.2: the divide-and-conquer sampler needs hypergeometric variates
 * (the number of samples that fall into one half of a universe, drawn without
 * replacement) and the G(n,p) adaptation of Sec. 4.3 needs binomial counts;
 * both are generated by acceptance-rejection in expected O(1) time.  The
 * rejection method used here is Stadlober's ratio-of-uniforms with the
 * table-mountain hat (Stadlober 1989/1990, the method the paper cites): a
 * point (X, V) uniform in (0,1] x [-s/2, s/2) gives W = a + V/X, which is
 * accepted with k = floor(W) when X^2 <= f(k)/f(mode).  Small means use
 * sequential inversion from the bottom of the support.
 *
 * All arithmetic is FP64 in the order written, using only the functions of
 * or_math.c.
 */
#include "or_internal.h"

/* Hat constants 2 sqrt(2/e) and 3 - 2 sqrt(3/e). */
#define RoU_D1 0x1.b72cd3f331398p+0
#define RoU_D2 0x1.cc3ebd3bc711ap-1

static double dmin(double a, double b) { return a < b ? a : b; }

/* ---------------- binomial ---------------- */

/* Inversion from 0 for n p < 10 (p <= 1/2):
 * f(0) = exp(n ln(1-p)), f(x+1) = f(x) * r * (n - x) / (x + 1), r = p/(1-p). */
static int binom_inversion(uint64_t n, double p, or_stream *s, uint64_t *out)
{
    double nd = (double)n;
    double q = 1.0 - p;
    double r = p / q;
    double f0 = or_exp(nd * or_log1m(p));
    for (int attempt = 0; attempt < OR_REJECT_CAP; attempt++) {
        double U = or_u01_open1(or_next_u64(s));
        uint64_t x = 0;
        double f = f0;
        for (;;) {
            if (U < f) {
                *out = x;
                return 0;
            }
            U = U - f;
            double xd = (double)x;
            f = ((f * r) * (nd - xd)) / (xd + 1.0);
            x = x + 1;
            if (x > n || f == 0.0)
                break; /* ran off the support through rounding: new uniform */
        }
    }
    return 6;
}

/* Ratio of uniforms for n p >= 10 (p <= 1/2). */
static int binom_rou(uint64_t n, double p, or_stream *s, uint64_t *out)
{
    double nd = (double)n;
    double q = 1.0 - p;
    double mean = nd * p;
    double var = mean * q;
    double M = __builtin_floor((nd + 1.0) * p);
    double a = mean + 0.5;
    double sw = RoU_D1 * __builtin_sqrt(var + 0.5) + RoU_D2;
    double lpq = or_log(p) - or_log1m(p);
    for (int it = 0; it < OR_REJECT_CAP; it++) {
        double X = or_u01_open0(or_next_u64(s));
        double Y = or_u01_open1(or_next_u64(s));
        double W = a + (sw * (Y - 0.5)) / X;
        if (W < 0.0 || W >= nd + 1.0)
            continue;
        double k = __builtin_floor(W);
        /* ln f(k) - ln f(M) = (k-M) ln(p/q) - [ln k! - ln M!] - [ln (n-k)! - ln (n-M)!] */
        double delta = ((k - M) * lpq - or_lnfact_diff(M, k - M)) - or_lnfact_diff(nd - M, M - k);
        double lx = or_log(X);
        if (lx + lx <= delta) {
            *out = (uint64_t)k;
            return 0;
        }
    }
    return 6;
}

static int binom_upto(uint64_t n, double p, or_stream *s, uint64_t *x, uint64_t nmax)
{
    if (n == 0 || p <= 0.0) {
        *x = 0;
        return 0;
    }
    if (p >= 1.0) {
        *x = n;
        return 0;
    }
    if (n > nmax)
        return 2;
    int flip = p > 0.5;
    double pp = flip ? 1.0 - p : p;
    uint64_t r;
    int rc = ((double)n * pp < 10.0) ? binom_inversion(n, pp, s, &r) : binom_rou(n, pp, s, &r);
    if (rc)
        return rc;
    *x = flip ? n - r : r;
    return 0;
}

int or_binom_s(uint64_t n, double p, or_stream *s, uint64_t *x)
{
    return binom_upto(n, p, s, x, OR_M_MAX);
}

/* The same variate for n up to 2^53 (every count and n - x stays exact in a
 * double): the chunk counts of G(n,p), Sec. 4.3. */
int or_binom_big(uint64_t n, double p, or_stream *s, uint64_t *x)
{
    return binom_upto(n, p, s, x, OR_BINOM_N_MAX);
}

/* ---------------- hypergeometric ---------------- */

/* Binomial(t, 1/2) as the number of one bits among t fair bits, taken from
 * the stream's u64 words in order (low bits of the last partial word). */
static uint64_t popcount_binomial(uint64_t t, or_stream *s)
{
    uint64_t X = 0;
    uint64_t left = t;
    while (left > 0) {
        uint64_t w = or_next_u64(s);
        if (left < 64)
            w &= ((uint64_t)1 << left) - 1;
        X += (uint64_t)__builtin_popcountll(w);
        left = left < 64 ? 0 : left - 64;
    }
    return X;
}

/* Inversion from 0 (support starts at 0 because K, t <= N/2).  The pmf is
 * symmetric in K and t; with A = min(K,t):
 *   ln f(0) = D(N-K-t, A) - D(N-A, A),  D(a,d) = ln (a+d)! - ln a!
 *   f(x+1)/f(x) = (K-x)(t-x) / ((x+1)(N-K-t+x+1)). */
static int hyper_inversion(u128 N, u128 K, u128 t, or_stream *s, uint64_t *out)
{
    u128 A = K < t ? K : t;
    double Kd = or_dbl128(K), td = or_dbl128(t), Ad = or_dbl128(A);
    double rest = or_dbl128(N - K - t);
    double lnf0 = or_lnfact_diff(rest, Ad) - or_lnfact_diff(or_dbl128(N - A), Ad);
    double f0 = or_exp(lnf0);
    for (int attempt = 0; attempt < OR_REJECT_CAP; attempt++) {
        double U = or_u01_open1(or_next_u64(s));
        uint64_t x = 0;
        double f = f0;
        for (;;) {
            if (U < f) {
                *out = x;
                return 0;
            }
            U = U - f;
            double xd = (double)x;
            f = f * (((Kd - xd) * (td - xd)) / ((xd + 1.0) * ((rest + xd) + 1.0)));
            x = x + 1;
            if ((double)x > Ad || f == 0.0)
                break;
        }
    }
    return 6;
}

/* Ratio of uniforms: mean = tK/N, var = (N-t) t p q / (N-1), mode
 * M = floor((t+1)(K+1)/(N+2)), hat centre mean + 1/2, width
 * D1 sqrt(var + 1/2) + D2. */
static int hyper_rou(u128 N, u128 K, u128 t, or_stream *s, uint64_t *out)
{
    double Nd = or_dbl128(N), Kd = or_dbl128(K), td = or_dbl128(t);
    double rest = or_dbl128(N - K - t);
    double p = Kd / Nd;
    double q = 1.0 - p;
    double mean = (td * Kd) / Nd;
    double var = ((((Nd - td) * td) * p) * q) / (Nd - 1.0);
    double M = __builtin_floor(((td + 1.0) * (Kd + 1.0)) / (Nd + 2.0));
    double a = mean + 0.5;
    double sw = RoU_D1 * __builtin_sqrt(var + 0.5) + RoU_D2;
    double xmax = dmin(Kd, td);
    for (int it = 0; it < OR_REJECT_CAP; it++) {
        double X = or_u01_open0(or_next_u64(s));
        double Y = or_u01_open1(or_next_u64(s));
        double W = a + (sw * (Y - 0.5)) / X;
        if (W < 0.0 || W >= xmax + 1.0)
            continue;
        double k = __builtin_floor(W);
        /* ln f(k) - ln f(M) as a sum of four factorial differences */
        double delta = (((-or_lnfact_diff(M, k - M)) - or_lnfact_diff(Kd - M, M - k))
                        - or_lnfact_diff(td - M, M - k)) - or_lnfact_diff(rest + M, k - M);
        double lx = or_log(X);
        if (lx + lx <= delta) {
            *out = (uint64_t)k;
            return 0;
        }
    }
    return 6;
}

/* K and t already reduced to at most N/2, both >= 1. */
static int hyper_core(u128 N, u128 K, uint64_t t, or_stream *s, uint64_t *x)
{
    if (((u128)t << 32) <= N) {
        /* t draws from a universe at least 2^32 t: replacement changes the law
         * by at most (t-1)/(N-1) < 2^-32 in total variation, so draw the
         * binomial; an exactly even split with few draws counts fair bits. */
        if (K + K == N && t <= ((uint64_t)1 << 15)) {
            *x = popcount_binomial(t, s);
            return 0;
        }
        return or_binom_s(t, or_dbl128(K) / or_dbl128(N), s, x);
    }
    double mean = (or_dbl128((u128)t) * or_dbl128(K)) / or_dbl128(N);
    if (mean < 10.0)
        return hyper_inversion(N, K, (u128)t, s, x);
    return hyper_rou(N, K, (u128)t, s, x);
}

/* Hypergeometric(N, K, t): the number of marked items among t drawn without
 * replacement from N items of which K are marked (Sec. 2.2: the sample count
 * of one half of a split universe).  Symmetries bring K and t to <= N/2. */
int or_hyper_s(u128 N, u128 K, uint64_t t, or_stream *s, uint64_t *x)
{
    if (K > N || (u128)t > N)
        return 1;
    if (t > OR_M_MAX)
        return 2;
    if (t == 0 || K == 0) {
        *x = 0;
        return 0;
    }
    if (K == N) {
        *x = t;
        return 0;
    }
    if ((u128)t == N) {
        *x = (uint64_t)K;
        return 0;
    }
    u128 K1 = K;
    int flipK = 0;
    if (K + K > N) {
        K1 = N - K;
        flipK = 1;
    }
    uint64_t t1 = t;
    int flipT = 0;
    if ((u128)t + (u128)t > N) {
        t1 = (uint64_t)(N - t);
        flipT = 1;
    }
    uint64_t r;
    int rc = hyper_core(N, K1, t1, s, &r);
    if (rc)
        return rc;
    if (flipT)
        r = (uint64_t)(K1 - r); /* marked among the complementary draws */
    if (flipK)
        r = t - r;              /* swap marked and unmarked */
    *x = r;
    return 0;
}

int or_hypergeometric(uint64_t N_lo, uint64_t N_hi, uint64_t K_lo, uint64_t K_hi,
                      uint64_t t, uint64_t seed, uint64_t node, uint32_t tag, uint64_t *x)
{
    or_stream s = or_stream_make(seed, node, tag);
    u128 N = ((u128)N_hi << 64) | N_lo;
    u128 K = ((u128)K_hi << 64) | K_lo;
    return or_hyper_s(N, K, t, &s, x);
}

int or_binomial(uint64_t n, double p, uint64_t seed, uint64_t node, uint32_t tag, uint64_t *x)
{
    or_stream s = or_stream_make(seed, node, tag);
    return or_binom_s(n, p, &s, x);
}
