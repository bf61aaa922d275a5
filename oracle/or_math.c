/*
 * Oracle: FP64 elementary functions (test infrastructure; see oracle.h).
 *
 * The variates of Sec. 2.2 (hypergeometric, binomial) and the geometric skips
 * of the G(n,p) sampler need ln, exp and ln k!.  To make two independent
 * implementations agree bit for bit, libm is never called: every function
 * below uses only IEEE-754 binary64 +, -, *, /, sqrt in round-to-nearest,
 * floor, and exact bit manipulation of the exponent, in the operation order
 * written here.  Compile with -ffp-contract=off (no fused multiply-add).
 */
#include <string.h>
#include "or_internal.h"

#define SQRT_HALF 0x1.6a09e667f3bcdp-1
#define LN2 0x1.62e42fefa39efp-1
#define INV_LN2 0x1.71547652b82fep+0
#define LN2_HI 0x1.62e42fee00000p-1
#define LN2_LO 0x1.a39ef35793c76p-33
#define HALF_LN_2PI 0x1.d67f1c864beb5p-1

static uint64_t bits_of(double x) { uint64_t b; memcpy(&b, &x, 8); return b; }
static double of_bits(uint64_t b) { double x; memcpy(&x, &b, 8); return x; }

/* x = f * 2^e with f in [0.5, 1), for finite x > 0. */
static double frexp_pos(double x, int *e)
{
    uint64_t b = bits_of(x);
    int ex = (int)((b >> 52) & 0x7ff);
    int adj = 0;
    if (ex == 0) { /* subnormal: scale into the normal range first (exact) */
        x = x * 0x1p54;
        b = bits_of(x);
        ex = (int)((b >> 52) & 0x7ff);
        adj = 54;
    }
    *e = ex - 1022 - adj;
    return of_bits((b & 0x800fffffffffffffULL) | ((uint64_t)1022 << 52));
}

/* 2^k for -1022 <= k <= 1023, built from bits (exact). */
static double pow2i(int k) { return of_bits((uint64_t)(k + 1023) << 52); }

/* Horner sum of the atanh series 1 + z/3 + z^2/5 + ... + z^11/23 with
 * coefficients c_j = 1/(2j+1), each the IEEE quotient 1.0/(2j+1). */
static double atanh_poly(double z)
{
    double P = 1.0 / 23.0;
    for (int j = 10; j >= 0; j--)
        P = 1.0 / (double)(2 * j + 1) + z * P;
    return P;
}

/* ln x for finite x > 0: ln x = e ln 2 + 2 atanh(s), s = (f-1)/(f+1),
 * f in [sqrt(1/2), sqrt(2)), so |s| <= 0.1716 and the truncated series
 * term is below 2e-20 relative. */
double or_log(double x)
{
    int e;
    double f = frexp_pos(x, &e);
    if (f < SQRT_HALF) {
        f = f + f;
        e = e - 1;
    }
    double s = (f - 1.0) / (f + 1.0);
    double z = s * s;
    double P = atanh_poly(z);
    return (double)e * LN2 + (s + s) * P;
}

/* ln(1-p) for 0 < p < 1.  Small p uses ln(1-p) = 2 atanh(-p/(2-p)) so no
 * digits are lost forming 1-p. */
double or_log1m(double p)
{
    if (p < 0.25) {
        double s = -p / (2.0 - p);
        double z = s * s;
        return (s + s) * atanh_poly(z);
    }
    return or_log(1.0 - p);
}

/* exp x: k = rint(x / ln 2), r = x - k ln2 (Cody-Waite split of ln 2),
 * Taylor polynomial of degree 17 in Horner form with coefficients 1/j!
 * (e_0 = 1, e_j = e_{j-1}/j), scaled by an exact power of two.
 * Defined on [-700, 700]; below returns 0, above returns +inf. */
double or_exp(double x)
{
    if (x < -700.0)
        return 0.0;
    if (x > 700.0)
        return 1.0 / 0.0;
    double kd = x * INV_LN2;
    /* round half to even, exactly: floor-based with tie correction */
    double fl = __builtin_floor(kd);
    double diff = kd - fl;
    double k = fl;
    if (diff > 0.5 || (diff == 0.5 && __builtin_fmod(fl, 2.0) != 0.0))
        k = fl + 1.0;
    double r = (x - k * LN2_HI) - k * LN2_LO;
    double ej[18];
    ej[0] = 1.0;
    for (int j = 1; j <= 17; j++)
        ej[j] = ej[j - 1] / (double)j;
    double t = ej[17];
    for (int j = 16; j >= 0; j--)
        t = ej[j] + r * t;
    return t * pow2i((int)k);
}

/* ln k! for an integer-valued double k >= 0.  k < 32: running sum of
 * or_log(j), j = 2..k, in ascending order.  Otherwise Stirling's series for
 * ln Gamma(x), x = k+1, with four correction terms. */
static double stirling_tail(double x)
{
    double w = 1.0 / x;
    double w2 = w * w;
    double C1 = 1.0 / 12.0, C3 = 1.0 / 360.0, C5 = 1.0 / 1260.0, C7 = 1.0 / 1680.0;
    return w * (C1 - w2 * (C3 - w2 * (C5 - w2 * C7)));
}

double or_lnfact(double k)
{
    if (k < 32.0) {
        double sum = 0.0;
        int kk = (int)k;
        for (int j = 2; j <= kk; j++)
            sum = sum + or_log((double)j);
        return sum;
    }
    double x = k + 1.0;
    return (((x - 0.5) * or_log(x)) - x) + HALF_LN_2PI + stirling_tail(x);
}

/* D(a, d) = ln (a+d)! - ln a!  for integer-valued doubles a >= 0, a+d >= 0.
 * When both arguments are large and close, the Stirling difference is taken
 * in a form without cancellation:
 *   (x1 - 1/2) ln(x2/x1) + d ln x2 - d + S(x2) - S(x1),  x1 = a+1, x2 = x1+d,
 * with ln(x2/x1) = 2 atanh(d / (x1 + x2)). */
double or_lnfact_diff(double a, double d)
{
    if (d == 0.0)
        return 0.0;
    double lo = a + d < a ? a + d : a;
    double ad = d < 0.0 ? -d : d;
    if (lo >= 64.0 && 4.0 * ad <= lo) {
        double x1 = a + 1.0;
        double x2 = x1 + d;
        double s = d / (x1 + x2);
        double z = s * s;
        double L = (s + s) * atanh_poly(z);
        return ((((x1 - 0.5) * L) + d * or_log(x2)) - d) + (stirling_tail(x2) - stirling_tail(x1));
    }
    return or_lnfact(a + d) - or_lnfact(a);
}
