// Device primitives of the communication-free Erdos-Renyi generators.
//
// * Philox4x32-10 node streams (Salmon et al., SC 2011): the paper's
//   pseudorandomisation of Sec. 2.2 -- every recursion subtree draws its
//   variates from a generator seeded by (global seed, subtree id) -- with the
//   subtree id carried in the counter instead of a hash.
// * FP64 ln / exp / ln k! built from IEEE-exact + - * / sqrt only, in a fixed
//   operation order, so that device and host procedures agree bit for bit.
//   Every translation unit is compiled with -fmad=false.
// * Hypergeometric and binomial variates (Sec. 2.2: acceptance-rejection in
//   expected O(1), Stadlober's ratio of uniforms) and the fair-bit binomial.
// * Lemire's bounded integers for Floyd's leaf sampler, and division by the
//   invariant n-1 through a multiplier (Granlund & Montgomery, PLDI 1994).
#pragma once
#include <cstdint>
#include <cstring>

namespace kg {

typedef unsigned __int128 u128;

// ---------------------------------------------------------------- status
enum : int {
  ST_OK = 0,
  ST_ARG = 1,
  ST_RANGE = 2,
  ST_CAPACITY = 3,
  ST_CUDA = 4,
  ST_TIMEOUT = 5,
  ST_INTERNAL = 6,
};

// ---------------------------------------------------------------- stream tags
enum : uint32_t {
  TAG_CHUNK_TREE = 1u,  // directed chunk split tree, node = heap index
  TAG_QUAD = 2u,        // undirected quadrant tree, node = block ranges
  TAG_TILE = 3u,        // tile tree inside a chunk, node = chunk<<32 | heap
  TAG_LEAF = 4u,        // Floyd draws of a leaf, node = chunk<<32 | heap
  TAG_GNP = 5u,         // geometric skips of a G(n,p) tile, node = chunk<<32 | tile
  TAG_GNP_COUNT = 6u,   // binomial sample count of a G(n,p) chunk, node = chunk id
};

// Limits of the procedure.
constexpr uint64_t M_MAX = uint64_t(1) << 44;  // largest m / binomial n
constexpr uint64_t BINOM_N_MAX = uint64_t(1) << 53;  // largest n of a G(n,p) chunk count
constexpr int D_MAX = 24;                      // largest tile-tree depth
constexpr int LEVEL_MAX = 31;                  // heap index < 2^32
constexpr int REJECT_CAP = 1000000;            // rejection loop cap

// ---------------------------------------------------------------- Philox4x32-10
__host__ __device__ __forceinline__ void philox10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                  uint32_t c3, uint32_t k0, uint32_t k1,
                                                  uint32_t w[4]) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
#ifdef __CUDA_ARCH__
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
#else
    const uint64_t p0 = uint64_t(0xD2511F53u) * c0, p1 = uint64_t(0xCD9E8D57u) * c2;
    const uint32_t hi0 = uint32_t(p0 >> 32), lo0 = uint32_t(p0);
    const uint32_t hi1 = uint32_t(p1 >> 32), lo1 = uint32_t(p1);
#endif
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  w[0] = c0;
  w[1] = c1;
  w[2] = c2;
  w[3] = c3;
}

// A node stream: u64 number i is half (i & 1) of Philox block i >> 1 with the
// counter (i >> 1, lo32(node), hi32(node), tag); a half reads (wA << 32) | wB.
struct Stream {
  uint32_t k0, k1, n0, n1, tag;
  uint64_t next;
  uint64_t cached_block;
  uint32_t w[4];

  __host__ __device__ __forceinline__ Stream(uint64_t seed, uint64_t node, uint32_t tag_)
      : k0(uint32_t(seed)), k1(uint32_t(seed >> 32)), n0(uint32_t(node)),
        n1(uint32_t(node >> 32)), tag(tag_), next(0), cached_block(~uint64_t(0)) {}

  __host__ __device__ __forceinline__ uint64_t at(uint64_t i) {
    const uint64_t b = i >> 1;
    if (b != cached_block) {
      philox10(uint32_t(b), n0, n1, tag, k0, k1, w);
      cached_block = b;
    }
    return (i & 1) ? ((uint64_t(w[2]) << 32) | w[3]) : ((uint64_t(w[0]) << 32) | w[1]);
  }
  __host__ __device__ __forceinline__ uint64_t u64() { return at(next++); }
};

__host__ __device__ __forceinline__ uint64_t stream_u64(uint64_t seed, uint64_t node, uint32_t tag,
                                                        uint64_t i) {
  uint32_t w[4];
  philox10(uint32_t(i >> 1), uint32_t(node), uint32_t(node >> 32), tag, uint32_t(seed),
           uint32_t(seed >> 32), w);
  return (i & 1) ? ((uint64_t(w[2]) << 32) | w[3]) : ((uint64_t(w[0]) << 32) | w[1]);
}

// (0,1] and [0,1) uniforms from the top 53 bits.
__host__ __device__ __forceinline__ double u01_oc(uint64_t x) {
  return double((x >> 11) + 1) * 0x1p-53;
}
__host__ __device__ __forceinline__ double u01_co(uint64_t x) { return double(x >> 11) * 0x1p-53; }

// ---------------------------------------------------------------- conversions
// Nearest-even conversion of a 128-bit integer: keep the top 64 bits with a
// sticky bit for everything shifted out, convert, scale by the exact power.
__host__ __device__ __forceinline__ double dbl(u128 x) {
  const uint64_t hi = uint64_t(x >> 64);
  if (hi == 0) return double(uint64_t(x));
#ifdef __CUDA_ARCH__
  const int nb = 128 - __clzll((long long)hi);
#else
  const int nb = 128 - __builtin_clzll(hi);
#endif
  const int s = nb - 64;
  const u128 lost_mask = (u128(1) << s) - 1;
  const uint64_t y = uint64_t(x >> s) | ((x & lost_mask) != 0 ? 1ull : 0ull);
  double r = double(y);
  // multiply by 2^s (s <= 64), exact
  uint64_t pb = uint64_t(s + 1023) << 52;
  double p;
  memcpy(&p, &pb, 8);
  return r * p;
}

__host__ __device__ __forceinline__ uint64_t bits(double x) {
  uint64_t b;
  memcpy(&b, &x, 8);
  return b;
}
__host__ __device__ __forceinline__ double from_bits(uint64_t b) {
  double x;
  memcpy(&x, &b, 8);
  return x;
}

// ---------------------------------------------------------------- FP64 functions
constexpr double SQRT_HALF = 0x1.6a09e667f3bcdp-1;
constexpr double LN2 = 0x1.62e42fefa39efp-1;
constexpr double INV_LN2 = 0x1.71547652b82fep+0;
constexpr double LN2_HI = 0x1.62e42fee00000p-1;
constexpr double LN2_LO = 0x1.a39ef35793c76p-33;
constexpr double HALF_LN_2PI = 0x1.d67f1c864beb5p-1;

// 1 + z/3 + z^2/5 + ... + z^11/23 in Horner form, c_j = 1/(2j+1) as IEEE quotients.
__host__ __device__ __forceinline__ double atanh_series(double z) {
  double P = 1.0 / 23.0;
#pragma unroll
  for (int j = 10; j >= 0; --j) P = 1.0 / double(2 * j + 1) + z * P;
  return P;
}

// ln x, x > 0 finite: x = f 2^e, f moved into [sqrt(1/2), sqrt(2)),
// ln x = e ln2 + 2 atanh((f-1)/(f+1)).
__host__ __device__ __forceinline__ double kg_log(double x) {
  uint64_t b = bits(x);
  int ex = int((b >> 52) & 0x7ff);
  int adj = 0;
  if (ex == 0) {  // subnormal: scale up exactly
    x = x * 0x1p54;
    b = bits(x);
    ex = int((b >> 52) & 0x7ff);
    adj = 54;
  }
  int e = ex - 1022 - adj;
  double f = from_bits((b & 0x800fffffffffffffull) | (uint64_t(1022) << 52));
  if (f < SQRT_HALF) {
    f = f + f;
    e = e - 1;
  }
  const double s = (f - 1.0) / (f + 1.0);
  const double z = s * s;
  const double P = atanh_series(z);
  return double(e) * LN2 + (s + s) * P;
}

// ln(1-p), 0 < p < 1; small p via 2 atanh(-p/(2-p)).
__host__ __device__ __forceinline__ double kg_log1m(double p) {
  if (p < 0.25) {
    const double s = -p / (2.0 - p);
    const double z = s * s;
    return (s + s) * atanh_series(z);
  }
  return kg_log(1.0 - p);
}

// exp x on [-700, 700] (0 below, +inf above): x = k ln2 + r with a two-part
// ln2, degree-17 Taylor polynomial (coefficients e_j = e_{j-1}/j), times 2^k.
__host__ __device__ __forceinline__ double kg_exp(double x) {
  if (x < -700.0) return 0.0;
  if (x > 700.0) return from_bits(0x7ff0000000000000ull);
  const double k = rint(x * INV_LN2);
  const double r = (x - k * LN2_HI) - k * LN2_LO;
  double ej[18];
  ej[0] = 1.0;
#pragma unroll
  for (int j = 1; j <= 17; ++j) ej[j] = ej[j - 1] / double(j);
  double t = ej[17];
#pragma unroll
  for (int j = 16; j >= 0; --j) t = ej[j] + r * t;
  return t * from_bits(uint64_t(int(k) + 1023) << 52);
}

// Stirling correction 1/(12x) - 1/(360x^3) + 1/(1260x^5) - 1/(1680x^7).
__host__ __device__ __forceinline__ double stirling_tail(double x) {
  const double w = 1.0 / x;
  const double w2 = w * w;
  return w * (1.0 / 12.0 - w2 * (1.0 / 360.0 - w2 * (1.0 / 1260.0 - w2 * (1.0 / 1680.0))));
}

// ln k! for integer-valued k >= 0 (ascending sum of logs below 32).
__host__ __device__ __forceinline__ double kg_lnfact(double k) {
  if (k < 32.0) {
    double sum = 0.0;
    const int kk = int(k);
    for (int j = 2; j <= kk; ++j) sum = sum + kg_log(double(j));
    return sum;
  }
  const double x = k + 1.0;
  return (((x - 0.5) * kg_log(x)) - x) + HALF_LN_2PI + stirling_tail(x);
}

// D(a, d) = ln (a+d)! - ln a!; large close arguments use
// (x1 - 1/2) 2atanh(d/(x1+x2)) + d ln x2 - d + S(x2) - S(x1).
__host__ __device__ __forceinline__ double kg_lnfact_diff(double a, double d) {
  if (d == 0.0) return 0.0;
  const double lo = (a + d < a) ? a + d : a;
  const double ad = d < 0.0 ? -d : d;
  if (lo >= 64.0 && 4.0 * ad <= lo) {
    const double x1 = a + 1.0;
    const double x2 = x1 + d;
    const double s = d / (x1 + x2);
    const double z = s * s;
    const double L = (s + s) * atanh_series(z);
    return ((((x1 - 0.5) * L) + d * kg_log(x2)) - d) + (stirling_tail(x2) - stirling_tail(x1));
  }
  return kg_lnfact(a + d) - kg_lnfact(a);
}

// ---------------------------------------------------------------- variates
constexpr double RoU_D1 = 0x1.b72cd3f331398p+0;  // 2 sqrt(2/e)
constexpr double RoU_D2 = 0x1.cc3ebd3bc711ap-1;  // 3 - 2 sqrt(3/e)

__host__ __device__ __forceinline__ int binom_inversion(uint64_t n, double p, Stream& s,
                                                        uint64_t& out) {
  const double nd = double(n);
  const double q = 1.0 - p;
  const double r = p / q;
  const double f0 = kg_exp(nd * kg_log1m(p));
  for (int attempt = 0; attempt < REJECT_CAP; ++attempt) {
    double U = u01_co(s.u64());
    uint64_t x = 0;
    double f = f0;
    for (;;) {
      if (U < f) {
        out = x;
        return ST_OK;
      }
      U = U - f;
      const double xd = double(x);
      f = ((f * r) * (nd - xd)) / (xd + 1.0);
      x = x + 1;
      if (x > n || f == 0.0) break;
    }
  }
  return ST_INTERNAL;
}

__host__ __device__ __forceinline__ int binom_rou(uint64_t n, double p, Stream& s, uint64_t& out) {
  const double nd = double(n);
  const double q = 1.0 - p;
  const double mean = nd * p;
  const double var = mean * q;
  const double M = floor((nd + 1.0) * p);
  const double a = mean + 0.5;
  const double sw = RoU_D1 * sqrt(var + 0.5) + RoU_D2;
  const double lpq = kg_log(p) - kg_log1m(p);
  for (int it = 0; it < REJECT_CAP; ++it) {
    const double X = u01_oc(s.u64());
    const double Y = u01_co(s.u64());
    const double W = a + (sw * (Y - 0.5)) / X;
    if (W < 0.0 || W >= nd + 1.0) continue;
    const double k = floor(W);
    const double delta =
        ((k - M) * lpq - kg_lnfact_diff(M, k - M)) - kg_lnfact_diff(nd - M, M - k);
    const double lx = kg_log(X);
    if (lx + lx <= delta) {
      out = uint64_t(k);
      return ST_OK;
    }
  }
  return ST_INTERNAL;
}

// Binomial(n, p): inversion for n min(p,1-p) < 10, else ratio of uniforms;
// n up to nmax (M_MAX for the hypergeometric's binomial regime, BINOM_N_MAX
// for the chunk counts of G(n,p): every count and n - x stay exact doubles).
__host__ __device__ __forceinline__ int binomial(uint64_t n, double p, Stream& s, uint64_t& out,
                                                 uint64_t nmax = M_MAX) {
  if (n == 0 || p <= 0.0) {
    out = 0;
    return ST_OK;
  }
  if (p >= 1.0) {
    out = n;
    return ST_OK;
  }
  if (n > nmax) return ST_RANGE;
  const bool flip = p > 0.5;
  const double pp = flip ? 1.0 - p : p;
  uint64_t r = 0;
  const int st = (double(n) * pp < 10.0) ? binom_inversion(n, pp, s, r) : binom_rou(n, pp, s, r);
  if (st) return st;
  out = flip ? n - r : r;
  return ST_OK;
}

// Binomial(t, 1/2) as the number of ones among t fair bits: u64 words
// s.next, s.next+1, ... (low bits of the last partial word).
__host__ __device__ __forceinline__ uint64_t popcount_bits(uint64_t t, Stream& s) {
  uint64_t X = 0;
  uint64_t left = t;
  while (left > 0) {
    uint64_t w = s.u64();
    if (left < 64) w &= (uint64_t(1) << left) - 1;
#ifdef __CUDA_ARCH__
    X += uint64_t(__popcll(w));
#else
    X += uint64_t(__builtin_popcountll(w));
#endif
    left = left < 64 ? 0 : left - 64;
  }
  return X;
}

// Hypergeometric inversion from 0 (K, t <= N/2): with A = min(K, t),
// ln f(0) = D(N-K-t, A) - D(N-A, A), f(x+1)/f(x) = (K-x)(t-x)/((x+1)(N-K-t+x+1)).
__host__ __device__ __forceinline__ int hyper_inversion(u128 N, u128 K, u128 t, Stream& s,
                                                        uint64_t& out) {
  const u128 A = K < t ? K : t;
  const double Kd = dbl(K), td = dbl(t), Ad = dbl(A);
  const double rest = dbl(N - K - t);
  const double lnf0 = kg_lnfact_diff(rest, Ad) - kg_lnfact_diff(dbl(N - A), Ad);
  const double f0 = kg_exp(lnf0);
  for (int attempt = 0; attempt < REJECT_CAP; ++attempt) {
    double U = u01_co(s.u64());
    uint64_t x = 0;
    double f = f0;
    for (;;) {
      if (U < f) {
        out = x;
        return ST_OK;
      }
      U = U - f;
      const double xd = double(x);
      f = f * (((Kd - xd) * (td - xd)) / ((xd + 1.0) * ((rest + xd) + 1.0)));
      x = x + 1;
      if (double(x) > Ad || f == 0.0) break;
    }
  }
  return ST_INTERNAL;
}

// Ratio of uniforms for the hypergeometric law (K, t <= N/2, mean >= 10).
__host__ __device__ __forceinline__ int hyper_rou(u128 N, u128 K, u128 t, Stream& s,
                                                  uint64_t& out) {
  const double Nd = dbl(N), Kd = dbl(K), td = dbl(t);
  const double rest = dbl(N - K - t);
  const double p = Kd / Nd;
  const double q = 1.0 - p;
  const double mean = (td * Kd) / Nd;
  const double var = ((((Nd - td) * td) * p) * q) / (Nd - 1.0);
  const double M = floor(((td + 1.0) * (Kd + 1.0)) / (Nd + 2.0));
  const double a = mean + 0.5;
  const double sw = RoU_D1 * sqrt(var + 0.5) + RoU_D2;
  const double xmax = Kd < td ? Kd : td;
  for (int it = 0; it < REJECT_CAP; ++it) {
    const double X = u01_oc(s.u64());
    const double Y = u01_co(s.u64());
    const double W = a + (sw * (Y - 0.5)) / X;
    if (W < 0.0 || W >= xmax + 1.0) continue;
    const double k = floor(W);
    const double delta = (((-kg_lnfact_diff(M, k - M)) - kg_lnfact_diff(Kd - M, M - k)) -
                          kg_lnfact_diff(td - M, M - k)) -
                         kg_lnfact_diff(rest + M, k - M);
    const double lx = kg_log(X);
    if (lx + lx <= delta) {
      out = uint64_t(k);
      return ST_OK;
    }
  }
  return ST_INTERNAL;
}

// Reduced hypergeometric problem: 1 <= K <= N/2, 1 <= t <= N/2.
struct HyperPlan {
  u128 N, K1;
  uint64_t t, t1;
  bool flipK, flipT;
  int kind;  // 0 = done (value in `fixed`), 1 = fair bits, 2 = general
  uint64_t fixed;
};

// Trivial cases, symmetries, and the choice of the fair-bit branch.
__host__ __device__ __forceinline__ int hyper_plan(u128 N, u128 K, uint64_t t, HyperPlan& h) {
  h.N = N;
  h.t = t;
  h.kind = 0;
  h.fixed = 0;
  if (K > N || u128(t) > N) return ST_ARG;
  if (t > M_MAX) return ST_RANGE;
  if (t == 0 || K == 0) return ST_OK;
  if (K == N) {
    h.fixed = t;
    return ST_OK;
  }
  if (u128(t) == N) {
    h.fixed = uint64_t(K);
    return ST_OK;
  }
  h.flipK = K + K > N;
  h.K1 = h.flipK ? N - K : K;
  h.flipT = u128(t) + u128(t) > N;
  h.t1 = h.flipT ? uint64_t(N - t) : t;
  const bool binreg = (u128(h.t1) << 32) <= N;
  h.kind = (binreg && h.K1 + h.K1 == N && h.t1 <= (uint64_t(1) << 15)) ? 1 : 2;
  return ST_OK;
}

__host__ __device__ __forceinline__ uint64_t hyper_finish(const HyperPlan& h, uint64_t r) {
  if (h.flipT) r = uint64_t(h.K1 - r);
  if (h.flipK) r = h.t - r;
  return r;
}

// General branch (kind 2) of a planned draw.
__host__ __device__ __forceinline__ int hyper_general(const HyperPlan& h, Stream& s,
                                                      uint64_t& r) {
  const u128 N = h.N, K = h.K1;
  const uint64_t t = h.t1;
  if ((u128(t) << 32) <= N) return binomial(t, dbl(K) / dbl(N), s, r);
  const double mean = (dbl(u128(t)) * dbl(K)) / dbl(N);
  if (mean < 10.0) return hyper_inversion(N, K, u128(t), s, r);
  return hyper_rou(N, K, u128(t), s, r);
}

// Hypergeometric(N, K, t) by one thread.
__host__ __device__ __forceinline__ int hypergeometric(u128 N, u128 K, uint64_t t, Stream& s,
                                                       uint64_t& out) {
  HyperPlan h;
  int st = hyper_plan(N, K, t, h);
  if (st) return st;
  if (h.kind == 0) {
    out = h.fixed;
    return ST_OK;
  }
  uint64_t r;
  if (h.kind == 1) {
    r = popcount_bits(h.t1, s);
  } else {
    st = hyper_general(h, s, r);
    if (st) return st;
  }
  out = hyper_finish(h, r);
  return ST_OK;
}

// Fair-bit count by a whole warp: words [w0, w0 + ceil(t/64)) of the stream,
// lane l takes Philox blocks b0 + l, b0 + l + 32, ...
__device__ __forceinline__ uint64_t popcount_bits_warp(uint64_t seed, uint64_t node, uint32_t tag,
                                                       uint64_t w0, uint64_t t) {
  const unsigned lane = threadIdx.x & 31;
  const uint64_t nw = (t + 63) >> 6;
  const uint64_t w1 = w0 + nw;
  const uint64_t b0 = w0 >> 1, b1 = (w1 - 1) >> 1;
  const uint64_t last = w1 - 1;
  const unsigned tail = unsigned(t & 63);
  unsigned long long acc = 0;
  for (uint64_t b = b0 + lane; b <= b1; b += 32) {
    uint32_t w[4];
    philox10(uint32_t(b), uint32_t(node), uint32_t(node >> 32), tag, uint32_t(seed),
             uint32_t(seed >> 32), w);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint64_t idx = 2 * b + h;
      if (idx < w0 || idx >= w1) continue;
      uint64_t x = h ? ((uint64_t(w[2]) << 32) | w[3]) : ((uint64_t(w[0]) << 32) | w[1]);
      if (idx == last && tail) x &= (uint64_t(1) << tail) - 1;
      acc += __popcll(x);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  return acc;
}

// ---------------------------------------------------------------- leaf draws
// Lemire: high word of x * range; reject when the low word is below
// (2^64 - range) mod range; retry r draws u64 #i of the stream tagged
// TAG_LEAF | r << 8.  `x` is the leaf stream's u64 #i.
__host__ __device__ __forceinline__ uint64_t mul_hi64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
  return __umul64hi(a, b);
#else
  return uint64_t((u128(a) * b) >> 64);
#endif
}

// 2^64 mod r (= (2^64 - r) mod r, Lemire's threshold) by doubling 1 modulo r
// 64 times; only the rejection branch needs it, and it keeps that branch free
// of a division routine.
__host__ __device__ __forceinline__ uint64_t pow2_64_mod(uint64_t r) {
  uint64_t rem = r == 1 ? 0 : 1;
  for (int b = 0; b < 64; ++b) {
    const uint64_t t = rem << 1;
    rem = ((rem >> 63) || t >= r) ? t - r : t;
  }
  return rem;
}

__host__ __device__ __forceinline__ uint64_t lemire_draw(uint64_t x, uint64_t range, uint64_t seed,
                                                         uint64_t node, uint64_t i) {
  uint64_t hi = mul_hi64(x, range);
  uint64_t lo = x * range;
  if (lo < range) {  // probability below range / 2^64
    const uint64_t thr = pow2_64_mod(range);
    uint32_t r = 1;
    while (lo < thr) {
      x = stream_u64(seed, node, TAG_LEAF | (r << 8), i);
      ++r;
      hi = mul_hi64(x, range);
      lo = x * range;
    }
  }
  return hi;
}

// ---------------------------------------------------------------- invariant division
// q = floor(x / D) for all 64-bit x, D >= 1 fixed: with l = ceil(log2 D),
// m = floor(2^64 (2^l - D) / D) + 1, t = mulhi(m, x),
// q = (t + ((x - t) >> min(l,1))) >> max(l-1, 0).
struct DivU64 {
  uint64_t D, m;
  int sh1, sh2;
};

inline DivU64 make_div(uint64_t D) {
  DivU64 r;
  r.D = D;
  int l = 0;
  while (l < 64 && (u128(1) << l) < u128(D)) ++l;
  r.m = uint64_t(((u128(1) << 64) * ((u128(1) << l) - D)) / D) + 1;
  r.sh1 = l < 1 ? l : 1;
  r.sh2 = l > 1 ? l - 1 : 0;
  return r;
}

__host__ __device__ __forceinline__ uint64_t div_q(const DivU64& d, uint64_t x) {
#ifdef __CUDA_ARCH__
  const uint64_t t = __umul64hi(d.m, x);
#else
  const uint64_t t = uint64_t((u128(d.m) * x) >> 64);
#endif
  return (t + ((x - t) >> d.sh1)) >> d.sh2;
}

// SplitMix64 finaliser (Steele, Lea, Flood 2014) for the edge digest.
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t edge_hash(uint64_t u, uint64_t v) {
  return mix64(u ^ ((v << 32) | (v >> 32)));
}

}  // namespace kg
