// Warp-cooperative hypergeometric and binomial variates: one draw by a whole
// warp, bit-identical to the one-thread procedure of kg_device.cuh.
//
// The ratio-of-uniforms loops (Sec. 2.2's acceptance-rejection, Stadlober's
// method) take candidate j from words w0 + 2j and w0 + 2j + 1 of the node
// stream and accept the first candidate that passes its test.  A candidate
// consumes only its own two words, so candidates can be evaluated in any
// order: here a group of lanes evaluates one candidate, one term of the
// acceptance test per lane (every term is the same function of the same
// arguments as in the sequential loop, and the group leader combines them in
// the same order), and the first accepted candidate in stream order is the
// result.  The sequential loop's dependent FP64 chain of ~1.5 iterations x
// 5 terms becomes one term plus a few additions, and no lane of the warp
// waits for another lane's rejections.  Inversion (small means) stays on one
// lane.  Every lane of the warp must call with the same arguments; every lane
// returns the same value.
#pragma once
#include "kg_device.cuh"

namespace kg {

// Binomial(n, p) by ratio of uniforms (np >= 10, p <= 1/2): binom_rou.
__device__ __forceinline__ int binom_rou_warp(uint64_t n, double p, uint64_t seed, uint64_t node,
                                              uint32_t tag, uint64_t w0, uint64_t& out) {
  constexpr int NT = 3, G = 32 / NT;  // terms per candidate, candidates per round
  const unsigned lane = threadIdx.x & 31;
  const unsigned g = lane / NT, tau = lane % NT;
  const double nd = double(n);
  const double q = 1.0 - p;
  const double mean = nd * p;
  const double var = mean * q;
  const double M = floor((nd + 1.0) * p);
  const double a = mean + 0.5;
  const double sw = RoU_D1 * sqrt(var + 0.5) + RoU_D2;
  const double lpq = kg_log(p) - kg_log1m(p);
  for (uint64_t j0 = 0; j0 < uint64_t(REJECT_CAP); j0 += G) {
    const uint64_t j = j0 + g;
    const bool live = g < unsigned(G) && j < uint64_t(REJECT_CAP);
    bool valid = false;
    double k = 0.0, term = 0.0;
    if (live) {
      const double X = u01_oc(stream_u64(seed, node, tag, w0 + 2 * j));
      const double Y = u01_co(stream_u64(seed, node, tag, w0 + 2 * j + 1));
      const double W = a + (sw * (Y - 0.5)) / X;
      valid = !(W < 0.0 || W >= nd + 1.0);
      if (valid) {
        k = floor(W);
        if (tau == 0)
          term = kg_lnfact_diff(M, k - M);
        else if (tau == 1)
          term = kg_lnfact_diff(nd - M, M - k);
        else
          term = kg_log(X);
      }
    }
    const double t1 = __shfl_down_sync(0xffffffffu, term, 1);
    const double t2 = __shfl_down_sync(0xffffffffu, term, 2);
    bool acc = false;
    if (live && tau == 0 && valid) {
      const double delta = ((k - M) * lpq - term) - t1;
      acc = t2 + t2 <= delta;
    }
    const unsigned msk = __ballot_sync(0xffffffffu, acc);
    if (msk) {
      out = uint64_t(__shfl_sync(0xffffffffu, k, __ffs(msk) - 1));
      return ST_OK;
    }
  }
  return ST_INTERNAL;
}

// Hypergeometric by ratio of uniforms (K, t <= N/2, mean >= 10): hyper_rou.
__device__ __forceinline__ int hyper_rou_warp(u128 N, u128 K, u128 t, uint64_t seed, uint64_t node,
                                              uint32_t tag, uint64_t w0, uint64_t& out) {
  constexpr int NT = 5, G = 32 / NT;
  const unsigned lane = threadIdx.x & 31;
  const unsigned g = lane / NT, tau = lane % NT;
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
  for (uint64_t j0 = 0; j0 < uint64_t(REJECT_CAP); j0 += G) {
    const uint64_t j = j0 + g;
    const bool live = g < unsigned(G) && j < uint64_t(REJECT_CAP);
    bool valid = false;
    double k = 0.0, term = 0.0;
    if (live) {
      const double X = u01_oc(stream_u64(seed, node, tag, w0 + 2 * j));
      const double Y = u01_co(stream_u64(seed, node, tag, w0 + 2 * j + 1));
      const double W = a + (sw * (Y - 0.5)) / X;
      valid = !(W < 0.0 || W >= xmax + 1.0);
      if (valid) {
        k = floor(W);
        // the four log-factorial differences share one call site
        double fa = M, fd = k - M;
        if (tau == 1) {
          fa = Kd - M;
          fd = M - k;
        } else if (tau == 2) {
          fa = td - M;
          fd = M - k;
        } else if (tau == 3) {
          fa = rest + M;
        }
        term = tau < 4 ? kg_lnfact_diff(fa, fd) : kg_log(X);
      }
    }
    const double t1 = __shfl_down_sync(0xffffffffu, term, 1);
    const double t2 = __shfl_down_sync(0xffffffffu, term, 2);
    const double t3 = __shfl_down_sync(0xffffffffu, term, 3);
    const double t4 = __shfl_down_sync(0xffffffffu, term, 4);
    bool acc = false;
    if (live && tau == 0 && valid) {
      const double delta = (((-term) - t1) - t2) - t3;
      acc = t4 + t4 <= delta;
    }
    const unsigned msk = __ballot_sync(0xffffffffu, acc);
    if (msk) {
      out = uint64_t(__shfl_sync(0xffffffffu, k, __ffs(msk) - 1));
      return ST_OK;
    }
  }
  return ST_INTERNAL;
}

// Broadcast of a lane-0 result and status to the warp.
__device__ __forceinline__ int warp_bcast(int st, uint64_t& x) {
  x = __shfl_sync(0xffffffffu, x, 0);
  return __shfl_sync(0xffffffffu, st, 0);
}

// binomial() by the warp: same branches, inversion on lane 0.
__device__ __forceinline__ int binomial_warp(uint64_t n, double p, uint64_t seed, uint64_t node,
                                             uint32_t tag, uint64_t w0, uint64_t& out,
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
  int st = ST_OK;
  if (double(n) * pp < 10.0) {
    if ((threadIdx.x & 31) == 0) {
      Stream s(seed, node, tag);
      s.next = w0;
      st = binom_inversion(n, pp, s, r);
    }
    st = warp_bcast(st, r);
  } else {
    st = binom_rou_warp(n, pp, seed, node, tag, w0, r);
  }
  if (st) return st;
  out = flip ? n - r : r;
  return ST_OK;
}

// hypergeometric() by the warp, from word 0 of the node stream.
__device__ __forceinline__ int hypergeometric_warp(u128 N, u128 K, uint64_t t, uint64_t seed,
                                                   uint64_t node, uint32_t tag, uint64_t& out) {
  HyperPlan h;
  int st = hyper_plan(N, K, t, h);
  if (st) return st;
  if (h.kind == 0) {
    out = h.fixed;
    return ST_OK;
  }
  uint64_t r = 0;
  if (h.kind == 1) {
    r = popcount_bits_warp(seed, node, tag, 0, h.t1);
  } else {
    const u128 NN = h.N, KK = h.K1;
    const uint64_t tt = h.t1;
    if ((u128(tt) << 32) <= NN) {
      st = binomial_warp(tt, dbl(KK) / dbl(NN), seed, node, tag, 0, r);
    } else if ((dbl(u128(tt)) * dbl(KK)) / dbl(NN) < 10.0) {
      if ((threadIdx.x & 31) == 0) {
        Stream s(seed, node, tag);
        st = hyper_inversion(NN, KK, u128(tt), s, r);
      }
      st = warp_bcast(st, r);
    } else {
      st = hyper_rou_warp(NN, KK, u128(tt), seed, node, tag, 0, r);
    }
    if (st) return st;
  }
  out = hyper_finish(h, r);
  return ST_OK;
}

}  // namespace kg
