// Hot leaf kernel: Floyd's sampler on one tile per block of 128 threads.
//
// Per tile of k <= k_max samples in a universe [lo, lo + L):
//   1. draw i (uniform on [0, L-k+i], Lemire) -- thread t owns the draw pairs
//      2(t + 128 s), 2(t + 128 s) + 1 that share one Philox block; the values
//      stay in registers;
//   2. bucket b(x) = floor(x nb / L) (a multiplier, monotone in x), counted
//      with shared-memory atomics that also hand each draw its slot;
//   3. exclusive scan of the bucket counts; scatter into A;
//   4. each draw's final rank = bucket start + #{smaller values in its bucket}
//      + #{equal values at a lower slot}; written to B -- B is the sorted
//      multiset, and any equal pair means Floyd replaced a value;
//   5. if all draws are distinct the sample is exactly {t_i}; otherwise the
//      replacements are resolved in draw order (rare when k^2 << L);
//   6. B[r] -> (u, v) -> 16- or 8-byte stores to consecutive output slots.
#pragma once
#include "kg_gnm.cuh"

namespace kg {

constexpr int FAST_THREADS = 256;
constexpr int FAST_PAIRS = K_MAX / (2 * FAST_THREADS);  // draw pairs per thread at k_max

// Philox round keys of one seed: key + r * Weyl constant, r = 0..9.
struct RoundKeys {
  uint32_t k0[10], k1[10];
};
inline RoundKeys round_keys(uint64_t seed) {
  RoundKeys rk;
  uint32_t a = uint32_t(seed), b = uint32_t(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    rk.k0[r] = a;
    rk.k1[r] = b;
    a += 0x9E3779B9u;
    b += 0xBB67AE85u;
  }
  return rk;
}

// Philox4x32-10 with precomputed round keys (same function as philox10).
__device__ __forceinline__ void philox10_rk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                            const RoundKeys& rk, uint32_t w[4]) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = uint64_t(0xD2511F53u) * c0;
    const uint64_t p1 = uint64_t(0xCD9E8D57u) * c2;
    const uint32_t n0 = uint32_t(p1 >> 32) ^ c1 ^ rk.k0[r];
    const uint32_t n2 = uint32_t(p0 >> 32) ^ c3 ^ rk.k1[r];
    c1 = uint32_t(p1);
    c3 = uint32_t(p0);
    c0 = n0;
    c2 = n2;
  }
  w[0] = c0;
  w[1] = c1;
  w[2] = c2;
  w[3] = c3;
}

// Bucket of a draw: floor(v * nbmul / 2^64) clamped to nb-1, or v itself
// when the universe has at most nb values.  Monotone in v.
__device__ __forceinline__ uint32_t bucket_of(uint64_t v, uint64_t nbmul, uint32_t nb) {
  if (!nbmul) return uint32_t(v);
  const uint64_t q = __umul64hi(v, nbmul);
  return q < nb ? uint32_t(q) : nb - 1;
}

// Per-tile parameters, computed for all tiles at once (tile_desc_kernel, or
// the batched engine's descriptor kernel) so that the leaf blocks start
// without a serial section.  flags: 0 = sample this tile, 1 = over k_max
// (left to the re-split kernel), 2 = nothing to do.
template <class Ctx>
struct TileDesc {
  uint64_t lo, L, base, cid, nbmul, U, W, seed;
  uint32_t k, nb, tau;
  int d, flags;
  Ctx gx;
  __host__ __device__ __forceinline__ uint64_t node(int level, uint64_t j) const {
    return (cid << 32) | ((uint64_t(1) << level) + j);
  }
};

// Fills the tile fields from (U, d, tau, k); the caller sets base, cid, seed, gx.
template <class Ctx>
__device__ __forceinline__ void desc_fill(TileDesc<Ctx>& td, uint64_t U, int d, uint64_t tau,
                                          uint64_t k, uint32_t k_max, int* err) {
  td.U = U;
  td.d = d;
  td.tau = uint32_t(tau);
  td.W = tile_width(U, d);
  td.lo = node_bound(U, td.W, d, d, tau);
  td.L = node_bound(U, td.W, d, d, u128(tau) + 1) - td.lo;
  td.k = uint32_t(k > 0xffffffffull ? 0xffffffffull : k);
  td.flags = 2;
  if (k == 0) return;
  if (k > 0xffffffffull) {
    set_error(err, ST_INTERNAL);
    return;
  }
  if (k > td.L) {
    set_error(err, ST_INTERNAL);
    return;
  }
  if (k > k_max) {
    td.flags = 1;
    return;
  }
  td.flags = 0;
  uint32_t nb = 32;
  while (nb < k) nb <<= 1;
  td.nb = nb;
  // bucket multiplier floor(2^64 nb / L) (0 means: bucket = value)
  td.nbmul = (td.L <= nb) ? 0 : uint64_t(double(nb) * 0x1p64 / double(td.L));
}

template <class Geom>
__global__ void __launch_bounds__(256)
    tile_desc_kernel(Geom g, uint64_t c_begin, int d, uint32_t k_max, uint64_t seed,
                     const uint64_t* __restrict__ tile_cnt, const uint64_t* __restrict__ tile_off,
                     uint64_t ntiles, TileDesc<typename Geom::Ctx>* __restrict__ desc,
                     unsigned long long* big, unsigned long long* nbig, int* err) {
  for (uint64_t t = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < ntiles;
       t += uint64_t(gridDim.x) * blockDim.x) {
    TileDesc<typename Geom::Ctx> td;
    const uint64_t c = c_begin + (t >> d);
    const uint64_t tau = t & ((uint64_t(1) << d) - 1);
    desc_fill(td, g.universe(c), d, tau, tile_cnt[t], k_max, err);
    td.base = tile_off[t];
    td.cid = g.chunk_id(c);
    td.seed = seed;
    td.gx = g.ctx(c);
    if (td.flags == 1) big[atomicAdd(nbig, 1ull)] = t;
    desc[t] = td;
  }
}

struct FastSmem {
  uint64_t A[K_MAX];          // draws scattered by bucket, then sorted in place;
                              // with DIGEST the rows u afterwards
  uint16_t hist[K_MAX + 2];   // bucket counts -> starts; per-draw codes in the rare path
  uint32_t bitT[K_MAX / 32], bitJ[K_MAX / 32];
};

// TILE_SEED: every tile carries its own seed (batched instances); otherwise
// the round keys of the one seed come in as a kernel parameter.
template <class Geom, class Sink, bool DIGEST, bool TILE_SEED>
__global__ void __launch_bounds__(FAST_THREADS, 5)
    leaf_fast_kernel(Geom g, Sink sink, int d, RoundKeys rk,
                     const TileDesc<typename Geom::Ctx>* __restrict__ desc, uint64_t ntiles,
                     int* err, DigestOut dig) {
  __shared__ FastSmem sm;
  __shared__ unsigned bh[65];
  __shared__ unsigned long long red_d[FAST_THREADS / 32];
  __shared__ unsigned red_c1[FAST_THREADS / 32], red_nr[FAST_THREADS / 32];
  __shared__ uint64_t s_fu, s_lu;
  __shared__ uint32_t s_fl, s_ll;
  const int tid = threadIdx.x;

  for (uint32_t b = tid; b < (K_MAX + 2) / 2; b += FAST_THREADS)
    reinterpret_cast<unsigned*>(sm.hist)[b] = 0;
  __syncthreads();
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const TileDesc<typename Geom::Ctx> td = desc[t];
    if (td.flags != 0) continue;  // uniform over the block
    const uint32_t k = td.k, nb = td.nb;
    const uint64_t L = td.L, Lk = L - k, node = td.node(td.d, td.tau), nbmul = td.nbmul;
    const uint64_t seed = td.seed;

    // ---- 1./2. draws in registers, bucket counts and slots
    uint64_t x[2 * FAST_PAIRS];
    uint32_t slot[2 * FAST_PAIRS];
#pragma unroll
    for (int s = 0; s < FAST_PAIRS; ++s) {
      const uint32_t i = 2 * (tid + FAST_THREADS * s);
      if (i >= k) break;
      uint32_t w[4];
      if (TILE_SEED)
        philox10(i >> 1, uint32_t(node), uint32_t(node >> 32), TAG_LEAF, uint32_t(seed),
                 uint32_t(seed >> 32), w);
      else
        philox10_rk(i >> 1, uint32_t(node), uint32_t(node >> 32), TAG_LEAF, rk, w);
      x[2 * s] = lemire_draw((uint64_t(w[0]) << 32) | w[1], Lk + i + 1, seed, node, i);
      x[2 * s + 1] = (i + 1 < k)
                         ? lemire_draw((uint64_t(w[2]) << 32) | w[3], Lk + i + 2, seed, node, i + 1)
                         : 0;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (i + h < k) {
          const uint64_t v = x[2 * s + h];
          slot[2 * s + h] = bucket_of(v, nbmul, nb);
        }
      }
    }
    // bucket counts: 16-bit counters packed in pairs, updated with 32-bit atomics
    unsigned* h32 = reinterpret_cast<unsigned*>(sm.hist);
#pragma unroll
    for (int s = 0; s < FAST_PAIRS; ++s) {
      const uint32_t i = 2 * (tid + FAST_THREADS * s);
      if (i >= k) break;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (i + h < k) {
          const uint32_t b = slot[2 * s + h];
          const unsigned old = atomicAdd(&h32[b >> 1], (b & 1) ? 0x10000u : 1u);
          // keep bucket in the low 16 bits, the within-bucket slot above
          slot[2 * s + h] = b | (((b & 1) ? (old >> 16) : (old & 0xffffu)) << 16);
        }
      }
    }
    __syncthreads();
    // ---- 3. exclusive scan of hist[0..nb) in place, hist[nb] = k
    {
      const uint32_t per = (nb + FAST_THREADS - 1) / FAST_THREADS;
      const uint32_t b0 = tid * per;
      uint32_t s = 0;
      for (uint32_t q = 0; q < per; ++q)
        if (b0 + q < nb) s += sm.hist[b0 + q];
      uint32_t tot;
      uint32_t run = block_inclusive_scan<FAST_THREADS>(s, tot) - s;
      for (uint32_t q = 0; q < per; ++q)
        if (b0 + q < nb) {
          const uint32_t c = sm.hist[b0 + q];
          sm.hist[b0 + q] = uint16_t(run);
          run += c;
        }
      if (tid == 0) sm.hist[nb] = uint16_t(k);
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < FAST_PAIRS; ++s) {
      const uint32_t i = 2 * (tid + FAST_THREADS * s);
      if (i >= k) break;
#pragma unroll
      for (int h = 0; h < 2; ++h)
        if (i + h < k) {
          const uint32_t b = slot[2 * s + h] & 0xffffu;
          const uint32_t p = sm.hist[b] + (slot[2 * s + h] >> 16);
          sm.A[p] = x[2 * s + h];
          slot[2 * s + h] = b | (p << 16);  // bucket and scatter position
        }
    }
    __syncthreads();
    // ---- 4. rank inside the bucket (ties by scatter position); the rank lies
    // in the bucket's own slot range, so after a barrier the values are
    // written back in place
    int dup = 0;
    uint32_t rank[2 * FAST_PAIRS];
#pragma unroll
    for (int s = 0; s < FAST_PAIRS; ++s) {
      const uint32_t i = 2 * (tid + FAST_THREADS * s);
      if (i >= k) break;
#pragma unroll
      for (int h = 0; h < 2; ++h)
        if (i + h < k) {
          const uint64_t v = x[2 * s + h];
          const uint32_t p = slot[2 * s + h] >> 16;
          const uint32_t b = slot[2 * s + h] & 0xffffu;
          const uint32_t s0 = sm.hist[b], s1 = sm.hist[b + 1];
          uint32_t r = s0;
          for (uint32_t q = s0; q < s1; ++q) {
            const uint64_t y = sm.A[q];
            r += (y < v) || (y == v && q < p);
            dup |= (y == v && q != p);
          }
          rank[2 * s + h] = r;
        }
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < FAST_PAIRS; ++s) {
      const uint32_t i = 2 * (tid + FAST_THREADS * s);
      if (i >= k) break;
#pragma unroll
      for (int h = 0; h < 2; ++h)
        if (i + h < k) sm.A[rank[2 * s + h]] = x[2 * s + h];
    }
    const int any_dup = __syncthreads_or(dup);
    uint64_t* res = sm.A;
    if (any_dup) {
      // ---- 5. sequential resolution in draw order.  A value v < L-k can only
      // be taken by an earlier draw of v itself (first occurrence wins); the
      // values L-k .. L-1 are tracked in a bitmap because replacements land
      // there.  Per draw a 16-bit code: the first sorted position of v, or
      // 0x8000 | (v - (L-k)) for the top k values.
#pragma unroll
      for (int s = 0; s < FAST_PAIRS; ++s) {
        const uint32_t i = 2 * (tid + FAST_THREADS * s);
        if (i >= k) break;
#pragma unroll
        for (int h = 0; h < 2; ++h)
          if (i + h < k) {
            const uint64_t v = x[2 * s + h];
            uint16_t code;
            if (v >= Lk) {
              code = uint16_t(0x8000u | uint32_t(v - Lk));
            } else {
              uint32_t a = 0, e = k;
              while (a < e) {
                const uint32_t mid = (a + e) >> 1;
                if (sm.A[mid] < v)
                  a = mid + 1;
                else
                  e = mid;
              }
              code = uint16_t(a);
            }
            sm.hist[i + h] = code;
          }
      }
      for (uint32_t w = tid; w < K_MAX / 32; w += FAST_THREADS) sm.bitT[w] = sm.bitJ[w] = 0;
      __syncthreads();
      if (tid == 0) {
        for (uint32_t i = 0; i < k; ++i) {
          const uint32_t code = sm.hist[i];
          if (!(code & 0x8000u)) {
            const uint32_t fp = code;
            if (sm.bitT[fp >> 5] & (1u << (fp & 31)))
              sm.bitJ[i >> 5] |= 1u << (i & 31);
            else
              sm.bitT[fp >> 5] |= 1u << (fp & 31);
          } else {
            const uint32_t bj = code & 0x7fffu;
            if (sm.bitJ[bj >> 5] & (1u << (bj & 31)))
              sm.bitJ[i >> 5] |= 1u << (i & 31);
            else
              sm.bitJ[bj >> 5] |= 1u << (bj & 31);
          }
        }
        // the taken set in increasing order, compacted in place (the write
        // index never passes the read index)
        uint32_t o = 0;
        uint64_t prev = 0;
        for (uint32_t r = 0; r < k; ++r) {
          const uint64_t v = sm.A[r];
          if (v >= Lk) break;
          const bool first = (r == 0 || prev != v);
          prev = v;
          if (first && (sm.bitT[r >> 5] & (1u << (r & 31)))) sm.A[o++] = v;
        }
        for (uint32_t bj = 0; bj < k; ++bj)
          if (sm.bitJ[bj >> 5] & (1u << (bj & 31))) {
            if (o < k) sm.A[o] = Lk + bj;
            ++o;
          }
        if (o != k) set_error(err, ST_INTERNAL);
      }
      __syncthreads();
    }
    // ---- 6. emit
    unsigned long long dsum = 0;
    const uint64_t lo = td.lo, base = td.base;
    const typename Geom::Ctx gx = td.gx;
    for (uint32_t r = tid; r < k; r += FAST_THREADS) {
      uint64_t u, v;
      g.map(gx, lo + res[r], u, v);
      sink.write(base + r, u, v);
      if (DIGEST) {
        dsum += edge_hash(u, v);
        res[r] = u;
      }
    }
    if (DIGEST) {
      for (int b = tid; b < 65; b += FAST_THREADS) bh[b] = 0;
      __syncthreads();
      uint32_t c1 = 0, nr = 0, fl = 0, ll = 0;
      uint64_t fu = 0, lu = 0;
      for (uint32_t r = tid; r < k; r += FAST_THREADS) {
        const uint64_t u = res[r];
        if (r > 0 && res[r - 1] == u) continue;
        uint32_t len = 1;
        while (r + len < k && res[r + len] == u) ++len;
        ++nr;
        const bool first = (r == 0), last = (r + len == k);
        if (first) {
          fu = u;
          fl = len;
        }
        if (last) {
          lu = u;
          ll = len;
        }
        if (!first && !last) {
          if (len == 1)
            ++c1;
          else
            atomicAdd(&bh[len < 64 ? len : 64], 1u);
        }
      }
      // block totals (FAST_THREADS threads)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
        c1 += __shfl_xor_sync(0xffffffffu, c1, o);
        nr += __shfl_xor_sync(0xffffffffu, nr, o);
      }
      const int lane = tid & 31, wid = tid >> 5;
      if (lane == 0) {
        red_d[wid] = dsum;
        red_c1[wid] = c1;
        red_nr[wid] = nr;
      }
      if (fl) {
        s_fu = fu;
        s_fl = fl;
      }
      if (ll) {
        s_lu = lu;
        s_ll = ll;
      }
      __syncthreads();
      const uint64_t cl = t >> d;
      if (tid == 0) {
        unsigned long long D = 0;
        unsigned C1 = 0, NR = 0;
        for (int w = 0; w < FAST_THREADS / 32; ++w) {
          D += red_d[w];
          C1 += red_c1[w];
          NR += red_nr[w];
        }
        atomicAdd(&dig.digest[cl], D);
        if (C1) atomicAdd(&dig.hist[cl * 65 + 1], (unsigned long long)C1);
        TileRec rc;
        rc.first_u = s_fu;
        rc.first_len = s_fl;
        rc.last_u = s_lu;
        rc.last_len = s_ll;
        rc.nruns = NR;
        rc.pad = 0;
        dig.rec[t] = rc;
      }
      for (int b = tid; b < 65; b += FAST_THREADS)
        if (bh[b]) atomicAdd(&dig.hist[cl * 65 + b], (unsigned long long)bh[b]);
    }
    // clear the bucket counters for the next tile (all of them: the rare path
    // reuses the array)
    for (uint32_t b = tid; b < (K_MAX + 2) / 2; b += FAST_THREADS)
      reinterpret_cast<unsigned*>(sm.hist)[b] = 0;
    __syncthreads();
  }
}

}  // namespace kg
