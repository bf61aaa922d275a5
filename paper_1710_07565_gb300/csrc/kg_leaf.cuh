// Hot leaf kernel: Floyd's sampler on one tile per block of 256 threads.
//
// Per tile of k <= k_max samples in a universe [lo, lo + L):
//   1. draw i (uniform on [0, L-k+i], Lemire) -- thread t owns the draw pairs
//      2(t + 256 s), 2(t + 256 s) + 1 that share one Philox block; the values
//      stay in registers;
//   2. bucket b(x), monotone in x, over nb >= 2k equal-width buckets, counted
//      with shared-memory atomics on packed 16-bit counters that also hand
//      each draw its slot in the bucket;
//   3. exclusive scan of the counts (16-byte groups per thread);
//   4. scatter to A[start(b) + slot]: A is sorted up to the order inside
//      buckets;
//   5. the draw at slot 0 of every bucket with several values sorts that
//      bucket in place (mean occupancy <= 1/2, so buckets are tiny); an equal
//      pair means Floyd replaced a value;
//   6. if all draws are distinct the sample is exactly {t_i}; otherwise the
//      replacements are resolved in draw order (rare when k^2 << L);
//   7. A[r] -> (u, v) -> 16- or 8-byte stores to consecutive output slots,
//      with the order-independent digest and the row runs when asked.
#pragma once
#include <type_traits>

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

// Bucket of a draw, monotone in v: the high word of (v >> bsh) * bmul, or v
// itself when the universe has at most nb values (bmul = 0).  With
// L' = ((L-1) >> bsh) + 1 <= 2^32 and bmul = floor(2^32 nb / L'), every
// v < L lands in [0, nb) and the buckets have equal widths (up to rounding).
__device__ __forceinline__ uint32_t bucket_of(uint64_t v, uint32_t bsh, uint32_t bmul) {
  return bmul ? __umulhi(uint32_t(v >> bsh), bmul) : uint32_t(v);
}

// Buckets per tile: at least twice k (mean occupancy <= 1/2) and at least
// FAST_THREADS * 8, so that every thread owns whole 16-byte groups of packed
// 16-bit counters in the scan.
constexpr uint32_t NB_MIN = 2048;
constexpr uint32_t NB_MAX = 2 * K_MAX < NB_MIN ? NB_MIN : 2 * K_MAX;
static_assert(NB_MIN % (8 * FAST_THREADS) == 0, "whole 16-byte counter groups per thread");

// Per-tile parameters, computed for all tiles at once (tile_desc_kernel, or
// the batched engine's descriptor kernel) so that the leaf blocks start
// without a serial section.  flags: 0 = sample this tile, 1 = over k_max
// (left to the re-split kernel), 2 = nothing to do, 3 = left by the sparse
// leaf kernel to the general one (on the fallback list).  aux0 / aux1:
// per-tile constants of the directed offset map (lo mod (n-1) and the row of
// offset lo), zero for the other geometries.
template <class Ctx>
struct TileDesc {
  uint64_t lo, L, base, cid, U, W, seed;
  uint64_t aux0, aux1;
  uint32_t k, nb, tau, bmul, bsh;
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
  td.aux0 = 0;
  td.aux1 = 0;
  td.flags = 2;
  td.nb = NB_MIN;
  td.bmul = 0;
  td.bsh = 0;
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
  uint32_t nb = NB_MIN;
  while (nb < 2 * k) nb <<= 1;
  td.nb = nb;
  if (td.L > nb) {
    const int bits = 64 - __clzll(td.L - 1);  // bit length of L - 1
    td.bsh = bits > 32 ? uint32_t(bits - 32) : 0u;
    const uint64_t Lp = ((td.L - 1) >> td.bsh) + 1;  // in (nb, 2^32]
    td.bmul = uint32_t((uint64_t(nb) << 32) / Lp);
  }
}

// The sparse leaf kernel (kg_leaf_sparse.cuh) samples tiles of the directed
// geometry with at most SP_KMAX draws over SP_NB buckets; it is used where
// Floyd's replacements are rare, and leaves to the general kernel every tile
// it cannot take (flags 3, or a repeated draw found while sorting).
#ifndef KG_SP_THREADS
#define KG_SP_THREADS 256
#endif
constexpr int SP_THREADS = KG_SP_THREADS;
constexpr int SP_MIN_BLOCKS = SP_THREADS == 256 ? 5 : 6;  // resident blocks per SM
constexpr int SP_KMAX = 1536;
constexpr int SP_PAIRS = SP_KMAX / (2 * SP_THREADS);  // draw pairs per thread
constexpr uint32_t SP_NB = 2048;
constexpr int SP_CPT = int(SP_NB) / SP_THREADS;       // bucket counters per thread
static_assert(SP_CPT % 4 == 0, "whole 16-byte counter groups per thread");
static_assert(SP_KMAX % (2 * SP_THREADS) == 0, "whole draw pairs per thread");

// Which tiles of a run the sparse kernel takes (on = 0: none).  ymax = 2^(31+s)
// (saturated): the directed map's 32-bit quotient estimate needs the in-tile
// offsets y = (lo mod (n-1)) + x below it.
struct SparseRoute {
  int on;
  uint64_t ymax;
};

// The same constants for a row width D >= 4 on the device (s <= 30 keeps
// 2^(32+s) in 64 bits); false if D is out of that range.
__device__ __forceinline__ bool sparse_map_dev(uint64_t D, uint32_t& M, int& s) {
  if (D < 4 || D >= (uint64_t(1) << 32)) return false;
  s = 62 - __clzll(D);  // floor(log2 D) - 1
  M = uint32_t((uint64_t(1) << (32 + s)) / D);
  return true;
}

// Per-tile offset map of the sparse kernel for geometries whose row width
// varies by tile: offset x of the tile is y = y0 + x past the start of row
// u0; row u0 + floor(y / D), column position w = y mod D, and the column is
// w + [w >= u] (directed: the diagonal is skipped) or col0 + w (a rectangle
// of an undirected instance).
struct SparseTileMap {
  uint64_t D, y0, u0, col0;
  uint32_t M;
  int s, skip;
};

// The map of a rectangle tile of an undirected geometry (the descriptor
// kernel routes only those to the sparse kernel, with aux0 = lo mod s_j and
// aux1 = the row of lo).
__device__ __forceinline__ void sparse_tile_map(const TileDesc<UndGeom::Ctx>& td,
                                                SparseTileMap& m) {
  m.D = td.gx.sj;
  m.col0 = td.gx.rj;
  m.skip = 0;
  m.y0 = td.aux0;
  m.u0 = td.aux1;
  if (!sparse_map_dev(m.D, m.M, m.s)) {
    m.M = 0;
    m.s = 0;
  }
}

// Descriptors of tiles [0, ntiles) of chunks c_begin... .  Tiles over k_max go
// to big[0 ..) (count nbig[0]), tiles routed away from the sparse kernel to
// big[ntiles-1 ...) downwards (count nbig[1]); no tile is on both lists.
template <class Geom>
__global__ void __launch_bounds__(256)
    tile_desc_kernel(Geom g, uint64_t c_begin, int d, uint32_t k_max, uint64_t seed,
                     const uint64_t* __restrict__ tile_cnt, const uint64_t* __restrict__ tile_off,
                     uint64_t ntiles, TileDesc<typename Geom::Ctx>* __restrict__ desc,
                     unsigned long long* big, unsigned long long* nbig, int* err,
                     SparseRoute route) {
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
    if constexpr (std::is_same<Geom, DirGeom>::value) {
      // offset lo of the chunk = row q, column position lo - q (n-1)
      const uint64_t q = div_q(g.div, td.lo);
      td.aux0 = td.lo - q * (g.n - 1);
      td.aux1 = td.gx.r0 + q;
      if (route.on && td.flags == 0) {
        const bool mapok = td.aux0 < route.ymax && td.L - 1 < route.ymax - td.aux0;
        if (td.k > uint32_t(SP_KMAX) || td.L <= SP_NB || !mapok) {
          td.flags = 3;
          big[ntiles - 1 - atomicAdd(nbig + 1, 1ull)] = t;
        }
      }
    } else if constexpr (std::is_same<typename Geom::Ctx, UndGeom::Ctx>::value) {
      // undirected: rectangle tiles with valid map constants go to the sparse
      // kernel, triangles and the rest to its fallback list
      if (route.on && td.flags == 0) {
        bool ok = !td.gx.tri && td.k <= uint32_t(SP_KMAX) && td.L > SP_NB;
        if (ok) {
          uint32_t M;
          int sh;
          ok = sparse_map_dev(td.gx.sj, M, sh);
          if (ok) {
            const uint64_t q = rect_row(td.lo, td.gx.sj);
            td.aux0 = td.lo - q * td.gx.sj;
            td.aux1 = td.gx.ri + q;
            const uint64_t ymax = uint64_t(1) << (31 + sh);
            ok = td.aux0 < ymax && td.L - 1 < ymax - td.aux0;
          }
        }
        if (!ok) {
          td.flags = 3;
          big[ntiles - 1 - atomicAdd(nbig + 1, 1ull)] = t;
        }
      }
    }
    if (td.flags == 1) big[atomicAdd(nbig, 1ull)] = t;
    desc[t] = td;
  }
}

struct FastSmem {
  uint64_t A[K_MAX];             // draws scattered by bucket, then sorted in place
  uint64_t D[K_MAX];             // draws in draw order
  uint32_t hist[NB_MAX / 2 + 1]; // packed 16-bit bucket counts -> starts (+ sentinel);
                                 // per-draw 16-bit codes in the rare path
  uint32_t bitT[K_MAX / 32], bitJ[K_MAX / 32];
  uint32_t multi[K_MAX / 2];     // buckets holding several values: start | count << 16
};

// Insertion sort of A[s0, s1) (one bucket, a handful of values); returns
// whether two values are equal.
__device__ __forceinline__ int sort_bucket(uint64_t* A, uint32_t s0, uint32_t s1) {
  int dup = 0;
  for (uint32_t i = s0 + 1; i < s1; ++i) {
    const uint64_t v = A[i];
    uint32_t j = i;
    uint64_t y = A[j - 1];
    while (y > v) {
      A[j] = y;
      --j;
      if (j == s0) break;
      y = A[j - 1];
    }
    dup |= (j > s0 && A[j - 1] == v);
    A[j] = v;
  }
  return dup;
}

// TILE_SEED: every tile carries its own seed (batched instances); otherwise
// the round keys of the one seed come in as a kernel parameter.  With nlist
// set, the kernel samples only the *nlist tiles list[ntiles-1], list[ntiles-2],
// ... (the sparse kernel's fallback list; flags 0 or 3), else tiles
// [0, ntiles) with flags 0.
template <class Geom, class Sink, bool DIGEST, bool TILE_SEED>
__global__ void __launch_bounds__(FAST_THREADS, 4)
    leaf_fast_kernel(Geom g, Sink sink, int d, RoundKeys rk,
                     const TileDesc<typename Geom::Ctx>* __restrict__ desc, uint64_t ntiles,
                     int* err, DigestOut dig, const unsigned long long* __restrict__ list = nullptr,
                     const unsigned long long* __restrict__ nlist = nullptr) {
  __shared__ __align__(16) FastSmem sm;
  __shared__ unsigned bh[65];
  __shared__ unsigned long long red_d[FAST_THREADS / 32];
  __shared__ unsigned red_c1[FAST_THREADS / 32], red_nr[FAST_THREADS / 32];
  __shared__ uint64_t s_fu, s_lu;
  __shared__ uint32_t s_fl, s_ll;
  __shared__ unsigned s_nmulti;
  using Desc = TileDesc<typename Geom::Ctx>;
  // the descriptors of this tile and the next one, staged in shared memory so
  // that their fields are read where they are used instead of being held in
  // registers for the whole tile
  __shared__ __align__(16) Desc s_td[2];
  const int tid = threadIdx.x;
  uint16_t* const st16 = reinterpret_cast<uint16_t*>(sm.hist);
  auto stage = [&](uint64_t tt, int slot) {
    static_assert(sizeof(Desc) % 4 == 0, "descriptor size");
    const uint32_t* src = reinterpret_cast<const uint32_t*>(desc + tt);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&s_td[slot]);
    for (uint32_t w = tid; w < sizeof(Desc) / 4; w += FAST_THREADS) dst[w] = src[w];
  };

  const uint64_t count = nlist ? uint64_t(*nlist) : ntiles;
  auto tile_at = [&](uint64_t i) { return nlist ? uint64_t(list[ntiles - 1 - i]) : i; };
  for (uint32_t b = tid; b < NB_MAX / 2 + 1; b += FAST_THREADS) sm.hist[b] = 0;
  if (blockIdx.x < count) stage(tile_at(blockIdx.x), 0);
  __syncthreads();
  int cur = 0;
  for (uint64_t it = blockIdx.x; it < count; it += gridDim.x, cur ^= 1) {
    const Desc& td = s_td[cur];
    const uint64_t t = tile_at(it);
    const uint64_t itn = it + gridDim.x;
    const bool take = td.flags == 0 || (nlist && td.flags == 3);
    if (!take || !sink.fits(td.base, td.k)) {  // uniform over the block
      if (take && tid == 0) set_error(err, ST_CAPACITY);  // the tile is dropped
      if (itn < count) stage(tile_at(itn), cur ^ 1);
      __syncthreads();
      continue;
    }
    const uint32_t k = td.k, nb = td.nb, bsh = td.bsh, bmul = td.bmul;
    const uint64_t Lk = td.L - k, node = td.node(td.d, td.tau);
    const uint64_t seed = td.seed;

    // ---- 1./2. draws, staged in D in draw order; bucket counts, and each
    // draw's slot in its bucket (kept in registers)
    uint32_t bs[2 * FAST_PAIRS];  // bucket | slot << 16
    // Lemire's rejection test is done in the loop, the rejected draws (below
    // L / 2^64 per draw) are redrawn after it, so that the retry code adds no
    // live registers to the loop
    uint32_t rejm = 0;
#pragma unroll
    for (int s = 0; s < FAST_PAIRS; ++s) {
      const uint32_t i = 2 * (tid + FAST_THREADS * s);
      if (i < k) {
        uint32_t w[4];
        if (TILE_SEED)
          philox10(i >> 1, uint32_t(node), uint32_t(node >> 32), TAG_LEAF, uint32_t(seed),
                   uint32_t(seed >> 32), w);
        else
          philox10_rk(i >> 1, uint32_t(node), uint32_t(node >> 32), TAG_LEAF, rk, w);
        const uint64_t a = (uint64_t(w[0]) << 32) | w[1], c = (uint64_t(w[2]) << 32) | w[3];
        const uint64_t r0 = Lk + i + 1, r1 = r0 + 1;
        const uint64_t x0 = mul_hi64(a, r0), x1 = mul_hi64(c, r1);
        const bool ok0 = a * r0 >= r0, ok1 = c * r1 >= r1;
        rejm |= (ok0 ? 0u : 1u << (2 * s)) | ((ok1 || i + 1 >= k) ? 0u : 2u << (2 * s));
        if (ok0) {
          const uint32_t b0 = bucket_of(x0, bsh, bmul);
          const uint32_t sh0 = (b0 & 1) << 4;
          const uint32_t old0 = atomicAdd(&sm.hist[b0 >> 1], 1u << sh0);
          bs[2 * s] = b0 | (((old0 >> sh0) & 0xffffu) << 16);
        }
        if (i + 1 < k) {
          if (ok1) {
            const uint32_t b1 = bucket_of(x1, bsh, bmul);
            const uint32_t sh1 = (b1 & 1) << 4;
            const uint32_t old1 = atomicAdd(&sm.hist[b1 >> 1], 1u << sh1);
            bs[2 * s + 1] = b1 | (((old1 >> sh1) & 0xffffu) << 16);
          }
          reinterpret_cast<ulonglong2*>(sm.D)[i >> 1] = make_ulonglong2(x0, x1);
        } else {
          sm.D[i] = x0;
        }
      }
    }
    if (rejm) {
#pragma unroll
      for (int j = 0; j < 2 * FAST_PAIRS; ++j)
        if (rejm & (1u << j)) {
          const uint32_t i = 2 * (tid + FAST_THREADS * (j >> 1)) + (j & 1);
          const uint64_t x = lemire_draw(stream_u64(seed, node, TAG_LEAF, i), Lk + i + 1, seed,
                                         node, i);
          const uint32_t b = bucket_of(x, bsh, bmul);
          const uint32_t sh = (b & 1) << 4;
          const uint32_t old = atomicAdd(&sm.hist[b >> 1], 1u << sh);
          bs[j] = b | (((old >> sh) & 0xffffu) << 16);
          sm.D[i] = x;
        }
    }
    __syncthreads();
    // every thread is past the previous tile: its descriptor slot takes the
    // next tile's (DIGEST: the barriers below publish it, so the tile ends
    // without one of its own)
    if (DIGEST && itn < count) stage(tile_at(itn), cur ^ 1);
    // ---- 3. exclusive scan of the packed counts: thread tid owns words
    // [tid*per, tid*per + per), per = nb / (2 FAST_THREADS) in {4, 8, ...}
    {
      const uint32_t per4 = nb / (8 * FAST_THREADS);  // uint4 groups per thread
      uint4* h4 = reinterpret_cast<uint4*>(sm.hist) + tid * per4;
      uint32_t sum = 0;
      for (uint32_t q = 0; q < per4; ++q) {
        const uint4 a = h4[q];
        sum += (a.x & 0xffffu) + (a.x >> 16) + (a.y & 0xffffu) + (a.y >> 16) +
               (a.z & 0xffffu) + (a.z >> 16) + (a.w & 0xffffu) + (a.w >> 16);
      }
      uint32_t tot;
      uint32_t run = block_inclusive_scan<FAST_THREADS>(sum, tot) - sum;
      for (uint32_t q = 0; q < per4; ++q) {
        uint4 a = h4[q];
        uint32_t c;
        c = (a.x & 0xffffu) + (a.x >> 16); a.x = run * 0x10001u + (a.x << 16); run += c;
        c = (a.y & 0xffffu) + (a.y >> 16); a.y = run * 0x10001u + (a.y << 16); run += c;
        c = (a.z & 0xffffu) + (a.z >> 16); a.z = run * 0x10001u + (a.z << 16); run += c;
        c = (a.w & 0xffffu) + (a.w >> 16); a.w = run * 0x10001u + (a.w << 16); run += c;
        h4[q] = a;
      }
      if (tid == 0) {
        sm.hist[nb >> 1] = k;  // start of the (absent) bucket nb
        s_nmulti = 0;
      }
      if (DIGEST)
        for (int b = tid; b < 65; b += FAST_THREADS) bh[b] = 0;
    }
    __syncthreads();  // bucket starts visible
    // ---- 4. scatter D[i] to A[start(b) + slot] (the bucket's values land in
    // [start(b), start(b+1)) in arbitrary order)
    {
      // the draw at slot 0 of a bucket with several values lists that bucket
      // (warp-aggregated append), so that the sorting below runs over a
      // compact list instead of diverging inside every warp
      const int lane = tid & 31;
#pragma unroll
      for (int s = 0; s < FAST_PAIRS; ++s) {
        const uint32_t i = 2 * (tid + FAST_THREADS * s);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          uint32_t item = 0;
          if (i + h < k) {
            const uint32_t v = bs[2 * s + h];
            const uint32_t b = v & 0xffffu, s0 = st16[b];
            sm.A[s0 + (v >> 16)] = sm.D[i + h];
            if ((v >> 16) == 0) {
              const uint32_t c = st16[b + 1] - s0;
              if (c > 1) item = s0 | (c << 16);
            }
          }
          if (2 * (FAST_THREADS * s) + h < k) {  // warp-uniform: some lane of the block is active
            const unsigned m = __ballot_sync(0xffffffffu, item != 0);
            if (m) {
              unsigned at = 0;
              if (lane == __ffs(m) - 1) at = atomicAdd(&s_nmulti, unsigned(__popc(m)));
              at = __shfl_sync(0xffffffffu, at, __ffs(m) - 1);
              if (item) sm.multi[at + __popc(m & ((1u << lane) - 1))] = item;
            }
          }
        }
      }
    }
    __syncthreads();
    // ---- 5. sort every listed bucket in place (mean occupancy <= 1/2: mostly
    // pairs); equal values mean Floyd replaced a draw
    int dup = 0;
    const uint32_t nmulti = s_nmulti;
    for (uint32_t e = tid; e < nmulti; e += FAST_THREADS) {
      const uint32_t item = sm.multi[e];
      const uint32_t s0 = item & 0xffffu, c = item >> 16;
      if (c == 2) {
        const uint64_t a = sm.A[s0], b = sm.A[s0 + 1];
        if (b < a) {
          sm.A[s0] = b;
          sm.A[s0 + 1] = a;
        }
        dup |= (a == b);
      } else if (c <= 4) {  // four loads at once, a 5-exchange network, c stores
        uint64_t y[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) y[q] = uint32_t(q) < c ? sm.A[s0 + q] : ~uint64_t(0);
        auto cx = [](uint64_t& a, uint64_t& b) {
          const uint64_t lo_ = a < b ? a : b, hi_ = a < b ? b : a;
          a = lo_;
          b = hi_;
        };
        cx(y[0], y[1]);
        cx(y[2], y[3]);
        cx(y[0], y[2]);
        cx(y[1], y[3]);
        cx(y[1], y[2]);
        dup |= (y[0] == y[1]) | (y[1] == y[2] && c > 2) | (y[2] == y[3] && c > 3);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (uint32_t(q) < c) sm.A[s0 + q] = y[q];
      } else {
        dup |= sort_bucket(sm.A, s0, s0 + c);
      }
    }
    const int any_dup = __syncthreads_or(dup);
    uint64_t* res = sm.A;
    if (any_dup) {
      // ---- 6. Floyd's replacements, resolved in parallel.  Draw i inserts
      // t_i unless t_i is already taken, else j_i = L-k+i (never taken
      // before step i).  A value below L-k can only be taken by a draw of
      // itself, so there the first draw of the value (in draw order) keeps
      // it and later ones are replaced.  A value v >= L-k is also the
      // replacement of draw p = v-(L-k) <= i: its first draw keeps it
      // exactly when draw p kept its own value (p = i: always), which chains
      // through earlier draws and is settled in rounds.  The kept values
      // below L-k are then compacted in sorted order, followed by the taken
      // values of [L-k, L) from a bitmap.
      uint32_t* first = sm.hist;                                   // per sorted position
      volatile uint8_t* status = reinterpret_cast<uint8_t*>(sm.multi);  // per draw: 0 keep,
                                                                   // 1 replaced, 2 open
      for (uint32_t r = tid; r < k; r += FAST_THREADS) first[r] = 0xffffffffu;
      for (uint32_t w = tid; w < K_MAX / 32; w += FAST_THREADS) sm.bitT[w] = sm.bitJ[w] = 0;
      __syncthreads();
      auto first_pos = [&](uint64_t v) {  // first sorted position of v
        uint32_t a = 0, e = k;
        while (a < e) {
          const uint32_t mid = (a + e) >> 1;
          if (sm.A[mid] < v)
            a = mid + 1;
          else
            e = mid;
        }
        return a;
      };
      for (uint32_t i = tid; i < k; i += FAST_THREADS) atomicMin(&first[first_pos(sm.D[i])], i);
      __syncthreads();
      for (uint32_t i = tid; i < k; i += FAST_THREADS) {
        const uint64_t v = sm.D[i];
        const bool is_first = first[first_pos(v)] == i;
        uint8_t st;
        if (!is_first)
          st = 1;
        else if (v < Lk || v - Lk == i)
          st = 0;
        else
          st = 2;
        status[i] = st;
      }
      __syncthreads();
      for (;;) {
        int open = 0;
        for (uint32_t i = tid; i < k; i += FAST_THREADS)
          if (status[i] == 2) {
            const uint8_t sp = status[uint32_t(sm.D[i] - Lk)];
            if (sp != 2)
              status[i] = sp;
            else
              open = 1;
          }
        if (!__syncthreads_or(open)) break;
      }
      for (uint32_t i = tid; i < k; i += FAST_THREADS) {
        const uint64_t v = sm.D[i];
        if (status[i]) {
          atomicOr(&sm.bitJ[i >> 5], 1u << (i & 31));  // j_i = L-k+i
        } else if (v >= Lk) {
          const uint32_t b = uint32_t(v - Lk);
          atomicOr(&sm.bitJ[b >> 5], 1u << (b & 31));
        } else {
          const uint32_t fp = first_pos(v);
          atomicOr(&sm.bitT[fp >> 5], 1u << (fp & 31));
        }
      }
      __syncthreads();
      // compaction into D: kept values below L-k (marked sorted positions),
      // then L-k + b for the marked b; word counts scanned by the block
      const uint32_t nw = (k + 31) >> 5;
      uint32_t cT = 0, cJ = 0;
      if (tid < nw) {
        cT = __popc(sm.bitT[tid]);
        cJ = __popc(sm.bitJ[tid]);
      }
      uint32_t totT, totJ;
      const uint32_t offT = block_inclusive_scan<FAST_THREADS>(cT, totT) - cT;
      const uint32_t offJ = block_inclusive_scan<FAST_THREADS>(cJ, totJ) - cJ;
      if (tid < nw) {
        uint32_t wT = sm.bitT[tid], wJ = sm.bitJ[tid], oT = offT, oJ = totT + offJ;
        while (wT) {
          const int b = __ffs(wT) - 1;
          wT &= wT - 1;
          sm.D[oT++] = sm.A[tid * 32 + b];
        }
        while (wJ) {
          const int b = __ffs(wJ) - 1;
          wJ &= wJ - 1;
          if (oJ < k) sm.D[oJ] = Lk + tid * 32 + b;
          ++oJ;
        }
      }
      if (tid == 0 && totT + totJ != k) set_error(err, ST_INTERNAL);
      res = sm.D;
      __syncthreads();
    }
    // the bucket counters are dead from here on: clear them for the next tile
    {
      const uint32_t per4 = nb / (8 * FAST_THREADS);
      uint4* h4 = reinterpret_cast<uint4*>(sm.hist) + tid * per4;
      for (uint32_t q = 0; q < per4; ++q) h4[q] = make_uint4(0, 0, 0, 0);
      if (tid == 0) sm.hist[nb >> 1] = 0;
    }
    // ---- 7. emit; lane l of warp w takes r = r0 + 32 w + l, so that every
    // warp holds 32 consecutive sorted edges.  DIGEST: the order-independent
    // digest, and the runs of equal rows u.  Offset x is in the row of x' < x
    // iff lo + x' >= the first offset of x's row, and x'' > x is iff
    // lo + x'' < that row's end (Geom::row_span); the neighbours' offsets are
    // read from A, so no division, no barrier and no stored rows are needed;
    // a run longer than one is measured by a scan of A from its start.
    unsigned long long dsum = 0;
    uint32_t c1 = 0, nr = 0;
    const uint64_t lo = td.lo, base = td.base;
    const typename Geom::Ctx gx = td.gx;
    const int lane = tid & 31;
    if constexpr (!DIGEST) {
      for (uint32_t r = tid; r < k; r += FAST_THREADS) {
        uint64_t u, v;
        g.map(gx, lo + res[r], u, v);
        sink.put(base + r, u, v);
      }
    } else {
      for (uint32_t r = tid; r < k; r += FAST_THREADS) {
        const uint64_t x = res[r];
        const uint64_t xp = r > 0 ? res[r - 1] : 0;  // the neighbours' offsets
        const uint64_t xn = r + 1 < k ? res[r + 1] : 0;
        {
          uint64_t u, v;
          g.map(gx, lo + x, u, v);
          sink.put(base + r, u, v);
          dsum += edge_hash(u, v);
          uint64_t rs, rl;  // the row's first offset and its length
          g.row_span(gx, lo + x, u, v, rs, rl);
          const uint64_t re = rs + rl;
          const bool st = r == 0 || lo + xp < rs;     // a run of row u starts at r
          const bool en = r + 1 == k || lo + xn >= re;  // ... and ends at r
          nr += st;
          c1 += st & en & (r != 0) & (r + 1 != k);     // one-edge runs inside the tile
          if (st & !en) {  // a run of two or more edges (rare when rows are sparse)
            uint32_t q = r + 2;
            while (q < k && lo + res[q] < re) ++q;
            const uint32_t len = q - r;
            const bool first = (r == 0), last = (q == k);
            if (first) {
              s_fu = u;
              s_fl = len;
            }
            if (last) {
              s_lu = u;
              s_ll = len;
            }
            if (!first && !last) atomicAdd(&bh[len < 64 ? len : 64], 1u);
          } else if (st & ((r == 0) | (r + 1 == k))) {  // a one-edge run at a tile end
            if (r == 0) {
              s_fu = u;
              s_fl = 1;
            }
            if (r + 1 == k) {
              s_lu = u;
              s_ll = 1;
            }
          }
        }
      }
      // block totals (FAST_THREADS threads)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
        c1 += __shfl_xor_sync(0xffffffffu, c1, o);
        nr += __shfl_xor_sync(0xffffffffu, nr, o);
      }
      const int wid = tid >> 5;
      if (lane == 0) {
        red_d[wid] = dsum;
        red_c1[wid] = c1;
        red_nr[wid] = nr;
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
    if constexpr (!DIGEST) {
      // the emission read A / D, which the next tile's draws overwrite
      if (itn < count) stage(tile_at(itn), cur ^ 1);
      __syncthreads();
    }
  }
}

}  // namespace kg
