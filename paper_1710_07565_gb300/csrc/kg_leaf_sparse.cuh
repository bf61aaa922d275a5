// Leaf kernel for sparse directed tiles: Floyd's sampler (the sequential base
// case of Sec. 2.2) on one tile per block of 256 threads, for tiles whose
// draws almost never repeat (k^2 << L, e.g. n = 2^36 with ~1024 samples in
// 2^49 pairs per tile).  It computes the same sample as leaf_fast_kernel with
// fewer instructions per edge:
//   1. draws as in leaf_fast_kernel (thread t owns the draw pairs
//      2(t + 256 s), +1, one Philox block each), bucketed over SP_NB = 2048
//      equal-width buckets by shared-memory atomics on 32-bit counters that
//      hand each draw its slot in its bucket;
//   2. one block scan turns the counts into bucket starts and, in the same
//      pass, lists the buckets holding several draws (no atomics, no ballots);
//   3. scatter to A[start + slot], then the listed buckets are sorted in
//      place; an equal pair means Floyd would replace a draw: such a tile
//      goes to the fallback list and the general kernel samples it;
//   4. emission: the offset map of Sec. 4.1 by a 32-bit quotient estimate
//      with one exact correction (the tile's first row and column come from
//      its descriptor), 16- or 8-byte stores to consecutive slots; with the
//      digest, a row run starts where the previous offset lies more than the
//      column position below, and ends where the next one lies at least the
//      rest of the row above, so no second pass over the rows is needed.
#pragma once
#include "kg_leaf.cuh"

namespace kg {

// Per-instance constants of the directed map: D = n - 1 >= 4,
// s = floor(log2 D) - 1, M = floor(2^(32+s) / D).  For y < 2^(31+s) the
// estimate q' = mulhi32(y >> s, M) satisfies q' <= floor(y / D) <= q' + 1.
struct SparseMap {
  uint64_t D;
  uint32_t M;
  int s;
};

inline SparseMap sparse_map(uint64_t n) {
  SparseMap mp;
  mp.D = n - 1;
  int lg = 63;
  while (!((mp.D >> lg) & 1)) --lg;
  mp.s = lg - 1;
  mp.M = uint32_t((u128(1) << (32 + mp.s)) / mp.D);
  return mp;
}

inline SparseRoute sparse_route(const SparseMap& mp, bool on) {
  SparseRoute r;
  r.on = on ? 1 : 0;
  r.ymax = (31 + mp.s >= 64) ? ~uint64_t(0) : (uint64_t(1) << (31 + mp.s));
  return r;
}

struct SparseSmem {
  uint64_t A[SP_KMAX];     // draws scattered by bucket, then sorted in place
  uint64_t D[SP_KMAX];     // draws in draw order
  uint32_t cnt[SP_NB];     // bucket counts, then bucket starts
  uint32_t multi[SP_KMAX / 2];  // buckets holding several draws: start | count << 16
};

// Geom: DirGeom (one map for the launch: mp), or a geometry whose tiles carry
// their own map (sparse_tile_map(descriptor, map)).  The Philox keys come from
// each tile's seed, added up round by round: holding ten precomputed round
// keys in registers measured slower here (more spills at 5 blocks per SM).
template <class Geom, class Sink, bool DIGEST>
__global__ void __launch_bounds__(SP_THREADS, SP_MIN_BLOCKS)
    leaf_sparse_kernel(SparseMap mp, Sink sink,
                       const TileDesc<typename Geom::Ctx>* __restrict__ desc, uint64_t ntiles,
                       int* err, DigestOut dig, unsigned long long* __restrict__ list,
                       unsigned long long* __restrict__ nlist) {
  constexpr bool DIR = std::is_same<Geom, DirGeom>::value;
  static_assert(DIR || !DIGEST, "the fused digest is for the directed geometry");
  __shared__ __align__(16) SparseSmem sm;
  __shared__ unsigned bh[65];
  __shared__ __align__(16) uint32_t wsum[SP_THREADS / 32];
  __shared__ unsigned long long red_d[SP_THREADS / 32];
  __shared__ unsigned red_c1[SP_THREADS / 32], red_nr[SP_THREADS / 32];
  __shared__ uint64_t s_fu, s_lu;
  __shared__ uint32_t s_fl, s_ll;
  __shared__ uint32_t s_nmulti;
  using Desc = TileDesc<typename Geom::Ctx>;
  __shared__ __align__(16) Desc s_td[2];
  __shared__ SparseTileMap s_map[2];  // per-tile maps (not DIR), staged with the descriptor
  const int tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
  auto stage = [&](uint64_t tt, int slot) {
    static_assert(sizeof(Desc) % 4 == 0, "descriptor size");
    const uint32_t* src = reinterpret_cast<const uint32_t*>(desc + tt);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&s_td[slot]);
    for (uint32_t w = tid; w < sizeof(Desc) / 4; w += SP_THREADS) dst[w] = src[w];
    if constexpr (!DIR) {
      if (tid == SP_THREADS - 1) sparse_tile_map(desc[tt], s_map[slot]);
    }
  };
  uint4* const cnt4 = reinterpret_cast<uint4*>(sm.cnt);

#pragma unroll
  for (int g4 = 0; g4 < SP_CPT / 4; ++g4) cnt4[(SP_CPT / 4) * tid + g4] = make_uint4(0, 0, 0, 0);
  if (DIGEST)
    for (int b = tid; b < 65; b += SP_THREADS) bh[b] = 0;
  if (blockIdx.x < ntiles) stage(blockIdx.x, 0);
  __syncthreads();
  int cur = 0;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x, cur ^= 1) {
    const Desc& td = s_td[cur];
    const uint64_t tn = t + gridDim.x;
    if (td.flags != 0 || !sink.fits(td.base, td.k)) {  // uniform over the block
      if (td.flags == 0 && tid == 0) set_error(err, ST_CAPACITY);  // the tile is dropped
      if (tn < ntiles) stage(tn, cur ^ 1);
      __syncthreads();
      continue;
    }
    const uint32_t k = td.k, bsh = td.bsh;
    // the descriptor's multiplier is for nb = 2048 or 4096 buckets; halving
    // it gives the 2048-bucket map (floor(floor(x) / 2) = floor(x / 2))
    const uint32_t bmul = td.bmul >> (td.nb >> 12);
    const uint64_t Lk = td.L - k, node = td.node(td.d, td.tau);

    // ---- 1. draws in draw order into D; bucket counts and slots
    uint32_t bs[2 * SP_PAIRS];  // bucket | slot << 16
    uint32_t rejm = 0;
#pragma unroll
    for (int s = 0; s < SP_PAIRS; ++s) {
      const uint32_t i = 2 * (tid + SP_THREADS * s);
      if (i < k) {
        uint32_t w[4];
        philox10(i >> 1, uint32_t(node), uint32_t(node >> 32), TAG_LEAF, uint32_t(td.seed),
                 uint32_t(td.seed >> 32), w);
        const uint64_t a = (uint64_t(w[0]) << 32) | w[1], c = (uint64_t(w[2]) << 32) | w[3];
        const uint64_t r0 = Lk + i + 1, r1 = r0 + 1;
        const uint64_t x0 = mul_hi64(a, r0), x1 = mul_hi64(c, r1);
        const bool ok0 = a * r0 >= r0, ok1 = c * r1 >= r1;
        rejm |= (ok0 ? 0u : 1u << (2 * s)) | ((ok1 || i + 1 >= k) ? 0u : 2u << (2 * s));
        if (ok0) {
          const uint32_t b0 = __umulhi(uint32_t(x0 >> bsh), bmul);
          bs[2 * s] = b0 | (atomicAdd(&sm.cnt[b0], 1u) << 16);
        }
        if (i + 1 < k) {
          if (ok1) {
            const uint32_t b1 = __umulhi(uint32_t(x1 >> bsh), bmul);
            bs[2 * s + 1] = b1 | (atomicAdd(&sm.cnt[b1], 1u) << 16);
          }
          reinterpret_cast<ulonglong2*>(sm.D)[i >> 1] = make_ulonglong2(x0, x1);
        } else {
          sm.D[i] = x0;
        }
      }
    }
    if (rejm) {  // Lemire's rejected draws (probability below L / 2^64 each)
#pragma unroll
      for (int j = 0; j < 2 * SP_PAIRS; ++j)
        if (rejm & (1u << j)) {
          const uint32_t i = 2 * (tid + SP_THREADS * (j >> 1)) + (j & 1);
          const uint64_t x = lemire_draw(stream_u64(td.seed, node, TAG_LEAF, i), Lk + i + 1,
                                         td.seed, node, i);
          const uint32_t b = __umulhi(uint32_t(x >> bsh), bmul);
          bs[j] = b | (atomicAdd(&sm.cnt[b], 1u) << 16);
          sm.D[i] = x;
        }
    }
    __syncthreads();
    // every thread is past the previous tile: its descriptor slot takes the next
    if (tn < ntiles) stage(tn, cur ^ 1);

    // ---- 2. bucket starts; buckets with several draws listed in order.
    // Thread tid owns counters [SP_CPT tid, SP_CPT (tid + 1)); one scan carries the draw
    // count (low 16 bits) and the number of multi-draw buckets (high 16).
    {
      uint32_t cs[SP_CPT];
#pragma unroll
      for (int g4 = 0; g4 < SP_CPT / 4; ++g4) {
        const uint4 cg = cnt4[(SP_CPT / 4) * tid + g4];
        cs[4 * g4] = cg.x;
        cs[4 * g4 + 1] = cg.y;
        cs[4 * g4 + 2] = cg.z;
        cs[4 * g4 + 3] = cg.w;
      }
      uint32_t pk = 0;
#pragma unroll
      for (int j = 0; j < SP_CPT; ++j) pk += cs[j] + (cs[j] > 1 ? 0x10000u : 0u);
      uint32_t inc = pk;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
      }
      if (lane == 31) wsum[wid] = inc;
      __syncthreads();
      uint32_t before = 0;
#pragma unroll
      for (int w = 0; w < SP_THREADS / 32; ++w) before += (w < wid) ? wsum[w] : 0u;
      uint32_t ex = before + inc - pk;
      uint32_t run = ex & 0xffffu, mpos = ex >> 16;
      uint32_t st[SP_CPT];
#pragma unroll
      for (int j = 0; j < SP_CPT; ++j) {
        st[j] = run;
        if (cs[j] > 1) sm.multi[mpos++] = run | (cs[j] << 16);
        run += cs[j];
      }
#pragma unroll
      for (int g4 = 0; g4 < SP_CPT / 4; ++g4)
        cnt4[(SP_CPT / 4) * tid + g4] =
            make_uint4(st[4 * g4], st[4 * g4 + 1], st[4 * g4 + 2], st[4 * g4 + 3]);
      if (tid == SP_THREADS - 1) s_nmulti = mpos;
    }
    __syncthreads();  // starts and the multi list visible

    // ---- 3. scatter, then sort the listed buckets
#pragma unroll
    for (int s = 0; s < SP_PAIRS; ++s) {
      const uint32_t i = 2 * (tid + SP_THREADS * s);
#pragma unroll
      for (int h = 0; h < 2; ++h)
        if (i + h < k) {
          const uint32_t v = bs[2 * s + h];
          sm.A[sm.cnt[v & 0xffffu] + (v >> 16)] = sm.D[i + h];
        }
    }
    __syncthreads();
    // the counters are dead: clear them for the next tile
#pragma unroll
    for (int g4 = 0; g4 < SP_CPT / 4; ++g4) cnt4[(SP_CPT / 4) * tid + g4] = make_uint4(0, 0, 0, 0);
    int dup = 0;
    const uint32_t nmulti = s_nmulti;
    for (uint32_t e = tid; e < nmulti; e += SP_THREADS) {
      const uint32_t item = sm.multi[e];
      const uint32_t s0 = item & 0xffffu, c = item >> 16;
      if (c == 2) {
        const uint64_t a = sm.A[s0], b = sm.A[s0 + 1];
        if (b < a) {
          sm.A[s0] = b;
          sm.A[s0 + 1] = a;
        }
        dup |= (a == b);
      } else {
        dup |= sort_bucket(sm.A, s0, s0 + c);
      }
    }
    if (__syncthreads_or(dup)) {
      // Floyd replaces a draw in this tile: the general kernel samples it
      if (tid == 0) list[ntiles - 1 - atomicAdd(nlist, 1ull)] = t;
      continue;
    }

    // ---- 4. emission: offset x of the tile is y = aux0 + x past the start of
    // row aux1; row u = aux1 + floor(y / D), column position w = y mod D,
    // v = w + [w >= u] (the diagonal is skipped)
    const uint64_t base = td.base;
    if constexpr (!DIR) {
      const SparseTileMap& tm = s_map[cur];
      const uint64_t rem0 = tm.y0, u0 = tm.u0, D = tm.D, col0 = tm.col0;
      const uint32_t M = tm.M;
      const int qs = tm.s, skip = tm.skip;
      for (uint32_t r = tid; r < k; r += SP_THREADS) {
        const uint64_t y = rem0 + sm.A[r];
        uint32_t q = __umulhi(uint32_t(y >> qs), M);
        uint64_t w = y - uint64_t(q) * D;
        if (w >= D) {
          w -= D;
          ++q;
        }
        const uint64_t u = u0 + q;
        sink.put(base + r, u, skip ? w + (w >= u ? 1 : 0) : col0 + w);
      }
      continue;
    }
    const uint64_t rem0 = td.aux0, u0 = td.aux1;
    const uint64_t D = mp.D;
    const uint32_t M = mp.M;
    const int qs = mp.s;
    if constexpr (!DIGEST) {
      for (uint32_t r = tid; r < k; r += SP_THREADS) {
        const uint64_t y = rem0 + sm.A[r];
        uint32_t q = __umulhi(uint32_t(y >> qs), M);
        uint64_t w = y - uint64_t(q) * D;
        if (w >= D) {
          w -= D;
          ++q;
        }
        const uint64_t u = u0 + q;
        sink.put(base + r, u, w + (w >= u ? 1 : 0));
      }
    } else {
      unsigned long long dsum = 0;
      uint32_t c1 = 0, nr = 0;
      for (uint32_t r = tid; r < k; r += SP_THREADS) {
        const uint64_t x = sm.A[r];
        const uint64_t y = rem0 + x;
        uint32_t q = __umulhi(uint32_t(y >> qs), M);
        uint64_t w = y - uint64_t(q) * D;
        if (w >= D) {
          w -= D;
          ++q;
        }
        const uint64_t u = u0 + q;
        const uint64_t v = w + (w >= u ? 1 : 0);
        sink.put(base + r, u, v);
        dsum += edge_hash(u, v);
        // a run of row u starts at r if the previous offset is in an earlier
        // row (more than w below x), and ends at r if the next offset is in a
        // later row (at least D - w above x)
        const bool first = (r == 0), last = (r + 1 == k);
        const bool st = first || x - sm.A[r - 1] > w;
        const bool en = last || sm.A[r + 1] - x >= D - w;
        nr += st;
        c1 += st & en & !first & !last;  // one-edge runs inside the tile
        if (st & !en) {  // a run of two or more edges (rare when rows are sparse)
          uint32_t e = r + 2;
          while (e < k && sm.A[e] - x < D - w) ++e;
          const uint32_t len = e - r;
          const bool lst = (e == k);
          if (first) {
            s_fu = u;
            s_fl = len;
          }
          if (lst) {
            s_lu = u;
            s_ll = len;
          }
          if (!first && !lst) atomicAdd(&bh[len < 64 ? len : 64], 1u);
        } else if (st & (first | last)) {  // a one-edge run at a tile end
          if (first) {
            s_fu = u;
            s_fl = 1;
          }
          if (last) {
            s_lu = u;
            s_ll = 1;
          }
        }
      }
      // block totals: the digest sum (mod 2^64), one-edge runs, runs
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
      c1 = __reduce_add_sync(0xffffffffu, c1);
      nr = __reduce_add_sync(0xffffffffu, nr);
      if (lane == 0) {
        red_d[wid] = dsum;
        red_c1[wid] = c1;
        red_nr[wid] = nr;
      }
      __syncthreads();
      const uint64_t cl = t >> td.d;
      if (tid == 0) {
        unsigned long long Dg = 0;
        unsigned C1 = 0, NR = 0;
#pragma unroll
        for (int w = 0; w < SP_THREADS / 32; ++w) {
          Dg += red_d[w];
          C1 += red_c1[w];
          NR += red_nr[w];
        }
        atomicAdd(&dig.digest[cl], Dg);
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
      for (int b = tid; b < 65; b += SP_THREADS)
        if (bh[b]) {
          atomicAdd(&dig.hist[cl * 65 + b], (unsigned long long)bh[b]);
          bh[b] = 0;
        }
    }
  }
}

}  // namespace kg
