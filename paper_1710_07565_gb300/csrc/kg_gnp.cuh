// G(n,p) (Sec. 4.3): every chunk is cut into tiles of T pairs, T the largest
// power of two <= max(1, k_leaf / p); inside a tile the kept pairs follow
// from geometric skips (Batagelj and Brandes, Sec. 3.1): after candidate x
// the next kept pair is x + floor(ln U * (1 / ln(1-p))), U uniform on (0,1],
// drawn from the stream of (chunk id, tile).  One thread per tile writes the
// kept offsets to its slots; a scan sizes the output; the emit pass maps the
// offsets to (u, v).  A tile with more kept pairs than slots (beyond ~30
// standard deviations) is regenerated by the emit pass instead.
#pragma once
#include "kg_batch.h"
#include "kg_common.cuh"

namespace kg {

struct GnpPlan {
  double p, inv_lq;      // p and 1 / ln(1-p)
  uint64_t T;            // tile length
  uint64_t tiles_per_chunk;
  uint32_t cap_t;        // slots per tile
  int all;               // p == 1: every pair
};

// The kept offsets of tile [lo, hi) in order, handed to f(i, x).
template <class F>
__device__ __forceinline__ uint64_t gnp_tile_walk(uint64_t seed, uint64_t node, uint64_t lo,
                                                  uint64_t hi, double inv_lq, F&& f) {
  Stream s(seed, node, TAG_GNP);
  uint64_t x = lo, i = 0;
  for (;;) {
    const double U = u01_oc(s.u64());
    const double g = floor(kg_log(U) * inv_lq);
    if (g >= double(hi - x)) break;
    x += uint64_t(g);
    f(i, x);
    ++i;
    x += 1;
    if (x >= hi) break;
  }
  return i;
}

// Pass 1: per tile, the skip walk into slots (offsets relative to the tile).
template <class Geom, class SlotT>
__global__ void __launch_bounds__(128)
    gnp_tiles(Geom g, GnpPlan pl, uint64_t seed, uint64_t C, SlotT* __restrict__ slots,
              uint64_t* __restrict__ cnt) {
  const uint64_t total = C * pl.tiles_per_chunk;
  for (uint64_t t = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
       t += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t c = t / pl.tiles_per_chunk, tau = t - c * pl.tiles_per_chunk;
    const uint64_t U = g.universe(c);
    const uint64_t lo = tau * pl.T;
    if (lo >= U) {
      cnt[t] = 0;
      continue;
    }
    const uint64_t hi = (U - lo > pl.T) ? lo + pl.T : U;
    if (pl.all) {
      cnt[t] = hi - lo;
      continue;
    }
    SlotT* sl = slots ? slots + t * pl.cap_t : nullptr;
    const uint32_t cap_t = pl.cap_t;
    cnt[t] = gnp_tile_walk(seed, (g.chunk_id(c) << 32) | tau, lo, hi, pl.inv_lq,
                           [&](uint64_t i, uint64_t x) {
                             if (i < cap_t) sl[i] = SlotT(x - lo);
                           });
  }
}

// Pass 2: per tile, kept offsets -> (u, v) at the scanned position.
template <class Geom, class SlotT, class Sink>
__global__ void __launch_bounds__(128)
    gnp_emit(Geom g, GnpPlan pl, uint64_t seed, uint64_t C, const SlotT* __restrict__ slots,
             const uint64_t* __restrict__ cnt, const uint64_t* __restrict__ off, Sink sink) {
  const uint64_t total = C * pl.tiles_per_chunk;
  // one warp per tile: lanes take consecutive kept pairs (coalesced stores)
  const unsigned lane = threadIdx.x & 31;
  const uint64_t warp = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  for (uint64_t t = warp; t < total; t += nwarps) {
    const uint64_t k = cnt[t];
    if (k == 0) continue;
    const uint64_t c = t / pl.tiles_per_chunk, tau = t - c * pl.tiles_per_chunk;
    const uint64_t lo = tau * pl.T;
    const typename Geom::Ctx gx = g.ctx(c);
    const uint64_t base = off[t];
    if (pl.all) {
      for (uint64_t i = lane; i < k; i += 32) {
        uint64_t u, v;
        g.map(gx, lo + i, u, v);
        sink.write(base + i, u, v);
      }
    } else if (k <= pl.cap_t) {
      const SlotT* sl = slots + t * pl.cap_t;
      for (uint64_t i = lane; i < k; i += 32) {
        uint64_t u, v;
        g.map(gx, lo + sl[i], u, v);
        sink.write(base + i, u, v);
      }
    } else if (lane == 0) {
      const uint64_t U = g.universe(c);
      const uint64_t hi = (U - lo > pl.T) ? lo + pl.T : U;
      gnp_tile_walk(seed, (g.chunk_id(c) << 32) | tau, lo, hi, pl.inv_lq,
                    [&](uint64_t i, uint64_t x) {
                      uint64_t u, v;
                      g.map(gx, x, u, v);
                      sink.write(base + i, u, v);
                    });
    }
  }
}

// Sec. 4.3 with binomial chunk counts: the sample count of chunk c is
// Binomial(U_c, p) from the stream (seed, chunk id, TAG_GNP_COUNT); the chunk
// is then sampled like a G(n,m) chunk.  One thread per chunk.
template <class Geom>
__global__ void __launch_bounds__(128)
    gnp_chunk_counts(Geom g, uint64_t C, double p, uint64_t seed, uint64_t* __restrict__ cnt,
                     int* err) {
  for (uint64_t c = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < C;
       c += uint64_t(gridDim.x) * blockDim.x) {
    Stream s(seed, g.chunk_id(c), TAG_GNP_COUNT);
    uint64_t x = 0;
    const int e = binomial(g.universe(c), p, s, x, BINOM_N_MAX);
    if (e) {
      set_error(err, e);
      x = 0;
    }
    cnt[c] = x;
  }
}

// One G(n,p)-by-binomial-counts size pass for many instances at once (the
// serving loop's sizing): instance i is taken by one warp, whose lanes draw
// the chunk binomials of gnp_chunk_counts (same streams, same universes:
// chunk boundaries floor(c n / P)) and add them up; sizes[i] is the entry
// count kg_gnp_binomial writes (twice the pairs when undirected).
__global__ void __launch_bounds__(128)
    gnpb_size_batch(const GnpbSizeReq* __restrict__ reqs, uint32_t count,
                    uint64_t* __restrict__ sizes, int* err) {
  const unsigned lane = threadIdx.x & 31;
  const uint64_t nwarps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  for (uint64_t i = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; i < count;
       i += nwarps) {
    const GnpbSizeReq q = reqs[i];
    const uint64_t P = q.chunks;
    auto rb = [&](uint64_t c) { return uint64_t((u128(c) * q.n) / P); };
    const uint64_t C = q.undirected ? P * (P + 1) / 2 : P;
    unsigned long long tot = 0;
    for (uint64_t c = lane; c < C; c += 32) {
      uint64_t U, cid;
      if (q.undirected) {
        uint32_t a, b;
        UndGeom::ij(c, a, b);
        const uint64_t sa = rb(uint64_t(a) + 1) - rb(a);
        U = (a == b) ? (sa ? uint64_t(u128(sa) * (sa - 1) / 2) : 0)
                     : sa * (rb(uint64_t(b) + 1) - rb(b));
        cid = uint64_t(a) * P + b;
      } else {
        U = (rb(c + 1) - rb(c)) * (q.n - 1);
        cid = c;
      }
      Stream st(q.seed, cid, TAG_GNP_COUNT);
      uint64_t x = 0;
      const int e = binomial(U, q.p, st, x, BINOM_N_MAX);
      if (e) {
        set_error(err, e);
        x = 0;
      }
      tot += x;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    if (lane == 0) sizes[i] = q.undirected ? 2 * tot : tot;
  }
}

}  // namespace kg
