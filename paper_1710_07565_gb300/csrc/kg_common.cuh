// Shared launch helpers, chunk geometries and block-level scans.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "kg_device.cuh"

namespace kg {

constexpr int K_LEAF = 1024;  // expected samples per tile (base-case threshold)
constexpr int K_MAX = 2048;   // a leaf with more samples is split once more
// leaf buckets are the next power of two >= k, so bucket arrays sized K_MAX
// hold every bucket index only when K_MAX itself is a power of two
static_assert((K_MAX & (K_MAX - 1)) == 0, "K_MAX must be a power of two");
constexpr int LEAF_THREADS = 256;

__device__ __forceinline__ void set_error(int* err, int code) {
  if (err) atomicCAS(err, 0, code);
}

// Chunk boundary r_c = floor(c n / P) ("sections of size roughly n/P",
// Sec. 4.2), without 128-bit division: with n = qP + r, floor(cn/P) = cq + floor(cr/P)
// and cr < 2^48 for c <= P <= 2^24, divided through an invariant multiplier.
struct RowBounds {
  uint64_t n, q, r;
  uint32_t P;
  DivU64 divP;
  static RowBounds make(uint64_t n_, uint32_t P_) {
    RowBounds b;
    b.n = n_;
    b.P = P_;
    b.q = n_ / P_;
    b.r = n_ % P_;
    b.divP = make_div(P_);
    return b;
  }
  __host__ __device__ __forceinline__ uint64_t operator()(uint64_t c) const {
    return c * q + div_q(divP, c * r);
  }
};

// Directed chunks (Sec. 4.1): chunk c = rows [r_c, r_{c+1}) x all n-1 columns
// other than the row itself; offsets are row-major, the diagonal skipped.
struct DirGeom {
  uint64_t n;
  uint32_t P;
  DivU64 div;  // division by n-1
  RowBounds rb;

  static DirGeom make(uint64_t n, uint32_t P) {
    DirGeom g;
    g.n = n;
    g.P = P;
    g.div = make_div(n > 1 ? n - 1 : 1);
    g.rb = RowBounds::make(n, P);
    return g;
  }

  __host__ __device__ __forceinline__ uint64_t chunk_id(uint64_t c) const { return c; }
  __host__ __device__ __forceinline__ uint64_t rows(uint64_t c) const { return rb(c + 1) - rb(c); }
  __host__ __device__ __forceinline__ uint64_t universe(uint64_t c) const {
    return rows(c) * (n - 1);
  }
  struct Ctx {
    uint64_t r0;
  };
  __host__ __device__ __forceinline__ Ctx ctx(uint64_t c) const { return Ctx{rb(c)}; }
  __host__ __device__ __forceinline__ void map(const Ctx& x, uint64_t off, uint64_t& u,
                                               uint64_t& v) const {
    const uint64_t q = div_q(div, off);
    const uint64_t w = off - q * (n - 1);
    u = x.r0 + q;
    v = w + (w >= u ? 1 : 0);
  }
  // first offset and length of the row of `off` (which maps to (u, v))
  __host__ __device__ __forceinline__ void row_span(const Ctx&, uint64_t off, uint64_t u,
                                                    uint64_t v, uint64_t& start,
                                                    uint64_t& len) const {
    start = off - (v - (v > u ? 1 : 0));
    len = n - 1;
  }
};

// Row of offset `off` in a rectangle of row length sj: off / sj, in 32-bit
// arithmetic when both fit (the common case), else 64-bit.
__host__ __device__ __forceinline__ uint64_t rect_row(uint64_t off, uint64_t sj) {
  if ((off | sj) <= 0xffffffffull) return uint32_t(off) / uint32_t(sj);
  return off / sj;
}

// Largest w >= 1 with w (w - 1) / 2 <= off (the row of a triangle offset):
// a square-root estimate (single precision below 2^40, double above),
// corrected exactly in integers.
__host__ __device__ __forceinline__ uint64_t tri_row(uint64_t off) {
  uint64_t w;
  if (off < (uint64_t(1) << 40)) {
    w = uint64_t((1.0f + sqrtf(1.0f + 8.0f * float(off))) * 0.5f);
    if (w < 1) w = 1;
    while (w * (w - 1) / 2 > off) --w;
    while ((w + 1) * w / 2 <= off) ++w;
    return w;
  }
  w = uint64_t((1.0 + sqrt(1.0 + 8.0 * double(off))) * 0.5);
  if (w < 1) w = 1;
  while (u128(w) * (w - 1) / 2 > off) --w;
  while (u128(w + 1) * w / 2 <= off) ++w;
  return w;
}

// Undirected chunks (Sec. 4.2): chunk (i, j), j <= i, of the triangular P x P
// chunk matrix; chunk index k enumerates (i, j) row by row, k = i(i+1)/2 + j,
// and the chunk's stream id is i P + j.  Rectangles (i > j) are row-major,
// triangles (i = j) hold u > v with offset (u-a)(u-a-1)/2 + (v-a).
struct UndGeom {
  uint64_t n;
  uint32_t P;
  RowBounds rb;

  __host__ __device__ __forceinline__ static void ij(uint64_t k, uint32_t& i, uint32_t& j) {
    uint64_t r = uint64_t(sqrt(8.0 * double(k) + 1.0) - 1.0) / 2;
    while (r * (r + 1) / 2 > k) --r;
    while ((r + 1) * (r + 2) / 2 <= k) ++r;
    i = uint32_t(r);
    j = uint32_t(k - r * (r + 1) / 2);
  }
  __host__ __device__ __forceinline__ uint64_t chunk_id(uint64_t k) const {
    uint32_t i, j;
    ij(k, i, j);
    return uint64_t(i) * P + j;
  }
  // rows of the chunk's row block
  __host__ __device__ __forceinline__ uint64_t rows(uint64_t k) const {
    uint32_t i, j;
    ij(k, i, j);
    return rb(uint64_t(i) + 1) - rb(i);
  }
  __host__ __device__ __forceinline__ uint64_t universe(uint64_t k) const {
    uint32_t i, j;
    ij(k, i, j);
    const uint64_t si = rb(uint64_t(i) + 1) - rb(i);
    if (i == j) return si ? uint64_t(u128(si) * (si - 1) / 2) : 0;
    const uint64_t sj = rb(uint64_t(j) + 1) - rb(j);
    return si * sj;
  }
  struct Ctx {
    uint64_t ri, rj, sj;
    bool tri;
  };
  __host__ __device__ __forceinline__ Ctx ctx(uint64_t k) const {
    uint32_t i, j;
    ij(k, i, j);
    Ctx x;
    x.ri = rb(i);
    x.rj = rb(j);
    x.sj = rb(uint64_t(j) + 1) - x.rj;
    x.tri = (i == j);
    return x;
  }
  __host__ __device__ __forceinline__ void map(const Ctx& x, uint64_t off, uint64_t& u,
                                               uint64_t& v) const {
    if (!x.tri) {
      const uint64_t q = rect_row(off, x.sj);
      u = x.ri + q;
      v = x.rj + (off - q * x.sj);
      return;
    }
    const uint64_t w = tri_row(off);
    u = x.ri + w;
    v = x.ri + (off - uint64_t(u128(w) * (w - 1) / 2));
  }
  // first offset and length of the row of `off` (which maps to (u, v))
  __host__ __device__ __forceinline__ void row_span(const Ctx& x, uint64_t off, uint64_t u,
                                                    uint64_t v, uint64_t& start,
                                                    uint64_t& len) const {
    if (!x.tri) {
      start = off - (v - x.rj);
      len = x.sj;
    } else {
      start = off - (v - x.ri);
      len = u - x.ri;
    }
  }
};

// Leaf universe of tile tau: [min(tau W, U), min((tau+1) W, U)), W = ceil(U/2^d).
__host__ __device__ __forceinline__ uint64_t tile_width(uint64_t U, int d) {
  return uint64_t((u128(U) + ((u128(1) << d) - 1)) >> d);
}
// Left end of tile-tree node (level, j): min(floor(j W 2^d / 2^level), U).
__host__ __device__ __forceinline__ uint64_t node_bound(uint64_t U, uint64_t W, int d, int level,
                                                        u128 j) {
  u128 x = j * u128(W);
  if (level <= d)
    x <<= (d - level);
  else
    x >>= (level - d);
  return x < u128(U) ? uint64_t(x) : U;
}

// ---------------------------------------------------------------- block scan
// Inclusive scan of one value per thread over the block; returns the block total.
template <int NT, class T>
__device__ __forceinline__ T block_inclusive_scan(T x, T& total) {
  __shared__ T warp_tot[NT / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  if (wid == 0) {
    T w = lane < NT / 32 ? warp_tot[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < NT / 32) warp_tot[lane] = w;
  }
  __syncthreads();
  if (wid > 0) x += warp_tot[wid - 1];
  total = warp_tot[NT / 32 - 1];
  __syncthreads();
  return x;
}

}  // namespace kg
