// Undirected generators (Sec. 4.2): the quadrant recursion over the
// triangular P x P chunk matrix, and the assembly of the sampled lower-triangle
// pairs into one (u, v)-sorted list holding every edge in both directions.
#pragma once
#include "kg_common.cuh"

namespace kg {

// ---------------------------------------------------------------- quadrant tree
// A node is a triangle of blocks [a, b) (a == c, b == d) or a rectangle of
// row blocks [a, b) x column blocks [c, d) strictly below the diagonal.
struct QNode {
  uint32_t a, b, c, d;
  uint64_t cnt;
};

__host__ __device__ __forceinline__ uint64_t quad_id(uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  return uint64_t(a) | (uint64_t(b - 1) << 16) | (uint64_t(c) << 32) | (uint64_t(d - 1) << 48);
}
__host__ __device__ __forceinline__ u128 tri_pairs(uint64_t S) {
  return S ? u128(S) * (S - 1) / 2 : 0;
}
__host__ __device__ __forceinline__ uint64_t und_chunk_index(uint32_t i, uint32_t j) {
  return uint64_t(i) * (i + 1) / 2 + j;
}

static __global__ void quad_init(QNode* list, uint32_t* counts, int nlevels, uint32_t P, uint64_t m) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    list[0] = QNode{0, P, 0, P, m};
    counts[0] = 1;
    for (int l = 1; l <= nlevels; ++l) counts[l] = 0;
  }
}

// One level: every node either is a chunk (its count is final) or draws its
// parts' counts from its own stream, in order, and appends the parts.
//  - triangle [a,b), l = ceil((b-a)/2): T1 = tri[a,a+l), R = rows [a+l,b) x
//    cols [a,a+l), T2 = tri[a+l,b); X1 = Hyp(N, |T1|, cnt),
//    X2 = Hyp(N - |T1|, |R|, cnt - X1), T2 gets the rest;
//  - rectangle: each dimension with more than one block halved at ceil, the
//    parts in row-major order, sequential conditional hypergeometrics.
// MINB = 4 (64 registers) for wide levels, where the spills cost less than
// the occupancy they buy (62 -> 47 ms for the 8.4 M-chunk tree at P = 4096);
// narrow levels are latency-bound and keep all the registers they want.
template <int MINB>
static __global__ void __launch_bounds__(256, MINB)
    quad_level(RowBounds rb, uint64_t seed, const QNode* __restrict__ in,
               const uint32_t* __restrict__ nin, QNode* __restrict__ out, uint32_t* nout,
               uint64_t* __restrict__ chunk_cnt, int* err) {
  const uint32_t count = *nin;
  for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < count;
       idx += gridDim.x * blockDim.x) {
    const QNode q = in[idx];
    const bool tri = (q.a == q.c && q.b == q.d);
    if (tri && q.b - q.a == 1) {
      chunk_cnt[und_chunk_index(q.a, q.a)] = q.cnt;
      continue;
    }
    if (!tri && q.b - q.a == 1 && q.d - q.c == 1) {
      chunk_cnt[und_chunk_index(q.a, q.c)] = q.cnt;
      continue;
    }
    Stream st(seed, quad_id(q.a, q.b, q.c, q.d), TAG_QUAD);
    if (tri) {
      const uint32_t l = (q.b - q.a + 1) / 2;
      const uint64_t ra = rb(q.a), rm = rb(q.a + l), rbb = rb(q.b);
      const uint64_t S1 = rm - ra, S2 = rbb - rm;
      const u128 T1 = tri_pairs(S1), R = u128(S2) * S1, T2 = tri_pairs(S2);
      const u128 N = T1 + R + T2;
      uint64_t X1 = 0, X2 = 0;
      int e = hypergeometric(N, T1, q.cnt, st, X1);
      if (!e) e = hypergeometric(N - T1, R, q.cnt - X1, st, X2);
      if (e) {
        set_error(err, e);
        X1 = X2 = 0;
      }
      const uint32_t o = atomicAdd(nout, 3u);
      out[o] = QNode{q.a, q.a + l, q.a, q.a + l, X1};
      out[o + 1] = QNode{q.a + l, q.b, q.a, q.a + l, X2};
      out[o + 2] = QNode{q.a + l, q.b, q.a + l, q.b, q.cnt - X1 - X2};
      continue;
    }
    uint32_t rlo[2] = {q.a, 0}, rhi[2] = {q.b, 0}, clo[2] = {q.c, 0}, chi[2] = {q.d, 0};
    int nr = 1, nc = 1;
    if (q.b - q.a >= 2) {
      const uint32_t s = q.a + (q.b - q.a + 1) / 2;
      rhi[0] = s;
      rlo[1] = s;
      rhi[1] = q.b;
      nr = 2;
    }
    if (q.d - q.c >= 2) {
      const uint32_t s = q.c + (q.d - q.c + 1) / 2;
      chi[0] = s;
      clo[1] = s;
      chi[1] = q.d;
      nc = 2;
    }
    QNode parts[4];
    u128 size[4];
    int np = 0;
    u128 N = 0;
    for (int i = 0; i < nr; ++i)
      for (int j = 0; j < nc; ++j) {
        parts[np] = QNode{rlo[i], rhi[i], clo[j], chi[j], 0};
        size[np] = u128(rb(rhi[i]) - rb(rlo[i])) * (rb(chi[j]) - rb(clo[j]));
        N += size[np];
        ++np;
      }
    uint64_t rem = q.cnt;
    for (int i = 0; i < np - 1; ++i) {
      uint64_t X = 0;
      const int e = hypergeometric(N, size[i], rem, st, X);
      if (e) {
        set_error(err, e);
        X = 0;
      }
      parts[i].cnt = X;
      N -= size[i];
      rem -= X;
    }
    parts[np - 1].cnt = rem;
    const uint32_t o = atomicAdd(nout, uint32_t(np));
    for (int i = 0; i < np; ++i) out[o + i] = parts[i];
  }
}

// ---------------------------------------------------------------- assembly
// The sampled pairs (u > v) of all chunks become the (u, v)-sorted list of
// both directions: degrees, row offsets (scan), scatter to row slots, and a
// sort of each row by v.  The rows' contents are unique, so the result does
// not depend on the order in which the scatter fills a row.
template <class Id>
__device__ __forceinline__ void load_pair(const Id* p, uint64_t i, uint64_t& u, uint64_t& v) {
  u = p[2 * i];
  v = p[2 * i + 1];
}

// one 8- or 16-byte store of the pair (u, v) at slot i
template <class Id>
__device__ __forceinline__ void store_pair(Id* out, uint64_t i, uint64_t u, uint64_t v) {
  if (sizeof(Id) == 4)
    reinterpret_cast<uint2*>(out)[i] = make_uint2(uint32_t(u), uint32_t(v));
  else
    reinterpret_cast<ulonglong2*>(out)[i] = make_ulonglong2(u, v);
}

// Rows [row_lo, row_lo + nrows) only: a pair (u, v) gives the entry (u, v)
// when u is in the window and (v, u) when v is (all rows: row_lo 0, nrows n).
template <class Id>
__global__ void und_degree(const Id* __restrict__ pairs, const uint64_t* __restrict__ npairs_dev,
                           uint64_t npairs_host, uint64_t row_lo, uint64_t nrows,
                           unsigned long long* __restrict__ deg) {
  const uint64_t np = npairs_dev ? *npairs_dev : npairs_host;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < np;
       i += uint64_t(gridDim.x) * blockDim.x) {
    uint64_t u, v;
    load_pair(pairs, i, u, v);
    if (u - row_lo < nrows) atomicAdd(&deg[u - row_lo], 1ull);
    if (v - row_lo < nrows) atomicAdd(&deg[v - row_lo], 1ull);
  }
}

template <class Id>
__global__ void und_scatter(const Id* __restrict__ pairs, const uint64_t* __restrict__ npairs_dev,
                            uint64_t npairs_host, uint64_t row_lo, uint64_t nrows,
                            unsigned long long* __restrict__ cursor, Id* __restrict__ out,
                            uint64_t cap, int* err) {
  const uint64_t np = npairs_dev ? *npairs_dev : npairs_host;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < np;
       i += uint64_t(gridDim.x) * blockDim.x) {
    uint64_t u, v;
    load_pair(pairs, i, u, v);
    if (u - row_lo < nrows) {
      const uint64_t p = atomicAdd(&cursor[u - row_lo], 1ull);
      if (p < cap)
        store_pair(out, p, u, v);
      else
        set_error(err, ST_CAPACITY);
    }
    if (v - row_lo < nrows) {
      const uint64_t q = atomicAdd(&cursor[v - row_lo], 1ull);
      if (q < cap)
        store_pair(out, q, v, u);
      else
        set_error(err, ST_CAPACITY);
    }
  }
}

// Per row block of the window: the digest of its entries and the histogram
// of its rows' degrees (rows [r_b, r_{b+1}) of block b_lo + (index)).  A CTA
// takes segments of 8192 consecutive rows (almost always inside one row
// block, 2^20 rows wide at scale): degrees 0..7 are counted in registers and
// summed over the warp, the rest and the digest in shared memory, and the
// segment's block receives one atomic per bin; rows of a second block in a
// segment go to global memory directly.
constexpr uint64_t DIGEST_SEG = 8192;

__device__ __forceinline__ uint64_t block_of_row(const RowBounds& rb, uint64_t u) {
  uint64_t b = uint64_t((u128(u) * rb.P) / rb.n);
  while (b + 1 < rb.P && rb(b + 1) <= u) ++b;
  while (b > 0 && rb(b) > u) --b;
  return b;
}

template <class Id>
__global__ void __launch_bounds__(256)
    und_block_digest(const Id* __restrict__ out, const uint64_t* __restrict__ rowptr,
                     uint64_t row_lo, uint64_t nrows, RowBounds rb, uint32_t b_lo,
                     unsigned long long* __restrict__ digest,
                     unsigned long long* __restrict__ hist) {
  __shared__ unsigned long long sh_hist[65];
  __shared__ unsigned long long sh_dig;
  const unsigned lane = threadIdx.x & 31;
  for (uint64_t s0 = uint64_t(blockIdx.x) * DIGEST_SEG; s0 < nrows;
       s0 += uint64_t(gridDim.x) * DIGEST_SEG) {
    const uint64_t s1 = s0 + DIGEST_SEG < nrows ? s0 + DIGEST_SEG : nrows;
    const uint64_t bA = block_of_row(rb, row_lo + s0);
    const bool one = block_of_row(rb, row_lo + s1 - 1) == bA;
    for (int i = threadIdx.x; i < 65; i += blockDim.x) sh_hist[i] = 0;
    if (threadIdx.x == 0) sh_dig = 0;
    __syncthreads();
    uint32_t c[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    unsigned long long dsum = 0;
    for (uint64_t r = s0 + threadIdx.x; r < s1; r += blockDim.x) {
      const uint64_t e0 = rowptr[r], e1 = rowptr[r + 1];
      const uint64_t deg = e1 - e0;
      unsigned long long ds = 0;
      for (uint64_t e = e0; e < e1; ++e) {
        uint64_t a, b2;
        load_pair(out, e, a, b2);
        ds += edge_hash(a, b2);
      }
      if (one || block_of_row(rb, row_lo + r) == bA) {
        dsum += ds;
#pragma unroll
        for (int d = 0; d < 8; ++d) c[d] += (deg == uint64_t(d));
        if (deg >= 8) atomicAdd(&sh_hist[deg < 64 ? deg : 64], 1ull);
      } else {  // the segment's second block
        const uint64_t bi = block_of_row(rb, row_lo + r) - b_lo;
        if (digest && ds) atomicAdd(&digest[bi], ds);
        if (hist) atomicAdd(&hist[bi * 65 + (deg < 64 ? deg : 64)], 1ull);
      }
    }
#pragma unroll
    for (int d = 0; d < 8; ++d) {
      const unsigned t = __reduce_add_sync(0xffffffffu, c[d]);
      if (lane == 0 && t) atomicAdd(&sh_hist[d], (unsigned long long)t);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
    if (lane == 0 && dsum) atomicAdd(&sh_dig, dsum);
    __syncthreads();
    const uint64_t bi = bA - b_lo;
    for (int i = threadIdx.x; i < 65; i += blockDim.x)
      if (hist && sh_hist[i]) atomicAdd(&hist[bi * 65 + i], sh_hist[i]);
    if (threadIdx.x == 0 && digest && sh_dig) atomicAdd(&digest[bi], sh_dig);
    __syncthreads();
  }
}

// Bitonic sort of 32 E values held by one warp, E consecutive values per lane
// (value index = lane E + e): exchanges at distance j < E stay in the lane,
// longer ones go through shuffles.
template <int E>
__device__ __forceinline__ void warp_bitonic(uint64_t (&x)[E], unsigned lane) {
#pragma unroll
  for (int k = 2; k <= 32 * E; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j >= E) {
        const int lj = j / E;
        const bool lower = (lane & lj) == 0;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const bool up = ((lane * E + e) & k) == 0;
          const uint64_t y = __shfl_xor_sync(0xffffffffu, x[e], lj);
          const uint64_t mn = x[e] < y ? x[e] : y, mx = x[e] < y ? y : x[e];
          x[e] = (lower == up) ? mn : mx;
        }
      } else {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int q = e ^ j;
          if (q > e) {
            const bool up = ((lane * E + e) & k) == 0;
            const uint64_t a = x[e], b = x[q];
            const bool sw = up ? (b < a) : (a < b);
            x[e] = sw ? b : a;
            x[q] = sw ? a : b;
          }
        }
      }
    }
  }
}

template <int E, class Id>
__device__ __forceinline__ void warp_sort_row_e(Id* out, uint64_t b, uint64_t deg, unsigned lane) {
  uint64_t x[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const uint64_t i = lane * E + e;
    x[e] = i < deg ? uint64_t(out[2 * (b + i) + 1]) : ~uint64_t(0);
  }
  warp_bitonic<E>(x, lane);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const uint64_t i = lane * E + e;
    if (i < deg) out[2 * (b + i) + 1] = Id(x[e]);
  }
}

constexpr uint64_t WARP_SORT_MAX = 256;

// Sorts the second ids of row entries [b, b + deg) by one warp (deg <= 256).
template <class Id>
__device__ __forceinline__ void warp_sort_row(Id* out, uint64_t b, uint64_t deg, unsigned lane) {
  if (deg <= 32)
    warp_sort_row_e<1>(out, b, deg, lane);
  else if (deg <= 64)
    warp_sort_row_e<2>(out, b, deg, lane);
  else if (deg <= 128)
    warp_sort_row_e<4>(out, b, deg, lane);
  else
    warp_sort_row_e<8>(out, b, deg, lane);
}

constexpr uint64_t LANE_SORT_MAX = 8;

// Sorts the second ids of row entries [b, b + deg), deg <= 8, by one thread:
// an 8-input sorting network (19 comparators) over registers padded with +inf.
template <class Id>
__device__ __forceinline__ void lane_sort_row(Id* out, uint64_t b, uint64_t deg) {
  uint64_t x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = uint64_t(i) < deg ? uint64_t(out[2 * (b + i) + 1]) : ~uint64_t(0);
  auto cx = [&](int i, int j) {
    const uint64_t a = x[i] < x[j] ? x[i] : x[j], c = x[i] < x[j] ? x[j] : x[i];
    x[i] = a;
    x[j] = c;
  };
  cx(0, 2); cx(1, 3); cx(4, 6); cx(5, 7);
  cx(0, 4); cx(1, 5); cx(2, 6); cx(3, 7);
  cx(0, 1); cx(2, 3); cx(4, 5); cx(6, 7);
  cx(2, 4); cx(3, 5);
  cx(1, 4); cx(3, 6);
  cx(1, 2); cx(3, 4); cx(5, 6);
#pragma unroll
  for (int i = 0; i < 8; ++i)
    if (uint64_t(i) < deg) out[2 * (b + i) + 1] = Id(x[i]);
}

// Rows of one warp's 32 consecutive rows: those of at most LANE_SORT_MAX
// entries by their own lane, those up to WARP_SORT_MAX by the whole warp one
// after the other, longer ones listed for und_sort_long.  Every lane of the
// warp calls it (b, deg: this lane's row; u: its row index).
template <class Id>
__device__ __forceinline__ void sort_rows_of_warp(Id* out, uint64_t b, uint64_t deg, uint64_t u,
                                                  unsigned lane, unsigned long long* long_rows,
                                                  unsigned long long* nlong) {
  if (deg >= 2 && deg <= LANE_SORT_MAX) lane_sort_row(out, b, deg);
  unsigned m = __ballot_sync(0xffffffffu, deg > LANE_SORT_MAX);
  while (m) {
    const int l = __ffs(m) - 1;
    m &= m - 1;
    const uint64_t bl = __shfl_sync(0xffffffffu, b, l), dl = __shfl_sync(0xffffffffu, deg, l);
    if (dl > WARP_SORT_MAX) {
      if (lane == unsigned(l)) long_rows[atomicAdd(nlong, 1ull)] = u;
    } else {
      warp_sort_row(out, bl, dl, lane);
    }
  }
}

template <class Id>
__global__ void __launch_bounds__(256)
    und_sort_short(const uint64_t* __restrict__ rowptr, uint64_t n, Id* __restrict__ out,
                   uint64_t cap, unsigned long long* long_rows, unsigned long long* nlong) {
  const unsigned lane = threadIdx.x & 31;
  const uint64_t warp = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  for (uint64_t u0 = warp * 32; u0 < n; u0 += nwarps * 32) {  // uniform over the warp
    const uint64_t u = u0 + lane;
    uint64_t b = 0, deg = 0;
    if (u < n) {
      b = rowptr[u];
      const uint64_t e = rowptr[u + 1] < cap ? rowptr[u + 1] : cap;
      deg = e > b ? e - b : 0;
    }
    sort_rows_of_warp(out, b, deg, u, lane, long_rows, nlong);
  }
}

constexpr int LONG_SMEM = 4096;

// One block per listed row: a sorting network whose comparisons all move the
// smaller value to the lower index (first step of each merge compares mirrored
// positions), so positions past the row behave as +infinity and are never
// touched.  Rows up to LONG_SMEM entries are sorted in shared memory, longer
// ones in place in global memory.
template <class Id>
__global__ void __launch_bounds__(256)
    und_sort_long(const uint64_t* __restrict__ rowptr, Id* __restrict__ out, uint64_t cap,
                  const unsigned long long* __restrict__ long_rows,
                  const unsigned long long* __restrict__ nlong) {
  __shared__ uint64_t sh[LONG_SMEM];
  const unsigned long long nl = *nlong;
  for (unsigned long long r = blockIdx.x; r < nl; r += gridDim.x) {
    const uint64_t u = long_rows[r];
    const uint64_t b = rowptr[u], e = rowptr[u + 1] < cap ? rowptr[u + 1] : cap;
    const uint64_t deg = e - b;
    uint64_t N = 1;
    int lgN = 0;
    while (N < deg) {
      N <<= 1;
      ++lgN;
    }
    const bool in_smem = deg <= LONG_SMEM;
    if (in_smem)
      for (uint64_t i = threadIdx.x; i < deg; i += blockDim.x) sh[i] = out[2 * (b + i) + 1];
    __syncthreads();
    auto get = [&](uint64_t i) -> uint64_t { return in_smem ? sh[i] : uint64_t(out[2 * (b + i) + 1]); };
    auto put = [&](uint64_t i, uint64_t x) {
      if (in_smem)
        sh[i] = x;
      else
        out[2 * (b + i) + 1] = Id(x);
    };
    for (int lk = 1; lk <= lgN; ++lk) {
      const uint64_t k = uint64_t(1) << lk;
      for (uint64_t i = threadIdx.x; i < N / 2; i += blockDim.x) {
        const uint64_t blk = i >> (lk - 1), off = i & (k / 2 - 1);
        const uint64_t lo = blk * k + off, hi = blk * k + k - 1 - off;
        if (hi < deg) {
          const uint64_t x = get(lo), y = get(hi);
          if (y < x) {
            put(lo, y);
            put(hi, x);
          }
        }
      }
      __syncthreads();
      for (int lj = lk - 2; lj >= 0; --lj) {
        const uint64_t j = uint64_t(1) << lj;
        for (uint64_t i = threadIdx.x; i < N / 2; i += blockDim.x) {
          const uint64_t blk = i >> lj, off = i & (j - 1);
          const uint64_t lo = blk * 2 * j + off, hi = lo + j;
          if (hi < deg) {
            const uint64_t x = get(lo), y = get(hi);
            if (y < x) {
              put(lo, y);
              put(hi, x);
            }
          }
        }
        __syncthreads();
      }
    }
    if (in_smem)
      for (uint64_t i = threadIdx.x; i < deg; i += blockDim.x) out[2 * (b + i) + 1] = Id(sh[i]);
    __syncthreads();
  }
}

}  // namespace kg

namespace kg {

// ---------------------------------------------------------------- bucketed assembly
// The window's rows are cut into buckets of 2^bsh consecutive rows, sized so
// that a bucket holds about ASM_TARGET entries.  (1) Every block histograms
// its contiguous share of the pairs by bucket in shared memory and stores
// its histogram; (2) per bucket, the blocks' counts become the blocks'
// offsets inside the bucket and a scan of the buckets' totals gives every
// bucket its final range of the output; (3) every block scatters its share's
// entries to its sub-range of each bucket; (4) one
// CTA per bucket loads the bucket's entries into shared memory, sorts them
// by row (counting sort) and each row by column, writes them back in order
// and fills the rows' offsets.  Buckets larger than shared memory are sorted
// in place in global memory instead.  The result is the same list as the
// atomic-per-entry assembly: rows hold unique columns, sorted.
constexpr int ASM_THREADS = 256;
constexpr uint32_t ASM_TARGET = 2048;    // expected entries per bucket
constexpr uint32_t ASM_CAP = 4096;       // entries a bucket may hold in shared memory
constexpr uint32_t ASM_BR_MAX = 2048;    // rows per bucket
constexpr uint32_t ASM_NB_MAX = 16384;   // buckets (per-block histogram in shared memory)
constexpr uint32_t ASM_ROW_LANE = 8;     // rows up to this length are sorted by one thread
constexpr uint32_t ASM_ROW_WARP = 256;   // ... up to this length by one warp, longer by the block

// An entry of a bucket as 8 bytes: its row inside the bucket (< 2^16) above
// bit 48, its column (< 2^48) below.  The scatter writes these keys to a
// staging array (half the bytes of a uint64 pair) and the bucket sort turns
// them back into (row, column) entries.
__device__ __forceinline__ uint64_t asm_key(uint64_t row_in_bucket, uint64_t col) {
  return (row_in_bucket << 48) | col;
}

constexpr int ASM_UNROLL = 4;          // pairs a thread loads before counting them
constexpr int ASM_SCATTER_UNROLL = 4;  // ... before scattering them
constexpr int ASM_HIST_BLOCKS = 2;     // count / scatter blocks per SM (64 KB histogram each)

// contiguous share [i0, i1) of the np pairs for block `blk` of `nblk`
__device__ __forceinline__ void asm_share(uint64_t np, uint32_t blk, uint32_t nblk, uint64_t& i0,
                                          uint64_t& i1) {
  const uint64_t per = (np + nblk - 1) / nblk;
  i0 = uint64_t(blk) * per;
  i1 = i0 + per < np ? i0 + per : np;
  if (i0 > np) i0 = np;
}

// (1) per block: the bucket histogram of its share, stored as row blockIdx.x
// of blk (nb counters per block, no atomics outside shared memory)
template <class Id>
__global__ void __launch_bounds__(ASM_THREADS)
    asm_bucket_count(const Id* __restrict__ pairs, const uint64_t* __restrict__ npairs_dev,
                     uint64_t npairs_host, uint64_t row_lo, uint64_t nrows, int bsh, uint32_t nb,
                     uint32_t* __restrict__ blk) {
  extern __shared__ uint32_t hcnt[];
  for (uint32_t i = threadIdx.x; i < nb; i += ASM_THREADS) hcnt[i] = 0;
  __syncthreads();
  uint64_t i0, i1;
  asm_share(npairs_dev ? *npairs_dev : npairs_host, blockIdx.x, gridDim.x, i0, i1);
  for (uint64_t i = i0 + threadIdx.x; i < i1; i += ASM_UNROLL * ASM_THREADS) {
    uint64_t u[ASM_UNROLL], v[ASM_UNROLL];
#pragma unroll
    for (int j = 0; j < ASM_UNROLL; ++j) {
      u[j] = v[j] = ~uint64_t(0);  // outside every window
      if (i + j * ASM_THREADS < i1) load_pair(pairs, i + j * ASM_THREADS, u[j], v[j]);
    }
#pragma unroll
    for (int j = 0; j < ASM_UNROLL; ++j) {
      if (u[j] - row_lo < nrows) atomicAdd(&hcnt[(u[j] - row_lo) >> bsh], 1u);
      if (v[j] - row_lo < nrows) atomicAdd(&hcnt[(v[j] - row_lo) >> bsh], 1u);
    }
  }
  __syncthreads();
  uint32_t* row = blk + uint64_t(blockIdx.x) * nb;
  for (uint32_t i = threadIdx.x; i < nb; i += ASM_THREADS) row[i] = hcnt[i];
}

// Per bucket b (one thread each): the counts of the G blocks become each
// block's offset inside the bucket (exclusive prefix over the blocks, in
// block order), and bcnt[b] the bucket's total.
static __global__ void __launch_bounds__(64)
    asm_bucket_colscan(uint32_t* __restrict__ blk, uint32_t G, uint32_t nb,
                       unsigned long long* __restrict__ bcnt) {
  const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  uint32_t run = 0;
  constexpr uint32_t U = 16;  // loads in flight before the dependent stores
  for (uint32_t g0 = 0; g0 < G; g0 += U) {
    uint32_t c[U];
#pragma unroll
    for (uint32_t j = 0; j < U; ++j) c[j] = g0 + j < G ? blk[uint64_t(g0 + j) * nb + b] : 0u;
#pragma unroll
    for (uint32_t j = 0; j < U; ++j)
      if (g0 + j < G) {
        blk[uint64_t(g0 + j) * nb + b] = run;
        run += c[j];
      }
  }
  bcnt[b] = run;
}

// (3) per block, the same share as in (1): every entry goes to its bucket's
// range at the block's offset in it (blk after asm_bucket_colscan)
template <class Id>
__global__ void __launch_bounds__(ASM_THREADS)
    asm_bucket_scatter(const Id* __restrict__ pairs, const uint64_t* __restrict__ npairs_dev,
                       uint64_t npairs_host, uint64_t row_lo, uint64_t nrows, int bsh, uint32_t nb,
                       const uint64_t* __restrict__ boff, const uint32_t* __restrict__ blk,
                       uint64_t* __restrict__ keys, uint64_t kcap, int* err) {
  extern __shared__ uint32_t hcur[];  // per bucket: this block's next slot in it
  const uint32_t* row = blk + uint64_t(blockIdx.x) * nb;
  for (uint32_t i = threadIdx.x; i < nb; i += ASM_THREADS) hcur[i] = row[i];
  __syncthreads();
  uint64_t i0, i1;
  asm_share(npairs_dev ? *npairs_dev : npairs_host, blockIdx.x, gridDim.x, i0, i1);
  for (uint64_t i = i0 + threadIdx.x; i < i1; i += ASM_SCATTER_UNROLL * ASM_THREADS) {
    uint64_t u[ASM_SCATTER_UNROLL], v[ASM_SCATTER_UNROLL];
#pragma unroll
    for (int j = 0; j < ASM_SCATTER_UNROLL; ++j) {
      u[j] = v[j] = ~uint64_t(0);  // outside every window
      if (i + j * ASM_THREADS < i1) load_pair(pairs, i + j * ASM_THREADS, u[j], v[j]);
    }
#pragma unroll
    for (int j = 0; j < ASM_SCATTER_UNROLL; ++j) {
      if (u[j] - row_lo < nrows) {
        const uint64_t rl = u[j] - row_lo;
        const uint32_t b = uint32_t(rl >> bsh);
        const uint64_t p = boff[b] + atomicAdd(&hcur[b], 1u);
        if (p < kcap)
          keys[p] = asm_key(rl & ((uint64_t(1) << bsh) - 1), v[j]);
        else
          set_error(err, ST_CAPACITY);
      }
      if (v[j] - row_lo < nrows) {
        const uint64_t rl = v[j] - row_lo;
        const uint32_t b = uint32_t(rl >> bsh);
        const uint64_t p = boff[b] + atomicAdd(&hcur[b], 1u);
        if (p < kcap)
          keys[p] = asm_key(rl & ((uint64_t(1) << bsh) - 1), u[j]);
        else
          set_error(err, ST_CAPACITY);
      }
    }
  }
}

// Per-row-block digest (sum of edge_hash over the entries) and out-degree
// histogram (65 bins, the last for 64 and more) of an assembly window, made
// while the entries are in shared memory; row block b of the window is
// b - b_lo.  Both pointers null: none.
struct AsmDigest {
  RowBounds rb;
  uint64_t b_lo;
  unsigned long long* digest;
  unsigned long long* hist;
};

struct AsmSmem {
  uint64_t key[ASM_CAP];   // (row in bucket) << 48 | column, as loaded
  uint64_t sorted[ASM_CAP];
  uint32_t rc[ASM_BR_MAX + 1];  // row counts -> row starts -> row cursors
  uint32_t nlong;
  // rows longer than ASM_ROW_WARP: a bucket of at most ASM_CAP entries has
  // fewer than ASM_CAP / ASM_ROW_WARP of them
  uint32_t longrow[ASM_CAP / ASM_ROW_WARP];
};

// Sorts row[0, len), len <= 8, by one thread: the 8-input network of
// lane_sort_row over registers padded with +infinity.
__device__ __forceinline__ void asm_lane_sort(uint64_t* row, uint32_t len) {
  uint64_t x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = uint32_t(i) < len ? row[i] : ~uint64_t(0);
  auto cx = [&](int i, int j) {
    const uint64_t a = x[i] < x[j] ? x[i] : x[j], c = x[i] < x[j] ? x[j] : x[i];
    x[i] = a;
    x[j] = c;
  };
  cx(0, 2); cx(1, 3); cx(4, 6); cx(5, 7);
  cx(0, 4); cx(1, 5); cx(2, 6); cx(3, 7);
  cx(0, 1); cx(2, 3); cx(4, 5); cx(6, 7);
  cx(2, 4); cx(3, 5);
  cx(1, 4); cx(3, 6);
  cx(1, 2); cx(3, 4); cx(5, 6);
#pragma unroll
  for (int i = 0; i < 8; ++i)
    if (uint32_t(i) < len) row[i] = x[i];
}

template <int E>
__device__ __forceinline__ void asm_warp_sort_e(uint64_t* row, uint32_t len, unsigned lane) {
  uint64_t x[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const uint32_t i = lane * E + e;
    x[e] = i < len ? row[i] : ~uint64_t(0);
  }
  warp_bitonic<E>(x, lane);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const uint32_t i = lane * E + e;
    if (i < len) row[i] = x[e];
  }
}

// Sorts row[0, len), len <= 256, by the whole warp (every lane calls it).
__device__ __forceinline__ void asm_warp_sort(uint64_t* row, uint32_t len, unsigned lane) {
  if (len <= 32)
    asm_warp_sort_e<1>(row, len, lane);
  else if (len <= 64)
    asm_warp_sort_e<2>(row, len, lane);
  else if (len <= 128)
    asm_warp_sort_e<4>(row, len, lane);
  else
    asm_warp_sort_e<8>(row, len, lane);
}

// Block-wide bitonic sort of x[0, n) (n <= ASM_CAP) in shared memory, ascending;
// positions past n act as +infinity (the first step of each merge compares
// mirrored positions and only moves the smaller value down).
__device__ __forceinline__ void asm_block_sort(uint64_t* x, uint32_t n) {
  uint32_t N = 1;
  int lgN = 0;
  while (N < n) {
    N <<= 1;
    ++lgN;
  }
  for (int lk = 1; lk <= lgN; ++lk) {
    const uint32_t k = 1u << lk;
    for (uint32_t i = threadIdx.x; i < N / 2; i += ASM_THREADS) {
      const uint32_t blk = i >> (lk - 1), off = i & (k / 2 - 1);
      const uint32_t lo = blk * k + off, hi = blk * k + k - 1 - off;
      if (hi < n && x[hi] < x[lo]) {
        const uint64_t t = x[lo];
        x[lo] = x[hi];
        x[hi] = t;
      }
    }
    __syncthreads();
    for (int lj = lk - 2; lj >= 0; --lj) {
      const uint32_t j = 1u << lj;
      for (uint32_t i = threadIdx.x; i < N / 2; i += ASM_THREADS) {
        const uint32_t blk = i >> lj, off = i & (j - 1);
        const uint32_t lo = blk * 2 * j + off, hi = lo + j;
        if (hi < n && x[hi] < x[lo]) {
          const uint64_t t = x[lo];
          x[lo] = x[hi];
          x[hi] = t;
        }
      }
      __syncthreads();
    }
  }
}

// One CTA per bucket (grid-stride): the bucket's entries sorted by (row,
// column) in shared memory, written back in place; rowptr[r] for its rows.
// Buckets over ASM_CAP entries go to big (sorted by asm_bucket_sort_global).
template <class Id>
__global__ void __launch_bounds__(ASM_THREADS)
    asm_bucket_sort(Id* __restrict__ out, const uint64_t* __restrict__ keys,
                    const uint64_t* __restrict__ boff, uint64_t row_lo,
                    uint64_t nrows, int bsh, uint32_t nb, uint64_t cap,
                    uint64_t* __restrict__ rowptr, unsigned long long* __restrict__ big,
                    unsigned long long* __restrict__ nbig, AsmDigest dig) {
  extern __shared__ __align__(16) unsigned char asm_raw[];
  AsmSmem& sm = *reinterpret_cast<AsmSmem*>(asm_raw);
  __shared__ unsigned long long sh_dig;
  __shared__ uint32_t sh_hist[65];
  const bool dg = dig.digest != nullptr || dig.hist != nullptr;
  for (uint32_t b = blockIdx.x; b < nb; b += gridDim.x) {
    const uint64_t e0 = boff[b], e1 = boff[b + 1];
    const uint64_t r0 = uint64_t(b) << bsh;
    const uint32_t nr = uint32_t(nrows - r0 < (uint64_t(1) << bsh) ? nrows - r0 : (1u << bsh));
    if (e1 > cap) {  // beyond the output (a capacity error was recorded): empty rows
      const uint64_t z = e0 < cap ? e0 : cap;
      for (uint32_t r = threadIdx.x; r < nr; r += ASM_THREADS) rowptr[r0 + r] = z;
      continue;
    }
    const uint64_t c64 = e1 - e0;
    if (c64 > ASM_CAP) {
      if (threadIdx.x == 0) big[atomicAdd(nbig, 1ull)] = b;
      continue;
    }
    const uint32_t c = uint32_t(c64);
    for (uint32_t r = threadIdx.x; r <= nr; r += ASM_THREADS) sm.rc[r] = 0;
    if (threadIdx.x == 0) sm.nlong = 0;
    if (threadIdx.x < 65) sh_hist[threadIdx.x] = 0;
    if (threadIdx.x == 0) sh_dig = 0;
    __syncthreads();
    // the bucket's keys, ASM_UNROLL loads in flight per thread
    for (uint32_t i = threadIdx.x; i < c; i += ASM_UNROLL * ASM_THREADS) {
      uint64_t k[ASM_UNROLL];
#pragma unroll
      for (int j = 0; j < ASM_UNROLL; ++j)
        if (i + j * ASM_THREADS < c) k[j] = keys[e0 + i + j * ASM_THREADS];
#pragma unroll
      for (int j = 0; j < ASM_UNROLL; ++j)
        if (i + j * ASM_THREADS < c) {
          sm.key[i + j * ASM_THREADS] = k[j];
          atomicAdd(&sm.rc[uint32_t(k[j] >> 48)], 1u);
        }
    }
    __syncthreads();
    // row starts: exclusive scan of the row counts (one thread per 8 rows)
    {
      const uint32_t per = (nr + ASM_THREADS - 1) / ASM_THREADS;
      const uint32_t a = threadIdx.x * per;
      uint32_t sum = 0;
      for (uint32_t q = 0; q < per && a + q < nr; ++q) sum += sm.rc[a + q];
      uint32_t tot;
      uint32_t run = block_inclusive_scan<ASM_THREADS>(sum, tot) - sum;
      for (uint32_t q = 0; q < per && a + q < nr; ++q) {
        const uint32_t cnt = sm.rc[a + q];
        sm.rc[a + q] = run;
        rowptr[r0 + a + q] = e0 + run;
        if (cnt > ASM_ROW_WARP) sm.longrow[atomicAdd(&sm.nlong, 1u)] = a + q;
        run += cnt;
      }
    }
    __syncthreads();
    // counting-sort placement (the order inside a row does not matter yet)
    for (uint32_t i = threadIdx.x; i < c; i += ASM_THREADS) {
      const uint64_t k = sm.key[i];
      sm.sorted[atomicAdd(&sm.rc[uint32_t(k >> 48)], 1u)] = k;
    }
    __syncthreads();
    // rc[r] is now the end of row r.  Every warp takes groups of 32 rows:
    // rows of at most ASM_ROW_LANE entries are sorted by their own lane, rows
    // up to ASM_ROW_WARP by the whole warp one after the other (a bitonic
    // network over registers and shuffles); longer rows wait for the block
    {
      const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
      for (uint32_t g = wid * 32; g < nr; g += ASM_THREADS) {  // uniform over the warp
        const uint32_t r = g + lane;
        uint32_t s0 = 0, len = 0;
        if (r < nr) {
          s0 = r ? sm.rc[r - 1] : 0;
          len = sm.rc[r] - s0;
        }
        if (len >= 2 && len <= ASM_ROW_LANE) asm_lane_sort(sm.sorted + s0, len);
        unsigned m = __ballot_sync(0xffffffffu, len > ASM_ROW_LANE && len <= ASM_ROW_WARP);
        while (m) {
          const int l = __ffs(m) - 1;
          m &= m - 1;
          const uint32_t bl = __shfl_sync(0xffffffffu, s0, l), dl = __shfl_sync(0xffffffffu, len, l);
          asm_warp_sort(sm.sorted + bl, dl, lane);
        }
      }
    }
    __syncthreads();
    // long rows by the whole block, one after the other
    const uint32_t nl = sm.nlong;
    for (uint32_t l = 0; l < nl; ++l) {
      const uint32_t r = sm.longrow[l];
      const uint32_t s1 = sm.rc[r], s0 = r ? sm.rc[r - 1] : 0;
      asm_block_sort(sm.sorted + s0, s1 - s0);
    }
    // the bucket's rows lie in one row block (almost always) or straddle several
    uint64_t bA = 0;
    bool one = true;
    if (dg) {
      bA = block_of_row(dig.rb, row_lo + r0);
      one = block_of_row(dig.rb, row_lo + r0 + nr - 1) == bA;
    }
    unsigned long long ds = 0;
    for (uint32_t i = threadIdx.x; i < c; i += ASM_THREADS) {
      const uint64_t k = sm.sorted[i];
      const uint64_t u = row_lo + r0 + (k >> 48), v = k & ((uint64_t(1) << 48) - 1);
      store_pair(out, e0 + i, u, v);
      if (dig.digest) {
        const unsigned long long h = edge_hash(u, v);
        if (one)
          ds += h;
        else
          atomicAdd(&dig.digest[block_of_row(dig.rb, u) - dig.b_lo], h);
      }
    }
    if (dg) {
      const unsigned lane = threadIdx.x & 31;
      if (dig.hist) {
        // rc[r] is the end of row r: degrees 0..7 counted in registers and
        // summed over the warp, longer ones in shared memory
        uint32_t c8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (uint32_t r = threadIdx.x; r < nr; r += ASM_THREADS) {
          const uint32_t deg = sm.rc[r] - (r ? sm.rc[r - 1] : 0u);
          const uint32_t bin = deg < 64 ? deg : 64;
          if (!one)
            atomicAdd(&dig.hist[(block_of_row(dig.rb, row_lo + r0 + r) - dig.b_lo) * 65 + bin], 1ull);
          else if (deg < 8)
            ++c8[deg];
          else
            atomicAdd(&sh_hist[bin], 1u);
        }
#pragma unroll
        for (int d = 0; d < 8; ++d) {
          const uint32_t t = __reduce_add_sync(0xffffffffu, c8[d]);
          if (lane == 0 && t) atomicAdd(&sh_hist[d], t);
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) ds += __shfl_xor_sync(0xffffffffu, ds, o);
      if (lane == 0 && ds) atomicAdd(&sh_dig, ds);
    }
    __syncthreads();
    // one atomic per bin and bucket (the same threads reset these at the next bucket)
    if (dg && one) {
      const uint64_t bi = bA - dig.b_lo;
      if (dig.digest && threadIdx.x == 0 && sh_dig) atomicAdd(&dig.digest[bi], sh_dig);
      if (dig.hist && threadIdx.x < 65 && sh_hist[threadIdx.x])
        atomicAdd(&dig.hist[bi * 65 + threadIdx.x], (unsigned long long)sh_hist[threadIdx.x]);
    }
  }
}

// The buckets over ASM_CAP entries: sorted in place in global memory by
// (row, column) (bitonic, one CTA per bucket), then each row's offset found
// by binary search.
template <class Id>
__global__ void __launch_bounds__(ASM_THREADS)
    asm_bucket_sort_global(Id* __restrict__ out, uint64_t* __restrict__ keys,
                           const uint64_t* __restrict__ boff, uint64_t row_lo, uint64_t nrows,
                           int bsh, uint64_t* __restrict__ rowptr,
                           const unsigned long long* __restrict__ big,
                           const unsigned long long* __restrict__ nbig, AsmDigest dig) {
  const unsigned long long nb = *nbig;
  for (unsigned long long q = blockIdx.x; q < nb; q += gridDim.x) {
    const uint32_t b = uint32_t(big[q]);
    const uint64_t e0 = boff[b], n = boff[b + 1] - e0;
    const uint64_t r0 = uint64_t(b) << bsh;
    const uint64_t nr = nrows - r0 < (uint64_t(1) << bsh) ? nrows - r0 : (uint64_t(1) << bsh);
    uint64_t* x = keys + e0;
    uint64_t N = 1;
    int lgN = 0;
    while (N < n) {
      N <<= 1;
      ++lgN;
    }
    // bitonic sort of the bucket's keys in place (positions past n act as +infinity)
    for (int lk = 1; lk <= lgN; ++lk) {
      const uint64_t k = uint64_t(1) << lk;
      for (uint64_t i = threadIdx.x; i < N / 2; i += ASM_THREADS) {
        const uint64_t blk = i >> (lk - 1), off = i & (k / 2 - 1);
        const uint64_t lo = blk * k + off, hi = blk * k + k - 1 - off;
        if (hi < n && x[hi] < x[lo]) {
          const uint64_t t = x[lo];
          x[lo] = x[hi];
          x[hi] = t;
        }
      }
      __syncthreads();
      for (int lj = lk - 2; lj >= 0; --lj) {
        const uint64_t j = uint64_t(1) << lj;
        for (uint64_t i = threadIdx.x; i < N / 2; i += ASM_THREADS) {
          const uint64_t blk = i >> lj, off = i & (j - 1);
          const uint64_t lo = blk * 2 * j + off, hi = lo + j;
          if (hi < n && x[hi] < x[lo]) {
            const uint64_t t = x[lo];
            x[lo] = x[hi];
            x[hi] = t;
          }
        }
        __syncthreads();
      }
    }
    // the entries in order, and the first entry of every row of the bucket
    for (uint64_t i = threadIdx.x; i < n; i += ASM_THREADS)
      store_pair(out, e0 + i, row_lo + r0 + (x[i] >> 48), x[i] & ((uint64_t(1) << 48) - 1));
    for (uint64_t r = threadIdx.x; r < nr; r += ASM_THREADS) {
      uint64_t a = 0, e = n;
      while (a < e) {
        const uint64_t mid = (a + e) >> 1;
        if ((x[mid] >> 48) < r)
          a = mid + 1;
        else
          e = mid;
      }
      rowptr[r0 + r] = e0 + a;
    }
    __syncthreads();
    // digest and degree histogram row by row (this path is rare: global atomics)
    if (dig.digest || dig.hist)
      for (uint64_t r = threadIdx.x; r < nr; r += ASM_THREADS) {
        const uint64_t s0 = rowptr[r0 + r], s1 = r + 1 < nr ? rowptr[r0 + r + 1] : e0 + n;
        const uint64_t row = row_lo + r0 + r;
        const uint64_t bi = block_of_row(dig.rb, row) - dig.b_lo;
        unsigned long long ds = 0;
        for (uint64_t e = s0; e < s1; ++e) ds += edge_hash(row, keys[e] & ((uint64_t(1) << 48) - 1));
        if (dig.digest && ds) atomicAdd(&dig.digest[bi], ds);
        if (dig.hist) atomicAdd(&dig.hist[bi * 65 + (s1 - s0 < 64 ? s1 - s0 : 64)], 1ull);
      }
    __syncthreads();
  }
}

}  // namespace kg
