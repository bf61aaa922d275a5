// C ABI: random geometric graphs RGG(n, r) in the unit square and cube
// (Sec. 5), with the count / prefix-sum / emit structure of the paper's GPU
// adaptation (Sec. 5, "Adaption to GPGPUs").
//
// Procedure (the same steps as the oracle, written independently):
//  * 32-bit fixed-point coordinates (x stands for x 2^-32); R = floor(r 2^32),
//    {u, v} is an edge iff sum_k (x_k(u) - x_k(v))^2 <= R^2 exactly.
//  * A grid of 2^g cells per dimension, cell side 2^(32-g) >= R, at most n
//    cells, g <= 15 (2D) / 10 (3D).
//  * Cell counts: the paper's recursive split of a cube into its 2^d subcubes,
//    each split done as d halvings (last dimension first), i.e. a binary tree
//    over the Morton index of the cells; node h draws the lower half's count
//    Binomial(c, 1/2) from its stream (tag 7): c fair bits for c <= 1024,
//    else the Sec. 2.2 binomial variate.
//  * Vertex ids follow the cells in row-major order (dimension 0 fastest),
//    then the draw order inside a cell; point j of the cell with Morton index
//    z takes the Philox block (j, z, tag 8): x_k = c_k 2^(32-g) + (w_k >> g).
//  * The neighbours of u lie in the cells that meet the box [x(u) - R,
//    x(u) + R]^d (a subset of the 3^d adjacent cells); visiting those cells in
//    row-major order and their points in id order gives every row sorted.
#include "kg.h"
#include "kg_common.cuh"
#include "kg_internal.h"
#include "kg_prof.h"
#include "kg_run.cuh"

namespace kg {
namespace {

constexpr uint32_t TAG_RGG_TREE = 7u;
constexpr uint32_t TAG_RGG_POINT = 8u;
constexpr uint64_t RGG_FAIR_BITS_MAX = 1024;
constexpr int RGG_CELLS_PER_BLOCK = 256;

cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

struct RggGrid {
  int dim, g;
  uint64_t n, R, cells;
};

int rgg_grid(int dim, uint64_t n, double r, RggGrid& G) {
  if (dim != 2 && dim != 3) return ST_ARG;
  if (!(r >= 0.0 && r <= 0.5)) return ST_ARG;  // also NaN
  if (n > 0xffffffffull) return ST_RANGE;
  G.dim = dim;
  G.n = n;
  G.R = uint64_t(r * 4294967296.0);  // exact scaling, truncation = floor
  const int gmax = dim == 2 ? 15 : 10;
  int g = 0;
  while (g < gmax) {
    const int h = g + 1;
    if ((uint64_t(1) << (32 - h)) < G.R) break;       // side would drop below R
    if ((uint64_t(1) << (dim * h)) > n) break;        // more cells than points
    g = h;
  }
  G.g = g;
  G.cells = uint64_t(1) << (dim * g);
  return ST_OK;
}

// In place over the Morton-indexed counts: node i of `level` keeps its count at
// position i << (D - level) and hands the upper half to i << (D - level) + half.
__global__ void __launch_bounds__(256)
    rgg_tree_level(uint32_t* __restrict__ cz, int D, int level, uint64_t root, uint64_t seed,
                   int* err) {
  const uint64_t nodes = uint64_t(1) << level;
  const int sh = D - level;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nodes;
       i += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t pos = i << sh;
    const uint64_t c = level == 0 ? root : cz[pos];
    uint64_t x = 0;
    if (c) {
      Stream s(seed, nodes + i, TAG_RGG_TREE);  // heap index of the node
      if (c <= RGG_FAIR_BITS_MAX) {
        x = popcount_bits(c, s);
      } else if (binomial(c, 0.5, s, x) != ST_OK) {
        set_error(err, ST_INTERNAL);
        x = 0;
      }
    }
    cz[pos] = uint32_t(x);
    cz[pos + (uint64_t(1) << (sh - 1))] = uint32_t(c - x);
  }
}

template <int DIM>
__host__ __device__ __forceinline__ uint64_t morton_of(const uint32_t* c, int g) {
  uint64_t z = 0;
  for (int b = 0; b < g; ++b)
#pragma unroll
    for (int k = 0; k < DIM; ++k) z |= uint64_t((c[k] >> b) & 1u) << (DIM * b + k);
  return z;
}

// Morton-indexed counts -> row-major counts (u64, the scan's input).
template <int DIM>
__global__ void __launch_bounds__(256)
    rgg_rowmajor(const uint32_t* __restrict__ cz, int g, uint64_t root,
                 uint64_t* __restrict__ cq) {
  const uint64_t cells = uint64_t(1) << (DIM * g);
  for (uint64_t z = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; z < cells;
       z += uint64_t(gridDim.x) * blockDim.x) {
    uint64_t q = 0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      uint64_t ck = 0;
      for (int b = 0; b < g; ++b) ck |= ((z >> (DIM * b + k)) & 1u) << b;
      q |= ck << (k * g);
    }
    cq[q] = g == 0 ? root : cz[z];
  }
}

// Points packed per vertex: (x, y) or (x, y, z, 0).
template <int DIM>
struct PtOf;
template <>
struct PtOf<2> {
  using T = uint2;
  __device__ __forceinline__ static uint32_t at(const uint2& p, int k) { return k ? p.y : p.x; }
};
template <>
struct PtOf<3> {
  using T = uint4;
  __device__ __forceinline__ static uint32_t at(const uint4& p, int k) {
    return k == 0 ? p.x : (k == 1 ? p.y : p.z);
  }
};

// One block per group of 256 consecutive cells: the group's points are spread
// over the block's threads, each finding its cell by a binary search over the
// group's starts in shared memory.
template <int DIM>
__global__ void __launch_bounds__(256)
    rgg_points(const uint64_t* __restrict__ S, int g, uint64_t seed,
               typename PtOf<DIM>::T* __restrict__ P, uint32_t* __restrict__ coords) {
  __shared__ uint64_t s_start[RGG_CELLS_PER_BLOCK + 1];
  const uint64_t cells = uint64_t(1) << (DIM * g);
  const uint32_t mask = (uint32_t(1) << g) - 1;
  const uint32_t k0 = uint32_t(seed), k1 = uint32_t(seed >> 32);
  for (uint64_t q0 = uint64_t(blockIdx.x) * RGG_CELLS_PER_BLOCK; q0 < cells;
       q0 += uint64_t(gridDim.x) * RGG_CELLS_PER_BLOCK) {
    const uint32_t nq =
        cells - q0 < RGG_CELLS_PER_BLOCK ? uint32_t(cells - q0) : uint32_t(RGG_CELLS_PER_BLOCK);
    for (uint32_t i = threadIdx.x; i <= nq; i += blockDim.x) s_start[i] = S[q0 + i];
    __syncthreads();
    const uint64_t p1 = s_start[nq];
    for (uint64_t p = s_start[0] + threadIdx.x; p < p1; p += blockDim.x) {
      uint32_t lo = 0, hi = nq;  // s_start[lo] <= p < s_start[hi]
      while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (s_start[mid] <= p)
          lo = mid;
        else
          hi = mid;
      }
      const uint64_t q = q0 + lo, j = p - s_start[lo];
      uint32_t c[DIM];
#pragma unroll
      for (int k = 0; k < DIM; ++k) c[k] = uint32_t(q >> (k * g)) & mask;
      const uint64_t z = morton_of<DIM>(c, g);
      uint32_t w[4];
      philox10(uint32_t(j), uint32_t(z), uint32_t(z >> 32), TAG_RGG_POINT, k0, k1, w);
      uint32_t x[3] = {0, 0, 0};
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        x[k] = uint32_t((uint64_t(c[k]) << (32 - g)) | (w[k] >> g));
        if (coords) coords[p * DIM + k] = x[k];
      }
      if constexpr (DIM == 2)
        P[p] = make_uint2(x[0], x[1]);
      else
        P[p] = make_uint4(x[0], x[1], x[2], 0u);
    }
    __syncthreads();
  }
}

// One 8- or 16-byte store of the entry (u, v) at slot i, marked evict-first
// so that the output stream does not push the points out of L2.
template <class Id>
__device__ __forceinline__ void rgg_store(Id* out, uint64_t i, uint64_t u, uint64_t v) {
  if (sizeof(Id) == 4)
    __stcs(reinterpret_cast<uint2*>(out) + i, make_uint2(uint32_t(u), uint32_t(v)));
  else
    __stcs(reinterpret_cast<ulonglong2*>(out) + i, make_ulonglong2(u, v));
}

// Count pass (EMIT = false: deg[u] = entries of row u) or emit pass (the
// entries of row u at rowptr[u] ..), one thread per vertex: the cells that
// meet the box [x(u) - R, x(u) + R]^d, row by row, their points in id order.
// Ids fit 32 bits (n < 2^32) and every coordinate difference that matters is
// <= R <= 2^31, so only the sum of squares needs 64 bits.
template <int DIM, bool EMIT, class Id>
__global__ void __launch_bounds__(256)
    rgg_edges(const typename PtOf<DIM>::T* __restrict__ P, uint32_t n, int g, uint32_t R,
              const uint64_t* __restrict__ S, unsigned long long* __restrict__ deg,
              const uint64_t* __restrict__ rowptr, Id* __restrict__ out, uint64_t cap,
              int* err) {
  using Pt = typename PtOf<DIM>::T;
  const int G = 1 << g;
  const int sh = 32 - g;
  const uint64_t R2 = uint64_t(R) * R;
  for (uint64_t uu = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; uu < n;
       uu += uint64_t(gridDim.x) * blockDim.x) {
    const uint32_t u = uint32_t(uu);
    const Pt pu = P[u];
    uint32_t xu[DIM];
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      xu[k] = PtOf<DIM>::at(pu, k);
      const int64_t a = int64_t(xu[k]) - R, b = int64_t(xu[k]) + R;
      lo[k] = a < 0 ? 0 : int(a >> sh);
      hi[k] = int(b >> sh) < G - 1 ? int(b >> sh) : G - 1;
    }
    uint64_t pos = EMIT ? rowptr[u] : 0;
    uint32_t cnt = 0;
    for (int d2 = lo[2]; d2 <= hi[2]; ++d2)
      for (int d1 = lo[1]; d1 <= hi[1]; ++d1) {
        const uint64_t row = (uint64_t(d2) * G + d1) * uint64_t(G);
        const uint32_t v0 = uint32_t(S[row + lo[0]]), v1 = uint32_t(S[row + hi[0] + 1]);
        for (uint32_t v = v0; v < v1; ++v) {
          const Pt pv = P[v];
          uint32_t m = 0;
          uint64_t s2 = 0;
#pragma unroll
          for (int k = 0; k < DIM; ++k) {
            const uint32_t dk = __usad(xu[k], PtOf<DIM>::at(pv, k), 0u);  // |x_k(u) - x_k(v)|
            m = m > dk ? m : dk;
            s2 += uint64_t(dk) * dk;  // may wrap when dk > R; then m > R
          }
          const bool hit = (m <= R) & (s2 <= R2) & (v != u);
          if (EMIT) {
            if (hit) {
              if (pos < cap)
                rgg_store(out, pos, u, v);
              else
                set_error(err, ST_CAPACITY);
              ++pos;
            }
          } else {
            cnt += hit;
          }
        }
      }
    if (!EMIT) deg[u] = cnt;
  }
}

enum class RggStop { CELLS, COUNT, EMIT };

// The whole procedure up to `stop`.  cq_out (optional) receives the row-major
// cell counts; d_count the number of entries (COUNT, EMIT).
template <int DIM>
int rgg_run(const RggGrid& G, uint64_t seed, RggStop stop, int id_bytes, void* d_out,
            uint64_t cap, uint64_t* d_count, uint32_t* d_coords, uint64_t* cq_out,
            cudaStream_t s) {
  int* err = device_error_word();
  if (!err) return ST_CUDA;
  Workspace ws(s);
  const int D = DIM * G.g;
  const uint64_t n = G.n;
  uint32_t* cz = ws.alloc<uint32_t>(G.cells);
  uint64_t* cq = cq_out ? cq_out : ws.alloc<uint64_t>(G.cells);
  if (!ws.ok()) return ST_CUDA;
  for (int level = 0; level < D; ++level) {
    ProfScope ps(PROF_RGG, s);
    rgg_tree_level<<<grid_for(uint64_t(1) << level, 256, sm_count() * 16), 256, 0, s>>>(cz, D, level,
                                                                                 n, seed, err);
    if (launch_ok()) return ST_CUDA;
  }
  {
    ProfScope ps(PROF_RGG, s);
    rgg_rowmajor<DIM><<<grid_for(G.cells, 256, sm_count() * 16), 256, 0, s>>>(cz, G.g, n, cq);
    if (launch_ok()) return ST_CUDA;
  }
  if (stop == RggStop::CELLS) return ST_OK;
  using Pt = typename PtOf<DIM>::T;
  uint64_t* S = ws.alloc<uint64_t>(G.cells + 1);
  Pt* P = ws.alloc<Pt>(n);
  unsigned long long* deg = ws.alloc<unsigned long long>(n);
  uint64_t* rowptr = ws.alloc<uint64_t>(n + 1);
  if (!ws.ok()) return ST_CUDA;
  int st = scan_exclusive_u64(cq, S, G.cells, ws, s);
  if (st) return st;
  {
    ProfScope ps(PROF_RGG, s);
    rgg_points<DIM><<<grid_for(G.cells, RGG_CELLS_PER_BLOCK, sm_count() * 8), 256, 0, s>>>(
        S, G.g, seed, P, d_coords);
    if (launch_ok()) return ST_CUDA;
  }
  const unsigned eblocks = grid_for(n, 256, sm_count() * 16);
  {
    ProfScope ps(PROF_RGG, s);
    rgg_edges<DIM, false, uint32_t><<<eblocks, 256, 0, s>>>(P, uint32_t(n), G.g, uint32_t(G.R), S,
                                                             deg, nullptr, nullptr, 0, err);
    if (launch_ok()) return ST_CUDA;
  }
  st = scan_exclusive_u64(reinterpret_cast<const uint64_t*>(deg), rowptr, n, ws, s);
  if (st) return st;
  if (cudaMemcpyAsync(d_count, rowptr + n, sizeof(uint64_t), cudaMemcpyDeviceToDevice, s) !=
      cudaSuccess)
    return ST_CUDA;
  if (stop == RggStop::COUNT) return ST_OK;
  ProfScope ps(PROF_RGG, s);
  if (id_bytes == 4)
    rgg_edges<DIM, true, uint32_t><<<eblocks, 256, 0, s>>>(P, uint32_t(n), G.g, uint32_t(G.R), S,
                                                            nullptr, rowptr,
                                                            static_cast<uint32_t*>(d_out), cap, err);
  else
    rgg_edges<DIM, true, uint64_t><<<eblocks, 256, 0, s>>>(P, uint32_t(n), G.g, uint32_t(G.R), S,
                                                            nullptr, rowptr,
                                                            static_cast<uint64_t*>(d_out), cap, err);
  return launch_ok();
}

int rgg_dispatch(const RggGrid& G, uint64_t seed, RggStop stop, int id_bytes, void* d_out,
                 uint64_t cap, uint64_t* d_count, uint32_t* d_coords, uint64_t* cq_out,
                 cudaStream_t s) {
  return G.dim == 2
             ? rgg_run<2>(G, seed, stop, id_bytes, d_out, cap, d_count, d_coords, cq_out, s)
             : rgg_run<3>(G, seed, stop, id_bytes, d_out, cap, d_count, d_coords, cq_out, s);
}

}  // namespace
}  // namespace kg

using namespace kg;

extern "C" {

kg_status kg_rgg_grid(int dim, uint64_t n, double r, int* g_out) {
  if (!g_out) return KG_ERR_ARG;
  RggGrid G;
  const int st = rgg_grid(dim, n, r, G);
  if (st) return kg_status(st);
  *g_out = G.g;
  return KG_OK;
}

kg_status kg_rgg_cell_counts(int dim, uint64_t n, double r, uint64_t seed, uint64_t* d_counts,
                             void* stream) {
  RggGrid G;
  const int st = rgg_grid(dim, n, r, G);
  if (st) return kg_status(st);
  if (!d_counts) return KG_ERR_ARG;
  return kg_status(rgg_dispatch(G, seed, RggStop::CELLS, 4, nullptr, 0, nullptr, nullptr,
                                d_counts, as_stream(stream)));
}

kg_status kg_rgg_count(int dim, uint64_t n, double r, uint64_t seed, uint64_t* d_count,
                       void* stream) {
  RggGrid G;
  const int st = rgg_grid(dim, n, r, G);
  if (st) return kg_status(st);
  if (!d_count) return KG_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  if (n == 0) return cudaMemsetAsync(d_count, 0, 8, s) == cudaSuccess ? KG_OK : KG_ERR_CUDA;
  return kg_status(
      rgg_dispatch(G, seed, RggStop::COUNT, 4, nullptr, 0, d_count, nullptr, nullptr, s));
}

kg_status kg_rgg(int dim, uint64_t n, double r, uint64_t seed, int id_bytes, void* d_out,
                 uint64_t cap_entries, uint64_t* d_count, uint32_t* d_coords, void* stream) {
  RggGrid G;
  const int st = rgg_grid(dim, n, r, G);
  if (st) return kg_status(st);
  if (id_bytes != 4 && id_bytes != 8) return KG_ERR_ARG;
  if (!d_count || (cap_entries > 0 && !d_out)) return KG_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  if (n == 0) return cudaMemsetAsync(d_count, 0, 8, s) == cudaSuccess ? KG_OK : KG_ERR_CUDA;
  return kg_status(rgg_dispatch(G, seed, RggStop::EMIT, id_bytes, d_out, cap_entries, d_count,
                                d_coords, nullptr, s));
}

}  // extern "C"
