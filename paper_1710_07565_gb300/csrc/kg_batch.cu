// Batched G(n,m): many independent instances (directed or undirected, each
// with its own n, m, seed and chunk count) generated by one fixed sequence of
// kernels over all instances.  kg_batch_create lays the instances out and
// uploads their table once; kg_batch_run only enqueues device work (no
// allocation, no host synchronisation), so the whole batch can be captured
// into one CUDA graph and replayed.  The output is the concatenation, in
// instance order, of what the per-instance entry points write.
#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "kg.h"
#include "kg_batch.h"
#include "kg_run.cuh"
#include "kg_und.cuh"
#include "kg_assemble.cuh"

namespace kg {

struct BInst {
  uint64_t n, m, seed;
  uint32_t P, undirected;
  uint32_t big, pad_;  // big: an undirected instance assembled by the per-instance sequence
  // binom: G(n,p) by binomial chunk counts (Sec. 4.3): the chunk counts are
  // Binomial(U_c, p) (their sum, m, is known beforehand from the count pass),
  // and the chunks are then sampled like G(n,m) chunks
  uint32_t binom, pad2_;
  double p;
  int d, D;
  uint64_t C;
  uint64_t chunk_base, tile_base, sample_base, pair_base, vert_base, out_base;
  // pairs of the small undirected instances before this one: the small
  // instances' pairs come first in the pair buffer (pair_base == spair_base
  // for them), the big ones' after all of them; vert_base counts the small
  // instances' vertices only
  uint64_t spair_base;
  RowBounds rb;
  DivU64 div;  // by n-1 (directed)
};

// Geometry context of one chunk of any instance.
struct BatchCtx {
  uint64_t nm1, r0, ri, rj, sj;
  DivU64 div;
  int kind;  // 0 directed, 1 undirected rectangle, 2 undirected triangle
};

struct BatchGeom {
  using Ctx = BatchCtx;
  __device__ __forceinline__ void map(const Ctx& x, uint64_t off, uint64_t& u, uint64_t& v) const {
    if (x.kind == 0) {
      const uint64_t q = div_q(x.div, off);
      const uint64_t w = off - q * x.nm1;
      u = x.r0 + q;
      v = w + (w >= u ? 1 : 0);
    } else if (x.kind == 1) {
      const uint64_t q = rect_row(off, x.sj);
      u = x.ri + q;
      v = x.rj + (off - q * x.sj);
    } else {
      const uint64_t w = tri_row(off);
      u = x.ri + w;
      v = x.ri + (off - uint64_t(u128(w) * (w - 1) / 2));
    }
  }
  __device__ __forceinline__ uint64_t rows(uint64_t) const { return 0; }
};

// The sparse leaf kernel's map of a directed or rectangle tile of a batch
// (batch_desc routes only those, with aux0 = lo mod D and aux1 = the row of lo).
__device__ __forceinline__ void sparse_tile_map(const TileDesc<BatchCtx>& td, SparseTileMap& m) {
  const int kind = td.gx.kind;
  m.D = kind == 0 ? td.gx.nm1 : td.gx.sj;
  m.col0 = kind == 0 ? 0 : td.gx.rj;
  m.skip = kind == 0;
  m.y0 = td.aux0;
  m.u0 = td.aux1;
  if (!sparse_map_dev(m.D, m.M, m.s)) {
    m.M = 0;
    m.s = 0;
  }
}

// Output positions below 2^62 go to the final output, those with bit 62 set
// to the undirected pair scratch.
constexpr uint64_t SCRATCH_BIT = uint64_t(1) << 62;

struct BatchSink {
  uint32_t* out;
  uint32_t* scratch;
  uint64_t cap_out, cap_scratch;
  int* err;
  __device__ __forceinline__ void write(uint64_t pos, uint64_t u, uint64_t v) const {
    uint32_t* dst = out;
    uint64_t cap = cap_out;
    if (pos & SCRATCH_BIT) {
      pos &= ~SCRATCH_BIT;
      dst = scratch;
      cap = cap_scratch;
    }
    if (pos >= cap) {
      set_error(err, ST_CAPACITY);
      return;
    }
    uint2 w;
    w.x = uint32_t(u);
    w.y = uint32_t(v);
    reinterpret_cast<uint2*>(dst)[pos] = w;
  }
  // whether slots [base, base + k) exist (base may carry SCRATCH_BIT)
  __device__ __forceinline__ bool fits(uint64_t base, uint64_t k) const {
    const uint64_t cap = (base & SCRATCH_BIT) ? cap_scratch : cap_out;
    base &= ~SCRATCH_BIT;
    return base <= cap && k <= cap - base;
  }
  // store to a slot already checked by fits()
  __device__ __forceinline__ void put(uint64_t pos, uint64_t u, uint64_t v) const {
    uint32_t* dst = (pos & SCRATCH_BIT) ? scratch : out;
    uint2 w;
    w.x = uint32_t(u);
    w.y = uint32_t(v);
    reinterpret_cast<uint2*>(dst)[pos & ~SCRATCH_BIT] = w;
  }
  __device__ __forceinline__ uint64_t read_u(uint64_t pos) const {
    const uint32_t* src = (pos & SCRATCH_BIT) ? scratch : out;
    return src[2 * (pos & ~SCRATCH_BIT)];
  }
};

// index i with base[i] <= x < base[i+1] (base non-decreasing, base[count] = total)
__device__ __forceinline__ uint32_t find_inst(const BInst* __restrict__ inst, uint32_t count,
                                              uint64_t x, int which) {
  uint32_t a = 0, b = count;
  while (b - a > 1) {
    const uint32_t mid = (a + b) >> 1;
    const uint64_t v = which == 0   ? inst[mid].tile_base
                       : which == 1 ? inst[mid].spair_base
                       : which == 2 ? inst[mid].vert_base
                                    : inst[mid].out_base;
    if (v <= x)
      a = mid;
    else
      b = mid;
  }
  return a;
}

// find_inst for 32 consecutive positions p (lane l holds p0 + l; every lane
// of the warp calls it): one search by lane 0, and a search of its own only
// for a lane past the next instance's start.
__device__ __forceinline__ uint32_t warp_find_inst(const BInst* __restrict__ inst, uint32_t count,
                                                   uint64_t p, int which, unsigned lane) {
  const uint64_t p0 = __shfl_sync(0xffffffffu, p, 0);
  uint32_t i0 = 0;
  if (lane == 0) i0 = find_inst(inst, count, p0, which);
  i0 = __shfl_sync(0xffffffffu, i0, 0);
  uint64_t nxt = ~uint64_t(0);
  if (i0 + 1 < count)
    nxt = which == 0   ? inst[i0 + 1].tile_base
          : which == 1 ? inst[i0 + 1].spair_base
          : which == 2 ? inst[i0 + 1].vert_base
                       : inst[i0 + 1].out_base;
  return p < nxt ? i0 : find_inst(inst, count, p, which);
}

__device__ __forceinline__ uint64_t b_universe(const BInst& I, uint64_t c) {
  if (!I.undirected) return (I.rb(c + 1) - I.rb(c)) * (I.n - 1);
  uint32_t i, j;
  UndGeom::ij(c, i, j);
  const uint64_t si = I.rb(uint64_t(i) + 1) - I.rb(i);
  if (i == j) return si ? uint64_t(u128(si) * (si - 1) / 2) : 0;
  return si * (I.rb(uint64_t(j) + 1) - I.rb(j));
}

__device__ __forceinline__ uint64_t b_chunk_id(const BInst& I, uint64_t c) {
  if (!I.undirected) return c;
  uint32_t i, j;
  UndGeom::ij(c, i, j);
  return uint64_t(i) * I.P + j;
}

// ---------------------------------------------------------------- trees
// One block per instance: the chunk counts, by the chunk split tree
// (directed), the quadrant tree (undirected) or the chunk binomials (G(n,p));
// an instance without tile levels (d = 0) copies them to its tile counts.
// The tile trees follow level by level over all instances (batch_tile_level).
constexpr int BT_MAXC = 32 * 33 / 2;  // undirected chunks at P <= 32

__global__ void __launch_bounds__(256)
    batch_trees(const BInst* __restrict__ inst, uint64_t* __restrict__ chunk_cnt,
                uint64_t* __restrict__ tile_cnt, int* err) {
  __shared__ uint64_t node_cnt[128];
  __shared__ QNode ql[2][BT_MAXC];
  __shared__ uint32_t qn[2];
  const BInst I = inst[blockIdx.x];
  const int tid = threadIdx.x;
  uint64_t* cc = chunk_cnt + I.chunk_base;
  if (I.binom) {
    // as gnp_chunk_counts: chunk c draws Binomial(U_c, p) from (seed, chunk id)
    for (uint64_t c = tid; c < I.C; c += blockDim.x) {
      Stream st(I.seed, b_chunk_id(I, c), TAG_GNP_COUNT);
      uint64_t x = 0;
      const int e = binomial(b_universe(I, c), I.p, st, x, BINOM_N_MAX);
      if (e) {
        set_error(err, e);
        x = 0;
      }
      cc[c] = x;
    }
  } else if (!I.undirected) {
    if (tid == 0) node_cnt[1] = I.m;
    __syncthreads();
    // one warp per node (warp-cooperative variates: P <= 64, so every level
    // holds at most 32 nodes for the block's warps)
    const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int level = 0; level <= I.D; ++level) {
      for (uint64_t j = wid; j < (uint64_t(1) << level); j += nw) {  // uniform over the warp
        const uint64_t h = (uint64_t(1) << level) + j;
        uint32_t a, b;
        if (!chunk_range(I.P, h, level, a, b)) continue;
        const uint64_t mc = node_cnt[h];
        if (b - a == 1) {
          if (lane == 0) cc[a] = mc;
          continue;
        }
        const uint32_t s = a + (b - a + 1) / 2;
        const uint64_t ra = I.rb(a);
        const u128 N = u128(I.rb(b) - ra) * (I.n - 1);
        const u128 NL = u128(I.rb(s) - ra) * (I.n - 1);
        uint64_t X = 0;
        const int e = hypergeometric_warp(N, NL, mc, I.seed, h, TAG_CHUNK_TREE, X);
        if (lane == 0) {
          if (e) {
            set_error(err, e);
            X = 0;
          }
          node_cnt[2 * h] = X;
          node_cnt[2 * h + 1] = mc - X;
        }
      }
      __syncthreads();
    }
  } else {
    if (tid == 0) {
      ql[0][0] = QNode{0, I.P, 0, I.P, I.m};
      qn[0] = 1;
      qn[1] = 0;
    }
    __syncthreads();
    for (int level = 0; level <= I.D; ++level) {
      const int cur = level & 1, nxt = cur ^ 1;
      const uint32_t count = qn[cur];
      for (uint32_t idx = tid; idx < count; idx += blockDim.x) {
        const QNode q = ql[cur][idx];
        const bool tri = (q.a == q.c && q.b == q.d);
        if ((tri && q.b - q.a == 1) || (!tri && q.b - q.a == 1 && q.d - q.c == 1)) {
          cc[und_chunk_index(q.a, q.c)] = q.cnt;
          continue;
        }
        Stream st(I.seed, quad_id(q.a, q.b, q.c, q.d), TAG_QUAD);
        QNode parts[4];
        u128 size[4];
        int np = 0;
        if (tri) {
          const uint32_t l = (q.b - q.a + 1) / 2;
          const uint64_t ra = I.rb(q.a), rm = I.rb(q.a + l), rbb = I.rb(q.b);
          const uint64_t S1 = rm - ra, S2 = rbb - rm;
          parts[0] = QNode{q.a, q.a + l, q.a, q.a + l, 0};
          parts[1] = QNode{q.a + l, q.b, q.a, q.a + l, 0};
          parts[2] = QNode{q.a + l, q.b, q.a + l, q.b, 0};
          size[0] = tri_pairs(S1);
          size[1] = u128(S2) * S1;
          size[2] = tri_pairs(S2);
          np = 3;
        } else {
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
          for (int i = 0; i < nr; ++i)
            for (int j = 0; j < nc; ++j) {
              parts[np] = QNode{rlo[i], rhi[i], clo[j], chi[j], 0};
              size[np] = u128(I.rb(rhi[i]) - I.rb(rlo[i])) * (I.rb(chi[j]) - I.rb(clo[j]));
              ++np;
            }
        }
        u128 N = 0;
        for (int i = 0; i < np; ++i) N += size[i];
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
        const uint32_t o = atomicAdd(&qn[nxt], uint32_t(np));
        for (int i = 0; i < np; ++i)
          if (o + i < BT_MAXC) ql[nxt][o + i] = parts[i];
      }
      __syncthreads();
      if (tid == 0) qn[cur] = 0;
      __syncthreads();
    }
  }
  __syncthreads();
  if (I.d == 0)
    for (uint64_t c = tid; c < I.C; c += blockDim.x) tile_cnt[I.tile_base + c] = cc[c];
}

// Level bases of the tile trees: row L (L < maxd) of `base` holds, for every
// instance i, the level-L nodes of the instances before i that have a level L
// (d > L: C 2^L nodes each), and in column count their total.
__global__ void __launch_bounds__(1024)
    batch_level_bases(const BInst* __restrict__ inst, uint32_t count, uint64_t* __restrict__ base) {
  const int L = int(blockIdx.x);
  uint64_t* b = base + uint64_t(L) * (count + 1);
  uint64_t carry = 0;
  for (uint32_t i0 = 0; i0 < count; i0 += 1024) {
    const uint32_t i = i0 + threadIdx.x;
    uint64_t x = 0;
    if (i < count && inst[i].d > L) x = inst[i].C << L;
    uint64_t tot;
    const uint64_t incl = block_inclusive_scan<1024>(x, tot);
    if (i < count) b[i] = carry + incl - x;
    carry += tot;
  }
  if (threadIdx.x == 0) b[count] = carry;
}

// Level L of every instance's tile tree (Sec. 4.1: a node's count splits
// between its two halves by a hypergeometric draw from the node's own
// stream), one thread per node over all instances: node t belongs to the
// instance i with base[i] <= t < base[i + 1].  Level L reads the chunk counts
// (L = 0) or level L - 1, and writes level L + 1; levels alternate between tmp
// and tile_cnt so that the last lands in tile_cnt.
__global__ void __launch_bounds__(256)
    batch_tile_level(const BInst* __restrict__ inst, uint32_t count, int L,
                     const uint64_t* __restrict__ base, const uint64_t* __restrict__ chunk_cnt,
                     uint64_t* __restrict__ tmp, uint64_t* __restrict__ tile_cnt, int* err) {
  const uint64_t total = base[count];
  for (uint64_t t = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
       t += uint64_t(gridDim.x) * blockDim.x) {
    uint32_t a = 0, b = count;
    while (b - a > 1) {
      const uint32_t mid = (a + b) >> 1;
      if (base[mid] <= t)
        a = mid;
      else
        b = mid;
    }
    const BInst& I = inst[a];
    const int d = I.d;
    const uint64_t node = t - base[a];
    const uint64_t c = node >> L;
    const uint64_t j = node & ((uint64_t(1) << L) - 1);
    const uint64_t* in =
        L == 0 ? chunk_cnt + I.chunk_base : (((d - L) & 1) ? tmp : tile_cnt) + I.tile_base;
    uint64_t* out = (((d - 1 - L) & 1) ? tmp : tile_cnt) + I.tile_base;
    const uint64_t U = b_universe(I, c);
    const uint64_t W = tile_width(U, d);
    const uint64_t lo = node_bound(U, W, d, L, j);
    const uint64_t hi = node_bound(U, W, d, L, u128(j) + 1);
    const uint64_t mid = node_bound(U, W, d, L + 1, u128(2) * j + 1);
    const uint64_t k = in[node];
    const uint64_t sid = (b_chunk_id(I, c) << 32) | ((uint64_t(1) << L) + j);
    uint64_t X = 0;
    int e = ST_INTERNAL;
    if (k <= hi - lo) {
      Stream st(I.seed, sid, TAG_TILE);
      e = hypergeometric(u128(hi - lo), u128(mid - lo), k, st, X);
    }
    if (e) {
      set_error(err, e);
      X = 0;
    }
    out[2 * node] = X;
    out[2 * node + 1] = k - X;
  }
}

// ---------------------------------------------------------------- tile descriptors

__global__ void __launch_bounds__(256)
    batch_desc(const BInst* __restrict__ inst, uint32_t count, uint64_t ntiles, uint32_t k_max,
               const uint64_t* __restrict__ tile_cnt, const uint64_t* __restrict__ tile_off,
               TileDesc<BatchCtx>* __restrict__ desc, unsigned long long* big,
               unsigned long long* nbig, int* err, bool sparse) {
  for (uint64_t t = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < ntiles;
       t += uint64_t(gridDim.x) * blockDim.x) {
    const uint32_t ii = find_inst(inst, count, t, 0);
    const BInst I = inst[ii];
    const uint64_t local = t - I.tile_base;
    const uint64_t c = local >> I.d;
    const uint64_t tau = local & ((uint64_t(1) << I.d) - 1);
    TileDesc<BatchCtx> td;
    desc_fill(td, b_universe(I, c), I.d, tau, tile_cnt[t], k_max, err);
    const uint64_t local_pos = tile_off[t] - I.sample_base;
    td.base = I.undirected ? (SCRATCH_BIT | (I.pair_base + local_pos)) : (I.out_base + local_pos);
    td.cid = b_chunk_id(I, c);
    td.seed = I.seed;
    BatchCtx x;
    x.nm1 = I.n - 1;
    x.div = I.div;
    if (!I.undirected) {
      x.kind = 0;
      x.r0 = I.rb(c);
    } else {
      uint32_t i, j;
      UndGeom::ij(c, i, j);
      x.kind = (i == j) ? 2 : 1;
      x.ri = I.rb(i);
      x.rj = I.rb(j);
      x.sj = I.rb(uint64_t(j) + 1) - x.rj;
    }
    td.gx = x;
    if (sparse && td.flags == 0) {
      // the sparse leaf kernel takes directed and rectangle tiles whose map
      // constants exist and whose in-row offsets stay below 2^(31+s); the
      // general kernel samples the rest from the fallback list
      bool ok = x.kind != 2 && td.k <= uint32_t(SP_KMAX) && td.L > SP_NB;
      if (ok) {
        const uint64_t D = x.kind == 0 ? x.nm1 : x.sj;
        uint32_t M;
        int sh;
        ok = sparse_map_dev(D, M, sh);
        if (ok) {
          const uint64_t q = x.kind == 0 ? div_q(x.div, td.lo) : rect_row(td.lo, D);
          td.aux0 = td.lo - q * D;
          td.aux1 = (x.kind == 0 ? x.r0 : x.ri) + q;
          const uint64_t ymax = uint64_t(1) << (31 + sh);
          ok = td.aux0 < ymax && td.L - 1 < ymax - td.aux0;
        }
      }
      if (!ok) {
        td.flags = 3;
        big[ntiles - 1 - atomicAdd(nbig + 1, 1ull)] = t;
      }
    }
    if (td.flags == 1) big[atomicAdd(nbig, 1ull)] = t;
    desc[t] = td;
  }
}

// ---------------------------------------------------------------- undirected assembly
__global__ void batch_und_degree(const BInst* __restrict__ inst, uint32_t count, uint64_t npairs,
                                 const uint32_t* __restrict__ pairs,
                                 unsigned long long* __restrict__ deg) {
  const unsigned lane = threadIdx.x & 31;
  for (uint64_t p0 = uint64_t(blockIdx.x) * blockDim.x + (threadIdx.x & ~31u); p0 < npairs;
       p0 += uint64_t(gridDim.x) * blockDim.x) {  // uniform over the warp
    const uint64_t p = p0 + lane;
    const BInst& I = inst[warp_find_inst(inst, count, p < npairs ? p : npairs - 1, 1, lane)];
    if (p < npairs && !I.big) {
      const uint64_t vb = I.vert_base;
      atomicAdd(&deg[vb + pairs[2 * p]], 1ull);
      atomicAdd(&deg[vb + pairs[2 * p + 1]], 1ull);
    }
  }
}

// absolute output position of the first entry of every undirected row
__global__ void batch_und_rowpos(const BInst* __restrict__ inst, uint32_t count, uint64_t nverts,
                                 const uint64_t* __restrict__ rowptr,
                                 unsigned long long* __restrict__ rowpos) {
  for (uint64_t r = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < nverts;
       r += uint64_t(gridDim.x) * blockDim.x) {
    const BInst& I = inst[find_inst(inst, count, r, 2)];
    rowpos[r] = rowptr[r] - rowptr[I.vert_base] + I.out_base;
  }
}

__global__ void batch_und_scatter(const BInst* __restrict__ inst, uint32_t count, uint64_t npairs,
                                  const uint32_t* __restrict__ pairs,
                                  unsigned long long* __restrict__ cursor,
                                  uint32_t* __restrict__ out, uint64_t cap, int* err) {
  const unsigned lane = threadIdx.x & 31;
  for (uint64_t p0 = uint64_t(blockIdx.x) * blockDim.x + (threadIdx.x & ~31u); p0 < npairs;
       p0 += uint64_t(gridDim.x) * blockDim.x) {  // uniform over the warp
    const uint64_t p = p0 + lane;
    const BInst& I = inst[warp_find_inst(inst, count, p < npairs ? p : npairs - 1, 1, lane)];
    if (p >= npairs || I.big) continue;
    const uint64_t vb = I.vert_base;
    const uint32_t u = pairs[2 * p], v = pairs[2 * p + 1];
    const uint64_t a = atomicAdd(&cursor[vb + u], 1ull);
    const uint64_t b = atomicAdd(&cursor[vb + v], 1ull);
    if (a < cap && b < cap) {
      reinterpret_cast<uint2*>(out)[a] = make_uint2(u, v);
      reinterpret_cast<uint2*>(out)[b] = make_uint2(v, u);
    } else {
      set_error(err, ST_CAPACITY);
    }
  }
}

// Rows of <= WARP_SORT_MAX entries sorted by their lane or their warp; longer rows listed.
__global__ void __launch_bounds__(256)
    batch_und_sort_short(uint64_t nverts, const unsigned long long* __restrict__ rowpos,
                         const unsigned long long* __restrict__ deg, uint32_t* __restrict__ out,
                         uint64_t cap, unsigned long long* long_rows, unsigned long long* nlong) {
  const unsigned lane = threadIdx.x & 31;
  const uint64_t warp = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  for (uint64_t r0 = warp * 32; r0 < nverts; r0 += nwarps * 32) {  // uniform over the warp
    const uint64_t r = r0 + lane;
    uint64_t b = 0, dg = 0;
    if (r < nverts) {
      b = rowpos[r];
      dg = deg[r];
      if (b + dg > cap) dg = 0;
    }
    sort_rows_of_warp(out, b, dg, r, lane, long_rows, nlong);
  }
}

__global__ void __launch_bounds__(256)
    batch_und_sort_long(const unsigned long long* __restrict__ rowpos,
                        const unsigned long long* __restrict__ deg, uint32_t* __restrict__ out,
                        const unsigned long long* __restrict__ long_rows,
                        const unsigned long long* __restrict__ nlong) {
  __shared__ uint64_t sh[LONG_SMEM];
  const unsigned long long nl = *nlong;
  for (unsigned long long q = blockIdx.x; q < nl; q += gridDim.x) {
    const uint64_t r = long_rows[q];
    const uint64_t b = rowpos[r], n = deg[r];
    uint64_t N = 1;
    int lgN = 0;
    while (N < n) {
      N <<= 1;
      ++lgN;
    }
    const bool in_smem = n <= LONG_SMEM;
    if (in_smem)
      for (uint64_t i = threadIdx.x; i < n; i += blockDim.x) sh[i] = out[2 * (b + i) + 1];
    __syncthreads();
    auto get = [&](uint64_t i) -> uint64_t { return in_smem ? sh[i] : uint64_t(out[2 * (b + i) + 1]); };
    auto put = [&](uint64_t i, uint64_t x) {
      if (in_smem)
        sh[i] = x;
      else
        out[2 * (b + i) + 1] = uint32_t(x);
    };
    for (int lk = 1; lk <= lgN; ++lk) {
      const uint64_t k = uint64_t(1) << lk;
      for (uint64_t i = threadIdx.x; i < N / 2; i += blockDim.x) {
        const uint64_t blk = i >> (lk - 1), off = i & (k / 2 - 1);
        const uint64_t lo = blk * k + off, hi = blk * k + k - 1 - off;
        if (hi < n) {
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
          if (hi < n) {
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
      for (uint64_t i = threadIdx.x; i < n; i += blockDim.x) out[2 * (b + i) + 1] = uint32_t(sh[i]);
    __syncthreads();
  }
}

// ---------------------------------------------------------------- per-instance digests
// digest[i] += sum of splitmix64(u ^ rotl(v, 32)) over the entries of
// instance i (kg_edge_digest of its output); a warp takes 32 consecutive
// entries and adds them with one atomic when they belong to one instance.
__global__ void __launch_bounds__(256)
    batch_digests(const BInst* __restrict__ inst, uint32_t count, uint64_t entries,
                  const uint32_t* __restrict__ out, unsigned long long* __restrict__ dig) {
  const unsigned lane = threadIdx.x & 31;
  for (uint64_t p0 = uint64_t(blockIdx.x) * blockDim.x + (threadIdx.x & ~31u); p0 < entries;
       p0 += uint64_t(gridDim.x) * blockDim.x) {  // uniform over the warp
    const uint64_t p = p0 + lane;
    const uint32_t ii = warp_find_inst(inst, count, p < entries ? p : entries - 1, 3, lane);
    unsigned long long h = 0;
    if (p < entries) {
      const uint2 e = reinterpret_cast<const uint2*>(out)[p];
      h = edge_hash(e.x, e.y);
    }
    const uint32_t i0 = __shfl_sync(0xffffffffu, ii, 0);
    if (__all_sync(0xffffffffu, ii == i0)) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
      if (lane == 0) atomicAdd(&dig[i0], h);
    } else if (p < entries) {
      atomicAdd(&dig[ii], h);
    }
  }
}

// ---------------------------------------------------------------- the plan
struct BatchPlan {
  int device;
  uint32_t count;
  uint64_t tiles, chunks, pairs, verts, entries, samples;
  uint64_t spairs;  // pairs of the small undirected instances (the first spairs of the buffer)
  std::vector<uint64_t> level_nodes;  // tile-tree nodes of level L over all instances (L < maxd)
  int has_und;
  std::vector<uint64_t> out_offsets;  // count + 1
  // device memory owned by the plan
  BInst* inst;
  uint64_t *chunk_cnt, *tile_tmp, *tile_cnt, *tile_off;
  uint64_t* lvl_base;  // level_nodes.size() rows of count + 1 (batch_level_bases)
  TileDesc<BatchCtx>* desc;
  unsigned long long *big, *nbig;
  uint32_t* pairs_buf;
  unsigned long long *deg, *rowpos, *cursor, *long_rows, *nlong;
  uint64_t* rowptr;
  ScanScratch scan_t, scan_v;  // the run's two scans (tiles, vertices)
  // undirected instances of at least BIG_PAIRS pairs: assembled one by one
  // with the per-instance sequence (scratch carved from big_arena each time)
  struct Big {
    uint64_t n, m, pair_base, out_base;
  };
  std::vector<Big> bigs;
  void* big_arena = nullptr;  // big_lanes areas of big_arena_bytes
  size_t big_arena_bytes = 0;
  // the big instances run on big_lanes streams forked from the caller's
  // stream and joined back (capturable): big k on lane big_lane[k], chosen
  // largest first onto the least loaded lane; one lane is the caller's stream
  static constexpr int BIG_LANES = 8;
  int big_lanes = 1;
  std::vector<int> big_lane;
  cudaStream_t big_s[BIG_LANES] = {};
  cudaEvent_t big_ev[BIG_LANES + 1] = {};
  // launch shapes chosen by kg_batch_tune (they do not change the output)
  unsigned tree_threads = 256;
  unsigned tiles_per_cta = 1;
  unsigned leaf_grid_cap = 0x7fffffffu;  // leaf blocks: ceil(tiles / tiles_per_cta)
  void* mem = nullptr;  // the plan's device memory (kg_batch_create), one allocation
};

constexpr uint64_t BIG_PAIRS = uint64_t(1) << 19;

static uint64_t piece(uint64_t b) { return (b + 255) & ~uint64_t(255); }

// Carves the plan's device arrays out of ws in one fixed order (a measuring
// workspace gives the bytes, a fixed arena the memory).
static bool plan_carve(BatchPlan& bp, Workspace& ws) {
  const uint64_t count = bp.count, chunks = bp.chunks, tiles = bp.tiles;
  const uint64_t pairs = bp.pairs, verts = bp.verts;
  bp.inst = ws.alloc<BInst>(count);
  bp.chunk_cnt = ws.alloc<uint64_t>(chunks);
  bp.tile_tmp = ws.alloc<uint64_t>(tiles);
  bp.tile_cnt = ws.alloc<uint64_t>(tiles);
  bp.tile_off = ws.alloc<uint64_t>(tiles + 1);
  bp.lvl_base = ws.alloc<uint64_t>(bp.level_nodes.size() * (count + 1));
  bp.desc = ws.alloc<TileDesc<BatchCtx>>(tiles);
  bp.big = ws.alloc<unsigned long long>(tiles);
  bp.nbig = ws.alloc<unsigned long long>(2);  // over k_max; left by the sparse kernel
  bp.pairs_buf = ws.alloc<uint32_t>(2 * pairs);
  bp.deg = ws.alloc<unsigned long long>(verts);
  bp.rowptr = ws.alloc<uint64_t>(verts + 1);
  bp.rowpos = ws.alloc<unsigned long long>(verts);
  bp.cursor = ws.alloc<unsigned long long>(verts);
  bp.long_rows = ws.alloc<unsigned long long>(verts);
  bp.nlong = ws.alloc<unsigned long long>(1);
  if (!scan_scratch(tiles, ws, bp.scan_t) || !scan_scratch(verts, ws, bp.scan_v)) return false;
  // scratch of the per-instance assembly (deg, rowptr, cursor, long rows,
  // count, scan) of the big undirected instances
  // (the largest need over them, measured on assemble()'s own carve; the
  // instances are assembled one after the other in stream order)
  uint64_t need = 0;
  for (const auto& g : bp.bigs)
    need = std::max<uint64_t>(need, assemble_scratch_bytes(g.n, 2 * g.m));
  bp.big_arena_bytes = 0;
  bp.big_arena = nullptr;
  if (need) {
    bp.big_arena_bytes = piece(need);
    bp.big_arena = ws.alloc<unsigned char>(bp.big_arena_bytes * uint64_t(bp.big_lanes));
  }
  return ws.ok();
}

// Host-side layout of a batch: validates the instances, fills their table
// (bases of chunks, tiles, samples, pairs, vertices and output entries, in
// instance order) and the plan's sizes.  No device memory is touched.
int batch_layout(const BatchSpec* specs, uint32_t count, std::vector<BInst>& tab, BatchPlan& bp) {
  tab.assign(count, BInst{});
  bp.count = count;
  bp.out_offsets.assign(count + 1, 0);
  bp.bigs.clear();
  bp.level_nodes.clear();
  uint64_t chunks = 0, tiles = 0, samples = 0, spairs = 0, bpairs = 0, verts = 0, entries = 0;
  for (uint32_t i = 0; i < count; ++i) {
    const BatchSpec& q = specs[i];
    BInst& I = tab[i];
    I.n = q.n;
    I.m = q.m;
    I.seed = q.seed;
    I.P = q.chunks;
    I.undirected = q.undirected ? 1 : 0;
    I.binom = q.binom ? 1 : 0;
    I.p = q.p;
    const uint32_t Pmax = I.undirected ? 32u : 64u;
    if (q.n == 0 || q.chunks == 0 || q.chunks > q.n || q.chunks > Pmax || q.n > (uint64_t(1) << 32))
      return ST_ARG;
    const u128 Ntot = I.undirected ? tri_pairs(q.n) : u128(q.n) * (q.n - 1);
    if (u128(q.m) > Ntot) return ST_ARG;
    if (q.m > M_MAX) return ST_RANGE;
    const u128 rmax = (u128(q.n) + q.chunks - 1) / q.chunks;
    const u128 Unom = I.undirected ? rmax * rmax : rmax * (q.n - 1);
    if (I.binom) {
      // as kg_gnp_binomial: chunk universes within the binomial's exact range,
      // the tile depth from the expected count p U_nom of the nominal chunk
      if (!(q.p >= 0.0 && q.p <= 1.0)) return ST_ARG;
      if (Unom > u128(BINOM_N_MAX)) return ST_RANGE;
      if (tile_depth_e(q.p * dbl(Unom), Unom, K_LEAF, I.d)) return ST_RANGE;
    } else if (tile_depth(q.m, Unom, Ntot, K_LEAF, I.d)) {
      return ST_RANGE;
    }
    I.D = 0;
    while ((uint64_t(1) << I.D) < q.chunks) ++I.D;
    I.C = I.undirected ? uint64_t(q.chunks) * (q.chunks + 1) / 2 : q.chunks;
    I.rb = RowBounds::make(q.n, q.chunks);
    I.div = make_div(q.n > 1 ? q.n - 1 : 1);
    I.chunk_base = chunks;
    I.tile_base = tiles;
    I.sample_base = samples;
    I.big = (I.undirected && q.m >= BIG_PAIRS) ? 1u : 0u;
    I.spair_base = spairs;
    I.pair_base = I.big ? bpairs : spairs;  // a big one's is moved past the small pairs below
    I.vert_base = verts;
    I.out_base = entries;
    I.pad_ = 0;
    I.pad2_ = 0;
    if (I.big) bp.bigs.push_back({q.n, q.m, bpairs, entries});
    bp.out_offsets[i] = entries;
    chunks += I.C;
    tiles += I.C << I.d;
    samples += q.m;
    if (bp.level_nodes.size() < size_t(I.d)) bp.level_nodes.resize(size_t(I.d), 0);
    for (int L = 0; L < I.d; ++L) bp.level_nodes[L] += I.C << L;
    if (I.big) {
      bpairs += q.m;
      entries += 2 * q.m;
    } else if (I.undirected) {
      spairs += q.m;
      verts += q.n;
      entries += 2 * q.m;
    } else {
      entries += q.m;
    }
  }
  for (BInst& I : tab)
    if (I.big) I.pair_base += spairs;
  for (auto& g : bp.bigs) g.pair_base += spairs;
  // lanes of the big instances: largest first onto the least loaded lane
  bp.big_lanes = int(std::min<size_t>(bp.bigs.size(), BatchPlan::BIG_LANES));
  if (bp.big_lanes < 1) bp.big_lanes = 1;
  bp.big_lane.assign(bp.bigs.size(), 0);
  {
    std::vector<size_t> order(bp.bigs.size());
    for (size_t k = 0; k < order.size(); ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(),
                     [&](size_t a, size_t b) { return bp.bigs[a].m > bp.bigs[b].m; });
    // lane 0 (the caller's stream) also assembles the small instances first
    std::vector<uint64_t> load(size_t(bp.big_lanes), 0);
    load[0] = spairs;
    for (size_t k : order) {
      const int l = int(std::min_element(load.begin(), load.end()) - load.begin());
      bp.big_lane[k] = l;
      load[size_t(l)] += bp.bigs[k].m;
    }
  }
  bp.out_offsets[count] = entries;
  bp.chunks = chunks;
  bp.tiles = tiles;
  bp.samples = samples;
  bp.pairs = spairs + bpairs;
  bp.spairs = spairs;
  bp.verts = verts;
  bp.entries = entries;
  bp.has_und = spairs > 0;
  return ST_OK;
}

size_t batch_plan_bytes(BatchPlan& bp) {
  Workspace meas = Workspace::measuring();
  BatchPlan copy = bp;
  if (!plan_carve(copy, meas)) return ~size_t(0);
  return meas.used();
}

static int batch_assemble_small(BatchPlan* bp, uint32_t* out, uint64_t cap, cudaStream_t s,
                                int* err);

static int batch_run_impl(BatchPlan* bp, uint32_t* out, uint64_t cap, cudaStream_t s) {
  int* err = device_error_word();
  if (!err) return ST_CUDA;
  const uint32_t count = bp->count;
  {
    ProfScope ps(PROF_CHUNK_TREE, s);
    batch_trees<<<count, bp->tree_threads, 0, s>>>(bp->inst, bp->chunk_cnt, bp->tile_cnt, err);
    if (launch_ok()) return ST_CUDA;
  }
  if (!bp->level_nodes.empty()) {
    ProfScope ps(PROF_TILE_TREE, s);
    batch_level_bases<<<unsigned(bp->level_nodes.size()), 1024, 0, s>>>(bp->inst, count,
                                                                         bp->lvl_base);
    if (launch_ok()) return ST_CUDA;
    for (size_t L = 0; L < bp->level_nodes.size(); ++L) {
      batch_tile_level<<<grid_for(bp->level_nodes[L], 256, sm_count() * 8), 256, 0, s>>>(
          bp->inst, count, int(L), bp->lvl_base + L * (uint64_t(count) + 1), bp->chunk_cnt,
          bp->tile_tmp, bp->tile_cnt, err);
      if (launch_ok()) return ST_CUDA;
    }
  }
  int st = scan_exclusive_u64(bp->tile_cnt, bp->tile_off, bp->tiles, bp->scan_t, s);
  if (st) return st;
  if (cudaMemsetAsync(bp->nbig, 0, 16, s) != cudaSuccess) return ST_CUDA;
  {
    ProfScope ps(PROF_OTHER, s);
    batch_desc<<<grid_for(bp->tiles, 256, sm_count() * 32), 256, 0, s>>>(
        bp->inst, count, bp->tiles, K_MAX, bp->tile_cnt, bp->tile_off, bp->desc, bp->big,
        bp->nbig, err, true);
    if (launch_ok()) return ST_CUDA;
  }
  BatchSink sink{out, bp->pairs_buf, cap, bp->pairs, err};
  const uint64_t gcap = bp->tiles < bp->leaf_grid_cap ? bp->tiles : bp->leaf_grid_cap;
  if (bp->tiles) {
    // directed and rectangle tiles without a repeated draw: the sparse kernel,
    // one block per tile; the rest (triangles, dense tiles, repeated draws)
    // from its fallback list by the general kernel
    {
      ProfScope ps(PROF_LEAF, s);
      const unsigned grid = unsigned(bp->tiles < 0x7fffffffull ? bp->tiles : 0x7fffffffull);
      leaf_sparse_kernel<BatchGeom, BatchSink, false><<<grid, SP_THREADS, 0, s>>>(
          SparseMap{}, sink, bp->desc, bp->tiles, err,
          DigestOut{nullptr, nullptr, nullptr}, bp->big, bp->nbig + 1);
      if (launch_ok()) return ST_CUDA;
    }
    ProfScope ps(PROF_LEAF, s);
    const uint64_t lg = gcap < uint64_t(sm_count()) * 8 ? gcap : uint64_t(sm_count()) * 8;
    leaf_fast_kernel<BatchGeom, BatchSink, false, true><<<unsigned(lg ? lg : 1), FAST_THREADS, 0, s>>>(
        BatchGeom{}, sink, 0, RoundKeys{}, bp->desc, bp->tiles, err,
        DigestOut{nullptr, nullptr, nullptr}, bp->big, bp->nbig + 1);
    if (launch_ok()) return ST_CUDA;
  }
  {
    ProfScope ps(PROF_OTHER, s);
    leaf_resplit_kernel<BatchGeom, BatchSink, false, TileDesc<BatchCtx>><<<sm_count(), LEAF_THREADS, 0, s>>>(
        BatchGeom{}, sink, K_MAX, bp->desc, err, DigestOut{nullptr, nullptr, nullptr}, bp->big,
        bp->nbig);
    if (launch_ok()) return ST_CUDA;
  }
  if (bp->bigs.empty()) return bp->has_und ? batch_assemble_small(bp, out, cap, s, err) : ST_OK;
  // the big undirected instances, each by the per-instance assembly, on
  // big_lanes streams (lane 0 is s, which first assembles the small
  // instances, concurrently with the other lanes' big ones); a lane's scratch
  // area is reused in its stream order
  const int nl = bp->big_lanes;
  cudaStream_t lane_s[BatchPlan::BIG_LANES];
  lane_s[0] = s;
  for (int l = 1; l < nl; ++l) lane_s[l] = bp->big_s[l];
  bool forked = false;
  if (nl > 1) {
    if (cudaEventRecord(bp->big_ev[0], s) != cudaSuccess) return ST_CUDA;
    for (int l = 1; l < nl; ++l)
      if (cudaStreamWaitEvent(lane_s[l], bp->big_ev[0], 0) != cudaSuccess) return ST_CUDA;
    forked = true;
  }
  if (bp->has_und) st = batch_assemble_small(bp, out, cap, s, err);
  for (size_t k = 0; k < bp->bigs.size() && st == ST_OK; ++k) {
    const auto& g = bp->bigs[k];
    const int l = bp->big_lane[k];
    Workspace wb(lane_s[l], static_cast<unsigned char*>(bp->big_arena) + uint64_t(l) * bp->big_arena_bytes,
                 bp->big_arena_bytes);
    st = assemble<uint32_t>(bp->pairs_buf + 2 * g.pair_base, nullptr, g.m, g.n,
                            out + 2 * g.out_base, 2 * g.m, wb, lane_s[l], err);
  }
  // every forked lane joins back, also after an error (a capture must end joined)
  if (forked)
    for (int l = 1; l < nl; ++l)
      if (cudaEventRecord(bp->big_ev[l], lane_s[l]) != cudaSuccess ||
          cudaStreamWaitEvent(s, bp->big_ev[l], 0) != cudaSuccess)
        st = ST_CUDA;
  return st;
}

// Streams and events of the big instances' lanes (lanes 1 .. big_lanes - 1).
static bool big_lanes_create(BatchPlan& bp) {
  for (int l = 1; l < bp.big_lanes; ++l)
    if (cudaStreamCreateWithFlags(&bp.big_s[l], cudaStreamNonBlocking) != cudaSuccess) return false;
  for (int l = 0; l < bp.big_lanes; ++l)
    if (cudaEventCreateWithFlags(&bp.big_ev[l], cudaEventDisableTiming) != cudaSuccess) return false;
  return true;
}

static void big_lanes_destroy(BatchPlan& bp) {
  for (int l = 0; l < BatchPlan::BIG_LANES; ++l) {
    if (bp.big_s[l]) cudaStreamDestroy(bp.big_s[l]);
    if (bp.big_ev[l]) cudaEventDestroy(bp.big_ev[l]);
    bp.big_s[l] = nullptr;
    bp.big_ev[l] = nullptr;
  }
}

// Undirected assembly of the small instances: one pass over all of them (their
// pairs are the first spairs of the pair buffer, their vertex ranges concatenated).
static int batch_assemble_small(BatchPlan* bp, uint32_t* out, uint64_t cap, cudaStream_t s,
                                int* err) {
  const uint32_t count = bp->count;
  const uint64_t V = bp->verts, Mp = bp->spairs;
  int st = ST_OK;
  if (cudaMemsetAsync(bp->deg, 0, V * 8, s) != cudaSuccess ||
      cudaMemsetAsync(bp->nlong, 0, 8, s) != cudaSuccess)
    return ST_CUDA;
  {
    ProfScope ps(PROF_ASSEMBLY, s);
    batch_und_degree<<<grid_for(Mp, 256, sm_count() * 32), 256, 0, s>>>(bp->inst, count, Mp,
                                                                 bp->pairs_buf, bp->deg);
    if (launch_ok()) return ST_CUDA;
  }
  st = scan_exclusive_u64(reinterpret_cast<const uint64_t*>(bp->deg), bp->rowptr, V, bp->scan_v, s);
  if (st) return st;
  {
    ProfScope ps(PROF_ASSEMBLY, s);
    batch_und_rowpos<<<grid_for(V, 256, sm_count() * 32), 256, 0, s>>>(bp->inst, count, V, bp->rowptr,
                                                                bp->rowpos);
    if (launch_ok()) return ST_CUDA;
  }
  if (cudaMemcpyAsync(bp->cursor, bp->rowpos, V * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return ST_CUDA;
  {
    ProfScope ps(PROF_ASSEMBLY, s);
    batch_und_scatter<<<grid_for(Mp, 256, sm_count() * 32), 256, 0, s>>>(bp->inst, count, Mp,
                                                                  bp->pairs_buf, bp->cursor, out,
                                                                  cap, err);
    if (launch_ok()) return ST_CUDA;
  }
  {
    ProfScope ps(PROF_ASSEMBLY, s);
    batch_und_sort_short<<<grid_for(V, 256, sm_count() * 32), 256, 0, s>>>(V, bp->rowpos, bp->deg, out, cap,
                                                                  bp->long_rows, bp->nlong);
    if (launch_ok()) return ST_CUDA;
  }
  {
    ProfScope ps(PROF_ASSEMBLY, s);
    batch_und_sort_long<<<sm_count() * 2, 256, 0, s>>>(bp->rowpos, bp->deg, out, bp->long_rows,
                                                bp->nlong);
    if (launch_ok()) return ST_CUDA;
  }
  return st;
}

struct BatchGroup {
  BatchPlan plan;
  std::vector<BInst> tab;
  unsigned long long* dig = nullptr;
};

int batch_group_prepare(const BatchSpec* specs, uint32_t count, BatchGroup** out,
                        size_t* dev_bytes, size_t* table_bytes) {
  BatchGroup* g = new BatchGroup();
  int st = batch_layout(specs, count, g->tab, g->plan);
  if (st) {
    delete g;
    return st;
  }
  if (cudaGetDevice(&g->plan.device) != cudaSuccess || !big_lanes_create(g->plan)) {
    big_lanes_destroy(g->plan);
    delete g;
    return ST_CUDA;
  }
  *dev_bytes = batch_plan_bytes(g->plan) + piece(uint64_t(count ? count : 1) * 8);
  *table_bytes = sizeof(BInst) * count;
  *out = g;
  return ST_OK;
}

int batch_group_launch(BatchGroup* g, void* dev_mem, size_t dev_bytes, void* h_table,
                       uint32_t* out, uint64_t cap, cudaStream_t s) {
  BatchPlan& bp = g->plan;
  Workspace ws(s, dev_mem, dev_bytes);
  if (!plan_carve(bp, ws)) return ST_INTERNAL;
  g->dig = ws.alloc<unsigned long long>(bp.count);
  if (!ws.ok()) return ST_INTERNAL;
  if (bp.count == 0) return ST_OK;
  memcpy(h_table, g->tab.data(), sizeof(BInst) * bp.count);
  if (cudaMemcpyAsync(bp.inst, h_table, sizeof(BInst) * bp.count, cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaMemsetAsync(g->dig, 0, sizeof(unsigned long long) * bp.count, s) != cudaSuccess)
    return ST_CUDA;
  if (bp.entries == 0) return ST_OK;
  int st = batch_run_impl(&bp, out, cap, s);
  if (st) return st;
  ProfScope ps(PROF_DIGEST, s);
  batch_digests<<<grid_for(bp.entries, 256, sm_count() * 16), 256, 0, s>>>(bp.inst, bp.count,
                                                                           bp.entries, out, g->dig);
  return launch_ok();
}

uint64_t batch_group_offset(const BatchGroup* g, uint32_t i) { return g->plan.out_offsets[i]; }

const uint64_t* batch_group_digests(const BatchGroup* g) {
  return reinterpret_cast<const uint64_t*>(g->dig);
}

void batch_group_free(BatchGroup* g) {
  if (!g) return;
  big_lanes_destroy(g->plan);
  delete g;
}

}  // namespace kg

using namespace kg;

struct kg_batch {
  BatchPlan plan;
};

extern "C" {

kg_status kg_batch_create(const kg_instance* h_inst, uint32_t count, int id_bytes,
                          kg_batch** out_batch) {
  if (!out_batch || (count && !h_inst) || id_bytes != 4) return KG_ERR_ARG;
  *out_batch = nullptr;
  std::vector<BatchSpec> specs(count);
  for (uint32_t i = 0; i < count; ++i) {
    const kg_instance& q = h_inst[i];
    specs[i] = BatchSpec{q.n, q.m, q.seed, 0.0, q.chunks, q.undirected ? 1 : 0, 0};
  }
  kg_batch* b = new kg_batch();
  BatchPlan& bp = b->plan;
  std::vector<BInst> tab;
  int st = batch_layout(specs.data(), count, tab, bp);
  if (st) {
    delete b;
    return kg_status(st);
  }
  if (cudaGetDevice(&bp.device) != cudaSuccess || !big_lanes_create(bp)) {
    big_lanes_destroy(bp);
    delete b;
    return KG_ERR_CUDA;
  }
  // the plan's device memory: one allocation, carved as the measuring pass counted
  const size_t bytes = batch_plan_bytes(bp);
  if (cudaMalloc(&bp.mem, bytes ? bytes : 256) != cudaSuccess) {
    big_lanes_destroy(bp);
    delete b;
    return KG_ERR_CUDA;
  }
  Workspace ws(nullptr, bp.mem, bytes ? bytes : 256);
  if (!plan_carve(bp, ws) ||
      cudaMemcpy(bp.inst, tab.data(), sizeof(BInst) * count, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(bp.mem);
    big_lanes_destroy(bp);
    delete b;
    return KG_ERR_CUDA;
  }
  *out_batch = b;
  return KG_OK;
}

kg_status kg_batch_destroy(kg_batch* b) {
  if (!b) return KG_OK;
  if (b->plan.mem) cudaFree(b->plan.mem);
  big_lanes_destroy(b->plan);
  delete b;
  return KG_OK;
}

uint64_t kg_batch_entries(const kg_batch* b) { return b ? b->plan.entries : 0; }

kg_status kg_batch_offsets(const kg_batch* b, uint64_t* h_offsets) {
  if (!b || !h_offsets) return KG_ERR_ARG;
  std::copy(b->plan.out_offsets.begin(), b->plan.out_offsets.end(), h_offsets);
  return KG_OK;
}

kg_status kg_batch_run(kg_batch* b, void* d_out, uint64_t cap_entries, void* stream) {
  if (!b) return KG_ERR_ARG;
  if (cap_entries < b->plan.entries) return KG_ERR_CAPACITY;
  if (b->plan.count == 0 || b->plan.entries == 0) return KG_OK;
  if (!d_out) return KG_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != b->plan.device) return KG_ERR_ARG;
  return kg_status(batch_run_impl(&b->plan, static_cast<uint32_t*>(d_out), cap_entries,
                                  static_cast<cudaStream_t>(stream)));
}

// Autotuning over launch shapes that do not change the output: threads per
// block of the per-instance tree kernel, and tiles per CTA of the leaf kernel
// (the leaf grid is ceil(tiles / tiles_per_cta) blocks striding over the
// tiles; 1 = one block per tile).  Choices are cached for the process, keyed
// by the GPU's name and the batch's size class (log2 of its instances and of
// its tiles): a batch of a class already tuned on this GPU takes the cached
// choice without timing anything.
namespace {
struct TuneKey {
  std::string gpu;
  int lg_count, lg_tiles;
  bool operator<(const TuneKey& o) const {
    return std::tie(gpu, lg_count, lg_tiles) < std::tie(o.gpu, o.lg_count, o.lg_tiles);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<unsigned, unsigned>> g_tune_cache;  // -> (tree threads, tiles per CTA)

int lg_ceil(uint64_t x) {
  int l = 0;
  while ((uint64_t(1) << l) < x && l < 63) ++l;
  return l;
}
}  // namespace

static unsigned grid_cap_for(uint64_t tiles, unsigned per_cta) {
  const uint64_t g = (tiles + per_cta - 1) / per_cta;
  return unsigned(g < 1 ? 1 : (g > 0x7fffffffull ? 0x7fffffffull : g));
}

kg_status kg_batch_tune(kg_batch* b, void* d_out, uint64_t cap_entries, int reps, void* stream) {
  if (!b || reps < 1) return KG_ERR_ARG;
  if (cap_entries < b->plan.entries) return KG_ERR_CAPACITY;
  if (b->plan.count == 0 || b->plan.entries == 0) return KG_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaDeviceProp prop;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
    return KG_ERR_CUDA;
  const TuneKey key{prop.name, lg_ceil(b->plan.count), lg_ceil(b->plan.tiles)};
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      b->plan.tree_threads = it->second.first;
      b->plan.tiles_per_cta = it->second.second;
      b->plan.leaf_grid_cap = grid_cap_for(b->plan.tiles, it->second.second);
      return KG_OK;
    }
  }
  const unsigned trees[] = {64, 128, 256};
  const unsigned per_cta[] = {1, 2, 4, 8, 16};
  float best = 1e30f;
  unsigned bt = 256, bp = 1;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return KG_ERR_CUDA;
  kg_status st = KG_OK;
  for (unsigned tt : trees)
    for (unsigned pc : per_cta) {
      b->plan.tree_threads = tt;
      b->plan.tiles_per_cta = pc;
      b->plan.leaf_grid_cap = grid_cap_for(b->plan.tiles, pc);
      float total = 0.f;
      for (int r = 0; r < reps && st == KG_OK; ++r) {
        cudaEventRecord(e0, s);
        st = kg_status(batch_run_impl(&b->plan, static_cast<uint32_t*>(d_out), cap_entries, s));
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) st = KG_ERR_CUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        total += ms;
      }
      if (st == KG_OK && total < best) {
        best = total;
        bt = tt;
        bp = pc;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->plan.tree_threads = bt;
  b->plan.tiles_per_cta = bp;
  b->plan.leaf_grid_cap = grid_cap_for(b->plan.tiles, bp);
  if (st == KG_OK) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = std::make_pair(bt, bp);
  }
  return st;
}

kg_status kg_batch_get_tuning(const kg_batch* b, uint32_t* tree_threads, uint32_t* tiles_per_cta) {
  if (!b) return KG_ERR_ARG;
  if (tree_threads) *tree_threads = b->plan.tree_threads;
  if (tiles_per_cta) *tiles_per_cta = b->plan.tiles_per_cta;
  return KG_OK;
}

}  // extern "C"
