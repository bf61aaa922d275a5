// C ABI: undirected G(n,m) (Sec. 4.2) and G(n,p) (Sec. 4.3), directed and
// undirected, with the assembly of undirected output in both directions.
#include <algorithm>
#include <vector>

#include "kg.h"
#include "kg_batch.h"
#include "kg_gnp.cuh"
#include "kg_run.cuh"
#include "kg_und.cuh"
#include "kg_assemble.cuh"

namespace kg {

static cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

// ---------------------------------------------------------------- undirected G(n,m)
struct UndParams {
  uint64_t n, m;
  uint32_t P;
  u128 Ntot, Unom;
  int d, D;
};

// windowed: the caller assembles only a window of rows (kg_gnm_undirected_rows),
// so n is limited by the chunk sizes instead of by whole-graph row arrays.
static int check_undirected(uint64_t n, uint64_t m, uint32_t P, uint32_t k_leaf, uint32_t k_max,
                            int id_bytes, UndParams& up, bool windowed = false) {
  if (n == 0 || P == 0 || uint64_t(P) > n) return ST_ARG;
  if (id_bytes != 4 && id_bytes != 8) return ST_ARG;
  if (k_leaf < 2 || k_max < k_leaf || k_max > uint32_t(K_MAX)) return ST_ARG;
  up.n = n;
  up.m = m;
  up.P = P;
  up.Ntot = tri_pairs(n);
  if (u128(m) > up.Ntot) return ST_ARG;
  if (m > M_MAX || P > 65536u) return ST_RANGE;
  if (windowed ? (n > (uint64_t(1) << 40)) : (n > (uint64_t(1) << 31))) return ST_RANGE;
  if (id_bytes == 4 && n > (uint64_t(1) << 32)) return ST_RANGE;
  const u128 rmax = (u128(n) + P - 1) / P;
  if (rmax >> 32) return ST_RANGE;
  up.Unom = rmax * rmax;
  int st = tile_depth(m, up.Unom, up.Ntot, k_leaf, up.d);
  if (st) return st;
  up.D = 0;
  while ((uint64_t(1) << up.D) < P) ++up.D;
  return ST_OK;
}

// Levels with at least this many nodes (bound) take the 64-register quad_level.
constexpr uint64_t QUAD_WIDE_NODES = uint64_t(1) << 18;

// Quadrant recursion: levels 0..D, node lists ping-pong, leaf counts per chunk.
static int run_quadtree(const UndParams& up, uint64_t seed, uint64_t* chunk_cnt, Workspace& ws,
                        cudaStream_t s, int* err) {
  const uint64_t C = uint64_t(up.P) * (up.P + 1) / 2;
  QNode* L0 = ws.alloc<QNode>(C);
  QNode* L1 = ws.alloc<QNode>(C);
  uint32_t* counts = ws.alloc<uint32_t>(up.D + 2);
  if (!ws.ok()) return ST_CUDA;
  const RowBounds rb = RowBounds::make(up.n, up.P);
  {
    ProfScope ps(PROF_CHUNK_TREE, s);
    quad_init<<<1, 32, 0, s>>>(L0, counts, up.D + 1, up.P, up.m);
    if (launch_ok()) return ST_CUDA;
  }
  for (int l = 0; l <= up.D; ++l) {
    const uint64_t bound = (l < 16) ? ((uint64_t(1) << l) * ((uint64_t(1) << l) + 1) / 2) : C;
    ProfScope ps(PROF_CHUNK_TREE, s);
    // one-warp blocks spread the few FP64-bound nodes of the top levels over the SMs
    const uint64_t nodes = bound < C ? bound : C;
    if (nodes >= QUAD_WIDE_NODES)
      quad_level<4><<<grid_for(nodes, 32, sm_count() * 64), 32, 0, s>>>(
          rb, seed, (l & 1) ? L1 : L0, counts + l, (l & 1) ? L0 : L1, counts + l + 1, chunk_cnt, err);
    else
      quad_level<1><<<grid_for(nodes, 32, sm_count() * 64), 32, 0, s>>>(
          rb, seed, (l & 1) ? L1 : L0, counts + l, (l & 1) ? L0 : L1, counts + l + 1, chunk_cnt, err);
    if (launch_ok()) return ST_CUDA;
  }
  return ST_OK;
}

template <class Id>
static int gnm_undirected_impl(const UndParams& up, uint64_t seed, uint32_t k_max, void* d_out,
                               uint64_t cap, cudaStream_t s, int* err) {
  Workspace ws(s);
  const uint64_t C = uint64_t(up.P) * (up.P + 1) / 2;
  uint64_t* chunk_cnt = ws.alloc<uint64_t>(C);
  Id* pairs = ws.alloc<Id>(2 * up.m);
  if (!ws.ok()) return ST_CUDA;
  int st = run_quadtree(up, seed, chunk_cnt, ws, s, err);
  if (st) return st;
  UndGeom g{up.n, up.P, RowBounds::make(up.n, up.P)};
  st = run_chunks(g, 0, C, chunk_cnt, up.d, k_max, seed, int(sizeof(Id)), pairs, up.m, ws, s, err);
  if (st) return st;
  return assemble<Id>(pairs, nullptr, up.m, up.n, static_cast<Id*>(d_out), cap, ws, s, err);
}

// ---------------------------------------------------------------- undirected rows by blocks
// The chunks (i, j <= i) a range of row blocks needs (Sec. 4.2: a PE
// regenerates the chunks of its row and of its column), given as a device
// list of chunk indices k = i(i+1)/2 + j (the row blocks' chunks, then the
// column blocks' chunks outside them).
struct UndListGeom {
  UndGeom base;
  const uint64_t* list;
  using Ctx = UndGeom::Ctx;
  __device__ __forceinline__ uint64_t chunk_id(uint64_t c) const { return base.chunk_id(list[c]); }
  __device__ __forceinline__ uint64_t rows(uint64_t c) const { return base.rows(list[c]); }
  __device__ __forceinline__ uint64_t universe(uint64_t c) const { return base.universe(list[c]); }
  __device__ __forceinline__ Ctx ctx(uint64_t c) const { return base.ctx(list[c]); }
  __device__ __forceinline__ void map(const Ctx& x, uint64_t off, uint64_t& u, uint64_t& v) const {
    base.map(x, off, u, v);
  }
  __device__ __forceinline__ void row_span(const Ctx& x, uint64_t off, uint64_t u, uint64_t v,
                                           uint64_t& start, uint64_t& len) const {
    base.row_span(x, off, u, v, start, len);
  }
};

__global__ void gather_counts(const uint64_t* __restrict__ src, const uint64_t* __restrict__ idx,
                              uint64_t n, uint64_t* __restrict__ dst) {
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += uint64_t(gridDim.x) * blockDim.x)
    dst[i] = src[idx[i]];
}

// the pairs actually in the buffer: min(total, cap)
__global__ void clamp_count(const uint64_t* total, uint64_t cap, uint64_t* out) {
  *out = *total < cap ? *total : cap;
}

template <class Id>
static int gnm_undirected_rows_impl(const UndParams& up, uint64_t seed, uint32_t b0, uint32_t b1,
                                    const uint64_t* d_counts, void* d_out, uint64_t cap,
                                    uint64_t* d_entries, uint64_t* d_digest, uint64_t* d_hist,
                                    cudaStream_t s, int* err) {
  Workspace ws(s);
  const uint32_t P = up.P;
  const uint64_t C = uint64_t(P) * (P + 1) / 2;
  int st;
  if (!d_counts) {
    uint64_t* c2 = ws.alloc<uint64_t>(C);
    if (!ws.ok()) return ST_CUDA;
    if ((st = run_quadtree(up, seed, c2, ws, s, err))) return st;
    d_counts = c2;
  }
  // chunks (i, j <= i) of the row blocks, then (i > j, j) of the column blocks
  // whose row block lies outside the range (those inside are already listed)
  std::vector<uint64_t> list;
  for (uint64_t i = b0; i < b1; ++i)
    for (uint64_t j = 0; j <= i; ++j) list.push_back(i * (i + 1) / 2 + j);
  for (uint64_t j = b0; j < b1; ++j)
    for (uint64_t i = std::max<uint64_t>(j + 1, b1); i < P; ++i)
      list.push_back(i * (i + 1) / 2 + j);
  const uint64_t L = list.size();
  uint64_t* dlist = ws.alloc<uint64_t>(L);
  uint64_t* cnt = ws.alloc<uint64_t>(L);
  uint64_t* off = ws.alloc<uint64_t>(L + 1);
  uint64_t* npairs = ws.alloc<uint64_t>(1);
  Id* pairs = ws.alloc<Id>(2 * (cap ? cap : 1));  // every pair gives an entry of the window
  if (!ws.ok()) return ST_CUDA;
  if (cudaMemcpyAsync(dlist, list.data(), L * 8, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return ST_CUDA;
  {
    ProfScope ps(PROF_OTHER, s);
    gather_counts<<<grid_for(L, 256, sm_count() * 8), 256, 0, s>>>(d_counts, dlist, L, cnt);
    if (launch_ok()) return ST_CUDA;
  }
  if ((st = scan_exclusive_u64(cnt, off, L, ws, s))) return st;
  const RowBounds rb = RowBounds::make(up.n, P);
  UndListGeom g{UndGeom{up.n, P, rb}, dlist};
  if ((st = run_chunks(g, 0, L, cnt, up.d, K_MAX, seed, int(sizeof(Id)), pairs, cap, ws, s, err)))
    return st;
  {
    ProfScope ps(PROF_OTHER, s);
    clamp_count<<<1, 1, 0, s>>>(off + L, cap, npairs);
    if (launch_ok()) return ST_CUDA;
  }
  const uint64_t row_lo = rb(b0), nrows = rb(b1) - row_lo;
  uint64_t* rowptr = nullptr;
  Id* out = static_cast<Id*>(d_out);
  if (d_digest || d_hist) {
    const uint64_t nb = b1 - b0;
    if ((d_digest && cudaMemsetAsync(d_digest, 0, nb * 8, s) != cudaSuccess) ||
        (d_hist && cudaMemsetAsync(d_hist, 0, nb * 65 * 8, s) != cudaSuccess))
      return ST_CUDA;
  }
  const AsmDigest dig{rb, b0, reinterpret_cast<unsigned long long*>(d_digest),
                      reinterpret_cast<unsigned long long*>(d_hist)};
  bool digested = false;
  if ((st = assemble<Id>(pairs, npairs, 0, up.n, out, cap, ws, s, err, row_lo, nrows, &rowptr,
                         cap, (d_digest || d_hist) ? &dig : nullptr, &digested)))
    return st;
  if (d_entries && cudaMemcpyAsync(d_entries, rowptr + nrows, 8, cudaMemcpyDeviceToDevice, s) !=
                       cudaSuccess)
    return ST_CUDA;
  if ((d_digest || d_hist) && !digested) {
    ProfScope ps(PROF_DIGEST, s);
    und_block_digest<Id><<<grid_for(nrows, unsigned(DIGEST_SEG), sm_count() * 16), 256, 0, s>>>(
        out, rowptr, row_lo, nrows, rb, b0, reinterpret_cast<unsigned long long*>(d_digest),
        reinterpret_cast<unsigned long long*>(d_hist));
    if (launch_ok()) return ST_CUDA;
  }
  return ST_OK;
}

// ---------------------------------------------------------------- G(n,p)
static uint64_t gnp_tile_len(double p, uint32_t k_leaf) {
  const double q = double(k_leaf) / p;
  if (!(q >= 2.0)) return 1;
  uint64_t T = 1;
  while (T < (uint64_t(1) << 62) && double(T * 2) <= q) T *= 2;
  return T;
}

__global__ void gnp_total(const uint64_t* off_end, uint64_t* d_count, uint64_t* npairs,
                          uint64_t mult, uint64_t cap, int* err) {
  const uint64_t tot = *off_end;
  *d_count = tot * mult;
  if (npairs) *npairs = (tot * mult <= cap) ? tot : cap / mult;
  if (tot * mult > cap) set_error(err, ST_CAPACITY);
}

template <class Geom, class Id, class SlotT>
static int gnp_impl(const Geom& g, uint64_t C, bool undirected, uint64_t n, const GnpPlan& pl,
                    uint64_t seed, void* d_out, uint64_t cap, uint64_t* d_count, cudaStream_t s,
                    int* err) {
  Workspace ws(s);
  const uint64_t tiles = C * pl.tiles_per_chunk;
  SlotT* slots = pl.cap_t ? ws.alloc<SlotT>(tiles * pl.cap_t) : nullptr;
  uint64_t* cnt = ws.alloc<uint64_t>(tiles);
  uint64_t* off = ws.alloc<uint64_t>(tiles + 1);
  uint64_t* npairs = ws.alloc<uint64_t>(1);
  if (!ws.ok()) return ST_CUDA;
  {
    ProfScope ps(PROF_GNP, s);
    gnp_tiles<Geom, SlotT><<<grid_for(tiles, 128, 1u << 20), 128, 0, s>>>(g, pl, seed, C, slots,
                                                                          cnt);
    if (launch_ok()) return ST_CUDA;
  }
  int st = scan_exclusive_u64(cnt, off, tiles, ws, s);
  if (st) return st;
  const uint64_t mult = undirected ? 2 : 1;
  {
    ProfScope ps(PROF_OTHER, s);
    gnp_total<<<1, 1, 0, s>>>(off + tiles, d_count, npairs, mult, cap, err);
    if (launch_ok()) return ST_CUDA;
  }
  if (!undirected) {
    PairSink<Id> sink{static_cast<Id*>(d_out), cap, err};
    ProfScope ps(PROF_LEAF, s);
    gnp_emit<Geom, SlotT, PairSink<Id>><<<grid_for(tiles, 4, sm_count() * 64), 128, 0, s>>>(
        g, pl, seed, C, slots, cnt, off, sink);
    return launch_ok();
  }
  const uint64_t pcap = cap / 2;
  Id* pairs = ws.alloc<Id>(2 * (pcap ? pcap : 1));
  if (!ws.ok()) return ST_CUDA;
  {
    // pairs beyond pcap are dropped by the sink without an error: the total
    // check above already recorded the capacity error
    PairSink<Id> sink{pairs, pcap, nullptr};
    ProfScope ps(PROF_LEAF, s);
    gnp_emit<Geom, SlotT, PairSink<Id>><<<grid_for(tiles, 4, sm_count() * 64), 128, 0, s>>>(
        g, pl, seed, C, slots, cnt, off, sink);
    if (launch_ok()) return ST_CUDA;
  }
  return assemble<Id>(pairs, npairs, 0, n, static_cast<Id*>(d_out), cap, ws, s, err);
}

// Count pass only: per-tile counts (no slots) and their sum.
template <class Geom>
static int gnp_count_impl(const Geom& g, uint64_t C, bool undirected, const GnpPlan& pl0,
                          uint64_t seed, uint64_t* d_count, cudaStream_t s, int* err) {
  Workspace ws(s);
  GnpPlan pl = pl0;
  pl.cap_t = 0;
  const uint64_t tiles = C * pl.tiles_per_chunk;
  uint64_t* cnt = ws.alloc<uint64_t>(tiles);
  uint64_t* off = ws.alloc<uint64_t>(tiles + 1);
  if (!ws.ok()) return ST_CUDA;
  {
    ProfScope ps(PROF_GNP, s);
    gnp_tiles<Geom, uint32_t><<<grid_for(tiles, 128, 1u << 20), 128, 0, s>>>(g, pl, seed, C,
                                                                             nullptr, cnt);
    if (launch_ok()) return ST_CUDA;
  }
  int st = scan_exclusive_u64(cnt, off, tiles, ws, s);
  if (st) return st;
  ProfScope ps(PROF_OTHER, s);
  gnp_total<<<1, 1, 0, s>>>(off + tiles, d_count, nullptr, undirected ? 2 : 1, ~uint64_t(0), err);
  return launch_ok();
}

template <class Geom, class Id>
static int gnp_dispatch_slots(const Geom& g, uint64_t C, bool und, uint64_t n, const GnpPlan& pl,
                              uint64_t seed, void* d_out, uint64_t cap, uint64_t* d_count,
                              cudaStream_t s, int* err) {
  if (pl.T <= (uint64_t(1) << 32))
    return gnp_impl<Geom, Id, uint32_t>(g, C, und, n, pl, seed, d_out, cap, d_count, s, err);
  return gnp_impl<Geom, Id, uint64_t>(g, C, und, n, pl, seed, d_out, cap, d_count, s, err);
}

}  // namespace kg

using namespace kg;

// ---------------------------------------------------------------- G(n,p), binomial counts
// Validation shared by kg_gnp_binomial and kg_gnp_binomial_count: chunk
// universes up to 2^53 (the binomial's exact range), the tile depth from the
// expected count p U_nom of the nominal chunk.
static int gnpb_prepare(int undirected, uint64_t n, double p, uint32_t chunks, int id_bytes,
                        uint64_t& C, int& d) {
  if (!(p >= 0.0 && p <= 1.0)) return ST_ARG;
  if (n == 0 || chunks == 0 || uint64_t(chunks) > n) return ST_ARG;
  if (id_bytes != 4 && id_bytes != 8) return ST_ARG;
  if (id_bytes == 4 && n > (uint64_t(1) << 32)) return ST_RANGE;
  const u128 rmax = (u128(n) + chunks - 1) / chunks;
  u128 Unom;
  if (undirected) {
    if (chunks > 65536u || n > (uint64_t(1) << 31)) return ST_RANGE;
    Unom = rmax * rmax;
    C = uint64_t(chunks) * (chunks + 1) / 2;
  } else {
    if (chunks > (1u << 24)) return ST_RANGE;
    Unom = rmax * (n - 1);
    C = chunks;
  }
  if (Unom > u128(BINOM_N_MAX)) return ST_RANGE;
  return tile_depth_e(p * dbl(Unom), Unom, K_LEAF, d);
}

namespace kg {
int gnpb_check(int undirected, uint64_t n, double p, uint32_t chunks, int id_bytes) {
  uint64_t C = 0;
  int d = 0;
  return gnpb_prepare(undirected, n, p, chunks, id_bytes, C, d);
}

int gnpb_size_many(const GnpbSizeReq* d_reqs, uint32_t count, uint64_t* d_sizes, cudaStream_t s) {
  int* err = device_error_word();
  if (!err) return ST_CUDA;
  if (count == 0) return ST_OK;
  ProfScope ps(PROF_CHUNK_TREE, s);
  gnpb_size_batch<<<grid_for(count, 4, sm_count() * 64), 128, 0, s>>>(d_reqs, count, d_sizes, err);
  return launch_ok();
}
}  // namespace kg

template <class Geom>
static int gnpb_counts(const Geom& g, uint64_t C, double p, uint64_t seed, uint64_t* cnt,
                       cudaStream_t s, int* err) {
  ProfScope ps(PROF_CHUNK_TREE, s);
  // one-warp blocks: a few hundred FP64 binomials spread over the SMs
  gnp_chunk_counts<Geom><<<grid_for(C, 32, sm_count() * 64), 32, 0, s>>>(g, C, p, seed, cnt, err);
  return launch_ok();
}

template <class Id>
static int gnpb_impl(int undirected, uint64_t n, double p, uint64_t seed, uint32_t P, uint64_t C,
                     int d, void* d_out, uint64_t cap, uint64_t* d_count, cudaStream_t s,
                     int* err) {
  Workspace ws(s);
  uint64_t* cnt = ws.alloc<uint64_t>(C);
  uint64_t* off = ws.alloc<uint64_t>(C + 1);
  uint64_t* npairs = ws.alloc<uint64_t>(1);
  if (!ws.ok()) return ST_CUDA;
  const uint64_t mult = undirected ? 2 : 1;
  int st;
  if (!undirected) {
    const DirGeom g = DirGeom::make(n, P);
    if ((st = gnpb_counts(g, C, p, seed, cnt, s, err))) return st;
    if ((st = scan_exclusive_u64(cnt, off, C, ws, s))) return st;
    {
      ProfScope ps(PROF_OTHER, s);
      gnp_total<<<1, 1, 0, s>>>(off + C, d_count, npairs, mult, cap, err);
      if (launch_ok()) return ST_CUDA;
    }
    return run_chunks(g, 0, C, cnt, d, K_MAX, seed, int(sizeof(Id)), d_out, cap, ws, s, err);
  }
  UndGeom g{n, P, RowBounds::make(n, P)};
  if ((st = gnpb_counts(g, C, p, seed, cnt, s, err))) return st;
  if ((st = scan_exclusive_u64(cnt, off, C, ws, s))) return st;
  {
    ProfScope ps(PROF_OTHER, s);
    gnp_total<<<1, 1, 0, s>>>(off + C, d_count, npairs, mult, cap, err);
    if (launch_ok()) return ST_CUDA;
  }
  const uint64_t pcap = cap / 2;
  Id* pairs = ws.alloc<Id>(2 * (pcap ? pcap : 1));
  if (!ws.ok()) return ST_CUDA;
  if ((st = run_chunks(g, 0, C, cnt, d, K_MAX, seed, int(sizeof(Id)), pairs, pcap, ws, s, err)))
    return st;
  return assemble<Id>(pairs, npairs, 0, n, static_cast<Id*>(d_out), cap, ws, s, err);
}

extern "C" {

kg_status kg_gnm_undirected_ex(uint64_t n, uint64_t m, uint64_t seed, uint32_t chunks,
                               uint32_t k_leaf, uint32_t k_max, int id_bytes, void* d_out,
                               uint64_t cap_edges, void* stream) {
  UndParams up;
  int st = check_undirected(n, m, chunks, k_leaf, k_max, id_bytes, up);
  if (st) return kg_status(st);
  if (cap_edges < 2 * m) return KG_ERR_CAPACITY;
  if (m == 0) return KG_OK;
  if (!d_out) return KG_ERR_ARG;
  int* err = device_error_word();
  if (!err) return KG_ERR_CUDA;
  cudaStream_t s = as_stream(stream);
  st = id_bytes == 4 ? gnm_undirected_impl<uint32_t>(up, seed, k_max, d_out, cap_edges, s, err)
                     : gnm_undirected_impl<uint64_t>(up, seed, k_max, d_out, cap_edges, s, err);
  return kg_status(st);
}

kg_status kg_gnm_undirected_chunk_counts(uint64_t n, uint64_t m, uint64_t seed, uint32_t chunks,
                                         uint64_t* d_counts, void* stream) {
  UndParams up;
  int st = check_undirected(n, m, chunks, K_LEAF, K_MAX, 8, up, true);
  if (st) return kg_status(st);
  if (!d_counts) return KG_ERR_ARG;
  int* err = device_error_word();
  if (!err) return KG_ERR_CUDA;
  cudaStream_t s = as_stream(stream);
  Workspace ws(s);
  return kg_status(run_quadtree(up, seed, d_counts, ws, s, err));
}

kg_status kg_gnm_undirected_rows(uint64_t n, uint64_t m, uint64_t seed, uint32_t chunks,
                                 uint32_t b_begin, uint32_t b_end, const uint64_t* d_counts,
                                 int id_bytes, void* d_out, uint64_t cap_edges, uint64_t* d_entries,
                                 uint64_t* d_block_digest, uint64_t* d_block_hist, void* stream) {
  UndParams up;
  int st = check_undirected(n, m, chunks, K_LEAF, K_MAX, id_bytes, up, true);
  if (st) return kg_status(st);
  if (b_begin >= b_end || b_end > chunks) return KG_ERR_ARG;
  if (!d_out && cap_edges > 0) return KG_ERR_ARG;
  int* err = device_error_word();
  if (!err) return KG_ERR_CUDA;
  cudaStream_t s = as_stream(stream);
  st = id_bytes == 4
           ? gnm_undirected_rows_impl<uint32_t>(up, seed, b_begin, b_end, d_counts, d_out,
                                                cap_edges, d_entries, d_block_digest, d_block_hist,
                                                s, err)
           : gnm_undirected_rows_impl<uint64_t>(up, seed, b_begin, b_end, d_counts, d_out,
                                                cap_edges, d_entries, d_block_digest, d_block_hist,
                                                s, err);
  return kg_status(st);
}

kg_status kg_gnm_undirected(uint64_t n, uint64_t m, uint64_t seed, uint32_t chunks, int id_bytes,
                            void* d_out, uint64_t cap_edges, void* stream) {
  return kg_gnm_undirected_ex(n, m, seed, chunks, K_LEAF, K_MAX, id_bytes, d_out, cap_edges,
                              stream);
}

// Validation and tile plan shared by kg_gnp_ex and kg_gnp_count.
// slots_per_tile >= 0 replaces the slot count of a tile (clamped to the tile
// length); negative keeps the default.
static int gnp_prepare(int undirected, uint64_t n, double p, uint32_t chunks, uint32_t k_leaf,
                       int id_bytes, GnpPlan& pl, uint64_t& C, int64_t slots_per_tile = -1) {
  if (!(p >= 0.0 && p <= 1.0) || k_leaf < 2) return ST_ARG;
  if (n == 0 || chunks == 0 || uint64_t(chunks) > n) return ST_ARG;
  if (id_bytes != 4 && id_bytes != 8) return ST_ARG;
  if (id_bytes == 4 && n > (uint64_t(1) << 32)) return ST_RANGE;
  const uint64_t rows_max = uint64_t((u128(n) + chunks - 1) / chunks);
  u128 Unom;
  if (undirected) {
    if (chunks > 65536u || n > (uint64_t(1) << 31)) return ST_RANGE;
    Unom = u128(rows_max) * rows_max;
    C = uint64_t(chunks) * (chunks + 1) / 2;
  } else {
    if (chunks > (1u << 24)) return ST_RANGE;
    Unom = u128(rows_max) * (n - 1);
    C = chunks;
  }
  if (Unom >> 64) return ST_RANGE;
  pl.p = p;
  pl.all = (p >= 1.0);
  pl.inv_lq = (pl.all || p == 0.0) ? 0.0 : 1.0 / kg_log1m(p);
  pl.T = pl.all ? (uint64_t(1) << 20) : (p == 0.0 ? (uint64_t(1) << 62) : gnp_tile_len(p, k_leaf));
  pl.tiles_per_chunk = uint64_t((Unom + pl.T - 1) / pl.T);
  if (pl.tiles_per_chunk > (uint64_t(1) << 32)) return ST_RANGE;
  const u128 tiles = u128(C) * pl.tiles_per_chunk;
  if (tiles > (u128(1) << 34)) return ST_RANGE;
  uint64_t cap_t = pl.all ? 0 : 2 * uint64_t(k_leaf) + 64;
  if (cap_t > pl.T) cap_t = pl.T;
  const uint64_t slot_bytes = (pl.T <= (uint64_t(1) << 32)) ? 4 : 8;
  // slots above this size: tiles are walked a second time instead
  if (uint64_t(tiles) * cap_t * slot_bytes > (uint64_t(12) << 30)) cap_t = 0;
  if (slots_per_tile >= 0 && !pl.all)
    cap_t = uint64_t(slots_per_tile) < pl.T ? uint64_t(slots_per_tile) : pl.T;
  pl.cap_t = uint32_t(cap_t);
  return ST_OK;
}

kg_status kg_gnp_ex_slots(int undirected, uint64_t n, double p, uint64_t seed, uint32_t chunks,
                          uint32_t k_leaf, int32_t slots_per_tile, int id_bytes, void* d_out,
                          uint64_t cap_edges, uint64_t* d_count, void* stream) {
  if (!d_count) return KG_ERR_ARG;
  if (slots_per_tile > (int32_t(1) << 20)) return KG_ERR_ARG;
  GnpPlan pl;
  uint64_t C = 0;
  int st = gnp_prepare(undirected, n, p, chunks, k_leaf, id_bytes, pl, C, slots_per_tile);
  if (st) return kg_status(st);
  cudaStream_t s = as_stream(stream);
  if (cudaMemsetAsync(d_count, 0, sizeof(uint64_t), s) != cudaSuccess) return KG_ERR_CUDA;
  if (p == 0.0 || n < 2) return KG_OK;
  if (!d_out && cap_edges > 0) return KG_ERR_ARG;
  int* err = device_error_word();
  if (!err) return KG_ERR_CUDA;
  if (undirected) {
    UndGeom g{n, chunks, RowBounds::make(n, chunks)};
    st = id_bytes == 4
             ? gnp_dispatch_slots<UndGeom, uint32_t>(g, C, true, n, pl, seed, d_out, cap_edges, d_count, s, err)
             : gnp_dispatch_slots<UndGeom, uint64_t>(g, C, true, n, pl, seed, d_out, cap_edges, d_count, s, err);
  } else {
    const DirGeom g = DirGeom::make(n, chunks);
    st = id_bytes == 4
             ? gnp_dispatch_slots<DirGeom, uint32_t>(g, C, false, n, pl, seed, d_out, cap_edges, d_count, s, err)
             : gnp_dispatch_slots<DirGeom, uint64_t>(g, C, false, n, pl, seed, d_out, cap_edges, d_count, s, err);
  }
  return kg_status(st);
}

kg_status kg_gnp_ex(int undirected, uint64_t n, double p, uint64_t seed, uint32_t chunks,
                    uint32_t k_leaf, int id_bytes, void* d_out, uint64_t cap_edges,
                    uint64_t* d_count, void* stream) {
  return kg_gnp_ex_slots(undirected, n, p, seed, chunks, k_leaf, -1, id_bytes, d_out, cap_edges,
                         d_count, stream);
}

kg_status kg_gnp_count(int undirected, uint64_t n, double p, uint64_t seed, uint32_t chunks,
                       uint32_t k_leaf, uint64_t* d_count, void* stream) {
  if (!d_count) return KG_ERR_ARG;
  GnpPlan pl;
  uint64_t C = 0;
  int st = gnp_prepare(undirected, n, p, chunks, k_leaf, 8, pl, C);
  if (st) return kg_status(st);
  cudaStream_t s = as_stream(stream);
  if (cudaMemsetAsync(d_count, 0, sizeof(uint64_t), s) != cudaSuccess) return KG_ERR_CUDA;
  if (p == 0.0 || n < 2) return KG_OK;
  int* err = device_error_word();
  if (!err) return KG_ERR_CUDA;
  if (undirected) {
    UndGeom g{n, chunks, RowBounds::make(n, chunks)};
    st = gnp_count_impl(g, C, true, pl, seed, d_count, s, err);
  } else {
    const DirGeom g = DirGeom::make(n, chunks);
    st = gnp_count_impl(g, C, false, pl, seed, d_count, s, err);
  }
  return kg_status(st);
}

kg_status kg_gnp_binomial(int undirected, uint64_t n, double p, uint64_t seed, uint32_t chunks,
                          int id_bytes, void* d_out, uint64_t cap_edges, uint64_t* d_count,
                          void* stream) {
  if (!d_count) return KG_ERR_ARG;
  uint64_t C = 0;
  int d = 0;
  int st = gnpb_prepare(undirected, n, p, chunks, id_bytes, C, d);
  if (st) return kg_status(st);
  cudaStream_t s = as_stream(stream);
  if (cudaMemsetAsync(d_count, 0, sizeof(uint64_t), s) != cudaSuccess) return KG_ERR_CUDA;
  if (p == 0.0 || n < 2) return KG_OK;
  if (!d_out && cap_edges > 0) return KG_ERR_ARG;
  int* err = device_error_word();
  if (!err) return KG_ERR_CUDA;
  st = id_bytes == 4 ? gnpb_impl<uint32_t>(undirected, n, p, seed, chunks, C, d, d_out, cap_edges,
                                           d_count, s, err)
                     : gnpb_impl<uint64_t>(undirected, n, p, seed, chunks, C, d, d_out, cap_edges,
                                           d_count, s, err);
  return kg_status(st);
}

kg_status kg_gnp_binomial_count(int undirected, uint64_t n, double p, uint64_t seed,
                                uint32_t chunks, uint64_t* d_count, void* stream) {
  if (!d_count) return KG_ERR_ARG;
  uint64_t C = 0;
  int d = 0;
  int st = gnpb_prepare(undirected, n, p, chunks, 8, C, d);
  if (st) return kg_status(st);
  cudaStream_t s = as_stream(stream);
  if (cudaMemsetAsync(d_count, 0, sizeof(uint64_t), s) != cudaSuccess) return KG_ERR_CUDA;
  if (p == 0.0 || n < 2) return KG_OK;
  int* err = device_error_word();
  if (!err) return KG_ERR_CUDA;
  Workspace ws(s);
  uint64_t* cnt = ws.alloc<uint64_t>(C);
  uint64_t* off = ws.alloc<uint64_t>(C + 1);
  if (!ws.ok()) return KG_ERR_CUDA;
  if (undirected) {
    UndGeom g{n, chunks, RowBounds::make(n, chunks)};
    st = gnpb_counts(g, C, p, seed, cnt, s, err);
  } else {
    const DirGeom g = DirGeom::make(n, chunks);
    st = gnpb_counts(g, C, p, seed, cnt, s, err);
  }
  if (st) return kg_status(st);
  if ((st = scan_exclusive_u64(cnt, off, C, ws, s))) return kg_status(st);
  ProfScope ps(PROF_OTHER, s);
  gnp_total<<<1, 1, 0, s>>>(off + C, d_count, nullptr, undirected ? 2 : 1, ~uint64_t(0), err);
  return kg_status(launch_ok());
}

kg_status kg_gnp_directed(uint64_t n, double p, uint64_t seed, uint32_t chunks, int id_bytes,
                          void* d_out, uint64_t cap_edges, uint64_t* d_count, void* stream) {
  return kg_gnp_ex(0, n, p, seed, chunks, K_LEAF, id_bytes, d_out, cap_edges, d_count, stream);
}

kg_status kg_gnp_undirected(uint64_t n, double p, uint64_t seed, uint32_t chunks, int id_bytes,
                            void* d_out, uint64_t cap_edges, uint64_t* d_count, void* stream) {
  return kg_gnp_ex(1, n, p, seed, chunks, K_LEAF, id_bytes, d_out, cap_edges, d_count, stream);
}

kg_status kg_gnp_size(int undirected, uint64_t n, double p, uint64_t seed, uint32_t chunks,
                      uint64_t* d_count, void* stream) {
  return kg_gnp_count(undirected, n, p, seed, chunks, K_LEAF, d_count, stream);
}

}  // extern "C"
