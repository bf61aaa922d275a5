// Orchestration shared by the entry points: tile-tree depth, and tile trees +
// scan + leaf kernels over a range of chunks of one geometry.
#pragma once
#include "kg_internal.h"
#include "kg_leaf.cuh"
#include "kg_leaf_sparse.cuh"
#include "kg_prof.h"

namespace kg {

// Tile-tree depth, one per instance: smallest d with E <= k_leaf 2^d, where E
// is the expected count of a chunk of nominal universe U_nom (d stops once
// 2^(d+1) > U_nom).
inline int tile_depth_e(double E, u128 Unom, uint32_t k_leaf, int& d_out) {
  int d = 0;
  for (;;) {
    if (E <= double(k_leaf) * double(uint64_t(1) << d)) break;
    if ((u128(2) << d) > Unom) break;
    if (d == D_MAX) return ST_RANGE;
    ++d;
  }
  d_out = d;
  return ST_OK;
}

// G(n,m): E = m (U_nom / N).
inline int tile_depth(uint64_t m, u128 Unom, u128 Ntot, uint32_t k_leaf, int& d_out) {
  return tile_depth_e(double(m) * (dbl(Unom) / dbl(Ntot)), Unom, k_leaf, d_out);
}

inline unsigned grid_for(uint64_t items, unsigned per_block, unsigned cap) {
  uint64_t b = (items + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return unsigned(b);
}

inline int launch_ok() { return cudaGetLastError() == cudaSuccess ? ST_OK : ST_CUDA; }

// Scratch of one run_chunks call, carved by one function before any launch,
// so that a measuring Workspace counts exactly the bytes a run takes.
template <class Ctx>
struct ChunkRunScratch {
  uint64_t *A = nullptr, *B = nullptr;  // tile-tree levels (ping-pong)
  uint64_t* tile_off = nullptr;         // T + 1 scanned tile counts
  ScanScratch scan;
  unsigned long long* digest = nullptr;  // per chunk, when the caller gives none
  unsigned long long* hist = nullptr;    // per chunk x 65, likewise
  TileRec* rec = nullptr;                // per tile run records
  // tiles over k_max from the front, tiles the sparse kernel leaves to the
  // general one from the back; nbig[0], nbig[1]: their counts
  unsigned long long *big = nullptr, *nbig = nullptr;
  TileDesc<Ctx>* desc = nullptr;         // per tile descriptors

  // C chunks with tile depth d; digest / hist: whether the caller gives them;
  // want: whether the digest and histogram are produced at all.
  bool carve(uint64_t C, int d, bool want, bool have_digest, bool have_hist, Workspace& ws) {
    const uint64_t T = C << d;
    if (d > 0) {
      A = ws.alloc<uint64_t>(T);
      B = ws.alloc<uint64_t>(T);
    }
    tile_off = ws.alloc<uint64_t>(T + 1);
    if (!scan_scratch(T, ws, scan)) return false;
    if (want) {
      if (!have_digest) digest = ws.alloc<unsigned long long>(C);
      if (!have_hist) hist = ws.alloc<unsigned long long>(C * 65);
      rec = ws.alloc<TileRec>(T);
    }
    big = ws.alloc<unsigned long long>(T);
    nbig = ws.alloc<unsigned long long>(2);
    desc = ws.alloc<TileDesc<Ctx>>(T);
    return ws.ok();
  }
};

// Whether the tiles of a directed run go to the sparse leaf kernel: Floyd's
// replacements must be rare (tile width W >= 2^26 pairs: a 2048-draw tile
// repeats a draw with probability below 1/32, a 1024-draw one below 1/128)
// and n - 1 >= 4 for the map's quotient estimate.
// Nominal universe of a run's chunks, on the host: the first chunk's
// (directed), a rectangle of two row blocks of ceil(n / P) rows (undirected).
template <class Geom>
inline uint64_t nominal_universe(const Geom& g, uint64_t c_begin);

// Tile-tree levels whose node universes are below EXACT_NODE_U draw exact
// hypergeometrics (ratio of uniforms over five log-factorial terms, rejection
// counts that differ from lane to lane): up to WARP_TREE_NODES_EXACT nodes
// they also go one warp per node.  Larger universes take the binomial
// approximation of the variate, cheap and even per lane, and go one lane per
// node from WARP_TREE_NODES on.
constexpr uint64_t WARP_TREE_NODES_EXACT = 16384;
constexpr uint64_t EXACT_NODE_U = uint64_t(1) << 40;

// The undirected geometry under a chunk-list geometry (or itself).
inline const UndGeom& und_base(const UndGeom& g) { return g; }
template <class G>
inline const UndGeom& und_base(const G& g) {
  return g.base;
}

template <class Geom>
inline uint64_t nominal_universe(const Geom& g, uint64_t c_begin) {
  if constexpr (std::is_same<Geom, DirGeom>::value) {
    return g.universe(c_begin);
  } else if constexpr (std::is_same<typename Geom::Ctx, UndGeom::Ctx>::value) {
    const UndGeom& b = und_base(g);
    const u128 r = (u128(b.n) + b.P - 1) / b.P;
    const u128 U = r * r;
    return (U >> 64) ? ~uint64_t(0) : uint64_t(U);
  } else {
    return ~uint64_t(0);
  }
}

template <class Geom>
inline bool use_sparse_leaf(const Geom& g, uint64_t c_begin, int d) {
  if constexpr (std::is_same<Geom, DirGeom>::value) {
    if (g.n < 5) return false;
    return tile_width(g.universe(c_begin), d) >= (uint64_t(1) << 26);
  } else if constexpr (std::is_same<typename Geom::Ctx, UndGeom::Ctx>::value) {
    // undirected: the nominal rectangle chunk (row blocks of ceil(n / P) rows)
    const UndGeom& b = und_base(g);
    const u128 r = (u128(b.n) + b.P - 1) / b.P;
    const u128 U = r * r;
    if (r < 4 || (U >> 64)) return false;
    return tile_width(uint64_t(U), d) >= (uint64_t(1) << 26);
  } else {
    return false;
  }
}

// Tile descriptors + leaf kernels over the T tiles of a run.
template <class Geom, class Sink, bool DIGEST>
inline int launch_leaf(const Geom& g, const Sink& sink, uint64_t c_begin, int d, uint32_t k_max,
                       uint64_t seed, const uint64_t* tile_cnt, const uint64_t* tile_off,
                       uint64_t T, int* err, DigestOut dig,
                       const ChunkRunScratch<typename Geom::Ctx>& sc, cudaStream_t s) {
  unsigned long long* big = sc.big;
  unsigned long long* nbig = sc.nbig;
  if (cudaMemsetAsync(nbig, 0, 2 * sizeof(unsigned long long), s) != cudaSuccess) return ST_CUDA;
  using Desc = TileDesc<typename Geom::Ctx>;
  // undirected tiles without the fused digest also have a sparse path
  constexpr bool SPARSE_UND = std::is_same<typename Geom::Ctx, UndGeom::Ctx>::value && !DIGEST;
  Desc* desc = sc.desc;
  const bool sparse = (std::is_same<Geom, DirGeom>::value || SPARSE_UND) && use_sparse_leaf(g, c_begin, d);
  SparseRoute route{0, 0};
  SparseMap mp{};
  if constexpr (std::is_same<Geom, DirGeom>::value) {
    if (sparse) {
      mp = sparse_map(g.n);
      route = sparse_route(mp, true);
    }
  } else if constexpr (SPARSE_UND) {
    route.on = sparse ? 1 : 0;  // per-tile maps: the descriptor kernel checks each tile
  }
  {
    ProfScope ps(PROF_OTHER, s);
    tile_desc_kernel<Geom><<<grid_for(T, 256, sm_count() * 32), 256, 0, s>>>(
        g, c_begin, d, k_max, seed, tile_cnt, tile_off, T, desc, big, nbig, err, route);
    if (launch_ok()) return ST_CUDA;
  }
  const unsigned grid = unsigned(T < 0x7fffffffull ? T : 0x7fffffffull);
  if constexpr (std::is_same<Geom, DirGeom>::value || SPARSE_UND) {
    if (sparse) {
      {
        ProfScope ps(PROF_LEAF, s);
        // one block per tile (a persistent grid of 1-16 waves measured no faster)
        leaf_sparse_kernel<Geom, Sink, DIGEST><<<grid, SP_THREADS, 0, s>>>(
            mp, sink, desc, T, err, dig, big, nbig + 1);
        if (launch_ok()) return ST_CUDA;
      }
      // the tiles the sparse kernel left (usually none): a fixed grid that
      // reads the list's length on the device
      ProfScope ps(PROF_OTHER, s);
      leaf_fast_kernel<Geom, Sink, DIGEST, false><<<sm_count() * 4, FAST_THREADS, 0, s>>>(
          g, sink, d, round_keys(seed), desc, T, err, dig, big, nbig + 1);
      if (launch_ok()) return ST_CUDA;
    }
  }
  if (!sparse) {
    ProfScope ps(PROF_LEAF, s);
    leaf_fast_kernel<Geom, Sink, DIGEST, false><<<grid, FAST_THREADS, 0, s>>>(
        g, sink, d, round_keys(seed), desc, T, err, dig);
    if (launch_ok()) return ST_CUDA;
  }
  ProfScope ps(PROF_OTHER, s);
  leaf_resplit_kernel<Geom, Sink, DIGEST, Desc><<<sm_count(), LEAF_THREADS, 0, s>>>(
      g, sink, k_max, desc, err, dig, big, nbig);
  return launch_ok();
}

// Tile trees + scan + leaves for chunks [c_begin, c_begin + C) of a geometry,
// with scratch carved beforehand (ChunkRunScratch::carve with the same C, d
// and digest arguments).  level0: the chunks' counts (device).  Pairs go to
// d_out[0 ..).  With digest pointers the leaf kernel also produces the
// per-chunk digest and out-degree histogram (directed geometry only).
template <class Geom>
int run_chunks_carved(const Geom& g, uint64_t c_begin, uint64_t C, const uint64_t* level0, int d,
                      uint32_t k_max, uint64_t seed, int id_bytes, void* d_out, uint64_t cap,
                      const ChunkRunScratch<typename Geom::Ctx>& sc, cudaStream_t s, int* err,
                      uint64_t* digest, uint64_t* hist) {
  const uint64_t T = C << d;
  const uint64_t* in = level0;
  for (int level = 0; level < d; ++level) {
    uint64_t* out = (level & 1) ? sc.B : sc.A;
    const uint64_t nodes = C << level;
    ProfScope ps(PROF_TILE_TREE, s);
    if (nodes <= WARP_TREE_NODES ||
        (nodes <= WARP_TREE_NODES_EXACT && (nominal_universe(g, c_begin) >> level) < EXACT_NODE_U))
      // few nodes: one warp per variate, so that the level waits for one
      // variate's chain instead of the slowest of 32 lanes
      tile_tree_level_warp<Geom><<<grid_for(nodes, 4, sm_count() * 64), 128, 0, s>>>(
          g, c_begin, C, d, level, seed, in, out, err);
    else
      // one-warp blocks, one node per lane: the levels spread over all SMs
      tile_tree_level<Geom><<<grid_for(nodes, 32, sm_count() * 64), 32, 0, s>>>(
          g, c_begin, C, d, level, seed, in, out, err);
    if (launch_ok()) return ST_CUDA;
    in = out;
  }
  uint64_t* tile_off = sc.tile_off;
  int st = scan_exclusive_u64(in, tile_off, T, sc.scan, s);
  if (st) return st;
  const bool want = digest || hist;
  DigestOut dig{nullptr, nullptr, nullptr};
  if (want) {
    dig.digest = digest ? reinterpret_cast<unsigned long long*>(digest) : sc.digest;
    dig.hist = hist ? reinterpret_cast<unsigned long long*>(hist) : sc.hist;
    dig.rec = sc.rec;
    if (cudaMemsetAsync(dig.digest, 0, C * sizeof(uint64_t), s) != cudaSuccess ||
        cudaMemsetAsync(dig.hist, 0, C * 65 * sizeof(uint64_t), s) != cudaSuccess ||
        cudaMemsetAsync(dig.rec, 0, T * sizeof(TileRec), s) != cudaSuccess)
      return ST_CUDA;
  }
  if (id_bytes == 4) {
    PairSink<uint32_t> sink{static_cast<uint32_t*>(d_out), cap, err};
    st = want ? launch_leaf<Geom, PairSink<uint32_t>, true>(g, sink, c_begin, d, k_max, seed, in,
                                                             tile_off, T, err, dig, sc, s)
              : launch_leaf<Geom, PairSink<uint32_t>, false>(g, sink, c_begin, d, k_max, seed, in,
                                                              tile_off, T, err, dig, sc, s);
  } else {
    PairSink<uint64_t> sink{static_cast<uint64_t*>(d_out), cap, err};
    st = want ? launch_leaf<Geom, PairSink<uint64_t>, true>(g, sink, c_begin, d, k_max, seed, in,
                                                             tile_off, T, err, dig, sc, s)
              : launch_leaf<Geom, PairSink<uint64_t>, false>(g, sink, c_begin, d, k_max, seed, in,
                                                              tile_off, T, err, dig, sc, s);
  }
  if (st || !want) return st;
  ProfScope ps(PROF_DIGEST, s);
  chunk_run_merge<Geom><<<grid_for(C, 128, sm_count() * 8), 128, 0, s>>>(g, c_begin, C, d, dig.rec,
                                                                   dig.hist);
  return launch_ok();
}

template <class Geom>
int run_chunks(const Geom& g, uint64_t c_begin, uint64_t C, const uint64_t* level0, int d,
               uint32_t k_max, uint64_t seed, int id_bytes, void* d_out, uint64_t cap,
               Workspace& ws, cudaStream_t s, int* err, uint64_t* digest = nullptr,
               uint64_t* hist = nullptr) {
  ChunkRunScratch<typename Geom::Ctx> sc;
  if (!sc.carve(C, d, digest || hist, digest != nullptr, hist != nullptr, ws)) return ST_CUDA;
  return run_chunks_carved(g, c_begin, C, level0, d, k_max, seed, id_bytes, d_out, cap, sc, s, err,
                           digest, hist);
}

}  // namespace kg
