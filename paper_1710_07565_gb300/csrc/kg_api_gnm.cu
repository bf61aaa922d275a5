// C ABI: directed G(n,m) (Sec. 4.1), its chunk counts and chunk ranges, the
// edge digest, and the status / error-word plumbing shared by all entry points.
#include <mutex>
#include <unordered_map>

#include "kg.h"
#include "kg_digest.cuh"
#include "kg_run.cuh"

namespace kg {

// ---------------------------------------------------------------- error word, pool
static std::mutex g_words_mu;
static std::unordered_map<int, int*> g_words;  // device -> error word

int* device_error_word() {
  std::mutex& mu = g_words_mu;
  std::unordered_map<int, int*>& words = g_words;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  auto it = words.find(dev);
  if (it != words.end()) return it->second;
  int* p = nullptr;
  if (cudaMalloc(&p, sizeof(int)) != cudaSuccess) return nullptr;
  if (cudaMemset(p, 0, sizeof(int)) != cudaSuccess) return nullptr;
  // keep freed scratch cached in the device's stream-ordered pool
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = ~uint64_t(0);
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  words[dev] = p;
  return p;
}

int sm_count() {
  static std::mutex mu;
  static std::unordered_map<int, int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 152;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
    n = 152;
  cache[dev] = n;
  return n;
}

// ---------------------------------------------------------------- directed
struct DirParams {
  uint64_t n, m;
  uint32_t P;
  u128 Ntot, Unom;
  int d, D;  // tile depth, chunk-tree depth ceil(log2 P)
};

static int check_directed(uint64_t n, uint64_t m, uint32_t P, uint32_t k_leaf, uint32_t k_max,
                          int id_bytes, DirParams& dp) {
  if (n == 0 || P == 0 || uint64_t(P) > n) return ST_ARG;
  if (id_bytes != 4 && id_bytes != 8) return ST_ARG;
  if (k_leaf < 2 || k_max < k_leaf || k_max > uint32_t(K_MAX)) return ST_ARG;
  dp.n = n;
  dp.m = m;
  dp.P = P;
  dp.Ntot = u128(n) * (n - 1);
  if (u128(m) > dp.Ntot) return ST_ARG;
  if (m > M_MAX) return ST_RANGE;
  if (P > (1u << 24)) return ST_RANGE;
  if (id_bytes == 4 && n > (uint64_t(1) << 32)) return ST_RANGE;
  const uint64_t rows_max = uint64_t((u128(n) + P - 1) / P);
  dp.Unom = u128(rows_max) * (n - 1);
  if (dp.Unom >> 64) return ST_RANGE;
  int st = tile_depth(m, dp.Unom, dp.Ntot, k_leaf, dp.d);
  if (st) return st;
  dp.D = 0;
  while ((uint64_t(1) << dp.D) < P) ++dp.D;
  return ST_OK;
}

static DirGeom dir_geom(uint64_t n, uint32_t P) { return DirGeom::make(n, P); }

// Chunk split tree: bands of 8 levels, one block per subtree root.
// node_cnt: scratch of 2^(D+1) counts (chunk_tree_nodes).
static uint64_t chunk_tree_nodes(const DirParams& dp) { return uint64_t(2) << dp.D; }

static int run_chunk_tree(const DirParams& dp, uint64_t seed, uint64_t* cnt, uint64_t* node_cnt,
                          cudaStream_t s, int* err) {
  // the top levels one warp per node, level by level; the rest in bands of
  // 8 levels, one block per subtree root and one thread per node
  int l = 0;
  for (; l <= dp.D && (uint64_t(1) << l) <= WARP_TREE_NODES; ++l) {
    ProfScope ps(PROF_CHUNK_TREE, s);
    chunk_tree_level_warp<<<grid_for(uint64_t(1) << l, 4, sm_count() * 64), 128, 0, s>>>(
        RowBounds::make(dp.n, dp.P), seed, dp.m, l, node_cnt, cnt, err);
    if (launch_ok()) return ST_CUDA;
  }
  for (int l0 = l; l0 <= dp.D; l0 += 8) {
    const int l1 = (l0 + 8 < dp.D + 1) ? l0 + 8 : dp.D + 1;
    ProfScope ps(PROF_CHUNK_TREE, s);
    chunk_tree_band<<<unsigned(1) << l0, 256, 0, s>>>(RowBounds::make(dp.n, dp.P), seed, dp.m, l0,
                                                       l1, node_cnt, cnt, err);
    if (launch_ok()) return ST_CUDA;
  }
  return ST_OK;
}

static int run_chunk_tree(const DirParams& dp, uint64_t seed, uint64_t* cnt, Workspace& ws,
                          cudaStream_t s, int* err) {
  uint64_t* node_cnt = ws.alloc<uint64_t>(chunk_tree_nodes(dp));
  if (!ws.ok()) return ST_CUDA;
  return run_chunk_tree(dp, seed, cnt, node_cnt, s, err);
}

// Everything a whole directed instance takes from scratch, carved in one
// place: the chunk counts, the chunk-tree nodes and the run over all chunks.
struct DirectedScratch {
  uint64_t* cnt = nullptr;
  uint64_t* node_cnt = nullptr;
  ChunkRunScratch<DirGeom::Ctx> run;
  bool carve(const DirParams& dp, Workspace& ws) {
    cnt = ws.alloc<uint64_t>(dp.P);
    node_cnt = ws.alloc<uint64_t>(chunk_tree_nodes(dp));
    return run.carve(dp.P, dp.d, false, false, false, ws) && ws.ok();
  }
};

// Bytes of scratch a whole directed instance takes (a measuring pass of the
// same carve that the run uses).
static uint64_t directed_scratch_bytes(const DirParams& dp) {
  Workspace meas = Workspace::measuring();
  DirectedScratch sc;
  if (!sc.carve(dp, meas)) return ~uint64_t(0);
  return meas.used();
}

}  // namespace kg

using namespace kg;

static cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

extern "C" {

const char* kg_status_str(kg_status s) {
  switch (s) {
    case KG_OK: return "ok";
    case KG_ERR_ARG: return "invalid argument";
    case KG_ERR_RANGE: return "size out of supported range";
    case KG_ERR_CAPACITY: return "output capacity too small";
    case KG_ERR_CUDA: return "CUDA error";
    case KG_ERR_TIMEOUT: return "device wait timed out";
    case KG_ERR_INTERNAL: return "internal limit reached";
  }
  return "unknown status";
}

kg_status kg_shutdown(void) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return KG_ERR_CUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return KG_ERR_CUDA;
  {
    std::lock_guard<std::mutex> lock(g_words_mu);
    auto it = g_words.find(dev);
    if (it != g_words.end()) {
      cudaFree(it->second);
      g_words.erase(it);
    }
  }
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) return KG_ERR_CUDA;
  uint64_t thr = 0;  // the pool's default: release at every synchronisation
  if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr) != cudaSuccess ||
      cudaMemPoolTrimTo(pool, 0) != cudaSuccess)
    return KG_ERR_CUDA;
  return KG_OK;
}

kg_status kg_last_error(void* stream) {
  int* err = device_error_word();
  if (!err) return KG_ERR_CUDA;
  if (cudaStreamSynchronize(as_stream(stream)) != cudaSuccess) return KG_ERR_CUDA;
  int h = 0;
  if (cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return KG_ERR_CUDA;
  if (cudaMemset(err, 0, sizeof(int)) != cudaSuccess) return KG_ERR_CUDA;
  return kg_status(h);
}

kg_status kg_gnm_directed_chunk_counts(uint64_t n, uint64_t m, uint64_t seed, uint32_t chunks,
                                       uint64_t* d_counts, void* stream) {
  DirParams dp;
  int st = check_directed(n, m, chunks, K_LEAF, K_MAX, 8, dp);
  if (st) return kg_status(st);
  if (!d_counts) return KG_ERR_ARG;
  int* err = device_error_word();
  if (!err) return KG_ERR_CUDA;
  Workspace ws(as_stream(stream));
  return kg_status(run_chunk_tree(dp, seed, d_counts, ws, as_stream(stream), err));
}

kg_status kg_gnm_directed_ex(uint64_t n, uint64_t m, uint64_t seed, uint32_t chunks,
                             uint32_t k_leaf, uint32_t k_max, int id_bytes, void* d_out,
                             uint64_t cap_edges, void* stream) {
  DirParams dp;
  int st = check_directed(n, m, chunks, k_leaf, k_max, id_bytes, dp);
  if (st) return kg_status(st);
  if (cap_edges < m) return KG_ERR_CAPACITY;
  if (m == 0) return KG_OK;
  if (!d_out) return KG_ERR_ARG;
  int* err = device_error_word();
  if (!err) return KG_ERR_CUDA;
  cudaStream_t s = as_stream(stream);
  Workspace ws(s);
  DirectedScratch sc;
  if (!sc.carve(dp, ws)) return KG_ERR_CUDA;
  st = run_chunk_tree(dp, seed, sc.cnt, sc.node_cnt, s, err);
  if (st) return kg_status(st);
  st = run_chunks_carved(dir_geom(n, chunks), 0, chunks, sc.cnt, dp.d, k_max, seed, id_bytes,
                         d_out, cap_edges, sc.run, s, err, nullptr, nullptr);
  return kg_status(st);
}

kg_status kg_gnm_directed(uint64_t n, uint64_t m, uint64_t seed, uint32_t chunks, int id_bytes,
                          void* d_out, uint64_t cap_edges, void* stream) {
  return kg_gnm_directed_ex(n, m, seed, chunks, K_LEAF, K_MAX, id_bytes, d_out, cap_edges, stream);
}

kg_status kg_gnm_directed_range(uint64_t n, uint64_t m, uint64_t seed, uint32_t chunks,
                                uint32_t c_begin, uint32_t c_end, const uint64_t* d_counts,
                                int id_bytes, void* d_out, uint64_t cap_edges,
                                uint64_t* d_chunk_digest, uint64_t* d_chunk_hist, void* stream) {
  DirParams dp;
  int st = check_directed(n, m, chunks, K_LEAF, K_MAX, id_bytes, dp);
  if (st) return kg_status(st);
  if (c_begin > c_end || c_end > chunks || !d_counts) return KG_ERR_ARG;
  const uint64_t C = c_end - c_begin;
  if (C == 0) return KG_OK;
  if (!d_out && cap_edges > 0) return KG_ERR_ARG;
  int* err = device_error_word();
  if (!err) return KG_ERR_CUDA;
  cudaStream_t s = as_stream(stream);
  Workspace ws(s);
  const DirGeom g = dir_geom(n, chunks);
  st = run_chunks(g, c_begin, C, d_counts + c_begin, dp.d, K_MAX, seed, id_bytes, d_out, cap_edges,
                  ws, s, err, d_chunk_digest, d_chunk_hist);
  return kg_status(st);
}

kg_status kg_edge_digest(const void* d_edges, uint64_t count, int id_bytes, uint64_t* d_digest,
                         void* stream) {
  if ((id_bytes != 4 && id_bytes != 8) || !d_digest || (count && !d_edges)) return KG_ERR_ARG;
  return kg_status(edge_digest(d_edges, count, id_bytes, d_digest, as_stream(stream)));
}

}  // extern "C"

// ---------------------------------------------------------------- no-allocation variant
// Directed G(n,m) for callers that cannot allocate device memory.  The
// scratch lives in one file-scope device array; every call shares it.
namespace kg {
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[KG_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device with cudaGetSymbolAddress (with that device current) and cached.
void* noalloc_scratch_address() {
  static std::mutex mu;
  static std::unordered_map<int, void*> addr;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  auto it = addr.find(dev);
  if (it != addr.end()) return it->second;
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return nullptr;
  addr[dev] = p;
  return p;
}

}  // namespace
}  // namespace kg

extern "C" kg_status kg_gnm_directed_noalloc(uint64_t n, uint64_t m, uint64_t seed, uint32_t chunks,
                                             int id_bytes, void* d_out, uint64_t cap_edges,
                                             int* d_status, void* stream) {
  DirParams dp;
  int st = check_directed(n, m, chunks, K_LEAF, K_MAX, id_bytes, dp);
  if (st) return kg_status(st);
  if (!d_status) return KG_ERR_ARG;
  if (cap_edges < m) return KG_ERR_CAPACITY;
  // the same carve, measured: an instance whose scratch does not fit is
  // rejected here, before anything is enqueued
  if (directed_scratch_bytes(dp) > uint64_t(KG_NOALLOC_SCRATCH_BYTES)) return KG_ERR_RANGE;
  if (m > 0 && !d_out) return KG_ERR_ARG;
  void* arena = noalloc_scratch_address();
  if (!arena) return KG_ERR_CUDA;
  cudaStream_t s = as_stream(stream);
  Workspace ws(s, arena, KG_NOALLOC_SCRATCH_BYTES);
  DirectedScratch sc;
  if (!sc.carve(dp, ws)) return KG_ERR_INTERNAL;  // cannot happen after the check above
  // device-side checks report into the caller's status word, cleared first
  int* err = d_status;
  if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) return KG_ERR_CUDA;
  if (m == 0) return KG_OK;
  st = run_chunk_tree(dp, seed, sc.cnt, sc.node_cnt, s, err);
  if (st) return kg_status(st);
  st = run_chunks_carved(dir_geom(n, chunks), 0, chunks, sc.cnt, dp.d, K_MAX, seed, id_bytes,
                         d_out, cap_edges, sc.run, s, err, nullptr, nullptr);
  return kg_status(st);
}

// Scratch bytes kg_gnm_directed_noalloc needs for an instance (host only, no
// device work): what its arena check compares with KG_NOALLOC_SCRATCH_BYTES.
extern "C" kg_status kg_gnm_directed_noalloc_scratch(uint64_t n, uint64_t m, uint32_t chunks,
                                                     uint64_t* h_bytes) {
  DirParams dp;
  int st = check_directed(n, m, chunks, K_LEAF, K_MAX, 8, dp);
  if (st) return kg_status(st);
  if (!h_bytes) return KG_ERR_ARG;
  *h_bytes = directed_scratch_bytes(dp);
  return KG_OK;
}
