// Exclusive prefix sum of per-chunk / per-tile sample counts.  The scan sizes
// the output exactly: the offsets of every tile follow from the counts with
// no atomics (reduce-then-scan over blocks of SCAN_ITEMS values).
#include "kg_common.cuh"
#include "kg_internal.h"
#include "kg_prof.h"

namespace kg {

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_PER_THREAD = 8;
constexpr int SCAN_ITEMS = SCAN_THREADS * SCAN_PER_THREAD;

__global__ void __launch_bounds__(SCAN_THREADS)
    scan_reduce_kernel(const uint64_t* __restrict__ in, uint64_t n, uint64_t* __restrict__ part) {
  const uint64_t base = uint64_t(blockIdx.x) * SCAN_ITEMS;
  uint64_t s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_PER_THREAD; ++k) {
    const uint64_t i = base + uint64_t(k) * SCAN_THREADS + threadIdx.x;
    if (i < n) s += in[i];
  }
  uint64_t tot;
  block_inclusive_scan<SCAN_THREADS>(s, tot);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// Per block: exclusive scan of its items plus the block's carry-in.  Warp w
// owns the 256 consecutive items base + 256 w + [0, 256), read and written in
// eight coalesced rows of 32 (lane l holds item 32 k + l of row k); each row
// is scanned across the lanes and carries its total into the next row.
__global__ void __launch_bounds__(SCAN_THREADS)
    scan_apply_kernel(const uint64_t* __restrict__ in, uint64_t n, const uint64_t* __restrict__ carry,
                      uint64_t* __restrict__ out) {
  __shared__ uint64_t warp_base[SCAN_THREADS / 32];
  const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint64_t wbase = uint64_t(blockIdx.x) * SCAN_ITEMS + uint64_t(wid) * (32 * SCAN_PER_THREAD);
  uint64_t v[SCAN_PER_THREAD];
#pragma unroll
  for (int k = 0; k < SCAN_PER_THREAD; ++k) {
    const uint64_t i = wbase + uint64_t(k) * 32 + lane;
    v[k] = i < n ? in[i] : 0;
  }
  // exclusive prefix of every item within the warp's 256
  uint64_t run = 0;
#pragma unroll
  for (int k = 0; k < SCAN_PER_THREAD; ++k) {
    uint64_t x = v[k];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= unsigned(o)) x += y;
    }
    const uint64_t excl = run + x - v[k];
    run += __shfl_sync(0xffffffffu, x, 31);
    v[k] = excl;
  }
  // warp totals to warp bases (one warp scans the sixteen totals)
  if (lane == 0) warp_base[wid] = run;
  __syncthreads();
  if (wid == 0) {
    const uint64_t t = lane < SCAN_THREADS / 32 ? warp_base[lane] : 0;
    uint64_t x = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= unsigned(o)) x += y;
    }
    if (lane < SCAN_THREADS / 32) warp_base[lane] = x - t + (carry ? carry[blockIdx.x] : 0);
  }
  __syncthreads();
  const uint64_t add = warp_base[wid];
#pragma unroll
  for (int k = 0; k < SCAN_PER_THREAD; ++k) {
    const uint64_t i = wbase + uint64_t(k) * 32 + lane;
    if (i < n) out[i] = v[k] + add;
  }
  // the total after the last item
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == SCAN_THREADS - 1) out[n] = run + add;
}

bool scan_scratch(uint64_t n, Workspace& ws, ScanScratch& sc) {
  sc.levels = 0;
  for (;;) {
    if (n == 0) return ws.ok();
    const uint64_t nb = (n + SCAN_ITEMS - 1) / SCAN_ITEMS;
    if (nb == 1) return ws.ok();
    if (sc.levels == ScanScratch::LEVELS) return false;
    sc.part[sc.levels] = ws.alloc<uint64_t>(nb);
    sc.carry[sc.levels] = ws.alloc<uint64_t>(nb + 1);
    ++sc.levels;
    n = nb;
  }
}

static int scan_level(const uint64_t* in, uint64_t* out, uint64_t n, const ScanScratch& sc,
                      int level, cudaStream_t s) {
  if (n == 0) {
    return cudaMemsetAsync(out, 0, sizeof(uint64_t), s) == cudaSuccess ? ST_OK : ST_CUDA;
  }
  const uint64_t nb = (n + SCAN_ITEMS - 1) / SCAN_ITEMS;
  if (nb == 1) {
    ProfScope ps(PROF_SCAN, s);
    scan_apply_kernel<<<1, SCAN_THREADS, 0, s>>>(in, n, nullptr, out);
    return cudaGetLastError() == cudaSuccess ? ST_OK : ST_CUDA;
  }
  if (level >= sc.levels) return ST_INTERNAL;
  uint64_t* part = sc.part[level];
  uint64_t* carry = sc.carry[level];
  {
    ProfScope ps(PROF_SCAN, s);
    scan_reduce_kernel<<<unsigned(nb), SCAN_THREADS, 0, s>>>(in, n, part);
  }
  const int st = scan_level(part, carry, nb, sc, level + 1, s);
  if (st) return st;
  ProfScope ps(PROF_SCAN, s);
  scan_apply_kernel<<<unsigned(nb), SCAN_THREADS, 0, s>>>(in, n, carry, out);
  return cudaGetLastError() == cudaSuccess ? ST_OK : ST_CUDA;
}

int scan_exclusive_u64(const uint64_t* in, uint64_t* out, uint64_t n, const ScanScratch& sc,
                       cudaStream_t s) {
  return scan_level(in, out, n, sc, 0, s);
}

int scan_exclusive_u64(const uint64_t* in, uint64_t* out, uint64_t n, Workspace& ws,
                       cudaStream_t s) {
  ScanScratch sc;
  if (!scan_scratch(n, ws, sc)) return ST_CUDA;
  return scan_level(in, out, n, sc, 0, s);
}

}  // namespace kg
