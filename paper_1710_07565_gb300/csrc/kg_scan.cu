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

// Per block: exclusive scan of its items plus the block's carry-in.
__global__ void __launch_bounds__(SCAN_THREADS)
    scan_apply_kernel(const uint64_t* __restrict__ in, uint64_t n, const uint64_t* __restrict__ carry,
                      uint64_t* __restrict__ out) {
  const uint64_t base = uint64_t(blockIdx.x) * SCAN_ITEMS;
  // thread t owns the SCAN_PER_THREAD consecutive items base + t*PER + k
  uint64_t v[SCAN_PER_THREAD];
  uint64_t s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_PER_THREAD; ++k) {
    const uint64_t i = base + uint64_t(threadIdx.x) * SCAN_PER_THREAD + k;
    v[k] = i < n ? in[i] : 0;
    s += v[k];
  }
  uint64_t tot;
  uint64_t incl = block_inclusive_scan<SCAN_THREADS>(s, tot);
  uint64_t run = incl - s + (carry ? carry[blockIdx.x] : 0);
#pragma unroll
  for (int k = 0; k < SCAN_PER_THREAD; ++k) {
    const uint64_t i = base + uint64_t(threadIdx.x) * SCAN_PER_THREAD + k;
    if (i < n) out[i] = run;
    run += v[k];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == SCAN_THREADS - 1) out[n] = run;
}

int scan_exclusive_u64(const uint64_t* in, uint64_t* out, uint64_t n, Workspace& ws,
                       cudaStream_t s) {
  if (n == 0) {
    return cudaMemsetAsync(out, 0, sizeof(uint64_t), s) == cudaSuccess ? ST_OK : ST_CUDA;
  }
  const uint64_t nb = (n + SCAN_ITEMS - 1) / SCAN_ITEMS;
  if (nb == 1) {
    ProfScope ps(PROF_SCAN, s);
    scan_apply_kernel<<<1, SCAN_THREADS, 0, s>>>(in, n, nullptr, out);
    return cudaGetLastError() == cudaSuccess ? ST_OK : ST_CUDA;
  }
  uint64_t* part = ws.alloc<uint64_t>(nb);
  uint64_t* carry = ws.alloc<uint64_t>(nb + 1);
  if (!ws.ok()) return ST_CUDA;
  {
    ProfScope ps(PROF_SCAN, s);
    scan_reduce_kernel<<<unsigned(nb), SCAN_THREADS, 0, s>>>(in, n, part);
  }
  const int st = scan_exclusive_u64(part, carry, nb, ws, s);
  if (st) return st;
  ProfScope ps(PROF_SCAN, s);
  scan_apply_kernel<<<unsigned(nb), SCAN_THREADS, 0, s>>>(in, n, carry, out);
  return cudaGetLastError() == cudaSuccess ? ST_OK : ST_CUDA;
}

}  // namespace kg
