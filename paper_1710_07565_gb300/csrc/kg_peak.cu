// Instrumentation kernels that measure the ceilings the generators are
// compared with on the GPU they run on: a write-only store stream (the bound
// of edge emission, which reads almost nothing) and the FP64 add / multiply
// rate under -fmad=false (the bound of the G(n,p) skip walk, one logarithm
// per kept pair).  No counterpart in the paper.
#include "kg.h"
#include "kg_common.cuh"
#include "kg_internal.h"
#include "kg_prof.h"

namespace kg {

// 16-byte stores over [buf, buf + n16 * 16): every thread stores 4 groups
// per step at a distance of the grid's width, so that each warp instruction
// covers 512 consecutive bytes; evict-first stores (mode 0) or write-back
// stores (mode 1).
template <int MODE>
__global__ void __launch_bounds__(256) store_stream(uint4* __restrict__ buf, uint64_t n16,
                                                   uint32_t value) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  const uint4 w = make_uint4(value, value ^ 0x9E3779B9u, value + 1u, ~value);
  uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  for (; i + 3 * stride < n16; i += 4 * stride) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (MODE == 0)
        __stcs(buf + i + q * stride, w);
      else
        buf[i + q * stride] = w;
    }
  }
  for (; i < n16; i += stride) {
    if (MODE == 0)
      __stcs(buf + i, w);
    else
      buf[i] = w;
  }
}

// FP64 chains: every thread runs 8 independent chains of x = x * a + b,
// with the multiply and the add rounded separately (the build's -fmad=false):
// 16 FP64 operations per iteration and thread.
__global__ void __launch_bounds__(256) fp64_chains(double* __restrict__ out, uint32_t iters,
                                                   double a, double b) {
  double x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = double(threadIdx.x + j) * 1e-3;
  for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = x[j] * a + b;
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s = s + x[j];
  if (s == 12345.678) out[0] = s;  // keeps the chains live; never true for these a, b
  if (threadIdx.x == 0 && blockIdx.x == 0) out[1] = s;
}

}  // namespace kg

using namespace kg;

extern "C" {

kg_status kg_peak_store(void* d_buf, uint64_t bytes, int mode, void* stream) {
  if (!d_buf || (reinterpret_cast<uintptr_t>(d_buf) & 15) || (bytes & 15) || mode < 0 || mode > 1)
    return KG_ERR_ARG;
  if (bytes == 0) return KG_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const unsigned grid = unsigned(sm_count() * 8);
  ProfScope ps(PROF_OTHER, s);
  if (mode == 0)
    store_stream<0><<<grid, 256, 0, s>>>(static_cast<uint4*>(d_buf), bytes / 16, 0x5EEDu);
  else
    store_stream<1><<<grid, 256, 0, s>>>(static_cast<uint4*>(d_buf), bytes / 16, 0x5EEDu);
  return cudaGetLastError() == cudaSuccess ? KG_OK : KG_ERR_CUDA;
}

kg_status kg_peak_fp64(double* d_out, uint32_t blocks, uint32_t iters, void* stream) {
  if (!d_out || blocks == 0 || iters == 0) return KG_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ProfScope ps(PROF_OTHER, s);
  // a slightly contracting affine map: the values stay finite and normal
  fp64_chains<<<blocks, 256, 0, s>>>(d_out, iters, 0.999999, 1e-6);
  return cudaGetLastError() == cudaSuccess ? KG_OK : KG_ERR_CUDA;
}

}  // extern "C"
