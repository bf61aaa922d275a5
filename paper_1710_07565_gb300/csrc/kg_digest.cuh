// Order-independent digests of edge lists: the sum of splitmix64(u ^ rotl(v,32))
// over the edges, and per chunk the histogram of out-degree values
// (vertices of the chunk's rows with out-degree 0..63, >= 64).
#pragma once
#include "kg_common.cuh"
#include "kg_internal.h"
#include "kg_prof.h"

namespace kg {

template <class Id>
__device__ __forceinline__ void load_edge(const void* e, uint64_t i, uint64_t& u, uint64_t& v) {
  if (sizeof(Id) == 4) {
    const uint2 w = reinterpret_cast<const uint2*>(e)[i];
    u = w.x;
    v = w.y;
  } else {
    const ulonglong2 w = reinterpret_cast<const ulonglong2*>(e)[i];
    u = w.x;
    v = w.y;
  }
}

template <class Id>
__global__ void edge_digest_kernel(const void* __restrict__ e, uint64_t count,
                                   unsigned long long* __restrict__ out) {
  unsigned long long s = 0;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count;
       i += uint64_t(gridDim.x) * blockDim.x) {
    uint64_t u, v;
    load_edge<Id>(e, i, u, v);
    s += edge_hash(u, v);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

inline int edge_digest(const void* e, uint64_t count, int id_bytes, uint64_t* out,
                       cudaStream_t s) {
  if (cudaMemsetAsync(out, 0, sizeof(uint64_t), s) != cudaSuccess) return ST_CUDA;
  if (count == 0) return ST_OK;
  uint64_t blocks = (count + 255) / 256;
  if (blocks > sm_count() * 32) blocks = sm_count() * 32;
  ProfScope ps(PROF_DIGEST, s);
  if (id_bytes == 4)
    edge_digest_kernel<uint32_t><<<unsigned(blocks), 256, 0, s>>>(
        e, count, reinterpret_cast<unsigned long long*>(out));
  else
    edge_digest_kernel<uint64_t><<<unsigned(blocks), 256, 0, s>>>(
        e, count, reinterpret_cast<unsigned long long*>(out));
  return cudaGetLastError() == cudaSuccess ? ST_OK : ST_CUDA;
}

}  // namespace kg
