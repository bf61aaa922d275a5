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
  if (blocks > 152 * 32) blocks = 152 * 32;
  ProfScope ps(PROF_DIGEST, s);
  if (id_bytes == 4)
    edge_digest_kernel<uint32_t><<<unsigned(blocks), 256, 0, s>>>(
        e, count, reinterpret_cast<unsigned long long*>(out));
  else
    edge_digest_kernel<uint64_t><<<unsigned(blocks), 256, 0, s>>>(
        e, count, reinterpret_cast<unsigned long long*>(out));
  return cudaGetLastError() == cudaSuccess ? ST_OK : ST_CUDA;
}

// One block per chunk: edges [off[c], off[c+1]) of the range output, sorted by u.
template <class Id, class Geom>
__global__ void chunk_digest_kernel(Geom g, uint64_t c_begin, uint64_t C,
                                    const uint64_t* __restrict__ off, const void* __restrict__ e,
                                    uint64_t cap, uint64_t* __restrict__ digest,
                                    uint64_t* __restrict__ hist) {
  __shared__ unsigned long long h[65];
  __shared__ unsigned long long dsum, distinct;
  for (uint64_t c = blockIdx.x; c < C; c += gridDim.x) {
    for (int b = threadIdx.x; b < 65; b += blockDim.x) h[b] = 0;
    if (threadIdx.x == 0) dsum = distinct = 0;
    __syncthreads();
    const uint64_t beg = off[c], end = off[c + 1] < cap ? off[c + 1] : cap;
    unsigned long long ls = 0, ld = 0;
    for (uint64_t i = beg + threadIdx.x; i < end; i += blockDim.x) {
      uint64_t u, v;
      load_edge<Id>(e, i, u, v);
      ls += edge_hash(u, v);
      uint64_t pu = ~uint64_t(0), pv;
      if (i > beg) load_edge<Id>(e, i - 1, pu, pv);
      if (i == beg || pu != u) {  // a run of out-edges of u starts here
        uint64_t j = i + 1;
        for (; j < end; ++j) {
          uint64_t uj, vj;
          load_edge<Id>(e, j, uj, vj);
          if (uj != u) break;
        }
        const uint64_t len = j - i;
        atomicAdd(&h[len < 64 ? len : 64], 1ull);
        ++ld;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ls += __shfl_xor_sync(0xffffffffu, ls, o);
      ld += __shfl_xor_sync(0xffffffffu, ld, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&dsum, ls);
      atomicAdd(&distinct, ld);
    }
    __syncthreads();
    const uint64_t cc = c_begin + c;
    const uint64_t rows = row_bound(g.n, g.P, cc + 1) - row_bound(g.n, g.P, cc);
    if (digest && threadIdx.x == 0) digest[c] = dsum;
    if (hist)
      for (int b = threadIdx.x; b < 65; b += blockDim.x)
        hist[c * 65 + b] = h[b] + (b == 0 ? rows - distinct : 0);
    __syncthreads();
  }
}

template <class Geom>
int chunk_digest(const Geom& g, uint64_t c_begin, uint64_t C, const uint64_t* off, int id_bytes,
                 const void* e, uint64_t cap, uint64_t* digest, uint64_t* hist, cudaStream_t s) {
  const unsigned blocks = unsigned(C < 152 * 64 ? C : 152 * 64);
  ProfScope ps(PROF_DIGEST, s);
  if (id_bytes == 4)
    chunk_digest_kernel<uint32_t, Geom><<<blocks, 256, 0, s>>>(g, c_begin, C, off, e, cap, digest,
                                                               hist);
  else
    chunk_digest_kernel<uint64_t, Geom><<<blocks, 256, 0, s>>>(g, c_begin, C, off, e, cap, digest,
                                                               hist);
  return cudaGetLastError() == cudaSuccess ? ST_OK : ST_CUDA;
}

}  // namespace kg
