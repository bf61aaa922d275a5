// Host-side launch sequence of the undirected assembly (Sec. 4.2): the sampled
// pairs (u > v) become the (u, v)-sorted list of both directions.
#pragma once
#include "kg_prof.h"
#include "kg_run.cuh"
#include "kg_und.cuh"

namespace kg {

// pairs (u > v) -> both directions, sorted by (u, v), into out[0 .. 2 npairs)
template <class Id>
inline int assemble(const Id* pairs, const uint64_t* npairs_dev, uint64_t npairs_host, uint64_t n,
                    Id* out, uint64_t cap, Workspace& ws, cudaStream_t s, int* err) {
  unsigned long long* deg = ws.alloc<unsigned long long>(n);
  uint64_t* rowptr = ws.alloc<uint64_t>(n + 1);
  unsigned long long* cursor = ws.alloc<unsigned long long>(n);
  unsigned long long* long_rows = ws.alloc<unsigned long long>(n);
  unsigned long long* nlong = ws.alloc<unsigned long long>(1);
  if (!ws.ok()) return ST_CUDA;
  if (cudaMemsetAsync(deg, 0, n * 8, s) != cudaSuccess ||
      cudaMemsetAsync(nlong, 0, 8, s) != cudaSuccess)
    return ST_CUDA;
  const uint64_t work = npairs_dev ? cap / 2 : npairs_host;
  {
    ProfScope ps(PROF_ASSEMBLY, s);
    und_degree<Id><<<grid_for(work, 256, 152 * 16), 256, 0, s>>>(pairs, npairs_dev, npairs_host,
                                                                 deg);
    if (launch_ok()) return ST_CUDA;
  }
  int st = scan_exclusive_u64(reinterpret_cast<const uint64_t*>(deg), rowptr, n, ws, s);
  if (st) return st;
  if (cudaMemcpyAsync(cursor, rowptr, n * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return ST_CUDA;
  {
    ProfScope ps(PROF_ASSEMBLY, s);
    und_scatter<Id><<<grid_for(work, 256, 152 * 16), 256, 0, s>>>(pairs, npairs_dev, npairs_host,
                                                                  cursor, out, cap, err);
    if (launch_ok()) return ST_CUDA;
  }
  {
    ProfScope ps(PROF_ASSEMBLY, s);
    und_sort_short<Id><<<grid_for(n, 8, 152 * 32), 256, 0, s>>>(rowptr, n, out, cap, long_rows,
                                                                nlong);
    if (launch_ok()) return ST_CUDA;
  }
  ProfScope ps(PROF_ASSEMBLY, s);
  und_sort_long<Id><<<152 * 2, 256, 0, s>>>(rowptr, out, cap, long_rows, nlong);
  return launch_ok();
}

}  // namespace kg
