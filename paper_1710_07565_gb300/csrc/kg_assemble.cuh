// Host-side launch sequence of the undirected assembly (Sec. 4.2): the sampled
// pairs (u > v) become the (u, v)-sorted list of both directions.
#pragma once
#include "kg_prof.h"
#include "kg_run.cuh"
#include "kg_und.cuh"

namespace kg {

// pairs (u > v) -> both directions, sorted by (u, v), into out[0 ..): the
// rows [row_lo, row_lo + nrows) (all n rows by default).  rowptr_out, when
// given, receives the nrows + 1 row offsets (device); its last entry is the
// number of entries written.
template <class Id>
inline int assemble(const Id* pairs, const uint64_t* npairs_dev, uint64_t npairs_host, uint64_t n,
                    Id* out, uint64_t cap, Workspace& ws, cudaStream_t s, int* err,
                    uint64_t row_lo = 0, uint64_t nrows = ~uint64_t(0),
                    uint64_t** rowptr_out = nullptr, uint64_t work_bound = 0) {
  if (nrows == ~uint64_t(0)) nrows = n;
  unsigned long long* deg = ws.alloc<unsigned long long>(nrows);
  uint64_t* rowptr = ws.alloc<uint64_t>(nrows + 1);
  unsigned long long* cursor = ws.alloc<unsigned long long>(nrows);
  unsigned long long* long_rows = ws.alloc<unsigned long long>(nrows);
  unsigned long long* nlong = ws.alloc<unsigned long long>(1);
  if (!ws.ok()) return ST_CUDA;
  if (rowptr_out) *rowptr_out = rowptr;
  if (cudaMemsetAsync(deg, 0, nrows * 8, s) != cudaSuccess ||
      cudaMemsetAsync(nlong, 0, 8, s) != cudaSuccess)
    return ST_CUDA;
  const uint64_t work = work_bound ? work_bound : (npairs_dev ? cap / 2 : npairs_host);
  {
    ProfScope ps(PROF_ASSEMBLY, s);
    und_degree<Id><<<grid_for(work, 256, sm_count() * 16), 256, 0, s>>>(pairs, npairs_dev, npairs_host,
                                                                 row_lo, nrows, deg);
    if (launch_ok()) return ST_CUDA;
  }
  int st = scan_exclusive_u64(reinterpret_cast<const uint64_t*>(deg), rowptr, nrows, ws, s);
  if (st) return st;
  if (cudaMemcpyAsync(cursor, rowptr, nrows * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return ST_CUDA;
  {
    ProfScope ps(PROF_ASSEMBLY, s);
    und_scatter<Id><<<grid_for(work, 256, sm_count() * 16), 256, 0, s>>>(
        pairs, npairs_dev, npairs_host, row_lo, nrows, cursor, out, cap, err);
    if (launch_ok()) return ST_CUDA;
  }
  {
    ProfScope ps(PROF_ASSEMBLY, s);
    und_sort_short<Id><<<grid_for(nrows, 256, sm_count() * 32), 256, 0, s>>>(rowptr, nrows, out, cap,
                                                                    long_rows, nlong);
    if (launch_ok()) return ST_CUDA;
  }
  ProfScope ps(PROF_ASSEMBLY, s);
  und_sort_long<Id><<<sm_count() * 2, 256, 0, s>>>(rowptr, out, cap, long_rows, nlong);
  return launch_ok();
}

}  // namespace kg
