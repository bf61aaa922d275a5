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
// Bucket shape of the bucketed assembly: bsh such that a bucket of 2^bsh rows
// holds about ASM_TARGET of the `entries` expected entries; false (the
// window then takes the atomic-per-entry path) if that takes more than
// ASM_NB_MAX buckets (larger buckets would overflow shared memory) or where
// that path is faster.
inline bool asm_shape(uint64_t nrows, uint64_t entries, int& bsh, uint32_t& nb) {
  const double avg = nrows ? double(entries) / double(nrows) : 0.0;
  bsh = 0;
  while ((1u << (bsh + 1)) <= ASM_BR_MAX && double(1u << (bsh + 1)) * avg <= double(ASM_TARGET))
    ++bsh;
  // too many buckets for the histogram: wider buckets while they expect at
  // most three quarters of what shared memory holds (a window of 2^24 rows at
  // 2.02 entries per row takes 2^14 buckets of 2^10 rows, ~2070 entries each)
  while (((nrows + (uint64_t(1) << bsh) - 1) >> bsh) > ASM_NB_MAX &&
         (1u << (bsh + 1)) <= ASM_BR_MAX &&
         double(1u << (bsh + 1)) * avg <= 0.75 * double(ASM_CAP))
    ++bsh;
  const uint64_t b = (nrows + (uint64_t(1) << bsh) - 1) >> bsh;
  nb = uint32_t(b < ASM_NB_MAX ? b : ASM_NB_MAX);
  // measured on GB300: the buckets win on windows of 2^22 rows and more and
  // on sparse rows (at most 4 entries on average); on smaller windows of
  // longer rows the atomic-per-entry counts stay in L2 and that path is
  // faster (n = 2^20 at 16 entries per row: 1.97 vs 2.37 ms)
  if (nrows < (uint64_t(1) << 22) && avg > 4.0) return false;
  return b <= ASM_NB_MAX && b > 0;
}

// Scratch of one assembly, carved in one place before any launch (so that a
// measuring Workspace gives its exact bytes).  buckets: the bucketed path
// (bsh, nb from asm_shape), else the atomic-per-entry path.
struct AsmScratch {
  bool buckets = false;
  int bsh = 0;
  uint32_t nb = 0;
  uint64_t* rowptr = nullptr;  // nrows + 1 row offsets (both paths)
  // bucketed path
  unsigned long long *bcnt = nullptr, *big = nullptr, *nbig = nullptr;
  uint32_t* blk = nullptr;  // G rows of nb per-block bucket counts, then offsets
  uint64_t* keys = nullptr;  // the scattered entries as 8-byte keys (asm_key), kcap of them
  uint64_t kcap = 0;
  uint32_t G = 0;           // blocks of the count and scatter kernels
  uint64_t* boff = nullptr;
  // atomic path
  unsigned long long *deg = nullptr, *cursor = nullptr, *long_rows = nullptr, *nlong = nullptr;
  ScanScratch scan;

  // nrows rows of the window; expect: the entries expected in it
  bool carve(uint64_t nrows, uint64_t expect, Workspace& ws) {
    buckets = nrows > 0 && asm_shape(nrows, expect, bsh, nb);
    rowptr = ws.alloc<uint64_t>(nrows + 1);
    if (buckets) {
      G = uint32_t(sm_count() * ASM_HIST_BLOCKS);
      bcnt = ws.alloc<unsigned long long>(nb);
      boff = ws.alloc<uint64_t>(uint64_t(nb) + 1);
      blk = ws.alloc<uint32_t>(uint64_t(G) * nb);
      kcap = expect;
      keys = ws.alloc<uint64_t>(kcap ? kcap : 1);
      big = ws.alloc<unsigned long long>(nb);
      nbig = ws.alloc<unsigned long long>(1);
      if (!scan_scratch(nb, ws, scan)) return false;
    } else {
      deg = ws.alloc<unsigned long long>(nrows);
      cursor = ws.alloc<unsigned long long>(nrows);
      long_rows = ws.alloc<unsigned long long>(nrows);
      nlong = ws.alloc<unsigned long long>(1);
      if (!scan_scratch(nrows, ws, scan)) return false;
    }
    return ws.ok();
  }
};

// Expected entries of an assembly window: the pairs' entries (both
// directions), or the output's capacity when the pair count is only known on
// the device.
inline uint64_t asm_expect(const void* npairs_dev, uint64_t npairs_host, uint64_t cap) {
  const uint64_t e = npairs_dev ? cap : 2 * npairs_host;
  return e < cap ? e : cap;
}

// Bytes of scratch assemble() takes for a window of nrows rows (measured).
inline uint64_t assemble_scratch_bytes(uint64_t nrows, uint64_t expect) {
  Workspace meas = Workspace::measuring();
  AsmScratch sc;
  if (!sc.carve(nrows, expect, meas)) return ~uint64_t(0);
  return meas.used();
}

template <class Id>
inline int assemble_buckets(const Id* pairs, const uint64_t* npairs_dev, uint64_t npairs_host,
                            Id* out, uint64_t cap, const AsmScratch& sc, cudaStream_t s, int* err,
                            uint64_t row_lo, uint64_t nrows, const AsmDigest& dig) {
  const int bsh = sc.bsh;
  const uint32_t nb = sc.nb;
  if (cudaMemsetAsync(sc.nbig, 0, 8, s) != cudaSuccess) return ST_CUDA;
  const size_t hsm = size_t(nb) * 4;
  const unsigned G = sc.G;  // the count and scatter kernels split the pairs alike
  static_assert(size_t(ASM_NB_MAX) * 4 <= 64 * 1024, "histogram in shared memory");
  if (cudaFuncSetAttribute(asm_bucket_count<Id>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           int(ASM_NB_MAX * 4)) != cudaSuccess ||
      cudaFuncSetAttribute(asm_bucket_scatter<Id>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           int(ASM_NB_MAX * 4)) != cudaSuccess ||
      cudaFuncSetAttribute(asm_bucket_sort<Id>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           int(sizeof(AsmSmem))) != cudaSuccess)
    return ST_CUDA;
  {
    ProfScope ps(PROF_ASSEMBLY, s);
    asm_bucket_count<Id><<<G, ASM_THREADS, hsm, s>>>(pairs, npairs_dev, npairs_host, row_lo, nrows,
                                                     bsh, nb, sc.blk);
    if (launch_ok()) return ST_CUDA;
  }
  {
    ProfScope ps(PROF_ASSEMBLY, s);
    asm_bucket_colscan<<<(nb + 63) / 64, 64, 0, s>>>(sc.blk, G, nb, sc.bcnt);
    if (launch_ok()) return ST_CUDA;
  }
  int st = scan_exclusive_u64(reinterpret_cast<const uint64_t*>(sc.bcnt), sc.boff, nb, sc.scan, s);
  if (st) return st;
  {
    ProfScope ps(PROF_ASSEMBLY, s);
    asm_bucket_scatter<Id><<<G, ASM_THREADS, hsm, s>>>(pairs, npairs_dev, npairs_host, row_lo,
                                                       nrows, bsh, nb, sc.boff, sc.blk, sc.keys,
                                                       sc.kcap, err);
    if (launch_ok()) return ST_CUDA;
  }
  {
    ProfScope ps(PROF_ASSEMBLY, s);
    asm_bucket_sort<Id><<<grid_for(nb, 1, sm_count() * 4), ASM_THREADS, sizeof(AsmSmem), s>>>(
        out, sc.keys, sc.boff, row_lo, nrows, bsh, nb, cap, sc.rowptr, sc.big, sc.nbig, dig);
    if (launch_ok()) return ST_CUDA;
  }
  {
    ProfScope ps(PROF_ASSEMBLY, s);
    asm_bucket_sort_global<Id><<<sm_count(), ASM_THREADS, 0, s>>>(
        out, sc.keys, sc.boff, row_lo, nrows, bsh, sc.rowptr, sc.big, sc.nbig, dig);
    if (launch_ok()) return ST_CUDA;
  }
  // the window's last offset: its entry count
  if (cudaMemcpyAsync(sc.rowptr + nrows, sc.boff + nb, 8, cudaMemcpyDeviceToDevice, s) !=
      cudaSuccess)
    return ST_CUDA;
  return ST_OK;
}

template <class Id>
inline int assemble(const Id* pairs, const uint64_t* npairs_dev, uint64_t npairs_host, uint64_t n,
                    Id* out, uint64_t cap, Workspace& ws, cudaStream_t s, int* err,
                    uint64_t row_lo = 0, uint64_t nrows = ~uint64_t(0),
                    uint64_t** rowptr_out = nullptr, uint64_t work_bound = 0,
                    const AsmDigest* dig = nullptr, bool* digested = nullptr) {
  if (nrows == ~uint64_t(0)) nrows = n;
  AsmScratch sc;
  if (!sc.carve(nrows, asm_expect(npairs_dev, npairs_host, cap), ws)) return ST_CUDA;
  if (rowptr_out) *rowptr_out = sc.rowptr;
  if (digested) *digested = false;
  if (sc.buckets) {
    // the bucketed path also makes the window's per-row-block digests and
    // degree histograms (zeroed by the caller) while the entries are on chip
    AsmDigest none{};
    const AsmDigest& dd = dig ? *dig : none;
    if (digested) *digested = dig != nullptr;
    return assemble_buckets<Id>(pairs, npairs_dev, npairs_host, out, cap, sc, s, err, row_lo, nrows,
                                dd);
  }
  uint64_t* rowptr = sc.rowptr;
  unsigned long long *deg = sc.deg, *cursor = sc.cursor, *long_rows = sc.long_rows,
                     *nlong = sc.nlong;
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
  int st = scan_exclusive_u64(reinterpret_cast<const uint64_t*>(deg), rowptr, nrows, sc.scan, s);
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
