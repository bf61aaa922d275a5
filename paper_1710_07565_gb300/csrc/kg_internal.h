// Host-side internals shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "kg_device.cuh"

namespace kg {

// Stream-ordered scratch: every allocation is released on the same stream
// when the workspace goes out of scope (cudaMallocAsync pool, no device sync).
class Workspace {
 public:
  explicit Workspace(cudaStream_t s) : s_(s) {}
  // Fixed-arena mode: carve 256-byte aligned pieces out of [arena, arena+bytes)
  // instead of allocating; nothing is freed.
  Workspace(cudaStream_t s, void* arena, size_t bytes)
      : s_(s), arena_(static_cast<unsigned char*>(arena)), arena_bytes_(bytes) {}
  // Measuring mode: every alloc returns nullptr and only adds the bytes the
  // fixed-arena mode would carve for it (used()); nothing may be launched
  // with its pointers.
  static Workspace measuring() {
    Workspace w(nullptr);
    w.measure_ = true;
    return w;
  }
  ~Workspace() {
    for (void* p : ptrs_) cudaFreeAsync(p, s_);
  }
  template <class T>
  T* alloc(uint64_t count) {
    const size_t bytes = size_t(count ? count : 1) * sizeof(T);
    if (measure_) {
      arena_used_ += (bytes + 255) & ~size_t(255);
      return nullptr;
    }
    if (arena_) {
      const size_t need = (bytes + 255) & ~size_t(255);
      if (arena_used_ + need > arena_bytes_) {
        ok_ = false;
        return nullptr;
      }
      T* p = reinterpret_cast<T*>(arena_ + arena_used_);
      arena_used_ += need;
      return p;
    }
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, s_) != cudaSuccess) {
      ok_ = false;
      return nullptr;
    }
    ptrs_.push_back(p);
    return static_cast<T*>(p);
  }
  bool ok() const { return ok_; }
  // bytes carved so far (fixed-arena and measuring modes)
  size_t used() const { return arena_used_; }

 private:
  cudaStream_t s_;
  std::vector<void*> ptrs_;
  bool ok_ = true;
  unsigned char* arena_ = nullptr;
  size_t arena_bytes_ = 0, arena_used_ = 0;
  bool measure_ = false;
};

// Exclusive scan of n u64 values: out[i] = sum in[0..i), out[n] = total.
int scan_exclusive_u64(const uint64_t* in, uint64_t* out, uint64_t n, Workspace& ws,
                       cudaStream_t s);

// The block partials of one scan of n values, carved before any launch (the
// same pieces, in the same order, that scan_exclusive_u64 takes).
struct ScanScratch {
  static constexpr int LEVELS = 8;
  uint64_t* part[LEVELS];
  uint64_t* carry[LEVELS];
  int levels = 0;
};
bool scan_scratch(uint64_t n, Workspace& ws, ScanScratch& sc);
int scan_exclusive_u64(const uint64_t* in, uint64_t* out, uint64_t n, const ScanScratch& sc,
                       cudaStream_t s);

// Device error word of the current device (allocated on first use).
int* device_error_word();

// Streaming multiprocessors of the current device (cached per device; 152 on
// a GB300 if the query fails), for grids sized in whole waves.
int sm_count();

}  // namespace kg
