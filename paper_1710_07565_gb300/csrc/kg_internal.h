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
  ~Workspace() {
    for (void* p : ptrs_) cudaFreeAsync(p, s_);
  }
  template <class T>
  T* alloc(uint64_t count) {
    const size_t bytes = size_t(count ? count : 1) * sizeof(T);
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

 private:
  cudaStream_t s_;
  std::vector<void*> ptrs_;
  bool ok_ = true;
  unsigned char* arena_ = nullptr;
  size_t arena_bytes_ = 0, arena_used_ = 0;
};

// Exclusive scan of n u64 values: out[i] = sum in[0..i), out[n] = total.
int scan_exclusive_u64(const uint64_t* in, uint64_t* out, uint64_t n, Workspace& ws,
                       cudaStream_t s);

// Device error word of the current device (allocated on first use).
int* device_error_word();

}  // namespace kg
