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
  ~Workspace() {
    for (void* p : ptrs_) cudaFreeAsync(p, s_);
  }
  template <class T>
  T* alloc(uint64_t count) {
    void* p = nullptr;
    const size_t bytes = size_t(count ? count : 1) * sizeof(T);
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
};

// Exclusive scan of n u64 values: out[i] = sum in[0..i), out[n] = total.
int scan_exclusive_u64(const uint64_t* in, uint64_t* out, uint64_t n, Workspace& ws,
                       cudaStream_t s);

// Device error word of the current device (allocated on first use).
int* device_error_word();

}  // namespace kg
