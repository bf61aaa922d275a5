// Launch accounting / per-kernel-class event timing (see kg_prof.cu).
#pragma once
#include <cuda_runtime.h>

#define KG_PROF_CLASSES 9

namespace kg {
enum ProfClass : int {
  PROF_CHUNK_TREE = 0,
  PROF_TILE_TREE = 1,
  PROF_SCAN = 2,
  PROF_LEAF = 3,
  PROF_DIGEST = 4,
  PROF_GNP = 5,
  PROF_ASSEMBLY = 6,
  PROF_OTHER = 7,
  PROF_RGG = 8,
};

// Counts one launch; when profiling is on, brackets it with events on `s`.
class ProfScope {
 public:
  ProfScope(int cls, cudaStream_t s);
  ~ProfScope();

 private:
  int cls_;
  cudaStream_t s_;
  void* a_;
};
}  // namespace kg
