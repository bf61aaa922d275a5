// Internal interface of the batched engine for the serving loop: a group of
// instances laid out on the host and run in device memory the caller owns
// (no allocation, no host synchronisation), with one order-independent
// digest per instance.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace kg {

// One instance: G(n,m) (binom = 0), or G(n,p) by binomial chunk counts
// (binom = 1, m = its exact sample count from kg_gnp_binomial_count).
struct BatchSpec {
  uint64_t n, m, seed;
  double p;
  uint32_t chunks;
  int undirected;
  int binom;
};

struct BatchGroup;

// Lays out `count` instances (uint32 ids).  *dev_bytes: device memory the
// group needs; *table_bytes: pinned host memory for its instance table.
int batch_group_prepare(const BatchSpec* specs, uint32_t count, BatchGroup** out,
                        size_t* dev_bytes, size_t* table_bytes);
// Enqueues the group on s: the instance table (staged in h_table, which must
// stay valid until s has passed this point), the generation into out
// (instance i at entries [batch_group_offset(i), batch_group_offset(i+1))),
// and the digests of the instances into the group's device array.
int batch_group_launch(BatchGroup* g, void* dev_mem, size_t dev_bytes, void* h_table,
                       uint32_t* out, uint64_t cap, cudaStream_t s);
uint64_t batch_group_offset(const BatchGroup* g, uint32_t i);
// device array of the group's count digests (valid after batch_group_launch)
const uint64_t* batch_group_digests(const BatchGroup* g);
void batch_group_free(BatchGroup* g);

// Validation of a G(n,p)-by-binomial-counts instance, as kg_gnp_binomial
// does it (ST_OK or the status it would return).
int gnpb_check(int undirected, uint64_t n, double p, uint32_t chunks, int id_bytes);

// Entry counts of `count` G(n,p)-by-binomial-counts instances (device array
// of GnpbSizeReq in, device sizes out), one kernel for all: each equals what
// kg_gnp_binomial_count writes for the same instance.
struct GnpbSizeReq {
  uint64_t n, seed;
  double p;
  uint32_t chunks;
  int undirected;
};
int gnpb_size_many(const GnpbSizeReq* d_reqs, uint32_t count, uint64_t* d_sizes, cudaStream_t s);

}  // namespace kg
