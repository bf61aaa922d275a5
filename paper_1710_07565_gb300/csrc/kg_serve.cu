// Serving: a continuous-batching request loop over the generators.
//
// Requests (G(n,m) or G(n,p), directed or undirected) are admitted in arrival
// order when their exact output size fits in a fixed device budget; the size
// of a G(n,m) request is m or 2m entries, that of a G(n,p) request is counted
// first on the device (kg_gnp_count: the same skip walks without storing
// them; kg_gnp_binomial_count: the chunk binomials of Sec. 4.3).
// Admitted requests run on a set of streams, so requests that arrive while
// others are on the GPU overlap with them.  Small G(n,m) and binomial G(n,p)
// requests (uint32 ids, at most 2^22 entries, chunk counts the batched engine
// takes) that are admitted together go to the GPU as one group: one batched
// launch sequence for all of them (the batched engine over a scratch arena
// the server owns), with one digest per request; larger requests run alone
// through their entry points.  A request's output is reduced on the device
// to its order-independent digest, copied to host memory, and its budget
// released -- which admits the next waiting requests.  The state of every
// request stays on the device until its digest is read.
#include <algorithm>
#include <chrono>
#include <deque>
#include <map>
#include <unordered_map>
#include <vector>

#include "kg.h"
#include "kg_batch.h"
#include "kg_internal.h"

namespace {

constexpr uint32_t MAX_INFLIGHT = 4096;
constexpr uint32_t GROUP_MAX = 1024;                    // requests per group
constexpr uint64_t GROUP_ENTRIES_MAX = uint64_t(1) << 24;  // entries of a grouped request
constexpr uint64_t STAGE_BYTES = uint64_t(64) << 20;    // pinned staging of the groups

enum ReqState { SIZING, WAITING, RUNNING };

struct Req {
  kg_request q;
  uint64_t id = 0, entries = 0, bytes = 0, off = 0;
  ReqState state = WAITING;
  int stream = 0;
  uint32_t slot = 0;
  cudaEvent_t ev = nullptr;
  double t_submit = 0, t_admit = 0;
  int64_t group = -1;   // the group it runs in, or -1 (alone)
  bool solo = false;    // not batchable (set after a failed group layout)
  bool failed = false;  // its size pass failed: finishes with KG_ERR_CUDA
};

// First-fit allocator over [0, size) in 256-byte units, coalescing on release.
struct FreeList {
  std::map<uint64_t, uint64_t> free_;  // offset -> size
  uint64_t in_use = 0;
  void init(uint64_t size) { free_[0] = size & ~uint64_t(255); }
  bool alloc(uint64_t bytes, uint64_t& off) {
    bytes = (bytes + 255) & ~uint64_t(255);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        off = it->first;
        const uint64_t rest = it->second - bytes;
        free_.erase(it);
        if (rest) free_[off + bytes] = rest;
        in_use += bytes;
        return true;
      }
    }
    return false;
  }
  void release(uint64_t off, uint64_t bytes) {
    bytes = (bytes + 255) & ~uint64_t(255);
    in_use -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

// Requests generated together by the batched engine.
struct Group {
  std::vector<uint64_t> ids;
  uint64_t out_off = 0, out_bytes = 0;  // one output block in the budget
  uint64_t ar_off = 0, ar_bytes = 0;    // scratch in the arena
  uint64_t pin_off = 0, pin_bytes = 0;  // pinned staging: instance table, then digests
  uint64_t tab_bytes = 0;
  cudaEvent_t ev = nullptr;
  kg::BatchGroup* plan = nullptr;
  bool failed = false;  // the launch failed: its requests finish with KG_ERR_CUDA
  size_t reported = 0;  // results already handed out (a poll may take part of a group)
};

}  // namespace

struct kg_server {
  int device = 0;
  unsigned char* pool = nullptr;
  uint64_t budget = 0, in_use = 0;
  std::map<uint64_t, uint64_t> free_;  // offset -> size, coalesced
  // the groups' scratch (device) and staging (pinned host)
  unsigned char* arena = nullptr;
  uint64_t arena_bytes = 0;
  unsigned char* stage = nullptr;
  FreeList arena_free, stage_free;
  std::unordered_map<int64_t, Group> groups;
  int64_t next_group = 0;
  // binomial G(n,p) requests waiting for their size pass, and size passes in
  // flight (one kernel for many requests)
  std::deque<uint64_t> to_size;
  struct SizeBatch {
    std::vector<uint64_t> ids;
    uint64_t ar_off = 0, ar_bytes = 0, pin_off = 0, pin_bytes = 0, sizes_at = 0;
    cudaEvent_t ev = nullptr;
  };
  std::vector<SizeBatch> sizing;
  std::vector<cudaStream_t> streams;
  uint32_t next_stream = 0;
  uint64_t next_id = 0;
  std::deque<uint64_t> waiting;        // admission order
  std::unordered_map<uint64_t, Req> reqs;
  uint64_t* d_slots = nullptr;         // per in-flight request: count, digest
  uint64_t* h_slots = nullptr;         // pinned mirrors
  std::vector<uint32_t> free_slots;
  std::vector<cudaEvent_t> free_events;
  std::chrono::steady_clock::time_point t0;

  double now_ms() const {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  bool alloc(uint64_t bytes, uint64_t& off) {
    bytes = (bytes + 255) & ~uint64_t(255);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        off = it->first;
        const uint64_t rest = it->second - bytes;
        free_.erase(it);
        if (rest) free_[off + bytes] = rest;
        in_use += bytes;
        return true;
      }
    }
    return false;
  }
  void release(uint64_t off, uint64_t bytes) {
    bytes = (bytes + 255) & ~uint64_t(255);
    in_use -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  cudaEvent_t event() {
    if (!free_events.empty()) {
      cudaEvent_t e = free_events.back();
      free_events.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    return e;
  }
  cudaStream_t pick_stream(int& idx) {
    idx = int(next_stream++ % streams.size());
    return streams[idx];
  }
};

static uint64_t req_bytes(const kg_request& q, uint64_t entries) {
  return entries * 2 * uint64_t(q.id_bytes);
}

// Launch the generator, then the digest of its output, then the digest's copy.
static kg_status launch(kg_server* S, Req& r) {
  const kg_request& q = r.q;
  cudaStream_t s = S->pick_stream(r.stream);
  void* out = S->pool + r.off;
  kg_status st;
  if (q.model == 0) {
    st = q.undirected ? kg_gnm_undirected(q.n, q.m, q.seed, q.chunks, q.id_bytes, out, r.entries, s)
                      : kg_gnm_directed(q.n, q.m, q.seed, q.chunks, q.id_bytes, out, r.entries, s);
  } else if (q.model == 1) {
    st = kg_gnp_ex(q.undirected, q.n, q.p, q.seed, q.chunks, 1024, q.id_bytes, out, r.entries,
                   S->d_slots + 2 * r.slot, s);
  } else {
    st = kg_gnp_binomial(q.undirected, q.n, q.p, q.seed, q.chunks, q.id_bytes, out, r.entries,
                         S->d_slots + 2 * r.slot, s);
  }
  if (st != KG_OK) return st;
  st = kg_edge_digest(out, r.entries, q.id_bytes, S->d_slots + 2 * r.slot + 1, s);
  if (st != KG_OK) return st;
  if (cudaMemcpyAsync(S->h_slots + 2 * r.slot + 1, S->d_slots + 2 * r.slot + 1, 8,
                      cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return KG_ERR_CUDA;
  r.ev = S->event();
  if (cudaEventRecord(r.ev, s) != cudaSuccess) return KG_ERR_CUDA;
  return KG_OK;
}

static void finish(kg_server* S, Req& r, kg_status st, kg_result* out) {
  out->id = r.id;
  out->entries = r.entries;
  out->digest = (st == KG_OK) ? S->h_slots[2 * r.slot + 1] : 0;
  out->t_submit_ms = r.t_submit;
  out->t_admit_ms = r.t_admit;
  out->t_done_ms = S->now_ms();
  out->status = st;
  out->pad = 0;
  if (r.state == RUNNING && r.group < 0) S->release(r.off, r.bytes);
  if (r.ev) S->free_events.push_back(r.ev);
  S->free_slots.push_back(r.slot);
}

// Whether a waiting request may join a group: the batched engine's instance
// limits (uint32 ids, chunks <= 64 directed / 32 undirected), G(n,m) or
// binomial G(n,p), at most 2^24 entries (the large ones fill the GPU alone),
// undirected at most 2^20 vertices (the group's per-vertex assembly arrays).
static bool batchable(const Req& r) {
  const kg_request& q = r.q;
  if (r.solo || q.id_bytes != 4 || (q.model != 0 && q.model != 2)) return false;
  if (q.n == 0 || q.n > (uint64_t(1) << 32) || q.chunks == 0 || q.chunks > q.n) return false;
  if (q.chunks > (q.undirected ? 32u : 64u)) return false;
  if (r.entries > GROUP_ENTRIES_MAX) return false;
  // undirected instances carry per-vertex assembly arrays in the group's scratch
  if (q.undirected && q.n > (uint64_t(1) << 20)) return false;
  return true;
}

static void release_group(kg_server* S, Group& g) {
  if (g.out_bytes) S->release(g.out_off, g.out_bytes);
  if (g.ar_bytes) S->arena_free.release(g.ar_off, g.ar_bytes);
  if (g.pin_bytes) S->stage_free.release(g.pin_off, g.pin_bytes);
  if (g.ev) S->free_events.push_back(g.ev);
  if (g.plan) kg::batch_group_free(g.plan);
  g = Group();
}

// Lays out the requests `ids` as one group and, if its output, scratch and
// staging fit, launches it.  Returns 1 when launched, 0 when something did
// not fit now or a group of several was refused (nothing is kept; the caller
// tries fewer), -1 when a single request cannot be grouped at all (refused by
// the layout, or larger than the whole scratch arena or staging area): it is
// then marked to run alone.
static int try_group(kg_server* S, const std::vector<uint64_t>& ids) {
  auto refuse = [&]() {
    if (ids.size() > 1) return 0;
    S->reqs[ids[0]].solo = true;
    return -1;
  };
  std::vector<kg::BatchSpec> specs;
  specs.reserve(ids.size());
  uint64_t entries = 0;
  for (uint64_t id : ids) {
    const Req& r = S->reqs[id];
    const kg_request& q = r.q;
    const uint64_t pairs = q.undirected ? r.entries / 2 : r.entries;
    specs.push_back(kg::BatchSpec{q.n, pairs, q.seed, q.model == 2 ? q.p : 0.0, q.chunks,
                                  q.undirected ? 1 : 0, q.model == 2 ? 1 : 0});
    entries += r.entries;
  }
  Group g;
  size_t dev_bytes = 0, tab_bytes = 0;
  if (kg::batch_group_prepare(specs.data(), uint32_t(specs.size()), &g.plan, &dev_bytes,
                              &tab_bytes) != kg::ST_OK) {
    g.plan = nullptr;
    return refuse();
  }
  g.out_bytes = entries ? entries * 8 : 256;
  g.ar_bytes = dev_bytes;
  g.tab_bytes = (tab_bytes + 255) & ~uint64_t(255);
  g.pin_bytes = g.tab_bytes + 8 * ids.size();
  if (g.ar_bytes > S->arena_bytes || g.pin_bytes > STAGE_BYTES) {
    kg::batch_group_free(g.plan);
    return refuse();
  }
  // each block is taken only if the previous ones were; on a miss the group
  // keeps exactly the blocks it holds, so that release_group returns those only
  const bool got_out = S->alloc(g.out_bytes, g.out_off);
  const bool got_ar = got_out && S->arena_free.alloc(g.ar_bytes, g.ar_off);
  const bool got_pin = got_ar && S->stage_free.alloc(g.pin_bytes, g.pin_off);
  if (!got_pin) {
    if (!got_out) g.out_bytes = 0;
    if (!got_ar) g.ar_bytes = 0;
    g.pin_bytes = 0;
    release_group(S, g);
    return 0;
  }
  int si = 0;
  cudaStream_t s = S->pick_stream(si);
  unsigned char* pin = S->stage + g.pin_off;
  uint32_t* out = reinterpret_cast<uint32_t*>(S->pool + g.out_off);
  int st = kg::batch_group_launch(g.plan, S->arena + g.ar_off, g.ar_bytes, pin, out, entries, s);
  if (st == kg::ST_OK &&
      cudaMemcpyAsync(pin + g.tab_bytes, kg::batch_group_digests(g.plan), 8 * ids.size(),
                      cudaMemcpyDeviceToHost, s) != cudaSuccess)
    st = kg::ST_CUDA;
  g.ev = S->event();
  if (st == kg::ST_OK && cudaEventRecord(g.ev, s) != cudaSuccess) st = kg::ST_CUDA;
  const int64_t gid = S->next_group++;
  const double now = S->now_ms();
  for (uint64_t id : ids) {
    Req& r = S->reqs[id];
    r.state = RUNNING;
    r.group = gid;
    r.t_admit = now;
    r.stream = si;
  }
  g.ids = ids;
  if (st != kg::ST_OK) {
    // the launch failed: the group finishes with the error once its stream has
    // passed what was enqueued
    g.failed = true;
    cudaStreamSynchronize(s);
  }
  S->groups.emplace(gid, std::move(g));
  return 1;
}

// Launches the collected requests `grp` (admitted in this order) as groups:
// the largest prefix whose output and scratch fit (halving), again for the
// rest; what does not fit now goes back to the front of the queue in order,
// a request the layout refuses goes back marked to run alone.  Returns false
// if requests went back for lack of space.
static bool flush_group(kg_server* S, std::vector<uint64_t>& grp) {
  size_t at = 0;
  bool all = true;
  while (at < grp.size()) {
    std::vector<uint64_t> cand(grp.begin() + at, grp.end());
    int got = 0;
    while (!cand.empty()) {
      got = try_group(S, cand);
      if (got != 0) break;
      cand.resize(cand.size() / 2);
    }
    if (got == 1) {
      at += cand.size();
      continue;
    }
    // nothing fits now, or a single request refused (marked solo): the rest
    // waits at the front of the queue, in order
    for (size_t i = grp.size(); i > at; --i) S->waiting.push_front(grp[i - 1]);
    all = got < 0;
    break;
  }
  grp.clear();
  return all;
}

// One size pass for the binomial G(n,p) requests waiting for it (up to
// SIZE_MAX_BATCH): their parameters staged in pinned memory, one kernel, the
// sizes copied back, one event.
constexpr uint32_t SIZE_MAX_BATCH = 4096;

static void launch_sizing(kg_server* S) {
  while (!S->to_size.empty()) {
    const uint32_t cnt = uint32_t(std::min<size_t>(S->to_size.size(), SIZE_MAX_BATCH));
    kg_server::SizeBatch b;
    const uint64_t par = ((sizeof(kg::GnpbSizeReq) * cnt) + 255) & ~uint64_t(255);
    b.sizes_at = par;
    b.ar_bytes = b.pin_bytes = par + 8 * uint64_t(cnt);
    if (!S->arena_free.alloc(b.ar_bytes, b.ar_off)) return;
    if (!S->stage_free.alloc(b.pin_bytes, b.pin_off)) {
      S->arena_free.release(b.ar_off, b.ar_bytes);
      return;
    }
    kg::GnpbSizeReq* hp = reinterpret_cast<kg::GnpbSizeReq*>(S->stage + b.pin_off);
    for (uint32_t i = 0; i < cnt; ++i) {
      const uint64_t id = S->to_size.front();
      S->to_size.pop_front();
      const kg_request& q = S->reqs[id].q;
      hp[i] = kg::GnpbSizeReq{q.n, q.seed, q.p, q.chunks, q.undirected ? 1 : 0};
      b.ids.push_back(id);
    }
    int si = 0;
    cudaStream_t s = S->pick_stream(si);
    unsigned char* dev = S->arena + b.ar_off;
    bool ok = cudaMemcpyAsync(dev, hp, sizeof(kg::GnpbSizeReq) * cnt, cudaMemcpyHostToDevice, s) ==
              cudaSuccess;
    ok = ok && kg::gnpb_size_many(reinterpret_cast<const kg::GnpbSizeReq*>(dev), cnt,
                                  reinterpret_cast<uint64_t*>(dev + b.sizes_at), s) == kg::ST_OK;
    ok = ok && cudaMemcpyAsync(S->stage + b.pin_off + b.sizes_at, dev + b.sizes_at, 8 * cnt,
                               cudaMemcpyDeviceToHost, s) == cudaSuccess;
    b.ev = S->event();
    ok = ok && cudaEventRecord(b.ev, s) == cudaSuccess;
    if (!ok) {
      // sizes unknown: these requests finish with an error at the next poll
      cudaStreamSynchronize(s);
      uint64_t* hs = reinterpret_cast<uint64_t*>(S->stage + b.pin_off + b.sizes_at);
      for (uint32_t i = 0; i < cnt; ++i) hs[i] = ~uint64_t(0);
    }
    S->sizing.push_back(std::move(b));
  }
}

extern "C" {

kg_status kg_server_create(uint64_t budget_bytes, uint32_t nstreams, kg_server** out) {
  if (!out || budget_bytes == 0 || nstreams == 0 || nstreams > 64) return KG_ERR_ARG;
  *out = nullptr;
  kg_server* S = new kg_server();
  S->t0 = std::chrono::steady_clock::now();
  if (cudaGetDevice(&S->device) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&S->pool), budget_bytes) != cudaSuccess) {
    delete S;
    return KG_ERR_CUDA;
  }
  S->budget = budget_bytes;
  S->free_[0] = budget_bytes & ~uint64_t(255);
  // scratch for the groups: an eighth of the budget, between 256 MB and 4 GB
  uint64_t ab = budget_bytes / 8;
  if (ab < (uint64_t(256) << 20)) ab = uint64_t(256) << 20;
  if (ab > (uint64_t(4) << 30)) ab = uint64_t(4) << 30;
  if (cudaMalloc(reinterpret_cast<void**>(&S->arena), ab) != cudaSuccess ||
      cudaMallocHost(reinterpret_cast<void**>(&S->stage), STAGE_BYTES) != cudaSuccess) {
    kg_server_destroy(S);
    return KG_ERR_CUDA;
  }
  S->arena_bytes = ab;
  S->arena_free.init(ab);
  S->stage_free.init(STAGE_BYTES);
  if (cudaMalloc(reinterpret_cast<void**>(&S->d_slots), 16 * MAX_INFLIGHT) != cudaSuccess ||
      cudaMallocHost(reinterpret_cast<void**>(&S->h_slots), 16 * MAX_INFLIGHT) != cudaSuccess) {
    kg_server_destroy(S);
    return KG_ERR_CUDA;
  }
  for (uint32_t i = 0; i < MAX_INFLIGHT; ++i) S->free_slots.push_back(MAX_INFLIGHT - 1 - i);
  for (uint32_t i = 0; i < nstreams; ++i) {
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      kg_server_destroy(S);
      return KG_ERR_CUDA;
    }
    S->streams.push_back(s);
  }
  *out = S;
  return KG_OK;
}

kg_status kg_server_destroy(kg_server* S) {
  if (!S) return KG_OK;
  for (cudaStream_t s : S->streams) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  for (auto& kv : S->reqs)
    if (kv.second.ev) cudaEventDestroy(kv.second.ev);
  for (auto& b : S->sizing)
    if (b.ev) cudaEventDestroy(b.ev);
  for (auto& kv : S->groups) {
    if (kv.second.ev) cudaEventDestroy(kv.second.ev);
    if (kv.second.plan) kg::batch_group_free(kv.second.plan);
  }
  for (cudaEvent_t e : S->free_events) cudaEventDestroy(e);
  if (S->pool) cudaFree(S->pool);
  if (S->arena) cudaFree(S->arena);
  if (S->stage) cudaFreeHost(S->stage);
  if (S->d_slots) cudaFree(S->d_slots);
  if (S->h_slots) cudaFreeHost(S->h_slots);
  delete S;
  return KG_OK;
}

kg_status kg_server_submit(kg_server* S, const kg_request* q, uint64_t* id_out) {
  if (!S || !q || (q->model < 0 || q->model > 2) || (q->id_bytes != 4 && q->id_bytes != 8))
    return KG_ERR_ARG;
  if (S->free_slots.empty()) return KG_ERR_CAPACITY;
  Req r;
  r.q = *q;
  r.id = S->next_id++;
  r.t_submit = S->now_ms();
  r.slot = S->free_slots.back();
  S->free_slots.pop_back();
  if (q->model == 0) {
    r.entries = q->undirected ? 2 * q->m : q->m;
    r.state = WAITING;
    S->waiting.push_back(r.id);
  } else if (q->model == 2) {
    // exact size first: binomial requests are sized together at the next poll
    const int st = kg::gnpb_check(q->undirected, q->n, q->p, q->chunks, q->id_bytes);
    if (st != kg::ST_OK) {
      S->free_slots.push_back(r.slot);
      return kg_status(st);
    }
    r.state = SIZING;
    S->to_size.push_back(r.id);
  } else {
    // exact size first: the count pass, its result copied to pinned memory
    cudaStream_t s = S->pick_stream(r.stream);
    kg_status st = kg_gnp_count(q->undirected, q->n, q->p, q->seed, q->chunks, 1024,
                                S->d_slots + 2 * r.slot, s);
    if (st == KG_OK &&
        cudaMemcpyAsync(S->h_slots + 2 * r.slot, S->d_slots + 2 * r.slot, 8, cudaMemcpyDeviceToHost,
                        s) != cudaSuccess)
      st = KG_ERR_CUDA;
    if (st != KG_OK) {
      S->free_slots.push_back(r.slot);
      return st;
    }
    r.ev = S->event();
    cudaEventRecord(r.ev, s);
    r.state = SIZING;
  }
  if (id_out) *id_out = r.id;
  S->reqs.emplace(r.id, r);
  return KG_OK;
}

// One scheduling pass: sized G(n,p) requests join the queue, waiting requests
// are admitted in order while their bytes fit, finished requests are reported.
kg_status kg_server_poll(kg_server* S, kg_result* out, uint32_t max_out, uint32_t* n_out) {
  if (!S || !n_out || (max_out && !out)) return KG_ERR_ARG;
  *n_out = 0;
  launch_sizing(S);
  std::vector<uint64_t> sized;
  // size passes that finished: their requests join the queue (a request whose
  // size could not be computed finishes with an error)
  for (size_t bi = 0; bi < S->sizing.size();) {
    kg_server::SizeBatch& b = S->sizing[bi];
    if (cudaEventQuery(b.ev) == cudaErrorNotReady) {
      ++bi;
      continue;
    }
    const uint64_t* hs = reinterpret_cast<const uint64_t*>(S->stage + b.pin_off + b.sizes_at);
    for (size_t i = 0; i < b.ids.size(); ++i) {
      Req& r = S->reqs[b.ids[i]];
      r.failed = hs[i] == ~uint64_t(0);
      r.entries = r.failed ? 0 : hs[i];
      r.state = WAITING;
      sized.push_back(r.id);
    }
    S->arena_free.release(b.ar_off, b.ar_bytes);
    S->stage_free.release(b.pin_off, b.pin_bytes);
    S->free_events.push_back(b.ev);
    S->sizing.erase(S->sizing.begin() + bi);
  }
  for (auto& kv : S->reqs) {
    Req& r = kv.second;
    if (r.state == SIZING && r.ev && cudaEventQuery(r.ev) == cudaSuccess) {
      r.entries = S->h_slots[2 * r.slot];
      S->free_events.push_back(r.ev);
      r.ev = nullptr;
      r.state = WAITING;
      sized.push_back(r.id);
    }
  }
  std::sort(sized.begin(), sized.end());
  for (uint64_t id : sized) S->waiting.push_back(id);
  // admission (arrival order; a request larger than the whole budget is refused)
  std::vector<uint64_t> grp;
  while (!S->waiting.empty() && *n_out < max_out) {
    Req& r = S->reqs[S->waiting.front()];
    if (r.failed) {
      S->waiting.pop_front();
      r.state = WAITING;
      finish(S, r, KG_ERR_CUDA, out + (*n_out)++);
      S->reqs.erase(r.id);
      continue;
    }
    r.bytes = req_bytes(r.q, r.entries);
    if (r.bytes > S->budget) {
      S->waiting.pop_front();
      finish(S, r, KG_ERR_CAPACITY, out + (*n_out)++);
      S->reqs.erase(r.id);
      continue;
    }
    if (batchable(r)) {
      // the batchable requests of this pass collect into one group, launched
      // when it is full or when the pass ends
      S->waiting.pop_front();
      grp.push_back(r.id);
      if (grp.size() == GROUP_MAX && !flush_group(S, grp)) break;
      continue;
    }
    if (!S->alloc(r.bytes ? r.bytes : 256, r.off)) break;
    if (!r.bytes) r.bytes = 256;
    S->waiting.pop_front();
    r.t_admit = S->now_ms();
    r.state = RUNNING;
    const kg_status st = launch(S, r);
    if (st != KG_OK) {
      finish(S, r, st, out + (*n_out)++);
      S->reqs.erase(r.id);
    }
  }
  flush_group(S, grp);
  // completions: whole groups, then requests that ran alone
  std::vector<int64_t> gdone;
  for (auto& kv : S->groups)
    if (cudaEventQuery(kv.second.ev) != cudaErrorNotReady) gdone.push_back(kv.first);
  std::sort(gdone.begin(), gdone.end());
  for (int64_t gid : gdone) {
    Group& g = S->groups[gid];
    const bool ok = !g.failed && cudaEventQuery(g.ev) == cudaSuccess;
    const uint64_t* dig = reinterpret_cast<const uint64_t*>(S->stage + g.pin_off + g.tab_bytes);
    for (; g.reported < g.ids.size() && *n_out < max_out; ++g.reported) {
      Req& r = S->reqs[g.ids[g.reported]];
      kg_result* o = out + (*n_out)++;
      finish(S, r, ok ? KG_OK : KG_ERR_CUDA, o);
      o->digest = ok ? dig[g.reported] : 0;
      S->reqs.erase(g.ids[g.reported]);
    }
    if (g.reported < g.ids.size()) break;  // the rest at the next poll
    release_group(S, g);
    S->groups.erase(gid);
  }
  std::vector<uint64_t> done;
  for (auto& kv : S->reqs)
    if (kv.second.state == RUNNING && kv.second.group < 0 &&
        cudaEventQuery(kv.second.ev) == cudaSuccess)
      done.push_back(kv.first);
  std::sort(done.begin(), done.end());
  for (uint64_t id : done) {
    if (*n_out >= max_out) break;
    Req& r = S->reqs[id];
    finish(S, r, KG_OK, out + (*n_out)++);
    S->reqs.erase(id);
  }
  return KG_OK;
}

kg_status kg_server_pending(const kg_server* S, uint32_t* sizing, uint32_t* waiting,
                            uint32_t* running, uint64_t* bytes_in_use) {
  if (!S) return KG_ERR_ARG;
  uint32_t a = 0, b = 0, c = 0;
  for (const auto& kv : S->reqs) {
    if (kv.second.state == SIZING) ++a;
    if (kv.second.state == WAITING) ++b;
    if (kv.second.state == RUNNING) ++c;
  }
  if (sizing) *sizing = a;
  if (waiting) *waiting = b;
  if (running) *running = c;
  if (bytes_in_use) *bytes_in_use = S->in_use;
  return KG_OK;
}

}  // extern "C"
