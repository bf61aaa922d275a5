// G(n,m) kernels: chunk split tree (Sec. 4.1), tile tree inside the chunks
// (the divide-and-conquer recursion of Sec. 2.2 continued below the chunk),
// and the leaf kernel that samples each tile without replacement (Floyd),
// sorts it in shared memory and emits (u, v) pairs with coalesced stores.
#pragma once
#include "kg_common.cuh"
#include "kg_warp_variates.cuh"

namespace kg {

// ---------------------------------------------------------------- chunk tree
// Range [a, b) of heap node h at depth `level`; false if an ancestor is a leaf.
__device__ __forceinline__ bool chunk_range(uint32_t P, uint64_t h, int level, uint32_t& a,
                                            uint32_t& b) {
  a = 0;
  b = P;
  for (int bit = level - 1; bit >= 0; --bit) {
    if (b - a < 2) return false;
    const uint32_t s = a + (b - a + 1) / 2;
    if ((h >> bit) & 1)
      a = s;
    else
      b = s;
  }
  return true;
}

// Levels [l0, l1) of the directed chunk tree, one block per subtree rooted at
// level l0.  Node h with range [a,b) and count mc splits at s = a + ceil((b-a)/2)
// (l = ceil(P/2)) by X = Hyp(rows[a,b)(n-1), rows[a,s)(n-1), mc).
static __global__ void chunk_tree_band(RowBounds rb, uint64_t seed, uint64_t m, int l0, int l1,
                                uint64_t* __restrict__ node_cnt, uint64_t* __restrict__ cnt,
                                int* err) {
  const uint64_t n = rb.n;
  const uint32_t P = rb.P;
  const uint64_t root = (uint64_t(1) << l0) + blockIdx.x;
  if (l0 == 0 && threadIdx.x == 0) node_cnt[1] = m;
  __syncthreads();
  for (int r = 0; r < l1 - l0; ++r) {
    const int level = l0 + r;
    const uint64_t nodes = uint64_t(1) << r;
    for (uint64_t j = threadIdx.x; j < nodes; j += blockDim.x) {
      const uint64_t h = (root << r) + j;
      uint32_t a, b;
      if (!chunk_range(P, h, level, a, b)) continue;
      const uint64_t mc = node_cnt[h];
      if (b - a == 1) {
        cnt[a] = mc;
        continue;
      }
      const uint32_t s = a + (b - a + 1) / 2;
      const uint64_t ra = rb(a);
      const u128 N = u128(rb(b) - ra) * (n - 1);
      const u128 NL = u128(rb(s) - ra) * (n - 1);
      Stream st(seed, h, TAG_CHUNK_TREE);
      uint64_t X = 0;
      const int e = hypergeometric(N, NL, mc, st, X);
      if (e) {
        set_error(err, e);
        X = 0;
      }
      node_cnt[2 * h] = X;
      node_cnt[2 * h + 1] = mc - X;
    }
    __syncthreads();
  }
}

// Level `level` of the directed chunk tree with one warp per node (the top
// levels, whose few nodes make the tree's dependent FP64 chain): the same
// split and variate as chunk_tree_band, drawn by the whole warp.
static __global__ void __launch_bounds__(128)
    chunk_tree_level_warp(RowBounds rb, uint64_t seed, uint64_t m, int level,
                          uint64_t* __restrict__ node_cnt, uint64_t* __restrict__ cnt, int* err) {
  const uint64_t n = rb.n;
  const uint64_t nodes = uint64_t(1) << level;
  const unsigned lane = threadIdx.x & 31;
  const uint64_t nwarps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  for (uint64_t j = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; j < nodes;
       j += nwarps) {
    const uint64_t h = nodes + j;
    uint32_t a, b;
    if (!chunk_range(rb.P, h, level, a, b)) continue;
    const uint64_t mc = level == 0 ? m : node_cnt[h];
    if (b - a == 1) {
      if (lane == 0) cnt[a] = mc;
      continue;
    }
    const uint32_t s = a + (b - a + 1) / 2;
    const uint64_t ra = rb(a);
    const u128 N = u128(rb(b) - ra) * (n - 1);
    const u128 NL = u128(rb(s) - ra) * (n - 1);
    uint64_t X = 0;
    const int e = hypergeometric_warp(N, NL, mc, seed, h, TAG_CHUNK_TREE, X);
    if (lane == 0) {
      if (e) {
        set_error(err, e);
        X = 0;
      }
      node_cnt[2 * h] = X;
      node_cnt[2 * h + 1] = mc - X;
    }
  }
}

// ---------------------------------------------------------------- tile tree
constexpr uint64_t SMALL_FAIR_BITS = 4096;  // fair-bit counts up to this size stay on one lane
// levels of at most this many nodes draw one variate per warp
// (tile_tree_level_warp, chunk_tree_level_warp), larger ones one per lane
constexpr uint64_t WARP_TREE_NODES = 2048;

// One level of the tile trees with one warp per node: the node and its split
// as in tile_tree_level, the variate drawn by the whole warp.
template <class Geom>
__global__ void __launch_bounds__(128)
    tile_tree_level_warp(Geom g, uint64_t c_begin, uint64_t C, int d, int level, uint64_t seed,
                         const uint64_t* __restrict__ in, uint64_t* __restrict__ out, int* err) {
  const uint64_t total = C << level;
  const unsigned lane = threadIdx.x & 31;
  const uint64_t nwarps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  for (uint64_t node = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; node < total;
       node += nwarps) {
    const uint64_t c = node >> level;
    const uint64_t j = node & ((uint64_t(1) << level) - 1);
    const uint64_t cc = c_begin + c;
    const uint64_t U = g.universe(cc);
    const uint64_t W = tile_width(U, d);
    const uint64_t lo = node_bound(U, W, d, level, j);
    const uint64_t hi = node_bound(U, W, d, level, u128(j) + 1);
    const uint64_t mid = node_bound(U, W, d, level + 1, u128(2) * j + 1);
    const uint64_t k = in[node];
    const uint64_t sid = (g.chunk_id(cc) << 32) | ((uint64_t(1) << level) + j);
    uint64_t X = 0;
    const int st = (k > hi - lo) ? ST_INTERNAL
                                 : hypergeometric_warp(u128(hi - lo), u128(mid - lo), k, seed,
                                                       sid, TAG_TILE, X);
    if (lane == 0) {
      if (st) {
        set_error(err, st);
        X = 0;
      }
      out[2 * node] = X;
      out[2 * node + 1] = k - X;
    }
  }
}

// One level of the tile trees of chunks [c_begin, c_begin + C): node (c, j) at
// `level` with count in[c 2^level + j] splits its universe at the middle tile
// boundary; out[2 (c 2^level + j)] gets X, out[... + 1] the rest.
// Lane i of a warp owns node 32w + i: FP64 draws run on all lanes at once;
// fair-bit binomials are then counted by the whole warp, one node at a time.
template <class Geom>
__global__ void __launch_bounds__(256)
    tile_tree_level(Geom g, uint64_t c_begin, uint64_t C, int d, int level, uint64_t seed,
                    const uint64_t* __restrict__ in, uint64_t* __restrict__ out, int* err) {
  const uint64_t nwarps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  const unsigned lane = threadIdx.x & 31;
  const uint64_t total = C << level;
  for (uint64_t base = ((uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5) * 32; base < total;
       base += nwarps * 32) {
    const uint64_t node = base + lane;
    const bool live = node < total;
    uint64_t X = 0, k = 0, sid = 0;
    int st = ST_OK;
    HyperPlan hp;
    hp.kind = 0;
    hp.fixed = 0;
    if (live) {
      const uint64_t c = node >> level;
      const uint64_t j = node & ((uint64_t(1) << level) - 1);
      const uint64_t cc = c_begin + c;
      const uint64_t U = g.universe(cc);
      const uint64_t W = tile_width(U, d);
      const uint64_t lo = node_bound(U, W, d, level, j);
      const uint64_t hi = node_bound(U, W, d, level, u128(j) + 1);
      const uint64_t mid = node_bound(U, W, d, level + 1, u128(2) * j + 1);
      k = in[node];
      sid = (g.chunk_id(cc) << 32) | ((uint64_t(1) << level) + j);
      st = (k > hi - lo) ? ST_INTERNAL : hyper_plan(u128(hi - lo), u128(mid - lo), k, hp);
      if (st == ST_OK) {
        if (hp.kind == 0) {
          X = hp.fixed;
        } else if (hp.kind == 2) {
          Stream s(seed, sid, TAG_TILE);
          uint64_t r = 0;
          st = hyper_general(hp, s, r);
          X = st ? 0 : hyper_finish(hp, r);
        } else if (hp.t1 <= SMALL_FAIR_BITS) {
          // a short fair-bit count runs on its own lane
          Stream s(seed, sid, TAG_TILE);
          X = hyper_finish(hp, popcount_bits(hp.t1, s));
        }
      }
    }
    unsigned todo = __ballot_sync(0xffffffffu, live && st == ST_OK && hp.kind == 1 &&
                                                   hp.t1 > SMALL_FAIR_BITS);
    while (todo) {
      const int src = __ffs(todo) - 1;
      todo &= todo - 1;
      const uint64_t ssid = __shfl_sync(0xffffffffu, sid, src);
      const uint64_t st1 = __shfl_sync(0xffffffffu, hp.t1, src);
      const uint64_t r = popcount_bits_warp(seed, ssid, TAG_TILE, 0, st1);
      if (lane == unsigned(src)) X = hyper_finish(hp, r);
    }
    if (live) {
      if (st) {
        set_error(err, st);
        X = 0;
      }
      out[2 * node] = X;
      out[2 * node + 1] = k - X;
    }
  }
}

// ---------------------------------------------------------------- leaf kernel
struct LeafSmem {
  uint64_t keys[K_MAX];    // draws t_i in draw order
  uint64_t sorted[K_MAX];  // the same values sorted
  uint32_t hist[K_MAX];    // bucket counts, then bucket ends
  uint16_t first_pos[K_MAX];
  uint32_t bitT[K_MAX / 32], bitJ[K_MAX / 32];
  // control for the re-split walk
  int stack_level[LEVEL_MAX + 2];
  uint64_t stack_j[LEVEL_MAX + 2], stack_k[LEVEL_MAX + 2];
  int sp;
  int leaf_level;
  uint64_t leaf_j, leaf_k;
  int done;
};

// Edge sink: interleaved (u, v) pairs of Id (uint32_t or uint64_t); nothing
// is written at or beyond `cap` pairs (the device error word records it).
template <class Id>
struct PairSink {
  Id* out;
  uint64_t cap;
  int* err;
  __device__ __forceinline__ void write(uint64_t pos, uint64_t u, uint64_t v) const {
    if (pos >= cap) {
      set_error(err, ST_CAPACITY);
      return;
    }
    if (sizeof(Id) == 4) {
      uint2 w;
      w.x = uint32_t(u);
      w.y = uint32_t(v);
      reinterpret_cast<uint2*>(out)[pos] = w;
    } else {
      ulonglong2 w;
      w.x = u;
      w.y = v;
      __stcs(reinterpret_cast<ulonglong2*>(out) + pos, w);
    }
  }
  // whether slots [base, base + k) exist
  __device__ __forceinline__ bool fits(uint64_t base, uint64_t k) const {
    return base <= cap && k <= cap - base;
  }
  // store to a slot already checked by fits()
  __device__ __forceinline__ void put(uint64_t pos, uint64_t u, uint64_t v) const {
    if (sizeof(Id) == 4) {
      uint2 w;
      w.x = uint32_t(u);
      w.y = uint32_t(v);
      reinterpret_cast<uint2*>(out)[pos] = w;
    } else {
      ulonglong2 w;
      w.x = u;
      w.y = v;
      __stcs(reinterpret_cast<ulonglong2*>(out) + pos, w);
    }
  }
  __device__ __forceinline__ uint64_t read_u(uint64_t pos) const {
    if (pos >= cap) return ~uint64_t(0);
    return sizeof(Id) == 4 ? uint64_t(reinterpret_cast<const uint2*>(out)[pos].x)
                           : reinterpret_cast<const ulonglong2*>(out)[pos].x;
  }
};

// Floyd's sampler on one leaf: k distinct values of [0, L) (draw i is uniform
// on [0, L-k+i]; a value already taken is replaced by L-k+i), sorted by a
// bucket pass in shared memory; then offsets lo + value are mapped to (u, v)
// and written to positions base, base+1, ... .  All threads of the block call it.
template <class Geom, class Sink, bool DIGEST>
__device__ uint64_t* leaf_sample_emit(const Geom& g, const typename Geom::Ctx& gx,
                                      const Sink& sink, LeafSmem& sm, uint64_t seed,
                                      uint64_t node, uint64_t lo, uint64_t L, uint32_t k,
                                      uint64_t base, int* err, unsigned long long& dsum) {
  const int tid = threadIdx.x;
  const uint64_t Lk = L - k;
  // 1. draws: thread handles pairs (i, i+1) that share one Philox block
  for (uint32_t i = 2 * tid; i < k; i += 2 * LEAF_THREADS) {
    uint32_t w[4];
    philox10(i >> 1, uint32_t(node), uint32_t(node >> 32), TAG_LEAF, uint32_t(seed),
             uint32_t(seed >> 32), w);
    const uint64_t x0 = (uint64_t(w[0]) << 32) | w[1];
    sm.keys[i] = lemire_draw(x0, Lk + i + 1, seed, node, i);
    if (i + 1 < k) {
      const uint64_t x1 = (uint64_t(w[2]) << 32) | w[3];
      sm.keys[i + 1] = lemire_draw(x1, Lk + i + 2, seed, node, i + 1);
    }
  }
  // 2. bucket sort by the top bits: nb buckets (power of two >= k)
  uint32_t nb = 64;
  while (nb < k) nb <<= 1;
  const int lognb = __ffs(nb) - 1;
  const int bl = (L > 1) ? 64 - __clzll((long long)(L - 1)) : 0;  // bits of L-1
  const int shift = bl > lognb ? bl - lognb : 0;
  for (uint32_t b = tid; b < nb; b += LEAF_THREADS) sm.hist[b] = 0;
  __syncthreads();
  for (uint32_t i = tid; i < k; i += LEAF_THREADS) atomicAdd(&sm.hist[sm.keys[i] >> shift], 1u);
  __syncthreads();
  {
    // exclusive scan of hist[0..nb): each thread owns nb/LEAF_THREADS (or 1) entries
    const uint32_t per = (nb + LEAF_THREADS - 1) / LEAF_THREADS;
    const uint32_t b0 = tid * per;
    uint32_t s = 0;
    for (uint32_t q = 0; q < per; ++q)
      if (b0 + q < nb) s += sm.hist[b0 + q];
    uint32_t tot;
    uint32_t run = block_inclusive_scan<LEAF_THREADS>(s, tot) - s;
    for (uint32_t q = 0; q < per; ++q)
      if (b0 + q < nb) {
        const uint32_t c = sm.hist[b0 + q];
        sm.hist[b0 + q] = run;
        run += c;
      }
  }
  __syncthreads();
  for (uint32_t i = tid; i < k; i += LEAF_THREADS) {
    const uint64_t x = sm.keys[i];
    const uint32_t pos = atomicAdd(&sm.hist[x >> shift], 1u);
    sm.sorted[pos] = x;
  }
  __syncthreads();
  // hist[b] is now the end of bucket b; sort inside each bucket
  for (uint32_t b = tid; b < nb; b += LEAF_THREADS) {
    const uint32_t s0 = b ? sm.hist[b - 1] : 0, s1 = sm.hist[b];
    for (uint32_t x = s0 + 1; x < s1; ++x) {
      const uint64_t key = sm.sorted[x];
      uint32_t y = x;
      while (y > s0 && sm.sorted[y - 1] > key) {
        sm.sorted[y] = sm.sorted[y - 1];
        --y;
      }
      sm.sorted[y] = key;
    }
  }
  __syncthreads();
  // 3. all draws distinct  <=>  Floyd never replaced a value: S = {t_i}
  int dup = 0;
  for (uint32_t r = tid + 1; r < k; r += LEAF_THREADS) dup |= (sm.sorted[r] == sm.sorted[r - 1]);
  uint64_t* res = sm.sorted;
  if (__syncthreads_or(dup)) {
    // Sequential resolution in draw order.  A value v < L-k can only be taken
    // by an earlier draw of v itself (first occurrence wins); the values
    // L-k .. L-1 are tracked in a bitmap because replacements land there.
    for (uint32_t i = tid; i < k; i += LEAF_THREADS) {
      const uint64_t v = sm.keys[i];
      uint32_t a = 0, b = k;  // lower_bound in sorted
      while (a < b) {
        const uint32_t mid = (a + b) >> 1;
        if (sm.sorted[mid] < v)
          a = mid + 1;
        else
          b = mid;
      }
      sm.first_pos[i] = uint16_t(a);
    }
    for (uint32_t w = tid; w < K_MAX / 32; w += LEAF_THREADS) sm.bitT[w] = sm.bitJ[w] = 0;
    __syncthreads();
    if (tid == 0) {
      for (uint32_t i = 0; i < k; ++i) {
        const uint64_t v = sm.keys[i];
        if (v < Lk) {
          const uint32_t fp = sm.first_pos[i];
          if (sm.bitT[fp >> 5] & (1u << (fp & 31)))
            sm.bitJ[i >> 5] |= 1u << (i & 31);
          else
            sm.bitT[fp >> 5] |= 1u << (fp & 31);
        } else {
          const uint32_t bj = uint32_t(v - Lk);
          if (sm.bitJ[bj >> 5] & (1u << (bj & 31)))
            sm.bitJ[i >> 5] |= 1u << (i & 31);
          else
            sm.bitJ[bj >> 5] |= 1u << (bj & 31);
        }
      }
      // the taken set in increasing order, written over keys[]
      uint32_t o = 0;
      for (uint32_t r = 0; r < k; ++r) {
        const uint64_t v = sm.sorted[r];
        if (v >= Lk) break;
        if ((r == 0 || sm.sorted[r - 1] != v) && (sm.bitT[r >> 5] & (1u << (r & 31))))
          sm.keys[o++] = v;
      }
      for (uint32_t bj = 0; bj < k; ++bj)
        if (sm.bitJ[bj >> 5] & (1u << (bj & 31))) sm.keys[o++] = Lk + bj;
      if (o != k) set_error(err, ST_INTERNAL);
    }
    __syncthreads();
    res = sm.keys;
  }
  // 4. emit: consecutive ranks to consecutive threads (coalesced stores);
  // with DIGEST the row u replaces the offset in place for the run analysis
  for (uint32_t r = tid; r < k; r += LEAF_THREADS) {
    uint64_t u, v;
    g.map(gx, lo + res[r], u, v);
    sink.write(base + r, u, v);
    if (DIGEST) {
      dsum += edge_hash(u, v);
      res[r] = u;
    }
  }
  __syncthreads();
  return res;
}

// ---------------------------------------------------------------- fused digest
// Per tile: the digest sum, the out-degree histogram of runs of equal u that
// lie strictly inside the tile, and a record of the first / last run, which
// may continue in the neighbouring tiles (merged per chunk afterwards).
struct TileRec {
  uint64_t first_u, last_u;
  uint32_t first_len, last_len, nruns, pad;
};

struct DigestOut {
  unsigned long long* digest;  // per chunk of the range
  unsigned long long* hist;    // per chunk x 65
  TileRec* rec;                // per tile of the range
};

struct NoDigest {};

template <class Acc>
__device__ __forceinline__ void tile_runs(const Acc& u_at, uint32_t k, uint32_t& c1, uint32_t& nr,
                                          unsigned* bh, uint64_t& fu, uint32_t& fl, uint64_t& lu,
                                          uint32_t& ll) {
  for (uint32_t r = threadIdx.x; r < k; r += LEAF_THREADS) {
    const uint64_t u = u_at(r);
    if (r > 0 && u_at(r - 1) == u) continue;
    uint32_t len = 1;
    while (r + len < k && u_at(r + len) == u) ++len;
    ++nr;
    const bool first = (r == 0), last = (r + len == k);
    if (first) {
      fu = u;
      fl = len;
    }
    if (last) {
      lu = u;
      ll = len;
    }
    if (!first && !last) {
      if (len == 1)
        ++c1;
      else
        atomicAdd(&bh[len < 64 ? len : 64], 1u);
    }
  }
}

// Block-wide totals of one tile, added to its chunk; thread 0 writes the record.
__device__ __forceinline__ void tile_digest_finish(
    const DigestOut& dig, uint64_t t, uint64_t c_local, unsigned long long dsum, uint32_t c1,
    uint32_t nr, uint64_t fu, uint32_t fl, uint64_t lu, uint32_t ll, unsigned* bh,
    unsigned long long* red_d, unsigned* red_c1, unsigned* red_nr, uint64_t& s_fu, uint32_t& s_fl,
    uint64_t& s_lu, uint32_t& s_ll) {
  const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
    c1 += __shfl_xor_sync(0xffffffffu, c1, o);
    nr += __shfl_xor_sync(0xffffffffu, nr, o);
  }
  if (lane == 0) {
    red_d[wid] = dsum;
    red_c1[wid] = c1;
    red_nr[wid] = nr;
  }
  if (fl) {  // the thread that saw rank 0
    s_fu = fu;
    s_fl = fl;
  }
  if (ll) {  // the thread that saw the last rank
    s_lu = lu;
    s_ll = ll;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long D = 0;
    unsigned C1 = 0, NR = 0;
    for (int w = 0; w < LEAF_THREADS / 32; ++w) {
      D += red_d[w];
      C1 += red_c1[w];
      NR += red_nr[w];
    }
    atomicAdd(&dig.digest[c_local], D);
    if (C1) atomicAdd(&dig.hist[c_local * 65 + 1], (unsigned long long)C1);
    TileRec rc;
    rc.first_u = s_fu;
    rc.first_len = s_fl;
    rc.last_u = s_lu;
    rc.last_len = s_ll;
    rc.nruns = NR;
    rc.pad = 0;
    dig.rec[t] = rc;
  }
  for (int b = threadIdx.x; b < 65; b += LEAF_THREADS)
    if (bh[b]) atomicAdd(&dig.hist[c_local * 65 + b], (unsigned long long)bh[b]);
  __syncthreads();
}

// Per chunk: merge the first / last runs of consecutive tiles into whole rows,
// histogram them, and count the rows without out-edges into bin 0.
template <class Geom>
__global__ void chunk_run_merge(Geom g, uint64_t c_begin, uint64_t C, int d,
                                const TileRec* __restrict__ rec,
                                unsigned long long* __restrict__ hist) {
  for (uint64_t c = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < C;
       c += uint64_t(gridDim.x) * blockDim.x) {
    unsigned long long* h = hist + c * 65;
    bool open = false;
    uint64_t ou = 0, ol = 0, distinct = 0;
    const uint64_t t0 = c << d, t1 = (c + 1) << d;
    for (uint64_t t = t0; t < t1; ++t) {
      const TileRec r = rec[t];
      if (r.nruns == 0) continue;
      distinct += r.nruns;
      if (open && r.first_u == ou) {
        --distinct;
        if (r.nruns == 1) {
          ol += r.first_len;
          continue;
        }
        ol += r.first_len;
        atomicAdd(&h[ol < 64 ? ol : 64], 1ull);
        ou = r.last_u;
        ol = r.last_len;
        continue;
      }
      if (open) atomicAdd(&h[ol < 64 ? ol : 64], 1ull);
      if (r.nruns == 1) {
        open = true;
        ou = r.first_u;
        ol = r.first_len;
      } else {
        atomicAdd(&h[r.first_len < 64 ? r.first_len : 64], 1ull);
        open = true;
        ou = r.last_u;
        ol = r.last_len;
      }
    }
    if (open) atomicAdd(&h[ol < 64 ? ol : 64], 1ull);
    const uint64_t rows = g.rows(c_begin + c);
    atomicAdd(&h[0], (unsigned long long)(rows - distinct));
  }
}

// Tiles with more than k_max samples: split further (levels below d) by the
// same hypergeometric rule, left to right, until every leaf holds at most
// k_max samples; the leaves are emitted in order from the tile's offset.
// Everything about the tile comes from its descriptor.
template <class Geom, class Sink, bool DIGEST, class Desc>
__global__ void __launch_bounds__(LEAF_THREADS)
    leaf_resplit_kernel(Geom g, Sink sink, uint32_t k_max, const Desc* __restrict__ desc,
                        int* err, DigestOut dig, const unsigned long long* __restrict__ big,
                        const unsigned long long* __restrict__ nbig) {
  __shared__ LeafSmem sm;
  __shared__ unsigned bh[65];
  __shared__ unsigned long long red_d[LEAF_THREADS / 32];
  __shared__ unsigned red_c1[LEAF_THREADS / 32], red_nr[LEAF_THREADS / 32];
  __shared__ uint64_t s_fu, s_lu;
  __shared__ uint32_t s_fl, s_ll;
  const unsigned long long nb = *nbig;
  for (unsigned long long bi = blockIdx.x; bi < nb; bi += gridDim.x) {
    const uint64_t t = big[bi];
    const Desc td = desc[t];
    const uint64_t k = td.k;
    const uint64_t seed = td.seed;
    unsigned long long dsum = 0;
    uint32_t c1 = 0, nr = 0;
    uint64_t fu = 0, lu = 0;
    uint32_t fl = 0, ll = 0;
    if (DIGEST) {
      for (int b = threadIdx.x; b < 65; b += LEAF_THREADS) bh[b] = 0;
    }
    const int d = td.d;
    const uint64_t U = td.U, W = td.W, cid = td.cid;
    uint64_t base = td.base;
    const uint64_t base0 = base;
    if (threadIdx.x == 0) {
      sm.stack_level[0] = d;
      sm.stack_j[0] = td.tau;
      sm.stack_k[0] = k;
      sm.sp = 1;
    }
    for (;;) {
      __syncthreads();
      if (threadIdx.x == 0) {
        sm.done = 1;
        while (sm.sp > 0) {
          --sm.sp;
          int lv = sm.stack_level[sm.sp];
          uint64_t j = sm.stack_j[sm.sp], kk = sm.stack_k[sm.sp];
          bool bad = false;
          for (;;) {
            const uint64_t lo = node_bound(U, W, d, lv, j);
            const uint64_t hi = node_bound(U, W, d, lv, u128(j) + 1);
            if (kk > hi - lo) {
              set_error(err, ST_INTERNAL);
              bad = true;
              break;
            }
            if (kk <= k_max || hi - lo < 2) break;
            if (lv + 1 > LEVEL_MAX) {
              set_error(err, ST_INTERNAL);
              bad = true;
              break;
            }
            const uint64_t mid = node_bound(U, W, d, lv + 1, u128(2) * j + 1);
            Stream s(seed, (cid << 32) | ((uint64_t(1) << lv) + j), TAG_TILE);
            uint64_t X = 0;
            const int e = hypergeometric(u128(hi - lo), u128(mid - lo), kk, s, X);
            if (e) {
              set_error(err, e);
              bad = true;
              break;
            }
            sm.stack_level[sm.sp] = lv + 1;
            sm.stack_j[sm.sp] = 2 * j + 1;
            sm.stack_k[sm.sp] = kk - X;
            ++sm.sp;
            ++lv;
            j = 2 * j;
            kk = X;
          }
          if (bad) {
            sm.sp = 0;
            break;
          }
          if (kk > 0) {
            sm.leaf_level = lv;
            sm.leaf_j = j;
            sm.leaf_k = kk;
            sm.done = 0;
            break;
          }
        }
      }
      __syncthreads();
      if (sm.done) break;
      const int lv = sm.leaf_level;
      const uint64_t j = sm.leaf_j;
      const uint32_t kk = uint32_t(sm.leaf_k);
      const uint64_t lo = node_bound(U, W, d, lv, j);
      const uint64_t hi = node_bound(U, W, d, lv, u128(j) + 1);
      leaf_sample_emit<Geom, Sink, DIGEST>(g, td.gx, sink, sm, seed,
                                           (cid << 32) | ((uint64_t(1) << lv) + j), lo, hi - lo,
                                           kk, base, err, dsum);
      base += kk;
    }
    if (DIGEST) {
      // the tile's rows are read back from the output just written
      __syncthreads();
      auto at = [&sink, base0](uint32_t r) { return sink.read_u(base0 + r); };
      tile_runs(at, uint32_t(base - base0), c1, nr, bh, fu, fl, lu, ll);
      tile_digest_finish(dig, t, t >> d, dsum, c1, nr, fu, fl, lu, ll, bh, red_d, red_c1, red_nr,
                         s_fu, s_fl, s_lu, s_ll);
    }
  }
}

}  // namespace kg
