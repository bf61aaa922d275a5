/*
 * kg.h -- C ABI of the GB300 communication-free Erdos-Renyi generators.
 *
 * Implements the generators of "Communication-free Massively Distributed
 * Graph Generation" (Funke, Lamm, Meyer, Penschuck, Sanders, Schulz, Strash,
 * von Looz): directed G(n,m) (Sec. 4.1), undirected G(n,m) (Sec. 4.2) and
 * G(n,p) (Sec. 4.3), all built on the divide-and-conquer sampling of
 * Sec. 2.2.  Every chunk of the adjacency matrix draws its random numbers from
 * a counter-based generator keyed by (seed, chunk / subtree id), so the output
 * is a pure function of (n, m or p, seed, chunks): the same call always
 * returns the same bytes, however the GPU schedules the work.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Vertices are 0 .. n-1.  Simple graphs only: no self-loops, no parallel
 *    edges (Sec. 2).
 *  - Output edges are interleaved pairs (u, v) of `id_bytes` bytes each
 *    (id_bytes = 4: uint32 pairs, 8 bytes per edge, requires n <= 2^32;
 *    id_bytes = 8: uint64 pairs, 16 bytes per edge), sorted by (u, v).
 *    Undirected generators write every edge in both directions.
 *  - d_* pointers are device pointers owned by the caller; the library keeps
 *    none of them after the call.  Scratch memory is taken from and returned
 *    to the stream-ordered pool of the current device (cudaMallocAsync).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are asynchronous: they enqueue kernels and return.
 *  - Argument errors are reported synchronously and nothing is enqueued.
 *    Errors found on the device (capacity, internal limits) set a per-device
 *    error word that kg_last_error() reads; nothing is ever written beyond
 *    cap_edges entries of d_out.
 *  - `chunks` is P of the paper: the number of row chunks (directed) or the
 *    side of the triangular P x P chunk matrix (undirected).  Changing P
 *    changes which graph is drawn but not the distribution.
 */
#ifndef KG_H
#define KG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum kg_status {
  KG_OK = 0,
  KG_ERR_ARG = 1,      /* invalid argument (reported before any work) */
  KG_ERR_RANGE = 2,    /* valid but beyond the supported sizes */
  KG_ERR_CAPACITY = 3, /* output buffer too small */
  KG_ERR_CUDA = 4,     /* a CUDA call failed */
  KG_ERR_TIMEOUT = 5,  /* a bounded device wait ran out */
  KG_ERR_INTERNAL = 6  /* an internal limit was reached (not expected) */
} kg_status;

/*
 * Directed G(n,m), Sec. 4.1 (Theorem 1): m ordered pairs drawn uniformly
 * without replacement from the n(n-1) pairs u != v.  The rows are cut into P
 * chunks (chunk c = rows [floor(cn/P), floor((c+1)n/P))); the chunk sample
 * counts come from a binary split tree of hypergeometric variates (Sec. 2.2);
 * each chunk then refines its count over a tile tree and samples every tile
 * with Floyd's algorithm.
 *   n >= 1; 1 <= chunks <= min(n, 2^24); m <= n(n-1); m <= 2^44;
 *   ceil(n/P)(n-1) < 2^64; cap_edges >= m.
 * Writes exactly m pairs to d_out.
 */
kg_status kg_gnm_directed(uint64_t n, uint64_t m, uint64_t seed, uint32_t chunks, int id_bytes,
                          void* d_out, uint64_t cap_edges, void* stream);

/* Same with explicit leaf parameters: k_leaf = expected samples per tile
 * (the base-case threshold of Sec. 2.2, >= 2), k_max = the count above which a
 * tile is split once more (k_leaf <= k_max <= 2048).  kg_gnm_directed uses
 * k_leaf = 1024, k_max = 2048.  Different values draw different graphs. */
kg_status kg_gnm_directed_ex(uint64_t n, uint64_t m, uint64_t seed, uint32_t chunks,
                             uint32_t k_leaf, uint32_t k_max, int id_bytes, void* d_out,
                             uint64_t cap_edges, void* stream);

/* Chunk sample counts of directed G(n,m) (the split tree alone):
 * d_counts[c] for c < chunks (device, uint64). */
kg_status kg_gnm_directed_chunk_counts(uint64_t n, uint64_t m, uint64_t seed, uint32_t chunks,
                                       uint64_t* d_counts, void* stream);

/* The edges of chunks [c_begin, c_end) of directed G(n,m) only -- what PE
 * c_begin..c_end-1 of the paper generates, with no communication.
 * d_counts: the full chunk-count array from kg_gnm_directed_chunk_counts.
 * Writes sum(d_counts[c_begin..c_end)) pairs to d_out (the caller sizes
 * cap_edges from the counts).  If d_chunk_digest is non-NULL it receives,
 * per chunk of the range, the order-independent digest
 *   sum over edges of splitmix64(u xor rotl64(v, 32))  (mod 2^64);
 * if d_chunk_hist is non-NULL it receives, per chunk, 65 uint64 counters:
 * the number of vertices of the chunk with out-degree 0..63 and >= 64. */
kg_status kg_gnm_directed_range(uint64_t n, uint64_t m, uint64_t seed, uint32_t chunks,
                                uint32_t c_begin, uint32_t c_end, const uint64_t* d_counts,
                                int id_bytes, void* d_out, uint64_t cap_edges,
                                uint64_t* d_chunk_digest, uint64_t* d_chunk_hist, void* stream);

/*
 * Undirected G(n,m), Sec. 4.2 (Theorem 2): m unordered pairs drawn uniformly
 * without replacement.  The lower triangle of the adjacency matrix is cut
 * into the triangular P x P chunk matrix; the quadrant recursion (split
 * l = ceil(P/2), two triangles and one rectangle per triangle node) gives each
 * chunk its count; chunk (i, j) draws from the stream of id i*P + j, the
 * seed both PEs i and j of the paper share.
 *   n >= 1; 1 <= chunks <= min(n, 2^16); m <= n(n-1)/2; m <= 2^44;
 *   n <= 2^31; cap_edges >= 2m.
 * Writes exactly 2m pairs (both directions).
 */
kg_status kg_gnm_undirected(uint64_t n, uint64_t m, uint64_t seed, uint32_t chunks, int id_bytes,
                            void* d_out, uint64_t cap_edges, void* stream);
kg_status kg_gnm_undirected_ex(uint64_t n, uint64_t m, uint64_t seed, uint32_t chunks,
                               uint32_t k_leaf, uint32_t k_max, int id_bytes, void* d_out,
                               uint64_t cap_edges, void* stream);

/*
 * Undirected G(n,m) by row blocks, Sec. 4.2 at scale: the graph of
 * kg_gnm_undirected (same n, m, seed, chunks; default leaf sizes), but only
 * the rows of row blocks [b_begin, b_end) -- every entry (u, v) with
 * floor(b_begin n / P) <= u < floor(b_end n / P), both directions, sorted by
 * (u, v).  As a PE of the paper does, the call regenerates from their shared
 * seeds the chunks of those row blocks and of those column blocks, so
 * consecutive ranges concatenate to the whole list and no range needs another.
 *   n <= 2^40, ceil(n / chunks) < 2^32, 1 <= chunks <= min(n, 2^16), m <= 2^44,
 *   m <= n(n-1)/2; id_bytes 4 needs n <= 2^32; 0 <= b_begin < b_end <= chunks.
 * d_counts: the chunk counts of kg_gnm_undirected_chunk_counts (device,
 * P(P+1)/2 uint64 in the order k = i(i+1)/2 + j), or NULL to draw them here.
 * *d_entries (device, optional) receives the number of entries; beyond
 * cap_edges the device error word becomes KG_ERR_CAPACITY.  Optional per
 * row block of the range: d_block_digest[b - b_begin], the order-independent
 * digest of its entries, and d_block_hist[(b - b_begin) * 65 + d], the number
 * of its rows with degree d (d >= 64 in the last bin).
 */
kg_status kg_gnm_undirected_chunk_counts(uint64_t n, uint64_t m, uint64_t seed, uint32_t chunks,
                                         uint64_t* d_counts, void* stream);
kg_status kg_gnm_undirected_rows(uint64_t n, uint64_t m, uint64_t seed, uint32_t chunks,
                                 uint32_t b_begin, uint32_t b_end, const uint64_t* d_counts,
                                 int id_bytes, void* d_out, uint64_t cap_edges, uint64_t* d_entries,
                                 uint64_t* d_block_digest, uint64_t* d_block_hist, void* stream);

/*
 * G(n,p), Sec. 4.3: every pair independently with probability p, by
 * geometric skips (Batagelj and Brandes, Sec. 3.1) over tiles of each chunk;
 * a tile's skips come from the stream of (chunk id, tile), so the chunk law is
 * fixed by its seed alone.  Directed pairs are ordered (E[m] = p n(n-1));
 * undirected pairs are unordered (E[m] = p n(n-1)/2) and written both ways.
 *   0 <= p <= 1; chunk limits as above (undirected: n <= 2^31).
 * *d_count (device, uint64) receives the number of pairs written; if it
 * exceeds cap_edges only the first cap_edges are written and the device
 * error word becomes KG_ERR_CAPACITY.
 */
kg_status kg_gnp_directed(uint64_t n, double p, uint64_t seed, uint32_t chunks, int id_bytes,
                          void* d_out, uint64_t cap_edges, uint64_t* d_count, void* stream);
kg_status kg_gnp_undirected(uint64_t n, double p, uint64_t seed, uint32_t chunks, int id_bytes,
                            void* d_out, uint64_t cap_edges, uint64_t* d_count, void* stream);
/* As above with the tile parameter k_leaf (tile length = largest power of two
 * <= max(1, k_leaf/p); default 1024). */
kg_status kg_gnp_ex(int undirected, uint64_t n, double p, uint64_t seed, uint32_t chunks,
                    uint32_t k_leaf, int id_bytes, void* d_out, uint64_t cap_edges,
                    uint64_t* d_count, void* stream);

/* Test and instrumentation hook of kg_gnp_ex (no counterpart in the paper):
 * the skip walk of a tile stores its kept offsets in slots_per_tile slots
 * (clamped to the tile length) instead of the default min(2 k_leaf + 64, T),
 * or 0 slots above 12 GB of slots.  A tile with more kept pairs than slots is
 * walked a second time by the emit pass; slots_per_tile = 0 walks every tile
 * twice, as the default does for instances whose slots would pass 12 GB;
 * negative keeps the default.  The output is the same bytes whatever the
 * slot count.  slots_per_tile <= 2^20, else KG_ERR_ARG. */
kg_status kg_gnp_ex_slots(int undirected, uint64_t n, double p, uint64_t seed, uint32_t chunks,
                          uint32_t k_leaf, int32_t slots_per_tile, int id_bytes, void* d_out,
                          uint64_t cap_edges, uint64_t* d_count, void* stream);

/*
 * G(n,p) by binomial chunk counts, Sec. 4.3: the sample count of every chunk
 * is a binomial variate Binomial(U_c, p) drawn from the stream of (seed, chunk
 * id), and the chunk is then sampled exactly like a G(n,m) chunk (tile tree +
 * Floyd's algorithm).  Same law as kg_gnp_ex, a different graph for the same
 * seed.  Chunks as for G(n,m); the chunk universes must not exceed 2^53
 * pairs (KG_ERR_RANGE), so that the binomial's counts stay exact doubles.
 * *d_count (device, uint64) receives the number of entries (both directions
 * when undirected); beyond cap_edges the device error word becomes
 * KG_ERR_CAPACITY.  kg_gnp_binomial_count writes only *d_count (the chunk
 * binomials and their sum), the exact size of the same call's output.
 */
kg_status kg_gnp_binomial(int undirected, uint64_t n, double p, uint64_t seed, uint32_t chunks,
                          int id_bytes, void* d_out, uint64_t cap_edges, uint64_t* d_count,
                          void* stream);
kg_status kg_gnp_binomial_count(int undirected, uint64_t n, double p, uint64_t seed,
                                uint32_t chunks, uint64_t* d_count, void* stream);

/*
 * kg_gnm_directed_noalloc -- directed G(n,m) that allocates no memory.
 * The paper has no counterpart to this entry point; it exists for callers
 * that must not let a library allocate device memory: a framework whose
 * caching allocator already holds (almost) all of the GPU's memory, where a
 * pool allocation would fail or fragment it, or an application that sets
 * up all its memory before its steady-state loop and forbids allocation
 * inside it, because allocation can synchronise the device and its latency
 * has no bound.
 *
 * Output: the same bytes as kg_gnm_directed with the same arguments.
 * Scratch: one array of KG_NOALLOC_SCRATCH_BYTES bytes compiled into the
 * library as a file-scope __device__ variable; every GPU that loads the
 * library holds it until the process exits.  An instance needs about 144
 * bytes per tile (tiles = chunks * 2^d, d the tile-tree depth: the smallest d
 * with m * ceil(n/chunks) / n <= 1024 * 2^d), plus a few KB: up to about
 * 233,000 tiles, i.e. m up to about 2.3 * 10^8 at the default leaf size.  The need is
 * computed by the same code that carves the array (and reported by
 * kg_gnm_directed_noalloc_scratch); an instance that does not fit is
 * rejected with KG_ERR_RANGE before any work is enqueued, and d_status is
 * then left untouched.
 * The call itself makes no cudaMalloc / cudaFree / pool allocation.
 * Set-up: the first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and caches it; make that
 * first call before any stream capture.
 * Sharing: all calls use the same array, which keeps whatever the last call
 * left in it; each call clears what must start at zero.  Calls whose work
 * overlaps on the GPU (other streams, or a second call before the first one
 * finished on another stream) race on the array and give wrong results --
 * serialise them.
 * d_status: caller-owned device int, set to 0 by the call and then to the
 * first status a device-side check raises (KG_ERR_CAPACITY, KG_ERR_INTERNAL);
 * read it after the stream has finished.  It must not be NULL.  This entry
 * point does not use the error word of kg_last_error().
 */
#define KG_NOALLOC_SCRATCH_BYTES (32u << 20)
kg_status kg_gnm_directed_noalloc(uint64_t n, uint64_t m, uint64_t seed, uint32_t chunks,
                                  int id_bytes, void* d_out, uint64_t cap_edges, int* d_status,
                                  void* stream);
/* Bytes of the fixed array kg_gnm_directed_noalloc would use for (n, m,
 * chunks), to *h_bytes (host memory); host-only, touches no device.  The call
 * fits when the result is <= KG_NOALLOC_SCRATCH_BYTES. */
kg_status kg_gnm_directed_noalloc_scratch(uint64_t n, uint64_t m, uint32_t chunks,
                                          uint64_t* h_bytes);

/*
 * Batched G(n,m): many independent instances generated together (the paper
 * runs one instance on many PEs; batching runs many instances on one GPU).
 * kg_batch_create validates the instances, lays out their outputs one after
 * another in instance order, allocates the plan's device memory and uploads
 * the instance table -- once (it synchronises).  kg_batch_run then only
 * enqueues kernels on `stream`: no allocation, no host synchronisation, a
 * fixed launch sequence, so it can be captured into a CUDA graph and
 * replayed.  The output of instance i occupies entries
 * [offsets[i], offsets[i+1]) of d_out (kg_batch_offsets) and is bit-identical
 * to what kg_gnm_directed / kg_gnm_undirected write for the same instance
 * (uint32 ids only: id_bytes must be 4).  Limits per instance: chunks <= 64
 * (directed) or <= 32 (undirected), n <= 2^32, m <= 2^44.  Undirected
 * instances of 2^19 pairs or more are assembled on up to 8 stream lanes: the
 * caller's stream and up to 7 streams that kg_batch_create creates (forked
 * from `stream` by events and joined back, so that all of kg_batch_run's
 * work is ordered before what follows on `stream`); kg_batch_destroy
 * releases them.  One batch runs on one stream at a time.
 * kg_batch_tune times the launch shapes that do not change the output
 * (threads per block of the chunk-count kernel: 64, 128, 256; tiles per CTA
 * of the general leaf kernel, which samples the tiles the sparse leaf kernel
 * leaves: 1, 2, 4, 8, 16) on the caller's buffer and keeps the fastest.
 * Choices are cached for the process by GPU name and size class (log2 of the
 * instance and tile counts): a batch of a class already tuned on the same GPU
 * takes the cached choice without timing.  kg_batch_get_tuning reports the
 * batch's current choice.
 */
typedef struct kg_instance {
  uint64_t n, m, seed;
  uint32_t chunks;
  int32_t undirected; /* 0: directed, 1: undirected */
} kg_instance;
typedef struct kg_batch kg_batch;
kg_status kg_batch_create(const kg_instance* h_instances, uint32_t count, int id_bytes,
                          kg_batch** out_batch);
uint64_t kg_batch_entries(const kg_batch* batch);
kg_status kg_batch_offsets(const kg_batch* batch, uint64_t* h_offsets /* count + 1 */);
kg_status kg_batch_run(kg_batch* batch, void* d_out, uint64_t cap_entries, void* stream);
kg_status kg_batch_tune(kg_batch* batch, void* d_out, uint64_t cap_entries, int reps, void* stream);
kg_status kg_batch_get_tuning(const kg_batch* batch, uint32_t* tree_threads,
                              uint32_t* tiles_per_cta);
kg_status kg_batch_destroy(kg_batch* batch);

/* Exact size of a G(n,p) output before generating it: *d_count (device)
 * receives the number of entries kg_gnp_ex would write with the same
 * arguments (both directions for undirected), from the same skip walks
 * without storing them. */
kg_status kg_gnp_count(int undirected, uint64_t n, double p, uint64_t seed, uint32_t chunks,
                       uint32_t k_leaf, uint64_t* d_count, void* stream);
/* kg_gnp_count with the default tile parameter (k_leaf = 1024): the exact
 * size of what kg_gnp_directed (undirected = 0) or kg_gnp_undirected
 * (undirected = 1) writes for the same arguments. */
kg_status kg_gnp_size(int undirected, uint64_t n, double p, uint64_t seed, uint32_t chunks,
                      uint64_t* d_count, void* stream);

/*
 * Serving: a continuous-batching request loop (host scheduling, device work).
 * kg_server_create reserves `budget_bytes` of device memory for outputs and
 * `streams` CUDA streams.  kg_server_submit queues a request; a G(n,p)
 * request is first sized exactly on the device (kg_gnp_count).  Each
 * kg_server_poll admits waiting requests in arrival order while their exact
 * output (entries * 2 * id_bytes bytes) fits in the free budget, launches
 * them on the streams (so new requests overlap with running ones), and
 * reports finished requests: the output is reduced on the device to its
 * digest (as kg_edge_digest), copied to host memory, and its budget freed.
 * Times are milliseconds since kg_server_create (host clock).  The
 * generators' own scratch comes from the device's stream-ordered pool, not
 * from the budget.  A request larger than the whole budget finishes with
 * KG_ERR_CAPACITY.  The digest of a request does not depend on what else is
 * running.  Small requests (model 0 or 2, id_bytes = 4, at most 2^24 entries,
 * chunks <= 64 directed or <= 32 undirected, undirected n <= 2^20) admitted
 * in one poll are generated together, as groups of up to 1024, by the batched
 * engine (kg_batch_run's kernels) in a scratch arena of budget / 8 (clamped
 * to 256 MB .. 4 GB) allocated beside the budget; a poll may hand out part of
 * a finished group and the rest at the next poll.  Not thread-safe: one host
 * thread drives a server.
 */
typedef struct kg_request {
  int32_t model;      /* 0: G(n,m), 1: G(n,p) by skips (kg_gnp_ex),
                         2: G(n,p) by binomial chunk counts (kg_gnp_binomial) */
  int32_t undirected; /* 0 or 1 */
  uint64_t n, m;      /* m for G(n,m) */
  double p;           /* p for G(n,p) */
  uint64_t seed;
  uint32_t chunks;
  int32_t id_bytes;   /* 4 or 8 */
} kg_request;
typedef struct kg_result {
  uint64_t id, entries, digest;
  double t_submit_ms, t_admit_ms, t_done_ms;
  int32_t status, pad;
} kg_result;
typedef struct kg_server kg_server;
kg_status kg_server_create(uint64_t budget_bytes, uint32_t streams, kg_server** out_server);
kg_status kg_server_submit(kg_server* server, const kg_request* request, uint64_t* id_out);
kg_status kg_server_poll(kg_server* server, kg_result* h_results, uint32_t max_results,
                         uint32_t* n_results);
kg_status kg_server_pending(const kg_server* server, uint32_t* sizing, uint32_t* waiting,
                            uint32_t* running, uint64_t* bytes_in_use);
kg_status kg_server_destroy(kg_server* server);

/*
 * Random geometric graph RGG(n, r), Sec. 5: n points uniform in the unit
 * square (dim = 2) or cube (dim = 3), an edge between every two points at
 * Euclidean distance <= r.  Coordinates are 32-bit fixed point (the integer x
 * stands for x 2^-32); with R = floor(r 2^32), {u, v} is an edge iff
 * sum_k (x_k(u) - x_k(v))^2 <= R^2, decided in exact integer arithmetic.
 * The points are placed as in Sec. 5: a grid of 2^g cells per dimension
 * (side 2^(32-g) >= R, at most n cells; kg_rgg_grid), the cell counts from
 * the recursive split of the cube into its 2^d subcubes (each split as d
 * halvings drawing Binomial(c, 1/2) from the stream of its tree node), and
 * the points of a cell from the stream of that cell.  Vertex ids follow the
 * cells in row-major order (dimension 0 fastest), then the order in which a
 * cell's points are drawn.  The output is a pure function of (dim, n, r,
 * seed).
 *   dim in {2, 3}; 0 <= r <= 1/2 (else KG_ERR_ARG); n < 2^32 (else
 *   KG_ERR_RANGE).
 */
/* g of the grid (host only, synchronous). */
kg_status kg_rgg_grid(int dim, uint64_t n, double r, int* g_out);
/* Points per cell: d_counts (device, 2^(dim g) uint64, row-major cells). */
kg_status kg_rgg_cell_counts(int dim, uint64_t n, double r, uint64_t seed, uint64_t* d_counts,
                             void* stream);
/* Exact number of entries kg_rgg writes (twice the edge count), to *d_count. */
kg_status kg_rgg_count(int dim, uint64_t n, double r, uint64_t seed, uint64_t* d_count,
                       void* stream);
/* All edges in both directions, sorted by (u, v), as id_bytes-wide pairs in
 * d_out (at most cap_entries of them; more set the error word to
 * KG_ERR_CAPACITY and are dropped); *d_count = entries.  d_coords (device,
 * optional) receives the n x dim fixed-point coordinates, vertex-major.
 * Scratch from the stream-ordered pool: 24 n (dim 2) or 32 n (dim 3) bytes
 * (packed points, degrees, row offsets) plus 20 bytes per cell. */
kg_status kg_rgg(int dim, uint64_t n, double r, uint64_t seed, int id_bytes, void* d_out,
                 uint64_t cap_entries, uint64_t* d_count, uint32_t* d_coords, void* stream);

/* Order-independent digest of an edge list (see kg_gnm_directed_range):
 * *d_digest = sum of splitmix64(u xor rotl64(v, 32)) over `count` pairs. */
kg_status kg_edge_digest(const void* d_edges, uint64_t count, int id_bytes, uint64_t* d_digest,
                         void* stream);

/* Synchronises `stream`, returns and clears the current device's error word. */
kg_status kg_last_error(void* stream);

/* Human-readable name of a status. */
const char* kg_status_str(kg_status s);

/* Releases what the library holds on the current device: waits for the
 * device to finish, frees the device error word (a pending error is
 * discarded) and returns the scratch cached in the device's stream-ordered
 * pool to the driver.  Batches and servers are owned by the caller and are
 * not touched.  Any entry point may be called afterwards: the state is made
 * again on first use.  Not thread-safe against concurrent calls. */
kg_status kg_shutdown(void);

/*
 * Instrumentation (no counterpart in the paper).
 * kg_launch_count: number of kernels this library has launched in the process.
 * kg_profile_begin / kg_profile_end: while enabled, every launch is bracketed
 * by a CUDA event pair recorded on the stream it is launched on; _end waits
 * for those events and returns, per kernel class, the summed milliseconds and
 * the number of launches (arrays of KG_PROF_CLASSES entries, host memory).
 * Classes: 0 chunk split tree, 1 tile tree, 2 scan, 3 leaf sampler/emitter,
 * 4 digest, 5 G(n,p) tile sampler, 6 undirected assembly, 7 other,
 * 8 random geometric graph.
 */
#define KG_PROF_CLASSES 9
unsigned long long kg_launch_count(void);
/* Ceilings measured with the library's own kernels (the caller times them,
 * e.g. with CUDA events on `stream`):
 * kg_peak_store writes `bytes` (a multiple of 16; d_buf 16-byte aligned) with
 * 16-byte stores, evict-first (mode 0) or write-back (mode 1), in a grid of
 * 8 blocks of 256 threads per SM -- the write-only bandwidth that bounds edge
 * emission.  kg_peak_fp64 runs `blocks` blocks of 256 threads, each thread
 * `iters` iterations of 8 independent chains x = x*a + b with separately
 * rounded multiply and add (16 FP64 operations per iteration and thread) --
 * the FP64 add/multiply rate that bounds the G(n,p) skip walk; d_out (2
 * doubles) receives a checksum. */
kg_status kg_peak_store(void* d_buf, uint64_t bytes, int mode, void* stream);
kg_status kg_peak_fp64(double* d_out, uint32_t blocks, uint32_t iters, void* stream);
kg_status kg_profile_begin(void);
kg_status kg_profile_end(double* ms, unsigned long long* launches);

#ifdef __cplusplus
}
#endif
#endif /* KG_H */
