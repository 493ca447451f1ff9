/*
 * gga.h -- C ABI of a GB300-native GGArray.
 *
 * A GGArray (Meneses, Navarro and Ferrada, "GGArray: A Dynamically Growable
 * GPU Array", arXiv 2209.00103) is an array of LFVectors, one per thread
 * block (Sec. IV, Fig. 1-2).  LFVector l is a list of buckets; bucket b holds
 * B * 2^b elements (Algorithm 2) and is allocated only when an insertion
 * reaches it (Algorithm 1).  Buckets never move once allocated.
 *
 * Conventions shared by every entry point:
 *  - All data pointers are DEVICE pointers unless a parameter says "host".
 *    The caller owns every buffer it passes; the handle owns its metadata and
 *    its buckets.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Every call enqueues its work on `stream` and returns without
 *    waiting, except where it says "synchronizes".  Calls on one handle must
 *    be ordered on one stream (or otherwise serialised by the caller); calls
 *    that overlap on the GPU race.
 *  - Return value: GGA_OK, or an error code below.  Argument errors are found
 *    on the host and nothing is enqueued.  Errors found by the GPU (pool
 *    exhausted, index out of range, destination too small, count/value
 *    mismatch) are latched in a device status word of the handle and
 *    returned by the next synchronizing call (gga_size, gga_last_error).
 *  - Element order: within an LFVector, elements appear round by round;
 *    within a round by increasing thread id; a thread's elements are
 *    contiguous (Sec. III-B: positions come from a prefix sum over the
 *    block's threads).  The global order is LFVector-major (Sec. IV: the
 *    prefix sum of LFVector sizes gives each LFVector's first global index).
 */
#ifndef GGA_H
#define GGA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  GGA_OK = 0,
  GGA_ERR_INVALID = 1,         /* bad argument, or (device) counts do not sum to n_values */
  GGA_ERR_POOL_EXHAUSTED = 2,  /* (device) a bucket did not fit in the pool */
  GGA_ERR_OUT_OF_RANGE = 3,    /* (device) read/write index >= size */
  GGA_ERR_DST_TOO_SMALL = 4,   /* (device) flatten destination capacity < size */
  GGA_ERR_CUDA = 5,            /* a CUDA runtime call failed */
  GGA_ERR_TIMEOUT = 6,         /* (device) a bounded wait gave up */
  GGA_ERR_TOO_LARGE = 7        /* gga_insert_noalloc: the call needs more than its fixed scratch */
};

/* Sweep modes for gga_sweep (Sec. VI-B, rw_g and rw_b). */
enum {
  GGA_RW_G = 0,  /* one thread per element, global index -> (LFVector, bucket, offset) */
  GGA_RW_B = 1   /* follows the block structure: bucket by bucket, no search */
};

/* Count distributions for gga_insert_generated. */
enum {
  GGA_DIST_BERNOULLI = 0,  /* Bernoulli(1/2): top bit of the draw */
  GGA_DIST_UNIFORM3 = 1,   /* Uniform{0,1,2}: (hi32 * 3) >> 32 */
  GGA_DIST_GEOMETRIC = 2,  /* Geometric(1/2) - 1: trailing one bits, at most 63 */
  GGA_DIST_POISSON = 3     /* #{k : hi32 >= thresholds[k]} */
};

#define GGA_MAX_BUCKETS 48
#define GGA_MAX_THRESHOLDS 16

typedef struct gga_array* gga_handle;
typedef struct gga_pool_t* gga_pool;

typedef struct {
  uint32_t n_lfvectors;        /* L >= 1: LFVectors = thread blocks */
  uint32_t threads_per_block;  /* T in [1, 1024]: threads inserting into one LFVector */
  uint64_t base_bucket;        /* B: first bucket size in elements, a power of two */
  uint32_t elem_bytes;         /* E: 4, 8 or 16 */
  uint32_t reserved;           /* must be 0 */
  uint64_t pool_bytes;         /* bytes of the bucket pool (HBM slab) */
} gga_params;

/* Counter-based draws for gga_insert_generated: thread t of block l
 * (gtid = l*T + t) in round r draws h = SplitMix64 output number
 * ((r << 32) | gtid) + 1 of the stream seeded with `seed`, i.e.
 * mix64(seed + ((r << 32 | gtid) + 1) * 0x9E3779B97F4A7C15), takes a count c
 * from h by `dist`, and inserts values va*gtid + vb*r + vc*k (k < c, mod 2^64)
 * stored as E bytes: E=4 low 32 bits, E=8 all, E=16 the record
 * {uint64 v, float(v & 0xFFFF), float((v >> 16) & 0xFFFF)}. */
typedef struct {
  uint64_t seed;
  uint32_t dist;                             /* GGA_DIST_* */
  uint32_t n_thresholds;                     /* for GGA_DIST_POISSON, <= 16 */
  uint32_t thresholds[GGA_MAX_THRESHOLDS];
  uint64_t va, vb, vc;
  uint32_t round0;                           /* round number of the first round */
  uint32_t reserved;
} gga_gen_spec;

/* Memory accounting returned by gga_memory (bytes). */
typedef struct {
  uint64_t bucket_bytes;     /* sum over LFVectors of capacity * E (Sec. V "memory used") */
  uint64_t live_bytes;       /* size * E ("memory needed") */
  uint64_t pool_bytes;       /* pool slab size */
  uint64_t pool_bump_bytes;  /* slab bytes ever handed out by the bump pointer */
  uint64_t free_list_bytes;  /* bytes parked on the per-size free lists */
  uint64_t metadata_bytes;   /* descriptors, offsets, bucket tables, work lists */
} gga_mem;

/*
 * gga_pool_create -- a bucket pool several GGArrays can share (Algorithm 2's
 * malloc done on the device: a bump pointer over one slab plus one free
 * queue per power-of-two bucket size; buckets handed back are reused first).
 *  pool_bytes       : slab size.
 *  slab_dev         : device slab of pool_bytes bytes, 256-byte aligned,
 *                     borrowed (must outlive the pool); NULL = allocate one.
 *  min_bucket_bytes : smallest bucket (B * E) any array in the pool will
 *                     use; the queues take pool_bytes / min_bucket_bytes * 16
 *                     bytes of device memory at most.
 * Arrays made with gga_create_in_pool allocate from it.  All calls on arrays
 * of one pool must be ordered on the device (one stream, or events):
 * allocation and release are not safe to overlap.
 */
int gga_pool_create(uint64_t pool_bytes, void* slab_dev, uint64_t min_bucket_bytes, void* stream, gga_pool* out);

/* gga_pool_destroy -- free the pool (its arrays must be destroyed first).
 * Synchronizes the device. */
int gga_pool_destroy(gga_pool pool);

/* gga_pool_info -- out4 (host) = {slab bytes, slab bytes handed out by the
 * bump pointer, bytes waiting in the free queues, bytes of queue storage}.
 * Synchronizes. */
int gga_pool_info(gga_pool pool, uint64_t* out4, void* stream);

/*
 * gga_create_in_pool -- like gga_create, but buckets come from a shared
 * pool (p->pool_bytes is ignored).  GGA_ERR_INVALID if B * E is smaller than
 * the pool's min_bucket_bytes.  gga_destroy returns the array's buckets to
 * the pool.
 */
int gga_create_in_pool(const gga_params* p, gga_pool pool, void* stream, gga_handle* out);

/*
 * gga_create -- make an empty GGArray (Sec. IV).
 *  p        : parameters (host pointer, read during the call).
 *  pool_dev : device slab of p->pool_bytes bytes to carve buckets from, 256-byte
 *             aligned, borrowed (must outlive the handle); NULL = the handle
 *             allocates its own slab.
 *  out      : receives the handle (host pointer).
 * Buckets are allocated lazily (Algorithm 1), so the new array holds no
 * bucket.  Errors: GGA_ERR_INVALID (L = 0, T not in [1,1024], B not a power
 * of two, E not in {4,8,16}, pool not aligned), GGA_ERR_CUDA.
 */
int gga_create(const gga_params* p, void* pool_dev, void* stream, gga_handle* out);

/*
 * gga_insert -- `rounds` rounds of block-level push_back (Algorithm 1).
 *  counts_dev : uint32 [rounds][L][T]; counts[r][l][t] = elements thread t of
 *               block l inserts in round r.
 *  values_dev : n_values elements of E bytes, packed in (round, block, thread,
 *               k) order -- the order the per-block prefix sums assign.
 * Each round, each block reserves its run with one size update, allocates
 * the buckets the run reaches (Algorithm 2, from the device pool), and the
 * elements are written at their prefix-sum positions.  Then the global size
 * and the prefix sum of LFVector sizes are updated (Sec. IV).
 * Device errors: GGA_ERR_INVALID if the counts do not sum to n_values
 * (nothing is inserted); GGA_ERR_POOL_EXHAUSTED if a bucket does not fit: the
 * affected LFVector keeps the rounds that fit and drops the rest, other
 * LFVectors are unaffected.  Scratch: the handle keeps a scratch buffer of
 * about 16*rounds*L bytes and grows it (stream-ordered) when needed.
 */
int gga_insert(gga_handle h, const uint32_t* counts_dev, uint32_t rounds,
               const void* values_dev, uint64_t n_values, void* stream);

/*
 * gga_insert_noalloc -- gga_insert for callers that must not allocate GPU
 * memory while they run: code that owns a fixed memory budget reserved up
 * front (for example through a caching allocator that holds the rest of the
 * device), or latency-critical loops where a cudaMalloc/cudaMallocAsync could
 * block or fail.  The paper has no counterpart; it is an interface variant.
 *  Arguments, element order, results and device errors are those of
 *  gga_insert; the handle is created beforehand with gga_create as usual.
 *  Scratch: gga_insert keeps its per-call scratch (the tile totals of the
 *  count pass, the first-value index of every (round, block) run and every
 *  round's position in each LFVector's batch) in a buffer it grows on
 *  demand.  This variant instead uses one fixed 32 MiB array compiled into
 *  the library as a static __device__ variable, so it calls no cudaMalloc,
 *  cudaFree or allocating library routine.  Every GPU on which a handle
 *  was created holds those 32 MiB until the process exits.  A call needs at
 *  most about 16.5 * rounds * L bytes of it (rounds * L <= ~2 million, e.g.
 *  512 rounds of 1024 LFVectors use 8.5 MiB); a call that needs more
 *  returns GGA_ERR_TOO_LARGE and enqueues nothing.
 *  Set-up: the array's device address is looked up once per device
 *  (cudaGetSymbolAddress, with that device current).  gga_create and
 *  gga_create_in_pool do that lookup on the handle's device, which is also
 *  when the library's module holding the array is loaded there and its
 *  32 MiB are committed (CUDA loads modules lazily by default): create the
 *  handles before reserving the rest of the device.  If that lookup failed
 *  at creation, the first call on the device makes it again (make such a
 *  call before any stream capture) and returns GGA_ERR_CUDA if it fails
 *  again; the runtime's last-error state is left clear either way.  The
 *  current device must be the handle's.
 *  Sharing: all calls, on all handles, share the one array and it keeps the
 *  last call's contents (a call writes every part of it before reading it).
 *  Calls that overlap on the GPU -- on different streams, or from different
 *  threads -- race on it; order them.
 */
int gga_insert_noalloc(gga_handle h, const uint32_t* counts_dev, uint32_t rounds,
                       const void* values_dev, uint64_t n_values, void* stream);

/*
 * gga_reserve -- resize without inserting (the "grow" step of the paper's
 * growable-array experiment, Sec. VI-C / Table II: capacity is raised when
 * necessary before an insertion).  target_dev: device, L uint64 (8-byte
 * aligned); afterwards LFVector l's capacity is at least target_dev[l]
 * elements: the buckets that capacity reaches are taken from the pool
 * (Algorithm 2), as an insertion of that many elements would take them.
 * Sizes and contents do not change; capacity never shrinks.  An LFVector
 * whose buckets do not fit keeps the longest prefix that did and
 * GGA_ERR_POOL_EXHAUSTED is latched.
 */
int gga_reserve(gga_handle h, const uint64_t* target_dev, void* stream);

/*
 * gga_insert_generated -- the same insertion with counts and values drawn
 * inside the inserting threads (spec above), as a kernel calling push_back
 * does.  spec is a host pointer.  Device errors as gga_insert.
 */
int gga_insert_generated(gga_handle h, const gga_gen_spec* spec, uint32_t rounds, void* stream);

/*
 * Device API (the paper's model, Sec. III-B and Algorithm 1: push_back is
 * called by the threads of a block inside a user kernel).  The device side
 * is the header-only include/gga_device.cuh (gga::block_push_back,
 * gga::lfv_at, gga::global_at); these calls connect it to a handle.
 *
 * gga_device_view -- *view_dev (host) receives a DEVICE pointer to the
 *  handle's gga_dev_view, to be passed to user kernels as a
 *  `const gga_dev_view*`.  The pointer stays valid, and its contents fixed,
 *  until gga_destroy; no stream work.
 *
 * gga_device_commit -- enqueue, after the user kernel(s) that pushed into
 *  the array, the step every insertion ends with: the prefix sum of LFVector
 *  sizes (Sec. IV) and the global size are recomputed and the pool's queued
 *  buckets the kernels took are accounted.  Required before any other call
 *  on the handle, or on another handle of the same pool, that follows the
 *  pushes.  Errors the kernels found (gga_device.cuh lists them) are latched
 *  in the handle's status word and returned by gga_last_error / gga_size.
 *
 * gga_push_generated -- gga_insert_generated written as a user kernel of
 *  the device API: one block of T threads per LFVector, one push per round
 *  through a gga::BlockPusher, then gga_device_commit.  Same draws, same
 *  result, same errors as gga_insert_generated; it is the per-round form of
 *  Algorithm 1, which gga_insert_generated batches over rounds.  Each push
 *  is assembled in shared memory and written with 128-bit stores.
 *
 * gga_push_expand -- pushes of values read from device memory, written as a
 *  user kernel of the device API (one block per LFVector of T <= 512 slots,
 *  each thread playing 4 consecutive slots -- 2 for 16-byte elements --;
 *  gga::block_push_rounds, 4 rounds per call for 4-byte elements, 2 for
 *  8- and 16-byte), then gga_device_commit.  In
 *  round r, thread t of block l appends counts_dev[r][l][t] copies of
 *  inputs_dev[r][l][t].  counts_dev: device, uint32 [rounds][L][T], 4-byte
 *  aligned; inputs_dev: device, E-byte elements [rounds][L][T], E-byte
 *  aligned; both caller-owned, read on `stream`.  The result equals
 *  gga_insert with the same counts and values_dev = every input repeated
 *  its count times, in (round, block, thread) order (Algorithm 1 with the
 *  positions of Sec. III-B).  GGA_ERR_INVALID on the host for a null
 *  pointer, misalignment or T > 512; GGA_ERR_POOL_EXHAUSTED latched when a
 *  call's buckets do not fit (the LFVector keeps the longest prefix of
 *  whole rounds of that call that fits and stops).
 */
int gga_device_view(gga_handle h, const void** view_dev);
int gga_device_commit(gga_handle h, void* stream);
int gga_push_generated(gga_handle h, const gga_gen_spec* spec, uint32_t rounds, void* stream);
int gga_push_expand(gga_handle h, const uint32_t* counts_dev, const void* inputs_dev, uint32_t rounds,
                    void* stream);

/*
 * gga_read -- out_dev[i] = element at global index idx_dev[i], i < n (rw_g
 * addressing, Sec. VI-B: search over the prefix sum of sizes -- started from
 * the proportional guess i * L / N --, then the bucket and offset of the
 * LFVector-local index).  idx_dev: uint64 [n], 8-byte aligned; out_dev: n
 * elements of E bytes.  An index >= size latches GGA_ERR_OUT_OF_RANGE and
 * its output element is zeroed.
 */
int gga_read(gga_handle h, const uint64_t* idx_dev, uint64_t n, void* out_dev, void* stream);

/*
 * gga_write -- element at global index idx_dev[i] = in_dev[i], i < n.
 * idx_dev: uint64 [n], 8-byte aligned; in_dev: n elements of E bytes,
 * E-aligned.  Duplicate indices race (the GPU keeps one of the values); an
 * index >= size latches GGA_ERR_OUT_OF_RANGE and is skipped.  A batch of
 * 2^20 writes or more is grouped by ranges of global indices first and
 * applied range by range (the writes that share a 32-byte sector then meet
 * in L2); its bins, (4 + E) * n + 4 KB bytes of device memory, are allocated
 * stream-ordered on the first such call and kept by the handle (reused and
 * grown by later calls, freed by gga_destroy).  If they cannot be allocated
 * the writes go directly.
 */
int gga_write(gga_handle h, const uint64_t* idx_dev, uint64_t n, const void* in_dev, void* stream);

/*
 * gga_sweep -- the r/w operation of Sec. VI-C: add `delta` to every element,
 * `repeats` times (the paper adds +1 thirty times), elements taken as
 * unsigned E-byte integers with wrap-around (E = 4 or 8; 16-byte records are
 * GGA_ERR_INVALID).  mode GGA_RW_G visits elements by global index, GGA_RW_B
 * by the block structure (Sec. VI-B).  Both give the same result.
 */
int gga_sweep(gga_handle h, int mode, uint64_t delta, uint32_t repeats, void* stream);

/*
 * gga_flatten -- copy the GGArray into the contiguous array dst_dev in global
 * order (abstract and Sec. VI-C: insertion phase, then flatten, then regular
 * r/w on a static array).  dst_dev holds dst_capacity_elems elements of E
 * bytes and must be E-aligned.  If the size exceeds the capacity, nothing is
 * copied and GGA_ERR_DST_TOO_SMALL is latched.  Buckets are streamed with
 * TMA bulk copies.
 */
int gga_flatten(gga_handle h, void* dst_dev, uint64_t dst_capacity_elems, void* stream);

/*
 * gga_size -- global size and per-LFVector sizes/capacities (Sec. IV).
 * Synchronizes `stream`.
 *  total_host       : receives the global size (host pointer), may be NULL.
 *  sizes_dev        : uint64 [L] per-LFVector sizes, or NULL.
 *  caps_dev         : uint64 [L] capacities B*(2^nbuckets - 1), or NULL.
 * Returns the latched device error, if any (it stays latched).
 */
int gga_size(gga_handle h, uint64_t* total_host, uint64_t* sizes_dev, uint64_t* caps_dev, void* stream);

/* gga_offsets -- the prefix sum of LFVector sizes, uint64 [L+1] (Sec. IV). */
int gga_offsets(gga_handle h, uint64_t* offsets_dev, void* stream);

/*
 * gga_clear -- empty the array: every bucket goes back to the pool's
 * per-size free lists (reused by later insertions), sizes become 0.
 */
int gga_clear(gga_handle h, void* stream);

/* gga_memory -- memory accounting (host pointer out).  Synchronizes. */
int gga_memory(gga_handle h, gga_mem* out, void* stream);

/* gga_last_error -- synchronize, return the latched device error and clear it. */
int gga_last_error(gga_handle h, void* stream);

/*
 * gga_twophase_spawn -- one spawning generation of the two-phase case study
 * (Sec. VI-D: an insertion phase grows the array from inside the
 * application kernel, then the data is flattened for a regular work phase).
 * Elements are 16-byte records {uint64 id, float pos, float vel} (E must be
 * 16).  Every parent record of LFVector l spawns Geometric(1/2) - 1 children
 * into l: the count of the parent at local index j is the number of trailing
 * one bits of SplitMix64 output ((gen << 48) | (offsets[l] + j)) + 1 of the
 * stream seeded with `seed` (offsets as when the call starts); children are
 * appended in parent order, a parent's children consecutively, and copy the
 * parent's pos and vel with id = ((gen + 1) << 56) | (l << 40) | (local index
 * of the child).  Parents are all records present when the call starts
 * (only_newborn = 0), or for only_newborn = 1 the records from born_dev[l]
 * (uint64 [L], device, updated to the size at the start of the call).
 * Device errors as gga_insert (pool exhausted: the LFVector keeps the
 * children of its first parents, a multiple of 1024 of them, whose children
 * fit, and spawns no more in this call).
 */
int gga_twophase_spawn(gga_handle h, uint32_t gen, uint64_t seed, int only_newborn, uint64_t* born_dev,
                       void* stream);

/*
 * gga_twophase_work -- the case study's work phase on a flattened array of n
 * records (16-byte aligned device pointer): `passes` streaming passes, each
 * adding vel to pos of every record (one round-to-nearest float add).
 */
int gga_twophase_work(void* records_dev, uint64_t n, uint32_t passes, void* stream);

/*
 * Batched growth: many arrays grown in one persistent launch.
 *
 * A job names an array, the draws of its counts and values (the spec of
 * gga_insert_generated) and a target size.  LFVector l of the array targets
 * target / L elements, plus one for the first target % L LFVectors.  It runs
 * rounds r = spec.round0, round0 + 1, ... while below its target: every
 * thread draws its count for the round, and a thread's elements past the
 * target are not inserted (the block scan clips them), so the LFVector
 * holds the prefix of its draw sequence up to the target.  Arrays may have
 * different T (<= 1024), B, E and pools.
 */
typedef struct gga_batch_t* gga_batch;

typedef struct {
  gga_handle array;
  gga_gen_spec spec;
  uint64_t target;
} gga_batch_job;

/* gga_batch_create -- build the batch's device tables (allocates; jobs is a
 * host array read during the call; the arrays must outlive the batch). */
int gga_batch_create(const gga_batch_job* jobs, uint32_t n_jobs, void* stream, gga_batch* out);

/* gga_batch_grow -- grow every job's array to its target: one persistent
 * kernel over all (array, LFVector) items, one kernel for the pools, one to
 * finalize the arrays.  Allocates nothing, does not synchronize.  Device
 * errors are latched in each array (pool exhausted: the LFVector keeps the
 * rounds that fit). */
int gga_batch_grow(gga_batch b, void* stream);

/* gga_batch_clear -- empty every array of the batch (buckets back to their
 * pools) in two kernels. */
int gga_batch_clear(gga_batch b, void* stream);

/* gga_batch_capture -- capture clear + grow on `stream` (not the legacy
 * default stream) into a CUDA graph kept by the batch; gga_batch_replay
 * launches it. */
int gga_batch_capture(gga_batch b, void* stream);
int gga_batch_replay(gga_batch b, void* stream);

/* gga_batch_destroy -- free the batch's tables (not its arrays). */
int gga_batch_destroy(gga_batch b);

/*
 * Request batches for serving many live arrays (continuous batching: the
 * requests that arrived while earlier work ran are launched together).
 *
 * gga_append_batch -- append reqs[i].n elements to reqs[i].array for all i.
 * One kernel reserves every (request, LFVector) share (one size update, the
 * buckets it reaches from the pool: Algorithm 1 and 2) and recomputes each
 * array's offsets; a second kernel writes the elements, 16K elements per
 * block.  Requests are launched in groups of at most 480 requests and 8192
 * (request, LFVector) pairs; the first call on a pool allocates that pool's
 * 128 KB of reservation records (kept until gga_pool_destroy).  Every LFVector l of
 * the array gets n / L elements, one more for the first n % L; element k
 * appended to LFVector l has the value tag * 2^24 + l * 2^20 + k (stored as
 * E bytes like gga_insert_generated's values), so n / L must be below 2^20.
 * All arrays must share one pool and appear at most once (GGA_ERR_INVALID).
 * If the pool cannot hold an LFVector's share, that LFVector takes none of
 * it and GGA_ERR_POOL_EXHAUSTED is latched (callers admit requests so that
 * this does not happen).
 */
typedef struct {
  gga_handle array;
  uint64_t n;
  uint64_t tag;
} gga_append_req;

int gga_append_batch(const gga_append_req* reqs, uint32_t n, void* stream);

/*
 * gga_read_batch -- for every request, read n elements at global indices
 * floor(u_k * N / 2^32), u_k = the high 32 bits of SplitMix64 output k + 1
 * of the stream seeded with `seed`, N = the array's size when the read runs
 * (Sec. IV's global indexing), into out (device, n elements of E bytes;
 * zeros if the array is empty).  One block per request.
 */
typedef struct {
  gga_handle array;
  uint64_t n;
  uint64_t seed;
  void* out;
} gga_read_req;

int gga_read_batch(const gga_read_req* reqs, uint32_t n, void* stream);

/* gga_destroy -- free the handle's metadata and its private pool (a borrowed
 * slab is left to its owner); an array of a shared pool first returns its
 * buckets to the pool.  Synchronizes the device. */
int gga_destroy(gga_handle h);

#ifdef __cplusplus
}
#endif

#endif /* GGA_H */
