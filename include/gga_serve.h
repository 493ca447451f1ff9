/*
 * gga_serve.h -- a native request server over many live GGArrays (the
 * serving pattern built on the GGArray's operations: append = Algorithm 1
 * and 2 through gga_append_batch, read = Sec. IV's global indexing through
 * gga_read_batch, flatten = the contiguous copy, after which the array is
 * retired with gga_clear).  The paper has no server; this is the host-side
 * scheduler of a serving workload (continuous batching of requests against
 * many live arrays), written natively so that the host's per-request work
 * stays small next to the GPU's.
 *
 * The scheduling rules (also the rules of the Python reference model in
 * paper_2209_00103_gb300/serving.py, which is tested on the CPU):
 *  - requests arrive at their trace times (seconds after the call starts);
 *    per array they run in arrival order: a request becomes ready when every
 *    earlier request of its array has completed (or was rejected);
 *  - each step takes ready requests oldest first, at most one per array and
 *    at most max_batch (batched = 0: one request per step, each waited for);
 *    an append is admitted only if a host mirror of the pool's allocator
 *    (free buckets per power-of-two byte class, then the bump pointer) says
 *    its buckets fit, else it waits, oldest first, to be tried again after a
 *    flatten returned memory, and is rejected deadline_s after its arrival;
 *  - a step is one gga_append_batch, one gga_read_batch and its flattens
 *    (each followed by gga_clear of the array), on `stream`; up to
 *    max_inflight steps are in flight; a request completes when its step's
 *    event has completed.
 * Latency = completion time seen by the host - arrival time.
 */
#ifndef GGA_SERVE_H
#define GGA_SERVE_H

#include <stdint.h>

#include "gga.h"

#ifdef __cplusplus
extern "C" {
#endif

enum { GGA_REQ_APPEND = 0, GGA_REQ_READ = 1, GGA_REQ_FLATTEN = 2 };

typedef struct {
  uint32_t n_arrays;       /* arrays[0..n_arrays) all of L LFVectors, first bucket B, E-byte elements */
  uint32_t L, B, E;
  uint32_t read_n;         /* elements per read request */
  uint32_t max_inflight;   /* steps in flight (>= 1) */
  uint32_t max_batch;      /* requests per step (>= 1) */
  int32_t batched;         /* 0: one request per step, each step waited for */
  double deadline_s;       /* how long an append may wait for pool memory */
  uint64_t pool_bytes;     /* the shared pool's slab bytes (the mirror's capacity) */
} gga_serve_config;

typedef struct {
  uint64_t steps;               /* launch steps */
  uint64_t step_requests;       /* requests over all steps */
  uint64_t appended_elements;   /* elements of admitted appends */
  double wall_s;                /* from the call's start to the last completion */
  double first_full_s;          /* arrival of the first append that did not fit (< 0: none) */
} gga_serve_stats;

/* Called (when given) for every read and flatten request once its step has
 * completed: dev_ptr holds n_elems elements of E bytes on the device, valid
 * only during the call. */
typedef void (*gga_serve_result_fn)(void* ctx, uint64_t request, const void* dev_ptr, uint64_t n_elems);

/*
 * gga_serve_run -- run a trace of n_req requests (host arrays, request r =
 * (t_arrival[r] seconds, type[r] in GGA_REQ_*, array[r] < n_arrays, n[r]
 * elements for appends (1 <= n[r], n[r] / L < 2^20), tag[r] = the append's
 * value tag and the read's seed)), arrival times ascending.  arrays: host
 * array of n_arrays handles created in `pool` with the config's shape and
 * empty at the call (their sizes are tracked on the host from here on).
 * read_out_dev: device, (max_inflight + 1) * max_batch * read_n elements
 * (read results land there); flat_arena_dev: device, flat_arena_elems
 * elements used round robin for flatten results (a result larger than the
 * arena gets its own stream-ordered allocation, freed after its step).
 * latency_s (host, n_req doubles) receives each request's latency (NaN when
 * not completed), state (host, n_req bytes) 1 = completed, 2 = rejected.
 * stats: host, optional.  Returns GGA_OK, GGA_ERR_INVALID for bad
 * arguments (nothing run), or the first error a library call returned
 * (the run stops there).
 */
int gga_serve_run(const gga_serve_config* cfg, gga_handle const* arrays, uint64_t n_req, const double* t_arrival,
                  const int8_t* type, const int64_t* array, const int64_t* n, const int64_t* tag,
                  void* read_out_dev, void* flat_arena_dev, uint64_t flat_arena_elems, double* latency_s,
                  int8_t* state, gga_serve_result_fn on_result, void* ctx, gga_serve_stats* stats, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GGA_SERVE_H */
