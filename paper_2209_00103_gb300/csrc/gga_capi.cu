// gga_capi.cu -- the extern "C" entry points declared in include/gga.h.
//
// A handle owns one metadata allocation (sizes, offsets, bucket tables, work
// lists, pool state, status words), an insertion scratch buffer that grows
// stream-ordered when a call needs more rounds, and -- unless the caller lent
// one -- the bucket slab.  Everything the operations compute runs in the
// kernels of gga_insert.cu and gga_access.cu; this file checks arguments,
// lays out memory and enqueues launches.
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>

#include "gga_core.cuh"

namespace gga {
uint64_t count_tiles(uint64_t n_rows, uint32_t T, bool vec_ok);
}

// A bucket pool: one slab, its bump pointer and the per-class free queues.
struct gga_pool_t {
  gga::PoolState* state;   // device
  void* slab;
  bool own_slab;
  void* rings;             // device, uint64 slots of all classes
  uint64_t ring_slots;
  uint64_t bytes;
  uint64_t min_bucket_bytes;
  int device;
  uint64_t* serve_records;  // device, made on first use by a batched append
  uint64_t serve_slots;
  std::mutex serve_mu;
};

struct gga_array {
  gga_params p;
  uint32_t log2B;
  int device;
  int num_sms;
  void* meta;
  size_t meta_bytes;
  gga_pool_t* pool;
  bool own_pool;
  void* scratch;
  size_t scratch_bytes;
  uint32_t scratch_rounds;
  gga::ArrayView view;
  gga::InsertScratch ins;   // pointers into meta (fixed part) and scratch (per-call part)
  unsigned long long* memstats;
  gga::ArrayView* dview;    // device copy of `view`, for kernels that take many arrays
  void* wscratch;           // binned random writes: bins of (address, value), kept between calls
  size_t wscratch_bytes;
};

namespace {

inline cudaStream_t S(void* s) { return static_cast<cudaStream_t>(s); }

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

bool valid_params(const gga_params* p) {
  if (!p) return false;
  if (p->n_lfvectors == 0 || p->threads_per_block == 0 || p->threads_per_block > 1024) return false;
  if (p->base_bucket == 0 || (p->base_bucket & (p->base_bucket - 1)) != 0) return false;
  if (p->base_bucket > (1ull << 40)) return false;
  if (!(p->elem_bytes == 4 || p->elem_bytes == 8 || p->elem_bytes == 16)) return false;
  if (p->reserved != 0) return false;
  return true;
}

// Per-call scratch of gga_insert, laid out for up to R_cap rounds:
// [tile prefixes [tiles+1] | row prefixes [rows+1] | pre [L][R+1]].
uint64_t max_tiles(uint32_t L, uint32_t T, uint32_t R) {
  const uint64_t rows = static_cast<uint64_t>(R) * L;
  const uint64_t a = gga::count_tiles(rows, T, false), b = gga::count_tiles(rows, T, true);
  return a > b ? a : b;
}

size_t insert_scratch_bytes(uint32_t L, uint32_t T, uint32_t R) {
  const uint64_t rows = static_cast<uint64_t>(R) * L;
  size_t b = align_up(max_tiles(L, T, R) * 8 + 8, 256);
  b += align_up((rows + 1) * 8, 256);
  b += align_up(static_cast<uint64_t>(L) * (R + 1) * 8, 256);
  return b;
}

void bind_scratch(gga_array* h, uint32_t R_cap, uint32_t R) {
  const uint32_t L = h->p.n_lfvectors;
  char* c = static_cast<char*>(h->scratch);
  h->ins.tile_pre = reinterpret_cast<uint64_t*>(c);
  c += align_up(max_tiles(L, h->p.threads_per_block, R_cap) * 8 + 8, 256);
  h->ins.row_pre = reinterpret_cast<uint64_t*>(c);
  c += align_up((static_cast<uint64_t>(R) * L + 1) * 8, 256);
  h->ins.pre = reinterpret_cast<uint64_t*>(c);
}

int ensure_scratch(gga_array* h, uint32_t R, cudaStream_t st) {
  if (R > h->scratch_rounds) {
    uint32_t cap = h->scratch_rounds * 2 > R ? h->scratch_rounds * 2 : R;
    const size_t nb = insert_scratch_bytes(h->p.n_lfvectors, h->p.threads_per_block, cap);
    if (h->scratch && cudaFreeAsync(h->scratch, st) != cudaSuccess) return GGA_ERR_CUDA;
    h->scratch = nullptr;
    h->scratch_bytes = 0;
    h->scratch_rounds = 0;
    if (cudaMallocAsync(&h->scratch, nb, st) != cudaSuccess) return GGA_ERR_CUDA;
    if (cudaMemsetAsync(h->scratch, 0, nb, st) != cudaSuccess) return GGA_ERR_CUDA;
    h->scratch_bytes = nb;
    h->scratch_rounds = cap;
  }
  bind_scratch(h, h->scratch_rounds, R);
  return GGA_OK;
}

// Make a pool of `bytes` (slab lent, or allocated when slab == nullptr).
// Queues exist for the byte classes from that of min_bucket_bytes up; a
// class's queue holds at most min(bytes >> c, lfv_hint * k) entries, k = 8
// for the 256-byte class (several small bucket indices share it), 1 above;
// lfv_hint = 0 means no hint (bounded by the slab only).
int pool_make(uint64_t bytes, void* slab, uint64_t min_bucket_bytes, uint64_t lfv_hint, cudaStream_t st,
              gga_pool_t** out) {
  gga_pool_t* pl = new (std::nothrow) gga_pool_t();
  if (!pl) return GGA_ERR_CUDA;
  pl->bytes = bytes;
  pl->min_bucket_bytes = min_bucket_bytes;
  pl->own_slab = slab == nullptr;
  pl->slab = slab;
  pl->rings = nullptr;
  pl->state = nullptr;
  pl->serve_records = nullptr;
  pl->serve_slots = 0;
  if (cudaGetDevice(&pl->device) != cudaSuccess) {
    delete pl;
    return GGA_ERR_CUDA;
  }
  gga::PoolState ps;
  std::memset(&ps, 0, sizeof(ps));
  uint64_t slots = 0;
  for (uint32_t c = gga::class_of(min_bucket_bytes ? min_bucket_bytes : 1); c < 64; ++c) {
    uint64_t n = bytes >> c;
    if (lfv_hint) {
      const uint64_t h = lfv_hint * (c == 8 ? 8 : 1);
      if (h < n) n = h;
    }
    ps.ring_off[c] = slots;
    ps.ring_cap[c] = n;
    slots += n;
  }
  pl->ring_slots = slots;
  int rc = GGA_OK;
  if (pl->own_slab && bytes > 0 && cudaMalloc(&pl->slab, bytes) != cudaSuccess) rc = GGA_ERR_CUDA;
  if (rc == GGA_OK && slots && cudaMalloc(&pl->rings, slots * 8) != cudaSuccess) rc = GGA_ERR_CUDA;
  if (rc == GGA_OK && cudaMalloc(reinterpret_cast<void**>(&pl->state), sizeof(gga::PoolState)) != cudaSuccess)
    rc = GGA_ERR_CUDA;
  if (rc == GGA_OK) {
    ps.cap = bytes;
    ps.base = reinterpret_cast<unsigned long long>(pl->slab);
    ps.rings = reinterpret_cast<unsigned long long>(pl->rings);
    if (cudaMemcpyAsync(pl->state, &ps, sizeof(ps), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      rc = GGA_ERR_CUDA;
  }
  if (rc != GGA_OK) {
    if (pl->state) cudaFree(pl->state);
    if (pl->rings) cudaFree(pl->rings);
    if (pl->own_slab && pl->slab) cudaFree(pl->slab);
    delete pl;
    return rc;
  }
  *out = pl;
  return GGA_OK;
}

int pool_free(gga_pool_t* pl) {
  int rc = GGA_OK;
  if (cudaDeviceSynchronize() != cudaSuccess) rc = GGA_ERR_CUDA;
  if (pl->state && cudaFree(pl->state) != cudaSuccess) rc = GGA_ERR_CUDA;
  if (pl->rings && cudaFree(pl->rings) != cudaSuccess) rc = GGA_ERR_CUDA;
  if (pl->own_slab && pl->slab && cudaFree(pl->slab) != cudaSuccess) rc = GGA_ERR_CUDA;
  if (pl->serve_records && cudaFree(pl->serve_records) != cudaSuccess) rc = GGA_ERR_CUDA;
  delete pl;
  return rc;
}

// Bytes parked in a pool's queues and its bump high-water mark (synchronizes).
int pool_read(gga_pool_t* pl, cudaStream_t st, uint64_t* bump, uint64_t* free_bytes) {
  gga::PoolState ps;
  if (cudaMemcpyAsync(&ps, pl->state, sizeof(ps), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return GGA_ERR_CUDA;
  *bump = ps.bump < ps.cap ? ps.bump : ps.cap;
  uint64_t fb = 0;
  for (int c = 0; c < 64; ++c)
    if (ps.ring_cap[c]) fb += (ps.ring_tail[c] - ps.ring_head[c]) << c;
  *free_bytes = fb;
  return GGA_OK;
}

int sync_status(gga_array* h, cudaStream_t st, bool clear) {
  uint32_t status = 0;
  if (cudaMemcpyAsync(&status, h->view.status, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) return GGA_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return GGA_ERR_CUDA;
  if (clear && status) {
    if (cudaMemsetAsync(h->view.status, 0, 4, st) != cudaSuccess) return GGA_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return GGA_ERR_CUDA;
  }
  return static_cast<int>(status);
}

}  // namespace

namespace gga {
ArrayView* handle_dview(gga_handle h) { return h ? h->dview : nullptr; }
PoolState* handle_pool(gga_handle h) { return h ? h->pool->state : nullptr; }

// Reservation records of batched appends on the handle's pool: 2 * slots
// uint64 (first index, then count, per (request, LFVector)), allocated once.
uint64_t* handle_serve_records(gga_handle h, uint64_t slots) {
  if (!h) return nullptr;
  gga_pool_t* pl = h->pool;
  std::lock_guard<std::mutex> lock(pl->serve_mu);
  if (pl->serve_records && pl->serve_slots >= slots) return pl->serve_records;
  if (pl->serve_records) return nullptr;
  void* p = nullptr;
  if (cudaMalloc(&p, 2 * slots * sizeof(uint64_t)) != cudaSuccess) return nullptr;
  pl->serve_records = static_cast<uint64_t*>(p);
  pl->serve_slots = slots;
  return pl->serve_records;
}

bool handle_parts(gga_handle h, ArrayView* view, InsertScratch* ins, int* device, int* num_sms) {
  if (!h) return false;
  if (view) *view = h->view;
  if (ins) *ins = h->ins;
  if (device) *device = h->device;
  if (num_sms) *num_sms = h->num_sms;
  return true;
}
}  // namespace gga

// Metadata and scratch of a handle living in `pool`.
static int handle_make(const gga_params* p, gga_pool_t* pool, bool own_pool, cudaStream_t st, gga_handle* out) {
  gga_array* h = new (std::nothrow) gga_array();
  if (!h) return GGA_ERR_CUDA;
  h->p = *p;
  h->log2B = 0;
  while ((1ull << h->log2B) < p->base_bucket) ++h->log2B;
  h->pool = pool;
  h->own_pool = own_pool;
  if (cudaGetDevice(&h->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
    delete h;
    return GGA_ERR_CUDA;
  }
  const uint64_t L = p->n_lfvectors;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  const size_t o_sizes = take(L * 8), o_offsets = take((L + 1) * 8), o_buckets = take(L * gga::kMaxBuckets * 8),
               o_nb = take(L * 4), o_fl = take((L + 1) * 8), o_ib = take(L * 8), o_il = take(L * 8),
               o_cp = take((L + 1) * 8), o_status = take(4), o_counters = take(16), o_mem = take(16),
               o_view = take(sizeof(gga::ArrayView));
  h->meta_bytes = off;
  if (cudaMalloc(&h->meta, h->meta_bytes) != cudaSuccess) {
    delete h;
    return GGA_ERR_CUDA;
  }
  char* m = static_cast<char*>(h->meta);
  gga::ArrayView& v = h->view;
  v.sizes = reinterpret_cast<uint64_t*>(m + o_sizes);
  v.offsets = reinterpret_cast<uint64_t*>(m + o_offsets);
  v.buckets = reinterpret_cast<uint64_t*>(m + o_buckets);
  v.nbuckets = reinterpret_cast<uint32_t*>(m + o_nb);
  v.fl_prefix = reinterpret_cast<uint64_t*>(m + o_fl);
  v.pool = pool->state;
  v.status = reinterpret_cast<uint32_t*>(m + o_status);
  v.B = p->base_bucket;
  v.L = p->n_lfvectors;
  v.T = p->threads_per_block;
  v.E = p->elem_bytes;
  v.log2B = h->log2B;
  h->ins.ins_base = reinterpret_cast<uint64_t*>(m + o_ib);
  h->ins.ins_len = reinterpret_cast<uint64_t*>(m + o_il);
  h->ins.cp_prefix = reinterpret_cast<uint64_t*>(m + o_cp);
  h->ins.counters = reinterpret_cast<uint32_t*>(m + o_counters);
  h->memstats = reinterpret_cast<unsigned long long*>(m + o_mem);
  h->scratch = nullptr;
  h->scratch_bytes = 0;
  h->scratch_rounds = 0;
  h->dview = reinterpret_cast<gga::ArrayView*>(m + o_view);
  int rc = cudaMemsetAsync(h->meta, 0, h->meta_bytes, st) == cudaSuccess ? GGA_OK : GGA_ERR_CUDA;
  if (rc == GGA_OK && cudaMemcpyAsync(h->dview, &h->view, sizeof(gga::ArrayView), cudaMemcpyHostToDevice, st) !=
                          cudaSuccess)
    rc = GGA_ERR_CUDA;
  // The insertion scratch is made by the first gga_insert that needs it.
  if (rc == GGA_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = GGA_ERR_CUDA;
  if (rc != GGA_OK) {
    h->own_pool = false;   // the caller disposes of the pool
    gga_destroy(h);
    return rc;
  }
  // Commit gga_insert_noalloc's fixed scratch on this device now, so that
  // no call of that entry point is the one that places it.
  gga::noalloc_prepare(h->device);
  *out = h;
  return GGA_OK;
}

extern "C" {

int gga_pool_create(uint64_t pool_bytes, void* slab_dev, uint64_t min_bucket_bytes, void* stream, gga_pool* out) {
  if (!out || pool_bytes == 0 || min_bucket_bytes == 0) return GGA_ERR_INVALID;
  if (slab_dev && (reinterpret_cast<uintptr_t>(slab_dev) & (gga::kGrain - 1)) != 0) return GGA_ERR_INVALID;
  *out = nullptr;
  return pool_make(pool_bytes, slab_dev, min_bucket_bytes, 0, S(stream), out);
}

int gga_pool_destroy(gga_pool pool) {
  if (!pool) return GGA_ERR_INVALID;
  return pool_free(pool);
}

int gga_pool_info(gga_pool pool, uint64_t* out4, void* stream) {
  if (!pool || !out4) return GGA_ERR_INVALID;
  uint64_t bump = 0, fb = 0;
  const int rc = pool_read(pool, S(stream), &bump, &fb);
  if (rc != GGA_OK) return rc;
  out4[0] = pool->bytes;
  out4[1] = bump;
  out4[2] = fb;
  out4[3] = pool->ring_slots * 8;
  return GGA_OK;
}

int gga_create(const gga_params* p, void* pool_dev, void* stream, gga_handle* out) {
  if (!out || !valid_params(p)) return GGA_ERR_INVALID;
  if (pool_dev && (reinterpret_cast<uintptr_t>(pool_dev) & (gga::kGrain - 1)) != 0) return GGA_ERR_INVALID;
  *out = nullptr;
  cudaStream_t st = S(stream);
  gga_pool_t* pool = nullptr;
  int rc = pool_make(p->pool_bytes, pool_dev, p->base_bucket * p->elem_bytes, p->n_lfvectors, st, &pool);
  if (rc != GGA_OK) return rc;
  rc = handle_make(p, pool, true, st, out);
  if (rc != GGA_OK) pool_free(pool);
  return rc;
}

int gga_create_in_pool(const gga_params* p, gga_pool pool, void* stream, gga_handle* out) {
  if (!out || !pool || !valid_params(p)) return GGA_ERR_INVALID;
  if (gga::alloc_bytes_for(p->base_bucket * p->elem_bytes) < gga::alloc_bytes_for(pool->min_bucket_bytes))
    return GGA_ERR_INVALID;   // the pool does not serve this array's smallest bucket
  *out = nullptr;
  return handle_make(p, pool, false, S(stream), out);
}

int gga_insert(gga_handle h, const uint32_t* counts_dev, uint32_t rounds, const void* values_dev,
               uint64_t n_values, void* stream) {
  if (!h) return GGA_ERR_INVALID;
  if (rounds == 0) return n_values == 0 ? GGA_OK : GGA_ERR_INVALID;
  if (!counts_dev || (n_values > 0 && !values_dev)) return GGA_ERR_INVALID;
  if ((reinterpret_cast<uintptr_t>(values_dev) % h->p.elem_bytes) != 0 && n_values > 0) return GGA_ERR_INVALID;
  if ((reinterpret_cast<uintptr_t>(counts_dev) & 3) != 0) return GGA_ERR_INVALID;
  cudaStream_t st = S(stream);
  int rc = ensure_scratch(h, rounds, st);
  if (rc != GGA_OK) return rc;
  return gga::launch_insert(h->view, h->ins, counts_dev, rounds, values_dev, n_values, h->num_sms, st);
}

int gga_reserve(gga_handle h, const uint64_t* target_dev, void* stream) {
  if (!h || !target_dev) return GGA_ERR_INVALID;
  if ((reinterpret_cast<uintptr_t>(target_dev) & 7) != 0) return GGA_ERR_INVALID;
  return gga::launch_reserve(h->view, target_dev, S(stream));
}

int gga_insert_generated(gga_handle h, const gga_gen_spec* spec, uint32_t rounds, void* stream) {
  if (!h || !spec) return GGA_ERR_INVALID;
  if (spec->dist > GGA_DIST_POISSON || spec->n_thresholds > GGA_MAX_THRESHOLDS) return GGA_ERR_INVALID;
  if (spec->dist == GGA_DIST_POISSON && spec->n_thresholds == 0) return GGA_ERR_INVALID;
  if (rounds == 0) return GGA_OK;
  return gga::launch_insert_generated(h->view, *spec, rounds, h->ins.counters, h->num_sms, S(stream));
}

int gga_read(gga_handle h, const uint64_t* idx_dev, uint64_t n, void* out_dev, void* stream) {
  if (!h || (n > 0 && (!idx_dev || !out_dev))) return GGA_ERR_INVALID;
  if ((reinterpret_cast<uintptr_t>(out_dev) % h->p.elem_bytes) != 0) return GGA_ERR_INVALID;
  if ((reinterpret_cast<uintptr_t>(idx_dev) & 7) != 0) return GGA_ERR_INVALID;
  return gga::launch_read(h->view, idx_dev, n, out_dev, h->num_sms, S(stream));
}

int gga_write(gga_handle h, const uint64_t* idx_dev, uint64_t n, const void* in_dev, void* stream) {
  if (!h || (n > 0 && (!idx_dev || !in_dev))) return GGA_ERR_INVALID;
  if ((reinterpret_cast<uintptr_t>(in_dev) % h->p.elem_bytes) != 0) return GGA_ERR_INVALID;
  if ((reinterpret_cast<uintptr_t>(idx_dev) & 7) != 0) return GGA_ERR_INVALID;
  // Large batches go through bins kept in the handle (grown stream-ordered;
  // if the allocation fails the writes go directly).
  const size_t need = gga::wbin_scratch_bytes(n, h->p.elem_bytes);
  if (need > h->wscratch_bytes) {
    cudaStream_t st = S(stream);
    if (h->wscratch) cudaFreeAsync(h->wscratch, st);
    h->wscratch = nullptr;
    h->wscratch_bytes = 0;
    if (cudaMallocAsync(&h->wscratch, need, st) == cudaSuccess && cudaMemsetAsync(h->wscratch, 0, 1024, st) == cudaSuccess) {
      h->wscratch_bytes = need;
    } else {
      cudaGetLastError();
      if (h->wscratch) cudaFreeAsync(h->wscratch, st);
      h->wscratch = nullptr;
    }
  }
  return gga::launch_write(h->view, idx_dev, n, in_dev, h->num_sms, need ? h->wscratch : nullptr, S(stream));
}

int gga_sweep(gga_handle h, int mode, uint64_t delta, uint32_t repeats, void* stream) {
  if (!h || (mode != GGA_RW_G && mode != GGA_RW_B)) return GGA_ERR_INVALID;
  if (h->p.elem_bytes == 16) return GGA_ERR_INVALID;
  return gga::launch_sweep(h->view, mode, delta, repeats, h->num_sms, S(stream));
}

int gga_flatten(gga_handle h, void* dst_dev, uint64_t dst_capacity_elems, void* stream) {
  if (!h || (!dst_dev && dst_capacity_elems > 0)) return GGA_ERR_INVALID;
  if ((reinterpret_cast<uintptr_t>(dst_dev) % h->p.elem_bytes) != 0) return GGA_ERR_INVALID;
  return gga::launch_flatten(h->view, dst_dev, dst_capacity_elems, h->num_sms, S(stream));
}

int gga_size(gga_handle h, uint64_t* total_host, uint64_t* sizes_dev, uint64_t* caps_dev, void* stream) {
  if (!h) return GGA_ERR_INVALID;
  cudaStream_t st = S(stream);
  const uint32_t L = h->p.n_lfvectors;
  if (sizes_dev &&
      cudaMemcpyAsync(sizes_dev, h->view.sizes, L * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return GGA_ERR_CUDA;
  if (caps_dev && gga::launch_caps(h->view, caps_dev, st) != GGA_OK) return GGA_ERR_CUDA;
  uint64_t n = 0;
  if (cudaMemcpyAsync(&n, h->view.offsets + L, sizeof(uint64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return GGA_ERR_CUDA;
  const int rc = sync_status(h, st, false);
  if (total_host) *total_host = n;
  return rc;
}

int gga_offsets(gga_handle h, uint64_t* offsets_dev, void* stream) {
  if (!h || !offsets_dev) return GGA_ERR_INVALID;
  return cudaMemcpyAsync(offsets_dev, h->view.offsets, (h->p.n_lfvectors + 1ull) * sizeof(uint64_t),
                         cudaMemcpyDeviceToDevice, S(stream)) == cudaSuccess
             ? GGA_OK
             : GGA_ERR_CUDA;
}

int gga_clear(gga_handle h, void* stream) {
  if (!h) return GGA_ERR_INVALID;
  return gga::launch_clear(h->view, S(stream));
}

int gga_memory(gga_handle h, gga_mem* out, void* stream) {
  if (!h || !out) return GGA_ERR_INVALID;
  cudaStream_t st = S(stream);
  if (cudaMemsetAsync(h->memstats, 0, 16, st) != cudaSuccess) return GGA_ERR_CUDA;
  if (gga::launch_memory(h->view, reinterpret_cast<uint64_t*>(h->memstats), st) != GGA_OK) return GGA_ERR_CUDA;
  unsigned long long ms[2];
  if (cudaMemcpyAsync(ms, h->memstats, 16, cudaMemcpyDeviceToHost, st) != cudaSuccess) return GGA_ERR_CUDA;
  uint64_t bump = 0, fb = 0;
  const int rc = pool_read(h->pool, st, &bump, &fb);
  if (rc != GGA_OK) return rc;
  out->bucket_bytes = ms[0];
  out->live_bytes = ms[1];
  out->pool_bytes = h->pool->bytes;
  out->pool_bump_bytes = bump;
  out->free_list_bytes = fb;
  out->metadata_bytes = h->meta_bytes + (h->own_pool ? h->pool->ring_slots * 8 : 0);
  return GGA_OK;
}

int gga_last_error(gga_handle h, void* stream) {
  if (!h) return GGA_ERR_INVALID;
  return sync_status(h, S(stream), true);
}

int gga_twophase_spawn(gga_handle h, uint32_t gen, uint64_t seed, int only_newborn, uint64_t* born_dev,
                       void* stream) {
  if (!h || h->p.elem_bytes != 16 || (only_newborn && !born_dev)) return GGA_ERR_INVALID;
  if (born_dev && (reinterpret_cast<uintptr_t>(born_dev) & 7) != 0) return GGA_ERR_INVALID;
  return gga::launch_twophase_spawn(h->view, gen, seed, only_newborn ? 1 : 0, born_dev, S(stream));
}

int gga_twophase_work(void* records_dev, uint64_t n, uint32_t passes, void* stream) {
  if (n > 0 && (!records_dev || (reinterpret_cast<uintptr_t>(records_dev) & 15) != 0)) return GGA_ERR_INVALID;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return GGA_ERR_CUDA;
  return gga::launch_twophase_work(records_dev, n, passes, sms, S(stream));
}

int gga_destroy(gga_handle h) {
  if (!h) return GGA_ERR_INVALID;
  int rc = GGA_OK;
  // In a shared pool the buckets go back to its queues first.
  if (!h->own_pool && h->pool && h->meta && gga::launch_clear(h->view, nullptr) != GGA_OK) rc = GGA_ERR_CUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) rc = GGA_ERR_CUDA;
  if (h->scratch && cudaFree(h->scratch) != cudaSuccess) rc = GGA_ERR_CUDA;
  if (h->wscratch && cudaFree(h->wscratch) != cudaSuccess) rc = GGA_ERR_CUDA;
  if (h->meta && cudaFree(h->meta) != cudaSuccess) rc = GGA_ERR_CUDA;
  if (h->own_pool && h->pool && pool_free(h->pool) != GGA_OK) rc = GGA_ERR_CUDA;
  delete h;
  return rc;
}

}  // extern "C"
