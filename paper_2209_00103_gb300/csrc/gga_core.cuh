// gga_core.cuh -- device-side building blocks of the library's kernels.
//
// The array's layout in HBM, the device pool, the bucket index math, the
// prefix-sum search and bucket allocation are in the public header
// gga_layout.cuh (shared with the device API that user kernels include);
// this file adds what only the library's kernels use: retry and spin
// bounds, pool queue pushes and fix-up, the mbarrier / bulk-copy PTX
// wrappers and the launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gga.h"
#include "gga_layout.cuh"

namespace gga {

constexpr uint64_t kUnitMask = (1ull << 40) - 1;
constexpr uint32_t kCasLimit = 1u << 20;     // bound on lock-free retry loops
constexpr uint32_t kSpinLimit = 1u << 22;    // bound on spin waits (~0.5 s with backoff)
constexpr uint32_t kChunkBytes = 16384;      // flatten / rw_b work unit

// upper_bound over a sorted uint64 array a[0..n): first i with a[i] > x.
__device__ __forceinline__ uint32_t upper_bound_u64(const uint64_t* a, uint32_t n, uint64_t x) {
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (a[mid] <= x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// Warp reduction.

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// Device pool queue operations (the pops are in gga_layout.cuh).

// Queue a bucket of byte class c (clear kernels only).  Returns false if the
// pool does not serve the class.
__device__ __forceinline__ bool ring_push(PoolState* p, uint32_t c, uint64_t addr) {
  const unsigned long long rc = p->ring_cap[c];
  if (rc == 0) return false;
  const unsigned long long j = atomicAdd(&p->ring_tail[c], 1ull);
  reinterpret_cast<uint64_t*>(p->rings)[p->ring_off[c] + j % rc] = addr;
  return true;
}

// After an insertion kernel: fold its pops into the queue heads (one thread).
__device__ __forceinline__ void ring_fixup(PoolState* p) {
  for (int c = 0; c < kPoolClasses; ++c) {
    if (p->ring_cap[c] == 0) continue;
    const unsigned long long h = p->ring_head[c] + p->ring_taken[c];
    p->ring_head[c] = h < p->ring_tail[c] ? h : p->ring_tail[c];
    p->ring_taken[c] = 0;
  }
}

// Chunks of kChunkBytes covering the live part of LFVector of `size`
// elements, bucket by bucket (flatten / rw_b work units).
__device__ __forceinline__ uint64_t bucket_chunks(uint64_t size, uint32_t log2B, uint32_t E) {
  uint64_t n = 0;
  for (uint32_t b = 0; b < static_cast<uint32_t>(kMaxBuckets); ++b) {
    const uint64_t first = bucket_first(b, log2B);
    if (first >= size) break;
    uint64_t len = bucket_len(b, log2B);
    if (size - first < len) len = size - first;
    n += (len * E + kChunkBytes - 1) / kChunkBytes;
  }
  return n;
}

// ---------------------------------------------------------------------------
// PTX wrappers: mbarrier and bulk (non-tensor) TMA copies.

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase; false if it gave up after `limit`
// attempts (the kernels then latch GGA_ERR_TIMEOUT and return).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t limit = kSpinLimit) {
  for (uint32_t it = 0; it < limit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
  }
  return false;
}

// Raise the transaction count a phase waits for, without arriving.
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Plain arrival (release at CTA scope).
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Global -> shared bulk copy completing on an mbarrier.  16-byte aligned
// addresses, size a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* smem_dst, const void* gsrc, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(smem_dst)),
      "l"(gsrc), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Shared -> global bulk copy tracked by bulk groups.
__device__ __forceinline__ void bulk_s2g(void* gdst, const void* smem_src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(smem_u32(smem_src)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// Bulk prefetch of [gsrc, gsrc + bytes) into L2 (a hint: nothing waits for
// it).  gsrc 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_prefetch_l2(const void* gsrc, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(gsrc), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_wait_read_all() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// ---------------------------------------------------------------------------
// Element types by size.

template <int E> struct Elem;
template <> struct Elem<4> { typedef uint32_t T; };
template <> struct Elem<8> { typedef unsigned long long T; };
template <> struct Elem<16> { typedef uint4 T; };

// 16 bytes seen as E-byte elements or as one 128-bit word.
template <int E>
union Vec16 {
  typename Elem<E>::T e[16 / E];
  uint4 v;
};

// ---------------------------------------------------------------------------
// Host-side launchers (defined in the .cu files).

struct InsertScratch {
  uint64_t* row_pre;              // [n_rows] run's first-value index inside its count tile
  uint64_t* pre;                  // [L][R + 1] run start of every round, relative to the batch base
  uint64_t* tile_pre;             // [n_tiles + 1] tile totals, then their exclusive prefix
  uint64_t* ins_base;             // [L] LFVector size before the batch
  uint64_t* ins_len;              // [L] committed elements of the batch
  uint64_t* cp_prefix;            // [L+1] prefix of copy chunks
  uint32_t* counters;             // [1] last-block-done counter of reserve
};

int launch_insert(const ArrayView& v, const InsertScratch& s, const uint32_t* counts, uint32_t rounds,
                  const void* values, uint64_t n_values, int num_sms, cudaStream_t st);
int launch_insert_generated(const ArrayView& v, const gga_gen_spec& spec, uint32_t rounds,
                            uint32_t* done_counter, int num_sms, cudaStream_t st);
int launch_finalize(const ArrayView& v, cudaStream_t st);
int launch_read(const ArrayView& v, const uint64_t* idx, uint64_t n, void* out, int num_sms, cudaStream_t st);
// scratch: nullptr, or wbin_scratch_bytes(n, E) bytes whose first 1 KB is
// zero before the first call (the binned path for n >= 2^20 keeps it so).
int launch_write(const ArrayView& v, const uint64_t* idx, uint64_t n, const void* in, int num_sms, void* scratch,
                 cudaStream_t st);
uint64_t wbin_scratch_bytes(uint64_t n, uint32_t E);
int launch_sweep(const ArrayView& v, int mode, uint64_t delta, uint32_t repeats, int num_sms, cudaStream_t st);
int launch_flatten(const ArrayView& v, void* dst, uint64_t cap_elems, int num_sms, cudaStream_t st);
int launch_reserve(const ArrayView& v, const uint64_t* target, cudaStream_t st);
int launch_clear(const ArrayView& v, cudaStream_t st);
int launch_caps(const ArrayView& v, uint64_t* caps, cudaStream_t st);
int launch_memory(const ArrayView& v, uint64_t* out2, cudaStream_t st);

int launch_twophase_spawn(const ArrayView& v, uint32_t gen, uint64_t seed, int only_newborn, uint64_t* born,
                          cudaStream_t st);
int launch_twophase_work(void* records, uint64_t n, uint32_t passes, int num_sms, cudaStream_t st);

// Handle internals for entry points defined outside gga_capi.cu (null
// output pointers are skipped).
bool handle_parts(gga_handle h, ArrayView* view, InsertScratch* ins, int* device, int* num_sms);
ArrayView* handle_dview(gga_handle h);
PoolState* handle_pool(gga_handle h);
uint64_t* handle_serve_records(gga_handle h, uint64_t slots);
uint64_t count_tiles(uint64_t n_rows, uint32_t T, bool vec_ok);
// Places gga_insert_noalloc's fixed scratch on device `dev` (current).
void noalloc_prepare(int dev);

}  // namespace gga
