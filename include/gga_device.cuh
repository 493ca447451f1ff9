// gga_device.cuh -- device API of the GB300 GGArray, for user kernels.
//
// The paper's model (Sec. III-B, Algorithm 1): the threads of a block
// insert into their own LFVector from inside a kernel.  Every thread
// contributes `count` elements; positions come from a prefix sum over the
// block's threads; one thread reserves the block's run on the LFVector and
// allocates the buckets it reaches (Algorithm 2, from a device pool, no
// host round trip); after a block barrier every thread writes its elements.
//
// Usage (header-only; compile with -I<this directory>, sm_103a):
//
//   #include "gga_device.cuh"
//   __global__ void k(const gga_dev_view* v, ...) {
//     uint32_t c = ...;                               // my element count
//     gga::block_push_back<uint32_t>(v, blockIdx.x, c,
//         [&](uint32_t k) { return my_value(k); });   // element k of mine
//   }
//
//   host:  const void* v;  gga_device_view(h, &v);     // device pointer
//          k<<<L, T, 0, s>>>((const gga_dev_view*)v, ...);
//          gga_device_commit(h, s);                   // before any other call on h
//
// For many pushes into one LFVector in one kernel, gga::BlockPusher keeps
// the LFVector's size in every thread and needs one block barrier per push
// (two when the push reaches new buckets), against two for each
// block_push_back call.
//
// Rules (the paper's phase separation, Sec. VI):
//  - every thread of the block calls block_push_back with the same
//    LFVector l (it holds two block barriers); l < L;
//  - at most one block pushes into a given LFVector at a time, and no other
//    call on the array (read, write, sweep, flatten, clear, insert) overlaps
//    the kernel on the GPU; kernels pushing into arrays of one pool are
//    ordered on the device, as every insertion is;
//  - gga_device_commit(h, stream) follows the kernel on the same stream: it
//    recomputes the prefix sum of LFVector sizes (Sec. IV) and returns the
//    pool's queued buckets the kernel took.  Global indices (global_at,
//    gga_read, ...) see the pushes only after it.
// Errors are latched in the array's device status word and returned by
// gga_last_error / gga_size: GGA_ERR_INVALID for l >= L or
// sizeof(T) != E (nothing pushed), GGA_ERR_POOL_EXHAUSTED when a bucket
// does not fit (that block's call pushes nothing; buckets it did get stay
// with the LFVector for its next growth).
//
// The library's own kernels are built on the same definitions.
//
// Layout in HBM (one set per handle):
//   sizes    [L]        uint64  LFVector sizes
//   offsets  [L+1]      uint64  prefix sum of sizes (Sec. IV), offsets[L] = N
//   buckets  [L][48]    uint64  bucket base addresses, 0 = nil (Algorithm 1)
//   nbuckets [L]        uint32  buckets allocated so far (always a prefix)
//   pool                PoolState: bump pointer + per-size free lists
//   status              uint32  first device-detected error
// Buckets live in one pre-reserved slab; bucket b of every LFVector holds
// B * 2^b elements (Algorithm 2) and starts on a 256-byte boundary.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gga.h"

namespace gga {

constexpr int kMaxBuckets = GGA_MAX_BUCKETS;
constexpr int kPoolClasses = 64;
constexpr uint64_t kGrain = 256;             // bucket alignment / allocation granule

// Device pool (Algorithm 2's malloc, without the host).  Buckets are carved
// from one slab by a bump pointer; buckets handed back (gga_clear,
// gga_destroy) wait in one ring queue per power-of-two byte class and are
// reused first.  Queues are touched with atomicAdd only: insertion kernels
// (and kernels calling block_push_back) pop (ring_taken), clear kernels push
// (ring_tail), never both in one kernel, and kernels using one pool are
// ordered on the device (one stream, or events); a one-thread fix-up after
// each insertion (gga_device_commit after a user kernel) folds the pops into
// ring_head.  A class's queue has room for every bucket of that class the
// slab can hold (or, for a handle's private pool, that its LFVectors can
// hold), so pushes never overrun it.
struct PoolState {
  unsigned long long bump;                        // slab bytes handed out (passes cap once exhausted)
  unsigned long long cap;                         // slab bytes
  unsigned long long base;                        // slab address
  unsigned long long ring_head[kPoolClasses];     // first queued entry
  unsigned long long ring_tail[kPoolClasses];     // one past the last queued entry
  unsigned long long ring_taken[kPoolClasses];    // pops by the running insertion kernel
  unsigned long long ring_off[kPoolClasses];      // first slot of the class in `rings`
  unsigned long long ring_cap[kPoolClasses];      // slots of the class (0: class not served)
  unsigned long long rings;                       // address of the uint64 slots
};

struct ArrayView {
  uint64_t* sizes;
  uint64_t* offsets;
  uint64_t* buckets;
  uint32_t* nbuckets;
  PoolState* pool;
  uint32_t* status;
  uint64_t* fl_prefix;   // [L+1] prefix of 16 KB bucket chunks per LFVector (flatten, rw_b)
  uint64_t B;
  uint32_t L, T, E, log2B;
};

// ---------------------------------------------------------------------------
// Errors.

__device__ __forceinline__ void latch_error(uint32_t* status, uint32_t code) {
  atomicCAS(status, 0u, code);
}

// ---------------------------------------------------------------------------
// Index math (Algorithm 2 bucket sizes): LFVector-local index j lies in
// bucket b with B(2^b - 1) <= j < B(2^(b+1) - 1), i.e. B*2^b <= j + B <
// B*2^(b+1).  So the highest set bit of j + B is log2(B) + b, and the offset
// is (j + B) - 2^hb.  No loop.

__device__ __forceinline__ void bucket_of(uint64_t j, uint32_t log2B, uint32_t& b, uint64_t& off) {
  const uint64_t x = j + (1ull << log2B);
  const uint32_t hb = 63u - static_cast<uint32_t>(__clzll(static_cast<long long>(x)));
  b = hb - log2B;
  off = x - (1ull << hb);
}

__host__ __device__ __forceinline__ uint64_t bucket_first(uint32_t b, uint32_t log2B) {
  return ((1ull << b) - 1ull) << log2B;   // B (2^b - 1)
}

__host__ __device__ __forceinline__ uint64_t bucket_len(uint32_t b, uint32_t log2B) {
  return 1ull << (log2B + b);             // B 2^b
}

// Number of buckets reached by indices 0..size-1.
__device__ __forceinline__ uint32_t buckets_for(uint64_t size, uint32_t log2B) {
  if (size == 0) return 0;
  uint32_t b;
  uint64_t off;
  bucket_of(size - 1, log2B, b, off);
  return b + 1;
}
// LFVector holding global index g < N: the prefix sum of sizes (Sec. IV) is
// searched from a proportional guess l = g * L / N, corrected by up to four
// steps to a neighbour (sizes of similar LFVectors land here), else by a
// binary search.  Returns the l with offsets[l] <= g < offsets[l + 1].  The
// offsets go through the read-only cache (`off` must point to global memory,
// never to a shared-memory copy): no block-wide staging, so a block costs
// nothing before its first access.
__device__ __forceinline__ uint32_t find_lfv(const uint64_t* off, uint32_t L, uint64_t N, uint64_t g) {
  // The guess only starts the search, so fp32 rounding in it is harmless.
  const float guess = __ull2float_rz(g) * (static_cast<float>(L) / __ull2float_rz(N));
  uint32_t l = guess < static_cast<float>(L) ? __float2uint_rz(guess) : L - 1;
  if (l >= L) l = L - 1;
#pragma unroll 1
  for (int s = 0; s < 4; ++s) {
    if (__ldg(off + l) > g) { --l; continue; }
    if (__ldg(off + l + 1) <= g) { ++l; continue; }
    return l;
  }
  uint32_t lo = 0, hi = L + 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(off + mid) <= g) lo = mid + 1; else hi = mid;
  }
  return lo - 1;
}

// ---------------------------------------------------------------------------
// Warp scan (Sec. III-B: shuffle prefix sum inside the block), for full
// warps of blocks whose x extent is a multiple of 32.

template <typename V>
__device__ __forceinline__ V warp_incl_scan(V v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const V n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += n;
  }
  return v;
}

// ---------------------------------------------------------------------------
// Device pool operations.

__host__ __device__ __forceinline__ uint64_t alloc_bytes_for(uint64_t bytes) {
  return bytes < kGrain ? kGrain : bytes;   // bucket sizes are powers of two
}

__host__ __device__ __forceinline__ uint32_t class_of(uint64_t bytes) {
  const uint64_t a = alloc_bytes_for(bytes);
  uint32_t c = 0;
  while ((1ull << c) < a) ++c;
  return c;
}

// Pop a queued bucket of byte class c, or 0 if the queue ran dry.
__device__ __forceinline__ uint64_t ring_pop(PoolState* p, uint32_t c) {
  const unsigned long long rc = p->ring_cap[c];
  if (rc == 0) return 0;
  const unsigned long long i = atomicAdd(&p->ring_taken[c], 1ull);
  const unsigned long long pos = p->ring_head[c] + i;
  if (pos >= p->ring_tail[c]) return 0;
  return reinterpret_cast<const uint64_t*>(p->rings)[p->ring_off[c] + pos % rc];
}

// Allocate buckets nb..need-1 of LFVector l (Algorithm 2 for every bucket a
// reservation reaches).  Queued buckets first; the rest with one bump of the
// slab for all of them.  A bucket index that cannot be served ends the
// allocated prefix; buckets obtained beyond it stay in the table as spares
// for the next growth.  Returns the new length of the allocated prefix.
__device__ inline uint32_t grow_buckets(const ArrayView& v, uint32_t l, uint32_t nb, uint32_t need) {
  uint64_t* tab = v.buckets + static_cast<uint64_t>(l) * kMaxBuckets;
  if (need > static_cast<uint32_t>(kMaxBuckets)) need = kMaxBuckets;
  uint64_t miss = 0, bump_bytes = 0;
  for (uint32_t b = nb; b < need; ++b) {
    if (tab[b] != 0) continue;
    const uint64_t a = ring_pop(v.pool, class_of(bucket_len(b, v.log2B) * v.E));
    if (a) {
      tab[b] = a;
    } else {
      miss |= 1ull << b;
      bump_bytes += alloc_bytes_for(bucket_len(b, v.log2B) * v.E);
    }
  }
  if (bump_bytes) {
    uint64_t off = atomicAdd(&v.pool->bump, static_cast<unsigned long long>(bump_bytes));
    const uint64_t cap = v.pool->cap, base = v.pool->base;
    for (uint32_t b = nb; b < need; ++b) {
      if (!((miss >> b) & 1ull)) continue;
      const uint64_t sz = alloc_bytes_for(bucket_len(b, v.log2B) * v.E);
      if (off + sz > cap) break;
      tab[b] = base + off;
      off += sz;
    }
  }
  uint32_t got = nb;
  while (got < need && tab[got] != 0) ++got;
  return got;
}

// grow_buckets by a whole warp (every lane calls it with the same
// arguments): lane i takes bucket nb + i (+32, ...), so the queue pops of an
// LFVector's buckets are in flight together instead of one after another;
// the misses get one bump of the slab for all of them, in bucket order.
// Same result as grow_buckets (which queued bucket of a class a bucket gets
// may differ; contents, sizes and capacities do not).
__device__ inline uint32_t grow_buckets_warp(const ArrayView& v, uint32_t l, uint32_t nb, uint32_t need) {
  const uint32_t lane = threadIdx.x & 31;
  uint64_t* tab = v.buckets + static_cast<uint64_t>(l) * kMaxBuckets;
  if (need > static_cast<uint32_t>(kMaxBuckets)) need = kMaxBuckets;
  uint32_t got = nb;
  bool open = true;   // the allocated prefix has not ended yet
  for (uint32_t b0 = nb; b0 < need; b0 += 32) {
    const uint32_t b = b0 + lane;
    const bool in = b < need;
    uint64_t a = in ? tab[b] : 0;
    const bool pop = in && a == 0;
    const uint64_t sz = pop ? alloc_bytes_for(bucket_len(b, v.log2B) * v.E) : 0;
    if (pop) a = ring_pop(v.pool, class_of(bucket_len(b, v.log2B) * v.E));
    const uint64_t mb = (pop && a == 0) ? sz : 0;
    const uint64_t incl = warp_incl_scan(mb);
    const uint64_t total = __shfl_sync(0xffffffffu, incl, 31);
    if (total) {
      uint64_t off0 = 0;
      if (lane == 0) off0 = atomicAdd(&v.pool->bump, static_cast<unsigned long long>(total));
      off0 = __shfl_sync(0xffffffffu, off0, 0);
      if (mb) {
        const uint64_t off = off0 + incl - mb;   // bucket order; once one does not fit, none after it does
        if (off + mb <= v.pool->cap) a = v.pool->base + off;
      }
    }
    if (pop && a) tab[b] = a;
    const uint32_t present = __ballot_sync(0xffffffffu, in && a != 0);
    const uint32_t inmask = __ballot_sync(0xffffffffu, in);
    if (open) {
      const uint32_t gap = ~present & inmask;
      if (gap) {
        got = b0 + static_cast<uint32_t>(__ffs(static_cast<int>(gap)) - 1);
        open = false;
      } else {
        got = b0 + static_cast<uint32_t>(__popc(inmask));
      }
    }
  }
  return got;
}

// ---------------------------------------------------------------------------
// Device API.

// The thread's rank in its block (x fastest, then y, then z: the order in
// which the hardware forms warps) and the block's thread count.
__device__ __forceinline__ uint32_t block_rank() {
  return threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
}

__device__ __forceinline__ uint32_t block_threads() { return blockDim.x * blockDim.y * blockDim.z; }

// push_back of Algorithm 1 for a whole block: thread t appends `count`
// elements value_of_k(0), ..., value_of_k(count - 1) to LFVector l, after the
// elements of threads 0..t-1 of this call (the prefix sum of Sec. III-B) and
// after everything pushed before.  All threads of the block call it with
// the same l.  Returns true when the block's elements were appended (the
// same value in every thread); `first`, if given, receives the thread's
// first LFVector-local index (meaningful when count > 0).
template <class T, class F>
__device__ bool block_push_back(const ArrayView* view, uint32_t l, uint32_t count, F value_of_k,
                                uint64_t* first = nullptr) {
  __shared__ unsigned long long s_warp[32];   // warp totals, then their exclusive prefix
  __shared__ unsigned long long s_base;
  __shared__ uint32_t s_ok;
  const ArrayView& v = *view;
  if (l >= v.L || sizeof(T) != v.E) {   // block-uniform: every thread leaves here
    if (block_rank() == 0) latch_error(v.status, GGA_ERR_INVALID);
    return false;
  }
  const uint32_t nt = block_threads(), t = block_rank();
  const uint32_t lane = t & 31, w = t >> 5, nw = (nt + 31) >> 5;
  const uint32_t in_warp = nt - (w << 5) < 32 ? nt - (w << 5) : 32;   // lanes present in this warp
  const uint32_t mask = in_warp == 32 ? 0xffffffffu : (1u << in_warp) - 1u;

  // 1. Block exclusive scan of the counts (shuffles, then the warp totals).
  uint64_t x = count;
#pragma unroll
  for (uint32_t o = 1; o < 32; o <<= 1) {
    const uint64_t n = __shfl_up_sync(mask, x, o);
    if (lane >= o) x += n;
  }
  if (lane == in_warp - 1) s_warp[w] = x;
  __syncthreads();

  // 2. Warp 0: prefix of the warp totals, reservation (size_l += total) and
  //    the buckets the new run reaches (Algorithm 2).
  if (w == 0) {
    const uint64_t y = lane < nw ? s_warp[lane] : 0;
    uint64_t yi = y;
#pragma unroll
    for (uint32_t o = 1; o < 32; o <<= 1) {
      const uint64_t n = __shfl_up_sync(mask, yi, o);
      if (lane >= o) yi += n;
    }
    if (lane < nw) s_warp[lane] = yi - y;
    const uint64_t total = __shfl_sync(mask, yi, nw - 1);
    uint64_t base = 0;
    uint32_t nb = 0;
    if (lane == 0) {
      base = v.sizes[l];
      nb = v.nbuckets[l];
    }
    base = __shfl_sync(mask, base, 0);
    nb = __shfl_sync(mask, nb, 0);
    bool ok = true;
    if (total > 0) {
      const uint64_t end = base + total;
      const uint32_t need = end < base ? kMaxBuckets + 1u : buckets_for(end, v.log2B);
      if (need > nb) {
        uint32_t got;
        if (mask == 0xffffffffu && (blockDim.x & 31) == 0) {   // threadIdx.x & 31 is the lane
          got = grow_buckets_warp(v, l, nb, need);
        } else {
          got = 0;
          if (lane == 0) got = grow_buckets(v, l, nb, need);
          got = __shfl_sync(mask, got, 0);
        }
        ok = got >= need;
        if (lane == 0) {
          v.nbuckets[l] = got;
          if (!ok) latch_error(v.status, GGA_ERR_POOL_EXHAUSTED);
        }
      }
      if (lane == 0 && ok) v.sizes[l] = end;
    }
    if (lane == 0) {
      s_base = base;
      s_ok = ok ? 1u : 0u;
    }
  }
  __syncthreads();

  // 3. Every thread writes its run: bucket and offset of its first index,
  //    then onward through the buckets (a run crosses into the next bucket
  //    when it passes the end of one).
  const bool ok = s_ok != 0;
  const uint64_t j0 = s_base + s_warp[w] + (x - count);
  if (first) *first = j0;
  if (!ok) return false;
  if (count > 0) {
    const uint64_t* tab = v.buckets + static_cast<uint64_t>(l) * kMaxBuckets;
    uint32_t b;
    uint64_t off;
    bucket_of(j0, v.log2B, b, off);
    T* p = reinterpret_cast<T*>(tab[b]) + off;
    uint64_t left = bucket_len(b, v.log2B) - off;
    for (uint32_t k = 0; k < count; ++k) {
      if (left == 0) {
        ++b;
        p = reinterpret_cast<T*>(tab[b]);
        left = bucket_len(b, v.log2B);
      }
      *p++ = static_cast<T>(value_of_k(k));
      --left;
    }
  }
  return true;
}

// block_push_back into the block's own LFVector, l = blockIdx.x (the
// paper's one block per LFVector).
template <class T, class F>
__device__ bool block_push_back(const ArrayView* view, uint32_t count, F value_of_k, uint64_t* first = nullptr) {
  return block_push_back<T>(view, blockIdx.x, count, value_of_k, first);
}

// Capacity of the first nb buckets, B (2^nb - 1), saturating at 2^64 - 1.
__host__ __device__ __forceinline__ uint64_t prefix_capacity(uint32_t nb, uint32_t log2B) {
  return nb + log2B >= 64u ? ~0ull : bucket_first(nb, log2B);
}

// Shared memory of one BlockPusher (declare it __shared__, one per pusher).
struct PushShared {
  unsigned long long warp[2][32];   // warp totals, by call parity
  uint32_t nb[2];                   // allocated buckets after an allocating call
  uint32_t ok[2];                   // whether that call's buckets fit
};

// A block's cursor on one LFVector for many pushes in one kernel: the same
// appends as calling block_push_back once per push, with the LFVector's size
// and allocated capacity kept by every thread instead of re-read, and the
// shared scan slots alternating between calls, so a push that fits in the
// allocated buckets costs one block barrier; a push that reaches new
// buckets takes a second one (warp 0 allocates them, Algorithm 2).  Every
// thread of the block constructs it and calls push with the same sequence
// of calls.  While it is in use, the block pushes into LFVector l only
// through it (block_push_back on l would not be seen by the cursor).
//
//   __shared__ gga::PushShared sh;
//   gga::BlockPusher<uint32_t> p(view, l, sh);
//   for (...) p.push(count, [&](uint32_t k) { return value(k); });
template <class T>
struct BlockPusher {
  const ArrayView* view;
  PushShared* sh;
  uint64_t size, cap;
  uint32_t l, nb, par;
  bool valid;

  __device__ BlockPusher(const ArrayView* v, uint32_t lfv, PushShared& s)
      : view(v), sh(&s), size(0), cap(0), l(lfv), nb(0), par(0) {
    __syncthreads();   // this block's earlier writes to the LFVector are visible
    valid = lfv < v->L && sizeof(T) == v->E;
    if (!valid) {
      if (block_rank() == 0) latch_error(v->status, GGA_ERR_INVALID);
      return;
    }
    size = v->sizes[lfv];
    nb = v->nbuckets[lfv];
    cap = prefix_capacity(nb, v->log2B);
  }

  // Append count elements value_of_k(0..count-1) of this thread after those
  // of threads 0..t-1 of this call (block_push_back's order).  Returns true
  // (in every thread) when the block's elements were appended.
  template <class F>
  __device__ bool push(uint32_t count, F value_of_k, uint64_t* first = nullptr) {
    if (!valid) return false;
    const ArrayView& v = *view;
    const uint32_t nt = block_threads(), t = block_rank();
    const uint32_t lane = t & 31, w = t >> 5, nw = (nt + 31) >> 5;
    const uint32_t in_warp = nt - (w << 5) < 32 ? nt - (w << 5) : 32;
    const uint32_t mask = in_warp == 32 ? 0xffffffffu : (1u << in_warp) - 1u;
    const uint32_t pb = par;
    par ^= 1u;

    // 1. Warp scan of the counts (32-bit while a warp's sum cannot wrap).
    uint64_t x;
    if (__all_sync(mask, count < (1u << 26))) {
      uint32_t y = count;
#pragma unroll
      for (uint32_t o = 1; o < 32; o <<= 1) {
        const uint32_t n = __shfl_up_sync(mask, y, o);
        if (lane >= o) y += n;
      }
      x = y;
    } else {
      x = count;
#pragma unroll
      for (uint32_t o = 1; o < 32; o <<= 1) {
        const uint64_t n = __shfl_up_sync(mask, x, o);
        if (lane >= o) x += n;
      }
    }
    if (lane == in_warp - 1) sh->warp[pb][w] = x;
    __syncthreads();

    // 2. Every warp: the block total and its own offset from the warp totals.
    uint64_t total = 0, woff = 0;
    if (in_warp == 32) {
      const uint64_t y = lane < nw ? sh->warp[pb][lane] : 0;
      if (__all_sync(0xffffffffu, y < (1ull << 26))) {   // 32 of them cannot wrap 32 bits
        const uint32_t y32 = static_cast<uint32_t>(y);
        uint32_t yi = y32;
#pragma unroll
        for (uint32_t o = 1; o < 32; o <<= 1) {
          const uint32_t n = __shfl_up_sync(0xffffffffu, yi, o);
          if (lane >= o) yi += n;
        }
        total = __shfl_sync(0xffffffffu, yi, 31);
        woff = __shfl_sync(0xffffffffu, yi - y32, w);
      } else {
        uint64_t yi = y;
#pragma unroll
        for (uint32_t o = 1; o < 32; o <<= 1) {
          const uint64_t n = __shfl_up_sync(0xffffffffu, yi, o);
          if (lane >= o) yi += n;
        }
        total = __shfl_sync(0xffffffffu, yi, 31);
        woff = __shfl_sync(0xffffffffu, yi - y, w);
      }
    } else {
      for (uint32_t i = 0; i < nw; ++i) {
        const uint64_t y = sh->warp[pb][i];
        total += y;
        if (i < w) woff += y;
      }
    }

    // 3. Reservation.  All threads hold the same size and capacity, so they
    //    take the same branch.
    const uint64_t base = size;
    const uint64_t end = base + total;
    bool ok = true;
    if (end <= cap && end >= base) {
      size = end;
      if (t == 0 && total > 0) v.sizes[l] = end;
    } else {
      if (w == 0) {
        const uint32_t need = end < base ? kMaxBuckets + 1u : buckets_for(end, v.log2B);
        uint32_t got;
        if (mask == 0xffffffffu && (blockDim.x & 31) == 0) {
          got = grow_buckets_warp(v, l, nb, need);
        } else {
          got = 0;
          if (lane == 0) got = grow_buckets(v, l, nb, need);
          got = __shfl_sync(mask, got, 0);
        }
        if (lane == 0) {
          const bool fits = got >= need;
          v.nbuckets[l] = got;
          if (fits) v.sizes[l] = end;
          else latch_error(v.status, GGA_ERR_POOL_EXHAUSTED);
          sh->nb[pb] = got;
          sh->ok[pb] = fits ? 1u : 0u;
        }
      }
      __syncthreads();   // the buckets exist before any write
      nb = sh->nb[pb];
      cap = prefix_capacity(nb, v.log2B);
      ok = sh->ok[pb] != 0;
      if (ok) size = end;
    }

    // 4. Every thread writes its run.
    const uint64_t j0 = base + woff + (x - count);
    if (first) *first = j0;
    if (!ok) return false;
    if (count > 0) {
      const uint64_t* tab = v.buckets + static_cast<uint64_t>(l) * kMaxBuckets;
      uint32_t b;
      uint64_t off;
      bucket_of(j0, v.log2B, b, off);
      T* p = reinterpret_cast<T*>(tab[b]) + off;
      uint64_t left = bucket_len(b, v.log2B) - off;
      for (uint32_t k = 0; k < count; ++k) {
        if (left == 0) {
          ++b;
          p = reinterpret_cast<T*>(tab[b]);
          left = bucket_len(b, v.log2B);
        }
        *p++ = static_cast<T>(value_of_k(k));
        --left;
      }
    }
    return true;
  }

  // The LFVector's size as this cursor has it (the same in every thread).
  __device__ uint64_t lfv_size() const { return size; }
};

// Size of LFVector l (after the pushes of earlier calls in this kernel by
// the same block, or of earlier kernels).
__device__ __forceinline__ uint64_t lfv_size(const ArrayView* view, uint32_t l) { return view->sizes[l]; }

// Element j < lfv_size(view, l) of LFVector l.
template <class T>
__device__ __forceinline__ T& lfv_at(const ArrayView* view, uint32_t l, uint64_t j) {
  uint32_t b;
  uint64_t off;
  bucket_of(j, view->log2B, b, off);
  return reinterpret_cast<T*>(view->buckets[static_cast<uint64_t>(l) * kMaxBuckets + b])[off];
}

// Number of elements N and element g < N in the global (LFVector-major)
// order of Sec. IV.  Valid from gga_device_commit until the next growth;
// not in a kernel that pushes into the array.
__device__ __forceinline__ uint64_t global_size(const ArrayView* view) { return view->offsets[view->L]; }

template <class T>
__device__ __forceinline__ T& global_at(const ArrayView* view, uint64_t g) {
  const uint32_t l = find_lfv(view->offsets, view->L, view->offsets[view->L], g);
  return lfv_at<T>(view, l, g - view->offsets[l]);
}

}  // namespace gga

// The device view a user kernel receives (gga_device_view in gga.h).
typedef gga::ArrayView gga_dev_view;
