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
// A kernel launched with blocks of up to 1024 threads should say so
// (__launch_bounds__(1024)) so that the compiler keeps it within the
// register file.
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
// The view, the pool, the bucket math and the allocation these calls use
// are in gga_layout.cuh, shared with the library's own kernels.
#pragma once

#include "gga_layout.cuh"

namespace gga {

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
