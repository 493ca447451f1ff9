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
// block_push_back call; given a shared-memory stage it assembles each push
// there and writes it with aligned 128-bit stores (one more barrier).
// gga::block_push_rounds appends K rounds of pushes in one call (one
// reservation, three barriers, staged 128-bit stores): the form for
// kernels that can gather several rounds' counts before pushing.
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
  uint4* stage;          // shared memory for staged writes (two halves), or nullptr
  uint32_t half_elems;   // capacity of one half in elements (a multiple of 16 bytes)
  uint64_t size, cap;
  uint64_t pend_base;    // the staged push not yet written out: its first position,
  uint32_t pend_n;       //   its length (0: none)
  uint32_t pend_half;    //   and its half of the stage
  uint32_t l, nb, par;
  bool valid;

  // stage / stage_bytes (optional): a 16-byte aligned shared-memory buffer
  // owned by this pusher, used as two halves by alternate pushes.  With it,
  // a push whose run fits in a half is assembled there, and written out
  // with aligned 128-bit stores after the next push's first barrier (so
  // staging costs no barrier of its own); call flush() after the last push
  // (every thread), before anything reads the LFVector.  Without a stage,
  // or for a larger push, every thread stores its own elements.
  __device__ BlockPusher(const ArrayView* v, uint32_t lfv, PushShared& s, void* stage_smem = nullptr,
                         uint32_t stage_bytes = 0)
      : view(v), sh(&s), stage(static_cast<uint4*>(stage_smem)),
        half_elems(stage_smem ? (stage_bytes / 32u) * 16u / static_cast<uint32_t>(sizeof(T)) : 0u),
        size(0), cap(0), pend_base(0), pend_n(0), pend_half(0), l(lfv), nb(0), par(0) {
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
    write_pending();   // the previous push's stage is complete (barrier above)

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

    // 4. Every thread writes its run: into this push's half of the stage
    //    (written out by the next push or flush()), or straight to the
    //    buckets.  The half is next written two pushes later, after a
    //    barrier that every thread reaches only after its share of this
    //    write-out.
    const uint64_t j0 = base + woff + (x - count);
    if (first) *first = j0;
    if (!ok) return false;
    constexpr uint32_t VEC = 16 / sizeof(T);
    const uint32_t shv = static_cast<uint32_t>(base & (VEC - 1));
    if (stage && total > 0 && total + shv <= half_elems && v.B >= VEC) {   // block-uniform
      T* st = reinterpret_cast<T*>(stage) + static_cast<uint64_t>(pb) * half_elems;
      const uint32_t q0 = static_cast<uint32_t>(j0 - base) + shv;
      for (uint32_t k = 0; k < count; ++k) st[q0 + k] = static_cast<T>(value_of_k(k));
      pend_base = base;
      pend_n = static_cast<uint32_t>(total);
      pend_half = pb;
      return true;
    }
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

  // Writes out the staged push still pending (every thread calls it after
  // the last push; a no-op without a stage).
  __device__ void flush() {
    if (pend_n == 0) return;   // block-uniform
    __syncthreads();
    write_pending();
  }

  // The pending push's stage half goes to the buckets (block-wide, after a
  // barrier that follows its stage writes).
  __device__ void write_pending() {
    if (pend_n == 0) return;
    const ArrayView& v = *view;
    constexpr uint32_t VEC = 16 / sizeof(T);
    const uint32_t shv = static_cast<uint32_t>(pend_base & (VEC - 1));
    stage_to_buckets<T>(v.buckets + static_cast<uint64_t>(l) * kMaxBuckets, v.log2B, v.B, pend_base, pend_n, shv,
                        stage + static_cast<uint64_t>(pend_half) * (half_elems * sizeof(T) / 16u),
                        block_rank(), block_threads());
    pend_n = 0;
  }

  // The LFVector's size as this cursor has it (the same in every thread).
  __device__ uint64_t lfv_size() const { return size; }
};

// Shared memory of one RoundsPusher<T, K> (declare it __shared__, one per
// pusher).
template <int K>
struct RoundsShared {
  uint32_t wt[K][32];                  // per round, the warps' totals, then their offsets
  uint32_t rb[K + 1];                  // start of every round's run in the call; rb[K]: its total
  uint64_t tab[kMaxBuckets];           // the LFVector's bucket table (copy)
  uint32_t nb;                         // allocated buckets after the call
  uint32_t commit;                     // elements the call keeps
  uint32_t rounds;                     // rounds the call keeps
};

// A block's cursor on one LFVector for pushes of K rounds per call: call
// push(count, value_of) with every thread's counts of K rounds, and the
// block appends what K successive block_push_back calls would -- thread t
// pushes count[kr] elements value_of(kr, 0), ..., value_of(kr, count[kr]-1)
// in round kr: round-major, then thread, then k -- with one reservation for
// the K rounds (thread coarsening over rounds, Sec. III-B; Algorithm 1
// once per call).  A call takes three block barriers: warp 0 turns the
// warps' totals into offsets and reserves (allocating the buckets the run
// reaches, Algorithm 2) between the first two, the writes follow the
// second, the write-out the third.  With a shared-memory stage the call's run is assembled
// there and written with aligned 128-bit stores; without one (or when it
// does not fit) every thread stores its own elements.  `limit` caps the
// LFVector's size: positions at or past it are dropped (the clipping of a
// growth to a target).  A thread's count must stay below 2^26 and a call's
// elements below 2^32.  Every thread of the block constructs the cursor and
// makes the same calls; while it is in use the block pushes into LFVector l
// only through it.
//
//   __shared__ gga::RoundsShared<8> rs;
//   extern __shared__ uint4 stage[];
//   gga::RoundsPusher<uint32_t, 8> p(view, l, rs, stage, stage_bytes);
//   for (...) { uint32_t c[8] = ...; p.push(c, [&](uint32_t kr, uint32_t k) { ... }); }
template <class T, int K>
struct RoundsPusher {
  static_assert(K >= 1 && K <= 16, "1 to 16 rounds per call");
  static constexpr uint32_t VEC = 16 / sizeof(T);
  const ArrayView* view;
  RoundsShared<K>* sh;
  uint4* stage;
  uint32_t stage_elems;
  uint64_t size, cap, limit;
  uint32_t l, nb;
  bool valid;

  __device__ RoundsPusher(const ArrayView* v, uint32_t lfv, RoundsShared<K>& s, void* stage_smem = nullptr,
                          uint32_t stage_bytes = 0, uint64_t size_limit = ~0ull)
      : view(v), sh(&s), stage(static_cast<uint4*>(stage_smem)),
        stage_elems(stage_smem ? stage_bytes / static_cast<uint32_t>(sizeof(T)) : 0u),
        size(0), cap(0), limit(size_limit), l(lfv), nb(0) {
    __syncthreads();   // earlier users of the shared slots and of the LFVector are done
    valid = lfv < v->L && sizeof(T) == v->E;
    if (!valid) {
      if (block_rank() == 0) latch_error(v->status, GGA_ERR_INVALID);
      return;
    }
    size = v->sizes[lfv];
    nb = v->nbuckets[lfv];
    cap = prefix_capacity(nb, v->log2B);
    const uint64_t* tab = v->buckets + static_cast<uint64_t>(lfv) * kMaxBuckets;
    for (uint32_t i = block_rank(); i < nb; i += block_threads()) s.tab[i] = tab[i];
    __syncthreads();
  }

  // The LFVector's size as this cursor has it (the same in every thread).
  __device__ uint64_t lfv_size() const { return size; }

  // Returns the rounds appended (the same in every thread): K, or fewer when
  // the pool cannot hold the buckets of all K (the longest prefix of whole
  // rounds that fits is kept, GGA_ERR_POOL_EXHAUSTED is latched, and
  // buckets obtained beyond it stay with the LFVector).  *kept (optional)
  // receives the elements appended; first (optional) K slots with the
  // thread's first LFVector-local index of every round.
  //
  // CMAX > 0 promises count[k] <= CMAX (the fill loop is then unrolled).
  template <uint32_t CMAX = 0, class F>
  __device__ uint32_t push(const uint32_t (&count)[K], F value_of, uint32_t* kept = nullptr,
                           uint64_t* first = nullptr) {
    if (!valid) return 0;
    const ArrayView& v = *view;
    const uint32_t nt = block_threads(), t = block_rank();
    const uint32_t lane = t & 31, w = t >> 5, nw = (nt + 31) >> 5;
    const uint32_t in_warp = nt - (w << 5) < 32 ? nt - (w << 5) : 32;
    const uint32_t mask = in_warp == 32 ? 0xffffffffu : (1u << in_warp) - 1u;

    // 1. In-warp exclusive offsets per round: two rounds per 32-bit scan
    //    word while the warp's round sums fit 16 bits (counts < 2048).
    uint32_t q[K];
    uint32_t cmax = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) cmax = max(cmax, count[k]);
    if (__all_sync(mask, cmax < 2048u)) {
#pragma unroll
      for (int j = 0; j < (K + 1) / 2; ++j) {
        const int k1 = 2 * j + 1 < K ? 2 * j + 1 : 2 * j;
        const uint32_t word = count[2 * j] | (2 * j + 1 < K ? count[k1] << 16 : 0u);
        uint32_t inc = word;
#pragma unroll
        for (uint32_t o = 1; o < 32; o <<= 1) {
          const uint32_t n = __shfl_up_sync(mask, inc, o);
          if (lane >= o) inc += n;
        }
        q[2 * j] = (inc - word) & 0xFFFFu;
        if (2 * j + 1 < K) q[k1] = (inc - word) >> 16;
        if (lane == in_warp - 1) {
          sh->wt[2 * j][w] = inc & 0xFFFFu;
          if (2 * j + 1 < K) sh->wt[k1][w] = inc >> 16;
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        uint32_t inc = count[k];
#pragma unroll
        for (uint32_t o = 1; o < 32; o <<= 1) {
          const uint32_t n = __shfl_up_sync(mask, inc, o);
          if (lane >= o) inc += n;
        }
        q[k] = inc - count[k];
        if (lane == in_warp - 1) sh->wt[k][w] = inc;
      }
    }
    __syncthreads();

    // 2. Warp 0: the warps' offsets in every round (written back over their
    //    totals) and the rounds' starts (two rounds per scan word while the
    //    block's round sums fit 16 bits), then lane 0 reserves the call's
    //    run -- kept up to the limit -- and warp 0 allocates the buckets it
    //    reaches (Algorithm 2); the others wait at the barrier that follows.
    if (w == 0) {
      uint64_t rb = 0;
      if (in_warp == 32) {
        uint32_t ymax = 0;
#pragma unroll
        for (int k = 0; k < K; ++k) ymax = max(ymax, lane < nw ? sh->wt[k][lane] : 0u);
        if (__all_sync(0xffffffffu, ymax < 2048u)) {
#pragma unroll
          for (int j = 0; j < (K + 1) / 2; ++j) {
            const int k1 = 2 * j + 1 < K ? 2 * j + 1 : 2 * j;
            const uint32_t y0 = lane < nw ? sh->wt[2 * j][lane] : 0u;
            const uint32_t y1 = 2 * j + 1 < K && lane < nw ? sh->wt[k1][lane] : 0u;
            const uint32_t word = y0 | (y1 << 16);
            uint32_t inc = word;
#pragma unroll
            for (uint32_t o = 1; o < 32; o <<= 1) {
              const uint32_t n = __shfl_up_sync(0xffffffffu, inc, o);
              if (lane >= o) inc += n;
            }
            const uint32_t tot = __shfl_sync(0xffffffffu, inc, 31);
            if (lane < nw) {
              sh->wt[2 * j][lane] = static_cast<uint32_t>(rb) + ((inc - word) & 0xFFFFu);
              if (2 * j + 1 < K) sh->wt[k1][lane] = static_cast<uint32_t>(rb) + (tot & 0xFFFFu) + ((inc - word) >> 16);
            }
            if (lane == 0) {
              sh->rb[2 * j] = static_cast<uint32_t>(rb);
              if (2 * j + 1 < K) sh->rb[k1] = static_cast<uint32_t>(rb + (tot & 0xFFFFu));
            }
            rb += (tot & 0xFFFFu) + (2 * j + 1 < K ? (tot >> 16) : 0u);
          }
        } else {
#pragma unroll
          for (int k = 0; k < K; ++k) {
            const uint64_t y = lane < nw ? sh->wt[k][lane] : 0u;
            uint64_t inc = y;
#pragma unroll
            for (uint32_t o = 1; o < 32; o <<= 1) {
              const uint64_t n = __shfl_up_sync(0xffffffffu, inc, o);
              if (lane >= o) inc += n;
            }
            if (lane < nw) sh->wt[k][lane] = static_cast<uint32_t>(rb + inc - y);
            if (lane == 0) sh->rb[k] = static_cast<uint32_t>(rb);
            rb += __shfl_sync(0xffffffffu, inc, 31);
          }
        }
      } else if (lane == 0) {
        // Blocks of fewer than 32 threads: one warp, one lane does it.
#pragma unroll
        for (int k = 0; k < K; ++k) {
          sh->rb[k] = static_cast<uint32_t>(rb);
          const uint32_t y = sh->wt[k][0];
          sh->wt[k][0] = static_cast<uint32_t>(rb);
          rb += y;
        }
      }
      rb = __shfl_sync(mask, rb, 0);
      // Reservation: kept up to the limit; allocation when the kept run
      // passes the allocated capacity (warp-uniform branch).
      const uint64_t base = size;
      uint64_t commit = base >= limit ? 0 : (limit - base < rb ? limit - base : rb);
      uint32_t kr = K;
      uint32_t nb2 = nb;
      if (base + commit > cap) {
        const uint32_t need = buckets_for(base + commit, v.log2B);
        if (mask == 0xffffffffu && (blockDim.x & 31) == 0) {
          nb2 = grow_buckets_warp(v, l, nb, need);
        } else {
          nb2 = 0;
          if (lane == 0) nb2 = grow_buckets(v, l, nb, need);
          nb2 = __shfl_sync(mask, nb2, 0);
        }
        const uint64_t* tab = v.buckets + static_cast<uint64_t>(l) * kMaxBuckets;
        for (uint32_t i = nb + lane; i < nb2; i += in_warp) sh->tab[i] = tab[i];   // warp 0's lanes
        if (nb2 < need) {   // keep the longest prefix of whole rounds that fits
          __syncwarp(mask);
          const uint64_t capg = prefix_capacity(nb2, v.log2B);
          kr = 0;
          while (kr < static_cast<uint32_t>(K) &&
                 base + (kr + 1 < static_cast<uint32_t>(K) ? sh->rb[kr + 1] : rb) <= capg)
            ++kr;
          const uint64_t keep = kr < static_cast<uint32_t>(K) ? sh->rb[kr] : rb;
          if (keep < commit) commit = keep;
          if (lane == 0) latch_error(v.status, GGA_ERR_POOL_EXHAUSTED);
        }
        if (lane == 0) v.nbuckets[l] = nb2;
      }
      if (lane == 0) {
        if (commit > 0) v.sizes[l] = base + commit;
        sh->rb[K] = static_cast<uint32_t>(rb);
        sh->nb = nb2;
        sh->commit = static_cast<uint32_t>(commit);
        sh->rounds = kr;
      }
    }
    __syncthreads();   // synchronize(): the buckets exist before any write

    // 3. Every thread: the call's result, and its positions.
    const uint64_t base = size;
    const uint64_t total = sh->rb[K];
    const uint64_t commit = sh->commit;
    const uint32_t rounds = sh->rounds;
    if (sh->nb != nb) {
      nb = sh->nb;
      cap = prefix_capacity(nb, v.log2B);
    }
    size = base + commit;
#pragma unroll
    for (int k = 0; k < K; ++k) q[k] += sh->wt[k][w];

    // 4. Writes: into the stage at the run's positions, or to the buckets.
    const uint32_t shv = static_cast<uint32_t>(base & (VEC - 1));
    const uint32_t n = static_cast<uint32_t>(commit);
    const bool staged = n > 0 && n + shv <= stage_elems && v.B >= VEC;   // block-uniform
    const bool whole = n == total;                                       // nothing clipped
    T* st = reinterpret_cast<T*>(stage);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (first) first[k] = base + q[k];
      const uint32_t c = count[k];
      if (staged && whole && CMAX > 0) {
#pragma unroll
        for (uint32_t m = 0; m + 1 <= CMAX; ++m)
          if (m < c) st[q[k] + m + shv] = static_cast<T>(value_of(static_cast<uint32_t>(k), m));
      } else if (staged && whole) {
        for (uint32_t m = 0; m < c; ++m) st[q[k] + m + shv] = static_cast<T>(value_of(static_cast<uint32_t>(k), m));
      } else {
        for (uint32_t m = 0; m < c; ++m) {
          const uint32_t p = q[k] + m;
          if (p >= n) break;
          const T x = static_cast<T>(value_of(static_cast<uint32_t>(k), m));
          if (staged) {
            st[p + shv] = x;
          } else {
            uint32_t b;
            uint64_t off;
            bucket_of(base + p, v.log2B, b, off);
            reinterpret_cast<T*>(sh->tab[b])[off] = x;
          }
        }
      }
    }
    // Every thread is past its reads of sh->wt before the next call writes
    // them, and the stage is complete before it is written out; the next
    // call writes the stage only after its own first barrier.
    __syncthreads();
    if (staged) stage_to_buckets<T>(sh->tab, v.log2B, v.B, base, n, shv, stage, t, nt);
    if (kept) *kept = n;
    return rounds;
  }
};

// One call of K rounds without a cursor: the same appends as
// RoundsPusher<T, K>::push on a cursor made for this call (the LFVector's
// size is read from the array; shared slots of the function's own).  Every
// thread of the block calls it with the same l.  Returns the rounds
// appended (0 for l >= L or sizeof(T) != E, GGA_ERR_INVALID latched).
template <class T, int K, class F>
__device__ uint32_t block_push_rounds(const ArrayView* view, uint32_t l, const uint32_t (&count)[K], F value_of,
                                      void* stage_smem = nullptr, uint32_t stage_bytes = 0,
                                      uint64_t* first = nullptr) {
  __shared__ RoundsShared<K> s;
  RoundsPusher<T, K> p(view, l, s, stage_smem, stage_bytes);
  return p.push(count, value_of, nullptr, first);
}

// block_push_rounds into the block's own LFVector, l = blockIdx.x.
template <class T, int K, class F>
__device__ uint32_t block_push_rounds(const ArrayView* view, const uint32_t (&count)[K], F value_of,
                                      void* stage_smem = nullptr, uint32_t stage_bytes = 0,
                                      uint64_t* first = nullptr) {
  return block_push_rounds<T, K>(view, blockIdx.x, count, value_of, stage_smem, stage_bytes, first);
}

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
