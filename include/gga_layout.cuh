// gga_layout.cuh -- the GB300 GGArray's data in HBM and the device-side
// operations on it that every kernel shares: the array's view, the device
// pool, the bucket index math (Algorithm 2), the search over the prefix sum
// of LFVector sizes (Sec. IV) and bucket allocation (Algorithm 1's
// new_bucket, without the host).  Included by the library's kernels and by
// the device API (gga_device.cuh), which is what user kernels include.
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
// Staged writes (the write step of Algorithm 1 when a block's run of
// consecutive LFVector positions has been assembled in shared memory).
// stage holds positions base - shv .. base + n - 1 of LFVector l, position
// base + q at stage element q + shv, with shv = base mod (16 / sizeof(T));
// the whole block calls it after a barrier that follows the stage writes.
// Every 16-byte group of positions inside the run goes out as one aligned
// 128-bit store (a group never straddles buckets when B is a multiple of
// 16 / sizeof(T), and buckets start on 256-byte boundaries); the partial
// groups at the run's ends go element by element.  The buckets are those
// of `tab` (the LFVector's bucket table), already allocated.  Each thread
// keeps the bucket its last group fell in (first position, end, address)
// and looks the table up again only when its positions pass that bucket's
// end.

template <class T>
__device__ __forceinline__ void stage_to_buckets(const uint64_t* tab, uint32_t log2B, uint64_t B, uint64_t base,
                                                 uint32_t n, uint32_t shv, const uint4* stage4, uint32_t t,
                                                 uint32_t nt) {
  constexpr uint32_t VEC = 16 / sizeof(T);
  const T* stage = reinterpret_cast<const T*>(stage4);
  const bool group_ok = B >= VEC;
  const uint64_t gbeg = base - shv;
  const uint32_t nvec = (n + shv + VEC - 1) / VEC;
  uint64_t cfirst = 0, cend = 0, caddr = 0;   // the bucket of this thread's last group
  for (uint32_t vi = t; vi < nvec; vi += nt) {
    const uint64_t p = gbeg + static_cast<uint64_t>(vi) * VEC;
    const uint32_t lo = vi * VEC;   // stage index of position p
    if (group_ok && lo >= shv && lo + VEC <= n + shv) {
      if (p < cfirst || p >= cend) {
        uint32_t bb;
        uint64_t off;
        bucket_of(p, log2B, bb, off);
        cfirst = p - off;
        cend = cfirst + bucket_len(bb, log2B);
        caddr = tab[bb];
      }
      __stcs(reinterpret_cast<uint4*>(caddr + (p - cfirst) * sizeof(T)), stage4[vi]);
    } else {
#pragma unroll
      for (uint32_t e = 0; e < VEC; ++e) {
        const uint32_t si = lo + e;
        if (si < shv || si >= n + shv) continue;
        uint32_t bb;
        uint64_t off;
        bucket_of(p + e, log2B, bb, off);
        *reinterpret_cast<T*>(tab[bb] + off * sizeof(T)) = stage[si];
      }
    }
  }
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

}  // namespace gga
