// gga_access.cu -- element access over a GGArray.
//
//  * read / write (rw_g addressing, Sec. VI-B): global index g -> LFVector
//    l with offsets[l] <= g < offsets[l+1] (search over the prefix sum of
//    sizes, Sec. IV, started from a proportional guess) -> local
//    j = g - offsets[l] -> (bucket, offset) by the clz formula -> element.
//  * sweep (Sec. VI-C's r/w operation, +delta `repeats` times):
//      rw_g: one thread per element through the global index translation;
//      rw_b: bucket by bucket (the block structure), 16 KB chunks, 128-bit
//            loads and stores, no search.
//  * flatten: every 16 KB chunk of live bucket data is fetched into shared
//    memory with a TMA bulk copy (cp.async.bulk, mbarrier completion, four
//    stages in flight per block) and written to its place in the contiguous
//    destination -- by a TMA bulk store when the destination is 16-byte
//    aligned, otherwise by realigned 128-bit stores.
#include "gga_core.cuh"

namespace gga {


// ---------------------------------------------------------------------------
// Global index translation.

// Address of global element g < N (Sec. IV index translation, Algorithm 2
// bucket sizes).
__device__ __forceinline__ uint64_t element_addr(const ArrayView& v, uint64_t N, uint64_t g) {
  const uint32_t l = find_lfv(v.offsets, v.L, N, g);
  uint32_t b;
  uint64_t o;
  bucket_of(g - __ldg(v.offsets + l), v.log2B, b, o);
  return __ldg(v.buckets + static_cast<uint64_t>(l) * kMaxBuckets + b) + o * v.E;
}

// Random reads and writes.  Every access is one dependent DRAM burst, so the
// rate of bursts in flight decides the time: a full grid (one pass over the
// indices, 4 per thread) keeps more of them in flight than a persistent
// grid-stride loop (measured on GB300: 1.40 vs 1.76 ms for 2^26 int32
// reads, the same as a flat gather of the same indices).
constexpr int kRwPerThread = 4;

template <int E>
__global__ void __launch_bounds__(256) read_kernel(ArrayView v, const uint64_t* __restrict__ idx, uint64_t n,
                                                   typename Elem<E>::T* __restrict__ out) {
  typedef typename Elem<E>::T T;
  constexpr int U = kRwPerThread;
  const uint64_t N = __ldg(v.offsets + v.L);
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  bool bad = false;
  for (uint64_t i0 = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i0 < n; i0 += stride * U) {
    uint64_t g[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t i = i0 + u * stride;
      g[u] = i < n ? __ldcs(idx + i) : 0;
      if (i < n && g[u] >= N) bad = true;
    }
    uint64_t addr[U];
#pragma unroll
    for (int u = 0; u < U; ++u) addr[u] = (i0 + u * stride < n && g[u] < N) ? element_addr(v, N, g[u]) : 0;
    T x[U];
#pragma unroll
    for (int u = 0; u < U; ++u) x[u] = addr[u] ? *reinterpret_cast<const T*>(addr[u]) : T();
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t i = i0 + u * stride;
      if (i < n) __stcs(out + i, x[u]);
    }
  }
  if (bad) latch_error(v.status, GGA_ERR_OUT_OF_RANGE);
}

template <int E>
__global__ void __launch_bounds__(256) write_kernel(ArrayView v, const uint64_t* __restrict__ idx, uint64_t n,
                                                    const typename Elem<E>::T* __restrict__ in) {
  typedef typename Elem<E>::T T;
  constexpr int U = kRwPerThread;
  const uint64_t N = __ldg(v.offsets + v.L);
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  bool bad = false;
  for (uint64_t i0 = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i0 < n; i0 += stride * U) {
    uint64_t g[U];
    T x[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t i = i0 + u * stride;
      g[u] = ~0ull;
      if (i < n) {
        g[u] = __ldcs(idx + i);
        x[u] = __ldcs(in + i);
        if (g[u] >= N) bad = true;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (g[u] < N) *reinterpret_cast<T*>(element_addr(v, N, g[u])) = x[u];
  }
  if (bad) latch_error(v.status, GGA_ERR_OUT_OF_RANGE);
}

// ---------------------------------------------------------------------------
// Binned random writes (large batches).
//
// A random 4-byte store makes the L2 fetch the 32-byte sector it lands in and
// write the whole sector back; with ~2 writes per sector (2^26 writes into
// 2^28 int32) most of that traffic is paid twice.  A large batch is therefore
// first grouped by ranges of global indices ("bins" of ~8 MB of elements) and
// then applied bin after bin, so the writes that share a sector meet while it
// is held in L2: each touched sector is fetched and written back once.
//   count:   per-bin totals (block histogram over the tiles the block takes,
//            one global atomic per bin per block)
//   scan:    bin cursors = exclusive scan of the totals; totals reset
//   scatter: a tile of writes is sorted by bin in shared memory (counting
//            sort) and written as runs of (offset inside the bin, value) into
//            the bins: 4 + E bytes per write instead of 8 + E
//   apply:   each pair's global index (its bin, found from the bin ends, and
//            the offset) is translated to an element address and the value
//            stored, in bin order, each bin's memory streamed into L2 by bulk
//            prefetches issued a few bins ahead
// Writes with the same index keep one of their values, as in the direct path.
// Measured on GB300 for 2^26 int32 writes: 1.22 ms binned (1.41 ms with
// 64-bit global indices in the bins, 1.71 ms without the prefetch either)
// against 2.0-2.6 ms for a direct scatter (flat array, same indices).

constexpr uint32_t kWbinMaxBins = 256;
constexpr uint64_t kWbinMin = 1ull << 20;        // smaller batches write directly
constexpr uint64_t kWbinHeader = 4096;           // totals[256] u32 | cursors[256] u64 | valid u64
constexpr int kWbinThreads = 256;

// The bins hold, per write, the element's offset inside its bin (32 bits:
// a bin spans at most 2^32 elements, 2^shift with shift <= 32 for any array
// below 2^40 elements) and then, 256-byte aligned, the values.
uint64_t wbin_values_offset(uint64_t n) { return (kWbinHeader + n * 4 + 255) & ~255ull; }

template <int E> struct WbinTile { static constexpr int kPer = 16; };
template <> struct WbinTile<16> { static constexpr int kPer = 8; };
// Writes per thread in the apply (its own tiles): measured on GB300 for 2^26
// int32 writes, write phase 1.190 ms at 8, 1.204 ms at 16, 1.299 ms at 32.
template <int E> struct WbinApplyPer { static constexpr int kPer = 8; };

// Bin of global index g: g >> shift, with 2^shift elements ~ 8 MB, raised
// until at most kWbinMaxBins bins cover [0, N).
__device__ __forceinline__ uint32_t wbin_shift(uint64_t N, uint32_t E) {
  uint32_t s = 23 - (31 - __clz(static_cast<int>(E)));
  while (N > 0 && ((N - 1) >> s) >= kWbinMaxBins) ++s;
  return s;
}

__device__ __forceinline__ uint32_t* wbin_totals(uint8_t* scr) { return reinterpret_cast<uint32_t*>(scr); }
__device__ __forceinline__ unsigned long long* wbin_cursors(uint8_t* scr) {
  return reinterpret_cast<unsigned long long*>(scr + 1024);
}
__device__ __forceinline__ unsigned long long* wbin_valid(uint8_t* scr) {
  return reinterpret_cast<unsigned long long*>(scr + 3072);
}

template <int E>
__global__ void __launch_bounds__(kWbinThreads) wbin_count_kernel(ArrayView v, const uint64_t* __restrict__ idx,
                                                                  uint64_t n, uint8_t* scr) {
  constexpr int kPer = WbinTile<E>::kPer;
  __shared__ uint32_t h[kWbinMaxBins];
  const uint64_t N = __ldg(v.offsets + v.L);
  const uint32_t shift = wbin_shift(N, E);
  for (uint32_t b = threadIdx.x; b < kWbinMaxBins; b += blockDim.x) h[b] = 0;
  __syncthreads();
  bool bad = false;
  // Tiles of kWbinThreads * kPer indices, taken by the blocks in turn: a
  // tile's indices are all loaded before any is counted.
  const uint64_t tile = static_cast<uint64_t>(kWbinThreads) * kPer;
  for (uint64_t base = static_cast<uint64_t>(blockIdx.x) * tile; base < n;
       base += static_cast<uint64_t>(gridDim.x) * tile) {
    uint64_t g[kPer];
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const uint64_t i = base + static_cast<uint64_t>(u) * kWbinThreads + threadIdx.x;
      g[u] = i < n ? __ldcs(idx + i) : ~0ull;
    }
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      if (g[u] < N) atomicAdd(&h[static_cast<uint32_t>(g[u] >> shift)], 1u);
      else if (g[u] != ~0ull) bad = true;
    }
  }
  if (bad) latch_error(v.status, GGA_ERR_OUT_OF_RANGE);
  __syncthreads();
  uint32_t* tot = wbin_totals(scr);
  for (uint32_t b = threadIdx.x; b < kWbinMaxBins; b += blockDim.x)
    if (h[b]) atomicAdd(tot + b, h[b]);
}

// One block of kWbinMaxBins threads, one bin each.
__global__ void __launch_bounds__(kWbinMaxBins) wbin_scan_kernel(uint8_t* scr) {
  __shared__ uint64_t wsum[kWbinMaxBins / 32];
  uint32_t* tot = wbin_totals(scr);
  const uint64_t c = tot[threadIdx.x];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint64_t sc = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t t = __shfl_up_sync(0xffffffffu, sc, o);
    if (lane >= o) sc += t;
  }
  if (lane == 31) wsum[w] = sc;
  __syncthreads();
  uint64_t add = 0;
  for (int k = 0; k < w; ++k) add += wsum[k];
  wbin_cursors(scr)[threadIdx.x] = sc - c + add;
  tot[threadIdx.x] = 0;   // ready for the next batch
  if (threadIdx.x == kWbinMaxBins - 1) *wbin_valid(scr) = sc + add;
}

template <int E>
__global__ void __launch_bounds__(kWbinThreads) wbin_scatter_kernel(ArrayView v, const uint64_t* __restrict__ idx,
                                                                    const typename Elem<E>::T* __restrict__ in,
                                                                    uint64_t n, uint8_t* scr, uint32_t* out_off,
                                                                    typename Elem<E>::T* out_val) {
  typedef typename Elem<E>::T T;
  constexpr int kPer = WbinTile<E>::kPer;
  constexpr int kTile = kWbinThreads * kPer;
  __shared__ uint32_t h[kWbinMaxBins];
  __shared__ uint32_t off[kWbinMaxBins];
  __shared__ unsigned long long gbase[kWbinMaxBins];
  __shared__ uint32_t wsum[kWbinThreads / 32];
  extern __shared__ __align__(16) uint8_t s_dyn[];
  T* s_val = reinterpret_cast<T*>(s_dyn);
  uint32_t* s_off = reinterpret_cast<uint32_t*>(s_dyn + static_cast<size_t>(kTile) * E);
  uint8_t* s_bin = s_dyn + static_cast<size_t>(kTile) * (4 + E);
  const uint64_t N = __ldg(v.offsets + v.L);
  const uint32_t shift = wbin_shift(N, E);
  if (shift > 32) {   // bins past 2^32 elements: arrays of 2^40 elements and more
    if (blockIdx.x == 0 && threadIdx.x == 0) latch_error(v.status, GGA_ERR_INVALID);
    return;
  }
  for (uint32_t b = threadIdx.x; b < kWbinMaxBins; b += blockDim.x) h[b] = 0;
  __syncthreads();
  const uint64_t base = static_cast<uint64_t>(blockIdx.x) * kTile;
  uint64_t g[kPer];
  T x[kPer];
  uint32_t rank[kPer];
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const uint64_t i = base + static_cast<uint64_t>(u) * kWbinThreads + threadIdx.x;
    g[u] = ~0ull;
    if (i < n) {
      g[u] = __ldcs(idx + i);
      x[u] = __ldcs(in + i);
      if (g[u] >= N) g[u] = ~0ull;
    }
  }
#pragma unroll
  for (int u = 0; u < kPer; ++u)
    rank[u] = g[u] != ~0ull ? atomicAdd(&h[static_cast<uint32_t>(g[u] >> shift)], 1u) : 0u;
  __syncthreads();
  {
    // Exclusive scan of the tile's bin counts (one bin per thread) and one
    // reservation per non-empty bin in the global bin arrays.
    const uint32_t c = h[threadIdx.x];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t sc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, sc, o);
      if (lane >= o) sc += t;
    }
    if (lane == 31) wsum[w] = sc;
    __syncthreads();
    uint32_t add = 0;
    for (int k = 0; k < w; ++k) add += wsum[k];
    off[threadIdx.x] = sc - c + add;
    if (c) gbase[threadIdx.x] = atomicAdd(wbin_cursors(scr) + threadIdx.x, static_cast<unsigned long long>(c));
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    if (g[u] == ~0ull) continue;
    const uint32_t b = static_cast<uint32_t>(g[u] >> shift);
    const uint32_t p = off[b] + rank[u];
    s_off[p] = static_cast<uint32_t>(g[u] - (static_cast<uint64_t>(b) << shift));
    s_val[p] = x[u];
    s_bin[p] = static_cast<uint8_t>(b);
  }
  __syncthreads();
  const uint32_t valid = off[kWbinMaxBins - 1] + h[kWbinMaxBins - 1];
  for (uint32_t p = threadIdx.x; p < valid; p += blockDim.x) {
    const uint32_t b = s_bin[p];
    const unsigned long long q = gbase[b] + (p - off[b]);
    out_off[q] = s_off[p];
    out_val[q] = s_val[p];
  }
}

// Brings the array's elements of global indices [g0, g1) into L2, by warp
// 0 of the block (every lane calls it): lane i walks LFVectors l0 + i,
// l0 + i + 32, ... of the range (l0 found once), one bulk prefetch per run
// (one bucket of one LFVector), widened to 16-byte boundaries inside the
// bucket's allocation.
template <int E>
__device__ void prefetch_range_l2_warp(const ArrayView& v, uint64_t N, uint64_t g0, uint64_t g1) {
  const uint32_t lane = threadIdx.x & 31;
  uint32_t l0 = 0;
  if (lane == 0) l0 = find_lfv(v.offsets, v.L, N, g0);
  l0 = __shfl_sync(0xffffffffu, l0, 0);
  constexpr uint64_t kMaxPrefetch = static_cast<uint64_t>(1) << 30;
  for (uint32_t l = l0 + lane; l < v.L; l += 32) {
    const uint64_t lo = __ldg(v.offsets + l), hi = __ldg(v.offsets + l + 1);
    if (lo >= g1) break;   // offsets ascend: so do the later LFVectors of this lane
    uint64_t j = (g0 > lo ? g0 : lo) - lo;
    const uint64_t jend = (g1 < hi ? g1 : hi) - lo;
    while (j < jend) {
      uint32_t b;
      uint64_t o;
      bucket_of(j, v.log2B, b, o);
      const uint64_t run = min(bucket_len(b, v.log2B) - o, jend - j);
      const uint64_t base = __ldg(v.buckets + static_cast<uint64_t>(l) * kMaxBuckets + b);
      const uint64_t a0 = (base + o * E) & ~15ull, a1 = (base + (o + run) * E + 15) & ~15ull;
      for (uint64_t a = a0; a < a1; a += kMaxPrefetch)
        bulk_prefetch_l2(reinterpret_cast<const void*>(a),
                         static_cast<uint32_t>(a1 - a < kMaxPrefetch ? a1 - a : kMaxPrefetch));
      j += run;
    }
  }
}

// Bins fetched ahead: the block whose tile holds the first write of bin b
// prefetches the bin kWbinAheadBytes of array further on (blocks 0, 1, ...
// the bins before it, one each), so that a bin's sectors come from DRAM as
// one stream instead of one random fill per first write to each.  Measured on
// GB300 for 2^26 int32 writes into 2^28 elements (8 MB bins; write phase,
// ranges walked by one thread): no prefetch 1.71 ms, 2 bins ahead 1.65, 4
// 1.59, 8 1.53-1.55, 12 1.64, 16 1.79, 24 2.13 (the bins then no longer stay
// in the 129 MB L2 until their writes arrive); 8 bins walked by warp 0:
// 1.44-1.46 ms.
constexpr uint64_t kWbinAheadBytes = 64ull << 20;

template <int E>
__global__ void __launch_bounds__(kWbinThreads) wbin_apply_kernel(ArrayView v, const uint32_t* __restrict__ goff,
                                                                  const typename Elem<E>::T* __restrict__ val,
                                                                  uint8_t* scr) {
  typedef typename Elem<E>::T T;
  constexpr int kPer = WbinApplyPer<E>::kPer;
  const uint64_t total = *wbin_valid(scr);
  const uint64_t N = __ldg(v.offsets + v.L);
  if (threadIdx.x < 32 && N > 0) {   // warp 0: the prefetches of this tile
    const uint32_t shift = wbin_shift(N, E);
    const uint32_t nbins = static_cast<uint32_t>(((N - 1) >> shift) + 1);
    const uint64_t bin_bytes = static_cast<uint64_t>(E) << shift;
    const uint32_t ahead = bin_bytes >= kWbinAheadBytes ? 1u : static_cast<uint32_t>(kWbinAheadBytes / bin_bytes);
    // Blocks 0 .. ahead - 1 fetch the first bins, one each.
    if (blockIdx.x < ahead && blockIdx.x < nbins)
      prefetch_range_l2_warp<E>(v, N, static_cast<uint64_t>(blockIdx.x) << shift,
                                min(static_cast<uint64_t>(blockIdx.x + 1) << shift, N));
    const unsigned long long* ends = wbin_cursors(scr);   // advanced to the bin ends by the scatter
    const uint64_t t0 = static_cast<uint64_t>(blockIdx.x) * kWbinThreads * kPer;
    const uint64_t t1 = t0 + static_cast<uint64_t>(kWbinThreads) * kPer;
    // First bin starting at or after t0 (bin starts ascend): binary search.
    uint32_t lo = 0, hi = nbins;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if ((mid ? ends[mid - 1] : 0) < t0) lo = mid + 1;
      else hi = mid;
    }
    for (uint32_t b = lo; b < nbins; ++b) {
      const uint64_t start = b ? ends[b - 1] : 0;
      if (start >= t1) break;
      const uint32_t pb = b + ahead;   // this tile holds bin b's first write
      if (ends[b] != start && pb < nbins)
        prefetch_range_l2_warp<E>(v, N, static_cast<uint64_t>(pb) << shift, min(static_cast<uint64_t>(pb + 1) << shift, N));
    }
  }
  if (N == 0) return;
  const uint32_t shift = wbin_shift(N, E);
  const uint32_t nbins = static_cast<uint32_t>(((N - 1) >> shift) + 1);
  const unsigned long long* ends = wbin_cursors(scr);   // advanced to the bin ends by the scatter
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * kWbinThreads * kPer;
  for (uint64_t base = static_cast<uint64_t>(blockIdx.x) * kWbinThreads * kPer; base < total; base += stride) {
    uint32_t o[kPer];
    T x[kPer];
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const uint64_t i = base + static_cast<uint64_t>(u) * kWbinThreads + threadIdx.x;
      o[u] = 0;
      if (i < total) {
        o[u] = __ldcs(goff + i);
        x[u] = __ldcs(val + i);
      }
    }
    // The bin of the tile's first write (lane 0 searches the bin ends while
    // the loads above are in flight); a write's bin is that one or, past its
    // end, one of the next (the tile's writes are in bin order).
    uint32_t bf = 0;
    if (lane == 0) {
      uint32_t lo = 0, hi = nbins;
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (ends[mid] <= base) lo = mid + 1;
        else hi = mid;
      }
      bf = lo;
    }
    uint32_t b = __shfl_sync(0xffffffffu, bf, 0);
    unsigned long long e = ends[b];   // the thread's positions ascend with u: b only moves forward
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const uint64_t i = base + static_cast<uint64_t>(u) * kWbinThreads + threadIdx.x;
      if (i < total) {
        while (i >= e) e = ends[++b];
        const uint64_t g = (static_cast<uint64_t>(b) << shift) + o[u];
        *reinterpret_cast<T*>(element_addr(v, N, g)) = x[u];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Sweeps.

template <int E>
__device__ __forceinline__ typename Elem<E>::T add_rep(typename Elem<E>::T x, uint64_t delta, uint32_t repeats) {
  typedef typename Elem<E>::T T;
  for (uint32_t k = 0; k < repeats; ++k) x += static_cast<T>(delta);
  return x;
}

// rw_g: elements are visited by global index, one thread per element, each
// through the global translation (LFVector by the prefix sum of sizes, then
// bucket and offset).  A warp takes 32*U consecutive indices; lane 0 finds
// the LFVector of the first.  When all of them lie in that LFVector (the
// usual case: LFVectors hold far more than 32*U elements) every element
// takes its bucket and offset by the clz formula and its bucket address
// from the table in 32-bit arithmetic; otherwise each element is placed on
// its own (LFVector search included).  U = 16 loads per lane are in flight
// before the first store, with many more blocks than are resident: the
// sweep is bound by how many bytes are in flight and by the instructions
// per element (measured on GB300 for 2^28 int32: 0.63 ms with the 64-bit
// per-element path alone, 0.37 ms with the 32-bit path at three blocks per
// SM, 0.40 ms at four, where registers spill).
constexpr int kSweepGPerLane = 16;

template <int E>
__global__ void __launch_bounds__(256, E == 4 ? 3 : 2) sweep_g_kernel(ArrayView v, uint64_t delta, uint32_t repeats) {
  typedef typename Elem<E>::T T;
  constexpr int U = kSweepGPerLane;
  const uint64_t N = __ldg(v.offsets + v.L);
  const int lane = threadIdx.x & 31;
  const uint64_t warps = static_cast<uint64_t>(gridDim.x) * (blockDim.x >> 5);
  for (uint64_t wbase = (static_cast<uint64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32 * U;
       wbase < N; wbase += warps * 32 * U) {
    uint32_t l0 = 0;
    if (lane == 0) l0 = find_lfv(v.offsets, v.L, N, wbase);
    l0 = __shfl_sync(0xffffffffu, l0, 0);
    const uint64_t lo = __ldg(v.offsets + l0), hi = __ldg(v.offsets + l0 + 1);
    T* addr[U];
    if (wbase + 32 * U <= hi && hi - lo <= 0xFFFFFFFFull - (1ull << v.log2B)) {
      // Warp-uniform: all the warp's indices lie in LFVector l0, whose
      // positions (plus B) fit in 32 bits.  Every element still takes its
      // own bucket and offset (the clz formula) and its own bucket-table
      // entry, in 32-bit arithmetic.
      const uint64_t* tab = v.buckets + static_cast<uint64_t>(l0) * kMaxBuckets;
      const uint32_t B = 1u << v.log2B;
      const uint32_t x0 = static_cast<uint32_t>(wbase - lo) + static_cast<uint32_t>(lane) + B;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint32_t x = x0 + 32u * u;
        const uint32_t hb = 31u - static_cast<uint32_t>(__clz(static_cast<int>(x)));
        addr[u] = reinterpret_cast<T*>(__ldg(tab + (hb - v.log2B))) + (x - (1u << hb));
      }
    } else {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint64_t g = wbase + lane + 32 * u;
        addr[u] = nullptr;
        if (g < N) {
          const uint32_t l = (g >= lo && g < hi) ? l0 : find_lfv(v.offsets, v.L, N, g);
          uint32_t b;
          uint64_t o;
          bucket_of(g - __ldg(v.offsets + l), v.log2B, b, o);
          addr[u] = reinterpret_cast<T*>(__ldg(v.buckets + static_cast<uint64_t>(l) * kMaxBuckets + b)) + o;
        }
      }
    }
    T x[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (addr[u]) x[u] = *addr[u];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (addr[u]) *addr[u] = add_rep<E>(x[u], delta, repeats);
  }
}

// Cursor over the 16 KB chunks of live bucket data, in (LFVector, bucket,
// chunk) order: the work list of flatten and rw_b.
struct ChunkCursor {
  uint32_t l, b;
  uint64_t cib;        // chunk index inside bucket b
  uint64_t size;       // size of LFVector l
  uint64_t blen_bytes; // live bytes of bucket b
  uint64_t baddr;      // address of bucket b
};

__device__ __forceinline__ void cursor_load_bucket(const ArrayView& v, ChunkCursor& c) {
  const uint64_t first = bucket_first(c.b, v.log2B);
  uint64_t len = bucket_len(c.b, v.log2B);
  if (c.size - first < len) len = c.size - first;
  c.blen_bytes = len * v.E;
  c.baddr = v.buckets[static_cast<uint64_t>(c.l) * kMaxBuckets + c.b];
}

// Position the cursor at global chunk w (w < fl_prefix[L]).
__device__ inline void cursor_seek(const ArrayView& v, ChunkCursor& c, uint64_t w) {
  c.l = upper_bound_u64(v.fl_prefix, v.L + 1, w) - 1;
  uint64_t k = w - v.fl_prefix[c.l];
  c.size = v.sizes[c.l];
  c.b = 0;
  while (true) {
    cursor_load_bucket(v, c);
    const uint64_t nch = (c.blen_bytes + kChunkBytes - 1) / kChunkBytes;
    if (k < nch) break;
    k -= nch;
    ++c.b;
  }
  c.cib = k;
}

__device__ inline void cursor_next(const ArrayView& v, ChunkCursor& c) {
  ++c.cib;
  if (c.cib * kChunkBytes < c.blen_bytes) return;
  c.cib = 0;
  ++c.b;
  if (bucket_first(c.b, v.log2B) < c.size) {
    cursor_load_bucket(v, c);
    return;
  }
  // next non-empty LFVector
  c.b = 0;
  do {
    ++c.l;
    if (c.l >= v.L) return;
    c.size = v.sizes[c.l];
  } while (c.size == 0);
  cursor_load_bucket(v, c);
}

// rw_b: each block sweeps a contiguous range of chunks.
template <int E>
__global__ void __launch_bounds__(256) sweep_b_kernel(ArrayView v, uint64_t delta, uint32_t repeats) {
  typedef typename Elem<E>::T T;
  constexpr uint32_t VEC = 16 / E;
  const uint64_t total = v.fl_prefix[v.L];
  const uint64_t ipb = (total + gridDim.x - 1) / gridDim.x;
  const uint64_t w0 = static_cast<uint64_t>(blockIdx.x) * ipb;
  const uint64_t w1 = min(total, w0 + ipb);
  if (w0 >= w1) return;
  ChunkCursor c;
  cursor_seek(v, c, w0);
  for (uint64_t w = w0; w < w1; ++w) {
    const uint64_t start = c.cib * kChunkBytes;
    const uint32_t bytes = static_cast<uint32_t>(min(static_cast<uint64_t>(kChunkBytes), c.blen_bytes - start));
    uint8_t* p = reinterpret_cast<uint8_t*>(c.baddr) + start;
    const uint32_t nvec = bytes / 16;
    constexpr int U = kChunkBytes / 16 / 256;
    uint4 x[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t i = threadIdx.x + u * 256;
      if (i < nvec) x[u] = __ldcs(reinterpret_cast<const uint4*>(p) + i);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t i = threadIdx.x + u * 256;
      if (i < nvec) {
        T* e = reinterpret_cast<T*>(&x[u]);
#pragma unroll
        for (uint32_t k = 0; k < VEC; ++k) e[k] = add_rep<E>(e[k], delta, repeats);
        __stcs(reinterpret_cast<uint4*>(p) + i, x[u]);
      }
    }
    // tail (< 16 bytes)
    const uint32_t tail = (bytes - nvec * 16) / E;
    if (threadIdx.x < tail) {
      T* e = reinterpret_cast<T*>(p + nvec * 16) + threadIdx.x;
      *e = add_rep<E>(*e, delta, repeats);
    }
    cursor_next(v, c);
  }
}

// ---------------------------------------------------------------------------
// Flatten with TMA bulk copies.

constexpr int kFlStages = 4;
constexpr int kFlThreads = 128;

template <int E>
__global__ void __launch_bounds__(kFlThreads) flatten_kernel(ArrayView v, uint8_t* __restrict__ dst,
                                                             uint64_t cap_elems) {
  typedef typename Elem<E>::T T;
  constexpr uint32_t VEC = 16 / E;
  extern __shared__ __align__(128) uint8_t s_buf[];      // kFlStages * kChunkBytes
  __shared__ __align__(8) uint64_t s_full[kFlStages];
  __shared__ uint64_t s_dst[kFlStages];
  __shared__ uint32_t s_len[kFlStages];

  const uint64_t N = v.offsets[v.L];
  if (N > cap_elems) {
    if (blockIdx.x == 0 && threadIdx.x == 0) latch_error(v.status, GGA_ERR_DST_TOO_SMALL);
    return;
  }
  const uint64_t total = v.fl_prefix[v.L];
  const uint64_t ipb = (total + gridDim.x - 1) / gridDim.x;
  const uint64_t w0 = static_cast<uint64_t>(blockIdx.x) * ipb;
  const uint64_t w1 = min(total, w0 + ipb);
  if (w0 >= w1) return;
  const uint32_t n_items = static_cast<uint32_t>(w1 - w0);
  const uint32_t tid = threadIdx.x;

  ChunkCursor c;
  uint64_t dst_l = 0;   // destination element index of LFVector c.l's first element
  if (tid == 0) {
    for (int s = 0; s < kFlStages; ++s) mbar_init(&s_full[s], 1);
    fence_mbar_init();
    cursor_seek(v, c, w0);
    dst_l = v.offsets[c.l];
  }
  __syncthreads();

  // Producer (thread 0): issue the bulk load of the cursor's chunk into stage s.
  auto issue = [&](int s) {
    const uint64_t start = c.cib * kChunkBytes;
    const uint32_t bytes = static_cast<uint32_t>(min(static_cast<uint64_t>(kChunkBytes), c.blen_bytes - start));
    const uint32_t bytes16 = (bytes + 15u) & ~15u;   // stays inside the bucket's allocation
    s_len[s] = bytes;
    s_dst[s] = reinterpret_cast<uint64_t>(dst) + (dst_l + bucket_first(c.b, v.log2B)) * E + start;
    mbar_arrive_expect_tx(&s_full[s], bytes16);
    bulk_g2s(s_buf + static_cast<size_t>(s) * kChunkBytes, reinterpret_cast<const void*>(c.baddr + start), bytes16,
             &s_full[s]);
    const uint32_t l_before = c.l;
    cursor_next(v, c);
    if (c.l != l_before && c.l < v.L) dst_l = v.offsets[c.l];
  };

  if (tid == 0) {
    fence_proxy_async_smem();
    for (uint32_t i = 0; i < n_items && i < static_cast<uint32_t>(kFlStages); ++i) issue(static_cast<int>(i));
  }

  uint32_t consumed = 0;
  bool failed = false;
  for (uint32_t i = 0; i < n_items; ++i) {
    const int s = static_cast<int>(i % kFlStages);
    const uint32_t ph = (i / kFlStages) & 1u;
    const bool ok = mbar_wait_bounded(&s_full[s], ph);
    if (!__syncthreads_and(ok)) {
      failed = true;
      break;
    }
    consumed = i + 1;
    const uint64_t dp = s_dst[s];
    const uint32_t bytes = s_len[s];
    const uint8_t* sb = s_buf + static_cast<size_t>(s) * kChunkBytes;
    if ((dp & 15u) == 0) {
      const uint32_t body = bytes & ~15u;
      if (tid == 0 && body) {
        bulk_s2g(reinterpret_cast<void*>(dp), sb, body);
        bulk_commit();
      }
      const uint32_t tail = (bytes - body) / E;
      if (tid < tail)
        reinterpret_cast<T*>(dp + body)[tid] = reinterpret_cast<const T*>(sb + body)[tid];
    } else {
      // Realign: head elements up to the 16-byte boundary, then 128-bit stores.
      const uint32_t n = bytes / E;
      const uint32_t head = min(n, static_cast<uint32_t>((16u - (dp & 15u)) & 15u) / E);
      const T* se = reinterpret_cast<const T*>(sb);
      T* de = reinterpret_cast<T*>(dp);
      if (tid < head) de[tid] = se[tid];
      const uint32_t nvec = (n - head) / VEC;
      for (uint32_t vi = tid; vi < nvec; vi += kFlThreads) {
        Vec16<E> x;
#pragma unroll
        for (uint32_t e = 0; e < VEC; ++e) x.e[e] = se[head + vi * VEC + e];
        __stcs(reinterpret_cast<uint4*>(de + head) + vi, x.v);
      }
      const uint32_t done = head + nvec * VEC;
      if (tid < n - done) de[done + tid] = se[done + tid];
    }
    __syncthreads();   // stage s consumed by generic-proxy reads
    if (tid == 0 && i + kFlStages < n_items) {
      bulk_wait_read_all();   // a bulk store from stage s has finished reading it
      fence_proxy_async_smem();
      issue(s);
    }
  }
  if (tid == 0) {
    if (failed) {
      latch_error(v.status, GGA_ERR_TIMEOUT);
      // Wait (bounded) for every load still in flight before leaving.
      const uint32_t issued = min(n_items, consumed + static_cast<uint32_t>(kFlStages));
      for (uint32_t i = consumed; i < issued; ++i)
        mbar_wait_bounded(&s_full[i % kFlStages], (i / kFlStages) & 1u);
    }
    bulk_wait_all();
  }
}

// ---------------------------------------------------------------------------
// Clear, capacities, accounting.

// Every bucket (live or spare) goes back to the queue of its index.
__global__ void clear_kernel(ArrayView v) {
  const uint64_t gt = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const uint64_t l = gt / kMaxBuckets;
  const uint32_t b = static_cast<uint32_t>(gt % kMaxBuckets);
  if (l >= v.L) return;
  uint64_t* slot = v.buckets + l * kMaxBuckets + b;
  const uint64_t a = *slot;
  if (a) {
    if (!ring_push(v.pool, class_of(bucket_len(b, v.log2B) * v.E), a)) latch_error(v.status, GGA_ERR_INVALID);
    *slot = 0;
  }
}

__global__ void clear_sizes_kernel(ArrayView v) {
  const uint64_t l = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (l < v.L) {
    v.nbuckets[l] = 0;
    v.sizes[l] = 0;
  }
  if (l <= v.L) {
    v.offsets[l] = 0;
    v.fl_prefix[l] = 0;
  }
}

__global__ void caps_kernel(ArrayView v, uint64_t* caps) {
  const uint64_t l = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (l < v.L) caps[l] = bucket_first(v.nbuckets[l], v.log2B);
}

__global__ void memory_kernel(ArrayView v, unsigned long long* out) {
  const uint64_t l = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  uint64_t bb = 0, live = 0;
  if (l < v.L) {
    bb = bucket_first(v.nbuckets[l], v.log2B) * v.E;
    live = v.sizes[l] * v.E;
  }
  bb = warp_sum_u64(bb);
  live = warp_sum_u64(live);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&out[0], static_cast<unsigned long long>(bb));
    atomicAdd(&out[1], static_cast<unsigned long long>(live));
  }
}

// ---------------------------------------------------------------------------
// Launchers.


// Grid of one full wave: the blocks that fit on all SMs at once (grid-stride
// kernels then give every block the same share), but no more than the work.
template <typename K>
static unsigned wave_grid(K kern, int threads, size_t smem, int num_sms, uint64_t work_blocks) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  const uint64_t wave = static_cast<uint64_t>(num_sms) * per_sm;
  return static_cast<unsigned>(work_blocks < 1 ? 1 : (work_blocks < wave ? work_blocks : wave));
}

// One pass: every thread takes kRwPerThread indices (grid capped at 2^31 - 1
// blocks; beyond that the kernels stride).
static unsigned rw_grid(uint64_t n) {
  const uint64_t per_block = 256ull * kRwPerThread;
  const uint64_t blocks = (n + per_block - 1) / per_block;
  return static_cast<unsigned>(blocks < 1 ? 1 : (blocks > 0x7FFFFFFFull ? 0x7FFFFFFFull : blocks));
}

template <int E>
static void read_as(const ArrayView& v, const uint64_t* idx, uint64_t n, void* out, cudaStream_t st) {
  typedef typename Elem<E>::T T;
  read_kernel<E><<<rw_grid(n), 256, 0, st>>>(v, idx, n, static_cast<T*>(out));
}

template <int E>
static void write_as(const ArrayView& v, const uint64_t* idx, uint64_t n, const void* in, void* scratch,
                     cudaStream_t st) {
  typedef typename Elem<E>::T T;
  if (!scratch || n < kWbinMin) {
    write_kernel<E><<<rw_grid(n), 256, 0, st>>>(v, idx, n, static_cast<const T*>(in));
    return;
  }
  constexpr int kTile = kWbinThreads * WbinTile<E>::kPer;
  uint8_t* scr = static_cast<uint8_t*>(scratch);
  uint32_t* out_off = reinterpret_cast<uint32_t*>(scr + kWbinHeader);
  T* out_val = reinterpret_cast<T*>(scr + wbin_values_offset(n));
  const uint64_t tiles = (n + kTile - 1) / kTile;
  const unsigned grid = static_cast<unsigned>(tiles > 0x7FFFFFFFull ? 0x7FFFFFFFull : tiles);
  const int smem = kTile * (4 + E + 1);
  cudaFuncSetAttribute(wbin_scatter_kernel<E>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  // The count runs 4 blocks per SM that take the tiles in turn (one set of
  // global bin additions per block): measured on GB300 for 2^26 int32
  // writes, write phase 1.408 ms against 1.460 ms with one block per tile.
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  const uint64_t cgrid_cap = static_cast<uint64_t>(sms) * 4;
  const unsigned cgrid = grid > cgrid_cap ? static_cast<unsigned>(cgrid_cap) : grid;
  wbin_count_kernel<E><<<cgrid, kWbinThreads, 0, st>>>(v, idx, n, scr);
  wbin_scan_kernel<<<1, kWbinMaxBins, 0, st>>>(scr);
  wbin_scatter_kernel<E><<<grid, kWbinThreads, smem, st>>>(v, idx, static_cast<const T*>(in), n, scr, out_off,
                                                           out_val);
  constexpr int kTileA = kWbinThreads * WbinApplyPer<E>::kPer;
  const uint64_t tiles_a = (n + kTileA - 1) / kTileA;
  const unsigned grid_a = static_cast<unsigned>(tiles_a > 0x7FFFFFFFull ? 0x7FFFFFFFull : tiles_a);
  wbin_apply_kernel<E><<<grid_a, kWbinThreads, 0, st>>>(v, out_off, out_val, scr);
}

int launch_read(const ArrayView& v, const uint64_t* idx, uint64_t n, void* out, int num_sms, cudaStream_t st) {
  if (n == 0) return GGA_OK;
  (void)num_sms;
  if (v.E == 4) read_as<4>(v, idx, n, out, st);
  else if (v.E == 8) read_as<8>(v, idx, n, out, st);
  else read_as<16>(v, idx, n, out, st);
  return cudaGetLastError() == cudaSuccess ? GGA_OK : GGA_ERR_CUDA;
}

uint64_t wbin_scratch_bytes(uint64_t n, uint32_t E) {
  return n < kWbinMin ? 0 : wbin_values_offset(n) + n * E;
}

int launch_write(const ArrayView& v, const uint64_t* idx, uint64_t n, const void* in, int num_sms, void* scratch,
                 cudaStream_t st) {
  if (n == 0) return GGA_OK;
  (void)num_sms;
  if (v.E == 4) write_as<4>(v, idx, n, in, scratch, st);
  else if (v.E == 8) write_as<8>(v, idx, n, in, scratch, st);
  else write_as<16>(v, idx, n, in, scratch, st);
  return cudaGetLastError() == cudaSuccess ? GGA_OK : GGA_ERR_CUDA;
}

template <int E>
static void sweep_as(const ArrayView& v, int mode, uint64_t delta, uint32_t repeats, int num_sms,
                     cudaStream_t st) {
  if (mode == GGA_RW_G) {
    // The size is on the device, so the grid cannot follow it: 32 blocks per
    // SM (several times what is resident at once) stride over the array.
    sweep_g_kernel<E><<<static_cast<unsigned>(num_sms) * 32u, 256, 0, st>>>(v, delta, repeats);
  } else {
    const unsigned grid = wave_grid(sweep_b_kernel<E>, 256, 0, num_sms, ~0ull);
    sweep_b_kernel<E><<<grid, 256, 0, st>>>(v, delta, repeats);
  }
}

int launch_sweep(const ArrayView& v, int mode, uint64_t delta, uint32_t repeats, int num_sms, cudaStream_t st) {
  if (v.E == 4) sweep_as<4>(v, mode, delta, repeats, num_sms, st);
  else sweep_as<8>(v, mode, delta, repeats, num_sms, st);
  return cudaGetLastError() == cudaSuccess ? GGA_OK : GGA_ERR_CUDA;
}

int launch_flatten(const ArrayView& v, void* dst, uint64_t cap_elems, int num_sms, cudaStream_t st) {
  const size_t smem = static_cast<size_t>(kFlStages) * kChunkBytes;
  const unsigned grid = static_cast<unsigned>(num_sms) * 3;
  uint8_t* d = static_cast<uint8_t*>(dst);
#define GGA_FL(EE)                                                                                          \
  do {                                                                                                      \
    cudaFuncSetAttribute(flatten_kernel<EE>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)); \
    flatten_kernel<EE><<<grid, kFlThreads, smem, st>>>(v, d, cap_elems);                                   \
  } while (0)
  if (v.E == 4) GGA_FL(4);
  else if (v.E == 8) GGA_FL(8);
  else GGA_FL(16);
#undef GGA_FL
  return cudaGetLastError() == cudaSuccess ? GGA_OK : GGA_ERR_CUDA;
}

int launch_clear(const ArrayView& v, cudaStream_t st) {
  const uint64_t n = static_cast<uint64_t>(v.L) * kMaxBuckets;
  clear_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(v);
  clear_sizes_kernel<<<static_cast<unsigned>((v.L + 1 + 255) / 256), 256, 0, st>>>(v);
  return cudaGetLastError() == cudaSuccess ? GGA_OK : GGA_ERR_CUDA;
}

int launch_caps(const ArrayView& v, uint64_t* caps, cudaStream_t st) {
  caps_kernel<<<(v.L + 255) / 256, 256, 0, st>>>(v, caps);
  return cudaGetLastError() == cudaSuccess ? GGA_OK : GGA_ERR_CUDA;
}

int launch_memory(const ArrayView& v, uint64_t* out2, cudaStream_t st) {
  memory_kernel<<<(v.L + 255) / 256, 256, 0, st>>>(v, reinterpret_cast<unsigned long long*>(out2));
  return cudaGetLastError() == cudaSuccess ? GGA_OK : GGA_ERR_CUDA;
}

}  // namespace gga
