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
// Sweeps.

template <int E>
__device__ __forceinline__ typename Elem<E>::T add_rep(typename Elem<E>::T x, uint64_t delta, uint32_t repeats) {
  typedef typename Elem<E>::T T;
  for (uint32_t k = 0; k < repeats; ++k) x += static_cast<T>(delta);
  return x;
}

// rw_g: elements are visited by global index, one thread per element, each
// through the global translation (LFVector by the prefix sum of sizes, then
// bucket and offset).  A warp takes 32*U consecutive indices; lane 0's
// LFVector search is shared by the lanes whose index falls in the same
// LFVector, the others search for themselves.  U = 16 loads per lane are in
// flight before the first store, with many more blocks than are resident:
// the sweep is bound by how many bytes are in flight (measured on GB300:
// 0.69-0.75 ms for 2^28 int32 against 0.98 ms with U = 8 and one wave of
// blocks).
constexpr int kSweepGPerLane = 16;

template <int E>
__global__ void __launch_bounds__(256) sweep_g_kernel(ArrayView v, uint64_t delta, uint32_t repeats) {
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
static void write_as(const ArrayView& v, const uint64_t* idx, uint64_t n, const void* in, cudaStream_t st) {
  typedef typename Elem<E>::T T;
  write_kernel<E><<<rw_grid(n), 256, 0, st>>>(v, idx, n, static_cast<const T*>(in));
}

int launch_read(const ArrayView& v, const uint64_t* idx, uint64_t n, void* out, int num_sms, cudaStream_t st) {
  if (n == 0) return GGA_OK;
  (void)num_sms;
  if (v.E == 4) read_as<4>(v, idx, n, out, st);
  else if (v.E == 8) read_as<8>(v, idx, n, out, st);
  else read_as<16>(v, idx, n, out, st);
  return cudaGetLastError() == cudaSuccess ? GGA_OK : GGA_ERR_CUDA;
}

int launch_write(const ArrayView& v, const uint64_t* idx, uint64_t n, const void* in, int num_sms,
                 cudaStream_t st) {
  if (n == 0) return GGA_OK;
  (void)num_sms;
  if (v.E == 4) write_as<4>(v, idx, n, in, st);
  else if (v.E == 8) write_as<8>(v, idx, n, in, st);
  else write_as<16>(v, idx, n, in, st);
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
