// gga_serve.cu -- request batches over many live arrays (continuous batching).
//
// A serving loop gathers requests that arrived while earlier work ran and
// launches them together: one kernel appends to many arrays (one block per
// (request, LFVector): one reservation, the buckets it reaches from the
// shared pool, then aligned 128-bit writes of the new elements), one kernel
// reads random indices of many arrays.  The requests travel as kernel
// parameters, so nothing on the host must outlive the call.
//
// Appended values are self-describing: element k of LFVector l appended by
// a request with tag g is g * 2^24 + l * 2^20 + k (an append places n / L
// elements in every LFVector, one more in the first n % L).
#include <algorithm>
#include <vector>

#include "gga_gen.cuh"

namespace gga {
namespace {

constexpr int kServeMax = 480;       // requests per launch (kernel parameters stay below 32 KB)
constexpr int kServeThreads = 256;

struct AppendParams {
  uint32_t n_req;
  uint32_t pad;
  PoolState* pool;
  const ArrayView* view[kServeMax];
  uint64_t n[kServeMax];
  uint64_t tag[kServeMax];
  uint32_t block0[kServeMax + 1];   // first block of every request (prefix of L)
};

struct ReadParams {
  uint32_t n_req;
  uint32_t pad;
  const ArrayView* view[kServeMax];
  uint64_t n[kServeMax];
  uint64_t seed[kServeMax];
  void* out[kServeMax];
};

template <int E>
__device__ void append_run(const ArrayView& v, uint32_t l, uint64_t base, uint64_t c, uint64_t tag) {
  typedef typename Elem<E>::T T;
  constexpr uint32_t VEC = 16 / E;
  const uint64_t* bk = v.buckets + static_cast<uint64_t>(l) * kMaxBuckets;
  const uint64_t vbase = tag * (1ull << 24) + static_cast<uint64_t>(l) * (1ull << 20);
  const uint64_t end = base + c;
  const uint64_t gbeg = base & ~static_cast<uint64_t>(VEC - 1);
  const bool group_ok = v.B >= VEC;
  for (uint64_t p = gbeg + static_cast<uint64_t>(threadIdx.x) * VEC; p < end; p += static_cast<uint64_t>(blockDim.x) * VEC) {
    if (group_ok && p >= base && p + VEC <= end) {
      Vec16<E> x;
#pragma unroll
      for (uint32_t e = 0; e < VEC; ++e) x.e[e] = gen_value<E>(vbase + (p + e - base));
      uint32_t bb;
      uint64_t off;
      bucket_of(p, v.log2B, bb, off);
      __stcs(reinterpret_cast<uint4*>(bk[bb] + off * E), x.v);
    } else {
      for (uint32_t e = 0; e < VEC; ++e) {
        const uint64_t pe = p + e;
        if (pe < base || pe >= end) continue;
        uint32_t bb;
        uint64_t off;
        bucket_of(pe, v.log2B, bb, off);
        *reinterpret_cast<T*>(bk[bb] + off * E) = gen_value<E>(vbase + (pe - base));
      }
    }
  }
}

__global__ void __launch_bounds__(kServeThreads) append_batch_kernel(const __grid_constant__ AppendParams P) {
  __shared__ uint64_t s_base, s_len;
  // Which request and LFVector this block serves.
  uint32_t lo = 0, hi = P.n_req;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (P.block0[mid] <= blockIdx.x) lo = mid; else hi = mid;
  }
  const uint32_t r = lo;
  const ArrayView& v = *P.view[r];
  const uint32_t l = blockIdx.x - P.block0[r];
  const uint64_t c = P.n[r] / v.L + (l < P.n[r] % v.L ? 1 : 0);
  if (threadIdx.x == 0) {
    // One reservation for the LFVector's share, Algorithm 2 for its buckets.
    const uint64_t base = v.sizes[l];
    uint64_t len = c;
    if (c) {
      const uint32_t nb = v.nbuckets[l];
      const uint32_t need = buckets_for(base + c, v.log2B);
      if (need > nb) {
        const uint32_t got = grow_buckets(v, l, nb, need);
        v.nbuckets[l] = got;
        if (got < need) {
          len = 0;   // the append does not fit: this LFVector takes none of it
          latch_error(v.status, GGA_ERR_POOL_EXHAUSTED);
        }
      }
    }
    v.sizes[l] = base + len;
    s_base = base;
    s_len = len;
  }
  __syncthreads();   // synchronize(): buckets exist before any write
  if (s_len == 0) return;
  switch (v.E) {
    case 4: append_run<4>(v, l, s_base, s_len, P.tag[r]); break;
    case 8: append_run<8>(v, l, s_base, s_len, P.tag[r]); break;
    default: append_run<16>(v, l, s_base, s_len, P.tag[r]); break;
  }
}

__global__ void serve_fixup_kernel(PoolState* pool) { ring_fixup(pool); }

__global__ void __launch_bounds__(256) serve_finalize_kernel(const __grid_constant__ AppendParams P) {
  __shared__ uint64_t s_warp[33];
  finalize_block(*P.view[blockIdx.x], nullptr, nullptr, nullptr, 1, s_warp);
}

template <int E>
__device__ void read_run(const ArrayView& v, uint64_t n, uint64_t seed, void* out) {
  typedef typename Elem<E>::T T;
  T* o = static_cast<T*>(out);
  const uint64_t N = v.offsets[v.L];
  for (uint64_t k = threadIdx.x; k < n; k += blockDim.x) {
    T x = T();
    if (N) {
      const uint64_t g = ((splitmix(seed, k) >> 32) * N) >> 32;   // uniform over [0, N)
      const uint32_t l = upper_bound_u64(v.offsets, v.L + 1, g) - 1;
      uint32_t b;
      uint64_t off;
      bucket_of(g - v.offsets[l], v.log2B, b, off);
      x = *reinterpret_cast<const T*>(v.buckets[static_cast<uint64_t>(l) * kMaxBuckets + b] + off * E);
    }
    o[k] = x;
  }
}

__global__ void __launch_bounds__(kServeThreads) read_batch_kernel(const __grid_constant__ ReadParams P) {
  const ArrayView& v = *P.view[blockIdx.x];
  switch (v.E) {
    case 4: read_run<4>(v, P.n[blockIdx.x], P.seed[blockIdx.x], P.out[blockIdx.x]); break;
    case 8: read_run<8>(v, P.n[blockIdx.x], P.seed[blockIdx.x], P.out[blockIdx.x]); break;
    default: read_run<16>(v, P.n[blockIdx.x], P.seed[blockIdx.x], P.out[blockIdx.x]); break;
  }
}

}  // namespace
}  // namespace gga

extern "C" {

int gga_append_batch(const gga_append_req* reqs, uint32_t n, void* stream) {
  if (n == 0) return GGA_OK;
  if (!reqs) return GGA_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  gga::PoolState* pool = gga::handle_pool(reqs[0].array);
  std::vector<gga_handle> seen;
  seen.reserve(n);
  for (uint32_t i = 0; i < n; ++i) {
    if (!reqs[i].array || gga::handle_pool(reqs[i].array) != pool) return GGA_ERR_INVALID;
    gga::ArrayView v;
    gga::InsertScratch s;
    int dev, sms;
    gga::handle_parts(reqs[i].array, &v, &s, &dev, &sms);
    if (reqs[i].n / v.L >= (1ull << 20)) return GGA_ERR_INVALID;   // value layout holds k < 2^20
    seen.push_back(reqs[i].array);
  }
  std::sort(seen.begin(), seen.end());
  if (std::adjacent_find(seen.begin(), seen.end()) != seen.end()) return GGA_ERR_INVALID;   // one request per array

  for (uint32_t i0 = 0; i0 < n; i0 += gga::kServeMax) {
    const uint32_t m = std::min<uint32_t>(gga::kServeMax, n - i0);
    gga::AppendParams P;
    P.n_req = m;
    P.pad = 0;
    P.pool = pool;
    uint32_t blocks = 0;
    for (uint32_t j = 0; j < m; ++j) {
      gga::ArrayView v;
      gga::InsertScratch s;
      int dev, sms;
      gga::handle_parts(reqs[i0 + j].array, &v, &s, &dev, &sms);
      P.view[j] = gga::handle_dview(reqs[i0 + j].array);
      P.n[j] = reqs[i0 + j].n;
      P.tag[j] = reqs[i0 + j].tag;
      P.block0[j] = blocks;
      blocks += v.L;
    }
    P.block0[m] = blocks;
    gga::append_batch_kernel<<<blocks, gga::kServeThreads, 0, st>>>(P);
    gga::serve_fixup_kernel<<<1, 1, 0, st>>>(pool);
    gga::serve_finalize_kernel<<<m, 256, 0, st>>>(P);
  }
  return cudaGetLastError() == cudaSuccess ? GGA_OK : GGA_ERR_CUDA;
}

int gga_read_batch(const gga_read_req* reqs, uint32_t n, void* stream) {
  if (n == 0) return GGA_OK;
  if (!reqs) return GGA_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (uint32_t i0 = 0; i0 < n; i0 += gga::kServeMax) {
    const uint32_t m = std::min<uint32_t>(gga::kServeMax, n - i0);
    gga::ReadParams P;
    P.n_req = m;
    P.pad = 0;
    for (uint32_t j = 0; j < m; ++j) {
      const gga_read_req& q = reqs[i0 + j];
      if (!q.array || (q.n && !q.out)) return GGA_ERR_INVALID;
      P.view[j] = gga::handle_dview(q.array);
      P.n[j] = q.n;
      P.seed[j] = q.seed;
      P.out[j] = q.out;
    }
    gga::read_batch_kernel<<<m, gga::kServeThreads, 0, st>>>(P);
  }
  return cudaGetLastError() == cudaSuccess ? GGA_OK : GGA_ERR_CUDA;
}

}  // extern "C"
