// gga_serve.cu -- request batches over many live arrays (continuous batching).
//
// A serving loop gathers requests that arrived while earlier work ran and
// launches them together.  An append batch is two kernels: one block per
// request reserves every LFVector's share (one size update, the buckets it
// reaches from the shared pool) and recomputes the array's offsets; then
// blocks of 16K elements each write the new elements with aligned 128-bit
// stores, so a large append spreads over the GPU instead of holding one
// block per LFVector.  One kernel reads random indices of many arrays.  The
// requests travel as kernel parameters, so nothing on the host must outlive
// the call; the reservations go to a small record array of the pool.
//
// Appended values are self-describing: element k of LFVector l appended by
// a request with tag g is g * 2^24 + l * 2^20 + k (an append places n / L
// elements in every LFVector, one more in the first n % L).
#include <algorithm>
#include <vector>

#include "gga_gen.cuh"

namespace gga {
namespace {

constexpr int kServeMax = 480;         // requests per launch (kernel parameters stay below 32 KB)
constexpr int kServeThreads = 256;
constexpr uint32_t kServeSlots = 8192; // (request, LFVector) pairs per launch: one reservation record each
constexpr uint64_t kAppendChunk = 16384;   // elements one block of the write kernel stores

struct AppendParams {
  uint32_t n_req;
  uint32_t pad;
  uint64_t* res_base;               // per (request, LFVector): first reserved index
  uint64_t* res_len;                // and the number of elements it got (0 if the pool was short)
  const ArrayView* view[kServeMax];
  uint64_t n[kServeMax];
  uint64_t tag[kServeMax];
  uint32_t slot0[kServeMax + 1];    // first reservation record of every request (prefix of L)
  uint32_t chunk0[kServeMax + 1];   // first write block of every request (prefix of L * per_lfv)
  uint32_t per_lfv[kServeMax];      // write blocks per LFVector of the request
};

struct ReadParams {
  uint32_t n_req;
  uint32_t pad;
  const ArrayView* view[kServeMax];
  uint64_t n[kServeMax];
  uint64_t seed[kServeMax];
  void* out[kServeMax];
};

// Stores elements [start, start + cnt) of LFVector l, element p taking the
// value vfirst + (p - start); 16-byte groups inside the range go as one
// aligned 128-bit store (B >= 16 / E keeps a group inside one bucket).
template <int E>
__device__ void append_run(const ArrayView& v, uint32_t l, uint64_t start, uint64_t cnt, uint64_t vfirst) {
  typedef typename Elem<E>::T T;
  constexpr uint32_t VEC = 16 / E;
  const uint64_t* bk = v.buckets + static_cast<uint64_t>(l) * kMaxBuckets;
  const uint64_t end = start + cnt;
  const uint64_t gbeg = start & ~static_cast<uint64_t>(VEC - 1);
  const bool group_ok = v.B >= VEC;
  for (uint64_t p = gbeg + static_cast<uint64_t>(threadIdx.x) * VEC; p < end; p += static_cast<uint64_t>(blockDim.x) * VEC) {
    if (group_ok && p >= start && p + VEC <= end) {
      Vec16<E> x;
#pragma unroll
      for (uint32_t e = 0; e < VEC; ++e) x.e[e] = gen_value<E>(vfirst + (p + e - start));
      uint32_t bb;
      uint64_t off;
      bucket_of(p, v.log2B, bb, off);
      __stcs(reinterpret_cast<uint4*>(bk[bb] + off * E), x.v);
    } else {
      for (uint32_t e = 0; e < VEC; ++e) {
        const uint64_t pe = p + e;
        if (pe < start || pe >= end) continue;
        uint32_t bb;
        uint64_t off;
        bucket_of(pe, v.log2B, bb, off);
        *reinterpret_cast<T*>(bk[bb] + off * E) = gen_value<E>(vfirst + (pe - start));
      }
    }
  }
}

// One block per request: every LFVector's share is reserved (one size
// update, Algorithm 2 for the buckets it reaches) by its own thread, then
// the block recomputes the array's offsets from the new sizes.
__global__ void __launch_bounds__(kServeThreads) append_reserve_kernel(const __grid_constant__ AppendParams P) {
  __shared__ uint64_t s_warp[33];
  const uint32_t r = blockIdx.x;
  const ArrayView& v = *P.view[r];
  for (uint32_t l = threadIdx.x; l < v.L; l += blockDim.x) {
    const uint64_t c = P.n[r] / v.L + (l < P.n[r] % v.L ? 1 : 0);
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
    P.res_base[P.slot0[r] + l] = base;
    P.res_len[P.slot0[r] + l] = len;
  }
  __syncthreads();
  finalize_block(v, nullptr, nullptr, nullptr, 1, s_warp);
}

// Write blocks: kAppendChunk elements of one (request, LFVector) each.
__global__ void __launch_bounds__(kServeThreads) append_write_kernel(const __grid_constant__ AppendParams P) {
  uint32_t lo = 0, hi = P.n_req;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (P.chunk0[mid] <= blockIdx.x) lo = mid; else hi = mid;
  }
  const uint32_t r = lo;
  const ArrayView& v = *P.view[r];
  const uint32_t j = blockIdx.x - P.chunk0[r];
  const uint32_t l = j / P.per_lfv[r];
  const uint64_t k0 = static_cast<uint64_t>(j % P.per_lfv[r]) * kAppendChunk;
  const uint64_t base = P.res_base[P.slot0[r] + l];
  const uint64_t len = P.res_len[P.slot0[r] + l];
  if (k0 >= len) return;
  const uint64_t cnt = len - k0 < kAppendChunk ? len - k0 : kAppendChunk;
  const uint64_t vfirst = P.tag[r] * (1ull << 24) + static_cast<uint64_t>(l) * (1ull << 20) + k0;
  switch (v.E) {
    case 4: append_run<4>(v, l, base + k0, cnt, vfirst); break;
    case 8: append_run<8>(v, l, base + k0, cnt, vfirst); break;
    default: append_run<16>(v, l, base + k0, cnt, vfirst); break;
  }
}

__global__ void serve_fixup_kernel(PoolState* pool) { ring_fixup(pool); }

template <int E>
__device__ void read_run(const ArrayView& v, uint64_t n, uint64_t seed, void* out) {
  typedef typename Elem<E>::T T;
  T* o = static_cast<T*>(out);
  const uint64_t N = v.offsets[v.L];
  for (uint64_t k = threadIdx.x; k < n; k += blockDim.x) {
    T x = T();
    if (N) {
      const uint64_t g = ((splitmix(seed, k) >> 32) * N) >> 32;   // uniform over [0, N)
      const uint32_t l = find_lfv(v.offsets, v.L, N, g);
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
    if (v.L > gga::kServeSlots) return GGA_ERR_INVALID;
    seen.push_back(reqs[i].array);
  }
  std::sort(seen.begin(), seen.end());
  if (std::adjacent_find(seen.begin(), seen.end()) != seen.end()) return GGA_ERR_INVALID;   // one request per array

  uint64_t* res = gga::handle_serve_records(reqs[0].array, gga::kServeSlots);
  if (!res) return GGA_ERR_CUDA;
  // Launch groups: at most kServeMax requests and kServeSlots (request, LFVector) pairs each.
  uint32_t i0 = 0;
  while (i0 < n) {
    gga::AppendParams P;
    P.pad = 0;
    P.res_base = res;
    P.res_len = res + gga::kServeSlots;
    uint32_t m = 0, slots = 0, chunks = 0;
    while (i0 + m < n && m < static_cast<uint32_t>(gga::kServeMax)) {
      gga::ArrayView v;
      gga::InsertScratch s;
      int dev, sms;
      gga::handle_parts(reqs[i0 + m].array, &v, &s, &dev, &sms);
      if (slots + v.L > gga::kServeSlots) break;
      const uint64_t per = (reqs[i0 + m].n / v.L + 1 + gga::kAppendChunk - 1) / gga::kAppendChunk;
      P.view[m] = gga::handle_dview(reqs[i0 + m].array);
      P.n[m] = reqs[i0 + m].n;
      P.tag[m] = reqs[i0 + m].tag;
      P.slot0[m] = slots;
      P.chunk0[m] = chunks;
      P.per_lfv[m] = static_cast<uint32_t>(per);
      slots += v.L;
      chunks += static_cast<uint32_t>(per) * v.L;
      ++m;
    }
    P.n_req = m;
    P.slot0[m] = slots;
    P.chunk0[m] = chunks;
    gga::append_reserve_kernel<<<m, gga::kServeThreads, 0, st>>>(P);
    gga::serve_fixup_kernel<<<1, 1, 0, st>>>(pool);
    gga::append_write_kernel<<<chunks, gga::kServeThreads, 0, st>>>(P);
    i0 += m;
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
