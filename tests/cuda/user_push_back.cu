// A user's kernels on the device API: they include only the public header
// (include/gga_device.cuh) and push into, and read from, a GGArray through
// the view gga_device_view returns.  Built by the tests with nvcc into a
// library of its own (it does not link the GGArray library).
#include <cuda_runtime.h>
#include <stdint.h>

#include "gga_device.cuh"

namespace {

// Rounds of pushes: block i handles LFVectors l = i, i + gridDim.x, ...
// (reversed when `reverse`), round by round; thread t of LFVector l pushes
// counts[r][l][t] values vals[r][l][t][0..count) and records its first
// LFVector-local index in first[r][l][t].  Threads are laid out in 2-D when
// blockDim.y > 1 (rank = x + blockDim.x * y).
template <class T>
__global__ void __launch_bounds__(1024) push_rounds(const gga_dev_view* v, const uint32_t* counts, const T* vals, uint64_t* first, uint32_t R,
                            uint32_t L, uint32_t NT, uint32_t kmax, int reverse, int stop_on_fail) {
  const uint32_t t = gga::block_rank();
  for (uint32_t i = blockIdx.x; i < L; i += gridDim.x) {
    const uint32_t l = reverse ? L - 1 - i : i;
    for (uint32_t r = 0; r < R; ++r) {
      const uint64_t row = (static_cast<uint64_t>(r) * L + l) * NT + t;
      const uint32_t c = counts[row];
      const T* mine = vals + row * kmax;
      uint64_t j0 = ~0ull;
      const bool ok = gga::block_push_back<T>(v, l, c, [&](uint32_t k) { return mine[k]; }, &j0);
      first[row] = ok ? j0 : ~0ull;
      if (!ok && stop_on_fail) break;
    }
  }
}

// The same rounds through a BlockPusher per LFVector (one shared slot set,
// reused by the block's successive cursors).
template <class T>
__global__ void __launch_bounds__(1024) push_rounds_cursor(const gga_dev_view* v, const uint32_t* counts, const T* vals, uint64_t* first,
                                   uint32_t R, uint32_t L, uint32_t NT, uint32_t kmax, int reverse, int stop_on_fail) {
  __shared__ gga::PushShared sh;
  const uint32_t t = gga::block_rank();
  for (uint32_t i = blockIdx.x; i < L; i += gridDim.x) {
    const uint32_t l = reverse ? L - 1 - i : i;
    gga::BlockPusher<T> pusher(v, l, sh);
    for (uint32_t r = 0; r < R; ++r) {
      const uint64_t row = (static_cast<uint64_t>(r) * L + l) * NT + t;
      const uint32_t c = counts[row];
      const T* mine = vals + row * kmax;
      uint64_t j0 = ~0ull;
      const bool ok = pusher.push(c, [&](uint32_t k) { return mine[k]; }, &j0);
      first[row] = ok ? j0 : ~0ull;
      if (!ok && stop_on_fail) break;
    }
  }
}

// The same rounds through the other forms of the device API: mode 2, a
// BlockPusher with a shared-memory stage (staged 128-bit writes); mode 3,
// block_push_rounds with K = 4 rounds per call and a stage; mode 4,
// block_push_rounds with K = 3 and no stage.  A block_push_rounds call
// that keeps fewer than K rounds counts as a failed push.
template <class T, int K>
__device__ void push_rounds_k(const gga_dev_view* v, const uint32_t* counts, const T* vals, uint64_t* first,
                              uint32_t R, uint32_t L, uint32_t NT, uint32_t kmax, uint32_t l, int stop_on_fail,
                              void* stage, uint32_t stage_bytes) {
  const uint32_t t = gga::block_rank();
  for (uint32_t r0 = 0; r0 < R; r0 += K) {
    uint32_t c[K];
    const T* mine[K];
    for (int k = 0; k < K; ++k) {
      const uint32_t r = r0 + k;
      const uint64_t row = (static_cast<uint64_t>(r < R ? r : 0) * L + l) * NT + t;
      c[k] = r < R ? counts[row] : 0u;
      mine[k] = vals + row * kmax;
    }
    uint64_t j0[K];
    const uint32_t done = gga::block_push_rounds<T, K>(
        v, l, c, [&](uint32_t kr, uint32_t k) { return mine[kr][k]; }, stage, stage_bytes, j0);
    for (int k = 0; k < K; ++k) {
      const uint32_t r = r0 + k;
      if (r < R) first[(static_cast<uint64_t>(r) * L + l) * NT + t] = static_cast<uint32_t>(k) < done ? j0[k] : ~0ull;
    }
    if (done < static_cast<uint32_t>(K) && stop_on_fail) break;
  }
}

template <class T>
__global__ void __launch_bounds__(1024) push_rounds_mode(const gga_dev_view* v, const uint32_t* counts,
                                                         const T* vals, uint64_t* first, uint32_t R, uint32_t L,
                                                         uint32_t NT, uint32_t kmax, int reverse, int stop_on_fail,
                                                         int mode, uint32_t stage_bytes) {
  __shared__ gga::PushShared sh;
  extern __shared__ uint4 stage[];
  const uint32_t t = gga::block_rank();
  for (uint32_t i = blockIdx.x; i < L; i += gridDim.x) {
    const uint32_t l = reverse ? L - 1 - i : i;
    if (mode == 2) {
      gga::BlockPusher<T> pusher(v, l, sh, stage, stage_bytes);
      for (uint32_t r = 0; r < R; ++r) {
        const uint64_t row = (static_cast<uint64_t>(r) * L + l) * NT + t;
        const T* mine = vals + row * kmax;
        uint64_t j0 = ~0ull;
        const bool ok = pusher.push(counts[row], [&](uint32_t k) { return mine[k]; }, &j0);
        first[row] = ok ? j0 : ~0ull;
        if (!ok && stop_on_fail) break;
      }
      pusher.flush();
    } else if (mode == 3) {
      push_rounds_k<T, 4>(v, counts, vals, first, R, L, NT, kmax, l, stop_on_fail, stage, stage_bytes);
    } else {
      push_rounds_k<T, 3>(v, counts, vals, first, R, L, NT, kmax, l, stop_on_fail, nullptr, 0);
    }
    __syncthreads();   // the next LFVector's pushes reuse the shared slots and the stage
  }
}

// Rounds whose values are a formula of (round, LFVector, thread, k), for
// counts too large to hold their values in an array: element k of thread t
// of LFVector l in round r is (r << 56) | (l << 48) | (t << 32) | k.
__global__ void __launch_bounds__(1024) push_formula(const gga_dev_view* v, const uint32_t* counts, uint32_t R, uint32_t L, uint32_t NT,
                             int cursor) {
  __shared__ gga::PushShared sh;
  const uint32_t t = gga::block_rank();
  const uint32_t l = blockIdx.x;
  const auto value = [&](uint32_t r) {
    return [=](uint32_t k) {
      return (static_cast<unsigned long long>(r) << 56) | (static_cast<unsigned long long>(l) << 48) |
             (static_cast<unsigned long long>(t) << 32) | k;
    };
  };
  if (cursor) {
    gga::BlockPusher<unsigned long long> pusher(v, l, sh);
    for (uint32_t r = 0; r < R; ++r) pusher.push(counts[(static_cast<uint64_t>(r) * L + l) * NT + t], value(r));
  } else {
    for (uint32_t r = 0; r < R; ++r)
      gga::block_push_back<unsigned long long>(v, l, counts[(static_cast<uint64_t>(r) * L + l) * NT + t], value(r));
  }
}

// One LFVector per block, the short form (l = blockIdx.x), one round.
template <class T>
__global__ void __launch_bounds__(1024) push_own(const gga_dev_view* v, const uint32_t* counts, const T* vals, uint32_t kmax) {
  const uint32_t t = gga::block_rank();
  const uint64_t row = static_cast<uint64_t>(blockIdx.x) * gga::block_threads() + t;
  const T* mine = vals + row * kmax;
  gga::block_push_back<T>(v, counts[row], [&](uint32_t k) { return mine[k]; });
}

template <class T>
__global__ void read_global(const gga_dev_view* v, const uint64_t* g, uint64_t n, T* out, uint64_t* n_out) {
  const uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i == 0) *n_out = gga::global_size(v);
  if (i < n) out[i] = gga::global_at<T>(v, g[i]);
}

template <class T>
__global__ void read_local(const gga_dev_view* v, const uint32_t* l, const uint64_t* j, uint64_t n, T* out,
                           uint64_t* sizes) {
  const uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) {
    out[i] = gga::lfv_at<T>(v, l[i], j[i]);
    sizes[i] = gga::lfv_size(v, l[i]);
  }
}

// Calls the device API must reject: an LFVector index past the end (mode 0)
// or an element type whose size is not the array's (mode 1).
__global__ void push_rejected(const gga_dev_view* v, int mode, uint32_t* ok_out) {
  bool ok;
  if (mode == 0) ok = gga::block_push_back<uint32_t>(v, v->L, 1u, [](uint32_t) { return 7u; });
  else ok = gga::block_push_back<uint16_t>(v, 0u, 1u, [](uint32_t) { return static_cast<uint16_t>(7); });
  if (threadIdx.x == 0) ok_out[blockIdx.x] = ok ? 1u : 0u;
}

int launched() { return cudaGetLastError() == cudaSuccess ? 0 : 5; }

}  // namespace

extern "C" {

int user_push_rounds(const void* view, const uint32_t* counts, const void* vals, uint64_t* first, uint32_t R,
                     uint32_t L, uint32_t bx, uint32_t by, uint32_t kmax, uint32_t E, uint32_t blocks, int reverse,
                     int stop_on_fail, void* stream) {
  const gga_dev_view* v = static_cast<const gga_dev_view*>(view);
  const dim3 block(bx, by);
  const uint32_t nt = bx * by;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (E == 4)
    push_rounds<uint32_t><<<blocks, block, 0, st>>>(v, counts, static_cast<const uint32_t*>(vals), first, R, L, nt,
                                                    kmax, reverse, stop_on_fail);
  else if (E == 8)
    push_rounds<unsigned long long><<<blocks, block, 0, st>>>(
        v, counts, static_cast<const unsigned long long*>(vals), first, R, L, nt, kmax, reverse, stop_on_fail);
  else
    push_rounds<uint4><<<blocks, block, 0, st>>>(v, counts, static_cast<const uint4*>(vals), first, R, L, nt, kmax,
                                                 reverse, stop_on_fail);
  return launched();
}

int user_push_rounds_cursor(const void* view, const uint32_t* counts, const void* vals, uint64_t* first, uint32_t R,
                            uint32_t L, uint32_t bx, uint32_t by, uint32_t kmax, uint32_t E, uint32_t blocks,
                            int reverse, int stop_on_fail, void* stream) {
  const gga_dev_view* v = static_cast<const gga_dev_view*>(view);
  const dim3 block(bx, by);
  const uint32_t nt = bx * by;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (E == 4)
    push_rounds_cursor<uint32_t><<<blocks, block, 0, st>>>(v, counts, static_cast<const uint32_t*>(vals), first, R,
                                                           L, nt, kmax, reverse, stop_on_fail);
  else if (E == 8)
    push_rounds_cursor<unsigned long long><<<blocks, block, 0, st>>>(
        v, counts, static_cast<const unsigned long long*>(vals), first, R, L, nt, kmax, reverse, stop_on_fail);
  else
    push_rounds_cursor<uint4><<<blocks, block, 0, st>>>(v, counts, static_cast<const uint4*>(vals), first, R, L, nt,
                                                        kmax, reverse, stop_on_fail);
  return launched();
}

int user_push_rounds_mode(const void* view, const uint32_t* counts, const void* vals, uint64_t* first, uint32_t R,
                          uint32_t L, uint32_t bx, uint32_t by, uint32_t kmax, uint32_t E, uint32_t blocks,
                          int reverse, int stop_on_fail, int mode, uint32_t stage_bytes, void* stream) {
  const gga_dev_view* v = static_cast<const gga_dev_view*>(view);
  const dim3 block(bx, by);
  const uint32_t nt = bx * by;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t smem = stage_bytes;
  if (E == 4) {
    cudaFuncSetAttribute(push_rounds_mode<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, stage_bytes);
    push_rounds_mode<uint32_t><<<blocks, block, smem, st>>>(v, counts, static_cast<const uint32_t*>(vals), first, R,
                                                            L, nt, kmax, reverse, stop_on_fail, mode, stage_bytes);
  } else if (E == 8) {
    cudaFuncSetAttribute(push_rounds_mode<unsigned long long>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         stage_bytes);
    push_rounds_mode<unsigned long long><<<blocks, block, smem, st>>>(
        v, counts, static_cast<const unsigned long long*>(vals), first, R, L, nt, kmax, reverse, stop_on_fail, mode,
        stage_bytes);
  } else {
    cudaFuncSetAttribute(push_rounds_mode<uint4>, cudaFuncAttributeMaxDynamicSharedMemorySize, stage_bytes);
    push_rounds_mode<uint4><<<blocks, block, smem, st>>>(v, counts, static_cast<const uint4*>(vals), first, R, L, nt,
                                                         kmax, reverse, stop_on_fail, mode, stage_bytes);
  }
  return launched();
}

int user_push_formula(const void* view, const uint32_t* counts, uint32_t R, uint32_t L, uint32_t NT, int cursor,
                      void* stream) {
  push_formula<<<L, NT, 0, static_cast<cudaStream_t>(stream)>>>(static_cast<const gga_dev_view*>(view), counts, R, L,
                                                                 NT, cursor);
  return launched();
}

int user_push_own(const void* view, const uint32_t* counts, const void* vals, uint32_t L, uint32_t T, uint32_t kmax,
                  void* stream) {
  push_own<uint32_t><<<L, T, 0, static_cast<cudaStream_t>(stream)>>>(
      static_cast<const gga_dev_view*>(view), counts, static_cast<const uint32_t*>(vals), kmax);
  return launched();
}

int user_read_global(const void* view, const uint64_t* g, uint64_t n, void* out, uint64_t* n_out, uint32_t E,
                     void* stream) {
  const gga_dev_view* v = static_cast<const gga_dev_view*>(view);
  const unsigned grid = static_cast<unsigned>((n + 255) / 256 > 0 ? (n + 255) / 256 : 1);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (E == 4) read_global<uint32_t><<<grid, 256, 0, st>>>(v, g, n, static_cast<uint32_t*>(out), n_out);
  else if (E == 8) read_global<unsigned long long><<<grid, 256, 0, st>>>(v, g, n, static_cast<unsigned long long*>(out), n_out);
  else read_global<uint4><<<grid, 256, 0, st>>>(v, g, n, static_cast<uint4*>(out), n_out);
  return launched();
}

int user_read_local(const void* view, const uint32_t* l, const uint64_t* j, uint64_t n, void* out, uint64_t* sizes,
                    uint32_t E, void* stream) {
  const gga_dev_view* v = static_cast<const gga_dev_view*>(view);
  const unsigned grid = static_cast<unsigned>((n + 255) / 256 > 0 ? (n + 255) / 256 : 1);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (E == 4) read_local<uint32_t><<<grid, 256, 0, st>>>(v, l, j, n, static_cast<uint32_t*>(out), sizes);
  else if (E == 8) read_local<unsigned long long><<<grid, 256, 0, st>>>(v, l, j, n, static_cast<unsigned long long*>(out), sizes);
  else read_local<uint4><<<grid, 256, 0, st>>>(v, l, j, n, static_cast<uint4*>(out), sizes);
  return launched();
}

int user_push_rejected(const void* view, int mode, uint32_t* ok_out, void* stream) {
  push_rejected<<<2, 64, 0, static_cast<cudaStream_t>(stream)>>>(static_cast<const gga_dev_view*>(view), mode, ok_out);
  return launched();
}

}  // extern "C"
