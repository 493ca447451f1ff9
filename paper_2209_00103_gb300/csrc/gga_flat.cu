// gga_flat.cu -- Sec. III-B's parallel insertion approaches on a flat array
// (the paper's insertion experiment, Sec. VI-A).
//   atomic: each thread: pos = atomicAdd(size, 1)
//   scan:   each block: warp shuffle scan of the threads' counts, one pass
//           over the warp totals in shared memory, one atomicAdd(size, total)
//           by the block, then every thread writes at base + its prefix.
#include <cuda_runtime.h>

#include "gga.h"
#include "gga_flat.h"

namespace {

__global__ void flat_insert_atomic_kernel(uint32_t* __restrict__ a, uint64_t cap, unsigned long long* size,
                                          uint64_t n, uint32_t first) {
  const uint64_t t = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const unsigned long long pos = atomicAdd(size, 1ull);
  if (pos < cap) a[pos] = first + static_cast<uint32_t>(t);
}

__global__ void flat_insert_scan_kernel(uint32_t* __restrict__ a, uint64_t cap, unsigned long long* size,
                                        uint64_t n, uint32_t first) {
  __shared__ uint32_t s_warp[32];
  __shared__ unsigned long long s_base;
  const uint64_t t = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const uint32_t c = t < n ? 1u : 0u;                 // this experiment inserts one element per thread
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t incl = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_warp[w] = incl;
  __syncthreads();
  if (w == 0) {
    const int nw = static_cast<int>(blockDim.x >> 5);
    uint32_t x = lane < nw ? s_warp[lane] : 0u;
    uint32_t sc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, sc, o);
      if (lane >= o) sc += y;
    }
    if (lane < nw) s_warp[lane] = sc - x;               // exclusive prefix of the warp totals
    if (lane == 31) s_base = sc ? atomicAdd(size, static_cast<unsigned long long>(sc)) : 0ull;
  }
  __syncthreads();
  if (c) {
    const unsigned long long pos = s_base + s_warp[w] + (incl - c);
    if (pos < cap) a[pos] = first + static_cast<uint32_t>(t);
  }
}

}  // namespace

extern "C" int gga_flat_insert(int mode, uint32_t* array, uint64_t capacity, uint64_t* size_dev, uint64_t n_threads,
                               uint32_t threads_per_block, uint32_t first_value, void* stream) {
  if (!array || !size_dev || threads_per_block < 32 || threads_per_block > 1024 || threads_per_block % 32)
    return GGA_ERR_INVALID;
  if (mode != GGA_FLAT_ATOMIC && mode != GGA_FLAT_SCAN) return GGA_ERR_INVALID;
  if (n_threads == 0) return GGA_OK;
  const uint64_t blocks = (n_threads + threads_per_block - 1) / threads_per_block;
  if (blocks > 0x7FFFFFFFull) return GGA_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned long long* sz = reinterpret_cast<unsigned long long*>(size_dev);
  if (mode == GGA_FLAT_ATOMIC)
    flat_insert_atomic_kernel<<<static_cast<unsigned>(blocks), threads_per_block, 0, st>>>(array, capacity, sz,
                                                                                           n_threads, first_value);
  else
    flat_insert_scan_kernel<<<static_cast<unsigned>(blocks), threads_per_block, 0, st>>>(array, capacity, sz,
                                                                                         n_threads, first_value);
  return cudaGetLastError() == cudaSuccess ? GGA_OK : GGA_ERR_CUDA;
}
