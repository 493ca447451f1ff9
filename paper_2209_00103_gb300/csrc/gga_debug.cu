// gga_debug.cu -- test hook for the bounded-wait failure path: a wait that
// nothing completes gives up after its limit and reports GGA_ERR_TIMEOUT.
#include "gga_core.cuh"
#include "gga_debug.h"

namespace gga {
namespace {

__global__ void wait_timeout_kernel(uint32_t attempts, int arrive, uint32_t* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (arrive && threadIdx.x == 0) mbar_arrive(&bar);
  const bool got = mbar_wait_bounded(&bar, 0, attempts);
  if (threadIdx.x == 0) *status = got ? GGA_OK : GGA_ERR_TIMEOUT;
}

}  // namespace
}  // namespace gga

extern "C" int gga_debug_wait_timeout(uint32_t attempts, int arrive, void* stream) {
  if (attempts == 0 || attempts > (1u << 20)) return GGA_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t* d = nullptr;
  uint32_t h = GGA_ERR_CUDA;
  if (cudaMallocAsync(reinterpret_cast<void**>(&d), sizeof(uint32_t), st) != cudaSuccess) return GGA_ERR_CUDA;
  gga::wait_timeout_kernel<<<1, 32, 0, st>>>(attempts, arrive, d);
  const bool ok = cudaGetLastError() == cudaSuccess &&
                  cudaMemcpyAsync(&h, d, sizeof(uint32_t), cudaMemcpyDeviceToHost, st) == cudaSuccess;
  cudaFreeAsync(d, st);
  if (cudaStreamSynchronize(st) != cudaSuccess || !ok) return GGA_ERR_CUDA;
  return static_cast<int>(h);
}
