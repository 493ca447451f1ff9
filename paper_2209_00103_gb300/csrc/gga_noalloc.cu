// gga_noalloc.cu -- gga_insert_noalloc: insertion that allocates no GPU memory.
//
// gga_insert grows a per-handle scratch buffer with cudaMallocAsync whenever a
// call needs more rounds than any call before it.  Callers that run inside a
// fixed, pre-reserved memory budget (a caching allocator that already holds
// the device's memory) or inside latency-critical loops cannot let a call
// allocate: the allocation may block, synchronize or fail at a bad moment.
// This entry point runs the same three insertion kernels with their per-call
// scratch placed in one fixed array that is part of the library image, so
// nothing is allocated during the call.  It is an interface variant; the
// paper has no counterpart.
//
// The array lives in device memory of every GPU that uses the library, for
// the life of the process.  Host code cannot use its name as an address (in
// host code the name denotes a host-side shadow), so the device address is
// looked up once per device with cudaGetSymbolAddress, with that device
// current, and passed to the kernels.  Under CUDA's lazy module loading the
// array is placed on a device only when it is first looked up there; handle
// creation does that lookup (noalloc_prepare), so the 32 MiB are committed
// while the caller creates its arrays, not inside a gga_insert_noalloc call.
#include <mutex>

#include "gga_core.cuh"

// Fixed scratch of gga_insert_noalloc: 32 MiB.
static constexpr size_t kNoAllocScratchBytes = static_cast<size_t>(32) << 20;
static __device__ __align__(256) unsigned char gga_noalloc_scratch[kNoAllocScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};

inline size_t up256(size_t x) { return (x + 255) / 256 * 256; }

// Device address of the fixed scratch on the current device, looked up on
// the first request there.  Returns nullptr on failure, with the runtime's
// last-error state cleared so that a later, unrelated launch check does not
// report this failure.
void* scratch_on_device(int dev) {
  if (dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (g_scratch_addr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, gga_noalloc_scratch) != cudaSuccess) {
      (void)cudaGetLastError();
      return nullptr;
    }
    g_scratch_addr[dev] = p;
  }
  return g_scratch_addr[dev];
}

}  // namespace

namespace gga {

// Called by handle creation with the handle's device current: places the
// fixed scratch on that device now.  A failure here is not an error of the
// creation (the array itself does not need the scratch); the next
// gga_insert_noalloc on the device tries again and reports GGA_ERR_CUDA.
void noalloc_prepare(int dev) { (void)scratch_on_device(dev); }

}  // namespace gga

extern "C" int gga_insert_noalloc(gga_handle h, const uint32_t* counts_dev, uint32_t rounds,
                                  const void* values_dev, uint64_t n_values, void* stream) {
  gga::ArrayView v;
  gga::InsertScratch s;
  int hdev = -1, num_sms = 0;
  if (!gga::handle_parts(h, &v, &s, &hdev, &num_sms)) return GGA_ERR_INVALID;
  if (rounds == 0) return n_values == 0 ? GGA_OK : GGA_ERR_INVALID;
  if (!counts_dev || (n_values > 0 && !values_dev)) return GGA_ERR_INVALID;
  if ((reinterpret_cast<uintptr_t>(values_dev) % v.E) != 0 && n_values > 0) return GGA_ERR_INVALID;
  if ((reinterpret_cast<uintptr_t>(counts_dev) & 3) != 0) return GGA_ERR_INVALID;

  // Scratch layout for this call: [tile prefixes | row prefixes | round positions].
  const uint64_t rows = static_cast<uint64_t>(rounds) * v.L;
  const bool vec_ok = (reinterpret_cast<uintptr_t>(counts_dev) & 15) == 0;
  const uint64_t tiles = gga::count_tiles(rows, v.T, vec_ok);
  const size_t b_tiles = up256(tiles * 8 + 8);
  const size_t b_voff = up256((rows + 1) * 8);
  const size_t b_pre = up256(static_cast<uint64_t>(v.L) * (rounds + 1ull) * 8);
  if (b_tiles + b_voff + b_pre > kNoAllocScratchBytes) return GGA_ERR_TOO_LARGE;

  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return GGA_ERR_CUDA;
  if (dev != hdev) return GGA_ERR_INVALID;
  char* base = static_cast<char*>(scratch_on_device(dev));
  if (!base) return GGA_ERR_CUDA;
  s.tile_pre = reinterpret_cast<uint64_t*>(base);
  s.row_pre = reinterpret_cast<uint64_t*>(base + b_tiles);
  s.pre = reinterpret_cast<uint64_t*>(base + b_tiles + b_voff);

  // The array keeps whatever the previous call (on any handle) left there;
  // every part of it this call reads is written by this call's kernels first.
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return gga::launch_insert(v, s, counts_dev, rounds, values_dev, n_values, num_sms, st);
}
