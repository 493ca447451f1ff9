// gga_push.cu -- the device API's own entry points: the view a user kernel
// pushes through, the commit that follows such a kernel, the generated
// insertion written as a user kernel would write it (Algorithm 1 as the
// paper states it: one block per LFVector, one push per round, through the
// device API's BlockPusher), and pushes of values read from device memory
// (block_push_rounds, several rounds per call).
#include "gga_core.cuh"
#include "gga_device.cuh"
#include "gga_gen.cuh"

namespace gga {

// (The pushes store per thread: with about one element per thread and push,
// assembling each push in a shared-memory stage for 128-bit stores made the
// kernel slower on GB300, 2.93 ms against 2.28 ms for the paper-shaped
// workload, whether the stage cost a barrier of its own or was written out
// behind the next push's first barrier.)
// Block l draws round r's counts and values exactly as gga_insert_generated
// does (SplitMix64 on ((r << 32) | l*T + t)), and appends them with one push
// per round through a BlockPusher on LFVector l.  A round that does not fit
// ends the block's rounds (the rounds that fit are kept, as in every
// insertion).
// Stage of one block_push_rounds call of the memory-sourced pushes: K = 8
// rounds of 512 threads average 16 KB of int32 at one element per thread
// and round.
constexpr uint32_t kExpandStageBytes = 32768;

template <int E>
__global__ void __launch_bounds__(1024) push_generated_kernel(const ArrayView* view, GenParams g, uint32_t R) {
  typedef typename Elem<E>::T T;
  __shared__ PushShared sh;
  const uint32_t l = blockIdx.x;
  const uint64_t gtid = static_cast<uint64_t>(l) * blockDim.x + threadIdx.x;
  BlockPusher<T> pusher(view, l, sh);
#pragma unroll 1
  for (uint32_t i = 0; i < R; ++i) {
    const uint64_t r = static_cast<uint64_t>(g.round0) + i;
    const uint32_t c = gen_count(g, splitmix(g.seed, (r << 32) | gtid));
    const uint64_t v0 = g.va * gtid + g.vb * r;
    if (!pusher.push(c, [&](uint32_t k) { return gen_value<E>(v0 + g.vc * k); })) break;
  }
  pusher.flush();
}

int launch_push_generated(const ArrayView& v, const ArrayView* dview, const gga_gen_spec& spec, uint32_t rounds,
                          cudaStream_t st) {
  const GenParams g = make_gen_params(spec);
  if (v.E == 4) push_generated_kernel<4><<<v.L, v.T, 0, st>>>(dview, g, rounds);
  else if (v.E == 8) push_generated_kernel<8><<<v.L, v.T, 0, st>>>(dview, g, rounds);
  else push_generated_kernel<16><<<v.L, v.T, 0, st>>>(dview, g, rounds);
  if (cudaGetLastError() != cudaSuccess) return GGA_ERR_CUDA;
  return launch_finalize(v, st);
}

// Memory-sourced pushes through the device API: block l reads, for K
// rounds at a time, its threads' counts counts[r][l][t] and inputs
// inputs[r][l][t] (coalesced, all 2K loads of a thread issued before any is
// used) and appends, per thread and round, `count` copies of its input with
// one block_push_rounds call for the K rounds (staged, 128-bit stores).  A
// call that does not fit ends the block's rounds.
// Two resident blocks of 512 threads per SM: the 2K loads of a pass are
// then held in registers until used (with 40 registers they spill, and a
// spilled load is waited for at once, which serialises them).
#ifndef GGA_EXPAND_MINB
#define GGA_EXPAND_MINB 2
#endif
template <int E, int K>
__global__ void __launch_bounds__(512, GGA_EXPAND_MINB) push_expand_kernel(const ArrayView* view,
                                                             const uint32_t* __restrict__ counts,
                                                             const typename Elem<E>::T* __restrict__ inputs,
                                                             uint32_t R, uint32_t L, uint32_t T,
                                                             uint32_t stage_bytes) {
  typedef typename Elem<E>::T V;
  extern __shared__ uint4 s_stage[];
  const uint32_t l = blockIdx.x, t = threadIdx.x;
  // (A bulk L2 prefetch of the next pass's rows by thread 0 measured slower:
  // 1.51 ms against 1.37 ms for the paper-shaped workload.)
#pragma unroll 1
  for (uint32_t r0 = 0; r0 < R; r0 += K) {
    uint32_t c[K];
    V x[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const uint32_t r = r0 + k;
      c[k] = 0;
      x[k] = V();
      if (r < R && t < T) {
        const uint64_t i = (static_cast<uint64_t>(r) * L + l) * T + t;
        c[k] = __ldcs(counts + i);
        x[k] = __ldcs(inputs + i);
      }
    }
    const uint32_t done =
        block_push_rounds<V, K>(view, l, c, [&](uint32_t kr, uint32_t) { return x[kr]; }, s_stage, stage_bytes);
    if (done < static_cast<uint32_t>(K)) break;
  }
}

int launch_push_expand(const ArrayView& v, const ArrayView* dview, const uint32_t* counts, const void* inputs,
                       uint32_t rounds, cudaStream_t st) {
  const uint32_t NT = (v.T + 31) / 32 * 32;
  if (NT > 512) return GGA_ERR_INVALID;
  const size_t smem = kExpandStageBytes;
#define GGA_EXPAND(EE, KK)                                                                                     \
  do {                                                                                                         \
    cudaFuncSetAttribute(push_expand_kernel<EE, KK>, cudaFuncAttributeMaxDynamicSharedMemorySize,             \
                         static_cast<int>(smem));                                                              \
    push_expand_kernel<EE, KK><<<v.L, NT, smem, st>>>(                                                         \
        dview, counts, static_cast<const typename Elem<EE>::T*>(inputs), rounds, v.L, v.T,                     \
        static_cast<uint32_t>(smem));                                                                          \
  } while (0)
  if (v.E == 4) GGA_EXPAND(4, 8);
  else if (v.E == 8) GGA_EXPAND(8, 4);
  else GGA_EXPAND(16, 2);
#undef GGA_EXPAND
  if (cudaGetLastError() != cudaSuccess) return GGA_ERR_CUDA;
  return launch_finalize(v, st);
}

}  // namespace gga

extern "C" {

int gga_device_view(gga_handle h, const void** view_dev) {
  if (!h || !view_dev) return GGA_ERR_INVALID;
  *view_dev = gga::handle_dview(h);
  return *view_dev ? GGA_OK : GGA_ERR_INVALID;
}

int gga_device_commit(gga_handle h, void* stream) {
  gga::ArrayView v;
  if (!gga::handle_parts(h, &v, nullptr, nullptr, nullptr)) return GGA_ERR_INVALID;
  return gga::launch_finalize(v, static_cast<cudaStream_t>(stream));
}

int gga_push_expand(gga_handle h, const uint32_t* counts_dev, const void* inputs_dev, uint32_t rounds,
                    void* stream) {
  gga::ArrayView v;
  if (!h || !gga::handle_parts(h, &v, nullptr, nullptr, nullptr)) return GGA_ERR_INVALID;
  if (rounds == 0) return GGA_OK;
  if (!counts_dev || !inputs_dev || v.T > 512) return GGA_ERR_INVALID;
  if ((reinterpret_cast<uintptr_t>(counts_dev) & 3) != 0 || (reinterpret_cast<uintptr_t>(inputs_dev) % v.E) != 0)
    return GGA_ERR_INVALID;
  return gga::launch_push_expand(v, gga::handle_dview(h), counts_dev, inputs_dev, rounds,
                                 static_cast<cudaStream_t>(stream));
}

int gga_push_generated(gga_handle h, const gga_gen_spec* spec, uint32_t rounds, void* stream) {
  gga::ArrayView v;
  if (!h || !spec || !gga::handle_parts(h, &v, nullptr, nullptr, nullptr)) return GGA_ERR_INVALID;
  if (spec->dist > GGA_DIST_POISSON || spec->n_thresholds > GGA_MAX_THRESHOLDS) return GGA_ERR_INVALID;
  if (spec->dist == GGA_DIST_POISSON && spec->n_thresholds == 0) return GGA_ERR_INVALID;
  if (rounds == 0) return GGA_OK;
  return gga::launch_push_generated(v, gga::handle_dview(h), *spec, rounds, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
