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

// Memory-sourced pushes through the device API: block l appends, per
// thread slot t and round r, counts[r][l][t] copies of inputs[r][l][t],
// K rounds per gga::block_push_rounds call (staged, 128-bit stores).  A
// thread plays S consecutive slots S t, ..., S t + S - 1 and pushes their
// counts together (its elements are slot S t's copies, then S t + 1's, ...,
// which is their order in the LFVector): one scan slot and one share of
// every barrier then serve S slots, and the blocks (512 / S threads for
// T = 512) are small enough for all 1024 of the paper-shaped workload to
// be resident at once.  Each thread loads its 2 K S counts and inputs of a
// call before using any.  A call that does not fit ends the block's rounds.
// Measured on GB300 for the paper-shaped workload (1024 x 512, 512 rounds,
// int32): one slot per thread, K = 8, 2 blocks per SM: 1.42 ms (with the
// loads prefetched into shared memory by cp.async: 1.52 ms); S = 2, K = 4,
// 4 per SM: 0.98 ms; S = 4, K = 2, 8 per SM: 0.90 ms; S = 4, K = 4, 8 per
// SM: 0.84 ms.
template <int E, int K, int S, int MINB>
__global__ void __launch_bounds__(512 / S, MINB) push_expand_s_kernel(const ArrayView* view,
                                                                  const uint32_t* __restrict__ counts,
                                                                  const typename Elem<E>::T* __restrict__ inputs,
                                                                  uint32_t R, uint32_t L, uint32_t T,
                                                                  uint32_t stage_bytes) {
  typedef typename Elem<E>::T V;
  extern __shared__ uint4 s_stage[];
  const uint32_t l = blockIdx.x, t = S * threadIdx.x;
#pragma unroll 1
  for (uint32_t r0 = 0; r0 < R; r0 += K) {
    uint32_t c[K], cs[K][S];
    V x[K][S];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const uint32_t r = r0 + k;
      c[k] = 0;
#pragma unroll
      for (int i = 0; i < S; ++i) {
        cs[k][i] = 0;
        x[k][i] = V();
        if (r < R && t + i < T) {
          const uint64_t at = (static_cast<uint64_t>(r) * L + l) * T + t + i;
          cs[k][i] = __ldcs(counts + at);
          x[k][i] = __ldcs(inputs + at);
        }
        c[k] += cs[k][i];
      }
    }
    const uint32_t done = block_push_rounds<V, K>(
        view, l, c,
        [&](uint32_t kr, uint32_t m) {
          V v = x[kr][S - 1];
#pragma unroll
          for (int i = S - 2; i >= 0; --i) {
            uint32_t before = 0;
#pragma unroll
            for (int j = 0; j <= i; ++j) before += cs[kr][j];
            if (m < before) v = x[kr][i];
          }
          return v;
        },
        s_stage, stage_bytes);
    if (done < static_cast<uint32_t>(K)) break;
  }
}

template <int E, int K, int S, int MINB>
int launch_expand_s(const ArrayView& v, const ArrayView* dview, const uint32_t* counts, const void* inputs,
                    uint32_t rounds, cudaStream_t st) {
  const uint32_t NTS = ((v.T + S - 1) / S + 31) / 32 * 32;
  // Stage: twice a call's elements at one per slot of 512 (larger calls go unstaged).
  const size_t smem = static_cast<size_t>(K) * 512u * E * 2u;
  auto kern = push_expand_s_kernel<E, K, S, MINB>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  kern<<<v.L, NTS, smem, st>>>(dview, counts, static_cast<const typename Elem<E>::T*>(inputs), rounds, v.L, v.T,
                               static_cast<uint32_t>(smem));
  if (cudaGetLastError() != cudaSuccess) return GGA_ERR_CUDA;
  return launch_finalize(v, st);
}

int launch_push_expand(const ArrayView& v, const ArrayView* dview, const uint32_t* counts, const void* inputs,
                       uint32_t rounds, cudaStream_t st) {
  if (v.T > 512) return GGA_ERR_INVALID;
  if (v.E == 4) return launch_expand_s<4, 4, 4, 8>(v, dview, counts, inputs, rounds, st);
  if (v.E == 8) return launch_expand_s<8, 2, 4, 8>(v, dview, counts, inputs, rounds, st);
  return launch_expand_s<16, 2, 2, 4>(v, dview, counts, inputs, rounds, st);
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
