// gga_push.cu -- the device API's own entry points: the view a user kernel
// pushes through, the commit that follows such a kernel, and the generated
// insertion written as a user kernel would write it (Algorithm 1 as the
// paper states it: one block per LFVector, one push per round, through the
// device API's BlockPusher).
#include "gga_core.cuh"
#include "gga_device.cuh"
#include "gga_gen.cuh"

namespace gga {

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

int gga_push_generated(gga_handle h, const gga_gen_spec* spec, uint32_t rounds, void* stream) {
  gga::ArrayView v;
  if (!h || !spec || !gga::handle_parts(h, &v, nullptr, nullptr, nullptr)) return GGA_ERR_INVALID;
  if (spec->dist > GGA_DIST_POISSON || spec->n_thresholds > GGA_MAX_THRESHOLDS) return GGA_ERR_INVALID;
  if (spec->dist == GGA_DIST_POISSON && spec->n_thresholds == 0) return GGA_ERR_INVALID;
  if (rounds == 0) return GGA_OK;
  return gga::launch_push_generated(v, gga::handle_dview(h), *spec, rounds, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
