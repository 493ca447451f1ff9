// gga_gen.cuh -- device helpers shared by the insertion kernels: the
// counter-based draws of the generated workloads, and the block-wide
// finalize (prefix sum of LFVector sizes, Sec. IV; work lists).
#pragma once

#include "gga_core.cuh"

namespace gga {

struct GenParams {
  uint64_t seed, va, vb, vc;
  uint32_t dist, nthr, round0, pad;
  uint32_t thr[GGA_MAX_THRESHOLDS];
};

// SplitMix64 (Steele, Lea and Flood, 2014): output number key+1 of the
// stream seeded with `seed`.
__device__ __forceinline__ uint64_t splitmix(uint64_t seed, uint64_t key) {
  uint64_t z = seed + (key + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint32_t gen_count(const GenParams& g, uint64_t h) {
  switch (g.dist) {
    case GGA_DIST_BERNOULLI:
      return static_cast<uint32_t>(h >> 63);
    case GGA_DIST_UNIFORM3:
      return static_cast<uint32_t>(((h >> 32) * 3ull) >> 32);
    case GGA_DIST_GEOMETRIC: {
      const uint64_t inv = ~h;
      return inv == 0 ? 63u : min(63u, static_cast<uint32_t>(__ffsll(static_cast<long long>(inv)) - 1));
    }
    default: {
      const uint32_t u = static_cast<uint32_t>(h >> 32);
      uint32_t c = 0;
#pragma unroll
      for (uint32_t k = 0; k < GGA_MAX_THRESHOLDS; ++k) c += (k < g.nthr) & (u >= g.thr[k]);
      return c;
    }
  }
}

template <int E>
__device__ __forceinline__ typename Elem<E>::T gen_value(uint64_t v);
template <>
__device__ __forceinline__ uint32_t gen_value<4>(uint64_t v) { return static_cast<uint32_t>(v); }
template <>
__device__ __forceinline__ unsigned long long gen_value<8>(uint64_t v) { return v; }
template <>
__device__ __forceinline__ uint4 gen_value<16>(uint64_t v) {
  const float x = static_cast<float>(static_cast<uint32_t>(v & 0xFFFFull));
  const float y = static_cast<float>(static_cast<uint32_t>((v >> 16) & 0xFFFFull));
  return make_uint4(static_cast<uint32_t>(v), static_cast<uint32_t>(v >> 32), __float_as_uint(x), __float_as_uint(y));
}


inline GenParams make_gen_params(const gga_gen_spec& spec) {
  GenParams g;
  g.seed = spec.seed;
  g.va = spec.va;
  g.vb = spec.vb;
  g.vc = spec.vc;
  g.dist = spec.dist;
  g.nthr = spec.n_thresholds;
  g.round0 = spec.round0;
  g.pad = 0;
  for (int i = 0; i < GGA_MAX_THRESHOLDS; ++i) g.thr[i] = spec.thresholds[i];
  return g;
}

// ---------------------------------------------------------------------------
// Finalize: prefix sum of sizes, flatten/rw_b chunk prefix, copy chunk prefix.
// Run by one block (any multiple of 32 threads, <= 1024).

__device__ __forceinline__ uint64_t block_excl_scan_u64(uint64_t x, uint64_t* s_warp, uint64_t& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint64_t inc = warp_incl_scan(x);
  if (lane == 31) s_warp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const uint64_t w = lane < nw ? s_warp[lane] : 0;
    const uint64_t wi = warp_incl_scan(w);
    if (lane < nw) s_warp[lane] = wi - w;
    if (lane == 31) s_warp[32] = wi;
  }
  __syncthreads();
  const uint64_t res = s_warp[warp] + inc - x;
  total = s_warp[32];
  __syncthreads();
  return res;
}

__device__ inline void finalize_block(const ArrayView& v, const uint64_t* ins_base, const uint64_t* ins_len,
                               uint64_t* cp_prefix, uint32_t copy_chunk_elems, uint64_t* s_warp) {
  uint64_t run_off = 0, run_fl = 0, run_cp = 0;
  for (uint32_t l0 = 0; l0 < v.L; l0 += blockDim.x) {
    const uint32_t l = l0 + threadIdx.x;
    uint64_t size = 0, fl = 0, cp = 0;
    if (l < v.L) {
      size = __ldcg(v.sizes + l);
      fl = bucket_chunks(size, v.log2B, v.E);
      if (cp_prefix) {
        const uint64_t b0 = __ldcg(ins_base + l), n = __ldcg(ins_len + l);
        cp = n ? (b0 + n - 1) / copy_chunk_elems - b0 / copy_chunk_elems + 1 : 0;
      }
    }
    uint64_t tot;
    const uint64_t eo = block_excl_scan_u64(size, s_warp, tot);
    if (l < v.L) v.offsets[l] = run_off + eo;
    run_off += tot;
    const uint64_t ef = block_excl_scan_u64(fl, s_warp, tot);
    if (l < v.L) v.fl_prefix[l] = run_fl + ef;
    run_fl += tot;
    if (cp_prefix) {
      const uint64_t ec = block_excl_scan_u64(cp, s_warp, tot);
      if (l < v.L) cp_prefix[l] = run_cp + ec;
      run_cp += tot;
    }
  }
  if (threadIdx.x == 0) {
    v.offsets[v.L] = run_off;
    v.fl_prefix[v.L] = run_fl;
    if (cp_prefix) cp_prefix[v.L] = run_cp;
  }
}


}  // namespace gga
