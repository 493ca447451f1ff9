// gga_twophase.cu -- the two-phase case study (Sec. VI-D) on the GGArray.
//
// Insertion phase: an application kernel grows the array from inside the
// kernel.  Every parent record spawns Geometric(1/2) - 1 children that the
// kernel push_backs into the parent's own LFVector (Algorithm 1 called by the
// application, with thread coarsening).  Work phase: the array is flattened
// (gga_flatten) and a streaming kernel updates the contiguous copy.
//
// Records are 16 bytes {uint64 id, float pos, float vel}.  The count of the
// parent at local index j of LFVector l in generation `gen` is the number of
// trailing one bits of SplitMix64 draw ((gen << 48) | (offsets[l] + j)) + 1 of
// the stream seeded with `seed`; children follow parent order, a parent's
// children consecutively, and child k of a parent is the parent with
// id = ((gen + 1) << 56) | (l << 40) | (the child's LFVector-local index).
#include "gga_core.cuh"

namespace gga {

int launch_finalize(const ArrayView& v, cudaStream_t st);

namespace {

__device__ __forceinline__ uint64_t splitmix2(uint64_t seed, uint64_t key) {
  uint64_t z = seed + (key + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Geometric(1/2) - 1: trailing one bits of h, at most 63.
__device__ __forceinline__ uint32_t trailing_ones(uint64_t h) {
  const uint64_t inv = ~h;
  return inv == 0 ? 63u : min(63u, static_cast<uint32_t>(__ffsll(static_cast<long long>(inv)) - 1));
}

__device__ __forceinline__ uint32_t warp_scan_packed(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += n;
  }
  return v;
}

constexpr int kSpawnP = 8;   // parents per thread per pass (coarsening)

// One block per LFVector.  Parents of a pass are j = c0 + p*NT + t (p < P),
// so the block reads them coalesced and their order is (p, t): the same
// round-major order the packed two-counter scan produces.  The children of
// round p of a warp form one run of the LFVector; the warp writes that run
// cooperatively, lane i taking children i, i+32, ...: the lane finds the
// child's parent (the last lane whose exclusive count is <= i, a five-step
// shuffle search), takes the parent's pos and vel by shuffle and stores the
// child at its bucket position.  Consecutive lanes store consecutive
// children, so the stores are coalesced without a shared-memory stage, and
// no lane loops over a long run of its own.
template <int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) spawn_kernel(ArrayView v, uint32_t gen, uint64_t seed, int only_newborn,
                                                           uint64_t* born) {
  constexpr int KP = kSpawnP / 2;
  __shared__ uint32_t s_wt[KP][32];
  __shared__ uint32_t s_rb[kSpawnP + 1];
  __shared__ uint64_t s_base;
  __shared__ uint32_t s_commit, s_nb;
  __shared__ int s_stop;

  const uint32_t l = blockIdx.x, t = threadIdx.x, NT = blockDim.x;
  const int lane = t & 31, warp = t >> 5, nwarps = NT >> 5;
  const uint64_t* bk = v.buckets + static_cast<uint64_t>(l) * kMaxBuckets;
  const uint64_t s = v.sizes[l];                       // parents end here
  const uint64_t first = only_newborn ? born[l] : 0;   // ... and start here
  const uint64_t goff = v.offsets[l];                  // global index of local 0 at generation start
  const uint64_t id_hi = (static_cast<uint64_t>(gen + 1) << 56) | (static_cast<uint64_t>(l) << 40);
  if (t == 0) {
    s_base = s;
    s_nb = v.nbuckets[l];
    s_stop = 0;
  }
  __syncthreads();

  for (uint64_t c0 = first; c0 < s; c0 += static_cast<uint64_t>(NT) * kSpawnP) {
    uint2 pv[kSpawnP];   // parents' pos and vel (the children's copy)
    uint32_t pk[KP], inc[KP];
#pragma unroll
    for (int j2 = 0; j2 < KP; ++j2) {
      uint32_t c[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int p = 2 * j2 + h;
        const uint64_t j = c0 + static_cast<uint64_t>(p) * NT + t;
        c[h] = 0;
        pv[p] = make_uint2(0, 0);
        if (j < s) {
          uint32_t bb;
          uint64_t off;
          bucket_of(j, v.log2B, bb, off);
          const uint4 rec = *reinterpret_cast<const uint4*>(bk[bb] + off * 16);
          pv[p] = make_uint2(rec.z, rec.w);
          c[h] = trailing_ones(splitmix2(seed, (static_cast<uint64_t>(gen) << 48) | (goff + j)));
        }
      }
      pk[j2] = c[0] | (c[1] << 16);
      inc[j2] = warp_scan_packed(pk[j2]);
      if (lane == 31) s_wt[j2][warp] = inc[j2];
    }
    __syncthreads();
    if (warp == 0) {
      uint32_t rb = 0;
#pragma unroll
      for (int j2 = 0; j2 < KP; ++j2) {
        const uint32_t w = lane < nwarps ? s_wt[j2][lane] : 0u;
        const uint32_t wi = warp_scan_packed(w);
        if (lane < nwarps) s_wt[j2][lane] = wi - w;
        const uint32_t tot = __shfl_sync(0xffffffffu, wi, 31);
        if (lane == 0) {
          s_rb[2 * j2] = rb;
          rb += tot & 0xFFFFu;
          s_rb[2 * j2 + 1] = rb;
          rb += tot >> 16;
        }
      }
      if (lane == 0) {
        s_rb[kSpawnP] = rb;
        // Leader: one reservation for the pass, Algorithm 2 for the buckets.
        const uint64_t base = s_base;
        uint32_t commit = rb;
        if (rb > 0) {
          const uint32_t nb = s_nb;
          const uint32_t need = buckets_for(base + rb, v.log2B);
          if (need > nb) {
            const uint32_t got = grow_buckets(v, l, nb, need);
            s_nb = got;
            v.nbuckets[l] = got;
            if (got < need) {
              const uint64_t cap = bucket_first(got, v.log2B);
              int kf = 0;
              while (kf < kSpawnP && base + s_rb[kf + 1] <= cap) ++kf;
              commit = s_rb[kf];
              s_stop = 1;
              latch_error(v.status, GGA_ERR_POOL_EXHAUSTED);
            }
          }
        }
        s_commit = commit;
        v.sizes[l] = base + commit;
      }
    }
    __syncthreads();   // synchronize(): the buckets exist before any write

    const uint64_t base = s_base;
    const uint32_t commit = s_commit;
#pragma unroll
    for (int j2 = 0; j2 < KP; ++j2) {
      const uint32_t wo = s_wt[j2][warp];                       // the warp's offset in rounds 2j2, 2j2+1
      const uint32_t ex = inc[j2] - pk[j2];                     // the lane's, inside the warp
      const uint32_t wt = __shfl_sync(0xffffffffu, inc[j2], 31);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int p = 2 * j2 + h;
        const uint32_t exl = (ex >> (16 * h)) & 0xFFFFu;
        const uint32_t wtot = (wt >> (16 * h)) & 0xFFFFu;
        const uint32_t q0 = s_rb[p] + ((wo >> (16 * h)) & 0xFFFFu);   // block position of the warp's run
        for (uint32_t i0 = 0; i0 < wtot; i0 += 32) {
          const uint32_t q = i0 + lane;
          uint32_t src = 0;
#pragma unroll
          for (uint32_t step = 16; step > 0; step >>= 1) {
            const uint32_t e = __shfl_sync(0xffffffffu, exl, src + step);
            if (e <= q) src += step;
          }
          const uint32_t pos = __shfl_sync(0xffffffffu, pv[p].x, src);
          const uint32_t vel = __shfl_sync(0xffffffffu, pv[p].y, src);
          if (q < wtot && q0 + q < commit) {
            const uint64_t local = base + q0 + q;
            const uint64_t id = id_hi | local;
            uint32_t bb;
            uint64_t off;
            bucket_of(local, v.log2B, bb, off);
            __stcs(reinterpret_cast<uint4*>(bk[bb] + off * 16),
                   make_uint4(static_cast<uint32_t>(id), static_cast<uint32_t>(id >> 32), pos, vel));
          }
        }
      }
    }
    // No block barrier here: the next pass writes s_rb, s_commit and the
    // warp-offset entries of s_wt only after its first barrier, which every
    // thread reaches after finishing this pass; the one entry a warp writes
    // before that barrier (lane 31: s_wt[.][warp]) is its own, read by its
    // lanes above (the warp synchronizes first).  s_base is written by
    // thread 0 and read by thread 0 (the leader) before the next pass's
    // second barrier and by the others after it; s_stop was set before this
    // pass's second barrier.
    __syncwarp();
    if (t == 0) s_base = base + commit;
    if (s_stop) break;
  }
  if (t == 0 && only_newborn) born[l] = s;
}

// One streaming pass over flattened records: pos += vel.
__global__ void __launch_bounds__(256) work_pass_kernel(uint4* __restrict__ rec, uint64_t n) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  constexpr int U = 4;
  for (uint64_t i0 = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i0 < n; i0 += stride * U) {
    uint4 r[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (i0 + u * stride < n) r[u] = __ldcs(rec + i0 + u * stride);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (i0 + u * stride < n) {
        r[u].z = __float_as_uint(__fadd_rn(__uint_as_float(r[u].z), __uint_as_float(r[u].w)));
        __stcs(rec + i0 + u * stride, r[u]);
      }
    }
  }
}

}  // namespace

int launch_twophase_spawn(const ArrayView& v, uint32_t gen, uint64_t seed, int only_newborn, uint64_t* born,
                          cudaStream_t st) {
  // The children's order and values depend on parent indices only, so the
  // block size is free: 1024 threads, one block per SM, whatever T is.
  // With 1024 LFVectors that is 6.7 waves of blocks (7 rounds), against 3.4
  // (4 rounds) with two 512-thread blocks per SM.
  spawn_kernel<1024, 1><<<v.L, 1024, 0, st>>>(v, gen, seed, only_newborn, born);
  if (cudaGetLastError() != cudaSuccess) return GGA_ERR_CUDA;
  return launch_finalize(v, st);
}

int launch_twophase_work(void* records, uint64_t n, uint32_t passes, int num_sms, cudaStream_t st) {
  if (n == 0) return GGA_OK;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, work_pass_kernel, 256, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const uint64_t want = (n + 255) / 256;
  const uint64_t wave = static_cast<uint64_t>(num_sms) * per_sm;
  const unsigned grid = static_cast<unsigned>(want < wave ? want : wave);
  for (uint32_t p = 0; p < passes; ++p)
    work_pass_kernel<<<grid, 256, 0, st>>>(static_cast<uint4*>(records), n);
  return cudaGetLastError() == cudaSuccess ? GGA_OK : GGA_ERR_CUDA;
}

}  // namespace gga
