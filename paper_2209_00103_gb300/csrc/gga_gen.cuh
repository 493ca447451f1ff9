// gga_gen.cuh -- device helpers shared by the insertion kernels: the
// counter-based draws of the generated workloads, and the block-wide
// finalize (prefix sum of LFVector sizes, Sec. IV; work lists).
#pragma once

#include <type_traits>

#include "gga_core.cuh"

namespace gga {

struct GenParams {
  uint64_t seed, va, vb, vc;
  uint32_t dist, nthr, round0;
  uint32_t thr_sorted;   // 1: thr[0..nthr) ascending (set on the host)
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

// SEARCH: g lives in shared memory, where a binary search over the
// thresholds costs a few indexed loads; for kernel parameters (constant
// bank) the unrolled count reads each threshold as an operand instead, and
// an indexed read would copy the parameters to local memory.
template <bool SEARCH = false>
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
      // c = #{k < nthr : u >= thr[k]}.  Ascending thresholds (the CDF of the
      // distribution, the usual case) make that set a prefix, whose length
      // a binary search finds in five steps; other tables are counted.
      const uint32_t u = static_cast<uint32_t>(h >> 32);
      uint32_t c = 0;
      if (SEARCH && g.thr_sorted) {
#pragma unroll
        for (uint32_t step = 16; step > 0; step >>= 1)
          if (c + step <= g.nthr && u >= g.thr[c + step - 1]) c += step;
      } else {
#pragma unroll
        for (uint32_t k = 0; k < GGA_MAX_THRESHOLDS; ++k) c += (k < g.nthr) & (u >= g.thr[k]);
      }
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
  g.thr_sorted = 1;
  for (int i = 0; i < GGA_MAX_THRESHOLDS; ++i) g.thr[i] = spec.thresholds[i];
  for (uint32_t i = 1; i < spec.n_thresholds && i < GGA_MAX_THRESHOLDS; ++i)
    if (g.thr[i] < g.thr[i - 1]) g.thr_sorted = 0;
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


// ---------------------------------------------------------------------------
// Growth of one LFVector by rounds of in-thread insertions (the in-kernel
// push_back of Algorithm 1, positions from Sec. III-B's block prefix sum),
// K rounds per pass.  Shared by the generated insertion (one block per
// LFVector, a fixed number of rounds) and the batched growth (a persistent
// block per item, rounds until the LFVector's target).
//
// Per pass every thread draws its counts for K rounds (virtual threads
// t = t0 * kv + i, kv = ceil(T / blockDim) <= KV), the per-thread round sums
// are scanned two rounds per 32-bit word (sums < 2^16 per block: counts are
// below 64 and blockDim * kv <= 1024), thread 0 makes one size reservation
// for the pass -- clipped at `target`, and, if the pool cannot hold the
// buckets it reaches, cut back to the longest prefix of whole rounds that
// fits -- and takes the buckets (Algorithm 2); then (synchronize) the values
// go to a shared-memory stage at their positions and the block streams the
// stage to the buckets with aligned 128-bit stores (a pass larger than the
// stage writes straight to the buckets).  Elements past the target are the
// ones a round-by-round growth would clip (positions are round-major).

__device__ __forceinline__ uint32_t warp_incl_scan_u32(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += n;
  }
  return v;
}

struct GenShared {
  uint32_t wt[4][32];   // packed warp prefixes (K / 2 <= 4 words)
  uint32_t rb[9];       // pass-relative start of every round (K <= 8)
  uint64_t base;        // LFVector size before the pass
  uint32_t commit, nb;
  int stop;             // 1: pool exhausted, 2: target reached
};

template <int E>
__device__ __forceinline__ void put_gen_elem(uint64_t addr, typename Elem<E>::T x) {
  *reinterpret_cast<typename Elem<E>::T*>(addr) = x;
}

// Returns the number of rounds it drew.  Every thread of the block calls it.
// SEARCH as for gen_count (g in shared memory).
template <int E, int K, int KV, bool SEARCH = false>
__device__ uint32_t grow_passes(const ArrayView& v, const GenParams& g, uint32_t l, uint32_t R, uint64_t target,
                                GenShared& sh, uint4* stage4, uint32_t cap) {
  typedef typename Elem<E>::T T;
  constexpr uint32_t VEC = 16 / E;
  constexpr int KP = K / 2;
  static_assert(K % 2 == 0 && K <= 8, "K rounds per pass: even, at most 8");
  T* stage = reinterpret_cast<T*>(stage4);
  const uint32_t t0 = threadIdx.x, NT = blockDim.x;
  const int lane = t0 & 31, warp = t0 >> 5, nwarps = NT >> 5;
  const uint32_t kv = KV == 1 ? 1u : (v.T + NT - 1) / NT;
  const uint64_t tfirst = static_cast<uint64_t>(t0) * kv;        // first virtual thread
  const uint64_t gfirst = static_cast<uint64_t>(l) * v.T + tfirst;
  const uint64_t* bk = v.buckets + static_cast<uint64_t>(l) * kMaxBuckets;
  const bool group_ok = v.B >= VEC;
  if (t0 == 0) {
    sh.base = v.sizes[l];
    sh.nb = v.nbuckets[l];
    sh.stop = sh.base >= target ? 2 : 0;
  }
  __syncthreads();
  uint32_t r0 = 0;
  while (r0 < R && sh.stop == 0) {
    const uint32_t kk = min(static_cast<uint32_t>(K), R - r0);
    uint32_t pk[KP], inc[KP], cc[K];
#pragma unroll
    for (int j = 0; j < KP; ++j) {
      uint32_t c[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint32_t k = 2 * j + h;
        const uint64_t r = static_cast<uint64_t>(g.round0) + r0 + k;
        uint32_t c0 = 0, c1 = 0;
        if (k < kk) {
          if (tfirst < v.T) c0 = gen_count<SEARCH>(g, splitmix(g.seed, (r << 32) | gfirst));
          if (KV > 1 && kv > 1 && tfirst + 1 < v.T)
            c1 = gen_count<SEARCH>(g, splitmix(g.seed, (r << 32) | (gfirst + 1)));
        }
        cc[k] = c0 | (c1 << 8);
        c[h] = c0 + c1;
      }
      pk[j] = c[0] | (c[1] << 16);
      inc[j] = warp_incl_scan_u32(pk[j]);
      if (lane == 31) sh.wt[j][warp] = inc[j];
    }
    __syncthreads();
    if (warp == 0) {
      uint32_t rb = 0;
#pragma unroll
      for (int j = 0; j < KP; ++j) {
        const uint32_t w = lane < nwarps ? sh.wt[j][lane] : 0u;
        const uint32_t wi = warp_incl_scan_u32(w);
        if (lane < nwarps) sh.wt[j][lane] = wi - w;
        const uint32_t tot = __shfl_sync(0xffffffffu, wi, 31);
        if (lane == 0) {
          sh.rb[2 * j] = rb;
          rb += tot & 0xFFFFu;
          sh.rb[2 * j + 1] = rb;
          rb += tot >> 16;
        }
      }
      if (lane == 0) {
        sh.rb[K] = rb;
        const uint64_t base = sh.base;
        const uint64_t rem = target - base;   // > 0 while the loop runs
        uint32_t commit = rb < rem ? rb : static_cast<uint32_t>(rem);
        if (commit > 0) {
          const uint32_t nb = sh.nb;
          const uint32_t need = buckets_for(base + commit, v.log2B);
          if (need > nb) {
            const uint32_t got = grow_buckets(v, l, nb, need);
            sh.nb = got;
            v.nbuckets[l] = got;
            if (got < need) {
              const uint64_t capg = bucket_first(got, v.log2B);
              int kf = 0;
              while (kf < K && base + sh.rb[kf + 1] <= capg) ++kf;
              if (sh.rb[kf] < commit) commit = sh.rb[kf];
              sh.stop = 1;
              latch_error(v.status, GGA_ERR_POOL_EXHAUSTED);
            }
          }
        }
        if (sh.stop == 0 && base + commit >= target) sh.stop = 2;
        sh.commit = commit;
        v.sizes[l] = base + commit;
      }
    }
    __syncthreads();   // synchronize(): the buckets exist before any write

    const uint64_t base = sh.base;
    const uint32_t commit = sh.commit;
    const uint32_t shv = static_cast<uint32_t>(base & (VEC - 1));   // stage index = pass position + shv
    const bool staged = commit + shv <= cap;
#pragma unroll
    for (int j = 0; j < KP; ++j) {
      const uint32_t ex = sh.wt[j][warp] + inc[j] - pk[j];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint32_t k = 2 * j + h;
        uint32_t st = sh.rb[k] + ((ex >> (16 * h)) & 0xFFFFu);
#pragma unroll
        for (int i = 0; i < KV; ++i) {
          const uint32_t c = (cc[k] >> (8 * i)) & 0xFFu;
          if (c == 0) continue;
          // A 4-byte element keeps the low 32 bits of the value, which
          // 32-bit arithmetic gives exactly.
          typedef typename std::conditional<E == 4, uint32_t, uint64_t>::type V;
          V val = static_cast<V>(g.va) * static_cast<V>(gfirst + i) +
                  static_cast<V>(g.vb) * static_cast<V>(static_cast<uint64_t>(g.round0) + r0 + k);
          for (uint32_t m = 0; m < c; ++m, val += static_cast<V>(g.vc)) {
            const uint32_t q = st + m;
            if (q >= commit) break;
            if (staged) {
              stage[q + shv] = gen_value<E>(val);
            } else {
              uint32_t bb;
              uint64_t off;
              bucket_of(base + q, v.log2B, bb, off);
              put_gen_elem<E>(bk[bb] + off * E, gen_value<E>(val));
            }
          }
          st += c;
        }
      }
    }
    __syncthreads();
    if (staged && commit) {
      const uint64_t gbeg = base - shv;
      const uint32_t nvec = (commit + shv + VEC - 1) / VEC;
      for (uint32_t vi = t0; vi < nvec; vi += NT) {
        const uint64_t p = gbeg + static_cast<uint64_t>(vi) * VEC;
        const uint32_t lo = vi * VEC;   // stage index of p
        if (group_ok && lo >= shv && lo + VEC <= commit + shv) {
          uint32_t bb;
          uint64_t off;
          bucket_of(p, v.log2B, bb, off);
          __stcs(reinterpret_cast<uint4*>(bk[bb] + off * E), stage4[vi]);
        } else {
#pragma unroll
          for (uint32_t e = 0; e < VEC; ++e) {
            const uint32_t si = lo + e;
            if (si < shv || si >= commit + shv) continue;
            uint32_t bb;
            uint64_t off;
            bucket_of(p + e, v.log2B, bb, off);
            put_gen_elem<E>(bk[bb] + off * E, stage[si]);
          }
        }
      }
    }
    // No barrier here: the next pass writes the stage, sh.wt, sh.rb and
    // sh.commit only after its first two barriers, which every thread reaches
    // after finishing this pass; sh.base is written by thread 0 and read by
    // thread 0 (the leader) before the next pass's second barrier and by the
    // others after it; sh.stop was set before this pass's second barrier.
    if (t0 == 0) sh.base = base + commit;
    r0 += kk;
  }
  __syncthreads();   // the caller may reuse the stage and sh
  return r0;
}

}  // namespace gga
