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
// stream seeded with `seed`.  The generator's state after key+1 steps is
// seed + (key+1) * GOLDEN (a Weyl sequence); the output is that state
// passed through the mixing function below.
constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;

__device__ __forceinline__ uint64_t splitmix_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// The high 32 bits of splitmix_mix(z): the final xor-shift by 31 changes
// the high word only by its own top bit, so the last step stays in 32 bits.
__device__ __forceinline__ uint32_t splitmix_mix_hi(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  const uint32_t h = static_cast<uint32_t>(z >> 32);
  return h ^ (h >> 31);
}

__device__ __forceinline__ uint64_t splitmix(uint64_t seed, uint64_t key) {
  return splitmix_mix(seed + (key + 1) * kGolden);
}

// The draws of one thread over consecutive rounds, for keys
// (round << 32) | gid.  Write gid = gh * 2^32 + gl (gl < 2^32); the key's
// high word is then uint32(round) | gh and its low word gl, so the state is
//   seed + (gl + 1) * GOLDEN + ((hi_word * GOLDEN) mod 2^32) * 2^32,
// where only the last term depends on the round: one 32-bit multiply and
// one 32-bit add into the state's high word per draw, instead of a 64-bit
// multiply.  Equal to splitmix(seed, (round << 32) | gid) for every gid.
struct RoundDraws {
  uint64_t base;   // seed + (gl + 1) * GOLDEN
  uint32_t gh;     // gid >> 32
  __device__ __forceinline__ RoundDraws() : base(0), gh(0) {}
  __device__ __forceinline__ RoundDraws(uint64_t seed, uint64_t gid)
      : base(seed + ((gid & 0xFFFFFFFFull) + 1ull) * kGolden), gh(static_cast<uint32_t>(gid >> 32)) {}
  __device__ __forceinline__ uint64_t state(uint64_t round) const {
    const uint32_t hw = (static_cast<uint32_t>(round) | gh) * static_cast<uint32_t>(kGolden);
    return base + (static_cast<uint64_t>(hw) << 32);
  }
};

// Count of one draw from the mixed state z.  DIST >= 0 fixes the
// distribution at compile time (GGA_DIST_*), -1 reads g.dist.  Every
// distribution but the geometric one uses only the high word of the draw.
// SEARCH: g lives in shared memory, where a binary search over the
// thresholds costs a few indexed loads; for kernel parameters (constant
// bank) the unrolled count reads each threshold as an operand instead, and
// an indexed read would copy the parameters to local memory.
template <bool SEARCH = false, int DIST = -1>
__device__ __forceinline__ uint32_t gen_count_state(const GenParams& g, uint64_t z) {
  const uint32_t dist = DIST >= 0 ? static_cast<uint32_t>(DIST) : g.dist;
  if (dist == GGA_DIST_GEOMETRIC) {
    const uint64_t inv = ~splitmix_mix(z);
    return inv == 0 ? 63u : min(63u, static_cast<uint32_t>(__ffsll(static_cast<long long>(inv)) - 1));
  }
  const uint32_t u = splitmix_mix_hi(z);
  if (dist == GGA_DIST_BERNOULLI) return u >> 31;
  if (dist == GGA_DIST_UNIFORM3) return __umulhi(u, 3u);
  // c = #{k < nthr : u >= thr[k]}.  Ascending thresholds (the CDF of the
  // distribution, the usual case) make that set a prefix, whose length a
  // binary search finds in five steps; other tables are counted.
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

// Count of draw h = splitmix(seed, key) (the whole 64-bit output).
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
// t = t0 * kv + i, kv = ceil(T / blockDim) <= KV <= 4), the per-thread round
// sums are scanned two rounds per 32-bit word (sums < 2^16 per block: counts
// are below 64 and blockDim * KV * 63 < 2^16), warp 0 scans the warp totals and its
// lane 0 makes one size reservation for the pass -- clipped at `target`,
// and, if the pool cannot hold the buckets it reaches, cut back to the
// longest prefix of whole rounds that fits -- and takes the buckets
// (Algorithm 2); then (synchronize) the values go to a shared-memory stage
// at their positions and the block streams the stage to the buckets with
// aligned 128-bit stores (a pass larger than the stage writes straight to
// the buckets).  Elements past the target are the ones a round-by-round
// growth would clip (positions are round-major).  The LFVector's bucket
// table is kept in shared memory, so the write-out finds a bucket's
// address without a global load.

__device__ __forceinline__ uint32_t warp_incl_scan_u32(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += n;
  }
  return v;
}

// Largest count a distribution draws (0 when it has no small bound).
template <int DIST>
__host__ __device__ constexpr uint32_t max_count() {
  return DIST == GGA_DIST_BERNOULLI ? 1u : (DIST == GGA_DIST_UNIFORM3 ? 2u : 0u);
}

struct GenShared {
  uint32_t wt[4][32];         // packed warp prefixes (K / 2 <= 4 words)
  uint32_t rb[9];             // pass-relative start of every round (K <= 8)
  uint64_t base;              // LFVector size before the pass
  uint32_t commit, nb;
  int stop;                   // 1: pool exhausted, 2: target reached
  uint64_t tab[kMaxBuckets];  // the LFVector's bucket table (copy)
  // Threshold counts (ascending thresholds) per interval of 2^24 draws:
  // ptab[i] holds c_i = #{k : thr[k] <= i * 2^24} in its top 7 bits and, in
  // its low 25, the offset of the next threshold thr[c_i] from i * 2^24 when
  // that threshold lies inside the interval, else 2^24 (no draw of the
  // interval reaches it).  A draw u of interval i counts c_i when its low 24
  // bits stay below that offset -- one table load -- and otherwise steps
  // over the thresholds from c_i + 1.
  uint32_t thr[GGA_MAX_THRESHOLDS];
  uint32_t ptab[256];
};

// Count of draw u (the high word) against ascending thresholds through the
// table: start from the thresholds below u's interval of 2^24, then step
// over those inside it.  Equal to #{k < nthr : u >= thr[k]}.
__device__ __forceinline__ uint32_t table_count(const GenShared& sh, uint32_t nthr, uint32_t u) {
  const uint32_t e = sh.ptab[u >> 24];
  uint32_t c = e >> 25;
  if ((u & 0xFFFFFFu) >= (e & 0x1FFFFFFu)) {
    ++c;
    while (c < nthr && u >= sh.thr[c]) ++c;
  }
  return c;
}

// Returns the number of rounds it drew; *done is set when the LFVector
// reached `target` or the pool ran out.  Every thread of the block calls
// it.  SEARCH as for gen_count (g in shared memory); DIST as for
// gen_count_state (-1: g.dist at run time).
template <int E, int K, int KV, bool SEARCH = false, int DIST = -1>
__device__ uint32_t grow_passes(const ArrayView& v, const GenParams& g, uint32_t l, uint32_t R, uint64_t target,
                                GenShared& sh, uint4* stage4, uint32_t cap, bool* done) {
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
  RoundDraws dv[KV];   // virtual threads gfirst, ..., gfirst + KV - 1
#pragma unroll
  for (int i = 0; i < KV; ++i) dv[i] = RoundDraws(g.seed, gfirst + i);
  if (t0 == 0) {
    sh.base = v.sizes[l];
    sh.nb = v.nbuckets[l];
    sh.stop = sh.base >= target ? 2 : 0;
  }
  {
    const uint32_t nb0 = v.nbuckets[l];
    for (uint32_t i = t0; i < nb0; i += NT) sh.tab[i] = bk[i];
  }
  const bool tabled = DIST == GGA_DIST_POISSON && g.thr_sorted;   // uniform
  if (tabled) {
    for (uint32_t i = t0; i < GGA_MAX_THRESHOLDS; i += NT) sh.thr[i] = g.thr[i];
    for (uint32_t i = t0; i < 256; i += NT) {
      uint32_t c = 0;
      for (uint32_t k = 0; k < g.nthr; ++k) c += g.thr[k] <= (i << 24) ? 1u : 0u;
      const uint64_t lo = static_cast<uint64_t>(i) << 24;
      const uint32_t rel = c < g.nthr && g.thr[c] < lo + (1u << 24) ? static_cast<uint32_t>(g.thr[c] - lo) : (1u << 24);
      sh.ptab[i] = (c << 25) | rel;
    }
  }
  __syncthreads();
  uint32_t r0 = 0;
  while (r0 < R && sh.stop == 0) {
    const uint32_t kk = min(static_cast<uint32_t>(K), R - r0);
    // pk: the thread's per-round sums, two rounds per word.  cw: with KV
    // virtual threads, the counts of the first KV - 1 of them, one byte
    // each (round k, virtual thread i at byte k * (KV - 1) + i; the last
    // one's count is the sum minus theirs); with one, the count is pk's
    // half-word.
    constexpr int KC = KV > 1 ? (K * (KV - 1) + 3) / 4 : 1;
    uint32_t pk[KP], inc[KP], cw[KC];
#pragma unroll
    for (int q = 0; q < KC; ++q) cw[q] = 0;
#pragma unroll
    for (int j = 0; j < KP; ++j) {
      uint32_t c[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint32_t k = 2 * j + h;
        const uint64_t r = static_cast<uint64_t>(g.round0) + r0 + k;
        uint32_t sum = 0;
#pragma unroll
        for (int i = 0; i < KV; ++i) {
          uint32_t ci = 0;
          if (k < kk && (KV == 1 || static_cast<uint32_t>(i) < kv) && tfirst + i < v.T) {
            if (DIST == GGA_DIST_POISSON && tabled) ci = table_count(sh, g.nthr, splitmix_mix_hi(dv[i].state(r)));
            else ci = gen_count_state<SEARCH, DIST>(g, dv[i].state(r));
          }
          if (KV > 1 && i < KV - 1) {
            const int q = static_cast<int>(k) * (KV - 1) + i;
            cw[KV > 1 ? q / 4 : 0] |= ci << (8 * (q % 4));
          }
          sum += ci;
        }
        c[h] = sum;
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
            for (uint32_t i = nb; i < got; ++i) sh.tab[i] = bk[i];
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
    // Fast path (block-uniform): the whole pass is kept and staged, so no
    // element needs the clipping test or the bucket math.
    const bool whole = staged && commit == sh.rb[K];
    typedef typename std::conditional<E == 4, uint32_t, uint64_t>::type V;
    // Element m of virtual thread i in round k: va * gid + vb * round + vc * m
    // (a 4-byte element keeps the low 32 bits, which 32-bit arithmetic gives
    // exactly).
    // The value parameters in registers: g may live in shared memory, where
    // the stage stores below could alias it and force a reload per element.
    const V va = static_cast<V>(g.va), vb = static_cast<V>(g.vb), vc = static_cast<V>(g.vc);
    const V vr = va * static_cast<V>(gfirst) + vb * static_cast<V>(static_cast<uint64_t>(g.round0) + r0);
    // Counts without a small bound, two virtual threads per thread (below):
    // one store loop over the run of both.  (With four the switch points
    // cost registers the kernels do not have.)
    constexpr bool kMergedRun = KV == 2 && !(DIST >= 0 && max_count<DIST>() > 0 && max_count<DIST>() <= 2);
#pragma unroll
    for (int j = 0; j < KP; ++j) {
      const uint32_t ex = sh.wt[j][warp] + inc[j] - pk[j];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint32_t k = 2 * j + h;
        uint32_t st = sh.rb[k] + ((ex >> (16 * h)) & 0xFFFFu);
        const uint32_t csum = (pk[j] >> (16 * h)) & 0xFFFFu;
        if (kMergedRun && whole) {
          // The thread's virtual threads own consecutive positions of the
          // round, so their elements form one run of csum positions from
          // st: one loop over the run, moving to the next virtual thread's
          // values at its first position (an empty virtual thread's switch
          // point equals the next one's, and the later switch wins).  One
          // shared-memory store per warp iteration over the run, against one
          // per iteration of each virtual thread's own loop.
          uint32_t sw[KV > 1 ? KV - 1 : 1];
          uint32_t acc = 0;
#pragma unroll
          for (int i = 0; i < KV - 1; ++i) {
            const int q = static_cast<int>(k) * (KV - 1) + i;
            acc += (cw[q / 4] >> (8 * (q % 4))) & 0xFFu;
            sw[i] = acc;
          }
          const V v0 = vr + vb * static_cast<V>(k);
          V val = v0;
          for (uint32_t m = 0; m < csum; ++m, val += vc) {
#pragma unroll
            for (int i = 0; i < KV - 1; ++i)
              if (m == sw[i]) val = v0 + va * static_cast<V>(i + 1);
            stage[st + m + shv] = gen_value<E>(val);
          }
          continue;
        }
        uint32_t before = 0;   // elements of the earlier virtual threads of this round
#pragma unroll
        for (int i = 0; i < KV; ++i) {
          uint32_t c = csum - before;
          if (KV > 1 && i < KV - 1) {
            const int q = static_cast<int>(k) * (KV - 1) + i;
            c = (cw[KV > 1 ? q / 4 : 0] >> (8 * (q % 4))) & 0xFFu;
          }
          before += c;
          V val = vr + va * static_cast<V>(i) + vb * static_cast<V>(k);
          if (whole && DIST >= 0 && max_count<DIST>() > 0 && max_count<DIST>() <= 2) {
            // At most two elements: predicated stores, no loop.
            if (c > 0) stage[st + shv] = gen_value<E>(val);
            if (max_count<DIST>() > 1 && c > 1) stage[st + 1 + shv] = gen_value<E>(val + vc);
          } else if (whole) {
            for (uint32_t m = 0; m < c; ++m, val += vc) stage[st + m + shv] = gen_value<E>(val);
          } else {
            for (uint32_t m = 0; m < c; ++m, val += vc) {
              const uint32_t q = st + m;
              if (q >= commit) break;
              if (staged) {
                stage[q + shv] = gen_value<E>(val);
              } else {
                uint32_t bb;
                uint64_t off;
                bucket_of(base + q, v.log2B, bb, off);
                reinterpret_cast<T*>(sh.tab[bb])[off] = gen_value<E>(val);
              }
            }
          }
          st += c;
        }
      }
    }
    __syncthreads();
    if (staged && commit) stage_to_buckets<T>(sh.tab, v.log2B, v.B, base, commit, shv, stage4, t0, NT);
    // No barrier here: the next pass writes the stage, sh.wt, sh.rb and
    // sh.commit only after its first two barriers, which every thread reaches
    // after finishing this pass; sh.base is written by thread 0 and read by
    // thread 0 (the leader) before the next pass's second barrier and by the
    // others after it; sh.stop was set before this pass's second barrier;
    // sh.tab only gains entries past those this pass reads.
    if (t0 == 0) sh.base = base + commit;
    r0 += kk;
  }
  *done = sh.stop != 0;
  __syncthreads();   // the caller may reuse the stage and sh
  return r0;
}

}  // namespace gga
