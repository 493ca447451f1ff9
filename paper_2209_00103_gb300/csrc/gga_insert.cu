// gga_insert.cu -- batched block-level insertion (Algorithm 1 over R rounds).
//
// Host-buffer form (gga_insert): counts[r][l][t] and values packed in
// (round, block, thread, k) order.  Three kernels:
//   1. count_scan: one streaming pass over the counts.  Row (r, l) of T counts
//      is reduced to the run length of block l in round r, and a single-pass
//      decoupled look-back scan (Merrill and Garland, 2016) over the rows in
//      memory order gives voff[r*L + l], the index of that run's first value.
//   2. reserve: one warp per LFVector.  A shuffle scan over the rounds gives
//      each round's position in the batch (the per-round size reservation of
//      Algorithm 1, done for all rounds at once), then the warp's leader
//      allocates every bucket the batch reaches from the device pool
//      (Algorithm 2) and commits the new size.  The last block to finish
//      recomputes the prefix sum of LFVector sizes (Sec. IV) and the work
//      lists of the copy, flatten and rw_b kernels.
//   3. copy: the elements are written at their prefix-sum positions.  Because
//      the values arrive packed in prefix-sum order, element q of LFVector l's
//      batch is value voff[r*L + l] + (q - pre[l][r]) for the round r whose run
//      holds q; the kernel walks destinations in 16-byte groups so every store
//      is a full aligned 128-bit store inside a bucket.
//
// In-kernel form (gga_insert_generated): each block is one LFVector; its
// threads draw their counts, run a warp-shuffle block scan (Sec. III-B), the
// leader thread reserves and allocates (Algorithms 1-2), __syncthreads is the
// synchronize() of Algorithm 1, and the block writes the run.  K rounds share
// one scan pass to amortise the barriers.
#include "gga_core.cuh"

namespace gga {

constexpr uint32_t kCopyChunkBytes = 32768;
constexpr uint32_t kCopyWindow = 1024;       // rounds kept in shared memory per copy chunk
constexpr int kCountThreads = 256;

// ---------------------------------------------------------------------------
// Finalize: prefix sum of sizes, flatten/rw_b chunk prefix, copy chunk prefix.
// Run by one block (any multiple of 32 threads, <= 1024).

__device__ uint64_t block_excl_scan_u64(uint64_t x, uint64_t* s_warp, uint64_t& total) {
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

__device__ void finalize_block(const ArrayView& v, const uint64_t* ins_base, const uint64_t* ins_len,
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

__global__ void __launch_bounds__(1024) finalize_kernel(ArrayView v) {
  __shared__ uint64_t s_warp[33];
  finalize_block(v, nullptr, nullptr, nullptr, 1, s_warp);
}

// ---------------------------------------------------------------------------
// 1. count_scan.

constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagPrefix = 2ull << 62;
constexpr unsigned long long kFlagError = 3ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1;

// Decoupled look-back by one full warp: publishes this tile's aggregate,
// sums predecessors' aggregates until one with an inclusive prefix, publishes
// the tile's inclusive prefix.  Returns the exclusive prefix on every lane.
// Tiles are numbered by a ticket taken at block start, so every predecessor
// is running or done; the wait is still bounded and an error poisons the
// chain instead of hanging it.
__device__ uint64_t lookback(uint32_t tile, uint64_t agg, unsigned long long* ts, uint32_t* err_flag) {
  const int lane = threadIdx.x & 31;
  volatile unsigned long long* vts = ts;
  if (tile == 0) {
    if (lane == 0) vts[0] = kFlagPrefix | (agg & kValMask);
    return 0;
  }
  if (lane == 0) vts[tile] = kFlagAgg | (agg & kValMask);
  uint64_t run = 0;
  int64_t pred = static_cast<int64_t>(tile) - 1;
  uint32_t spins = 0;
  bool bad = false;
  while (true) {
    const int64_t idx = pred - lane;
    const unsigned long long word = idx >= 0 ? static_cast<unsigned long long>(vts[idx]) : (kFlagPrefix + 0ull);
    const unsigned long long flag = word & ~kValMask;
    if (__any_sync(0xffffffffu, flag == 0)) {
      if (++spins > kSpinLimit) { bad = true; break; }
      __nanosleep(32);
      continue;
    }
    if (__any_sync(0xffffffffu, flag == kFlagError)) { bad = true; break; }
    const uint32_t pm = __ballot_sync(0xffffffffu, flag == kFlagPrefix);
    const uint64_t val = word & kValMask;
    if (pm) {
      const int first = __ffs(pm) - 1;
      run += warp_sum_u64(lane <= first ? val : 0);
      break;
    }
    run += warp_sum_u64(val);
    pred -= 32;
  }
  if (lane == 0) {
    vts[tile] = bad ? kFlagError : (kFlagPrefix | ((run + agg) & kValMask));
    if (bad) atomicExch(err_flag, 1u);
  }
  return run;
}

__host__ __device__ constexpr int count_rows_per_warp(int T_TPL) {
  return T_TPL == 0 ? 4 : (T_TPL >= 1024 ? 2 : 2048 / T_TPL);
}

__host__ __device__ constexpr int count_rows_per_tile(int T_TPL) {
  return (kCountThreads / 32) * count_rows_per_warp(T_TPL);
}

// T_TPL > 0: T == T_TPL (a multiple of 128) and counts 16-byte aligned, the
// row is read with 128-bit loads.  T_TPL == 0: any T, 32-bit loads.
template <int T_TPL>
__global__ void __launch_bounds__(kCountThreads) count_scan_kernel(const uint32_t* __restrict__ counts,
                                                                   uint64_t n_rows, uint32_t T, uint64_t n_tiles,
                                                                   uint64_t* __restrict__ voff,
                                                                   unsigned long long* tile_state,
                                                                   uint32_t* counters) {
  constexpr int RPW = count_rows_per_warp(T_TPL);
  constexpr int ROWS = count_rows_per_tile(T_TPL);
  __shared__ uint64_t s_tot[ROWS];
  __shared__ uint32_t s_tile;
  __shared__ uint64_t s_prefix, s_agg;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_tile = atomicAdd(&counters[0], 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint64_t row0 = static_cast<uint64_t>(tile) * ROWS;

  if constexpr (T_TPL > 0) {
    constexpr int PER = T_TPL / 128;  // 128-bit loads per lane per row
    uint4 x[RPW][PER];
#pragma unroll
    for (int rr = 0; rr < RPW; ++rr) {
      const uint64_t row = row0 + warp * RPW + rr;
#pragma unroll
      for (int k = 0; k < PER; ++k) {
        if (row < n_rows)
          x[rr][k] = __ldcs(reinterpret_cast<const uint4*>(counts + row * T_TPL) + k * 32 + lane);
        else
          x[rr][k] = make_uint4(0, 0, 0, 0);
      }
    }
#pragma unroll
    for (int rr = 0; rr < RPW; ++rr) {
      uint64_t s = 0;
#pragma unroll
      for (int k = 0; k < PER; ++k)
        s += static_cast<uint64_t>(x[rr][k].x) + x[rr][k].y + x[rr][k].z + x[rr][k].w;
      s = warp_sum_u64(s);
      if (lane == 0) s_tot[warp * RPW + rr] = s;
    }
  } else {
    for (int rr = 0; rr < RPW; ++rr) {
      const uint64_t row = row0 + warp * RPW + rr;
      uint64_t s = 0;
      if (row < n_rows) {
        const uint32_t* p = counts + row * T;
        for (uint32_t i = lane; i < T; i += 32) s += __ldcs(p + i);
      }
      s = warp_sum_u64(s);
      if (lane == 0) s_tot[warp * RPW + rr] = s;
    }
  }
  __syncthreads();
  if (warp == 0) {
    uint64_t run = 0;
    for (int seg = 0; seg < ROWS; seg += 32) {
      const uint64_t x = seg + lane < ROWS ? s_tot[seg + lane] : 0;
      const uint64_t inc = warp_incl_scan(x);
      if (seg + lane < ROWS) s_tot[seg + lane] = run + inc - x;
      run += __shfl_sync(0xffffffffu, inc, 31);
    }
    const uint64_t excl = lookback(tile, run, tile_state, &counters[2]);
    if (lane == 0) {
      s_prefix = excl;
      s_agg = run;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < ROWS; i += blockDim.x) {
    const uint64_t row = row0 + i;
    if (row < n_rows) voff[row] = s_prefix + s_tot[i];
  }
  if (tile == n_tiles - 1 && threadIdx.x == 0) voff[n_rows] = s_prefix + s_agg;
}

// ---------------------------------------------------------------------------
// 2. reserve: one warp per LFVector.

__global__ void __launch_bounds__(256) reserve_kernel(ArrayView v, InsertScratch s, uint64_t n_rows, uint32_t R,
                                                      uint64_t n_values, uint64_t n_tiles,
                                                      uint32_t copy_chunk_elems) {
  __shared__ uint64_t s_warp[33];
  __shared__ int s_last;
  const uint64_t gt = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const uint64_t nthreads = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  // The look-back state is consumed: clear it for the next call.
  for (uint64_t i = gt; i < n_tiles; i += nthreads) s.tile_state[i] = 0;

  const bool scan_ok = __ldcg(&s.counters[2]) == 0;
  const bool ok = scan_ok && __ldcg(&s.voff[n_rows]) == n_values;
  if (!ok && gt == 0) latch_error(v.status, scan_ok ? GGA_ERR_INVALID : GGA_ERR_TIMEOUT);

  const int lane = threadIdx.x & 31;
  const uint64_t l = gt >> 5;
  if (l < v.L) {
    const uint64_t base = v.sizes[l];
    uint64_t* pre_l = s.pre + l * (static_cast<uint64_t>(R) + 1);
    uint64_t S = 0;
    for (uint32_t r0 = 0; r0 < R; r0 += 32) {
      const uint32_t r = r0 + lane;
      uint64_t t = 0;
      if (ok && r < R) {
        const uint64_t row = static_cast<uint64_t>(r) * v.L + l;
        t = __ldcg(s.voff + row + 1) - __ldcg(s.voff + row);
      }
      const uint64_t inc = warp_incl_scan(t);
      if (r < R) pre_l[r] = S + inc - t;
      S += __shfl_sync(0xffffffffu, inc, 31);
    }
    __syncwarp();
    if (lane == 0) {
      pre_l[R] = S;
      uint64_t commit = S;
      if (S > 0) {
        const uint32_t nb = v.nbuckets[l];
        const uint32_t need = buckets_for(base + S, v.log2B);
        if (need > nb) {
          const uint32_t got = grow_buckets(v, static_cast<uint32_t>(l), nb, need);
          v.nbuckets[l] = got;
          if (got < need) {
            // Keep the longest prefix of rounds that fits (pool exhausted).
            const uint64_t cap = bucket_first(got, v.log2B);
            uint32_t lo = 0, hi = R;  // largest r with base + pre_l[r] <= cap
            while (lo < hi) {
              const uint32_t mid = (lo + hi + 1) >> 1;
              if (base + pre_l[mid] <= cap) lo = mid; else hi = mid - 1;
            }
            commit = pre_l[lo];
            latch_error(v.status, GGA_ERR_POOL_EXHAUSTED);
          }
        }
      }
      s.ins_base[l] = base;
      s.ins_len[l] = commit;
      v.sizes[l] = base + commit;
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&s.counters[1], 1u) == gridDim.x - 1;
  __syncthreads();
  if (s_last) {
    __threadfence();
    finalize_block(v, s.ins_base, s.ins_len, s.cp_prefix, copy_chunk_elems, s_warp);
    if (threadIdx.x == 0) {
      s.counters[0] = 0;
      s.counters[1] = 0;
      s.counters[2] = 0;
    }
  }
}

// ---------------------------------------------------------------------------
// 3. copy: destination-ordered write of every committed run.

template <int E>
__device__ __forceinline__ typename Elem<E>::T load_elem(const uint8_t* values, uint64_t i) {
  return __ldcs(reinterpret_cast<const typename Elem<E>::T*>(values) + i);
}

template <int E>
__device__ __forceinline__ void store_elem(uint64_t addr, typename Elem<E>::T x) {
  __stcs(reinterpret_cast<typename Elem<E>::T*>(addr), x);
}

// largest i in [0, n) with a[i] <= x (a[0] <= x assumed)
__device__ __forceinline__ uint32_t last_le(const uint64_t* a, uint32_t n, uint64_t x) {
  uint32_t lo = 0, hi = n;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (a[mid] <= x) lo = mid; else hi = mid;
  }
  return lo;
}

template <int E, bool SRC_VEC>
__global__ void __launch_bounds__(256) copy_kernel(ArrayView v, const uint8_t* __restrict__ values,
                                                   const uint64_t* __restrict__ voff, const uint64_t* __restrict__ pre,
                                                   uint32_t R, const uint64_t* __restrict__ ins_base,
                                                   const uint64_t* __restrict__ ins_len,
                                                   const uint64_t* __restrict__ cp_prefix) {
  typedef typename Elem<E>::T T;
  constexpr uint32_t VEC = 16 / E;
  constexpr uint32_t C = kCopyChunkBytes / E;
  __shared__ uint64_t s_pre[kCopyWindow + 1];
  __shared__ uint64_t s_src[kCopyWindow];
  __shared__ uint32_t s_rlo, s_rhi;

  const uint64_t total = cp_prefix[v.L];
  const uint64_t ipb = (total + gridDim.x - 1) / gridDim.x;
  const uint64_t w0 = static_cast<uint64_t>(blockIdx.x) * ipb;
  const uint64_t w1 = min(total, w0 + ipb);
  if (w0 >= w1) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool group_ok = v.B >= VEC;
  uint32_t l = upper_bound_u64(cp_prefix, v.L + 1, w0) - 1;

  for (uint64_t w = w0; w < w1; ++w) {
    while (cp_prefix[l + 1] <= w) ++l;
    const uint64_t base = ins_base[l], len = ins_len[l];
    const uint64_t chunk = base / C + (w - cp_prefix[l]);
    const uint64_t p0 = max(base, chunk * C), p1 = min(base + len, (chunk + 1) * C);
    const uint64_t q0 = p0 - base, q1 = p1 - base;
    const uint64_t* pre_l = pre + static_cast<uint64_t>(l) * (R + 1);
    const uint64_t* bk = v.buckets + static_cast<uint64_t>(l) * kMaxBuckets;

    // Rounds whose runs hold q0 and q1-1: 32-ary search by warp 0.
    if (warp == 0) {
      uint32_t lo_a = 0, hi_a = R + 1, lo_b = 0, hi_b = R + 1;
      while (hi_a - lo_a > 1 || hi_b - lo_b > 1) {
        const uint32_t sa = (hi_a - lo_a + 31) / 32, sb = (hi_b - lo_b + 31) / 32;
        const uint32_t ia = lo_a + lane * sa, ib = lo_b + lane * sb;
        const bool pa = ia < hi_a && pre_l[ia] <= q0;
        const bool pb = ib < hi_b && pre_l[ib] <= q1 - 1;
        const int ka = 31 - __clz(__ballot_sync(0xffffffffu, pa));
        const int kb = 31 - __clz(__ballot_sync(0xffffffffu, pb));
        const uint32_t nlo_a = lo_a + ka * sa, nlo_b = lo_b + kb * sb;
        hi_a = min(hi_a, nlo_a + sa);
        hi_b = min(hi_b, nlo_b + sb);
        lo_a = nlo_a;
        lo_b = nlo_b;
      }
      if (lane == 0) {
        s_rlo = lo_a;
        s_rhi = lo_b;
      }
    }
    __syncthreads();
    const uint32_t rlo = s_rlo, nw = s_rhi - s_rlo + 1;
    const bool windowed = nw <= kCopyWindow;
    if (windowed) {
      for (uint32_t i = threadIdx.x; i <= nw; i += blockDim.x) {
        s_pre[i] = pre_l[rlo + i];
        if (i < nw) s_src[i] = voff[static_cast<uint64_t>(rlo + i) * v.L + l];
      }
    }
    __syncthreads();

    const uint64_t gbeg = p0 & ~static_cast<uint64_t>(VEC - 1);
    for (uint64_t p = gbeg + static_cast<uint64_t>(threadIdx.x) * VEC; p < p1;
         p += static_cast<uint64_t>(blockDim.x) * VEC) {
      const bool full = group_ok && p >= p0 && p + VEC <= p1;
      if (full && windowed) {
        const uint64_t q = p - base;
        const uint32_t r = last_le(s_pre, nw, q);
        uint32_t bb;
        uint64_t off;
        bucket_of(p, v.log2B, bb, off);
        const uint64_t dst = bk[bb] + off * E;
        if (q + VEC <= s_pre[r + 1]) {
          const uint64_t src = s_src[r] + (q - s_pre[r]);
          if (SRC_VEC && (src % VEC) == 0) {
            __stcs(reinterpret_cast<uint4*>(dst), __ldcs(reinterpret_cast<const uint4*>(values) + src / VEC));
          } else {
            Vec16<E> x;
#pragma unroll
            for (uint32_t e = 0; e < VEC; ++e) x.e[e] = load_elem<E>(values, src + e);
            __stcs(reinterpret_cast<uint4*>(dst), x.v);
          }
        } else {
          Vec16<E> x;
#pragma unroll
          for (uint32_t e = 0; e < VEC; ++e) {
            const uint32_t re = last_le(s_pre, nw, q + e);
            x.e[e] = load_elem<E>(values, s_src[re] + (q + e - s_pre[re]));
          }
          __stcs(reinterpret_cast<uint4*>(dst), x.v);
        }
      } else {
        for (uint32_t e = 0; e < VEC; ++e) {
          const uint64_t pe = p + e;
          if (pe < p0 || pe >= p1) continue;
          const uint64_t q = pe - base;
          uint64_t src;
          if (windowed) {
            const uint32_t re = last_le(s_pre, nw, q);
            src = s_src[re] + (q - s_pre[re]);
          } else {
            const uint32_t re = last_le(pre_l, R + 1, q);
            src = voff[static_cast<uint64_t>(re) * v.L + l] + (q - pre_l[re]);
          }
          uint32_t bb;
          uint64_t off;
          bucket_of(pe, v.log2B, bb, off);
          store_elem<E>(bk[bb] + off * E, load_elem<E>(values, src));
        }
      }
    }
    __syncthreads();
  }
}

template <int T_TPL>
static void launch_count(const uint32_t* counts, uint64_t n_rows, uint32_t T, uint64_t* voff,
                         unsigned long long* ts, uint32_t* counters, cudaStream_t st) {
  const uint64_t n_tiles = (n_rows + count_rows_per_tile(T_TPL) - 1) / count_rows_per_tile(T_TPL);
  count_scan_kernel<T_TPL><<<static_cast<unsigned>(n_tiles), kCountThreads, 0, st>>>(counts, n_rows, T, n_tiles,
                                                                                      voff, ts, counters);
}

uint64_t count_tiles(uint64_t n_rows, uint32_t T, bool vec_ok) {
  int tpl = 0;
  if (vec_ok && (T == 128 || T == 256 || T == 512 || T == 1024)) tpl = static_cast<int>(T);
  const uint64_t rows = static_cast<uint64_t>(count_rows_per_tile(tpl));
  return (n_rows + rows - 1) / rows;
}

int launch_insert(const ArrayView& v, const InsertScratch& s, const uint32_t* counts, uint32_t R,
                  const void* values, uint64_t n_values, int num_sms, cudaStream_t st) {
  const uint64_t n_rows = static_cast<uint64_t>(R) * v.L;
  const bool vec_ok = (reinterpret_cast<uintptr_t>(counts) & 15) == 0;
  const uint64_t n_tiles = count_tiles(n_rows, v.T, vec_ok);
  if (vec_ok && v.T == 128) launch_count<128>(counts, n_rows, v.T, s.voff, s.tile_state, s.counters, st);
  else if (vec_ok && v.T == 256) launch_count<256>(counts, n_rows, v.T, s.voff, s.tile_state, s.counters, st);
  else if (vec_ok && v.T == 512) launch_count<512>(counts, n_rows, v.T, s.voff, s.tile_state, s.counters, st);
  else if (vec_ok && v.T == 1024) launch_count<1024>(counts, n_rows, v.T, s.voff, s.tile_state, s.counters, st);
  else launch_count<0>(counts, n_rows, v.T, s.voff, s.tile_state, s.counters, st);

  const uint32_t cce = kCopyChunkBytes / v.E;
  const unsigned rblocks = static_cast<unsigned>((static_cast<uint64_t>(v.L) * 32 + 255) / 256);
  reserve_kernel<<<rblocks, 256, 0, st>>>(v, s, n_rows, R, n_values, n_tiles, cce);

  const unsigned cgrid = static_cast<unsigned>(num_sms) * 4;
  const bool src_vec = (reinterpret_cast<uintptr_t>(values) & 15) == 0;
  const uint8_t* vals = static_cast<const uint8_t*>(values);
#define GGA_COPY(EE)                                                                                          \
  do {                                                                                                        \
    if (src_vec)                                                                                              \
      copy_kernel<EE, true><<<cgrid, 256, 0, st>>>(v, vals, s.voff, s.pre, R, s.ins_base, s.ins_len, s.cp_prefix); \
    else                                                                                                      \
      copy_kernel<EE, false><<<cgrid, 256, 0, st>>>(v, vals, s.voff, s.pre, R, s.ins_base, s.ins_len, s.cp_prefix); \
  } while (0)
  if (v.E == 4) GGA_COPY(4);
  else if (v.E == 8) GGA_COPY(8);
  else GGA_COPY(16);
#undef GGA_COPY
  return cudaGetLastError() == cudaSuccess ? GGA_OK : GGA_ERR_CUDA;
}

int launch_finalize(const ArrayView& v, cudaStream_t st) {
  finalize_kernel<<<1, 1024, 0, st>>>(v);
  return cudaGetLastError() == cudaSuccess ? GGA_OK : GGA_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// In-kernel generated insertion.

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
      for (uint32_t k = 0; k < g.nthr; ++k) c += u >= g.thr[k];
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

constexpr uint32_t kGenStageBytes = 65536;

template <int E> struct GenK { static constexpr int value = E == 16 ? 4 : 8; };

// One block per LFVector.  Per pass of K rounds: every thread draws its K
// counts, a warp-shuffle scan plus one shared-memory pass over the warp
// totals gives its positions, thread 0 reserves the pass's run and allocates
// the buckets it reaches, then (synchronize) every thread writes its values
// at its prefix-sum positions into a shared-memory stage and the block
// streams the stage to the buckets with aligned 128-bit stores.  A pass that
// does not fit the stage writes straight to the buckets instead.
template <int E, int K>
__global__ void __launch_bounds__(1024) gen_insert_kernel(ArrayView v, GenParams g, uint32_t R) {
  typedef typename Elem<E>::T T;
  constexpr uint32_t VEC = 16 / E;
  constexpr uint32_t CAP = kGenStageBytes / E;
  extern __shared__ uint4 s_stage4[];
  T* s_stage = reinterpret_cast<T*>(s_stage4);
  __shared__ uint64_t s_wtot[K][32];
  __shared__ uint64_t s_rbase[K + 1];
  __shared__ uint64_t s_base, s_commit;
  __shared__ int s_stop;

  const uint32_t l = blockIdx.x, t = threadIdx.x, NT = blockDim.x;
  const int lane = t & 31, warp = t >> 5, nwarps = NT >> 5;
  const uint64_t gtid = static_cast<uint64_t>(l) * v.T + t;
  const uint64_t* bk = v.buckets + static_cast<uint64_t>(l) * kMaxBuckets;
  const bool group_ok = v.B >= VEC;
  if (t == 0) {
    s_base = v.sizes[l];
    s_stop = 0;
  }
  __syncthreads();

  for (uint32_t r0 = 0; r0 < R; r0 += K) {
    const uint32_t kk = min(static_cast<uint32_t>(K), R - r0);
    uint64_t inc[K];
    uint32_t cnt[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const uint64_t r = static_cast<uint64_t>(g.round0) + r0 + k;
      cnt[k] = (t < v.T && static_cast<uint32_t>(k) < kk) ? gen_count(g, splitmix(g.seed, (r << 32) | gtid)) : 0u;
      inc[k] = warp_incl_scan(static_cast<uint64_t>(cnt[k]));
      if (lane == 31) s_wtot[k][warp] = inc[k];
    }
    __syncthreads();
    if (warp == 0) {
      uint64_t rb = 0;
      for (int k = 0; k < K; ++k) {
        const uint64_t w = lane < nwarps ? s_wtot[k][lane] : 0;
        const uint64_t wi = warp_incl_scan(w);
        if (lane < nwarps) s_wtot[k][lane] = rb + wi - w;   // pass-relative start of the warp's run
        if (lane == 0) s_rbase[k] = rb;
        rb += __shfl_sync(0xffffffffu, wi, 31);
      }
      if (lane == 0) {
        s_rbase[K] = rb;
        // Leader: one size reservation for the pass, then Algorithm 2 for
        // every bucket the run reaches.
        const uint64_t base = s_base;
        uint64_t commit = rb;
        if (rb > 0) {
          const uint32_t nb = v.nbuckets[l];
          const uint32_t need = buckets_for(base + rb, v.log2B);
          if (need > nb) {
            const uint32_t got = grow_buckets(v, l, nb, need);
            v.nbuckets[l] = got;
            if (got < need) {
              const uint64_t cap = bucket_first(got, v.log2B);
              int kf = 0;
              while (kf < K && base + s_rbase[kf + 1] <= cap) ++kf;
              commit = s_rbase[kf];
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

    const uint64_t base = s_base, commit = s_commit;
    const bool staged = commit <= CAP;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const uint64_t start = s_wtot[k][warp] + inc[k] - cnt[k];   // this thread's position in the pass
      const uint64_t r = static_cast<uint64_t>(g.round0) + r0 + k;
      for (uint32_t j = 0; j < cnt[k]; ++j) {
        const uint64_t q = start + j;
        if (q >= commit) break;
        const T x = gen_value<E>(g.va * gtid + g.vb * r + g.vc * j);
        if (staged) {
          s_stage[q] = x;
        } else {
          uint32_t bb;
          uint64_t off;
          bucket_of(base + q, v.log2B, bb, off);
          store_elem<E>(bk[bb] + off * E, x);
        }
      }
    }
    __syncthreads();
    if (staged) {
      const uint64_t gbeg = base & ~static_cast<uint64_t>(VEC - 1);
      const uint64_t end = base + commit;
      for (uint64_t p = gbeg + static_cast<uint64_t>(t) * VEC; p < end; p += static_cast<uint64_t>(NT) * VEC) {
        if (group_ok && p >= base && p + VEC <= end) {
          Vec16<E> x;
#pragma unroll
          for (uint32_t e = 0; e < VEC; ++e) x.e[e] = s_stage[p - base + e];
          uint32_t bb;
          uint64_t off;
          bucket_of(p, v.log2B, bb, off);
          __stcs(reinterpret_cast<uint4*>(bk[bb] + off * E), x.v);
        } else {
#pragma unroll
          for (uint32_t e = 0; e < VEC; ++e) {
            const uint64_t pe = p + e;
            if (pe < base || pe >= end) continue;
            uint32_t bb;
            uint64_t off;
            bucket_of(pe, v.log2B, bb, off);
            store_elem<E>(bk[bb] + off * E, s_stage[pe - base]);
          }
        }
      }
    }
    __syncthreads();
    if (t == 0) s_base = base + commit;
    const int stop = s_stop;
    __syncthreads();
    if (stop) break;
  }
}

int launch_insert_generated(const ArrayView& v, const gga_gen_spec& spec, uint32_t R, uint32_t* /*done*/,
                            int /*num_sms*/, cudaStream_t st) {
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
  const uint32_t NT = (v.T + 31) / 32 * 32;
  const size_t smem = kGenStageBytes;
#define GGA_GEN(EE)                                                                                          \
  do {                                                                                                       \
    cudaFuncSetAttribute(gen_insert_kernel<EE, GenK<EE>::value>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                         static_cast<int>(smem));                                                            \
    gen_insert_kernel<EE, GenK<EE>::value><<<v.L, NT, smem, st>>>(v, g, R);                                  \
  } while (0)
  if (v.E == 4) GGA_GEN(4);
  else if (v.E == 8) GGA_GEN(8);
  else GGA_GEN(16);
#undef GGA_GEN
  finalize_kernel<<<1, 1024, 0, st>>>(v);
  return cudaGetLastError() == cudaSuccess ? GGA_OK : GGA_ERR_CUDA;
}

}  // namespace gga
