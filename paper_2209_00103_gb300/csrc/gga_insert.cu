// gga_insert.cu -- batched block-level insertion (Algorithm 1 over R rounds).
//
// Host-buffer form (gga_insert): counts[r][l][t] and values packed in
// (round, block, thread, k) order.  Four kernels:
//   1. count: one streaming pass over the counts.  Row (r, l) of T counts is
//      reduced to the run length of block l in round r; each block takes a
//      tile of consecutive rows, writes every row's exclusive prefix inside
//      the tile and the tile's total.
//   2. tile_scan: one block turns the tile totals into tile prefixes, so the
//      first-value index of run (r, l) is voff(r*L + l) = tile prefix + row
//      prefix, with no inter-block waiting anywhere.
//   3. reserve: one warp per LFVector.  A shuffle scan over the rounds gives
//      each round's position in the batch (the per-round size reservation of
//      Algorithm 1, done for all rounds at once), then the warp's leader
//      allocates every bucket the batch reaches from the device pool
//      (Algorithm 2) and commits the new size.  The last block to finish
//      recomputes the prefix sum of LFVector sizes (Sec. IV) and the work
//      lists of the copy, flatten and rw_b kernels.
//   4. copy: the elements are written at their prefix-sum positions.  Because
//      the values arrive packed in prefix-sum order, element q of LFVector l's
//      batch is value voff(r*L + l) + (q - pre[l][r]) for the round r whose run
//      holds q; the kernel walks destinations in 16-byte groups so every store
//      is a full aligned 128-bit store inside a bucket.
//
// In-kernel form (gga_insert_generated): each block is one LFVector; its
// threads draw their counts, run a warp-shuffle block scan (Sec. III-B), the
// leader thread reserves and allocates (Algorithms 1-2), __syncthreads is the
// synchronize() of Algorithm 1, and the block writes the run.  K rounds share
// one scan pass to amortise the barriers.
#include "gga_core.cuh"
#include "gga_gen.cuh"

namespace gga {

constexpr uint32_t kCopyChunkBytes = 4096;                   // one warp's unit of destination
constexpr int kCopyThreads = 256;
constexpr int kCopyU = kCopyChunkBytes / 16 / 32;             // 16-byte groups per lane per chunk
constexpr int kCountThreads = 256;

// ---------------------------------------------------------------------------
// Finalize: prefix sum of sizes, flatten/rw_b chunk prefix, copy chunk prefix.
// Run by one block (any multiple of 32 threads, <= 1024).

__global__ void __launch_bounds__(1024) finalize_kernel(ArrayView v) {
  __shared__ uint64_t s_warp[33];
  if (threadIdx.x == 0) ring_fixup(v.pool);
  finalize_block(v, nullptr, nullptr, nullptr, 1, s_warp);
}

// ---------------------------------------------------------------------------
// 1. count and 2. tile_scan.

__host__ __device__ constexpr int count_rows_per_warp(int T_TPL) {
  return T_TPL == 0 ? 4 : (T_TPL >= 1024 ? 2 : 2048 / T_TPL);
}

__host__ __device__ constexpr int count_rows_per_tile(int T_TPL) {
  return (kCountThreads / 32) * count_rows_per_warp(T_TPL);
}

// First-value index of run `row` (row == n_rows gives the grand total).
__device__ __forceinline__ uint64_t voff_at(const InsertScratch& s, uint64_t row, uint32_t rows_per_tile,
                                            uint64_t n_rows, uint64_t n_tiles) {
  if (row >= n_rows) return s.tile_pre[n_tiles];
  return s.tile_pre[row / rows_per_tile] + s.row_pre[row];
}

// T_TPL > 0: T == T_TPL (a multiple of 128) and counts 16-byte aligned, the
// row is read with 128-bit loads.  T_TPL == 0: any T, 32-bit loads.
template <int T_TPL>
__global__ void __launch_bounds__(kCountThreads) count_kernel(const uint32_t* __restrict__ counts, uint64_t n_rows,
                                                              uint32_t T, uint32_t L, uint32_t R,
                                                              uint64_t* __restrict__ row_pre,
                                                              uint64_t* __restrict__ tile_agg,
                                                              uint64_t* __restrict__ pre) {
  constexpr int RPW = count_rows_per_warp(T_TPL);
  constexpr int ROWS = count_rows_per_tile(T_TPL);
  __shared__ uint64_t s_tot[ROWS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t tile = blockIdx.x;
  const uint64_t row0 = tile * ROWS;

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
      const uint64_t row = row0 + seg + lane;
      if (seg + lane < ROWS && row < n_rows) {
        row_pre[row] = run + inc - x;
        // The row's total also goes to its LFVector's line of `pre`
        // ([L][R+1], round-contiguous), where reserve reads and scans it.
        const uint64_t r = row / L;
        pre[(row - r * L) * (static_cast<uint64_t>(R) + 1) + r] = x;
      }
      run += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane == 0) tile_agg[tile] = run;
  }
}

// Exclusive scan of the tile totals in place; entry n_tiles gets the total.
// One block; warp w takes kTileScanItems x 32 consecutive tiles with
// coalesced loads (lane i reads tiles 32k + i), scans them with shuffles,
// one block scan combines the warp totals, then the warp writes its tiles
// back the same way.  (A run of consecutive tiles per thread made every
// load and store instruction touch 32 lines: 19 us for 16,384 tiles.)
constexpr int kTileScanItems = 16;

__global__ void __launch_bounds__(1024) tile_scan_kernel(uint64_t* tile, uint64_t n_tiles) {
  __shared__ uint64_t s_warp[33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t per_warp = 32ull * kTileScanItems;
  const uint64_t per_pass = per_warp * (blockDim.x >> 5);
  uint64_t run = 0;
  for (uint64_t t0 = 0; t0 < n_tiles; t0 += per_pass) {
    const uint64_t w0 = t0 + static_cast<uint64_t>(warp) * per_warp;
    uint64_t x[kTileScanItems];
#pragma unroll
    for (int k = 0; k < kTileScanItems; ++k) {
      const uint64_t i = w0 + 32 * k + lane;
      x[k] = i < n_tiles ? tile[i] : 0;
    }
    uint64_t carry = 0;   // sum of the warp's tiles before chunk k
#pragma unroll
    for (int k = 0; k < kTileScanItems; ++k) {
      const uint64_t inc = warp_incl_scan(x[k]);
      const uint64_t ex = carry + inc - x[k];
      carry += __shfl_sync(0xffffffffu, inc, 31);
      x[k] = ex;
    }
    uint64_t tot;
    const uint64_t e = block_excl_scan_u64(lane == 0 ? carry : 0, s_warp, tot);
    const uint64_t wbase = run + __shfl_sync(0xffffffffu, e, 0);
#pragma unroll
    for (int k = 0; k < kTileScanItems; ++k) {
      const uint64_t i = w0 + 32 * k + lane;
      if (i < n_tiles) tile[i] = wbase + x[k];
    }
    run += tot;
  }
  if (threadIdx.x == 0) tile[n_tiles] = run;
}

// ---------------------------------------------------------------------------
// 2. reserve: one warp per LFVector.

__global__ void __launch_bounds__(256) reserve_kernel(ArrayView v, InsertScratch s, uint32_t R, uint64_t n_values,
                                                      uint64_t n_tiles, uint32_t copy_chunk_elems) {
  __shared__ uint64_t s_warp[33];
  __shared__ int s_last;
  const uint64_t gt = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const bool ok = s.tile_pre[n_tiles] == n_values;
  if (!ok && gt == 0) latch_error(v.status, GGA_ERR_INVALID);

  const int lane = threadIdx.x & 31;
  const uint64_t l = gt >> 5;
  if (l < v.L) {
    const uint64_t base = v.sizes[l];
    uint64_t* pre_l = s.pre + l * (static_cast<uint64_t>(R) + 1);
    uint64_t S = 0;
    // Rounds in sweeps of 32 x kResK: every run length of a sweep (count
    // left it in pre_l[r], round-contiguous) is loaded before the first
    // scan, so the loads are in flight together; the scan overwrites it.
    constexpr int kResK = 16;
    for (uint32_t r0 = 0; r0 < R; r0 += 32 * kResK) {
      uint64_t t[kResK];
#pragma unroll
      for (int k = 0; k < kResK; ++k) {
        const uint32_t r = r0 + k * 32 + lane;
        t[k] = (ok && r < R) ? pre_l[r] : 0;
      }
#pragma unroll
      for (int k = 0; k < kResK; ++k) {
        const uint32_t r = r0 + k * 32 + lane;
        const uint64_t inc = warp_incl_scan(t[k]);
        if (r < R) pre_l[r] = S + inc - t[k];
        S += __shfl_sync(0xffffffffu, inc, 31);
      }
    }
    __syncwarp();
    if (lane == 0) pre_l[R] = S;
    // The whole warp allocates (S and base are the same in every lane).
    uint32_t nb = 0, need = 0, got = 0;
    if (S > 0) {
      nb = v.nbuckets[l];
      need = buckets_for(base + S, v.log2B);
      if (need > nb) got = grow_buckets_warp(v, static_cast<uint32_t>(l), nb, need);
    }
    __syncwarp();
    if (lane == 0) {
      uint64_t commit = S;
      if (S > 0 && need > nb) {
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
    if (threadIdx.x == 0) ring_fixup(v.pool);
    finalize_block(v, s.ins_base, s.ins_len, s.cp_prefix, copy_chunk_elems, s_warp);
    if (threadIdx.x == 0) s.counters[1] = 0;
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

// Elements src .. src+VEC-1 of the packed values as one 16-byte group.  With
// a 16-byte aligned buffer a misaligned group is read as the two aligned
// 16-byte words that cover it (the second holds element src+VEC-1, so it
// lies in the buffer's allocation) and the words are selected.
template <int E, bool SRC_VEC>
__device__ __forceinline__ uint4 load_group(const uint8_t* __restrict__ values, uint64_t src) {
  if constexpr (E == 16) {
    return __ldcs(reinterpret_cast<const uint4*>(values) + src);
  } else if constexpr (!SRC_VEC) {
    Vec16<E> x;
#pragma unroll
    for (uint32_t e = 0; e < 16 / E; ++e) x.e[e] = load_elem<E>(values, src + e);
    return x.v;
  } else {
    constexpr uint32_t VEC = 16 / E;
    const uint32_t d = static_cast<uint32_t>(src % VEC);
    const uint4* q = reinterpret_cast<const uint4*>(values) + src / VEC;
    const uint4 a = __ldcs(q);
    if (d == 0) return a;
    const uint4 b = __ldcs(q + 1);
    if constexpr (E == 8) return make_uint4(a.z, a.w, b.x, b.y);
    if (d == 1) return make_uint4(a.y, a.z, a.w, b.x);
    if (d == 2) return make_uint4(a.z, a.w, b.x, b.y);
    return make_uint4(a.w, b.x, b.y, b.z);
  }
}

// Last index i in [0, n) with a[i] <= x, searched by a whole warp 32-ary
// (a[0] <= x assumed).  Every lane returns the same index.
__device__ __forceinline__ uint32_t warp_last_le(const uint64_t* a, uint32_t n, uint64_t x) {
  const int lane = threadIdx.x & 31;
  uint32_t lo = 0, hi = n;
  while (hi - lo > 1) {
    const uint32_t st = (hi - lo + 31) / 32;
    const uint32_t i = lo + lane * st;
    const bool pr = i < hi && a[i] <= x;
    const int k = 31 - __clz(__ballot_sync(0xffffffffu, pr));
    const uint32_t nlo = lo + k * st;
    hi = min(hi, nlo + st);
    lo = nlo;
  }
  return lo;
}

// Each warp streams a contiguous range of 4 KB destination chunks.  A chunk
// lies in one LFVector's batch.  The warp keeps the run starts and
// first-value indices of 32 consecutive rounds of that LFVector in its own
// shared-memory window and reloads it only when a chunk runs past it (runs
// are usually longer than a chunk, so one window serves many chunks).  Lanes
// own 16-byte destination groups (coalesced 128-bit stores) and issue all
// their loads before their stores.  No block-wide barrier.
template <int E, bool SRC_VEC>
__global__ void __launch_bounds__(kCopyThreads) copy_kernel(ArrayView v, const uint8_t* __restrict__ values,
                                                            InsertScratch sc, uint32_t R, uint64_t n_rows,
                                                            uint64_t n_tiles, uint32_t rows_per_tile) {
  constexpr uint32_t VEC = 16 / E;
  constexpr uint32_t C = kCopyChunkBytes / E;
  constexpr int NW = kCopyThreads / 32;
  constexpr uint32_t NONE = 0xFFFFFFFFu;
  __shared__ uint64_t s_wp[NW][33];   // run starts of rounds wr .. wr+31 (batch-relative); [32] = sentinel
  __shared__ uint64_t s_wv[NW][32];   // first-value index of those runs
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint64_t* wp = s_wp[wib];
  uint64_t* wv = s_wv[wib];
  const uint64_t* __restrict__ cp_prefix = sc.cp_prefix;
  const uint64_t total = cp_prefix[v.L];
  const uint64_t gw = static_cast<uint64_t>(blockIdx.x) * NW + wib;
  const uint64_t nwarps = static_cast<uint64_t>(gridDim.x) * NW;
  const uint64_t w0 = total * gw / nwarps, w1 = total * (gw + 1) / nwarps;
  if (w0 >= w1) return;
  const bool group_ok = v.B >= VEC;

  uint32_t l = upper_bound_u64(cp_prefix, v.L + 1, w0) - 1;
  uint64_t base = sc.ins_base[l], len = sc.ins_len[l], lfv_first = cp_prefix[l], lfv_end = cp_prefix[l + 1];
  const uint64_t* pre_l = sc.pre + static_cast<uint64_t>(l) * (R + 1);
  const uint64_t* bk = v.buckets + static_cast<uint64_t>(l) * kMaxBuckets;
  uint32_t wr = NONE;          // round in window slot 0
  uint64_t covered = 0;        // positions below this lie in rounds wr .. wr+30

  for (uint64_t w = w0; w < w1; ++w) {
    if (w >= lfv_end) {
      while (cp_prefix[l + 1] <= w) ++l;
      base = sc.ins_base[l];
      len = sc.ins_len[l];
      lfv_first = cp_prefix[l];
      lfv_end = cp_prefix[l + 1];
      pre_l = sc.pre + static_cast<uint64_t>(l) * (R + 1);
      bk = v.buckets + static_cast<uint64_t>(l) * kMaxBuckets;
      wr = NONE;
    }
    const uint64_t chunk = base / C + (w - lfv_first);
    const uint64_t p0 = max(base, chunk * C), p1 = min(base + len, (chunk + 1) * C);
    const uint64_t q0 = p0 - base, q1 = p1 - base;
    if (wr == NONE || q1 > covered) {
      // (Re)load the window from the round holding q0.
      const uint32_t r0 = (wr != NONE && q0 < covered) ? wr + last_le(wp, 32, q0) : warp_last_le(pre_l, R + 1, q0);
      __syncwarp();
      const uint32_t r = r0 + lane;
      wp[lane] = r <= R ? pre_l[r] : ~0ull;
      wv[lane] = r < R ? voff_at(sc, static_cast<uint64_t>(r) * v.L + l, rows_per_tile, n_rows, n_tiles) : 0;
      if (lane == 0) wp[32] = ~0ull;
      __syncwarp();
      wr = r0;
      covered = wp[31];
    }

    const uint64_t gbeg = p0 & ~static_cast<uint64_t>(VEC - 1);
    // Bucket of the chunk's ends: most chunks lie in one bucket.
    uint32_t b0, b1;
    uint64_t o0, o1;
    bucket_of(p0, v.log2B, b0, o0);
    bucket_of(p1 - 1, v.log2B, b1, o1);
    const bool one_bucket = b0 == b1;
    const uint64_t dbase = bk[b0] + (gbeg - bucket_first(b0, v.log2B)) * E;   // address of gbeg if in bucket b0
    Vec16<E> x[kCopyU];
    uint32_t fast = 0, slow = 0;
    // Window index of this lane's current position; positions only grow.
    uint32_t i = last_le(wp, 32, max(gbeg + static_cast<uint64_t>(lane) * VEC, p0) - base);
#pragma unroll
    for (int u = 0; u < kCopyU; ++u) {
      const uint32_t du = (lane + 32 * u) * VEC;   // element offset from gbeg
      const uint64_t p = gbeg + du;
      const uint64_t q = p - base;
      if (p < p1) {
        if (group_ok && one_bucket && p >= p0 && p + VEC <= p1 && q + VEC <= covered) {
          while (wp[i + 1] <= q) ++i;
          fast |= 1u << u;
          if (q + VEC <= wp[i + 1]) {
            x[u].v = load_group<E, SRC_VEC>(values, wv[i] + (q - wp[i]));
          } else {
            uint32_t ie = i;
#pragma unroll
            for (uint32_t e = 0; e < VEC; ++e) {
              while (wp[ie + 1] <= q + e) ++ie;
              x[u].e[e] = load_elem<E>(values, wv[ie] + (q + e - wp[ie]));
            }
          }
        } else {
          slow |= 1u << u;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kCopyU; ++u)
      if ((fast >> u) & 1u)
        __stcs(reinterpret_cast<uint4*>(dbase + static_cast<uint64_t>(lane + 32 * u) * 16), x[u].v);
    // Partial groups at the ends of the batch, chunks across a bucket
    // boundary, tiny first buckets, positions past the window: element by
    // element.
    while (slow) {
      const int u = __ffs(slow) - 1;
      slow &= slow - 1;
      const uint64_t p = gbeg + static_cast<uint64_t>(lane + 32 * u) * VEC;
      for (uint32_t e = 0; e < VEC; ++e) {
        const uint64_t pe = p + e;
        if (pe < p0 || pe >= p1) continue;
        const uint64_t q = pe - base;
        uint64_t src;
        if (q < covered) {
          const uint32_t ie = last_le(wp, 32, q);
          src = wv[ie] + (q - wp[ie]);
        } else {
          const uint32_t re = last_le(pre_l, R + 1, q);
          src = voff_at(sc, static_cast<uint64_t>(re) * v.L + l, rows_per_tile, n_rows, n_tiles) + (q - pre_l[re]);
        }
        uint32_t bb;
        uint64_t off;
        bucket_of(pe, v.log2B, bb, off);
        store_elem<E>(bk[bb] + off * E, load_elem<E>(values, src));
      }
    }
  }
}

// ---------------------------------------------------------------------------
// 4. bulk copy (values 16-byte aligned): source-ordered streaming with TMA.
//
// The packed values are one contiguous stream in run order (round-major,
// then block), and the runs of 32 consecutive (round, block) rows form one
// contiguous span of it.  Each block takes an equal, 16-byte aligned range
// of the stream's bytes (so a few huge runs spread over every block as well
// as many small ones do); a warp-wide 32-way search over the units' first
// values finds the unit its range starts in.  Its producer warp resolves a
// unit lane-parallel (lane j = row j: the run's first-value index, its
// LFVector, its position there and the bucket address) and then cuts the
// part of the unit's span inside the block's range into 16 KB windows: for
// each, lane 0 fetches the window into a stage of a 3-deep shared-memory
// ring with one TMA bulk copy (cp.async.bulk, mbarrier completion) and the
// lanes write one descriptor per run piece in the window.  Four consumer
// warps write each piece from shared memory to its bucket: element stores up
// to the 16-byte boundary, then aligned 128-bit stores, then the tail.

constexpr uint32_t kBkWin = 16384;        // bytes per stage
constexpr int kBkStages = 3;
constexpr int kBkConsumers = 4;           // consumer warps per block (2: 0.645 ms, 4: 0.602 ms, 6: 0.600 ms
                                          // for the paper-shaped insertion on GB300)
constexpr int kBkThreads = 32 * (1 + kBkConsumers);
constexpr int kBkRows = 32;               // rows per unit

struct BkPiece {
  uint64_t pos;       // LFVector position of the piece's first element
  uint64_t addr;      // its address, or 0 if the consumer must look the bucket up
  uint32_t src_off;   // byte offset of the piece inside the stage
  uint32_t n;         // elements
  uint32_t l;         // LFVector
  uint32_t b;         // bucket of pos
};

template <int E>
__device__ __forceinline__ void warp_store_run(const uint8_t* src, uint64_t dst, uint32_t count, int lane) {
  typedef typename Elem<E>::T T;
  constexpr uint32_t VEC = 16 / E;
  const T* se = reinterpret_cast<const T*>(src);
  T* de = reinterpret_cast<T*>(dst);
  const uint32_t head = min(count, static_cast<uint32_t>((16u - (dst & 15u)) & 15u) / E);
  if (static_cast<uint32_t>(lane) < head) de[lane] = se[lane];
  const uint32_t nv = (count - head) / VEC;
  for (uint32_t vi = lane; vi < nv; vi += 32) {
    Vec16<E> x;
#pragma unroll
    for (uint32_t e = 0; e < VEC; ++e) x.e[e] = se[head + vi * VEC + e];
    __stcs(reinterpret_cast<uint4*>(de + head) + vi, x.v);
  }
  const uint32_t done = head + nv * VEC;
  if (static_cast<uint32_t>(lane) < count - done) de[done + lane] = se[done + lane];
}

template <int E>
__global__ void __launch_bounds__(kBkThreads) copy_bulk_kernel(ArrayView v, const uint8_t* __restrict__ values,
                                                               uint64_t n_values, InsertScratch sc, uint32_t R,
                                                               uint64_t n_rows, uint64_t n_tiles,
                                                               uint32_t rows_per_tile) {
  extern __shared__ __align__(128) uint8_t s_buf[];   // kBkStages * kBkWin
  __shared__ __align__(8) uint64_t s_full[kBkStages];
  __shared__ __align__(8) uint64_t s_empty[kBkStages];
  __shared__ BkPiece s_piece[kBkStages][kBkRows];
  __shared__ uint32_t s_np[kBkStages];
  __shared__ uint32_t s_last[kBkStages];

  // Counts that do not sum to n_values were already reported by reserve;
  // the spans would not describe the buffer, so nothing is read.
  if (sc.tile_pre[n_tiles] != n_values) return;
  const uint64_t n_units = (n_rows + kBkRows - 1) / kBkRows;
  // The block's bytes of the value stream.  Windows are 16-byte aligned and
  // may reach up to 15 bytes past the last value: the stream starts 16-byte
  // aligned and its end is not, in that case, so those bytes still lie in
  // the same allocation (allocations end on a 256-byte boundary).
  const uint64_t total = (n_values * E + 15) & ~static_cast<uint64_t>(15);
  const uint64_t share = ((total + gridDim.x - 1) / gridDim.x + 15) & ~static_cast<uint64_t>(15);
  const uint64_t blo = static_cast<uint64_t>(blockIdx.x) * share;
  const uint64_t bhi = min(total, blo + share);
  if (n_units == 0 || blo >= bhi) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kBkStages; ++s) {
      mbar_init(&s_full[s], 1);
      mbar_init(&s_empty[s], kBkConsumers);
    }
    fence_mbar_init();
  }
  __syncthreads();

  if (warp == 0) {
    // ------------------------------- producer -------------------------------
    uint32_t i = 0;          // stages published so far
    bool ok = true;
    // The last unit whose first value starts at or before blo (32-way search;
    // unit 0 starts at 0).
    uint64_t ulo = 0, uhi = n_units;
    while (uhi - ulo > 1) {
      const uint64_t step = (uhi - ulo + 31) / 32;
      const uint64_t pu = ulo + static_cast<uint64_t>(lane) * step;
      const bool le = pu < uhi && voff_at(sc, pu * kBkRows, rows_per_tile, n_rows, n_tiles) * E <= blo;
      const uint32_t m = __ballot_sync(0xffffffffu, le);
      const uint64_t k = static_cast<uint64_t>(31 - __clz(static_cast<int>(m | 1u)));
      ulo += k * step;
      uhi = min(uhi, ulo + step);
    }
    for (uint64_t u = ulo; u < n_units && ok; ++u) {
      const uint64_t row = u * kBkRows + lane;
      const bool valid = row < n_rows;
      // Round trip 1: first-value index of this row's run and of the next.
      const uint64_t vs = valid ? voff_at(sc, row, rows_per_tile, n_rows, n_tiles) : n_values;
      uint64_t ve = __shfl_down_sync(0xffffffffu, vs, 1);
      if (lane == 31) ve = valid ? voff_at(sc, row + 1, rows_per_tile, n_rows, n_tiles) : n_values;
      if (!valid) ve = vs;
      // Round trip 2: LFVector, committed length, position of the run.
      uint32_t l = 0, b = 0;
      uint64_t pos = 0, addr = 0;
      bool has = valid && ve > vs;
      if (has) {
        const uint64_t r = row / v.L;
        l = static_cast<uint32_t>(row - r * v.L);
        const uint64_t pr = sc.pre[static_cast<uint64_t>(l) * (R + 1) + r];
        has = pr + (ve - vs) <= sc.ins_len[l];   // rounds dropped on pool exhaustion are skipped
        pos = sc.ins_base[l] + pr;
      }
      // Round trip 3: bucket address of the run's first element.
      if (has) {
        uint64_t off;
        bucket_of(pos, v.log2B, b, off);
        addr = v.buckets[static_cast<uint64_t>(l) * kMaxBuckets + b] + off * E;
      }
      // The unit's span of values, cut into 16-byte aligned windows.
      const uint64_t span_lo = __shfl_sync(0xffffffffu, vs, 0) * E;
      const uint64_t span_hi = __shfl_sync(0xffffffffu, ve, 31) * E;
      if (span_lo >= bhi) break;                 // this and every later unit lie past the block's range
      if (span_hi <= span_lo) continue;
      const uint64_t w_first = max(span_lo & ~static_cast<uint64_t>(15), blo);
      const uint64_t w_end = min((span_hi + 15) & ~static_cast<uint64_t>(15), bhi);
      for (uint64_t wlo = w_first; wlo < w_end && ok; wlo += kBkWin, ++i) {
        const uint64_t whi = min(w_end, wlo + kBkWin);
        const int s = static_cast<int>(i % kBkStages);
        if (i >= static_cast<uint32_t>(kBkStages)) {
          const bool got = mbar_wait_bounded(&s_empty[s], ((i / kBkStages) - 1) & 1u);
          ok = __all_sync(0xffffffffu, got);
          if (!ok) break;
        }
        if (lane == 0) {
          fence_proxy_async_smem();
          mbar_expect_tx(&s_full[s], static_cast<uint32_t>(whi - wlo));
          bulk_g2s(s_buf + static_cast<size_t>(s) * kBkWin, values + wlo, static_cast<uint32_t>(whi - wlo),
                   &s_full[s]);
        }
        // This row's piece in the window.
        const uint64_t pe0 = max(vs, wlo / E), pe1 = min(ve, whi / E);
        const bool in = has && pe1 > pe0;
        const uint32_t mask = __ballot_sync(0xffffffffu, in);
        if (in) {
          const int k = __popc(mask & ((1u << lane) - 1u));
          BkPiece pc;
          pc.pos = pos + (pe0 - vs);
          pc.addr = pe0 == vs ? addr : 0;
          pc.b = b;
          if (pe0 != vs) {
            uint64_t off;
            bucket_of(pc.pos, v.log2B, pc.b, off);
          }
          pc.src_off = static_cast<uint32_t>(pe0 * E - wlo);
          pc.n = static_cast<uint32_t>(pe1 - pe0);
          pc.l = l;
          s_piece[s][k] = pc;
        }
        if (lane == 0) {
          s_np[s] = __popc(mask);
          s_last[s] = 0;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&s_full[s]);
      }
    }
    // Closing stage: no data, tells the consumers to stop.
    if (ok) {
      const int s = static_cast<int>(i % kBkStages);
      if (i >= static_cast<uint32_t>(kBkStages))
        ok = __all_sync(0xffffffffu, mbar_wait_bounded(&s_empty[s], ((i / kBkStages) - 1) & 1u));
      if (ok && lane == 0) {
        s_np[s] = 0;
        s_last[s] = 1;
        mbar_arrive(&s_full[s]);
      }
    }
    if (!ok && lane == 0) {
      latch_error(v.status, GGA_ERR_TIMEOUT);
      // Let every bulk copy this warp issued land before the block leaves.
      const uint32_t lo = i > static_cast<uint32_t>(kBkStages) ? i - kBkStages : 0;
      for (uint32_t j = lo; j < i; ++j) mbar_wait_bounded(&s_full[j % kBkStages], (j / kBkStages) & 1u);
    }
  } else {
    // ------------------------------- consumers ------------------------------
    const int cw = warp - 1;
    for (uint32_t i = 0;; ++i) {
      const int s = static_cast<int>(i % kBkStages);
      const bool got = __all_sync(0xffffffffu, mbar_wait_bounded(&s_full[s], (i / kBkStages) & 1u));
      if (!got) {
        if (lane == 0) latch_error(v.status, GGA_ERR_TIMEOUT);
        break;
      }
      const uint32_t np = s_np[s];
      const bool last = s_last[s] != 0;
      const uint8_t* sb = s_buf + static_cast<size_t>(s) * kBkWin;
      for (uint32_t k = cw; k < np; k += kBkConsumers) {
        const BkPiece pc = s_piece[s][k];
        uint64_t pos = pc.pos, addr = pc.addr;
        uint32_t n = pc.n, so = pc.src_off, b = pc.b;
        const uint64_t* bk = v.buckets + static_cast<uint64_t>(pc.l) * kMaxBuckets;
        if (addr == 0) addr = bk[b] + (pos - bucket_first(b, v.log2B)) * E;
        while (n) {
          const uint64_t room = bucket_first(b, v.log2B) + bucket_len(b, v.log2B) - pos;
          const uint32_t seg = room < n ? static_cast<uint32_t>(room) : n;
          warp_store_run<E>(sb + so, addr, seg, lane);
          n -= seg;
          if (!n) break;
          pos += seg;
          so += seg * E;
          ++b;
          addr = bk[b];
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&s_empty[s]);
      if (last) break;
    }
  }
}

template <int T_TPL>
static void launch_count(const uint32_t* counts, uint64_t n_rows, uint32_t T, uint32_t L, uint32_t R,
                         const InsertScratch& s, cudaStream_t st) {
  const uint64_t n_tiles = (n_rows + count_rows_per_tile(T_TPL) - 1) / count_rows_per_tile(T_TPL);
  count_kernel<T_TPL><<<static_cast<unsigned>(n_tiles), kCountThreads, 0, st>>>(counts, n_rows, T, L, R, s.row_pre,
                                                                                 s.tile_pre, s.pre);
}

static int count_template(uint32_t T, bool vec_ok) {
  return (vec_ok && (T == 128 || T == 256 || T == 512 || T == 1024)) ? static_cast<int>(T) : 0;
}

uint64_t count_tiles(uint64_t n_rows, uint32_t T, bool vec_ok) {
  const uint64_t rows = static_cast<uint64_t>(count_rows_per_tile(count_template(T, vec_ok)));
  return (n_rows + rows - 1) / rows;
}

int launch_insert(const ArrayView& v, const InsertScratch& s, const uint32_t* counts, uint32_t R,
                  const void* values, uint64_t n_values, int num_sms, cudaStream_t st) {
  const uint64_t n_rows = static_cast<uint64_t>(R) * v.L;
  const bool vec_ok = (reinterpret_cast<uintptr_t>(counts) & 15) == 0;
  const int tpl = count_template(v.T, vec_ok);
  const uint32_t rpt = static_cast<uint32_t>(count_rows_per_tile(tpl));
  const uint64_t n_tiles = count_tiles(n_rows, v.T, vec_ok);
  switch (tpl) {
    case 128: launch_count<128>(counts, n_rows, v.T, v.L, R, s, st); break;
    case 256: launch_count<256>(counts, n_rows, v.T, v.L, R, s, st); break;
    case 512: launch_count<512>(counts, n_rows, v.T, v.L, R, s, st); break;
    case 1024: launch_count<1024>(counts, n_rows, v.T, v.L, R, s, st); break;
    default: launch_count<0>(counts, n_rows, v.T, v.L, R, s, st); break;
  }
  tile_scan_kernel<<<1, 1024, 0, st>>>(s.tile_pre, n_tiles);

  const uint32_t cce = kCopyChunkBytes / v.E;
  const unsigned rblocks = static_cast<unsigned>((static_cast<uint64_t>(v.L) * 32 + 255) / 256);
  reserve_kernel<<<rblocks, 256, 0, st>>>(v, s, R, n_values, n_tiles, cce);

  const bool src_vec = (reinterpret_cast<uintptr_t>(values) & 15) == 0;
  const uint8_t* vals = static_cast<const uint8_t*>(values);
  if (src_vec) {
    if (n_values == 0) return cudaGetLastError() == cudaSuccess ? GGA_OK : GGA_ERR_CUDA;
    const size_t smem = static_cast<size_t>(kBkStages) * kBkWin;
#define GGA_BULK(EE)                                                                                        \
  do {                                                                                                      \
    cudaFuncSetAttribute(copy_bulk_kernel<EE>, cudaFuncAttributeMaxDynamicSharedMemorySize,                 \
                         static_cast<int>(smem));                                                           \
    int per_sm = 0;                                                                                         \
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, copy_bulk_kernel<EE>, kBkThreads, smem) !=   \
            cudaSuccess || per_sm < 1)                                                                      \
      per_sm = 1;                                                                                           \
    copy_bulk_kernel<EE><<<static_cast<unsigned>(num_sms * per_sm), kBkThreads, smem, st>>>(               \
        v, vals, n_values, s, R, n_rows, n_tiles, rpt);                                                     \
  } while (0)
    if (v.E == 4) GGA_BULK(4);
    else if (v.E == 8) GGA_BULK(8);
    else GGA_BULK(16);
#undef GGA_BULK
    return cudaGetLastError() == cudaSuccess ? GGA_OK : GGA_ERR_CUDA;
  }
  // Values not 16-byte aligned: destination-ordered copy with element loads.
  // One wave: as many blocks as fit on the SMs at once.
#define GGA_COPY(EE)                                                                                          \
  do {                                                                                                        \
    auto kern = src_vec ? copy_kernel<EE, true> : copy_kernel<EE, false>;                                     \
    int per_sm = 0;                                                                                           \
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kCopyThreads, 0) != cudaSuccess ||       \
        per_sm < 1)                                                                                           \
      per_sm = 1;                                                                                             \
    kern<<<static_cast<unsigned>(num_sms * per_sm), kCopyThreads, 0, st>>>(v, vals, s, R, n_rows, n_tiles, rpt); \
  } while (0)
  if (v.E == 4) GGA_COPY(4);
  else if (v.E == 8) GGA_COPY(8);
  else GGA_COPY(16);
#undef GGA_COPY
  return cudaGetLastError() == cudaSuccess ? GGA_OK : GGA_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Resize: the grow step of the growable-array experiment (Sec. VI-C, Table
// II: the capacity is raised when necessary, before the insertion).  Every
// LFVector l gets the buckets that make its capacity at least target[l]
// (Algorithm 2 for each missing bucket, from the pool); sizes do not change.
// One thread per LFVector; the pool's pops are folded by finalize_kernel.

__global__ void __launch_bounds__(256) reserve_capacity_kernel(ArrayView v, const uint64_t* __restrict__ target) {
  const uint32_t l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= v.L) return;
  const uint32_t nb = v.nbuckets[l];
  const uint32_t need = buckets_for(target[l], v.log2B);
  if (need > nb) {
    const uint32_t got = grow_buckets(v, l, nb, need);
    v.nbuckets[l] = got;
    if (got < need) latch_error(v.status, GGA_ERR_POOL_EXHAUSTED);
  }
}

int launch_reserve(const ArrayView& v, const uint64_t* target, cudaStream_t st) {
  reserve_capacity_kernel<<<(v.L + 255) / 256, 256, 0, st>>>(v, target);
  finalize_kernel<<<1, 1024, 0, st>>>(v);
  return cudaGetLastError() == cudaSuccess ? GGA_OK : GGA_ERR_CUDA;
}

int launch_finalize(const ArrayView& v, cudaStream_t st) {
  finalize_kernel<<<1, 1024, 0, st>>>(v);
  return cudaGetLastError() == cudaSuccess ? GGA_OK : GGA_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// In-kernel generated insertion.

// A pass's values are staged in shared memory (a pass averages 16 KB at
// K = 8 rounds, 512 threads, one int32 per thread and round; a pass that
// does not fit writes directly).  T in (256, 512] is played by blocks of
// T / GGA_GEN_VT threads, GGA_GEN_VT virtual threads each (one scan word
// and one share of every barrier serve them), GGA_GEN_MINB_VT resident per
// SM with a GGA_GEN_STAGE_VT-byte stage: measured on GB300 for the
// paper-shaped workload (1024 LFVectors x 512 threads x 512 rounds, int32),
// 128 threads x 4, 8 per SM: 0.737 ms; 256 x 2, 4 per SM: 0.753 ms; 512 x 1,
// 3 per SM (40 registers, 48 KB stage): 0.816 ms.  Other T use one virtual
// thread per thread, blocks of up to 512 threads 3 per SM (up to 1024: 1).
#ifndef GGA_GEN_VT
#define GGA_GEN_VT 4
#endif
#ifndef GGA_GEN_MINB_VT
#define GGA_GEN_MINB_VT 8
#endif
#ifndef GGA_GEN_MINB512
#define GGA_GEN_MINB512 3
#endif
#ifndef GGA_GEN_STAGE_VT
#define GGA_GEN_STAGE_VT 24576
#endif
constexpr uint32_t kGenStageBytes = 49152;
constexpr uint32_t kGenStageBytesVT = GGA_GEN_STAGE_VT;

template <int E> struct GenK { static constexpr int value = E == 16 ? 4 : 8; };

// One block per LFVector, R rounds in passes of K (grow_passes in
// gga_gen.cuh), with no target.
template <int E, int K, int KV, int MAXT, int MINB, int DIST>
__global__ void __launch_bounds__(MAXT, MINB) gen_insert_kernel(const __grid_constant__ ArrayView v,
                                                                const __grid_constant__ GenParams g, uint32_t R,
                                                                uint32_t stage_bytes) {
  extern __shared__ uint4 s_stage4[];
  __shared__ GenShared sh;
  bool done;
  grow_passes<E, K, KV, false, DIST>(v, g, blockIdx.x, R, ~0ull, sh, s_stage4, stage_bytes / E, &done);
}

int launch_insert_generated(const ArrayView& v, const gga_gen_spec& spec, uint32_t R, uint32_t* /*done*/,
                            int /*num_sms*/, cudaStream_t st) {
  const GenParams g = make_gen_params(spec);
  const bool vt = GGA_GEN_VT > 1 && v.T > 256 && v.T <= 512;
  const uint32_t NT = vt ? ((v.T + GGA_GEN_VT - 1) / GGA_GEN_VT + 31) / 32 * 32 : (v.T + 31) / 32 * 32;
  const size_t smem = vt ? kGenStageBytesVT : kGenStageBytes;
#define GGA_GEN_AD(EE, KK, KV, MT, MB, DD)                                                                   \
  do {                                                                                                       \
    cudaFuncSetAttribute(gen_insert_kernel<EE, KK, KV, MT, MB, DD>,                                          \
                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));               \
    gen_insert_kernel<EE, KK, KV, MT, MB, DD><<<v.L, NT, smem, st>>>(v, g, R, static_cast<uint32_t>(smem));   \
  } while (0)
  // The count distribution is a template argument: the draw loop then has
  // no per-draw dispatch.
#define GGA_GEN_AS(EE, KK, KV, MT, MB)                                                                       \
  do {                                                                                                       \
    switch (g.dist) {                                                                                        \
      case GGA_DIST_BERNOULLI: GGA_GEN_AD(EE, KK, KV, MT, MB, GGA_DIST_BERNOULLI); break;                    \
      case GGA_DIST_UNIFORM3: GGA_GEN_AD(EE, KK, KV, MT, MB, GGA_DIST_UNIFORM3); break;                      \
      case GGA_DIST_GEOMETRIC: GGA_GEN_AD(EE, KK, KV, MT, MB, GGA_DIST_GEOMETRIC); break;                    \
      default: GGA_GEN_AD(EE, KK, KV, MT, MB, GGA_DIST_POISSON); break;                                      \
    }                                                                                                        \
  } while (0)
  // Rounds per pass: a pass then averages <= 32 KB at one element per thread
  // and round (K halves for blocks of more than 512 threads beyond 4 bytes).
#define GGA_GEN(EE)                                                                                          \
  do {                                                                                                       \
    if (vt) GGA_GEN_AS(EE, GenK<EE>::value, (GGA_GEN_VT > 1 ? GGA_GEN_VT : 2), 512 / (GGA_GEN_VT > 1 ? GGA_GEN_VT : 2),   \
                       GGA_GEN_MINB_VT);                                                                     \
    else if (NT <= 512) GGA_GEN_AS(EE, GenK<EE>::value, 1, 512, GGA_GEN_MINB512);                            \
    else GGA_GEN_AS(EE, (EE == 4 ? 8 : GenK<EE>::value / 2), 1, 1024, 1);                                    \
  } while (0)
  if (v.E == 4) GGA_GEN(4);
  else if (v.E == 8) GGA_GEN(8);
  else GGA_GEN(16);
#undef GGA_GEN
#undef GGA_GEN_AS
#undef GGA_GEN_AD
  finalize_kernel<<<1, 1024, 0, st>>>(v);
  return cudaGetLastError() == cudaSuccess ? GGA_OK : GGA_ERR_CUDA;
}

}  // namespace gga
