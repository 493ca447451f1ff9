// gga_batch.cu -- many GGArrays grown in one persistent launch.
//
// A batch is a list of jobs: an array, the draws of its counts and values
// (as gga_insert_generated), and a target size.  gga_batch_grow runs one
// persistent kernel over all (array, LFVector) items, largest first, taken
// from an atomic ticket: a block grows its LFVector in passes of several
// rounds -- every thread draws its counts, a block scan gives positions,
// counts are clipped at the LFVector's target by the same scan, the leader
// reserves and allocates, the block stages the values and writes them with
// 128-bit stores (Algorithm 1 with thread coarsening: a block of 512 threads
// plays T <= 1024 threads).  Then one kernel folds the pool
// pops and one finalizes every array.  Nothing allocates and nothing waits
// on the host, so the whole step can be captured in a CUDA graph and
// replayed (gga_batch_capture / gga_batch_replay).
#include <algorithm>
#include <new>
#include <vector>

#include "gga_gen.cuh"

namespace gga {

int launch_clear(const ArrayView& v, cudaStream_t st);

namespace {

// Threads per block and virtual threads per thread (T <= kBatchThreads *
// kBatchKV = 1024) and resident blocks per SM.
#ifndef GGA_BATCH_THREADS
#define GGA_BATCH_THREADS 512
#endif
constexpr int kBatchThreads = GGA_BATCH_THREADS;
constexpr int kBatchKV = 1024 / kBatchThreads;
constexpr int kBatchMinBlocks = 1024 / kBatchThreads;
// Stage of a pass: 80 KB, two blocks per SM.  Measured on GB300 for the
// 4096-array workload (rounds per pass for 8- / 16-byte payloads): 48 KB
// with 4 / 2 rounds 4.30 ms, 80 KB with 4 / 4 rounds 4.24 ms, 96 KB with
// 4 / 4 4.25 ms, with 6 / 4 4.31 ms.
constexpr uint32_t kBatchStageBytes = 81920;
constexpr uint32_t kBatchMaxRounds = 1u << 20;

struct BatchJob {
  ArrayView v;
  GenParams g;
  uint64_t target;
};

struct BatchItem {
  uint32_t job;
  uint32_t l;
};

// Grow LFVector l of job J to its share of the target: rounds of in-thread
// insertions in passes of K (grow_passes in gga_gen.cuh), clipped at the
// target.  All threads of the block call it.
#ifndef GGA_BATCH_NOINLINE
#define GGA_BATCH_NOINLINE 0
#endif
// One distribution's pass loop; with GGA_BATCH_NOINLINE a function of its
// own, register-allocated apart from the other (payload, distribution) forms.
template <int E, int K, int DIST>
__device__ __forceinline__ uint32_t grow_item_passes_inl(const ArrayView& v, const GenParams& g, uint32_t l,
                                                         uint64_t target, GenShared& sh, uint4* stage, bool* done) {
  return grow_passes<E, K, kBatchKV, true, DIST>(v, g, l, kBatchMaxRounds, target, sh, stage, kBatchStageBytes / E,
                                                 done);
}
template <int E, int K, int DIST>
__device__ __noinline__ uint32_t grow_item_passes_call(const ArrayView& v, const GenParams& g, uint32_t l,
                                                       uint64_t target, GenShared& sh, uint4* stage, bool* done) {
  return grow_item_passes_inl<E, K, DIST>(v, g, l, target, sh, stage, done);
}
template <int E, int K, int DIST>
__device__ __forceinline__ uint32_t grow_item_passes(const ArrayView& v, const GenParams& g, uint32_t l,
                                                     uint64_t target, GenShared& sh, uint4* stage, bool* done) {
  return GGA_BATCH_NOINLINE ? grow_item_passes_call<E, K, DIST>(v, g, l, target, sh, stage, done)
                            : grow_item_passes_inl<E, K, DIST>(v, g, l, target, sh, stage, done);
}

template <int E>
__device__ void grow_item(const BatchJob& J, uint32_t l, GenShared& sh, uint4* stage) {
  const ArrayView& v = J.v;
  const uint64_t target = J.target / v.L + (l < J.target % v.L ? 1 : 0);
  // Rounds per pass: a pass of T <= 1024 threads at one element per thread
  // and round then averages <= 64 KB, inside the 80 KB stage.
  constexpr int K = E == 4 ? 8 : 4;
  uint32_t drawn;
  bool done;
  // One dispatch per item on the count distribution, none per draw.
  switch (J.g.dist) {
    case GGA_DIST_BERNOULLI:
      drawn = grow_item_passes<E, K, GGA_DIST_BERNOULLI>(v, J.g, l, target, sh, stage, &done);
      break;
    case GGA_DIST_UNIFORM3:
      drawn = grow_item_passes<E, K, GGA_DIST_UNIFORM3>(v, J.g, l, target, sh, stage, &done);
      break;
    case GGA_DIST_GEOMETRIC:
      drawn = grow_item_passes<E, K, GGA_DIST_GEOMETRIC>(v, J.g, l, target, sh, stage, &done);
      break;
    default:
      drawn = grow_item_passes<E, K, GGA_DIST_POISSON>(v, J.g, l, target, sh, stage, &done);
      break;
  }
  if (threadIdx.x == 0 && !done && drawn >= kBatchMaxRounds) latch_error(v.status, GGA_ERR_TIMEOUT);
  __syncthreads();
}

__global__ void __launch_bounds__(kBatchThreads, kBatchMinBlocks) batch_grow_kernel(const BatchJob* __restrict__ jobs,
                                                                      const BatchItem* __restrict__ items,
                                                                      uint32_t n_items, uint32_t* ticket) {
  extern __shared__ uint4 s_stage4[];
  __shared__ GenShared sh;
  __shared__ uint32_t s_item;
  // The item's job (its view and draws) in shared memory: the pass loop
  // reads these fields over and over, and from here they are shared-memory
  // loads instead of global ones.
  __shared__ __align__(16) BatchJob s_job;
  static_assert(sizeof(BatchJob) % 8 == 0, "job copied in 8-byte words");
  while (true) {
    if (threadIdx.x == 0) s_item = atomicAdd(ticket, 1u);
    __syncthreads();
    const uint32_t it = s_item;
    if (it >= n_items) break;
    const BatchItem item = items[it];
    if (threadIdx.x < sizeof(BatchJob) / 8)
      reinterpret_cast<unsigned long long*>(&s_job)[threadIdx.x] =
          reinterpret_cast<const unsigned long long*>(jobs + item.job)[threadIdx.x];
    __syncthreads();
    const BatchJob& J = s_job;
    switch (J.v.E) {
      case 4: grow_item<4>(J, item.l, sh, s_stage4); break;
      case 8: grow_item<8>(J, item.l, sh, s_stage4); break;
      default: grow_item<16>(J, item.l, sh, s_stage4); break;
    }
  }
}

// Fold the pops of the grow kernel into every pool's queue heads; reset
// the ticket for the next run.
__global__ void batch_fixup_kernel(PoolState* const* pools, uint32_t n_pools, uint32_t* ticket) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_pools) ring_fixup(pools[i]);
  if (i == 0) *ticket = 0;
}

__global__ void __launch_bounds__(256) batch_finalize_kernel(const BatchJob* __restrict__ jobs) {
  __shared__ uint64_t s_warp[33];
  finalize_block(jobs[blockIdx.x].v, nullptr, nullptr, nullptr, 1, s_warp);
}

// Every bucket of every item back to its pool's queue; sizes to zero.
__global__ void batch_clear_kernel(const BatchJob* __restrict__ jobs, const BatchItem* __restrict__ items) {
  const BatchItem item = items[blockIdx.x];
  const ArrayView& v = jobs[item.job].v;
  const uint64_t l = item.l;
  for (uint32_t b = threadIdx.x; b < static_cast<uint32_t>(kMaxBuckets); b += blockDim.x) {
    uint64_t* slot = v.buckets + l * kMaxBuckets + b;
    const uint64_t a = *slot;
    if (a) {
      if (!ring_push(v.pool, class_of(bucket_len(b, v.log2B) * v.E), a)) latch_error(v.status, GGA_ERR_INVALID);
      *slot = 0;
    }
  }
  if (threadIdx.x == 0) {
    v.sizes[l] = 0;
    v.nbuckets[l] = 0;
  }
}

}  // namespace
}  // namespace gga

struct gga_batch_t {
  gga::BatchJob* jobs;
  gga::BatchItem* items;
  gga::PoolState** pools;
  uint32_t* ticket;
  uint32_t n_jobs, n_items, n_pools;
  int num_sms;
  unsigned grid;
  cudaGraphExec_t graph;
  bool has_graph;
};

namespace {

int batch_grow(gga_batch_t* b, cudaStream_t st) {
  if (b->n_items) {
    gga::batch_grow_kernel<<<b->grid, gga::kBatchThreads, gga::kBatchStageBytes, st>>>(b->jobs, b->items,
                                                                                         b->n_items, b->ticket);
    gga::batch_fixup_kernel<<<(b->n_pools + 63) / 64 + 1, 64, 0, st>>>(b->pools, b->n_pools, b->ticket);
  }
  if (b->n_jobs) gga::batch_finalize_kernel<<<b->n_jobs, 256, 0, st>>>(b->jobs);
  return cudaGetLastError() == cudaSuccess ? GGA_OK : GGA_ERR_CUDA;
}

int batch_clear(gga_batch_t* b, cudaStream_t st) {
  if (b->n_items) gga::batch_clear_kernel<<<b->n_items, 64, 0, st>>>(b->jobs, b->items);
  if (b->n_jobs) gga::batch_finalize_kernel<<<b->n_jobs, 256, 0, st>>>(b->jobs);
  return cudaGetLastError() == cudaSuccess ? GGA_OK : GGA_ERR_CUDA;
}

}  // namespace

extern "C" {

int gga_batch_create(const gga_batch_job* jobs, uint32_t n_jobs, void* stream, gga_batch* out) {
  if (!out || (n_jobs && !jobs)) return GGA_ERR_INVALID;
  *out = nullptr;
  std::vector<gga::BatchJob> hj(n_jobs);
  std::vector<std::pair<uint64_t, gga::BatchItem>> hi;
  std::vector<gga::PoolState*> hp;
  int num_sms = 0;
  for (uint32_t j = 0; j < n_jobs; ++j) {
    gga::InsertScratch ins;
    int dev = 0;
    if (!gga::handle_parts(jobs[j].array, &hj[j].v, &ins, &dev, &num_sms)) return GGA_ERR_INVALID;
    const gga_gen_spec& sp = jobs[j].spec;
    if (sp.dist > GGA_DIST_POISSON || sp.n_thresholds > GGA_MAX_THRESHOLDS ||
        (sp.dist == GGA_DIST_POISSON && sp.n_thresholds == 0))
      return GGA_ERR_INVALID;
    hj[j].g = gga::make_gen_params(sp);
    hj[j].target = jobs[j].target;
    const uint32_t L = hj[j].v.L;
    for (uint32_t l = 0; l < L; ++l) {
      const uint64_t tl = jobs[j].target / L + (l < jobs[j].target % L ? 1 : 0);
      if (tl) hi.push_back({tl, gga::BatchItem{j, l}});
    }
    if (std::find(hp.begin(), hp.end(), hj[j].v.pool) == hp.end()) hp.push_back(hj[j].v.pool);
  }
  // Largest LFVectors first: the ticket then balances the tail.
  std::stable_sort(hi.begin(), hi.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
  std::vector<gga::BatchItem> items(hi.size());
  for (size_t i = 0; i < hi.size(); ++i) items[i] = hi[i].second;

  gga_batch_t* b = new (std::nothrow) gga_batch_t();
  if (!b) return GGA_ERR_CUDA;
  b->n_jobs = n_jobs;
  b->n_items = static_cast<uint32_t>(items.size());
  b->n_pools = static_cast<uint32_t>(hp.size());
  b->has_graph = false;
  b->jobs = nullptr;
  b->items = nullptr;
  b->pools = nullptr;
  b->ticket = nullptr;
  if (num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
  }
  b->num_sms = num_sms;
  int per_sm = 0;
  cudaFuncSetAttribute(gga::batch_grow_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       static_cast<int>(gga::kBatchStageBytes));
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gga::batch_grow_kernel, gga::kBatchThreads,
                                                    gga::kBatchStageBytes) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  b->grid = static_cast<unsigned>(num_sms * per_sm);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = GGA_OK;
  if (cudaMalloc(&b->jobs, sizeof(gga::BatchJob) * (n_jobs ? n_jobs : 1)) != cudaSuccess ||
      cudaMalloc(&b->items, sizeof(gga::BatchItem) * (items.empty() ? 1 : items.size())) != cudaSuccess ||
      cudaMalloc(&b->pools, sizeof(gga::PoolState*) * (hp.empty() ? 1 : hp.size())) != cudaSuccess ||
      cudaMalloc(&b->ticket, sizeof(uint32_t)) != cudaSuccess)
    rc = GGA_ERR_CUDA;
  if (rc == GGA_OK &&
      ((n_jobs && cudaMemcpyAsync(b->jobs, hj.data(), sizeof(gga::BatchJob) * n_jobs, cudaMemcpyHostToDevice, st) !=
                      cudaSuccess) ||
       (!items.empty() && cudaMemcpyAsync(b->items, items.data(), sizeof(gga::BatchItem) * items.size(),
                                          cudaMemcpyHostToDevice, st) != cudaSuccess) ||
       (!hp.empty() && cudaMemcpyAsync(b->pools, hp.data(), sizeof(gga::PoolState*) * hp.size(),
                                       cudaMemcpyHostToDevice, st) != cudaSuccess) ||
       cudaMemsetAsync(b->ticket, 0, sizeof(uint32_t), st) != cudaSuccess ||
       cudaStreamSynchronize(st) != cudaSuccess))
    rc = GGA_ERR_CUDA;
  if (rc != GGA_OK) {
    gga_batch_destroy(b);
    return rc;
  }
  *out = b;
  return GGA_OK;
}

int gga_batch_grow(gga_batch b, void* stream) {
  if (!b) return GGA_ERR_INVALID;
  return batch_grow(b, static_cast<cudaStream_t>(stream));
}

int gga_batch_clear(gga_batch b, void* stream) {
  if (!b) return GGA_ERR_INVALID;
  return batch_clear(b, static_cast<cudaStream_t>(stream));
}

int gga_batch_capture(gga_batch b, void* stream) {
  if (!b || !stream) return GGA_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (b->has_graph) {
    cudaGraphExecDestroy(b->graph);
    b->has_graph = false;
  }
  cudaGraph_t g;
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return GGA_ERR_CUDA;
  int rc = batch_clear(b, st);
  if (rc == GGA_OK) rc = batch_grow(b, st);
  if (cudaStreamEndCapture(st, &g) != cudaSuccess) return GGA_ERR_CUDA;
  if (rc != GGA_OK) {
    cudaGraphDestroy(g);
    return rc;
  }
  const cudaError_t e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return GGA_ERR_CUDA;
  b->has_graph = true;
  return GGA_OK;
}

int gga_batch_replay(gga_batch b, void* stream) {
  if (!b || !b->has_graph) return GGA_ERR_INVALID;
  return cudaGraphLaunch(b->graph, static_cast<cudaStream_t>(stream)) == cudaSuccess ? GGA_OK : GGA_ERR_CUDA;
}

int gga_batch_destroy(gga_batch b) {
  if (!b) return GGA_ERR_INVALID;
  int rc = GGA_OK;
  if (cudaDeviceSynchronize() != cudaSuccess) rc = GGA_ERR_CUDA;
  if (b->has_graph) cudaGraphExecDestroy(b->graph);
  if (b->jobs) cudaFree(b->jobs);
  if (b->items) cudaFree(b->items);
  if (b->pools) cudaFree(b->pools);
  if (b->ticket) cudaFree(b->ticket);
  delete b;
  return rc;
}

}  // extern "C"
