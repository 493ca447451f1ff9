// gga_server.cu -- gga_serve_run (include/gga_serve.h): the request server's
// scheduling loop in native code.  Host code only; the GPU work is the
// library's own entry points (gga_append_batch, gga_read_batch, gga_flatten,
// gga_clear) on one stream, tracked with events.  The rules are those of
// the Python reference model (serving.py, Server.run), step for step.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <limits>
#include <queue>
#include <thread>
#include <unordered_map>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "gga.h"
#include "gga_serve.h"

namespace {

constexpr int kClasses = 64;
constexpr uint32_t kLookAhead = 32;   // waiting appends tried per step after memory was freed

// Bucket classes (power-of-two bytes, at least 256) with counts.
typedef std::vector<std::pair<uint8_t, uint32_t>> Tally;

uint32_t bit_length(uint64_t x) { return x == 0 ? 0u : 64u - static_cast<uint32_t>(__builtin_clzll(x)); }

uint8_t byte_class(uint64_t nbytes) {
  return static_cast<uint8_t>(std::max<uint32_t>(8u, bit_length(std::max<uint64_t>(nbytes, 256) - 1)));
}

// Buckets reached by LFVector-local indices 0..size-1 (Algorithm 2's sizes B 2^b).
uint32_t buckets_for(uint64_t size, uint64_t B) {
  return size == 0 ? 0u : bit_length(size - 1 + B) - bit_length(B) + 1;
}

void tally_add(Tally& t, uint8_t c) {
  for (auto& p : t)
    if (p.first == c) {
      ++p.second;
      return;
    }
  t.emplace_back(c, 1u);
}

// Host copy of the pool's accounting: free buckets per class, bump pointer.
struct Mirror {
  uint64_t cap = 0, bump = 0;
  uint64_t free_[kClasses] = {};
  uint64_t need(const Tally& t) const {
    uint64_t b = 0;
    for (const auto& p : t)
      if (p.second > free_[p.first]) b += static_cast<uint64_t>(p.second - free_[p.first]) << p.first;
    return b;
  }
  bool fits(const Tally& t) const { return bump + need(t) <= cap; }
  void take(const Tally& t) {
    for (const auto& p : t) {
      uint64_t f = free_[p.first];
      if (p.second > f) {
        bump += static_cast<uint64_t>(p.second - f) << p.first;
        f = p.second;
      }
      free_[p.first] = f - p.second;
    }
  }
  void give(const Tally& t) {
    for (const auto& p : t) free_[p.first] += p.second;
  }
};

struct ArrayState {
  std::vector<uint64_t> sizes;
  std::deque<uint64_t> queue;
  bool busy = false;
};

struct Result {
  uint64_t r;
  const void* ptr;
  uint64_t n;
  void* owned;   // a stream-ordered allocation to free after the step, or nullptr
};

struct Step {
  cudaEvent_t ev;
  std::vector<uint64_t> taken;
  std::vector<Result> results;
};

typedef std::pair<double, uint64_t> Item;   // (arrival, request): oldest first
typedef std::priority_queue<Item, std::vector<Item>, std::greater<Item>> MinHeap;

}  // namespace

extern "C" int gga_serve_run(const gga_serve_config* cfg, gga_handle const* arrays, uint64_t m,
                             const double* t_arr, const int8_t* typ, const int64_t* arr, const int64_t* nn,
                             const int64_t* tag, void* read_out_dev, void* flat_arena_dev, uint64_t arena_elems,
                             double* lat, int8_t* state, gga_serve_result_fn on_result, void* ctx,
                             gga_serve_stats* stats, void* stream) {
  if (!cfg || !arrays || (m > 0 && (!t_arr || !typ || !arr || !nn || !tag || !lat || !state))) return GGA_ERR_INVALID;
  if (cfg->n_arrays == 0 || cfg->L == 0 || cfg->max_inflight == 0 || cfg->max_batch == 0 || cfg->read_n == 0 ||
      (cfg->E != 4 && cfg->E != 8 && cfg->E != 16) || cfg->B == 0 || (cfg->B & (cfg->B - 1)) != 0)
    return GGA_ERR_INVALID;
  for (uint64_t r = 0; r < m; ++r) {
    if (arr[r] < 0 || static_cast<uint64_t>(arr[r]) >= cfg->n_arrays || typ[r] < 0 || typ[r] > GGA_REQ_FLATTEN)
      return GGA_ERR_INVALID;
    if (typ[r] == GGA_REQ_APPEND && nn[r] < 1) return GGA_ERR_INVALID;
    if (typ[r] == GGA_REQ_READ && !read_out_dev) return GGA_ERR_INVALID;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint32_t L = cfg->L, E = cfg->E;
  const uint64_t B = cfg->B;
  const uint32_t max_batch = cfg->batched ? cfg->max_batch : 1u;
  const uint32_t slots = cfg->max_inflight + 1;

  std::vector<ArrayState> as(cfg->n_arrays);
  for (auto& a : as) a.sizes.assign(L, 0);
  Mirror mirror;
  mirror.cap = cfg->pool_bytes;
  for (uint64_t r = 0; r < m; ++r) {
    lat[r] = std::numeric_limits<double>::quiet_NaN();
    state[r] = 0;
  }
  std::vector<cudaEvent_t> events(slots);
  for (auto& e : events)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return GGA_ERR_CUDA;

  MinHeap heap, waiting;
  std::unordered_map<uint64_t, Tally> wait_cls;
  uint64_t freed = 0, checked = 0, nxt = 0, appended = 0, steps = 0, step_reqs = 0;
  double t_full = std::numeric_limits<double>::infinity();
  std::deque<Step> inflight;
  uint32_t slot = 0;
  uint64_t arena_ptr = 0;
  int rc = GGA_OK;
  const auto t0 = std::chrono::steady_clock::now();
  const auto now_s = [&]() { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); };
  const auto next_head = [&](ArrayState& a) {
    a.queue.pop_front();
    if (!a.queue.empty()) heap.emplace(t_arr[a.queue.front()], a.queue.front());
  };
  const auto append_classes = [&](const ArrayState& a, uint64_t n) {
    Tally t;
    for (uint32_t l = 0; l < L; ++l) {
      const uint64_t c = n / L + (l < n % L ? 1 : 0);
      const uint64_t s = a.sizes[l];
      for (uint32_t b = buckets_for(s, B); b < buckets_for(s + c, B); ++b) tally_add(t, byte_class((B << b) * E));
    }
    return t;
  };
  const auto all_classes = [&](const ArrayState& a) {
    Tally t;
    for (uint64_t s : a.sizes)
      for (uint32_t b = 0; b < buckets_for(s, B); ++b) tally_add(t, byte_class((B << b) * E));
    return t;
  };
  std::vector<uint64_t> appends, reads, flats, taken;
  std::vector<gga_append_req> areq;
  std::vector<gga_read_req> rreq;

  while (true) {
    const double now = now_s();
    // Arrivals: per array in order; a request is a ready head when its array has nothing ahead.
    while (nxt < m && t_arr[nxt] <= now) {
      ArrayState& a = as[arr[nxt]];
      a.queue.push_back(nxt);
      if (a.queue.size() == 1 && !a.busy) heap.emplace(t_arr[nxt], nxt);
      ++nxt;
    }
    // Completions.
    while (!inflight.empty() &&
           (cudaEventQuery(inflight.front().ev) == cudaSuccess || inflight.size() >= cfg->max_inflight)) {
      Step s = std::move(inflight.front());
      inflight.pop_front();
      if (cudaEventSynchronize(s.ev) != cudaSuccess) {
        rc = GGA_ERR_CUDA;
        break;
      }
      const double done = now_s();
      for (uint64_t r : s.taken) {
        lat[r] = done - t_arr[r];
        state[r] = 1;
        ArrayState& a = as[arr[r]];
        a.busy = false;
        next_head(a);
      }
      for (const Result& x : s.results) {
        if (on_result) on_result(ctx, x.r, x.ptr, x.n);
        if (x.owned) cudaFreeAsync(x.owned, st);
      }
    }
    if (rc != GGA_OK) break;
    // Appends past their deadline are rejected; their arrays move on.
    while (!waiting.empty() && now - waiting.top().first > cfg->deadline_s) {
      const uint64_t r = waiting.top().second;
      waiting.pop();
      wait_cls.erase(r);
      state[r] = 2;
      next_head(as[arr[r]]);
    }
    appends.clear();
    reads.clear();
    flats.clear();
    taken.clear();
    const auto admit = [&](uint64_t r, const Tally& cls) {
      ArrayState& a = as[arr[r]];
      mirror.take(cls);
      const uint64_t n = static_cast<uint64_t>(nn[r]);
      for (uint32_t l = 0; l < L; ++l) a.sizes[l] += n / L + (l < n % L ? 1 : 0);
      appends.push_back(r);
      a.busy = true;
      taken.push_back(r);
    };
    // Waiting appends, oldest first, once memory has been freed since they were last tried.
    if (!waiting.empty() && freed != checked) {
      checked = freed;
      std::vector<Item> keep;
      uint32_t tried = 0;
      while (!waiting.empty() && taken.size() < max_batch && tried < kLookAhead) {
        const Item it = waiting.top();
        waiting.pop();
        ++tried;
        auto w = wait_cls.find(it.second);
        if (mirror.fits(w->second)) {
          const Tally cls = std::move(w->second);
          wait_cls.erase(w);
          admit(it.second, cls);
        } else {
          keep.push_back(it);
        }
      }
      for (const Item& it : keep) waiting.push(it);
    }
    // Ready heads, oldest first; an append that does not fit goes to the waiting queue.
    while (!heap.empty() && taken.size() < max_batch) {
      const uint64_t r = heap.top().second;
      heap.pop();
      ArrayState& a = as[arr[r]];
      if (typ[r] == GGA_REQ_APPEND) {
        Tally cls = append_classes(a, static_cast<uint64_t>(nn[r]));
        if (mirror.fits(cls)) {
          admit(r, cls);
        } else {
          wait_cls.emplace(r, std::move(cls));
          waiting.emplace(t_arr[r], r);
          t_full = std::min(t_full, t_arr[r]);
        }
        continue;
      }
      (typ[r] == GGA_REQ_READ ? reads : flats).push_back(r);
      a.busy = true;
      taken.push_back(r);
    }
    if (!taken.empty()) {
      Step s;
      s.ev = events[slot];
      if (!appends.empty()) {
        areq.resize(appends.size());
        for (size_t i = 0; i < appends.size(); ++i) {
          const uint64_t r = appends[i];
          areq[i].array = arrays[arr[r]];
          areq[i].n = static_cast<uint64_t>(nn[r]);
          areq[i].tag = static_cast<uint64_t>(tag[r]);
          appended += areq[i].n;
        }
        rc = gga_append_batch(areq.data(), static_cast<uint32_t>(areq.size()), stream);
      }
      if (rc == GGA_OK && !reads.empty()) {
        rreq.resize(reads.size());
        for (size_t j = 0; j < reads.size(); ++j) {
          const uint64_t r = reads[j];
          char* out = static_cast<char*>(read_out_dev) +
                      ((static_cast<uint64_t>(slot) * cfg->max_batch + j) * cfg->read_n) * E;
          rreq[j].array = arrays[arr[r]];
          rreq[j].n = cfg->read_n;
          rreq[j].seed = static_cast<uint64_t>(tag[r]);
          rreq[j].out = out;
          s.results.push_back({r, out, cfg->read_n, nullptr});
        }
        rc = gga_read_batch(rreq.data(), static_cast<uint32_t>(rreq.size()), stream);
      }
      for (size_t i = 0; rc == GGA_OK && i < flats.size(); ++i) {
        const uint64_t r = flats[i];
        ArrayState& a = as[arr[r]];
        uint64_t n = 0;
        for (uint64_t x : a.sizes) n += x;
        void* dst = nullptr;
        void* owned = nullptr;
        if (n + 1 > arena_elems) {
          if (cudaMallocAsync(&owned, (n + 1) * E, st) != cudaSuccess) {
            rc = GGA_ERR_CUDA;
            break;
          }
          dst = owned;
        } else {
          if (arena_ptr + n + 1 > arena_elems) arena_ptr = 0;
          dst = static_cast<char*>(flat_arena_dev) + arena_ptr * E;
          arena_ptr += n + 1;
        }
        rc = gga_flatten(arrays[arr[r]], dst, n, stream);
        if (rc == GGA_OK) rc = gga_clear(arrays[arr[r]], stream);
        mirror.give(all_classes(a));
        std::fill(a.sizes.begin(), a.sizes.end(), 0);
        s.results.push_back({r, dst, n, owned});
      }
      if (rc != GGA_OK) break;
      ++steps;
      step_reqs += taken.size();
      freed += flats.size();
      s.taken = taken;
      if (cudaEventRecord(s.ev, st) != cudaSuccess) {
        rc = GGA_ERR_CUDA;
        break;
      }
      inflight.push_back(std::move(s));
      slot = (slot + 1) % slots;
      if (!cfg->batched && cudaEventSynchronize(inflight.back().ev) != cudaSuccess) {
        rc = GGA_ERR_CUDA;
        break;
      }
    } else if (inflight.empty()) {
      if (nxt >= m && heap.empty() && waiting.empty()) break;
      const double wait = nxt < m ? t_arr[nxt] - now_s() : 0.0005;
      if (wait > 0) std::this_thread::sleep_for(std::chrono::duration<double>(std::min(wait, 0.0005)));
    }
  }
  // On an error: let the enqueued work finish before returning.
  for (Step& s : inflight) {
    cudaEventSynchronize(s.ev);
    for (const Result& x : s.results)
      if (x.owned) cudaFreeAsync(x.owned, st);
  }
  cudaStreamSynchronize(st);
  for (auto& e : events) cudaEventDestroy(e);
  if (stats) {
    stats->steps = steps;
    stats->step_requests = step_reqs;
    stats->appended_elements = appended;
    stats->wall_s = now_s();
    stats->first_full_s = std::isinf(t_full) ? -1.0 : t_full;
  }
  return rc;
}
