// GGArray oracle: a plain, slow, single-threaded CPU model of the GGArray of
// Meneses, Navarro and Ferrada, "GGArray: A Dynamically Growable GPU Array"
// (arXiv 2209.00103).
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
// execute this file; only tests/, the smoke check and the bench's CPU-baseline
// leg use it.  It shares no code, header, table or constant generator with the
// CUDA implementation.
//
// What it models (each function below names the passage it follows):
//   * A GGArray is an array of LFVectors, one per thread block (Sec. IV,
//     Fig. 1-2).  Here each LFVector is a std::vector of E-byte elements in
//     insertion order.
//   * Insertion (Algorithm 1, Sec. III-B): in every round each thread t of
//     block l inserts c[r][l][t] elements; positions come from a prefix sum
//     over the threads of the block, "as if it was a contiguous array"
//     (Sec. III intro to parallel insertion).  So within a round the elements
//     of block l appear in increasing thread id, a thread's elements
//     contiguous and in increasing k.
//   * Buckets (Algorithm 2): bucket b of an LFVector holds
//     2^(log2(first_block_size) + b) = B * 2^b elements and is allocated only
//     when an insertion index reaches it (Algorithm 1, the nil test).
//   * The global view (Sec. IV, paragraph after Algorithm 2): a prefix sum of
//     the LFVector sizes gives the index of each LFVector's first element; a
//     global index is located by binary search over it.  The global order is
//     therefore LFVector-major.
//   * Flatten (abstract; Sec. VI-C discussion of two-phase applications):
//     moving the elements into one contiguous static array, which this model
//     reads as the concatenation of the LFVectors in block order.
//   * The r/w operation of Sec. VI-C: a kernel that adds +1 thirty times to
//     every element; modelled as "add delta, repeats times".
//
// Readings where the paper is silent (Sec. IV and Algorithms 1-2 leave these open):
//   * log in Algorithm 2 is log2 and B must be a power of two;
//   * buckets are allocated lazily, so an empty LFVector has capacity 0;
//   * a read/write of a global index >= size is an error;
//   * random writes are applied in the order given (later ones win).
//
// Build: g++ -O2 -std=c++17 -shared -fPIC gga_oracle.cpp -o liboracle.so
// (done on demand by oracle/__init__.py).

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

enum {
  ORC_OK = 0,
  ORC_ERR_INVALID = 1,
  ORC_ERR_OUT_OF_RANGE = 2,
  ORC_ERR_DST_TOO_SMALL = 3,
};

struct OracleArray {
  uint32_t L;   // number of LFVectors (= thread blocks)
  uint32_t T;   // threads per block
  uint64_t B;   // first bucket size in elements (first_block_size)
  uint32_t E;   // element size in bytes
  // lfv[l] holds LFVector l's elements back to back, E bytes each, in
  // insertion order.
  std::vector<std::vector<unsigned char>> lfv;
  // reserved[l]: the largest capacity asked for by a resize (0 if none).
  std::vector<uint64_t> reserved;
};

bool is_power_of_two(uint64_t x) { return x != 0 && (x & (x - 1)) == 0; }

uint64_t lfv_size(const OracleArray& a, uint32_t l) {
  return a.lfv[l].size() / a.E;
}

// Sec. IV, paragraph after Algorithm 2: offsets[l] = sum of the sizes of
// LFVectors 0..l-1; offsets[L] = global size.
std::vector<uint64_t> prefix_offsets(const OracleArray& a) {
  std::vector<uint64_t> off(a.L + 1, 0);
  for (uint32_t l = 0; l < a.L; ++l) off[l + 1] = off[l] + lfv_size(a, l);
  return off;
}

// Algorithm 2: bucket b holds B * 2^b elements.  The bucket of LFVector-local
// index j is found by walking the buckets in order and subtracting their
// sizes -- deliberately a loop, the plainest statement of the layout.
void bucket_of(uint64_t j, uint64_t B, uint32_t* b_out, uint64_t* off_out) {
  uint32_t b = 0;
  uint64_t first = 0;       // LFVector-local index of bucket b's slot 0
  uint64_t bsize = B;       // B * 2^b
  while (j >= first + bsize) {
    first += bsize;
    bsize *= 2;
    ++b;
  }
  *b_out = b;
  *off_out = j - first;
}

// Capacity after lazy allocation (Algorithm 1's nil test, Algorithm 2's bucket
// sizes): the buckets reached by indices 0..size-1 are allocated, so capacity
// is B*(2^k - 1) for the least k with B*(2^k - 1) >= size, and 0 when empty.
uint64_t capacity_of(uint64_t size, uint64_t B) {
  uint64_t k = 0;
  uint64_t cap = 0;
  while (cap < size) {
    cap += B << k;
    ++k;
  }
  return cap;
}

uint64_t buckets_of(uint64_t size, uint64_t B) {
  uint64_t k = 0;
  uint64_t cap = 0;
  while (cap < size) {
    cap += B << k;
    ++k;
  }
  return k;
}

// Locate global index g (Sec. IV: binary search over the prefix sum of
// LFVector sizes).  upper_bound returns the first offset > g; the LFVector
// before it is the last one starting at or before g, which skips empty ones.
bool locate(const std::vector<uint64_t>& off, uint64_t g, uint32_t* l, uint64_t* j) {
  if (g >= off.back()) return false;
  auto it = std::upper_bound(off.begin(), off.end(), g);
  uint32_t ll = static_cast<uint32_t>((it - off.begin()) - 1);
  *l = ll;
  *j = g - off[ll];
  return true;
}

// ---------------------------------------------------------------------------
// Counter-based generator (SplitMix64, Steele, Lea and Flood, OOPSLA 2014):
// output n of the stream seeded with s is mix64(s + n * 0x9E3779B97F4A7C15),
// with the published 64-bit finalizer.  Used only for the generated-insert
// workloads, where counts and values are drawn inside the inserting threads.
uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t splitmix_at(uint64_t seed, uint64_t key) {
  return mix64(seed + (key + 1) * 0x9E3779B97F4A7C15ULL);
}

// Draw a per-thread insertion count from one 64-bit word.
//   dist 0: Bernoulli(1/2)      -> top bit
//   dist 1: Uniform{0,1,2}      -> floor(3 * u32 / 2^32), u32 = high word
//   dist 2: Geometric(1/2) - 1  -> number of trailing one bits (max 63)
//   dist 3: Poisson(1)          -> #{k : u32 >= thr[k]}, thr given as data
uint32_t draw_count(uint32_t dist, uint64_t h, const uint32_t* thr, uint32_t nthr) {
  switch (dist) {
    case 0:
      return static_cast<uint32_t>(h >> 63);
    case 1:
      return static_cast<uint32_t>(((h >> 32) * 3ULL) >> 32);
    case 2: {
      uint32_t c = 0;
      while (c < 63 && ((h >> c) & 1ULL)) ++c;
      return c;
    }
    case 3: {
      uint32_t u = static_cast<uint32_t>(h >> 32);
      uint32_t c = 0;
      for (uint32_t k = 0; k < nthr; ++k)
        if (u >= thr[k]) ++c;
      return c;
    }
    default:
      return 0;
  }
}

// Self-describing value of element k of thread gtid in round r:
// v = a*gtid + b*r + c*k (mod 2^64), stored in E bytes.  For E = 16 the
// record is {int64 key = v, float x = v & 0xFFFF, float y = (v >> 16) & 0xFFFF},
// whose floats are integers below 2^16 and therefore exact.
void make_value(uint64_t v, uint32_t E, unsigned char* out) {
  if (E == 4) {
    uint32_t w = static_cast<uint32_t>(v);
    std::memcpy(out, &w, 4);
  } else if (E == 8) {
    std::memcpy(out, &v, 8);
  } else {
    float x = static_cast<float>(v & 0xFFFFULL);
    float y = static_cast<float>((v >> 16) & 0xFFFFULL);
    std::memcpy(out, &v, 8);
    std::memcpy(out + 8, &x, 4);
    std::memcpy(out + 12, &y, 4);
  }
}

}  // namespace

extern "C" {

// Create an empty GGArray of L LFVectors for blocks of T threads, first bucket
// B elements (power of two, Algorithm 2), E-byte elements (4, 8 or 16).
void* orc_create(uint32_t L, uint32_t T, uint64_t B, uint32_t E) {
  if (L == 0 || T == 0 || !is_power_of_two(B) || !(E == 4 || E == 8 || E == 16))
    return nullptr;
  OracleArray* a = new OracleArray();
  a->L = L;
  a->T = T;
  a->B = B;
  a->E = E;
  a->lfv.assign(L, {});
  a->reserved.assign(L, 0);
  return a;
}

void orc_destroy(void* h) { delete static_cast<OracleArray*>(h); }

// Algorithm 1 applied to R rounds.  counts is [R][L][T]; values holds the
// inserted elements packed in (round, block, thread, k) order, n_values of
// them.  For every round, block and thread (in that order) the thread's
// counts[r][l][t] elements are appended to LFVector l.  If sizes_per_round is
// not null it receives the size of every LFVector after every round, [R][L].
int orc_insert(void* h, const uint32_t* counts, uint32_t R, const void* values,
               uint64_t n_values, uint64_t* sizes_per_round) {
  OracleArray& a = *static_cast<OracleArray*>(h);
  uint64_t total = 0;
  for (uint64_t i = 0; i < static_cast<uint64_t>(R) * a.L * a.T; ++i) total += counts[i];
  if (total != n_values) return ORC_ERR_INVALID;
  const unsigned char* src = static_cast<const unsigned char*>(values);
  for (uint32_t r = 0; r < R; ++r) {
    for (uint32_t l = 0; l < a.L; ++l) {
      for (uint32_t t = 0; t < a.T; ++t) {
        uint32_t c = counts[(static_cast<uint64_t>(r) * a.L + l) * a.T + t];
        for (uint32_t k = 0; k < c; ++k) {
          a.lfv[l].insert(a.lfv[l].end(), src, src + a.E);  // vector(idx) = e
          src += a.E;
        }
      }
      if (sizes_per_round) sizes_per_round[static_cast<uint64_t>(r) * a.L + l] = lfv_size(a, l);
    }
  }
  return ORC_OK;
}

// Algorithm 1 with counts and values drawn inside each inserting thread
// (the form in which a kernel calls push_back itself).  For round
// r = round0 + i (i < R), thread t of block l (gtid = l*T + t) draws
// c = draw_count(dist, splitmix_at(seed, (r << 32) | gtid)) and appends the
// values va*gtid + vb*r + vc*k for k = 0..c-1.  counts_out, if not null,
// receives the drawn counts [R][L][T].
int orc_insert_generated(void* h, uint64_t seed, uint32_t dist, const uint32_t* thr,
                         uint32_t nthr, uint64_t va, uint64_t vb, uint64_t vc,
                         uint32_t round0, uint32_t R, uint32_t* counts_out) {
  OracleArray& a = *static_cast<OracleArray*>(h);
  if (dist > 3 || (dist == 3 && thr == nullptr)) return ORC_ERR_INVALID;
  std::vector<unsigned char> e(a.E);
  for (uint32_t i = 0; i < R; ++i) {
    uint64_t r = static_cast<uint64_t>(round0) + i;
    for (uint32_t l = 0; l < a.L; ++l) {
      for (uint32_t t = 0; t < a.T; ++t) {
        uint64_t gtid = static_cast<uint64_t>(l) * a.T + t;
        uint32_t c = draw_count(dist, splitmix_at(seed, (r << 32) | gtid), thr, nthr);
        if (counts_out) counts_out[(static_cast<uint64_t>(i) * a.L + l) * a.T + t] = c;
        for (uint32_t k = 0; k < c; ++k) {
          make_value(va * gtid + vb * r + vc * k, a.E, e.data());
          a.lfv[l].insert(a.lfv[l].end(), e.begin(), e.end());
        }
      }
    }
  }
  return ORC_OK;
}

// Growth to a target size (batched arrays): LFVector l's target is
// target / L plus one for the first target % L LFVectors.  LFVector l runs
// rounds r = round0, round0 + 1, ... while its size is below its target; in
// each round its threads t = 0..T-1 draw counts as in orc_insert_generated
// and push_back in thread order until the target is reached (a thread's
// elements past the target are not inserted).  Fails if some LFVector has
// not reached its target after max_rounds rounds.
int orc_grow_to_target(void* h, uint64_t seed, uint32_t dist, const uint32_t* thr, uint32_t nthr, uint64_t va,
                       uint64_t vb, uint64_t vc, uint32_t round0, uint64_t target, uint32_t max_rounds) {
  OracleArray& a = *static_cast<OracleArray*>(h);
  if (dist > 3 || (dist == 3 && thr == nullptr)) return ORC_ERR_INVALID;
  std::vector<unsigned char> e(a.E);
  for (uint32_t l = 0; l < a.L; ++l) {
    const uint64_t tl = target / a.L + (l < target % a.L ? 1 : 0);
    uint32_t n = 0;
    for (uint64_t r = round0; lfv_size(a, l) < tl; ++r, ++n) {
      if (n >= max_rounds) return ORC_ERR_INVALID;
      for (uint32_t t = 0; t < a.T && lfv_size(a, l) < tl; ++t) {
        const uint64_t gtid = static_cast<uint64_t>(l) * a.T + t;
        const uint32_t c = draw_count(dist, splitmix_at(seed, (r << 32) | gtid), thr, nthr);
        for (uint32_t k = 0; k < c && lfv_size(a, l) < tl; ++k) {
          make_value(va * gtid + vb * r + vc * k, a.E, e.data());
          a.lfv[l].insert(a.lfv[l].end(), e.begin(), e.end());
        }
      }
    }
  }
  return ORC_OK;
}

// Served append: LFVector l receives n / L elements (one more for the first
// n % L), element k with value tag * 2^24 + l * 2^20 + k, appended in order.
int orc_append(void* h, uint64_t n, uint64_t tag) {
  OracleArray& a = *static_cast<OracleArray*>(h);
  std::vector<unsigned char> e(a.E);
  for (uint32_t l = 0; l < a.L; ++l) {
    const uint64_t c = n / a.L + (l < n % a.L ? 1 : 0);
    for (uint64_t k = 0; k < c; ++k) {
      make_value(tag * (1ULL << 24) + static_cast<uint64_t>(l) * (1ULL << 20) + k, a.E, e.data());
      a.lfv[l].insert(a.lfv[l].end(), e.begin(), e.end());
    }
  }
  return ORC_OK;
}

// Served random read: out[k] = element at global index
// floor((splitmix_at(seed, k) >> 32) * N / 2^32), N = current size; zeros if
// the array is empty (Sec. IV's global indexing through the prefix sum).
int orc_read_random(void* h, uint64_t n, uint64_t seed, void* out) {
  OracleArray& a = *static_cast<OracleArray*>(h);
  std::vector<uint64_t> off = prefix_offsets(a);
  const uint64_t N = off.back();
  unsigned char* dst = static_cast<unsigned char*>(out);
  for (uint64_t k = 0; k < n; ++k) {
    if (N == 0) {
      std::memset(dst + k * a.E, 0, a.E);
      continue;
    }
    const uint64_t g = ((splitmix_at(seed, k) >> 32) * N) >> 32;
    uint32_t l;
    uint64_t j;
    locate(off, g, &l, &j);
    std::memcpy(dst + k * a.E, a.lfv[l].data() + j * a.E, a.E);
  }
  return ORC_OK;
}

// Global size (Sec. IV: the GGArray keeps the global size).
uint64_t orc_size(void* h) {
  OracleArray& a = *static_cast<OracleArray*>(h);
  uint64_t n = 0;
  for (uint32_t l = 0; l < a.L; ++l) n += lfv_size(a, l);
  return n;
}

void orc_sizes(void* h, uint64_t* out) {
  OracleArray& a = *static_cast<OracleArray*>(h);
  for (uint32_t l = 0; l < a.L; ++l) out[l] = lfv_size(a, l);
}

// Elements LFVector l's buckets must cover: its size, or more if a resize
// asked for more.
static uint64_t covered(const OracleArray& a, uint32_t l) {
  const uint64_t s = lfv_size(a, l);
  return s > a.reserved[l] ? s : a.reserved[l];
}

// Capacity and bucket count of every LFVector under lazy bucket allocation.
void orc_capacities(void* h, uint64_t* caps, uint64_t* nbuckets) {
  OracleArray& a = *static_cast<OracleArray*>(h);
  for (uint32_t l = 0; l < a.L; ++l) {
    if (caps) caps[l] = capacity_of(covered(a, l), a.B);
    if (nbuckets) nbuckets[l] = buckets_of(covered(a, l), a.B);
  }
}

// Resize (the grow step of Sec. VI-C's experiment): LFVector l's buckets
// are allocated until its capacity is at least target[l]; sizes and
// contents stay.
int orc_reserve(void* h, const uint64_t* target) {
  OracleArray& a = *static_cast<OracleArray*>(h);
  for (uint32_t l = 0; l < a.L; ++l)
    if (target[l] > a.reserved[l]) a.reserved[l] = target[l];
  return ORC_OK;
}

// Prefix sum of LFVector sizes, L+1 entries (Sec. IV).
void orc_offsets(void* h, uint64_t* out) {
  OracleArray& a = *static_cast<OracleArray*>(h);
  std::vector<uint64_t> off = prefix_offsets(a);
  std::copy(off.begin(), off.end(), out);
}

// (bucket, offset) of LFVector-local index j for first bucket size B.
void orc_bucket_of(uint64_t j, uint64_t B, uint32_t* b, uint64_t* off) { bucket_of(j, B, b, off); }

uint64_t orc_capacity_of(uint64_t size, uint64_t B) { return capacity_of(size, B); }

// rw_g-style random read (Sec. VI-B): out[i] = element at global index idx[i].
// Returns ORC_ERR_OUT_OF_RANGE (and writes zeros there) if an index >= size.
int orc_read(void* h, const uint64_t* idx, uint64_t n, void* out) {
  OracleArray& a = *static_cast<OracleArray*>(h);
  std::vector<uint64_t> off = prefix_offsets(a);
  unsigned char* dst = static_cast<unsigned char*>(out);
  int rc = ORC_OK;
  for (uint64_t i = 0; i < n; ++i) {
    uint32_t l;
    uint64_t j;
    if (!locate(off, idx[i], &l, &j)) {
      std::memset(dst + i * a.E, 0, a.E);
      rc = ORC_ERR_OUT_OF_RANGE;
      continue;
    }
    std::memcpy(dst + i * a.E, a.lfv[l].data() + j * a.E, a.E);
  }
  return rc;
}

// Random write: element at global index idx[i] = in[i], applied in order.
int orc_write(void* h, const uint64_t* idx, uint64_t n, const void* in) {
  OracleArray& a = *static_cast<OracleArray*>(h);
  std::vector<uint64_t> off = prefix_offsets(a);
  const unsigned char* src = static_cast<const unsigned char*>(in);
  int rc = ORC_OK;
  for (uint64_t i = 0; i < n; ++i) {
    uint32_t l;
    uint64_t j;
    if (!locate(off, idx[i], &l, &j)) {
      rc = ORC_ERR_OUT_OF_RANGE;
      continue;
    }
    std::memcpy(a.lfv[l].data() + j * a.E, src + i * a.E, a.E);
  }
  return rc;
}

// The r/w operation of Sec. VI-C: add delta to every element, repeats times
// (the paper adds +1 thirty times).  Elements are unsigned integers of E
// bytes with wrap-around; 16-byte records are not integers and are rejected.
int orc_sweep_add(void* h, uint64_t delta, uint32_t repeats) {
  OracleArray& a = *static_cast<OracleArray*>(h);
  if (a.E == 16) return ORC_ERR_INVALID;
  for (uint32_t l = 0; l < a.L; ++l) {
    uint64_t n = lfv_size(a, l);
    for (uint64_t j = 0; j < n; ++j) {
      unsigned char* p = a.lfv[l].data() + j * a.E;
      for (uint32_t rep = 0; rep < repeats; ++rep) {
        if (a.E == 4) {
          uint32_t w;
          std::memcpy(&w, p, 4);
          w += static_cast<uint32_t>(delta);
          std::memcpy(p, &w, 4);
        } else {
          uint64_t w;
          std::memcpy(&w, p, 8);
          w += delta;
          std::memcpy(p, &w, 8);
        }
      }
    }
  }
  return ORC_OK;
}

// Flatten: copy every element into one contiguous array in global order
// (LFVector 0's elements, then LFVector 1's, ...).  dst must hold capacity
// elements; fails with ORC_ERR_DST_TOO_SMALL when capacity < size.
int orc_flatten(void* h, void* dst, uint64_t capacity) {
  OracleArray& a = *static_cast<OracleArray*>(h);
  if (capacity < orc_size(h)) return ORC_ERR_DST_TOO_SMALL;
  unsigned char* out = static_cast<unsigned char*>(dst);
  for (uint32_t l = 0; l < a.L; ++l) {
    std::memcpy(out, a.lfv[l].data(), a.lfv[l].size());
    out += a.lfv[l].size();
  }
  return ORC_OK;
}

// Read LFVector l's elements (its local order) into out; returns its size.
uint64_t orc_lfvector(void* h, uint32_t l, void* out) {
  OracleArray& a = *static_cast<OracleArray*>(h);
  if (out) std::memcpy(out, a.lfv[l].data(), a.lfv[l].size());
  return lfv_size(a, l);
}

// Memory held by buckets: sum of capacities times E (Sec. V's "memory used").
uint64_t orc_bucket_bytes(void* h) {
  OracleArray& a = *static_cast<OracleArray*>(h);
  uint64_t bytes = 0;
  for (uint32_t l = 0; l < a.L; ++l) bytes += capacity_of(covered(a, l), a.B) * a.E;
  return bytes;
}

// ---------------------------------------------------------------------------
// Two-phase case study (Sec. VI-D): an insertion phase that grows the array
// from inside the kernel, then flatten, then regular passes over the static
// copy.  Records are 16 bytes {uint64 id, float pos, float vel}.

// Spawning generation `gen`: every parent record of LFVector l appends
// Geometric(1/2) - 1 children to the same LFVector (the push_back of
// Algorithm 1 called from inside the application kernel).  The count of the
// parent at LFVector-local index j is the trailing-ones count of
// splitmix_at(seed, (gen << 48) | g) with g = offsets[l] + j, the parent's
// global index when the generation starts.  Children are appended in parent
// order, a parent's children consecutively; a child copies its parent's pos
// and vel and gets id ((gen + 1) << 56) | (l << 40) | (its local index).
// Parents are all records present when the generation starts
// (only_newborn = 0), or only those appended by the previous generation
// (only_newborn = 1, born[l] holds where they start and is advanced).
int orc_spawn(void* h, uint32_t gen, uint64_t seed, int only_newborn, uint64_t* born) {
  OracleArray& a = *static_cast<OracleArray*>(h);
  if (a.E != 16) return ORC_ERR_INVALID;
  std::vector<uint64_t> off = prefix_offsets(a);
  for (uint32_t l = 0; l < a.L; ++l) {
    const uint64_t s = lfv_size(a, l);
    const uint64_t first = only_newborn ? born[l] : 0;
    for (uint64_t j = first; j < s; ++j) {
      const uint64_t key = (static_cast<uint64_t>(gen) << 48) | (off[l] + j);
      const uint32_t c = draw_count(2, splitmix_at(seed, key), nullptr, 0);
      unsigned char parent[16];
      std::memcpy(parent, a.lfv[l].data() + j * 16, 16);
      for (uint32_t k = 0; k < c; ++k) {
        const uint64_t local = lfv_size(a, l);
        const uint64_t id = (static_cast<uint64_t>(gen + 1) << 56) | (static_cast<uint64_t>(l) << 40) | local;
        std::memcpy(parent, &id, 8);
        a.lfv[l].insert(a.lfv[l].end(), parent, parent + 16);
      }
    }
    if (only_newborn) born[l] = s;
  }
  return ORC_OK;
}

// Work phase of the case study on the flattened records: pos += vel,
// `passes` times, one float addition each (Sec. VI-D's kernel "adds 1 to
// every element", here with a per-record increment).
void orc_work_passes(void* records, uint64_t n, uint32_t passes) {
  unsigned char* r = static_cast<unsigned char*>(records);
  for (uint32_t p = 0; p < passes; ++p) {
    for (uint64_t i = 0; i < n; ++i) {
      float pos, vel;
      std::memcpy(&pos, r + i * 16 + 8, 4);
      std::memcpy(&vel, r + i * 16 + 12, 4);
      pos = pos + vel;
      std::memcpy(r + i * 16 + 8, &pos, 4);
    }
  }
}

// The n-th draw of the counter-based generator and a count drawn from it,
// exposed so tests can compare this C implementation with other ones.
uint64_t orc_splitmix_at(uint64_t seed, uint64_t key) { return splitmix_at(seed, key); }

uint32_t orc_draw_count(uint32_t dist, uint64_t h, const uint32_t* thr, uint32_t nthr) {
  return draw_count(dist, h, thr, nthr);
}

}  // extern "C"
