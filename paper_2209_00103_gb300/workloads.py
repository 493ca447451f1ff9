"""Seeded synthetic inputs for the GGArray workloads.

This module only draws inputs: per-thread insertion counts, the values the
threads insert, and random indices.  It holds none of the GGArray's own
arithmetic (no bucket math, no reservation, no offsets) and imports neither
the CUDA binding nor the oracle, so tests can feed the same arrays to both.

All draws come from one counter-based generator, SplitMix64 (Steele, Lea and
Flood, OOPSLA 2014): draw ``n`` of the stream seeded with ``s`` is
``mix64(s + n * 0x9E3779B97F4A7C15)`` with the published finalizer.  The
counter ``n`` is ``key + 1`` where ``key`` packs what the draw belongs to,
e.g. ``(round << 32) | global_thread_id`` for insertion counts.

Workload shapes follow the paper's experiments: every block is one LFVector,
each of its threads inserts a few elements per round (Sec. III-B, Sec. VI-A),
values are self-describing integers so any misplaced element is visible.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
MASK64 = (1 << 64) - 1


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output finalizer on a uint64 array (wrap-around arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix_at(seed: int, keys) -> np.ndarray:
    """Draw number key+1 of the SplitMix64 stream seeded with ``seed``."""
    keys = np.asarray(keys, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(seed & MASK64) + (keys + np.uint64(1)) * GOLDEN
    return mix64(state)


def poisson1_thresholds(kmax: int = 12) -> np.ndarray:
    """floor(2^32 * CDF_Poisson(1)(k)) for k = 0..kmax-1, computed in double.

    A count is #{k : u32 >= thr[k]}, which is Poisson(1) truncated at kmax.
    """
    thr = []
    cdf = 0.0
    for k in range(kmax):
        cdf += math.exp(-1.0) / math.factorial(k)
        thr.append(min(int(math.floor(cdf * 2.0 ** 32)), 2 ** 32 - 1))
    return np.array(thr, dtype=np.uint32)


def draw_counts(dist: str, h: np.ndarray, thresholds: np.ndarray | None = None) -> np.ndarray:
    """Map 64-bit draws to insertion counts (uint32)."""
    h = np.asarray(h, dtype=np.uint64)
    if dist == "bernoulli":                          # Bernoulli(1/2): top bit
        return (h >> np.uint64(63)).astype(np.uint32)
    if dist == "uniform3":                           # Uniform{0,1,2}
        hi = h >> np.uint64(32)
        return ((hi * np.uint64(3)) >> np.uint64(32)).astype(np.uint32)
    if dist == "geometric":                          # Geometric(1/2) - 1 = trailing ones
        c = np.zeros(h.shape, dtype=np.uint32)
        x = h.copy()
        alive = np.ones(h.shape, dtype=bool)
        for _ in range(63):
            bit = (x & np.uint64(1)).astype(bool) & alive
            c += bit
            alive &= bit
            x >>= np.uint64(1)
            if not alive.any():
                break
        return c
    if dist == "poisson":                            # Poisson(1) by thresholds
        thr = poisson1_thresholds() if thresholds is None else thresholds
        u = (h >> np.uint64(32)).astype(np.uint64)
        c = np.zeros(h.shape, dtype=np.uint32)
        for t in thr:
            c += (u >= np.uint64(int(t))).astype(np.uint32)
        return c
    raise ValueError(dist)


def value_dtype(E: int) -> np.dtype:
    return {4: np.dtype(np.uint32), 8: np.dtype(np.uint64), 16: np.dtype((np.void, 16))}[E]


def encode_values(v: np.ndarray, E: int) -> np.ndarray:
    """Store uint64 self-describing values in E-byte elements.

    E=4 keeps the low 32 bits, E=8 all 64; E=16 builds the record
    {int64 key = v, float32 x = v & 0xFFFF, float32 y = (v >> 16) & 0xFFFF}.
    """
    v = np.asarray(v, dtype=np.uint64)
    if E == 4:
        return v.astype(np.uint32)
    if E == 8:
        return v.copy()
    rec = np.zeros(v.shape[0], dtype=[("key", "<u8"), ("x", "<f4"), ("y", "<f4")])
    rec["key"] = v
    rec["x"] = (v & np.uint64(0xFFFF)).astype(np.float32)
    rec["y"] = ((v >> np.uint64(16)) & np.uint64(0xFFFF)).astype(np.float32)
    return rec.view(np.dtype((np.void, 16))).reshape(-1)


@dataclass
class InsertSpec:
    """One batch of R insertion rounds of a GGArray of L blocks x T threads.

    Thread t of block l (gtid = gtid0 + l*T + t) draws its count for round r
    from ``splitmix_at(seed, (r << 32) | gtid)`` and inserts values
    ``va*gtid + vb*r + vc*k`` for k < count.  gtid0 = l0*T gives the inputs
    of blocks l0, l0+1, ... of a larger array exactly as that array's own
    spec would draw them.
    """
    L: int
    T: int
    E: int
    seed: int
    dist: str
    rounds: int
    round0: int = 0
    coeffs: tuple = (1, 0, 0)
    thresholds: np.ndarray | None = field(default=None, repr=False)
    gtid0: int = 0

    def counts(self) -> np.ndarray:
        """uint32 counts, shape [R][L][T]."""
        r = np.arange(self.round0, self.round0 + self.rounds, dtype=np.uint64)
        gtid = np.uint64(self.gtid0) + np.arange(self.L * self.T, dtype=np.uint64)
        keys = (r[:, None] << np.uint64(32)) | gtid[None, :]
        h = splitmix_at(self.seed, keys)
        c = draw_counts(self.dist, h, self.thresholds)
        return c.reshape(self.rounds, self.L, self.T)

    def values(self, counts: np.ndarray) -> np.ndarray:
        """Packed values in (round, block, thread, k) order, E bytes each."""
        R = counts.shape[0]
        flat = counts.reshape(-1).astype(np.int64)
        n = int(flat.sum())
        gtid = np.tile(np.uint64(self.gtid0) + np.arange(self.L * self.T, dtype=np.uint64), R)
        rnd = np.repeat(np.arange(self.round0, self.round0 + R, dtype=np.uint64), self.L * self.T)
        g_rep = np.repeat(gtid, flat)
        r_rep = np.repeat(rnd, flat)
        # k = position of an element within its thread's run.
        starts = np.repeat(np.cumsum(flat) - flat, flat)
        k = (np.arange(n, dtype=np.int64) - starts).astype(np.uint64)
        va, vb, vc = (np.uint64(int(c) & MASK64) for c in self.coeffs)
        with np.errstate(over="ignore"):
            v = va * g_rep + vb * r_rep + vc * k
        return encode_values(v, self.E)

    def make(self):
        c = self.counts()
        return c, self.values(c)


def expand_inputs(spec: "InsertSpec") -> np.ndarray:
    """Per-(round, block, thread) inputs [R][L][T] of the memory-sourced
    pushes: the value va*gtid + vb*r, E bytes each.  With spec.coeffs[2] = 0
    the spec's packed values are these inputs repeated count times."""
    r = np.arange(spec.round0, spec.round0 + spec.rounds, dtype=np.uint64)
    gtid = np.uint64(spec.gtid0) + np.arange(spec.L * spec.T, dtype=np.uint64)
    va, vb = (np.uint64(int(c) & MASK64) for c in spec.coeffs[:2])
    with np.errstate(over="ignore"):
        v = (va * gtid[None, :] + vb * r[:, None]).reshape(-1)
    return encode_values(v, spec.E)


def uniform_indices(seed: int, n: int, size: int) -> np.ndarray:
    """n indices uniform over [0, size) (size < 2^32): floor(u32 * size / 2^32)."""
    assert 0 < size < (1 << 32)
    h = splitmix_at(seed, np.arange(n, dtype=np.uint64))
    return ((h >> np.uint64(32)) * np.uint64(size)) >> np.uint64(32)


def index_keyed_values(seed: int, idx: np.ndarray, E: int) -> np.ndarray:
    """Values that depend only on the index written, so duplicate indices in a
    random write batch all carry the same value."""
    return encode_values(splitmix_at(seed, idx), E)


# ---------------------------------------------------------------------------
# The workloads.

@dataclass
class GrowthWorkload:
    """A GGArray grown from empty by R rounds of per-thread insertions, then
    read at random, written at random, swept and flattened."""
    name: str
    L: int
    T: int
    B: int
    E: int
    spec: InsertSpec
    n_random: int
    read_seed: int
    write_seed: int
    value_seed: int
    sweep_delta: int = 1
    sweep_repeats: int = 1


def tiny_bernoulli() -> GrowthWorkload:
    """32 blocks x 256 threads, first bucket 1024 int32, 10 rounds of
    Bernoulli(1/2) insertions with value gtid*10 + round (about 41k elements)."""
    spec = InsertSpec(L=32, T=256, E=4, seed=1, dist="bernoulli", rounds=10, coeffs=(10, 1, 0))
    return GrowthWorkload("tiny_bernoulli_32x256_B1024_int32", 32, 256, 1024, 4, spec,
                          n_random=4096, read_seed=101, write_seed=102, value_seed=103)


def paper_growth() -> GrowthWorkload:
    """1024 blocks x 512 threads, first bucket 4096 int32, 512 rounds of
    Uniform{0,1,2} insertions (about 2^28 elements, 1 GiB), value
    ((round*2 + k) << 19) | gtid; then 2^26 random reads and writes."""
    spec = InsertSpec(L=1024, T=512, E=4, seed=2, dist="uniform3", rounds=512,
                      coeffs=(1, 1 << 20, 1 << 19))
    return GrowthWorkload("paper_growth_1024x512_B4096_int32_2^28", 1024, 512, 4096, 4, spec,
                          n_random=1 << 26, read_seed=201, write_seed=202, value_seed=203)


def scaled_growth(rounds: int, L: int = 1024, T: int = 512, B: int = 4096) -> GrowthWorkload:
    """The paper-shaped growth workload with fewer rounds (same seed, same
    per-round draws), for tests and CPU samples."""
    spec = InsertSpec(L=L, T=T, E=4, seed=2, dist="uniform3", rounds=rounds,
                      coeffs=(1, 1 << 20, 1 << 19))
    return GrowthWorkload(f"paper_growth_{L}x{T}_B{B}_int32_R{rounds}", L, T, B, 4, spec,
                          n_random=min(1 << 26, L * T * rounds // 4 + 1),
                          read_seed=201, write_seed=202, value_seed=203)


# ---------------------------------------------------------------------------
# The same generator on torch tensors (any device), so full-size inputs can be
# drawn directly in device memory.  Bit patterns are carried in int64 tensors
# with wrap-around arithmetic; right shifts are made logical by masking.

def _s64(u: int) -> int:
    u &= MASK64
    return u - (1 << 64) if u >= (1 << 63) else u


def _lsr(x, s: int):
    return (x >> s) & ((1 << (64 - s)) - 1)


def mix64_t(z):
    z = (z ^ _lsr(z, 30)) * _s64(0xBF58476D1CE4E5B9)
    z = (z ^ _lsr(z, 27)) * _s64(0x94D049BB133111EB)
    return z ^ _lsr(z, 31)


def splitmix_at_t(seed: int, keys):
    """Torch twin of splitmix_at: keys int64 tensor -> int64 tensor of draws."""
    return mix64_t(_s64(seed) + (keys + 1) * _s64(int(GOLDEN)))


def draw_counts_t(dist: str, h, thresholds: np.ndarray | None = None):
    import torch
    hi = _lsr(h, 32)
    if dist == "bernoulli":
        c = _lsr(h, 63)
    elif dist == "uniform3":
        c = _lsr(hi * 3, 32)
    elif dist == "geometric":
        c = torch.zeros_like(h)
        alive = torch.ones_like(h, dtype=torch.bool)
        for s in range(63):
            bit = (_lsr(h, s) & 1).bool() & alive
            c += bit.to(h.dtype)
            alive &= bit
    elif dist == "poisson":
        thr = poisson1_thresholds() if thresholds is None else thresholds
        c = torch.zeros_like(h)
        for t in thr:
            c += (hi >= int(t)).to(h.dtype)
    else:
        raise ValueError(dist)
    return c.to(torch.int32)


def encode_values_t(v, E: int):
    """Torch twin of encode_values: int32 [n], int64 [n] or int64 [n, 2]."""
    import torch
    if E == 4:
        return (((v + (1 << 31)) & 0xFFFFFFFF) - (1 << 31)).to(torch.int32)
    if E == 8:
        return v.clone()
    x = (v & 0xFFFF).to(torch.float32).view(torch.int32).to(torch.int64) & 0xFFFFFFFF
    y = (_lsr(v, 16) & 0xFFFF).to(torch.float32).view(torch.int32).to(torch.int64) & 0xFFFFFFFF
    return torch.stack([v, x | (y << 32)], dim=1)


def make_insert_inputs_t(spec: "InsertSpec", device):
    """(counts int32 [R][L][T], packed values) for spec, drawn on `device`."""
    import torch
    R, LT = spec.rounds, spec.L * spec.T
    r = torch.arange(spec.round0, spec.round0 + R, dtype=torch.int64, device=device)
    gtid = torch.arange(LT, dtype=torch.int64, device=device)
    keys = (r[:, None] << 32) | gtid[None, :]
    counts = draw_counts_t(spec.dist, splitmix_at_t(spec.seed, keys), spec.thresholds)
    flat = counts.reshape(-1).to(torch.int64)
    n = int(flat.sum().item())
    g_rep = torch.repeat_interleave(gtid.repeat(R), flat, output_size=n)
    r_rep = torch.repeat_interleave(r.repeat_interleave(LT), flat, output_size=n)
    starts = torch.repeat_interleave(torch.cumsum(flat, 0) - flat, flat, output_size=n)
    k = torch.arange(n, dtype=torch.int64, device=device) - starts
    va, vb, vc = (_s64(int(c)) for c in spec.coeffs)
    v = va * g_rep + vb * r_rep + vc * k
    return counts.reshape(R, spec.L, spec.T), encode_values_t(v, spec.E)


def expand_inputs_t(spec: "InsertSpec", device):
    """expand_inputs on `device`: [R][L][T] elements (int32 / int64, or
    int64 pairs for 16-byte records)."""
    import torch
    r = torch.arange(spec.round0, spec.round0 + spec.rounds, dtype=torch.int64, device=device)
    gtid = torch.arange(spec.L * spec.T, dtype=torch.int64, device=device)
    va, vb = (_s64(int(c)) for c in spec.coeffs[:2])
    v = (va * gtid[None, :] + vb * r[:, None]).reshape(-1)
    e = encode_values_t(v, spec.E)
    return e.reshape((spec.rounds, spec.L, spec.T) + tuple(e.shape[1:]))


def uniform_indices_t(seed: int, n: int, size: int, device):
    import torch
    assert 0 < size < (1 << 32)
    h = splitmix_at_t(seed, torch.arange(n, dtype=torch.int64, device=device))
    return _lsr(_lsr(h, 32) * size, 32)


def index_keyed_values_t(seed: int, idx, E: int):
    return encode_values_t(splitmix_at_t(seed, idx), E)


# ---------------------------------------------------------------------------
# Two-phase case study (Sec. VI-D): initial 16-byte records, spawned
# generations, then flatten and streaming passes.

RECORD_DTYPE = np.dtype([("id", "<u8"), ("pos", "<f4"), ("vel", "<f4")])


def initial_records(n0: int) -> np.ndarray:
    """Record i = {id i, pos (i & 1023), vel ((7 i) & 15) / 16}: dyadic values,
    so 20 additions of vel stay exact in float32."""
    i = np.arange(n0, dtype=np.uint64)
    r = np.zeros(n0, dtype=RECORD_DTYPE)
    r["id"] = i
    r["pos"] = (i & np.uint64(1023)).astype(np.float32)
    r["vel"] = ((i * np.uint64(7)) & np.uint64(15)).astype(np.float32) / np.float32(16)
    return r


def initial_records_t(n0: int, device):
    """Torch twin of initial_records as int64 [n0, 2] (id, pos|vel bits)."""
    import torch
    i = torch.arange(n0, dtype=torch.int64, device=device)
    pos = (i & 1023).to(torch.float32).view(torch.int32).to(torch.int64) & 0xFFFFFFFF
    vel = (((i * 7) & 15).to(torch.float32) / 16).view(torch.int32).to(torch.int64) & 0xFFFFFFFF
    return torch.stack([i, pos | (vel << 32)], dim=1)


def split_counts(L: int, T: int, n0: int) -> np.ndarray:
    """One insertion round placing records [l*n0/L, (l+1)*n0/L) in LFVector l,
    spread over its T threads as evenly as possible: counts [1][L][T]."""
    per_l = np.diff((np.arange(L + 1, dtype=np.int64) * n0) // L)
    c = np.zeros((1, L, T), dtype=np.uint32)
    t = np.arange(T + 1, dtype=np.int64)
    for l in range(L):
        c[0, l] = np.diff((t * int(per_l[l])) // T)
    return c


@dataclass
class TwoPhaseWorkload:
    name: str
    L: int
    T: int
    B: int
    n0: int
    generations: int
    seed: int
    passes: int
    only_newborn: bool


def two_phase(only_newborn: bool = False, n0: int = 1 << 24, generations: int = 8) -> TwoPhaseWorkload:
    """2^24 initial records over 1024 LFVectors x 512 threads, 8 generations
    of Geometric(1/2)-1 children per record (mean 1), then flatten and 20
    passes of pos += vel.  only_newborn=False: every record present spawns
    (the population about doubles per generation); True: only the previous
    generation's children spawn."""
    tag = "newborn" if only_newborn else "all"
    return TwoPhaseWorkload(f"two_phase_{tag}_1024x512_B4096_n{n0}_g{generations}", 1024, 512, 4096, n0,
                            generations, 5, 20, only_newborn)
