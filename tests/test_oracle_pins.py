"""Pins for the GGArray oracle: it is checked against facts fixed by the paper
and by mathematics, never against itself.

* closed forms of the bucket layout of Algorithm 2 (first/last slot of each
  bucket, capacity after lazy allocation, capacity <= 2*size + B);
* brute force over tiny inputs against a second, independent model (a global
  list of tagged elements sorted by (block, round, thread, k), which is what
  the prefix-sum insertion of Sec. III-B and the LFVector-major global order
  of Sec. IV define);
* a one-LFVector GGArray behaves exactly like a plain list with appends;
* the self-describing values of the tiny workload decode to their inserting
  thread and round, grouped by block and sorted by (round, thread);
* published SplitMix64 outputs for the generator feeding both sides.
"""

import itertools
import os

import numpy as np
import pytest

import oracle
from paper_2209_00103_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Algorithm 2 bucket layout: bucket b holds B * 2^b elements.

@pytest.mark.parametrize("B", [1, 2, 4, 8, 1024, 4096, 1 << 16])
def test_bucket_first_and_last_slot(B):
    # Slots of buckets 0..b-1 number B + 2B + ... + 2^(b-1) B = B (2^b - 1).
    for b in range(0, 30):
        first = B * ((1 << b) - 1)
        last = first + B * (1 << b) - 1
        assert oracle.bucket_of(first, B) == (b, 0)
        assert oracle.bucket_of(last, B) == (b, B * (1 << b) - 1)


@pytest.mark.parametrize("B", [1, 2, 4, 16])
def test_bucket_walk_is_lexicographic_bijection(B):
    # Consecutive indices visit (bucket, offset) in order, each bucket filled
    # to exactly B * 2^b slots before the next one starts.
    b, off = 0, 0
    for j in range(1 << 13):
        assert oracle.bucket_of(j, B) == (b, off)
        off += 1
        if off == B << b:
            b, off = b + 1, 0


@pytest.mark.parametrize("B", [1, 4, 1024, 4096])
def test_capacity_closed_form(B):
    assert oracle.capacity_of(0, B) == 0              # lazy: nothing allocated
    assert oracle.capacity_of(1, B) == B              # bucket 0
    assert oracle.capacity_of(B, B) == B
    assert oracle.capacity_of(B + 1, B) == 3 * B      # buckets 0, 1
    assert oracle.capacity_of(3 * B, B) == 3 * B
    assert oracle.capacity_of(3 * B + 1, B) == 7 * B  # buckets 0, 1, 2
    rng = np.random.default_rng(5)
    for s in rng.integers(1, 1 << 40, size=2000):
        s = int(s)
        cap = oracle.capacity_of(s, B)
        assert s <= cap <= 2 * s + B                   # capacity bound
        k = (cap // B + 1).bit_length() - 1            # cap = B(2^k - 1)
        assert cap == B * ((1 << k) - 1)
        assert B * ((1 << (k - 1)) - 1) < s            # least such k


def test_paper_growth_memory_ratio_at_scale():
    # With ~2^18 elements per LFVector and B = 4096, six buckets hold
    # 4096*63 = 258048 < 2^18, so seven are needed: 520192 / 262144 ~ 1.98.
    cap = oracle.capacity_of(1 << 18, 4096)
    assert cap == 4096 * 127
    assert cap / (1 << 18) < 2.0


# --------------------------------------------------------------------------
# Brute force against an independent model.

def naive_model(counts, values):
    """Tag each packed value with (block, round, thread, k) and sort: the
    LFVector-major global order, rounds in sequence, threads by prefix sum."""
    R, L, T = counts.shape
    tagged = []
    i = 0
    for r in range(R):
        for l in range(L):
            for t in range(T):
                for k in range(int(counts[r, l, t])):
                    tagged.append(((l, r, t, k), values[i]))
                    i += 1
    tagged.sort(key=lambda x: x[0])
    flat = np.array([v for _, v in tagged], dtype=values.dtype)
    sizes = counts.sum(axis=(0, 2)).astype(np.uint64)
    return flat, sizes


def check_against_naive(L, T, B, counts, E=4):
    n = int(counts.sum())
    values = (np.arange(n, dtype=np.uint64) * 7919 + 13).astype(np.uint32 if E == 4 else np.uint64)
    a = oracle.OracleGGArray(L, T, B, E)
    a.insert(counts, values)
    flat, sizes = naive_model(counts, values)
    got = a.flatten()
    assert np.array_equal(got, flat)
    assert np.array_equal(a.sizes(), sizes)
    assert a.size() == n
    off = a.offsets()
    assert off[0] == 0 and np.array_equal(np.diff(off.astype(np.int64)), sizes.astype(np.int64))
    caps, nb = a.capacities()
    for l in range(L):
        s = int(sizes[l])
        assert int(caps[l]) == (0 if s == 0 else B * ((1 << int(nb[l])) - 1))
        assert s <= int(caps[l]) <= 2 * s + B
    if n:
        out, rc = a.read(np.arange(n, dtype=np.uint64))
        assert rc == oracle.OK and np.array_equal(out, flat)
    out, rc = a.read(np.array([n], dtype=np.uint64))
    assert rc == oracle.ERR_OUT_OF_RANGE
    a.close()


def test_brute_force_all_small_count_tensors():
    # Every count tensor with L*T*R <= 6 entries in {0,1,2}.
    shapes = [(1, 1, 1), (1, 2, 1), (2, 1, 1), (1, 2, 2), (2, 1, 2), (2, 2, 1),
              (1, 3, 2), (2, 3, 1), (1, 1, 3), (1, 2, 3), (2, 1, 3), (3, 2, 1)]
    n_cases = 0
    for (L, T, R) in shapes:
        for B in (1, 2, 4):
            for cs in itertools.product(range(3), repeat=L * T * R):
                counts = np.array(cs, dtype=np.uint32).reshape(R, L, T)
                check_against_naive(L, T, B, counts)
                n_cases += 1
    assert n_cases > 10000


def test_brute_force_random_small():
    rng = np.random.default_rng(11)
    for _ in range(300):
        L = int(rng.integers(1, 4))
        T = int(rng.integers(1, 5))
        R = int(rng.integers(1, 4))
        B = int(rng.choice([1, 2, 4]))
        E = int(rng.choice([4, 8]))
        counts = rng.integers(0, 3, size=(R, L, T)).astype(np.uint32)
        check_against_naive(L, T, B, counts, E)


def test_rounds_split_equals_batched():
    # Inserting R rounds in one call or round by round gives the same array,
    # and the per-round size series is the running sum of block totals.
    rng = np.random.default_rng(3)
    L, T, R, B = 5, 7, 6, 2
    counts = rng.integers(0, 3, size=(R, L, T)).astype(np.uint32)
    n = int(counts.sum())
    values = np.arange(n, dtype=np.uint32)
    a = oracle.OracleGGArray(L, T, B, 4)
    spr = a.insert(counts, values, per_round=True)
    b = oracle.OracleGGArray(L, T, B, 4)
    pos = 0
    for r in range(R):
        m = int(counts[r].sum())
        b.insert(counts[r:r + 1], values[pos:pos + m])
        pos += m
        assert np.array_equal(b.sizes(), spr[r])
    assert np.array_equal(a.flatten(), b.flatten())
    assert np.array_equal(spr[-1], counts.sum(axis=(0, 2)))
    assert np.array_equal(spr, np.cumsum(counts.sum(axis=2), axis=0))


def test_single_lfvector_is_a_list():
    # L = 1: the GGArray is one LFVector, so its content is plain append order.
    rng = np.random.default_rng(7)
    T, R = 9, 20
    counts = rng.integers(0, 4, size=(R, 1, T)).astype(np.uint32)
    plain = []
    v = 1000
    vals = []
    for r in range(R):
        for t in range(T):
            for _ in range(int(counts[r, 0, t])):
                plain.append(v)
                vals.append(v)
                v += 3
    a = oracle.OracleGGArray(1, T, 4, 4)
    a.insert(counts, np.array(vals, dtype=np.uint32))
    assert a.flatten().tolist() == plain
    assert a.lfvector(0).tolist() == plain


def test_insert_rejects_wrong_value_count():
    a = oracle.OracleGGArray(2, 2, 1, 4)
    counts = np.ones((1, 2, 2), dtype=np.uint32)
    with pytest.raises(oracle.OracleError):
        a.insert(counts, np.zeros(3, dtype=np.uint32))
    assert a.size() == 0


def test_create_rejects_invalid_params():
    for args in [(0, 1, 1, 4), (1, 0, 1, 4), (1, 1, 3, 4), (1, 1, 0, 4), (1, 1, 4, 2), (1, 1, 4, 12)]:
        with pytest.raises(oracle.OracleError):
            oracle.OracleGGArray(*args)


# --------------------------------------------------------------------------
# Reads, writes, the +1 r/w operation, flatten.

def test_read_write_and_sweep():
    rng = np.random.default_rng(9)
    L, T, R, B = 4, 8, 5, 2
    counts = rng.integers(0, 3, size=(R, L, T)).astype(np.uint32)
    counts[:, 2, :] = 0                        # an empty LFVector in the middle
    n = int(counts.sum())
    values = np.arange(n, dtype=np.uint32) + 5
    a = oracle.OracleGGArray(L, T, B, 4)
    a.insert(counts, values)
    flat = a.flatten().copy()
    # Writes in order: the later write to an index wins.
    idx = np.array([0, n - 1, 3, 3], dtype=np.uint64)
    vals = np.array([11, 22, 33, 44], dtype=np.uint32)
    assert a.write(idx, vals) == oracle.OK
    flat[0], flat[n - 1], flat[3] = 11, 22, 44
    assert np.array_equal(a.flatten(), flat)
    out, rc = a.read(np.array([3, 0, n - 1], dtype=np.uint64))
    assert rc == oracle.OK and out.tolist() == [44, 11, 22]
    # Out-of-range indices are reported; in-range ones still apply.
    assert a.write(np.array([n, 1], dtype=np.uint64), np.array([9, 77], dtype=np.uint32)) == oracle.ERR_OUT_OF_RANGE
    flat[1] = 77
    assert np.array_equal(a.flatten(), flat)
    # Sec. VI-C's r/w kernel: +1 thirty times, with uint32 wrap-around.
    a.write(np.array([2], dtype=np.uint64), np.array([0xFFFFFFF0], dtype=np.uint32))
    flat[2] = 0xFFFFFFF0
    a.sweep_add(1, 30)
    assert np.array_equal(a.flatten(), (flat.astype(np.uint64) + 30).astype(np.uint32))
    assert a.flatten()[2] == (0xFFFFFFF0 + 30) - (1 << 32)
    with pytest.raises(oracle.OracleError):
        a.flatten(capacity=n - 1)


def test_sweep_rejects_records():
    a = oracle.OracleGGArray(1, 1, 1, 16)
    with pytest.raises(oracle.OracleError):
        a.sweep_add(1, 1)


# --------------------------------------------------------------------------
# The counter-based generator.

def test_splitmix_published_outputs():
    want = [int(line, 16) for line in open(os.path.join(GOLDEN, "splitmix64_seed0.txt"))
            if line.startswith("0x")]
    got_np = [int(x) for x in wl.splitmix_at(0, np.arange(5, dtype=np.uint64))]
    got_c = [oracle.splitmix_at(0, k) for k in range(5)]
    assert got_np == want
    assert got_c == want


def test_count_draws_distribution_and_agreement():
    h = wl.splitmix_at(12345, np.arange(1 << 16, dtype=np.uint64))
    thr = wl.poisson1_thresholds()
    for dist, mean, p0 in [("bernoulli", 0.5, 0.5), ("uniform3", 1.0, 1 / 3),
                           ("geometric", 1.0, 0.5), ("poisson", 1.0, np.exp(-1))]:
        c = wl.draw_counts(dist, h, thr)
        assert abs(c.mean() - mean) < 0.02, dist
        assert abs((c == 0).mean() - p0) < 0.01, dist
        # C implementation agrees draw by draw.
        c_c = np.array([oracle.draw_count(dist, int(x), thr) for x in h[:2000]])
        assert np.array_equal(c_c, c[:2000]), dist
    u3 = wl.draw_counts("uniform3", h)
    assert set(np.unique(u3).tolist()) == {0, 1, 2}
    assert all(abs((u3 == v).mean() - 1 / 3) < 0.01 for v in range(3))


@pytest.mark.parametrize("E", [4, 8, 16])
def test_generated_insert_matches_packed_insert(E):
    # The oracle's in-thread draws and the numpy input generator are two
    # independent implementations of the same generator.
    for dist in ["bernoulli", "uniform3", "geometric", "poisson"]:
        spec = wl.InsertSpec(L=3, T=33, E=E, seed=77, dist=dist, rounds=4, round0=2,
                             coeffs=(10, 1 << 20, 1 << 19), thresholds=wl.poisson1_thresholds())
        counts, values = spec.make()
        a = oracle.OracleGGArray(3, 33, 4, E)
        a.insert(counts, values)
        b = oracle.OracleGGArray(3, 33, 4, E)
        cb = b.insert_generated(77, dist, spec.coeffs, 2, 4, thresholds=spec.thresholds,
                                return_counts=True)
        assert np.array_equal(cb, counts)
        assert a.flatten().tobytes() == b.flatten().tobytes()


def test_tiny_workload_self_describing_values():
    w = wl.tiny_bernoulli()
    counts, values = w.spec.make()
    a = oracle.OracleGGArray(w.L, w.T, w.B, w.E)
    a.insert(counts, values)
    flat = a.flatten().astype(np.int64)
    assert a.size() == int(counts.sum())
    assert 38000 < a.size() < 44000                       # ~ 32*256*10/2 = 40960
    gtid, rnd = flat // 10, flat % 10
    block = gtid // w.T
    tid = gtid % w.T
    # Grouped by block (LFVector-major global order) ...
    assert np.all(np.diff(block) >= 0)
    # ... and within a block sorted by (round, thread id) (prefix-sum order).
    key = block * 100000 + rnd * 1000 + tid
    assert np.all(np.diff(key) > 0)
    # The multiset of (gtid, round) is exactly the Bernoulli draws.
    want = np.argwhere(counts.reshape(10, -1) == 1)       # (round, gtid)
    got = np.stack([rnd, gtid], axis=1)
    assert np.array_equal(np.sort(want[:, 0] * 100000 + want[:, 1]),
                          np.sort(got[:, 0] * 100000 + got[:, 1]))
    # One +1 read-modify-write pass.
    a.sweep_add(1, 1)
    assert np.array_equal(a.flatten().astype(np.int64), flat + 1)
    # Offsets are block boundaries of the flattened sequence.
    off = a.offsets().astype(np.int64)
    for l in range(w.L):
        seg = gtid[off[l]:off[l + 1]] // w.T
        assert np.all(seg == l)


# --------------------------------------------------------------------------
# Two-phase case study: spawning generations against an independent numpy
# model (np.repeat of parents by their drawn counts), and the work phase
# against its closed form.

def spawn_model(lfvs, gen, seed, only_newborn, born):
    sizes = np.array([len(x) for x in lfvs], dtype=np.uint64)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    out = []
    for l, rec in enumerate(lfvs):
        s = len(rec)
        first = int(born[l]) if only_newborn else 0
        j = np.arange(first, s, dtype=np.uint64)
        keys = (np.uint64(gen) << np.uint64(48)) | (off[l] + j)
        c = wl.draw_counts("geometric", wl.splitmix_at(seed, keys))
        kids = np.repeat(rec[first:s], c.astype(np.int64))
        local = np.uint64(s) + np.arange(len(kids), dtype=np.uint64)
        kids["id"] = (np.uint64(gen + 1) << np.uint64(56)) | (np.uint64(l) << np.uint64(40)) | local
        out.append(np.concatenate([rec, kids]))
        if only_newborn:
            born[l] = s
    return out


@pytest.mark.parametrize("only_newborn", [False, True])
def test_spawn_matches_repeat_model(only_newborn):
    L, T, B, n0 = 5, 8, 4, 300
    counts = wl.split_counts(L, T, n0)
    recs = wl.initial_records(n0)
    a = oracle.OracleGGArray(L, T, B, 16)
    a.insert(counts, recs.view(np.dtype((np.void, 16))))
    per_l = counts.sum(axis=2)[0]
    bounds = np.concatenate([[0], np.cumsum(per_l)]).astype(np.int64)
    lfvs = [recs[bounds[l]:bounds[l + 1]].copy() for l in range(L)]
    born_o = np.zeros(L, dtype=np.uint64)
    born_m = np.zeros(L, dtype=np.uint64)
    for gen in range(5):
        a.spawn(gen, 5, only_newborn, born_o)
        lfvs = spawn_model(lfvs, gen, 5, only_newborn, born_m)
        assert np.array_equal(born_o, born_m)
        for l in range(L):
            assert a.lfvector(l).tobytes() == lfvs[l].tobytes(), (gen, l)
    # Children carry their parents' pos/vel and self-describing ids.
    flat = a.flatten().view(wl.RECORD_DTYPE)
    gen_of = (flat["id"] >> np.uint64(56)).astype(np.int64)
    assert gen_of.max() >= 3
    kids = flat[gen_of > 0]
    loc = kids["id"] & np.uint64((1 << 40) - 1)
    lv = (kids["id"] >> np.uint64(40)) & np.uint64(0xFFFF)
    off = a.offsets()
    glob = off[lv.astype(np.int64)] + loc
    assert np.array_equal(np.sort(glob), np.nonzero(gen_of > 0)[0].astype(np.uint64))


def test_work_passes_closed_form():
    r = wl.initial_records(5000)
    want = r["pos"].astype(np.float64) + 20 * r["vel"].astype(np.float64)
    got = oracle.work_passes(r.view(np.dtype((np.void, 16))).copy(), 20).view(wl.RECORD_DTYPE)
    assert np.array_equal(got["pos"].astype(np.float64), want)      # dyadic: exact
    assert np.array_equal(got["vel"], r["vel"]) and np.array_equal(got["id"], r["id"])


def test_split_counts_and_initial_records():
    c = wl.split_counts(7, 5, 1000)
    assert c.sum() == 1000
    per_l = c.sum(axis=2)[0]
    assert per_l.max() - per_l.min() <= 1
    r = wl.initial_records(2048)
    assert r["pos"][1024] == 0 and r["pos"][1023] == 1023
    assert r["vel"][1] == 7 / 16 and r["vel"][3] == 5 / 16


# --------------------------------------------------------------------------
# Growth to a target (batched arrays): sizes are the targets split over the
# LFVectors, and each LFVector is the prefix of the unclipped sequence the
# same draws produce (clipping by the scan = truncation in insertion order).

@pytest.mark.parametrize("dist", ["bernoulli", "uniform3", "geometric", "poisson"])
@pytest.mark.parametrize("E", [4, 8, 16])
def test_grow_to_target_is_a_truncated_generation(dist, E):
    L, T, B = 5, 24, 4
    thr = wl.poisson1_thresholds()
    coeffs = (0x10001, 0x9E3779B9, 7)
    for target in [0, 1, 4, 37, 1000, 4099]:
        a = oracle.OracleGGArray(L, T, B, E)
        a.grow_to_target(11, dist, coeffs, target, round0=3, thresholds=thr)
        per = [target // L + (1 if l < target % L else 0) for l in range(L)]
        assert a.sizes().tolist() == per
        full = oracle.OracleGGArray(L, T, B, E)
        full.insert_generated(11, dist, coeffs, 3, 600, thresholds=thr)
        for l in range(L):
            assert a.lfvector(l).tobytes() == full.lfvector(l)[:per[l]].tobytes()


# --------------------------------------------------------------------------
# Served appends and random reads.

def test_served_append_values_decode():
    L, T, B = 4, 8, 16
    a = oracle.OracleGGArray(L, T, B, 8)
    plan = [(10, 7), (1, 8), (0, 9), (1003, 10)]
    for n, tag in plan:
        a.append(n, tag)
    want_sizes = np.zeros(L, dtype=np.uint64)
    for n, _ in plan:
        want_sizes += np.array([n // L + (1 if l < n % L else 0) for l in range(L)], dtype=np.uint64)
    assert np.array_equal(a.sizes(), want_sizes)
    for l in range(L):
        v = a.lfvector(l).astype(np.uint64)
        tag, ll, k = v >> np.uint64(24), (v >> np.uint64(20)) & np.uint64(15), v & np.uint64((1 << 20) - 1)
        assert np.all(ll == l)
        # appended in request order, each request's share in k order
        exp = np.concatenate([np.stack([np.full(c, t, dtype=np.uint64), np.arange(c, dtype=np.uint64)], 1)
                              for n, t in plan for c in [n // L + (1 if l < n % L else 0)]])
        assert np.array_equal(np.stack([tag, k], 1), exp)


def test_served_random_read_matches_uniform_indices():
    L, T, B = 3, 8, 16
    a = oracle.OracleGGArray(L, T, B, 8)
    assert not a.read_random(5, 1).any()                      # empty array reads zeros
    a.append(10007, 3)
    flat = a.flatten()
    got = a.read_random(4096, 99)
    idx = wl.uniform_indices(99, 4096, a.size())
    assert np.array_equal(got, flat[idx.astype(np.int64)])


def _cap_closed_form(x: int, B: int) -> int:
    # least B(2^k - 1) >= x, by logarithm rather than by walking the buckets
    if x == 0:
        return 0
    k = int(np.ceil(np.log2(x / B + 1)))
    while B * ((1 << k) - 1) < x:       # guard the float rounding at the edges
        k += 1
    while k > 0 and B * ((1 << (k - 1)) - 1) >= x:
        k -= 1
    return B * ((1 << k) - 1)


@pytest.mark.parametrize("B", [1, 4, 256])
def test_reserve_capacity_and_contents(B):
    rng = np.random.default_rng(41 + B)
    L, T, E = 6, 8, 4
    o = oracle.OracleGGArray(L, T, B, E)
    counts = rng.integers(0, 3, size=(3, L, T)).astype(np.uint32)
    vals = (np.arange(int(counts.sum()), dtype=np.uint32) * 7 + 1)
    o.insert(counts, vals)
    sizes = o.sizes().astype(np.int64)
    before = o.flatten().copy()
    target = rng.integers(0, 5000, size=L).astype(np.uint64)
    target[0] = 0
    assert o.reserve(target) == oracle.OK
    caps, nb = o.capacities()
    for l in range(L):
        want = _cap_closed_form(max(int(sizes[l]), int(target[l])), B)
        assert int(caps[l]) == want
        assert int(caps[l]) >= int(target[l])
        assert int(caps[l]) == B * ((1 << int(nb[l])) - 1)
    assert o.flatten().tobytes() == before.tobytes()           # a resize moves nothing
    assert np.array_equal(o.sizes().astype(np.int64), sizes)
    assert o.bucket_bytes() == int(caps.sum()) * E
    # A smaller request changes nothing; an insertion past the reservation grows as usual.
    assert o.reserve(target // np.uint64(2)) == oracle.OK
    assert np.array_equal(o.capacities()[0], caps)
    big = np.zeros((1, L, T), dtype=np.uint32)
    big[0, 1, :] = 3000
    o.insert(big, np.zeros(int(big.sum()), dtype=np.uint32))
    caps2, _ = o.capacities()
    assert int(caps2[1]) == _cap_closed_form(max(int(sizes[1]) + 3000 * T, int(target[1])), B)
