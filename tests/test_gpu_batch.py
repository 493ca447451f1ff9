"""Batched growth: many arrays of uneven size, different T, B, E and count
distributions, grown to their targets in one persistent launch (also
captured in a CUDA graph and replayed) -- each array bit for bit against
the oracle."""

import numpy as np
import pytest
import torch

import oracle
from paper_2209_00103_gb300 import batching, gga
from paper_2209_00103_gb300 import workloads as wl

import oracle_pool
from harness import assert_same_state, dev_to_np

pytestmark = pytest.mark.gpu

DISTS = ["bernoulli", "uniform3", "geometric", "poisson"]


def make_jobs(rng, n, pool):
    thr = wl.poisson1_thresholds()
    jobs, refs = [], []
    for a in range(n):
        T = int(rng.choice([1, 32, 100, 128, 256, 512, 1024]))
        L = int(rng.choice([1, 2, 3, 8]))
        B = int(rng.choice([256, 512, 1024]))
        E = int(rng.choice([4, 8, 16]))
        target = int(rng.choice([0, 1, 17, 999, 5000, 40000]))
        dist = DISTS[a % 4]
        spec = gga.make_gen_spec(1000 + a, dist, (0x10001, 0x9E3779B9, 7), round0=a % 5,
                                 thresholds=thr if dist == "poisson" else None)
        g = gga.GGArray(L, T, B, E, shared_pool=pool)
        o = oracle.OracleGGArray(L, T, B, E)
        o.grow_to_target(1000 + a, dist, (0x10001, 0x9E3779B9, 7), target, round0=a % 5, thresholds=thr)
        jobs.append((g, spec, target))
        refs.append(o)
    return jobs, refs


def test_small_batch_matches_oracle():
    rng = np.random.default_rng(71)
    pool = gga.GGAPool(256 << 20, 256 * 4)
    jobs, refs = make_jobs(rng, 36, pool)
    batch = gga.GGABatch(jobs)
    batch.grow()
    for (g, _, target), o in zip(jobs, refs):
        assert_same_state(g, o)
        assert g.size()[0] == target
    # Clear and grow again (buckets come back from the pool's queues).
    bump = pool.info()["bump_bytes"]
    batch.clear()
    batch.grow()
    for (g, _, _), o in zip(jobs, refs):
        assert_same_state(g, o)
    assert pool.info()["bump_bytes"] == bump
    # Captured in a CUDA graph and replayed.
    s = torch.cuda.Stream()
    batch.capture(s)
    for _ in range(2):
        batch.replay(s)
    s.synchronize()
    for (g, _, _), o in zip(jobs, refs):
        assert_same_state(g, o)
    batch.close()
    for g, _, _ in jobs:
        g.close()
    pool.close()


@pytest.mark.parametrize("order", ["ascending", "shuffled"])
def test_threshold_tables_in_any_order(order):
    # A Poisson-style count is #{k : u >= thr[k]}.  The batch kernel finds
    # it by binary search when the table is ascending and counts it
    # otherwise; both must give the oracle's counts.  The shuffled table
    # also carries thresholds equal to each other and to 0 and 2^32 - 1.
    thr = np.array(list(wl.poisson1_thresholds()) + [0, 0xFFFFFFFF, 1 << 31], dtype=np.uint32)
    thr = np.sort(thr) if order == "ascending" else np.random.default_rng(5).permutation(thr)
    pool = gga.GGAPool(128 << 20, 256 * 4)
    jobs, refs = [], []
    for a, (T, E, target) in enumerate([(512, 4, 70000), (1024, 8, 30001), (100, 16, 9999), (32, 4, 5)]):
        spec = gga.make_gen_spec(40 + a, "poisson", (3, 1 << 20, 1), thresholds=thr)
        g = gga.GGArray(3, T, 256, E, shared_pool=pool)
        o = oracle.OracleGGArray(3, T, 256, E)
        o.grow_to_target(40 + a, "poisson", (3, 1 << 20, 1), target, thresholds=thr)
        jobs.append((g, spec, target))
        refs.append(o)
    batch = gga.GGABatch(jobs)
    batch.grow()
    for (g, _, target), o in zip(jobs, refs):
        assert_same_state(g, o)
        assert g.size()[0] == target
    batch.close()
    for g, _, _ in jobs:
        g.close()
    pool.close()


def test_batched_workload_4096_arrays():
    sizes = batching.batched_sizes()
    assert len(sizes) == 4096 and sizes.max() <= (16 << 20) and sizes.min() >= 1
    assert 30000 < np.median(sizes) < 140000
    rule = batching.tuned_rule()
    pool, arrays, batch, params = batching.build(sizes, rule)
    s = torch.cuda.Stream()
    batch.capture(s)
    batch.replay(s)
    batch.replay(s)
    s.synchronize()
    got = np.array([g.size()[0] for g in arrays])
    assert np.array_equal(got, sizes)                       # every array reached its target
    assert all(g.last_error() == gga.GGA_OK for g in arrays)
    assert batching.memory_ratio(arrays) <= 2.1
    # Every one of the 4096 arrays against the oracle (run in a spawned
    # worker pool; each side reduced to a digest of its sizes, capacities,
    # offsets and flattened contents).
    thr = wl.poisson1_thresholds()
    jobs = [(a, params[a][1], params[a][0], params[a][2], batching.payload_bytes(a), (3 << 32) | a, "poisson",
             (0x10001, 0x9E3779B9, 7), int(sizes[a]), thr) for a in range(len(sizes))]
    want = oracle_pool.grown_digests(jobs)
    bad = []
    for a, g in enumerate(arrays):
        n, rc, s_, c_ = g.sizes_caps()
        flat = dev_to_np(g.flatten(), g.E)[:n].tobytes() if n else b""
        got = oracle_pool.state_digest(s_.cpu().numpy(), c_.cpu().numpy(), g.offsets().cpu().numpy(), flat)
        if rc != gga.GGA_OK or got != want[a]:
            bad.append(a)
    assert not bad, bad[:10]
    # One array in full, element by element (a failure there shows where).
    a = int(np.argmax(sizes))
    T, L, B = params[a]
    o = oracle.OracleGGArray(L, T, B, batching.payload_bytes(a))
    o.grow_to_target((3 << 32) | a, "poisson", (0x10001, 0x9E3779B9, 7), int(sizes[a]), thresholds=thr)
    assert_same_state(arrays[a], o)
    batching.teardown(pool, arrays, batch)
