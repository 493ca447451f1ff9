"""Resize without insertion (the grow step of the paper's growable-array
experiment, Sec. VI-C / Table II) against the oracle: capacities, bucket
memory and contents after reserving, after inserting into the reservation,
and after a smaller request; a pool too small keeps the longest prefix."""

import numpy as np
import pytest
import torch

import oracle
from paper_2209_00103_gb300 import gga

from harness import assert_same_state, insert_both, make_pair, packed_values, random_counts

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()


@pytest.mark.parametrize("E", [4, 16])
def test_reserve_matches_oracle(E):
    rng = np.random.default_rng(61 + E)
    L, T, B = 40, 64, 256
    g, o = make_pair(L, T, B, E, expected_elems=600000)
    counts = random_counts(rng, 4, L, T)
    insert_both(g, o, counts, packed_values(int(counts.sum()), E, 3), E)
    target = rng.integers(0, 20000, size=L).astype(np.uint64)
    target[3] = 0
    g.reserve(_dev(target))
    assert o.reserve(target) == oracle.OK
    assert_same_state(g, o)
    assert g.memory()["bucket_bytes"] == o.bucket_bytes()
    counts2 = random_counts(rng, 6, L, T)
    insert_both(g, o, counts2, packed_values(int(counts2.sum()), E, 4), E)
    assert_same_state(g, o)
    g.reserve(_dev(target // np.uint64(2)))
    o.reserve(target // np.uint64(2))
    assert_same_state(g, o)
    assert g.memory()["bucket_bytes"] == o.bucket_bytes()
    g.clear()
    n, rc, sizes, caps = g.sizes_caps()
    assert rc == gga.GGA_OK and n == 0 and int(caps.sum()) == 0
    g.close()


def test_reserve_pool_exhaustion_keeps_prefix():
    L, T, B, E = 4, 32, 256, 4
    pool = 1 << 20
    g = gga.GGArray(L, T, B, E, pool)
    target = np.full(L, 1 << 20, dtype=np.uint64)        # 4 MiB of buckets per LFVector
    g.reserve(_dev(target))
    assert g.last_error() == gga.GGA_ERR_POOL_EXHAUSTED
    n, rc, sizes, caps = g.sizes_caps()
    assert rc == gga.GGA_OK and n == 0
    for c in caps.cpu().numpy():
        k = 0
        while B * ((1 << k) - 1) < int(c):
            k += 1
        assert int(c) == B * ((1 << k) - 1) and int(c) < (1 << 20)
    assert g.memory()["bucket_bytes"] <= pool
    g.close()


@pytest.mark.parametrize("L", [32, 512])
def test_doubling_schedule_matches_oracle(L):
    # The bench's doubling experiment at a small start: resize to twice the
    # size, insert one element per element, +1 thirty times, six times over.
    T, B, E = 64, 256, 4
    n0, iters = 3000, 6
    g, o = make_pair(L, T, B, E, expected_elems=n0 << iters)

    def split(n, parts):
        return np.array([n // parts + (1 if i < n % parts else 0) for i in range(parts)], dtype=np.int64)

    def counts_for(add):
        c = np.zeros((1, L, T), dtype=np.uint32)
        for l in range(L):
            c[0, l, :] = split(int(add[l]), T)
        return c

    sizes = split(n0, L)
    insert_both(g, o, counts_for(sizes), np.arange(n0, dtype=np.uint32), E)
    for it in range(iters):
        target = (2 * sizes).astype(np.uint64)
        g.reserve(_dev(target))
        o.reserve(target)
        n_add = int(sizes.sum())
        insert_both(g, o, counts_for(sizes), (np.arange(n_add, dtype=np.uint32) * 3 + it), E)
        g.sweep(gga.GGA_RW_B, 1, 30)
        o.sweep_add(1, 30)
        sizes = 2 * sizes
        assert_same_state(g, o)
    assert g.size()[0] == n0 << iters
    g.close()
