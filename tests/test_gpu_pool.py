"""Shared bucket pools: several GGArrays carve buckets from one slab; a
destroyed array's buckets return to the pool's free queues and are reused
by the next arrays before the bump pointer moves."""

import numpy as np
import pytest
import torch

import oracle
from paper_2209_00103_gb300 import gga

from harness import assert_same_state, counts_to_dev, packed_values, random_counts, values_to_dev

pytestmark = pytest.mark.gpu


def test_arrays_share_a_pool_and_match_the_oracle():
    rng = np.random.default_rng(61)
    pool = gga.GGAPool(64 << 20, 256 * 4)
    arrays = []
    for k, (L, T, B, E) in enumerate([(4, 64, 256, 4), (9, 128, 512, 8), (3, 32, 64, 16), (16, 256, 256, 4)]):
        g = gga.GGArray(L, T, B, E, shared_pool=pool)
        o = oracle.OracleGGArray(L, T, B, E)
        for r in range(3):
            counts = random_counts(rng, 5, L, T)
            values = packed_values(int(counts.sum()), E, seed=10 * k + r)
            g.insert(counts_to_dev(counts), values_to_dev(values, E))
            o.insert(counts, values)
        arrays.append((g, o))
    for g, o in arrays:
        assert_same_state(g, o)
    info = pool.info()
    assert info["bump_bytes"] <= info["pool_bytes"] and info["free_list_bytes"] == 0
    for g, _ in arrays:
        g.close()
    pool.close()


def test_destroyed_buckets_are_reused():
    rng = np.random.default_rng(67)
    pool = gga.GGAPool(32 << 20, 1024 * 4)
    L, T, B, E = 8, 128, 1024, 4
    counts = random_counts(rng, 40, L, T)
    values = packed_values(int(counts.sum()), E)
    g1 = gga.GGArray(L, T, B, E, shared_pool=pool)
    g1.insert(counts_to_dev(counts), values_to_dev(values, E))
    used = pool.info()["bump_bytes"]
    g1.close()
    info = pool.info()
    assert info["free_list_bytes"] == used          # every bucket went back
    g2 = gga.GGArray(L, T, B, E, shared_pool=pool)
    o = oracle.OracleGGArray(L, T, B, E)
    g2.insert(counts_to_dev(counts), values_to_dev(values, E))
    o.insert(counts, values)
    assert_same_state(g2, o)
    info = pool.info()
    assert info["bump_bytes"] == used and info["free_list_bytes"] == 0
    g2.close()
    pool.close()


def test_pool_rejects_smaller_buckets():
    pool = gga.GGAPool(1 << 20, 4096)
    with pytest.raises(gga.GGAError):
        gga.GGArray(2, 32, 256, 4, shared_pool=pool)     # 1 KB buckets, pool serves >= 4 KB
    g = gga.GGArray(2, 32, 1024, 4, shared_pool=pool)   # 4 KB: fine
    g.close()
    pool.close()
