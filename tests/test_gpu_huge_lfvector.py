"""One LFVector of more than 2^32 elements: L = 1, T = 1024, first bucket
4096 int32, 4,200,000 generated rounds of Uniform{0,1,2} (~4.30e9 elements,
~17 GB live, bucket 20 reached, ~34 GB of buckets).  Positions inside the
LFVector need 64 bits, so this is the case where the global sweep leaves
its 32-bit per-warp path (taken only while an LFVector's positions plus B
stay below 2^32) and every element goes through the 64-bit translation; the
random reads and writes and the flatten take the same 64-bit bucket math
(Algorithm 2's bucket sizes B 2^b, b up to 20).  Size and capacity, reads
around position 2^32 and at the edges of the last buckets, writes, both
sweeps and sampled positions of the flattened array are checked against the
oracle grown from the same draws."""

import numpy as np
import pytest
import torch

import oracle
from paper_2209_00103_gb300 import gga

pytestmark = pytest.mark.gpu

L, T, B, E, R = 1, 1024, 4096, 4, 4_200_000
SEED, DIST, COEFFS = 33, "uniform3", (7, 1 << 11, 3)


def bucket_first(b):
    return B * ((1 << b) - 1)


def test_one_lfvector_beyond_2_32_elements():
    free, _ = torch.cuda.mem_get_info()
    if free < (64 << 30):
        pytest.skip(f"needs ~56 GB of free device memory, {free >> 30} GB free")
    g = gga.GGArray(L, T, B, E, 36 << 30)
    g.insert_generated(gga.make_gen_spec(SEED, DIST, COEFFS), R)
    o = oracle.OracleGGArray(L, T, B, E)
    o.insert_generated(SEED, DIST, COEFFS, 0, R)
    n, rc, sizes, caps = g.sizes_caps()
    assert rc == gga.GGA_OK
    N = o.size()
    assert n == N and N > (1 << 32)
    assert int(sizes.cpu()[0]) == N
    assert int(caps.cpu()[0]) == int(o.capacities()[0][0]) == bucket_first(21)

    rng = np.random.default_rng(5)
    edges = [0, 1, (1 << 32) - 1, 1 << 32, (1 << 32) + 1, N - 1]
    for b in (18, 19, 20):
        edges += [bucket_first(b) - 1, bucket_first(b), bucket_first(b) + 1]
    idx = np.unique(np.concatenate([np.array([e for e in edges if e < N], dtype=np.uint64),
                                    rng.integers(0, N, 20000, dtype=np.uint64)]))
    idx_dev = torch.from_numpy(idx.view(np.int64)).cuda()

    def check():
        want, orc = o.read(idx)
        assert orc == oracle.OK
        got = g.read(idx_dev).cpu().numpy().view(np.uint32)
        assert np.array_equal(got, want)

    check()
    # Writes (the direct path: fewer than 2^20), distinct values.
    w = idx[::3]
    vals = (rng.integers(0, 1 << 32, w.shape[0], dtype=np.uint64)).astype(np.uint32)
    g.write(torch.from_numpy(w.view(np.int64)).cuda(), torch.from_numpy(vals.view(np.int32)).cuda())
    assert o.write(w, vals) == oracle.OK
    check()
    # Both sweeps over all ~4.3e9 elements.
    g.sweep(gga.GGA_RW_G, 3, 2)
    o.sweep_add(3, 2)
    check()
    g.sweep(gga.GGA_RW_B, 0xFFFFFFFF, 1)
    o.sweep_add(0xFFFFFFFF, 1)
    check()
    assert g.last_error() == gga.GGA_OK
    # Flatten: the positions of the sampled indices in the contiguous copy.
    dst = g.flatten()
    got = dst[idx_dev].cpu().numpy().view(np.uint32)
    want, _ = o.read(idx)
    assert np.array_equal(got, want)
    del dst
    g.close()
    o.close()
