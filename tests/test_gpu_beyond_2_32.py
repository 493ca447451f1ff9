"""Parity beyond 2^32 elements: a generated GGArray of ~4.36e9 int32 elements
(1024 LFVectors x 1024 threads, 4160 rounds of Uniform{0,1,2}, ~17 GB), so
global indices, offsets and flatten positions need 64 bits.  Three
LFVectors -- the first, one in the middle and the last, whose elements lie
past global index 2^32 -- are rebuilt by the oracle from their own draws;
sizes, capacities, sampled reads, writes (direct, and a batch large enough
to be binned), both sweeps and the flattened array are checked against it."""

import numpy as np
import pytest
import torch

import oracle
from paper_2209_00103_gb300 import gga
from paper_2209_00103_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

L, T, B, E, R = 1024, 1024, 4096, 4, 4160
SEED, DIST, COEFFS = 21, "uniform3", (3, 1 << 20, 1 << 9)


def lfv_oracle(l):
    spec = wl.InsertSpec(L=1, T=T, E=E, seed=SEED, dist=DIST, rounds=R, coeffs=COEFFS, gtid0=l * T)
    counts, values = spec.make()
    o = oracle.OracleGGArray(1, T, B, E)
    o.insert(counts, values)
    return o


def test_generated_array_beyond_2_32_elements():
    free, _ = torch.cuda.mem_get_info()
    if free < (64 << 30):
        pytest.skip(f"needs ~55 GB of free device memory, {free >> 30} GB free")
    g = gga.GGArray(L, T, B, E, 36 << 30)
    g.insert_generated(gga.make_gen_spec(SEED, DIST, COEFFS), R)
    n, rc, sizes, caps = g.sizes_caps()
    assert rc == gga.GGA_OK and n > (1 << 32)
    sizes = sizes.cpu().numpy().astype(np.int64)
    caps = caps.cpu().numpy().astype(np.int64)
    offs = g.offsets().cpu().numpy().astype(np.int64)
    assert offs[0] == 0 and np.array_equal(np.diff(offs), sizes) and offs[L] == n
    rng = np.random.default_rng(1)
    picks = {}
    for l in (0, 700, L - 1):
        o = lfv_oracle(l)
        assert sizes[l] == o.size()
        assert caps[l] == int(o.capacities()[0][0])
        j = np.unique(np.concatenate([[0, 1, sizes[l] - 1], rng.integers(0, sizes[l], 3000)])).astype(np.int64)
        want, orc = o.read(j.astype(np.uint64))
        assert orc == oracle.OK
        picks[l] = (j, want.astype(np.uint32), o)
    assert offs[L - 1] > (1 << 32)
    gidx = {l: torch.from_numpy(offs[l] + j).cuda() for l, (j, _, _) in picks.items()}

    def check(delta):
        for l, (j, want, _) in picks.items():
            got = g.read(gidx[l]).cpu().numpy().view(np.uint32)
            assert np.array_equal(got, want + np.uint32(delta)), l

    check(0)
    g.sweep(gga.GGA_RW_G, 1, 1)
    check(1)
    g.sweep(gga.GGA_RW_B, 2, 1)
    check(3)
    # Writes past 2^32, then read back.
    j, want, _ = picks[L - 1]
    newv = (np.arange(j.size, dtype=np.uint32) * np.uint32(2654435761)).view(np.int32)
    g.write(gidx[L - 1], torch.from_numpy(newv).cuda())
    assert np.array_equal(g.read(gidx[L - 1]).cpu().numpy(), newv)
    picks[L - 1] = (j, newv.view(np.uint32) - np.uint32(3), None)
    # A batch of 2^20 + 5 writes (the binned path: writes grouped by ranges of
    # global indices, each stored as its bin and its offset inside the bin)
    # into the three checked LFVectors, the last of them past 2^32; the
    # values are keyed by the index, so repeated indices agree.
    rng2 = np.random.default_rng(9)
    ls = np.array(sorted(picks), dtype=np.int64)
    nw = (1 << 20) + 5
    li = rng2.integers(0, ls.size, nw)
    loc = (rng2.random(nw) * sizes[ls[li]]).astype(np.int64)
    gw = offs[ls[li]] + loc
    assert gw.max() >= (1 << 32)
    vals = ((gw.astype(np.uint64) * np.uint64(2654435761)) & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    gw_dev = torch.from_numpy(gw).cuda()
    g.write(gw_dev, torch.from_numpy(vals.view(np.int32)).cuda())
    assert np.array_equal(g.read(gw_dev).cpu().numpy().view(np.uint32), vals)
    for l, (j, want, o) in list(picks.items()):
        m = ls[li] == l
        hit = dict(zip(loc[m].tolist(), vals[m].tolist()))
        w2 = want.copy()
        for k, jj in enumerate(j.tolist()):
            if jj in hit:
                w2[k] = np.uint32((hit[jj] - 3) & 0xFFFFFFFF)
        picks[l] = (j, w2, o)
    for l, (j, want, _) in picks.items():   # the sampled positions: written or kept
        got = g.read(gidx[l]).cpu().numpy().view(np.uint32)
        assert np.array_equal(got, want + np.uint32(3)), l
    # Flatten: the sampled positions of the contiguous copy.
    dst = gga.elem_tensor(n, E)
    g.flatten(dst)
    for l, (j, want, _) in picks.items():
        got = dst[gidx[l]].cpu().numpy().view(np.uint32)
        assert np.array_equal(got, want + np.uint32(3)), l
    assert g.last_error() == gga.GGA_OK
    del dst
    g.close()
