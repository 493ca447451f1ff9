"""GPU parity: the CUDA path (through the C ABI) against the oracle, bit for
bit -- flattened contents, per-LFVector sizes, capacities and offsets, random
reads and writes, both sweeps.  The GGArray is an exact integer structure, so
there is no tolerance."""

import numpy as np
import pytest
import torch

import oracle
from paper_2209_00103_gb300 import gga
from paper_2209_00103_gb300 import workloads as wl

from harness import (assert_same_state, counts_to_dev, dev_to_np, insert_both, make_pair, packed_values,
                     random_counts, values_to_dev)

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    yield
    torch.cuda.synchronize()


def check_random_rw(g, o, E, n_idx, seed):
    N = o.size()
    if N == 0:
        return
    idx = wl.uniform_indices(seed, n_idx, N) if N < (1 << 32) else None
    got = dev_to_np(g.read(torch.from_numpy(idx.view(np.int64)).cuda()), E)
    want, rc = o.read(idx)
    assert rc == oracle.OK
    assert got.tobytes() == want.tobytes()
    # index-keyed writes: duplicates carry equal values
    widx = wl.uniform_indices(seed + 1, n_idx, N)
    wv = wl.index_keyed_values(seed + 2, widx, E)
    g.write(torch.from_numpy(widx.view(np.int64)).cuda(), values_to_dev(wv, E))
    assert o.write(widx, wv) == oracle.OK


# ---------------------------------------------------------------------------

def test_tiny_workload_end_to_end():
    w = wl.tiny_bernoulli()
    counts, values = w.spec.make()
    g, o = make_pair(w.L, w.T, w.B, w.E)
    insert_both(g, o, counts, values, w.E)
    assert_same_state(g, o)
    # Self-describing values checked on the GPU output directly.
    flat = dev_to_np(g.flatten(), 4).astype(np.int64)
    gtid, rnd = flat // 10, flat % 10
    key = (gtid // w.T) * 100000 + rnd * 1000 + gtid % w.T
    assert np.all(np.diff(key) > 0)
    check_random_rw(g, o, 4, w.n_random, w.read_seed)
    assert_same_state(g, o)
    # One +1 read-modify-write pass, both sweep modes, then flatten again.
    g.sweep(gga.GGA_RW_B, 1, 1)
    o.sweep_add(1, 1)
    assert_same_state(g, o)
    g.sweep(gga.GGA_RW_G, 1, 30)
    o.sweep_add(1, 30)
    assert_same_state(g, o)
    assert g.last_error() == gga.GGA_OK
    g.close()


@pytest.mark.parametrize("E", [4, 8, 16])
@pytest.mark.parametrize("L,T,B,R", [(1, 1, 1, 1), (1, 5, 2, 7), (3, 32, 4, 3), (7, 33, 16, 5),
                                     (5, 128, 1024, 9), (4, 512, 4, 4), (2, 1024, 8, 3), (9, 100, 2, 6)])
def test_ragged_shapes(L, T, B, R, E):
    rng = np.random.default_rng(L * 1000 + T * 10 + B + R + E)
    counts = random_counts(rng, R, L, T, hi=4)
    if L > 2:
        counts[:, 1, :] = 0                      # an LFVector that stays empty
    counts[R // 2] = 0                           # an empty round
    values = packed_values(int(counts.sum()), E, seed=R)
    g, o = make_pair(L, T, B, E, expected_elems=int(counts.sum()))
    insert_both(g, o, counts, values, E)
    assert_same_state(g, o)
    check_random_rw(g, o, E, 1000, 7)
    assert_same_state(g, o)
    if E != 16:
        g.sweep(gga.GGA_RW_G, 3, 2)
        o.sweep_add(3, 2)
        g.sweep(gga.GGA_RW_B, 0xFFFFFFFF, 1)
        o.sweep_add(0xFFFFFFFF, 1)
        assert_same_state(g, o)
    g.close()


@pytest.mark.parametrize("E", [4, 8, 16])
def test_long_runs_cross_buckets_and_chunks(E):
    # A few threads insert thousands of elements: runs span many buckets and
    # copy/flatten chunks; other threads insert nothing.
    L, T, B, R = 3, 64, 4, 4
    counts = np.zeros((R, L, T), dtype=np.uint32)
    counts[0, 0, 5] = 70000
    counts[1, 0, 6] = 3
    counts[1, 2, 0] = 40001
    counts[2, 1, 63] = 9000
    counts[3, :, :] = 1
    values = packed_values(int(counts.sum()), E, seed=5)
    g, o = make_pair(L, T, B, E, expected_elems=int(counts.sum()))
    insert_both(g, o, counts, values, E)
    assert_same_state(g, o)
    g.close()


@pytest.mark.parametrize("counts_off,values_off", [(1, 0), (0, 1), (3, 3)])
def test_unaligned_input_pointers(counts_off, values_off):
    rng = np.random.default_rng(17)
    L, T, B, R, E = 6, 256, 64, 5, 4
    counts = random_counts(rng, R, L, T)
    values = packed_values(int(counts.sum()), E, seed=1)
    g, o = make_pair(L, T, B, E, expected_elems=int(counts.sum()))
    insert_both(g, o, counts, values, E, counts_off, values_off)
    assert_same_state(g, o)
    g.close()


def test_round_by_round_equals_batched():
    rng = np.random.default_rng(23)
    L, T, B, R, E = 16, 128, 32, 12, 4
    counts = random_counts(rng, R, L, T)
    values = packed_values(int(counts.sum()), E, seed=9)
    g1, o = make_pair(L, T, B, E, expected_elems=int(counts.sum()))
    g2, _ = make_pair(L, T, B, E, expected_elems=int(counts.sum()))
    spr = o.insert(counts, values, per_round=True)
    g1.insert(counts_to_dev(counts), values_to_dev(values, E))
    pos = 0
    for r in range(R):
        m = int(counts[r].sum())
        g2.insert(counts_to_dev(counts[r:r + 1]), values_to_dev(values[pos:pos + m], E))
        pos += m
        _, rc, sizes, _ = g2.sizes_caps()
        assert rc == gga.GGA_OK
        assert np.array_equal(sizes.cpu().numpy().astype(np.uint64), spr[r])
    assert_same_state(g1, o)
    assert_same_state(g2, o)
    g1.close()
    g2.close()


def test_many_rounds_grow_scratch():
    # More rounds than the initial scratch holds, then fewer again.
    rng = np.random.default_rng(29)
    L, T, B, E = 8, 64, 16, 4
    g, o = make_pair(L, T, B, E, pool_bytes=64 << 20)
    for R in (200, 3, 1000, 1):
        counts = random_counts(rng, R, L, T)
        values = packed_values(int(counts.sum()), E, seed=R)
        insert_both(g, o, counts, values, E)
        assert_same_state(g, o)
    g.close()


@pytest.mark.parametrize("E", [4, 8, 16])
@pytest.mark.parametrize("dist", ["bernoulli", "uniform3", "geometric", "poisson"])
def test_generated_insert_matches_oracle(dist, E):
    L, T, B = 11, 96, 8
    thr = wl.poisson1_thresholds()
    coeffs = (10, 1 << 20, 1 << 19)
    g, o = make_pair(L, T, B, E, pool_bytes=64 << 20)
    for round0, R in [(0, 5), (5, 12), (17, 1)]:
        spec = gga.make_gen_spec(99, dist, coeffs, round0=round0, thresholds=thr if dist == "poisson" else None)
        g.insert_generated(spec, R)
        o.insert_generated(99, dist, coeffs, round0, R, thresholds=thr)
        assert_same_state(g, o)
    g.close()


@pytest.mark.parametrize("T", [300, 512, 1000])
@pytest.mark.parametrize("dist,E", [("uniform3", 4), ("poisson", 16), ("geometric", 8)])
def test_generated_insert_wide_blocks(T, dist, E):
    # Blocks of more than 256 threads (the launches that may play two
    # virtual threads per thread), ragged T, rounds not a multiple of a pass.
    L, B = 37, 64
    thr = wl.poisson1_thresholds()
    coeffs = (3, 1 << 21, 7)
    g, o = make_pair(L, T, B, E, pool_bytes=256 << 20)
    for round0, R in [(0, 13), (13, 8)]:
        spec = gga.make_gen_spec(5, dist, coeffs, round0=round0, thresholds=thr if dist == "poisson" else None)
        g.insert_generated(spec, R)
        o.insert_generated(5, dist, coeffs, round0, R, thresholds=thr)
        assert_same_state(g, o)
    g.close()


def test_generated_and_packed_paths_agree():
    # The in-kernel generated insertion and gga_insert on the same draws.
    spec_np = wl.InsertSpec(L=32, T=256, E=4, seed=1, dist="bernoulli", rounds=10, coeffs=(10, 1, 0))
    counts, values = spec_np.make()
    g1, o = make_pair(32, 256, 1024, 4)
    g2, _ = make_pair(32, 256, 1024, 4)
    g1.insert(counts_to_dev(counts), values_to_dev(values, 4))
    g2.insert_generated(gga.make_gen_spec(1, "bernoulli", (10, 1, 0)), 10)
    o.insert(counts, values)
    assert_same_state(g1, o)
    assert_same_state(g2, o)
    g1.close()
    g2.close()


# ---------------------------------------------------------------------------
# Edge cases and device-detected errors.

def test_empty_array():
    g, o = make_pair(4, 32, 4, 4)
    assert_same_state(g, o, check_flatten=False)
    dst = torch.full((4,), -1, dtype=torch.int32, device="cuda")
    g.flatten(dst)
    assert g.last_error() == gga.GGA_OK
    assert dst.tolist() == [-1] * 4
    out = g.read(torch.tensor([0], dtype=torch.int64, device="cuda"))
    assert g.last_error() == gga.GGA_ERR_OUT_OF_RANGE
    assert out.tolist() == [0]
    g.close()


def test_out_of_range_and_small_destination():
    rng = np.random.default_rng(3)
    L, T, B, R, E = 4, 64, 4, 3, 4
    counts = random_counts(rng, R, L, T)
    values = packed_values(int(counts.sum()), E)
    g, o = make_pair(L, T, B, E)
    insert_both(g, o, counts, values, E)
    N = o.size()
    out = g.read(torch.tensor([0, N, N - 1], dtype=torch.int64, device="cuda"))
    assert g.last_error() == gga.GGA_ERR_OUT_OF_RANGE
    want, _ = o.read(np.array([0, N - 1], dtype=np.uint64))
    got = dev_to_np(out, 4)
    assert got[1] == 0 and got[0] == want[0] and got[2] == want[1]
    g.write(torch.tensor([N + 5], dtype=torch.int64, device="cuda"), torch.tensor([1], dtype=torch.int32, device="cuda"))
    assert g.last_error() == gga.GGA_ERR_OUT_OF_RANGE
    dst = torch.full((N - 1,), 7, dtype=torch.int32, device="cuda")
    g.flatten(dst)
    assert g.last_error() == gga.GGA_ERR_DST_TOO_SMALL
    assert bool((dst == 7).all())
    assert_same_state(g, o)
    g.close()


def test_count_value_mismatch_inserts_nothing():
    g, o = make_pair(2, 32, 4, 4)
    counts = np.ones((2, 2, 32), dtype=np.uint32)
    g.insert(counts_to_dev(counts), values_to_dev(np.arange(127, dtype=np.uint32), 4))
    n, rc = g.size()
    assert rc == gga.GGA_ERR_INVALID and n == 0
    assert g.last_error() == gga.GGA_ERR_INVALID
    assert g.last_error() == gga.GGA_OK
    # The array still works afterwards.
    insert_both(g, o, counts, np.arange(128, dtype=np.uint32), 4)
    assert_same_state(g, o)
    g.close()


def test_invalid_arguments_rejected_on_host():
    with pytest.raises(gga.GGAError):
        gga.GGArray(4, 32, 3, 4, 1 << 20)        # B not a power of two
    with pytest.raises(gga.GGAError):
        gga.GGArray(4, 32, 4, 12, 1 << 20)       # element size
    with pytest.raises(gga.GGAError):
        gga.GGArray(0, 32, 4, 4, 1 << 20)
    with pytest.raises(gga.GGAError):
        gga.GGArray(4, 2048, 4, 4, 1 << 20)
    g = gga.GGArray(2, 32, 4, 16, 1 << 20)
    with pytest.raises(gga.GGAError):
        g.sweep(gga.GGA_RW_B, 1)                 # records are not integers
    g.close()


def test_pool_exhaustion_keeps_fitting_prefix():
    # The pool fits a few buckets only.  LFVectors that cannot allocate keep
    # the rounds that fit; nothing else is disturbed.
    rng = np.random.default_rng(41)
    L, T, B, R, E = 8, 64, 64, 6, 4
    counts = random_counts(rng, R, L, T)
    values = packed_values(int(counts.sum()), E)
    pool = 3 * L * 64 * 4 + 3 * 128 * 4 * 4     # every LFVector gets ~2 buckets
    g = gga.GGArray(L, T, B, E, pool)
    o = oracle.OracleGGArray(L, T, B, E)
    spr = o.insert(counts, values, per_round=True)
    g.insert(counts_to_dev(counts), values_to_dev(values, E))
    n, rc, sizes, caps = g.sizes_caps()
    assert rc == gga.GGA_ERR_POOL_EXHAUSTED
    sizes = sizes.cpu().numpy().astype(np.uint64)
    caps = caps.cpu().numpy().astype(np.uint64)
    full = o.sizes()
    assert (sizes < full).any()
    flat = dev_to_np(g.flatten(), E)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    for l in range(L):
        s = int(sizes[l])
        # committed size is a round boundary of the oracle's size series
        assert s == 0 or s in set(spr[:, l].tolist())
        assert s <= caps[l]
        assert flat[off[l]:off[l] + s].tobytes() == o.lfvector(l)[:s].tobytes()
    mem = g.memory()
    assert mem["pool_bump_bytes"] <= pool
    g.close()


def test_clear_reuses_buckets_from_free_lists():
    rng = np.random.default_rng(43)
    L, T, B, R, E = 16, 128, 256, 8, 8
    counts = random_counts(rng, R, L, T)
    values = packed_values(int(counts.sum()), E)
    g, o = make_pair(L, T, B, E, pool_bytes=32 << 20)
    insert_both(g, o, counts, values, E)
    m1 = g.memory()
    g.clear()
    m2 = g.memory()
    assert m2["bucket_bytes"] == 0 and m2["live_bytes"] == 0
    assert m2["free_list_bytes"] >= m1["bucket_bytes"]
    o2 = oracle.OracleGGArray(L, T, B, E)
    g.insert(counts_to_dev(counts), values_to_dev(values, E))
    o2.insert(counts, values)
    assert_same_state(g, o2)
    m3 = g.memory()
    assert m3["pool_bump_bytes"] == m1["pool_bump_bytes"]   # all buckets came from the free lists
    assert m3["bucket_bytes"] == m1["bucket_bytes"]
    g.close()


def test_memory_accounting_matches_capacities():
    rng = np.random.default_rng(47)
    L, T, B, R, E = 32, 256, 1024, 20, 4
    counts = random_counts(rng, R, L, T)
    values = packed_values(int(counts.sum()), E)
    g, o = make_pair(L, T, B, E)
    insert_both(g, o, counts, values, E)
    m = g.memory()
    assert m["bucket_bytes"] == o.bucket_bytes()
    assert m["live_bytes"] == o.size() * E
    assert m["bucket_bytes"] <= 2 * m["live_bytes"] + L * B * E
    g.close()
