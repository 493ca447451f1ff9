"""Large random-write batches (2^20 writes or more go through bins of
global-index ranges, applied bin after bin): the state after the writes
equals the oracle's for every element type, with duplicate indices,
out-of-range indices, and batches of growing size that reuse and regrow the
handle's bins.  The full-size paper-shaped workload (2^26 writes into 2^28
int32, 128 bins) is checked in test_gpu_full_size."""

import numpy as np
import pytest
import torch

import oracle
from paper_2209_00103_gb300 import gga
from paper_2209_00103_gb300 import workloads as wl

from harness import assert_same_state, dev_to_np, insert_both, make_pair, packed_values, random_counts, values_to_dev

pytestmark = pytest.mark.gpu


def grown_pair(E, seed, R=500, L=48, T=128, B=256):
    rng = np.random.default_rng(seed)
    counts = random_counts(rng, R, L, T)
    n_vals = int(counts.sum())
    g, o = make_pair(L, T, B, E, expected_elems=n_vals)
    insert_both(g, o, counts, packed_values(n_vals, E, seed=E), E)
    return rng, g, o


@pytest.mark.parametrize("E", [4, 8, 16])
def test_binned_writes_match_oracle(E):
    rng, g, o = grown_pair(E, 900 + E)
    N = o.size()
    assert N > 2_000_000
    for k, n in enumerate([(1 << 20) + 12345, (1 << 21) + 7, 1 << 20]):
        idx = rng.integers(0, N, size=n, dtype=np.uint64)          # duplicates are certain
        vals = wl.index_keyed_values(1000 + k, idx, E)
        g.write(torch.from_numpy(idx.view(np.int64)).cuda(), values_to_dev(vals, E))
        assert o.write(idx, vals) == oracle.OK
        assert g.last_error() == gga.GGA_OK
    assert_same_state(g, o)
    g.close()


def test_binned_writes_out_of_range_are_skipped_and_reported():
    rng, g, o = grown_pair(4, 77)
    N = o.size()
    n = (1 << 20) + 3
    idx = rng.integers(0, N, size=n, dtype=np.uint64)
    idx[[0, 1000, n - 1]] = [N, N + 12345, np.uint64(1) << np.uint64(62)]
    vals = wl.index_keyed_values(5, idx, 4)
    g.write(torch.from_numpy(idx.view(np.int64)).cuda(), values_to_dev(vals, 4))
    assert o.write(idx, vals) == oracle.ERR_OUT_OF_RANGE
    assert g.last_error() == gga.GGA_ERR_OUT_OF_RANGE
    assert_same_state(g, o)                                         # every in-range write applied
    g.close()


def as_records(a: np.ndarray, E: int) -> np.ndarray:
    """Elements as one comparable item each (16-byte records as two uint64)."""
    if E == 16:
        return np.ascontiguousarray(a).view(np.uint64).reshape(-1, 2)
    return np.ascontiguousarray(a).view({4: np.uint32, 8: np.uint64}[E]).reshape(-1, 1)


@pytest.mark.parametrize("E", [4, 8, 16])
@pytest.mark.parametrize("n", [200_000, (1 << 20) + 999])   # the direct path, and the binned path
def test_conflicting_duplicate_writes_keep_one_written_value(E, n):
    # Writes whose duplicate indices carry different values: several results
    # are correct (the paper does not order concurrent writes), so the test
    # checks the validity rule -- every written element equals, bit for bit,
    # one of the values written to its index (a torn or mixed record fails),
    # and every other element is unchanged.
    rng, g, o = grown_pair(E, 300 + E)
    N = o.size()
    before = as_records(dev_to_np(g.flatten(), E)[:N], E)
    assert before.tobytes() == o.flatten().tobytes()
    hot = rng.integers(0, N, size=4096, dtype=np.uint64)          # many writes per hot index
    idx = np.where(rng.random(n) < 0.5, hot[rng.integers(0, hot.size, size=n)],
                   rng.integers(0, N, size=n, dtype=np.uint64)).astype(np.uint64)
    vals = wl.encode_values(wl.splitmix_at(4242 + E, np.arange(n, dtype=np.uint64)), E)   # distinct per write
    if E == 16:   # make the two halves of a record disagree with every other write's halves
        v = vals.view(np.uint64).reshape(-1, 2)
        v[:, 1] = wl.splitmix_at(99, np.arange(n, dtype=np.uint64))
    g.write(torch.from_numpy(idx.view(np.int64)).cuda(), values_to_dev(vals, E))
    assert g.last_error() == gga.GGA_OK
    after = as_records(dev_to_np(g.flatten(), E)[:N], E)
    written = np.zeros(N, dtype=bool)
    written[idx] = True
    assert np.array_equal(after[~written], before[~written])
    w = as_records(vals, E)
    match = np.all(after[idx] == w, axis=1)                       # write i's value is the one kept
    order = np.argsort(idx, kind="stable")
    sidx = idx[order]
    starts = np.flatnonzero(np.concatenate([[True], sidx[1:] != sidx[:-1]]))
    kept_one = np.logical_or.reduceat(match[order], starts)
    assert kept_one.all(), int((~kept_one).sum())
    assert np.bincount(np.searchsorted(sidx[starts], idx), minlength=starts.size).max() > 8   # real conflicts
    g.close()


def test_binned_writes_on_an_array_of_more_than_2_gb():
    # 16-byte elements, ~141M of them (2.26 GB): 256 bins of 8 MB no longer
    # cover the array, so the bins are widened (the shift is raised) -- the
    # branch the 1 GB workloads never take.
    L, T, B, E, R = 512, 512, 4096, 16, 540
    coeffs = (10, 1 << 20, 1)
    g = gga.GGArray(L, T, B, E, 5 << 30)
    o = oracle.OracleGGArray(L, T, B, E)
    g.insert_generated(gga.make_gen_spec(17, "uniform3", coeffs), R)
    o.insert_generated(17, "uniform3", coeffs, 0, R)
    N = o.size()
    assert N * E > (256 << 23)
    rng = np.random.default_rng(21)
    idx = rng.integers(0, N, size=(1 << 21) + 5, dtype=np.uint64)
    vals = wl.index_keyed_values(77, idx, E)
    g.write(torch.from_numpy(idx.view(np.int64)).cuda(), values_to_dev(vals, E))
    assert o.write(idx, vals) == oracle.OK
    assert g.last_error() == gga.GGA_OK
    assert_same_state(g, o)
    g.close()
    o.close()
