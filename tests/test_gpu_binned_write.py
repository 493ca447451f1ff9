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

from harness import assert_same_state, insert_both, make_pair, packed_values, random_counts, values_to_dev

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
