"""gga_insert_noalloc: insertion for callers that may not allocate GPU memory
during the call (a fixed, pre-reserved memory budget; latency-critical
loops).  Its per-call scratch is the library's fixed device array, so it must
give exactly what gga_insert gives -- also on the second call in a row, when
the array still holds the first call's leftovers.

This file is named to be collected last."""

import numpy as np
import pytest
import torch

from paper_2209_00103_gb300 import gga

from harness import counts_to_dev, dev_to_np, packed_values, random_counts, values_to_dev

pytestmark = pytest.mark.gpu


def state(g):
    n, rc, sizes, caps = g.sizes_caps()
    flat = dev_to_np(g.flatten(), g.E)[:n].tobytes() if n else b""
    return n, rc, sizes.cpu().numpy(), caps.cpu().numpy(), g.offsets().cpu().numpy(), flat


@pytest.mark.parametrize("E", [4, 16])
def test_noalloc_matches_gga_insert_on_two_calls(E):
    assert torch.cuda.is_available()
    rng = np.random.default_rng(101 + E)
    L, T, B = 96, 512, 64
    g_ref = gga.GGArray(L, T, B, E, 64 << 20)
    g_na = gga.GGArray(L, T, B, E, 64 << 20)
    # Two calls in a row; the second is smaller, so it meets the first's
    # leftovers in the fixed scratch.
    for R in (40, 7):
        counts = random_counts(rng, R, L, T)
        values = packed_values(int(counts.sum()), E, seed=R)
        c_dev, v_dev = counts_to_dev(counts), values_to_dev(values, E)
        g_ref.insert(c_dev, v_dev)
        gga.gga_insert_noalloc(g_na.h, c_dev, v_dev)
        n1, rc1, s1, k1, o1, f1 = state(g_ref)
        n2, rc2, s2, k2, o2, f2 = state(g_na)
        assert rc1 == rc2 == gga.GGA_OK
        assert n1 == n2 > 0
        assert np.array_equal(s1, s2) and np.array_equal(k1, k2) and np.array_equal(o1, o2)
        assert f1 == f2
    g_ref.close()
    g_na.close()


def test_noalloc_rejects_calls_beyond_its_scratch():
    L, T, B, E = 4096, 1, 4, 4
    g = gga.GGArray(L, T, B, E, 1 << 20)
    R = 1024                                   # 4M (round, block) runs: > 32 MiB of scratch
    counts = torch.zeros((R, L, T), dtype=torch.int32, device="cuda")
    with pytest.raises(gga.GGAError) as ei:
        gga.gga_insert_noalloc(g.h, counts, torch.empty(0, dtype=torch.int32, device="cuda"))
    assert ei.value.code == gga.GGA_ERR_TOO_LARGE
    n, rc = g.size()
    assert n == 0 and rc == gga.GGA_OK
    g.close()
