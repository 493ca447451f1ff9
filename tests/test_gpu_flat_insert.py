"""Sec. III-B's insertion approaches on a flat array: every thread's value
lands exactly once after the old size, the size advances by the thread
count, a block's run is contiguous and in thread order with the scan
approach, and nothing is written past the capacity."""

import numpy as np
import pytest
import torch

from paper_2209_00103_gb300 import gga

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", [gga.GGA_FLAT_ATOMIC, gga.GGA_FLAT_SCAN])
@pytest.mark.parametrize("T", [32, 128, 1024])
def test_flat_insert_places_every_value_once(mode, T):
    cap, old, n, first = 5_000_000, 1000, 3_000_017, 77
    a = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    a[:old] = torch.arange(old, dtype=torch.int32, device="cuda")
    size = torch.tensor([old], dtype=torch.int64, device="cuda")
    gga.gga_flat_insert(mode, a, size, n, T, first)
    assert int(size.item()) == old + n
    h = a.cpu().numpy()
    assert np.array_equal(h[:old], np.arange(old))
    got = h[old:old + n].astype(np.int64)
    assert np.array_equal(np.sort(got), first + np.arange(n))
    assert np.all(h[old + n:] == -1)
    if mode == gga.GGA_FLAT_SCAN:
        pos = np.empty(n, dtype=np.int64)
        pos[got - first] = np.arange(n)
        starts = pos[::T]
        for b in range(0, (n + T - 1) // T, 97):
            k = min(T, n - b * T)
            assert np.array_equal(pos[b * T:b * T + k], starts[b] + np.arange(k))


@pytest.mark.parametrize("mode", [gga.GGA_FLAT_ATOMIC, gga.GGA_FLAT_SCAN])
def test_flat_insert_respects_capacity(mode):
    a = torch.full((1000,), -1, dtype=torch.int32, device="cuda")
    guard = torch.full((4096,), -5, dtype=torch.int32, device="cuda")
    size = torch.tensor([900], dtype=torch.int64, device="cuda")
    gga.gga_flat_insert(mode, a, size, 500, 128, 0)
    assert int(size.item()) == 1400
    h = a.cpu().numpy()
    assert np.all(h[:900] == -1) and np.all(h[900:] >= 0)
    assert bool((guard == -5).all())
