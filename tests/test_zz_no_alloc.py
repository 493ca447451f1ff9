"""gga_insert_noalloc: insertion for callers that may not allocate GPU memory
during the call (a fixed, pre-reserved memory budget; latency-critical
loops).  Its per-call scratch is the library's fixed device array, so it must
give exactly what gga_insert gives -- also on the second call in a row, when
the array still holds the first call's leftovers -- and the device's memory
in use must not change across a call, not even transiently in the
stream-ordered pool.

This file is named to be collected last."""

import ctypes
import ctypes.util
import glob
import os

import numpy as np
import pytest
import torch

from paper_2209_00103_gb300 import gga

from harness import counts_to_dev, dev_to_np, packed_values, random_counts, values_to_dev

pytestmark = pytest.mark.gpu

# cudaMemPoolAttr values of the CUDA runtime API.
_RESERVED_MEM_CURRENT, _RESERVED_MEM_HIGH, _USED_MEM_CURRENT, _USED_MEM_HIGH = 5, 6, 7, 8


def _cudart():
    """The CUDA runtime the library itself links (shared cudart)."""
    cands = sorted(glob.glob(os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64", "libcudart.so*")))
    name = cands[-1] if cands else ctypes.util.find_library("cudart")
    assert name, "libcudart not found"
    return ctypes.CDLL(name)


class StreamPool:
    """The current device's stream-ordered memory pool (the one
    cudaMallocAsync draws from), with its high-water marks."""

    def __init__(self):
        self.rt = _cudart()
        dev = ctypes.c_int()
        assert self.rt.cudaGetDevice(ctypes.byref(dev)) == 0
        self.pool = ctypes.c_void_p()
        assert self.rt.cudaDeviceGetMemPool(ctypes.byref(self.pool), dev.value) == 0

    def attr(self, a):
        v = ctypes.c_uint64()
        assert self.rt.cudaMemPoolGetAttribute(self.pool, a, ctypes.byref(v)) == 0
        return v.value

    def reset_highs(self):
        zero = ctypes.c_uint64(0)
        for a in (_RESERVED_MEM_HIGH, _USED_MEM_HIGH):
            assert self.rt.cudaMemPoolSetAttribute(self.pool, a, ctypes.byref(zero)) == 0


def state(g):
    n, rc, sizes, caps = g.sizes_caps()
    flat = dev_to_np(g.flatten(), g.E)[:n].tobytes() if n else b""
    return n, rc, sizes.cpu().numpy(), caps.cpu().numpy(), g.offsets().cpu().numpy(), flat


def assert_same(g_ref, g_na):
    n1, rc1, s1, k1, o1, f1 = state(g_ref)
    n2, rc2, s2, k2, o2, f2 = state(g_na)
    assert rc1 == rc2 == gga.GGA_OK
    assert n1 == n2 > 0
    assert np.array_equal(s1, s2) and np.array_equal(k1, k2) and np.array_equal(o1, o2)
    assert f1 == f2


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
        assert_same(g_ref, g_na)
    g_ref.close()
    g_na.close()


def test_noalloc_allocates_nothing_on_two_handles():
    """Calls on two handles of different L, taken in turn, each with more
    rounds than any call before it on that handle (so gga_insert would grow
    its scratch there): the device's free memory and the stream-ordered
    pool's reserved and used high-water marks do not move across a call,
    and the results equal gga_insert's."""
    rng = np.random.default_rng(7)
    E, B = 4, 32
    shapes = [(96, 256), (37, 512)]
    refs = [gga.GGArray(L, T, B, E, 64 << 20) for L, T in shapes]
    nas = [gga.GGArray(L, T, B, E, 64 << 20) for L, T in shapes]
    sp = StreamPool()
    for R in (3, 17, 60):
        for (L, T), g_ref, g_na in zip(shapes, refs, nas):
            counts = random_counts(rng, R, L, T)
            values = packed_values(int(counts.sum()), E, seed=R * 1000 + L)
            c_dev, v_dev = counts_to_dev(counts), values_to_dev(values, E)
            g_ref.insert(c_dev, v_dev)   # also loads the insertion kernels' module before the check
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            res0, used0 = sp.attr(_RESERVED_MEM_CURRENT), sp.attr(_USED_MEM_CURRENT)
            sp.reset_highs()
            gga.gga_insert_noalloc(g_na.h, c_dev, v_dev)
            torch.cuda.synchronize()
            assert torch.cuda.mem_get_info()[0] == free0
            assert sp.attr(_RESERVED_MEM_HIGH) <= res0 and sp.attr(_USED_MEM_HIGH) <= used0
            assert_same(g_ref, g_na)
    for g in refs + nas:
        g.close()


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
