"""Shared test helpers: move seeded inputs to the device, run the same
workload through the CUDA path (via the C ABI) and through the oracle, and
compare results bit for bit."""

from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_2209_00103_gb300 import gga
from paper_2209_00103_gb300 import workloads as wl


def counts_to_dev(counts: np.ndarray, offset_elems: int = 0) -> torch.Tensor:
    c = np.ascontiguousarray(counts, dtype=np.uint32).view(np.int32)
    if offset_elems:
        buf = torch.zeros(c.size + offset_elems, dtype=torch.int32, device="cuda")
        buf[offset_elems:] = torch.from_numpy(c.reshape(-1)).cuda()
        return buf[offset_elems:].view(c.shape)
    return torch.from_numpy(c).cuda()


def values_to_dev(values: np.ndarray, E: int, offset_elems: int = 0) -> torch.Tensor:
    if E == 4:
        host = torch.from_numpy(np.ascontiguousarray(values).view(np.int32))
    elif E == 8:
        host = torch.from_numpy(np.ascontiguousarray(values).view(np.int64))
    else:
        host = torch.from_numpy(np.ascontiguousarray(values).view(np.int64).reshape(-1, 2))
    if offset_elems:
        shape = (host.shape[0] + offset_elems,) + tuple(host.shape[1:])
        buf = torch.zeros(shape, dtype=host.dtype, device="cuda")
        buf[offset_elems:] = host.cuda()
        return buf[offset_elems:]
    return host.cuda()


def dev_to_np(t: torch.Tensor, E: int) -> np.ndarray:
    a = t.detach().cpu().contiguous().numpy()
    if E == 4:
        return a.view(np.uint32).reshape(-1)
    if E == 8:
        return a.view(np.uint64).reshape(-1)
    return a.view(np.dtype((np.void, 16))).reshape(-1)


def np_to_dev_vals(v: np.ndarray, E: int) -> torch.Tensor:
    return values_to_dev(v, E)


def assert_same_state(g: gga.GGArray, o: oracle.OracleGGArray, check_flatten: bool = True):
    n, rc, sizes, caps = g.sizes_caps()
    assert rc == gga.GGA_OK, gga.ERROR_NAMES.get(rc)
    assert n == o.size()
    assert np.array_equal(sizes.cpu().numpy().astype(np.uint64), o.sizes())
    ocaps, _ = o.capacities()
    assert np.array_equal(caps.cpu().numpy().astype(np.uint64), ocaps)
    assert np.array_equal(g.offsets().cpu().numpy().astype(np.uint64), o.offsets())
    if check_flatten:
        flat = dev_to_np(g.flatten(), g.E)[:n]
        assert flat.tobytes() == o.flatten().tobytes()


def make_pair(L, T, B, E, pool_bytes=None, expected_elems=0):
    if pool_bytes is None:
        pool_bytes = max(1 << 20, 4 * expected_elems * E + L * 4 * B * E + (1 << 20))
    g = gga.GGArray(L, T, B, E, pool_bytes)
    o = oracle.OracleGGArray(L, T, B, E)
    return g, o


def insert_both(g, o, counts, values, E, counts_off=0, values_off=0):
    g.insert(counts_to_dev(counts, counts_off), values_to_dev(values, E, values_off))
    o.insert(counts, values)


def random_counts(rng, R, L, T, hi=3):
    return rng.integers(0, hi, size=(R, L, T)).astype(np.uint32)


def packed_values(n: int, E: int, seed: int = 0) -> np.ndarray:
    v = wl.splitmix_at(seed, np.arange(n, dtype=np.uint64))
    return wl.encode_values(v, E)
