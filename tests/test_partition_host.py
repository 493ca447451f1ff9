"""The partitioned GGArray's host logic on CPU, world size 2 over gloo
(rendezvous on 127.0.0.1): each rank holds a contiguous range of the
LFVectors (here the oracle stands in for the rank's GPU array), one
all-gather of the LFVector sizes gives the global offsets, each rank's
local flatten is its slice of the flattened array, and reads of global
indices are routed to the owning rank and back.  Checked against one
oracle holding all LFVectors (Sec. IV: LFVector-major global order over
the prefix sum of sizes)."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2209_00103_gb300 import partition
from paper_2209_00103_gb300 import workloads as wl


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def to_torch(a: np.ndarray, E: int) -> torch.Tensor:
    a = np.ascontiguousarray(a)
    if E == 4:
        return torch.from_numpy(a.view(np.int32).copy())
    if E == 8:
        return torch.from_numpy(a.view(np.int64).copy())
    return torch.from_numpy(a.view(np.int64).reshape(-1, 2).copy())


class OraclePart:
    """The local part of a rank, on the CPU: an oracle of its LFVectors."""

    def __init__(self, o, E):
        self.o, self.E = o, E

    def lfv_sizes(self):
        return torch.from_numpy(self.o.sizes().astype(np.int64))

    def read_local(self, idx):
        vals, rc = self.o.read(idx.numpy().astype(np.uint64))
        assert rc == oracle.OK
        return to_torch(vals, self.E)

    def flatten_local(self):
        return to_torch(self.o.flatten(), self.E)


def case(L, T, B, E, R, seed, empty_lfvs=()):
    rng = np.random.default_rng(seed)
    counts = rng.integers(0, 3, size=(R, L, T)).astype(np.uint32)
    for l in empty_lfvs:
        counts[:, l, :] = 0
    values = wl.encode_values(wl.splitmix_at(seed, np.arange(int(counts.sum()), dtype=np.uint64)), E)
    return counts, values


def slice_inputs(counts, values, l0, l1):
    """The counts and packed values of LFVectors [l0, l1) (values are packed
    in (round, LFVector, thread, k) order)."""
    R, L, T = counts.shape
    row = counts.sum(axis=2).reshape(-1).astype(np.int64)          # per (round, LFVector)
    start = np.concatenate([[0], np.cumsum(row)])
    keep = [values[start[r * L + l]:start[r * L + l + 1]] for r in range(R) for l in range(l0, l1)]
    return np.ascontiguousarray(counts[:, l0:l1, :]), np.concatenate(keep) if keep else values[:0]


def _worker(rank, world, port, q, L, T, B, E, R, seed, empty_lfvs, n_reads):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    counts, values = case(L, T, B, E, R, seed, empty_lfvs)
    l0, l1 = partition.lfv_range(L, world, rank)
    c, v = slice_inputs(counts, values, l0, l1)
    o = oracle.OracleGGArray(l1 - l0, T, B, E)
    o.insert(c, v)
    p = partition.PartitionedGGArray(OraclePart(o, E), L, world, rank)
    offsets = p.sync().numpy().copy()
    N = p.global_size()
    idx = torch.from_numpy(wl.uniform_indices(seed + 1, n_reads, N).view(np.int64)) if N else torch.zeros(0, dtype=torch.int64)
    got = p.read(idx).numpy().tobytes()
    start, part = p.flatten()
    q.put((rank, offsets.tobytes(), got, start, part.numpy().tobytes()))
    dist.destroy_process_group()


def run_ranks(world, *args):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q) + args) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    return out


@pytest.mark.parametrize("L,T,B,E,R,empty", [(8, 32, 4, 4, 5, ()), (7, 33, 8, 16, 3, (0, 1, 2)),
                                              (5, 64, 2, 8, 4, (3, 4))])
def test_two_rank_partition_matches_one_oracle(L, T, B, E, R, empty):
    seed, n_reads = 11 + L, 5000
    res = run_ranks(2, L, T, B, E, R, seed, empty, n_reads)
    counts, values = case(L, T, B, E, R, seed, empty)
    o = oracle.OracleGGArray(L, T, B, E)
    o.insert(counts, values)
    want_off = o.offsets().astype(np.int64).tobytes()
    N = o.size()
    idx = wl.uniform_indices(seed + 1, n_reads, N)
    want_reads, rc = o.read(idx)
    assert rc == oracle.OK
    flat = o.flatten()
    pieces = []
    for rank, off, got, start, part in res:
        assert off == want_off                                      # the all-gathered global offsets
        assert got == want_reads.tobytes()                          # routed reads, in request order
        pieces.append((start, part))
    assert b"".join(p for _, p in sorted(pieces)) == flat.tobytes()  # slices tile the flattened array
    assert sorted(pieces)[0][0] == 0


def test_lfvector_ranges_tile_the_array():
    for L in (1, 2, 7, 1024, 1025):
        for world in (1, 2, 3, 8):
            rs = [partition.lfv_range(L, world, r) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == L
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
            assert max(b - a for a, b in rs) - min(b - a for a, b in rs) <= 1
