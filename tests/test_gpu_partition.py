"""The partitioned GGArray's local part on the GPU (one rank: the library's
GGArray through GGArrayPart): offsets, reads and the flatten slice equal the
oracle's.  The exchange between ranks is tested on CPU ranks over gloo
(test_partition_host.py); every GPU run of this project has one GPU."""

import numpy as np
import pytest
import torch

import oracle
from paper_2209_00103_gb300 import gga, partition
from paper_2209_00103_gb300 import workloads as wl

from harness import counts_to_dev, dev_to_np, make_pair, packed_values, random_counts, values_to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("E", [4, 16])
def test_single_rank_partition_on_the_gpu(E):
    rng = np.random.default_rng(3 + E)
    L, T, B = 9, 64, 8
    counts = random_counts(rng, 6, L, T)
    values = packed_values(int(counts.sum()), E, seed=E)
    g, o = make_pair(L, T, B, E, pool_bytes=64 << 20)
    g.insert(counts_to_dev(counts), values_to_dev(values, E))
    o.insert(counts, values)
    p = partition.PartitionedGGArray(partition.GGArrayPart(g), L, 1, 0, device=torch.device("cuda"))
    off = p.sync()
    assert np.array_equal(off.cpu().numpy().astype(np.uint64), o.offsets())
    idx = wl.uniform_indices(5, 4000, o.size())
    got = dev_to_np(p.read(torch.from_numpy(idx.view(np.int64)).cuda()), E)
    want, rc = o.read(idx)
    assert rc == oracle.OK and got.tobytes() == want.tobytes()
    start, part = p.flatten()
    assert start == 0 and dev_to_np(part, E).tobytes() == o.flatten().tobytes()
    g.close()
