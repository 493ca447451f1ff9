"""Parity at full size: the paper-shaped growth workload (1024 blocks x 512
threads, first bucket 4096 int32, 512 rounds of Uniform{0,1,2}, ~2^28
elements), in the launch configuration bench.py times, against the oracle
on every element: sizes, capacities, offsets, 2^26 random reads, 2^26
random writes, both sweeps and the flattened array."""

import numpy as np
import pytest
import torch

import oracle
from paper_2209_00103_gb300 import gga
from paper_2209_00103_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_paper_growth_full_size():
    w = wl.paper_growth()
    dev = torch.device("cuda", 0)
    counts_t, values_t = wl.make_insert_inputs_t(w.spec, dev)
    N = int(values_t.shape[0])
    assert abs(N - (1 << 28)) < 200000
    g = gga.GGArray(w.L, w.T, w.B, w.E, int(2.5 * N * 4) + w.L * w.B * 16)
    g.insert(counts_t, values_t)
    counts = counts_t.cpu().numpy().view(np.uint32)
    values = values_t.cpu().numpy().view(np.uint32)
    del counts_t, values_t
    o = oracle.OracleGGArray(w.L, w.T, w.B, w.E)
    o.insert(counts, values)
    del counts, values

    n, rc, sizes, caps = g.sizes_caps()
    assert rc == gga.GGA_OK and n == o.size() == N
    assert np.array_equal(sizes.cpu().numpy().astype(np.uint64), o.sizes())
    ocaps, _ = o.capacities()
    assert np.array_equal(caps.cpu().numpy().astype(np.uint64), ocaps)
    assert np.array_equal(g.offsets().cpu().numpy().astype(np.uint64), o.offsets())
    mem = g.memory()
    assert mem["bucket_bytes"] == o.bucket_bytes()
    assert mem["bucket_bytes"] / mem["live_bytes"] <= 2.0          # the paper's <= 2x memory claim

    idx_r = wl.uniform_indices_t(w.read_seed, w.n_random, N, dev)
    got = g.read(idx_r).cpu().numpy().view(np.uint32)
    want, orc = o.read(idx_r.cpu().numpy().view(np.uint64))
    assert orc == oracle.OK and np.array_equal(got, want)
    del got, want

    idx_w = wl.uniform_indices_t(w.write_seed, w.n_random, N, dev)
    vals_w = wl.index_keyed_values_t(w.value_seed, idx_w, 4)
    g.write(idx_w, vals_w)
    assert o.write(idx_w.cpu().numpy().view(np.uint64), vals_w.cpu().numpy().view(np.uint32)) == oracle.OK

    g.sweep(gga.GGA_RW_B, 1, 1)
    o.sweep_add(1, 1)
    dst = gga.elem_tensor(N, 4, dev)
    g.flatten(dst)
    assert np.array_equal(dst.cpu().numpy().view(np.uint32), o.flatten())
    g.sweep(gga.GGA_RW_G, 1, 1)
    o.sweep_add(1, 1)
    g.flatten(dst)
    assert np.array_equal(dst.cpu().numpy().view(np.uint32), o.flatten())
    assert g.last_error() == gga.GGA_OK
    g.close()


def test_paper_growth_generated_full_size():
    # The in-kernel generated insertion of the same workload: same contents.
    w = wl.paper_growth()
    N = None
    g1 = gga.GGArray(w.L, w.T, w.B, w.E, 3 << 30)
    g1.insert_generated(gga.make_gen_spec(w.spec.seed, w.spec.dist, w.spec.coeffs), w.spec.rounds)
    counts_t, values_t = wl.make_insert_inputs_t(w.spec, torch.device("cuda", 0))
    N = int(values_t.shape[0])
    g2 = gga.GGArray(w.L, w.T, w.B, w.E, 3 << 30)
    g2.insert(counts_t, values_t)
    del counts_t, values_t
    n1, rc1 = g1.size()
    n2, rc2 = g2.size()
    assert rc1 == rc2 == gga.GGA_OK and n1 == n2 == N
    assert torch.equal(g1.flatten(), g2.flatten())
    assert torch.equal(g1.offsets(), g2.offsets())
    g1.close()
    g2.close()
