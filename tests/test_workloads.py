"""The numpy and torch implementations of the input generator agree draw
for draw (both feed the oracle and the CUDA path)."""

import numpy as np
import pytest
import torch

from paper_2209_00103_gb300 import workloads as wl


def test_splitmix_numpy_torch_agree():
    keys = np.arange(5000, dtype=np.uint64) * np.uint64(7919) + np.uint64(3)
    a = wl.splitmix_at(12345, keys)
    b = wl.splitmix_at_t(12345, torch.from_numpy(keys.view(np.int64))).numpy().view(np.uint64)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("E", [4, 8, 16])
@pytest.mark.parametrize("dist", ["bernoulli", "uniform3", "geometric", "poisson"])
def test_insert_inputs_numpy_torch_agree(dist, E):
    spec = wl.InsertSpec(L=3, T=40, E=E, seed=5, dist=dist, rounds=3, round0=4,
                         coeffs=(10, 1 << 20, (1 << 63) + 5), thresholds=wl.poisson1_thresholds())
    c_np, v_np = spec.make()
    c_t, v_t = wl.make_insert_inputs_t(spec, "cpu")
    assert np.array_equal(c_np.view(np.int32), c_t.numpy())
    assert v_np.tobytes() == v_t.contiguous().numpy().tobytes()


def test_indices_numpy_torch_agree():
    a = wl.uniform_indices(9, 3000, 123457)
    b = wl.uniform_indices_t(9, 3000, 123457, "cpu").numpy()
    assert np.array_equal(a.astype(np.int64), b)
    for E in (4, 8, 16):
        va = wl.index_keyed_values(4, a, E)
        vb = wl.index_keyed_values_t(4, torch.from_numpy(a.view(np.int64)), E)
        assert va.tobytes() == vb.contiguous().numpy().tobytes()


def test_gtid0_gives_one_blocks_inputs_of_a_larger_spec():
    # The inputs of block 4 of a 6-block spec, drawn on their own with
    # gtid0 = 4*T: the same counts and the same values, in the same order.
    kw = dict(T=32, E=4, seed=3, dist="uniform3", rounds=5, coeffs=(3, 1 << 20, 1 << 9))
    c, v = wl.InsertSpec(L=6, **kw).make()
    cp, vp = wl.InsertSpec(L=1, gtid0=4 * 32, **kw).make()
    assert np.array_equal(cp[:, 0, :], c[:, 4, :])
    flat = c.reshape(-1).astype(np.int64)
    starts = np.cumsum(flat) - flat
    sel = [v[int(starts[(r * 6 + 4) * 32]):int(starts[(r * 6 + 4) * 32]) + int(c[r, 4].sum())] for r in range(5)]
    assert np.array_equal(np.concatenate(sel), vp)
