"""The theoretical memory model (Sec. V) against facts that do not depend on
it: the GGArray capacity formula equals the oracle's bucket walk, the static
sizing overflows in the stated fraction of lognormal draws, sigma = 0 has
exact values, and every GGArray draw stays within 2 S + B L."""

import math

import numpy as np
import pytest

import oracle
from paper_2209_00103_gb300 import memory_model as mm


@pytest.mark.parametrize("B", [1, 3, 4, 256, 4096])
def test_ggarray_capacity_matches_oracle(B):
    for size in list(range(0, 300)) + [10 ** 6, 2 ** 28 - 1, 2 ** 28, 2 ** 28 + 1]:
        assert mm.ggarray_capacity(size, B) == oracle.capacity_of(size, B), (size, B)


@pytest.mark.parametrize("sigma", [0.5, 1.0, 2.0])
def test_static_sizing_fails_in_one_percent_of_draws(sigma):
    N = 10 ** 6
    z = np.random.default_rng(3).standard_normal(200_000)
    S = N * (1.0 + np.exp(sigma * z))
    frac = float(np.mean(S > mm.static_elems(N, sigma, 0.01)))
    assert abs(frac - 0.01) < 0.0015


def test_sigma_zero_exact_values():
    N, L, B = 1 << 20, 64, 256
    rows = mm.model(N=N, L=L, B=B, sigmas=[0.0], draws=10)
    r = rows[0]
    assert r.static == pytest.approx(1.0)
    assert r.semi_static == pytest.approx(1.0) and r.semi_static_peak == pytest.approx(1.5)
    per = (2 * N) // L
    want = L * oracle.capacity_of(per, B) / (2 * N)
    assert r.ggarray == pytest.approx(want) and r.ggarray_max == pytest.approx(want)


def test_ggarray_within_twice_plus_first_buckets():
    N, L, B = 1 << 22, 256, 1024
    rng = np.random.default_rng(5)
    for F in np.exp(2.0 * rng.standard_normal(500)):
        S = int(N * (1 + F))
        mem = mm.ggarray_elems(S, L, B)
        assert S <= mem <= 2 * S + B * L
        cap, peak = mm.semi_static_elems(N, S)
        assert S <= cap < 2 * S and peak <= 1.5 * cap
