"""Theoretical memory use (the paper's Sec. V): an array of N elements
receives N * F more, F ~ LogNormal(mu = 0, sigma), so the needed memory is
S = N (1 + F) elements.

* static: allocated once so that it overflows in at most `fail` of the runs:
  N (1 + exp(sigma * z)), z the (1 - fail) quantile of the standard normal
  (closed form).
* semi-static (host-resized doubling from N): the least N * 2^k >= S; while
  a resize copies, the old and the new buffer are both held (peak 1.5x the
  new capacity).
* GGArray: S split evenly over L LFVectors (the first S mod L get one more);
  LFVector capacity is the least B (2^k - 1) covering its share (Algorithm
  2's doubling buckets, allocated only when reached).

All three are reported as memory / needed, averaged over Monte Carlo draws
of F (and, for the GGArray, also the largest ratio seen).  Plain host code.
"""

from __future__ import annotations

import math
from dataclasses import dataclass
from statistics import NormalDist

import numpy as np


def static_elems(N: int, sigma: float, fail: float = 0.01) -> float:
    """Static capacity that holds N (1 + F) in all but `fail` of the runs."""
    z = NormalDist().inv_cdf(1.0 - fail)
    return N * (1.0 + math.exp(sigma * z))


def ggarray_capacity(size: int, B: int) -> int:
    """Least B (2^k - 1) >= size (0 when size is 0): the capacity of one
    LFVector whose buckets of B * 2^b elements are allocated when reached."""
    if size <= 0:
        return 0
    k = max(0, math.ceil(math.log2(size / B + 1)) - 1)
    while B * ((1 << k) - 1) < size:
        k += 1
    return B * ((1 << k) - 1)


def ggarray_elems(S: int, L: int, B: int) -> int:
    q, r = divmod(int(S), L)
    return r * ggarray_capacity(q + 1, B) + (L - r) * ggarray_capacity(q, B)


def semi_static_elems(N: int, S: int):
    """(final capacity, peak during the last resize)."""
    cap = N
    while cap < S:
        cap *= 2
    return cap, (cap + cap // 2 if cap > N else cap)


@dataclass
class ModelRow:
    sigma: float
    static: float
    semi_static: float
    semi_static_peak: float
    ggarray: float
    ggarray_max: float


def model(N: int = 1 << 24, L: int = 1024, B: int = 4096, sigmas=None, draws: int = 4000, seed: int = 8,
          fail: float = 0.01):
    """Memory / needed for sigma in [0, 2] (Sec. V)."""
    if sigmas is None:
        sigmas = [0.25 * i for i in range(9)]
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(draws)
    rows = []
    for sg in sigmas:
        F = np.exp(sg * z)
        S = np.floor(N * (1.0 + F)).astype(np.int64)
        st = static_elems(N, sg, fail)
        semi = np.array([semi_static_elems(N, int(s)) for s in S], dtype=np.float64)
        gg = np.array([ggarray_elems(int(s), L, B) for s in S], dtype=np.float64)
        rows.append(ModelRow(sigma=sg, static=float(np.mean(st / S)),
                             semi_static=float(np.mean(semi[:, 0] / S)),
                             semi_static_peak=float(np.mean(semi[:, 1] / S)),
                             ggarray=float(np.mean(gg / S)), ggarray_max=float(np.max(gg / S))))
    return rows


if __name__ == "__main__":
    import json
    for r in model():
        print(json.dumps({k: round(v, 4) for k, v in r.__dict__.items()}))
