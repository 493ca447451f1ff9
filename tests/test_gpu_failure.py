"""Failure detection without a GPU fault: a bounded wait that nothing
completes gives up and reports GGA_ERR_TIMEOUT through a status word, and the
context stays usable (the same process then runs normal work)."""

import numpy as np
import pytest
import torch

import oracle
from paper_2209_00103_gb300 import gga

from harness import assert_same_state, insert_both, make_pair, packed_values, random_counts

pytestmark = pytest.mark.gpu


def test_bounded_wait_completes_when_the_barrier_does():
    assert gga.gga_debug_wait_timeout(1000, True) == gga.GGA_OK


def test_bounded_wait_gives_up_and_reports_timeout():
    assert gga.gga_debug_wait_timeout(2000, False) == gga.GGA_ERR_TIMEOUT
    # The context is still usable.
    rng = np.random.default_rng(3)
    g, o = make_pair(8, 64, 256, 4, expected_elems=20000)
    counts = random_counts(rng, 5, 8, 64)
    insert_both(g, o, counts, packed_values(int(counts.sum()), 4, 1), 4)
    assert_same_state(g, o)
    g.close()
    assert gga.gga_debug_wait_timeout(10, True) == gga.GGA_OK
