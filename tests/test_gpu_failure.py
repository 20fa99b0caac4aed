"""Failure detection without a GPU fault (needs a GPU).

The step kernels' device-side waits -- the decoupled look-back on a
predecessor tile's status word, the mbarrier wait for a tile's bulk copies
-- are bounded.  lcs_selftest_waits runs each against a partner that never
answers (a status word nothing publishes, an mbarrier no copy completes)
and must come back, within a second or two, with LCS_ERR_TIMEOUT for both;
the GPU stays usable, which a normal run right after checks.  Host-side
failures (bad arguments, non-finite states, displacements beyond a
neighbour, capacity) are covered by the other GPU test files.
"""
import time

import numpy as np
import pytest

import synth
from helpers import gpu_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lcs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2604_11008_gb300 as m
    from paper_2604_11008_gb300 import build
    build.build()
    return m


def test_bounded_waits_give_up_and_report(lcs):
    t0 = time.perf_counter()
    lookback, mbarrier = lcs.selftest_waits()
    elapsed = time.perf_counter() - t0
    assert lookback == lcs.LCS_ERR_TIMEOUT
    assert mbarrier == lcs.LCS_ERR_TIMEOUT
    assert elapsed < 10.0, elapsed
    # the device is still usable: a normal run completes without error
    field, _, x, v, tau = synth.small_case(700, 16, 16, 3.0, 2000, 0.05, dt=0.01)
    sim = lcs.Simulator(field, x, v, 0.01, tau=tau, sub=(2, 2, 2), sort_every=3)
    sim.step(6)
    st = gpu_state(sim)
    assert np.array_equal(np.sort(st["ids"].astype(np.int64)), np.arange(2000))
