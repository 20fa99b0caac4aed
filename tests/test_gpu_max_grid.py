"""The largest grid the fixed-point positions allow: N = 1024 (positions are
x N/L * 2^52 in an int64, and 1024 * 2^52 = 2^62).  A 1024^3 field of a few
Fourier modes (25.8 GB as FP64, 34 GB as the library's float-pair copy),
4096 particles spread over the box plus particles on its faces, on cell
faces and on subdomain faces, 20 steps with migration and a cell sort after
every fifth step (27-bit cell keys: three radix passes), against the FP64
oracle: storage order and trajectories.  The particles start with random
velocities and move about a cell per step: the relative position error is
measured against the displacement, whose FP64 rounding floor (ulp(L)/2 per
step in the oracle) must stay well below the bar.
"""
import os

import numpy as np
import pytest

import oracle
import synth
from helpers import L, assert_same_storage, gpu_state, traj_errors

pytestmark = pytest.mark.gpu

N = 1024


@pytest.fixture(scope="module")
def lcs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    free, _ = torch.cuda.mem_get_info()
    if free < 80 * 2**30:
        pytest.skip("needs 80 GB of free device memory")
    if os.sysconf("SC_PHYS_PAGES") * os.sysconf("SC_PAGE_SIZE") < 96 * 2**30:
        pytest.skip("needs 96 GB of host memory for the oracle's copy of the field")
    import paper_2604_11008_gb300 as m
    from paper_2604_11008_gb300 import build
    build.build()
    return m


def test_max_grid_against_oracle(lcs):
    import torch
    modes = synth.draw_modes(6, 1.0, 6.0, synth.rng(1024, synth.STREAM_FIELD))
    field_d = synth.field_from_modes(modes, N, device="cuda")
    dt = 0.002
    g = synth.rng(1024, synth.STREAM_POS)
    x = synth.positions(4096, g)
    dx = L / N
    # particles on the box faces, just inside them, on cell faces and on the
    # faces between the 2 x 2 x 2 subdomains
    edge = np.array([0.0, np.nextafter(L, 0.0), dx, 511 * dx, 512 * dx, L / 2,
                     np.nextafter(L / 2, 0.0), 1023 * dx])
    extra = np.stack([np.resize(edge, 64), np.resize(edge[::-1], 64),
                      np.resize(np.roll(edge, 3), 64)])
    x = np.concatenate([x, extra], axis=1)
    n = x.shape[1]
    v = np.random.default_rng(1025).normal(0.0, 1.5, size=x.shape)
    tau = synth.lognormal_tau(n, 0.05, 0.5, dt, synth.rng(1024, synth.STREAM_TAU))
    P, steps, every = (2, 2, 2), 20, 5
    sim = lcs.Simulator(field_d, x, v, dt, tau=tau, sub=P, g=(0.0, 0.0, -9.8), sort_every=every,
                        sort_brick=8, track_images=True, kernel="df")
    sim.step(steps)
    st = gpu_state(sim)
    sim.close()
    field = field_d.cpu().numpy()
    del field_d
    torch.cuda.empty_cache()
    ref = oracle.initial_state(N, L, P, x, v, tau, track_img=True)
    oracle.run(ref, field, L, P, 0.0, dt, (0.0, 0.0, -9.8), steps, sort_every=every, brick=8)
    del field
    assert_same_storage(st, ref, N, P, brick=8)
    ex, ev, px, pv = traj_errors(st["x"], st["img"], st["v"], st["ids"], ref, x)
    assert max(ex, ev, px, pv) < 1e-12, (ex, ev, px, pv)
