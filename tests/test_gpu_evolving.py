"""Evolving field: U(X, t) linear in time between two snapshots (needs a GPU).

The fluid velocity of Eq. (6) is U(X, t) = (1 - th) U_a(X) + th U_b(X),
th = (t - t_a)/(t_b - t_a), with the Heun stages of step n at t_n = t_start +
n dt and t_n + dt.  Against the oracle on the same inputs: the FP64 and
float-float kernels within the FP64 bar, FP32/BF16 storage within theirs;
pushing a new snapshot mid-run continues the same time axis.
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import L, assert_same_storage, gpu_state, traj_errors

pytestmark = pytest.mark.gpu

DT = 0.005


@pytest.fixture(scope="module")
def lcs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2604_11008_gb300 as m
    from paper_2604_11008_gb300 import build
    build.build()
    return m


def fields(seed, N, count):
    """`count` independent snapshots with the same spectrum shape."""
    return [synth.small_case(seed + k, N, 32, 6.0, 1, None)[0] for k in range(count)]


def particles(seed, N, n):
    _, _, x, v, tau = synth.small_case(seed, N, 8, 2.0, n, 0.05, dt=DT)
    return x, v, tau


def oracle_run(x, v, tau, P, snaps, times, t_start, segments, sort_every=0, brick=4):
    """segments: [(steps, index of the first snapshot)], snapshot k at times[k]."""
    N = snaps[0].shape[-1]
    ref = oracle.initial_state(N, L, P, x, v, tau, track_img=True)
    k0 = 0
    for steps, s in segments:
        oracle.run(ref, snaps[s], L, P, 0.0, DT, (0.0, 0.0, -9.8), steps, sort_every=sort_every,
                   brick=brick, step0=k0, field_b=snaps[s + 1], t_start=t_start,
                   t_field=(times[s], times[s + 1]))
        k0 += steps
    return ref


@pytest.mark.parametrize("kernel,dtype,tol", [("fp64", "f64", 1e-12), ("df", "f64", 1e-12),
                                              ("auto", "f32", 1e-5), ("auto", "bf16", 1e-2)])
def test_evolving_field_against_oracle(lcs, kernel, dtype, tol):
    N, P = 24, (2, 2, 3)
    snaps = fields(200, N, 2)
    times = (0.0, 0.1)
    x, v, tau = particles(201, N, 15000)
    sim = lcs.Simulator(snaps[0], x, v, DT, tau=tau, g=(0.0, 0.0, -9.8), sub=P, kernel=kernel,
                        field_dtype=dtype, track_images=True, sort_every=5, sort_brick=4,
                        field_next=snaps[1], t_start=0.02, t_field=times)
    sim.step(30)   # t from 0.02 to 0.17: past t_b, the field extrapolates linearly
    st = gpu_state(sim)
    ref = oracle_run(x, v, tau, P, snaps, times, 0.02, [(30, 0)], sort_every=5)
    ex, ev, px, pv = traj_errors(st["x"], st["img"], st["v"], st["ids"], ref, x)
    assert max(ex, ev, px, pv) < tol, (ex, ev, px, pv)
    if tol == 1e-12:
        assert_same_storage(st, ref, N, P, 4)
        # the time dependence matters: the frozen first snapshot lands far away
        frozen = oracle.initial_state(N, L, P, x, v, tau, track_img=True)
        oracle.run(frozen, snaps[0], L, P, 0.0, DT, (0.0, 0.0, -9.8), 30, sort_every=5, brick=4)
        _, ev_f, _, _ = traj_errors(st["x"], st["img"], st["v"], st["ids"], frozen, x)
        assert ev_f > 1e-3, ev_f


@pytest.mark.parametrize("kernel", ["df", "fp64"])
def test_pushing_snapshots_continues_the_time_axis(lcs, kernel):
    N, P = 16, (2, 1, 2)
    snaps = fields(210, N, 4)
    times = (0.0, 0.05, 0.1, 0.15)
    x, v, tau = particles(211, N, 8000)
    sim = lcs.Simulator(snaps[0], x, v, DT, tau=tau, g=(0.0, 0.0, -9.8), sub=P, kernel=kernel,
                        track_images=True, field_next=snaps[1], t_start=0.0,
                        t_field=times[:2])
    sim.step(10)                      # t 0 -> 0.05
    sim.set_field(snaps[2], times[2])
    sim.step(10)                      # t 0.05 -> 0.1
    sim.set_field(snaps[3], times[3])
    sim.step(7)
    st = gpu_state(sim)
    ref = oracle_run(x, v, tau, P, snaps, times, 0.0, [(10, 0), (10, 1), (7, 2)])
    ex, ev, px, pv = traj_errors(st["x"], st["img"], st["v"], st["ids"], ref, x)
    assert max(ex, ev, px, pv) < 1e-12, (ex, ev, px, pv)
    # the first snapshot of the context is now snaps[2] (float pairs: 2^-48)
    got = sim.get_field().cpu().numpy()
    assert np.abs(got - snaps[2]).max() <= 2.0 ** -47 * np.abs(snaps[2]).max()


def test_batch_mixes_frozen_and_evolving_ensembles(lcs):
    N = 16
    snaps = fields(220, N, 2)
    specs = []
    for k in range(3):
        x, v, tau = particles(230 + k, N, 3000 + 1000 * k)
        sp = dict(field=snaps[0], x0=x, v0=v, dt=DT, tau=tau, sub=(2, 2, 2), kernel="df",
                  sort_every=4, track_images=True)
        if k != 1:
            sp.update(field_next=snaps[1], t_start=0.01 * k, t_field=(0.0, 0.2))
        specs.append(sp)
    batch = lcs.Simulator(None, None, None, None, ensembles=specs)
    batch.set_step_config(256, 2, 3)
    batch.step(12)
    for k, sp in enumerate(specs):
        solo = lcs.Simulator(**{kk: vv for kk, vv in sp.items()
                                if kk not in ("field", "x0", "v0", "dt")},
                             field=sp["field"], x0=sp["x0"], v0=sp["v0"], dt=sp["dt"])
        solo.set_step_config(256, 2, 3)
        solo.step(12)
        a, b = gpu_state(batch, k), gpu_state(solo)
        for key in ("seg", "ids", "x", "v"):
            assert np.array_equal(a[key], b[key]), (k, key)
        solo.close()


def test_evolving_field_arguments(lcs):
    N = 16
    snaps = fields(240, N, 2)
    x, v, tau = particles(241, N, 100)
    with pytest.raises(lcs.LcsError) as e:
        lcs.Simulator(snaps[0], x, v, DT, tau=tau, field_next=snaps[1], t_field=(0.1, 0.1))
    assert e.value.status == lcs.LCS_ERR_ARG
    with pytest.raises(lcs.LcsError) as e:
        lcs.Simulator(snaps[0], x, v, DT, tau=tau, field_next=snaps[1], ckpt_every=4,
                      track_images=True)
    assert e.value.status == lcs.LCS_ERR_ARG
    sim = lcs.Simulator(snaps[0], x, v, DT, tau=tau, field_next=snaps[1], t_field=(0.0, 1.0))
    with pytest.raises(lcs.LcsError) as e:
        sim.set_field(snaps[0], 0.5)          # not after t_b
    assert e.value.status == lcs.LCS_ERR_ARG
    sim.step(2)                               # a refused call latches nothing
    sim.sync()
    frozen = lcs.Simulator(snaps[0], x, v, DT, tau=tau)
    with pytest.raises(lcs.LcsError) as e:
        frozen.set_field(snaps[1], 2.0)
    assert e.value.status == lcs.LCS_ERR_ARG
