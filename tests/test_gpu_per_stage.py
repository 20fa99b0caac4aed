"""Migration after each Runge-Kutta stage (Sec. 3.2.2), needs a GPU.

With migrate_per_stage the particles move to the subdomain of their
predictor position X* before the second stage and again after X'.  The
storage order after every step must equal the oracle's per-stage migration
(bit for bit as per-subdomain id lists on the same inputs, up to particles
straddling a face), and the trajectories those of the single-migration step.
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import L, assert_same_storage, by_id, gpu_state, traj_errors

pytestmark = pytest.mark.gpu

G = (0.0, 0.0, -9.8)


@pytest.fixture(scope="module")
def lcs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2604_11008_gb300 as m
    from paper_2604_11008_gb300 import build
    build.build()
    return m


def case(seed, N, n, dt=0.01):
    field, _, x, v, tau = synth.small_case(seed, N, 16, N / 4.0, n, 0.05, dt=dt)
    v = np.ascontiguousarray(v + 2.0 * np.random.default_rng(seed).standard_normal(v.shape))
    return field, x, v, tau


@pytest.mark.parametrize("kernel,dtype,tol", [("df", "f64", 1e-12), ("fp64", "f64", 1e-12),
                                              ("auto", "f32", 1e-5), ("auto", "bf16", 1e-2)])
def test_per_stage_against_oracle(lcs, kernel, dtype, tol):
    N, P, steps = 24, (3, 2, 2), 20
    field, x, v, tau = case(400, N, 20000)
    sim = lcs.Simulator(field, x, v, 0.01, tau=tau, g=G, sub=P, kernel=kernel, field_dtype=dtype,
                        track_images=True, sort_every=6, sort_brick=4, migrate_per_stage=True)
    sim.step(steps)
    st = gpu_state(sim)
    ref = oracle.initial_state(N, L, P, x, v, tau, track_img=True)
    oracle.run(ref, field, L, P, 0.0, 0.01, G, steps, sort_every=6, brick=4, per_stage=True)
    ex, ev, px, pv = traj_errors(st["x"], st["img"], st["v"], st["ids"], ref, x)
    assert max(ex, ev, px, pv) < tol, (ex, ev, px, pv)
    if tol == 1e-12:
        assert_same_storage(st, ref, N, P, 4)


def test_per_stage_and_single_migration_agree_up_to_order(lcs):
    N, P = 24, (2, 3, 2)
    field, x, v, tau = case(401, N, 30000)
    out = []
    for per_stage in (False, True):
        sim = lcs.Simulator(field, x, v, 0.01, tau=tau, g=G, sub=P, kernel="df",
                            track_images=True, sort_every=0, migrate_per_stage=per_stage)
        sim.step(7)
        out.append(gpu_state(sim))
        sim.close()
    a, b = out
    assert np.array_equal(a["seg"], b["seg"]) and not np.array_equal(a["ids"], b["ids"])
    xa, va, ia = by_id(a["ids"], a["x"], a["v"], a["img"])
    xb, vb, ib = by_id(b["ids"], b["x"], b["v"], b["img"])
    assert np.abs((xa + L * ia) - (xb + L * ib)).max() < 1e-12
    assert np.abs(va - vb).max() < 1e-12 * np.abs(va).max()


@pytest.mark.parametrize("kernel,dtype,tol,items", [("df", "f64", 1e-12, 1),
                                                    ("df", "f64", 1e-12, 2),
                                                    ("fp64", "f64", 1e-12, 1),
                                                    ("auto", "f32", 1e-5, 2)])
def test_per_stage_with_evolving_field_against_oracle(lcs, kernel, dtype, tol, items):
    # stage 1 sees the field at t_n, stage 2 (after the particles moved to
    # the owner of X*) at t_n + dt; the step counter advances once per step
    N, P, steps, dt = 24, (2, 3, 2), 16, 0.005
    field, x, v, tau = case(430, N, 15000, dt=dt)
    field2 = synth.small_case(431, N, 16, N / 4.0, 1, None)[0]
    times = (0.0, 0.06)
    sim = lcs.Simulator(field, x, v, dt, tau=tau, g=G, sub=P, kernel=kernel, field_dtype=dtype,
                        track_images=True, sort_every=5, sort_brick=4, migrate_per_stage=True,
                        field_next=field2, t_start=0.01, t_field=times)
    sim.set_step_config(256, items, 3)
    sim.step(steps)
    st = gpu_state(sim)
    ref = oracle.initial_state(N, L, P, x, v, tau, track_img=True)
    oracle.run(ref, field, L, P, 0.0, dt, G, steps, sort_every=5, brick=4, per_stage=True,
               field_b=field2, t_start=0.01, t_field=times)
    ex, ev, px, pv = traj_errors(st["x"], st["img"], st["v"], st["ids"], ref, x)
    assert max(ex, ev, px, pv) < tol, (ex, ev, px, pv)
    if tol == 1e-12:
        assert_same_storage(st, ref, N, P, 4)
    # the time dependence matters: the frozen field lands far away
    frozen = oracle.initial_state(N, L, P, x, v, tau, track_img=True)
    oracle.run(frozen, field, L, P, 0.0, dt, G, steps, sort_every=5, brick=4, per_stage=True)
    _, ev_f, _, _ = traj_errors(st["x"], st["img"], st["v"], st["ids"], frozen, x)
    assert ev_f > 1e-3, ev_f


def test_per_stage_configurations_and_batches_agree(lcs):
    N = 16
    specs = []
    for k in range(3):
        field, x, v, tau = case(410 + k, N, 4000 + 3000 * k)
        specs.append(dict(field=field, x0=x, v0=v, dt=0.01, tau=tau, g=G, sub=(2, 2, 2),
                          kernel="df", sort_every=3, track_images=True, migrate_per_stage=True))
    res = []
    for cfg in ((256, 1, 3), (256, 2, 3)):
        batch = lcs.Simulator(None, None, None, None, ensembles=specs)
        batch.set_step_config(*cfg)
        batch.step(8)
        res.append([gpu_state(batch, k) for k in range(3)])
        batch.close()
    for k in range(3):
        for key in ("seg", "ids", "x", "v", "img"):
            assert np.array_equal(res[0][k][key], res[1][k][key]), (k, key)
    sp = specs[2]
    solo = lcs.Simulator(**{kk: vv for kk, vv in sp.items() if kk not in ("field", "x0", "v0", "dt")},
                         field=sp["field"], x0=sp["x0"], v0=sp["v0"], dt=sp["dt"])
    solo.set_step_config(256, 1, 3)
    solo.step(8)
    s = gpu_state(solo)
    for key in ("seg", "ids", "x", "v"):
        assert np.array_equal(s[key], res[0][2][key]), key


def test_per_stage_arguments(lcs):
    N = 16
    field, x, v, tau = case(420, N, 200)
    with pytest.raises(lcs.LcsError) as e:
        lcs.Simulator(field, x, v, 0.01, tau=tau, migrate_per_stage=True, ckpt_every=4,
                      track_images=True)
    assert e.value.status == lcs.LCS_ERR_ARG
    sim = lcs.Simulator(field, x, v, 0.01, tau=tau, migrate_per_stage=True)
    for cfg in ((256, 2, 0), (128, 2, 3)):
        with pytest.raises(lcs.LcsError) as e:
            sim.set_step_config(*cfg)
        assert e.value.status == lcs.LCS_ERR_ARG
    cfg = sim.tune(1)
    assert cfg in ((256, 2, 3), (256, 1, 3))
    mixed = [dict(field=field, x0=x, v0=v, dt=0.01, tau=tau, migrate_per_stage=m)
             for m in (True, False)]
    with pytest.raises(lcs.LcsError) as e:
        lcs.Simulator(None, None, None, None, ensembles=mixed)
    assert e.value.status == lcs.LCS_ERR_ARG
