"""Owned-field mode: every subdomain interpolates only from its own brick of
field cells plus a halo of two (needs a GPU).

This is the memory pattern of the multi-GPU decomposition (Sec. 2.1, 2.3):
the gathered cells and the arithmetic are those of the shared field, so the
state must equal the shared-field run bit for bit, for every field storage,
with one migration per step and with migration after each Runge-Kutta stage,
and meet the FP64 bar against the oracle.  A stencil outside its brick -- a
particle whose predictor lies more than one cell beyond its subdomain -- is
reported; with migration per stage the predictor is owned again before it is
gathered, so the same move is served.
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import L, assert_same_storage, gpu_state, traj_errors

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
    v = np.ascontiguousarray(v + np.random.default_rng(seed).standard_normal(v.shape))
    return field, x, v, tau


def run(lcs, field, x, v, tau, P, steps, **kw):
    sim = lcs.Simulator(field, x, v, 0.01, tau=tau, g=G, sub=P, track_images=True, **kw)
    sim.step(steps)
    st = gpu_state(sim)
    sim.close()
    return st


@pytest.mark.parametrize("per_stage", [False, True])
@pytest.mark.parametrize("kernel,dtype", [("df", "f64"), ("auto", "f32"), ("auto", "bf16")])
def test_owned_equals_shared(lcs, kernel, dtype, per_stage):
    N, P = 24, (2, 3, 2)
    field, x, v, tau = case(600, N, 20000)
    kw = dict(kernel=kernel, field_dtype=dtype, sort_every=5, sort_brick=4,
              migrate_per_stage=per_stage)
    shared = run(lcs, field, x, v, tau, P, 12, **kw)
    owned = run(lcs, field, x, v, tau, P, 12, owned_field=True, **kw)
    for key in ("seg", "ids", "x", "v", "img"):
        assert np.array_equal(owned[key], shared[key]), key


@pytest.mark.parametrize("items", [1, 2])
def test_owned_against_oracle(lcs, items):
    N, P, steps = 24, (3, 2, 2), 20
    field, x, v, tau = case(601, N, 15000)
    sim = lcs.Simulator(field, x, v, 0.01, tau=tau, g=G, sub=P, kernel="df", track_images=True,
                        sort_every=6, sort_brick=4, owned_field=True)
    sim.set_step_config(256, items, lcs.STEP_OWNED_FIELD)
    sim.step(steps)
    st = gpu_state(sim)
    ref = oracle.initial_state(N, L, P, x, v, tau, track_img=True)
    oracle.run(ref, field, L, P, 0.0, 0.01, G, steps, sort_every=6, brick=4)
    ex, ev, px, pv = traj_errors(st["x"], st["img"], st["v"], st["ids"], ref, x)
    assert max(ex, ev, px, pv) < 1e-12, (ex, ev, px, pv)
    assert_same_storage(st, ref, N, P, 4)


@pytest.mark.parametrize("per_stage", [False, True])
@pytest.mark.parametrize("kernel,dtype", [("df", "f64"), ("auto", "f32")])
def test_owned_evolving_field_equals_shared(lcs, kernel, dtype, per_stage):
    # both snapshots have bricks; a snapshot pushed mid-run rebuilds them
    N, P, dt = 24, (2, 2, 3), 0.005
    field, x, v, tau = case(605, N, 12000, dt=dt)
    snaps = [field] + [synth.small_case(606 + k, N, 16, N / 4.0, 1, None)[0] for k in range(2)]
    out = []
    for owned in (False, True):
        sim = lcs.Simulator(snaps[0], x, v, dt, tau=tau, g=G, sub=P, kernel=kernel,
                            field_dtype=dtype, track_images=True, sort_every=4, sort_brick=4,
                            migrate_per_stage=per_stage, owned_field=owned, field_next=snaps[1],
                            t_start=0.0, t_field=(0.0, 0.04))
        sim.step(8)
        sim.set_field(snaps[2], 0.08)
        sim.step(8)
        out.append(gpu_state(sim))
        sim.close()
    for key in ("seg", "ids", "x", "v", "img"):
        assert np.array_equal(out[0][key], out[1][key]), key


def test_thin_subdomains_with_overlapping_halos(lcs):
    # W = 1, 2, 4 cells per subdomain: the halos of neighbours overlap and
    # wrap around the periodic faces
    N, P = 8, (8, 4, 2)
    field, x, _, tau = case(602, N, 6000)
    v = np.zeros_like(x)
    kw = dict(kernel="df", sort_every=3)
    shared = run(lcs, field, x, v, tau, P, 10, **kw)
    owned = run(lcs, field, x, v, tau, P, 10, owned_field=True, **kw)
    for key in ("seg", "ids", "x", "v", "img"):
        assert np.array_equal(owned[key], shared[key]), key


def test_stencil_outside_the_brick_is_reported(lcs):
    # every particle moves 2.5 cells along x per step: within a neighbour
    # subdomain (W = 12 cells), but the predictor of a particle near the
    # upper face of its subdomain lies beyond the halo of two cells
    N, P, dt = 24, (2, 1, 1), 0.01
    field = np.zeros((3, N, N, N))
    rng = np.random.default_rng(603)
    x = np.ascontiguousarray(rng.uniform(0.0, L, (3, 4000)))
    v = np.zeros_like(x)
    v[0] = 2.5 * (L / N) / dt
    kw = dict(tau_const=1.0, sub=P)
    ok = lcs.Simulator(field, x, v, dt, **kw)
    ok.step(1)
    ok.sync()
    bad = lcs.Simulator(field, x, v, dt, owned_field=True, **kw)
    with pytest.raises(lcs.LcsError) as e:
        bad.step(1)
        bad.sync()
    assert e.value.status == lcs.LCS_ERR_DISPLACEMENT
    # migrating after each stage hands the particle to the predictor's owner
    per_stage = lcs.Simulator(field, x, v, dt, owned_field=True, migrate_per_stage=True, **kw)
    per_stage.step(2)
    per_stage.sync()
    ref = lcs.Simulator(field, x, v, dt, migrate_per_stage=True, **kw)
    ref.step(2)
    a, b = gpu_state(per_stage), gpu_state(ref)
    for key in ("seg", "ids", "x", "v"):
        assert np.array_equal(a[key], b[key]), key


def test_owned_field_arguments(lcs):
    N = 16
    field, x, v, tau = case(604, N, 500)
    for kw in (dict(kernel="fp64"), dict(ckpt_every=4, track_images=True)):
        with pytest.raises(lcs.LcsError) as e:
            lcs.Simulator(field, x, v, 0.01, tau=tau, sub=(2, 2, 2), owned_field=True, **kw)
        assert e.value.status == lcs.LCS_ERR_ARG, kw
    owned = lcs.Simulator(field, x, v, 0.01, tau=tau, sub=(2, 2, 2), owned_field=True)
    shared = lcs.Simulator(field, x, v, 0.01, tau=tau, sub=(2, 2, 2))
    for sim, cfg in ((owned, (256, 2, lcs.STEP_DEFERRED)), (shared, (256, 2, lcs.STEP_OWNED_FIELD))):
        with pytest.raises(lcs.LcsError) as e:
            sim.set_step_config(*cfg)
        assert e.value.status == lcs.LCS_ERR_ARG
    assert owned.tune(1)[2] == lcs.STEP_OWNED_FIELD
    assert (owned.tune_trials_ms[:12] == -1).all() and (owned.tune_trials_ms[12:] > 0).all()
    spec = dict(field=field, x0=x, v0=v, dt=0.01, tau=tau, sub=(2, 2, 2))
    with pytest.raises(lcs.LcsError) as e:
        lcs.Simulator(None, None, None, None, ensembles=[dict(spec, owned_field=True), spec])
    assert e.value.status == lcs.LCS_ERR_ARG


def test_owned_field_in_a_batch_of_uneven_ensembles(lcs):
    # three ensembles of different grids and subdomain shapes in one
    # context: each reads its own bricks through the shared launches
    specs = []
    for k, (N, P) in enumerate(((16, (2, 2, 2)), (24, (3, 2, 1)), (12, (1, 3, 2)))):
        field, x, v, tau = case(610 + k, N, 3000 + 2000 * k)
        specs.append(dict(field=field, x0=x, v0=v, dt=0.01, tau=tau, g=G, sub=P, kernel="df",
                          sort_every=4, track_images=True))
    out = []
    for owned in (False, True):
        sim = lcs.Simulator(None, None, None, None,
                            ensembles=[dict(sp, owned_field=owned) for sp in specs])
        sim.step(9)
        out.append([gpu_state(sim, k) for k in range(len(specs))])
        sim.close()
    for k in range(len(specs)):
        for key in ("seg", "ids", "x", "v", "img"):
            assert np.array_equal(out[0][k][key], out[1][k][key]), (k, key)
