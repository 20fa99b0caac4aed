"""Shared-memory staging in the step kernel (needs a GPU).

Mode 1 copies the box of field cells around each tile's particles into shared
memory and interpolates from there (a tile whose box does not fit reads global
memory); mode 2 brings each block's next tile of particle records into shared
memory with bulk asynchronous copies while the current tile is processed;
mode 3 integrates a block's next tile before resolving the previous tile's
scan prefix, parking that tile in shared memory.  The values read are the
same either way, so every configuration must
reproduce the plain kernel's state bit for bit; the staged-tile counter shows
which path the mode-1 tiles took.
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import L, assert_same_storage, gpu_state, traj_errors

pytestmark = pytest.mark.gpu

UNSTAGED = (256, 2, 0)
STAGED = ((256, 2, 1), (128, 2, 1))
PREFETCH = ((256, 2, 2), (128, 2, 2), (256, 1, 2))
DEFERRED = ((256, 2, 3), (128, 2, 3), (256, 1, 3), (128, 1, 3))


@pytest.fixture(scope="module")
def lcs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2604_11008_gb300 as m
    from paper_2604_11008_gb300 import build
    build.build()
    return m


def dense_case(seed, N, n, tau_median=0.05, g=(0.0, 0.0, -9.8)):
    """Many particles per cell, cell-sorted every step: tiles cover a few
    cells, so their boxes fit (and wrap around the periodic faces)."""
    field, _, x, v, tau = synth.small_case(seed, N, 12, N / 4.0, n, tau_median, dt=0.01)
    return dict(field=field, x0=x, v0=v, dt=0.01, tau=tau, tau_const=0.1, g=g)


def run(lcs, case, cfg, steps, **kw):
    sim = lcs.Simulator(case["field"], case["x0"], case["v0"], case["dt"], tau=case["tau"],
                        tau_const=case["tau_const"], g=case["g"], track_images=True, **kw)
    sim.set_step_config(*cfg)
    sim.step(steps)
    st = gpu_state(sim)
    staged = sim.staged_tiles
    sim.close()
    return st, staged


@pytest.mark.parametrize("kernel,dtype", [("df", "f64"), ("auto", "f32"), ("auto", "bf16")])
def test_staged_equals_unstaged_sorted(lcs, kernel, dtype):
    case = dense_case(900, 12, 60000)
    kw = dict(sub=(2, 2, 3), sort_every=1, sort_brick=2, kernel=kernel, field_dtype=dtype)
    ref, n0 = run(lcs, case, UNSTAGED, 7, **kw)
    assert n0 == 0
    for cfg in STAGED:
        st, n = run(lcs, case, cfg, 7, **kw)
        assert n > 0, cfg      # boxes of sorted tiles fit
        for key in ("seg", "ids", "x", "v", "img"):
            assert np.array_equal(st[key], ref[key]), (cfg, key)


@pytest.mark.parametrize("kernel,dtype", [("df", "f64"), ("auto", "f32")])
def test_staged_falls_back_when_boxes_do_not_fit(lcs, kernel, dtype):
    # unsorted particles spread over a 40^3 grid: each tile's box is the
    # whole domain, far beyond the 64 KB box
    case = dense_case(901, 40, 30000)
    kw = dict(sub=(1, 2, 1), sort_every=0, kernel=kernel, field_dtype=dtype)
    ref, _ = run(lcs, case, UNSTAGED, 5, **kw)
    st, n = run(lcs, case, STAGED[0], 5, **kw)
    assert n == 0
    for key in ("seg", "ids", "x", "v", "img"):
        assert np.array_equal(st[key], ref[key]), key


def test_staged_df_against_oracle(lcs):
    case = dense_case(902, 12, 20000)
    sub = (2, 1, 2)
    st, n = run(lcs, case, STAGED[0], 6, sub=sub, sort_every=2, sort_brick=2, kernel="df")
    assert n > 0
    ref = oracle.initial_state(12, L, sub, case["x0"], case["v0"], case["tau"], track_img=True)
    oracle.run(ref, case["field"], L, sub, case["tau_const"], case["dt"], case["g"], 6,
               sort_every=2, brick=2)
    assert_same_storage(st, ref, 12, sub, brick=2)
    ex, ev, px, pv = traj_errors(st["x"], st["img"], st["v"], st["ids"], ref, case["x0"])
    assert max(ex, ev, px, pv) < 1e-12, (ex, ev, px, pv)


def test_staged_config_errors(lcs):
    case = dense_case(903, 8, 100)
    sim = lcs.Simulator(case["field"], case["x0"], case["v0"], case["dt"], tau=case["tau"],
                        kernel="fp64")
    with pytest.raises(lcs.LcsError) as e:
        sim.set_step_config(256, 2, 1)   # the all-FP64 kernel has no staged form
    assert e.value.status == lcs.LCS_ERR_ARG
    with pytest.raises(lcs.LcsError) as e:
        sim.set_step_config(64, 2, 0)    # not one of the configurations
    assert e.value.status == lcs.LCS_ERR_ARG
    sim.set_step_config(128, 2, 0)
    sim.step(2)
    assert sim.staged_tiles == 0
    sim.close()


@pytest.mark.parametrize("kernel,dtype", [("fp64", "f64"), ("df", "f64"), ("auto", "f32"),
                                          ("auto", "bf16")])
@pytest.mark.parametrize("per_particle_tau,images", [(True, True), (False, False), (True, False)])
def test_prefetched_and_deferred_equal_plain(lcs, kernel, dtype, per_particle_tau, images):
    # ragged segments (window starts at every alignment), migration, sorting
    case = dense_case(904, 12, 9001)
    if not per_particle_tau:
        case["tau"] = None
    kw = dict(sub=(3, 2, 2), sort_every=3, sort_brick=2, kernel=kernel, field_dtype=dtype)

    def go(cfg):
        sim = lcs.Simulator(case["field"], case["x0"], case["v0"], case["dt"], tau=case["tau"],
                            tau_const=case["tau_const"], g=case["g"], track_images=images, **kw)
        sim.set_step_config(*cfg)
        sim.step(8)
        st = gpu_state(sim)
        sim.close()
        return st

    ref = go(UNSTAGED)
    for cfg in PREFETCH + DEFERRED:
        st = go(cfg)
        for key in ("seg", "ids", "x", "v", "img", "tau"):
            assert np.array_equal(st[key], ref[key]), (cfg, key)


@pytest.mark.parametrize("mode", [2, 3])
def test_prefetched_and_deferred_batch_against_oracle(lcs, mode):
    """Several ensembles in one launch, modes 2 and 3, against the FP64 oracle."""
    sp = []
    for k, (N, n, sub) in enumerate([(12, 3000, (2, 2, 2)), (8, 1, (1, 1, 1)),
                                     (16, 0, (2, 1, 1)), (12, 5000, (3, 1, 2))]):
        field, _, x, v, tau = synth.small_case(910 + k, N, 12, N / 4.0, max(n, 1), 0.05, dt=0.01)
        sp.append(dict(field=field, x0=x[:, :n], v0=v[:, :n], dt=0.01, tau=tau[:n],
                       tau_const=0.1, g=(0.0, 0.0, -9.8), sub=sub, sort_every=4, sort_brick=2,
                       kernel="df", track_images=True))
    batch = lcs.Simulator(None, None, None, None, ensembles=sp)
    batch.set_step_config(256, 2, mode)
    batch.step(9)
    for k in (0, 3):
        s = sp[k]
        N = s["field"].shape[-1]
        ref = oracle.initial_state(N, L, s["sub"], s["x0"], s["v0"], s["tau"], track_img=True)
        oracle.run(ref, s["field"], L, s["sub"], s["tau_const"], s["dt"], s["g"], 9,
                   sort_every=4, brick=2)
        st = gpu_state(batch, k)
        assert_same_storage(st, ref, N, s["sub"], brick=2)
        ex, ev, px, pv = traj_errors(st["x"], st["img"], st["v"], st["ids"], ref, s["x0"])
        assert max(ex, ev, px, pv) < 1e-12, (k, ex, ev, px, pv)
    batch.close()


@pytest.mark.parametrize("first,second", [(DEFERRED[2], UNSTAGED), (UNSTAGED, DEFERRED[2]),
                                          (DEFERRED[0], PREFETCH[0])])
def test_pending_sort_across_calls(lcs, first, second):
    """A cell sort whose permutation the next step kernel reads (modes 3 and
    4) is left pending between calls: a switch to a mode that reads records
    in storage order applies it first; the id-ordered read, an explicit sort
    and the state read all see the sorted records.  Every path gives the
    storage of a run in one mode."""
    case = dense_case(905, 12, 9001)
    kw = dict(sub=(3, 2, 2), sort_every=3, sort_brick=2, kernel="df", field_dtype="f64")

    def make(cfg):
        sim = lcs.Simulator(case["field"], case["x0"], case["v0"], case["dt"], tau=case["tau"],
                            tau_const=case["tau_const"], g=case["g"], track_images=True, **kw)
        sim.set_step_config(*cfg)
        return sim

    ref = make(UNSTAGED)
    ref.step(9)
    ref_x, ref_v = (t.cpu().numpy() for t in ref.final_state_by_id())
    ref.sort()
    ref.step(1)
    want = gpu_state(ref)
    ref.close()

    sim = make(first)
    sim.step(3)                    # the sort after step 3 may be left pending
    sim.set_step_config(*second)
    sim.step(6)                    # and the one after step 9
    x, v = (t.cpu().numpy() for t in sim.final_state_by_id())
    assert np.array_equal(x, ref_x) and np.array_equal(v, ref_v)
    sim.sort()
    sim.step(1)
    got = gpu_state(sim)
    sim.close()
    for key in ("seg", "ids", "x", "v", "img", "tau"):
        assert np.array_equal(got[key], want[key]), key


def test_state_read_through_pending_sort(lcs):
    """lcs_get_state right after a sort step reads the records through the
    pending permutation (which stays pending): the state equals that of a
    mode that applies every sort at once, then and after further steps."""
    case = dense_case(906, 12, 9001)
    kw = dict(sub=(3, 2, 2), sort_every=4, sort_brick=2, kernel="df", field_dtype="f64")

    def make(cfg):
        sim = lcs.Simulator(case["field"], case["x0"], case["v0"], case["dt"], tau=case["tau"],
                            tau_const=case["tau_const"], g=case["g"], track_images=True, **kw)
        sim.set_step_config(*cfg)
        return sim

    fused, plain = make(DEFERRED[2]), make(UNSTAGED)
    for n in (8, 3, 1):  # the first and the last read follow a sort
        fused.step(n)
        plain.step(n)
        a, b = gpu_state(fused), gpu_state(plain)
        for key in ("seg", "ids", "x", "v", "img", "tau"):
            assert np.array_equal(a[key], b[key]), (n, key)
    fused.close()
    plain.close()
