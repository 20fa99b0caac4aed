"""Batched ensembles (needs a GPU).

All ensembles of a context advance in the same persistent kernel launches;
each ensemble's particles see exactly the arithmetic and the stable orders of
a run of that ensemble alone, so batched and solo states must be identical
bit for bit.  The autotuner changes only the scan tile and the kernel mode, never the
results.
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import L, gpu_state

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


def specs(kernel, dtype):
    out = []
    cases = [  # N, n, sub, tau median (None: constant), sort_every, g
        (8, 1, (2, 2, 2), None, 0, (0.0, 0.0, 0.0)),
        (12, 700, (3, 1, 2), 0.05, 4, (0.0, 0.0, -9.8)),
        (16, 5000, (2, 2, 2), None, 5, (0.0, 0.0, 0.0)),
        (24, 20000, (3, 3, 3), 0.05, 4, (0.0, -1.0, 0.0)),
        (16, 0, (1, 1, 1), None, 3, (0.0, 0.0, 0.0)),
        (20, 9000, (1, 1, 1), 0.1, 0, (0.0, 0.0, -9.8)),
    ]
    for k, (N, n, sub, tm, se, g) in enumerate(cases):
        field, _, x, v, tau = synth.small_case(500 + k, N, 12, N / 4.0, max(n, 1), tm, dt=0.01)
        x, v = x[:, :n], v[:, :n]
        tau = None if tau is None else tau[:n]
        out.append(dict(field=field, x0=x, v0=v, dt=0.01, tau=tau, tau_const=0.1, g=g, sub=sub,
                        sort_every=se, sort_brick=4, kernel=kernel, field_dtype=dtype,
                        track_images=True))
    return out


@pytest.mark.parametrize("kernel,dtype", [("df", "f64"), ("auto", "f32"), ("fp64", "f64")])
def test_batch_equals_solo_runs(lcs, kernel, dtype):
    sp = specs(kernel, dtype)
    batch = lcs.Simulator(None, None, None, None, ensembles=sp)
    batch.step(13)  # sorts after steps 3, 4, 5, 6, 8, 9, 10, 12 depending on the ensemble
    for k, s in enumerate(sp):
        solo = lcs.Simulator(**{kk: vv for kk, vv in s.items() if kk not in ("field", "x0", "v0",
                                                                                "dt")},
                             field=s["field"], x0=s["x0"], v0=s["v0"], dt=s["dt"])
        solo.step(13)
        a, b = gpu_state(batch, k), gpu_state(solo)
        for key in ("seg", "ids", "x", "v", "img"):
            assert np.array_equal(a[key], b[key]), (k, key)
        solo.close()


def test_batch_against_oracle(lcs):
    sp = specs("df", "f64")
    batch = lcs.Simulator(None, None, None, None, ensembles=sp)
    batch.step(9)
    for k in (2, 3):
        s = sp[k]
        N = s["field"].shape[-1]
        ref = oracle.initial_state(N, L, s["sub"], s["x0"], s["v0"], s["tau"], track_img=True)
        oracle.run(ref, s["field"], L, s["sub"], s["tau_const"], s["dt"], s["g"], 9,
                   sort_every=s["sort_every"], brick=4)
        st = gpu_state(batch, k)
        assert np.array_equal(st["seg"], ref.seg)
        assert np.array_equal(st["ids"].astype(np.uint32), ref.ids)
        assert np.abs(st["x"] - ref.x).max() < 1e-12


def test_tune_keeps_results(lcs):
    sp = specs("df", "f64")
    a = lcs.Simulator(None, None, None, None, ensembles=sp)
    b = lcs.Simulator(None, None, None, None, ensembles=sp)
    cfg = b.tune(2)   # 12 configurations x 2 steps (the owned-field mode is skipped)
    a.step(2 * int((b.tune_trials_ms > 0).sum()))
    assert cfg in ((256, 2, 0), (256, 1, 0), (128, 2, 0), (256, 2, 1), (128, 2, 1),
                   (256, 2, 2), (128, 2, 2), (256, 1, 2), (256, 2, 3), (128, 2, 3),
                   (256, 1, 3), (128, 1, 3))
    assert (b.tune_trials_ms[:12] > 0).all()
    assert (b.tune_trials_ms[12:] == -1).all()
    # a configuration per class of ensembles (grid size, decade of np)
    allowed = {(256, 2, 0), (256, 1, 0), (128, 2, 0), (256, 2, 1), (128, 2, 1), (256, 2, 2),
               (128, 2, 2), (256, 1, 2), (256, 2, 3), (128, 2, 3), (256, 1, 3), (128, 1, 3)}
    cfgs = [b.step_config_of(k) for k in range(len(sp))]
    assert cfgs[0] == cfg and all(c in allowed for c in cfgs)
    for k in range(len(sp)):
        sa, sb = gpu_state(a, k), gpu_state(b, k)
        for key in ("seg", "ids", "x", "v"):
            assert np.array_equal(sa[key], sb[key]), (k, key)
    a.step(4)
    b.step(4)   # graphs rebuilt with the tuned tile
    for k in range(len(sp)):
        assert np.array_equal(gpu_state(a, k)["x"], gpu_state(b, k)["x"])


def test_mixed_storage_is_rejected(lcs):
    sp = specs("df", "f64")[:2]
    sp[1]["field_dtype"] = "f32"
    with pytest.raises(lcs.LcsError) as e:
        lcs.Simulator(None, None, None, None, ensembles=sp)
    assert e.value.status == lcs.LCS_ERR_ARG


def test_batch_workload_ensembles_equal_solo(lcs):
    """The 48-ensemble batching workload (grids 64-256^3, FP32 fields), at 1/100
    of its particle counts: every ensemble of the batch equals its solo run."""
    ens = synth.batch_ensembles(48, device="cuda", scale=0.01)
    sp = [dict(field=e["field"], x0=e["x0"], v0=e["v0"], dt=e["dt"], tau=e["tau"],
               sub=(2, 2, 2), sort_every=10, field_dtype="f32") for e in ens]
    batch = lcs.Simulator(None, None, None, None, ensembles=sp)
    batch.step(12)
    for k in (0, 7, 23, 47):
        s = sp[k]
        solo = lcs.Simulator(s["field"], s["x0"], s["v0"], s["dt"], tau=s["tau"], sub=s["sub"],
                             sort_every=10, field_dtype="f32")
        solo.step(12)
        a, b = gpu_state(batch, k), gpu_state(solo)
        assert np.array_equal(a["ids"], b["ids"]) and np.array_equal(a["x"], b["x"])
        solo.close()


def test_step_runs_in_one_graph_equal_single_steps(lcs):
    """lcs_step records runs of steps up to the step period (lcm of the sort
    and checkpoint intervals) as one graph each; any split of the same steps
    into calls gives the same state bit for bit."""
    sp = specs("df", "f64")
    a = lcs.Simulator(None, None, None, None, ensembles=sp)
    b = lcs.Simulator(None, None, None, None, ensembles=sp)
    for n in (37, 3, 60):
        a.step(n)
        for _ in range(n):
            b.step(1)
        for k in range(len(sp)):
            sa, sb = gpu_state(a, k), gpu_state(b, k)
            for key in ("seg", "ids", "x", "v", "img"):
                assert np.array_equal(sa[key], sb[key]), (n, k, key)
    # sort intervals 3, 4, 5: period 60, so the 100 steps of `a` took one
    # graph launch per run -- (0, 37), (37, 3), (40, 20), (0, 40) -- and `b` 100
    assert a.graph_launches == 4 and b.graph_launches == 100, (a.graph_launches,
                                                               b.graph_launches)
