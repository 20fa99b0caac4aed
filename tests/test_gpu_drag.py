"""Nonlinear drag factor of Eq. (7) against the oracle (needs a GPU).

f = 1 + 0.15 Re_p^0.687, Re_p = 2 r |V - U| / nu, r from
tau_p = (2/9)(rho_p/rho) r^2 / nu (Sec. 2.2).  The FP64 and float-float
kernels must meet the FP64 bar (1e-12); the
FP32 / BF16 kernels use FP32 powf and must meet their bars against the oracle
on the same rounded field and on the FP64 field.  The float-float kernel's
power is its own table-driven float-float log2 / exp2; slips over twelve
decades run it across its whole reduction range.  With a small viscosity the
particle Reynolds numbers reach O(1-10), so f departs from 1 by tens of
percent and a wrong factor could not hide inside the tolerances.
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import L, assert_same_storage, by_id, gpu_state, traj_errors

pytestmark = pytest.mark.gpu

NU, RHO = 2e-3, 843.0
DRAG = (1, NU, RHO)


@pytest.fixture(scope="module")
def lcs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2604_11008_gb300 as m
    from paper_2604_11008_gb300 import build
    build.build()
    return m


def case(seed=120, N=24, n=20000):
    field, _, x, v, tau = synth.small_case(seed, N, 32, 6.0, n, 0.05, dt=0.005)
    v = np.ascontiguousarray(0.5 * np.random.default_rng(seed).standard_normal(x.shape))
    return field, x, v, tau


def run_gpu(lcs, field, x, v, tau, P, steps, **kw):
    sim = lcs.Simulator(field, x, v, 0.005, tau=tau, g=(0.0, 0.0, -9.8), sub=P,
                        track_images=True, drag="nonlinear", nu=NU, density_ratio=RHO, **kw)
    sim.step(steps)
    st = gpu_state(sim)
    sim.close()
    return st


def test_reynolds_numbers_are_order_one():
    field, x, v, tau = case()
    u = np.stack(oracle.interp(field, L, x))
    r = np.sqrt(9 * NU * tau / (2 * RHO))
    re = 2 * r * np.linalg.norm(v - u, axis=0) / NU
    assert np.median(re) > 0.5 and re.max() > 5


@pytest.mark.parametrize("kernel", ["fp64", "df"])
def test_nonlinear_drag_fp64_trajectories(lcs, kernel):
    field, x, v, tau = case()
    P, steps = (2, 3, 2), 30
    st = run_gpu(lcs, field, x, v, tau, P, steps, kernel=kernel, sort_every=7, sort_brick=4)
    ref = oracle.initial_state(24, L, P, x, v, tau, track_img=True)
    oracle.run(ref, field, L, P, 0.0, 0.005, (0.0, 0.0, -9.8), steps, sort_every=7, brick=4,
               drag=DRAG)
    ex, ev, px, pv = traj_errors(st["x"], st["img"], st["v"], st["ids"], ref, x)
    assert max(ex, ev, px, pv) < 1e-12, (ex, ev, px, pv)
    assert_same_storage(st, ref, 24, P, 4)
    # the drag law matters at this size: Stokes drag lands far away
    stokes = oracle.initial_state(24, L, P, x, v, tau, track_img=True)
    oracle.run(stokes, field, L, P, 0.0, 0.005, (0.0, 0.0, -9.8), steps, sort_every=7, brick=4)
    ex_s, ev_s, px_s, pv_s = traj_errors(st["x"], st["img"], st["v"], st["ids"], stokes, x)
    assert ev_s > 1e-3, ev_s


@pytest.mark.parametrize("kernel", ["df", "fp64"])
def test_nonlinear_drag_over_decades_of_slip(lcs, kernel):
    # |V - U| from 1e-9 to 1e3 (Re_p from about 1e-9 to 1e3), every particle
    # checked on its own against the oracle
    N, n, P, steps, dt = 16, 6000, (2, 2, 2), 4, 0.001
    field, x, _, tau = case(seed=123, N=N, n=n)
    u = np.stack(oracle.interp(field, L, x))
    rng = np.random.default_rng(123)
    d = rng.standard_normal(x.shape)
    d *= 10.0 ** rng.uniform(-9, 3, n) / np.linalg.norm(d, axis=0)
    v = np.ascontiguousarray(u + d)
    sim = lcs.Simulator(field, x, v, dt, tau=tau, sub=P, track_images=True, kernel=kernel,
                        drag="nonlinear", nu=NU, density_ratio=RHO)
    sim.step(steps)
    st = gpu_state(sim)
    ref = oracle.initial_state(N, L, P, x, v, tau, track_img=True)
    oracle.run(ref, field, L, P, 0.0, dt, (0.0, 0.0, 0.0), steps, drag=DRAG)
    ex, ev, px, pv = traj_errors(st["x"], st["img"], st["v"], st["ids"], ref, x)
    assert max(ex, ev, px, pv) < 1e-12, (ex, ev, px, pv)
    xg, vg, ig = by_id(st["ids"], st["x"], st["v"], st["img"])
    xr, vr, ir = by_id(ref.ids, ref.x, ref.v, ref.img)
    dv = np.linalg.norm(vg - vr, axis=0) / np.linalg.norm(vr, axis=0)
    dx = np.linalg.norm(xg + L * ig - xr - L * ir, axis=0) / np.linalg.norm(xr + L * ir - x, axis=0)
    assert dv.max() < 1e-11 and dx.max() < 1e-11, (dv.max(), dx.max())


@pytest.mark.parametrize("dtype,tol_q,tol_64", [("f32", 1e-6, 1e-5), ("bf16", 1e-5, 1e-2)])
def test_nonlinear_drag_precision_variants(lcs, dtype, tol_q, tol_64):
    field, x, v, tau = case(seed=121)
    P, steps = (2, 2, 2), 30
    st = run_gpu(lcs, field, x, v, tau, P, steps, field_dtype=dtype)
    fq = oracle.round_f32(field) if dtype == "f32" else oracle.round_bf16(field)
    for f_ref, tol in ((fq, tol_q), (field, tol_64)):
        ref = oracle.initial_state(24, L, P, x, v, tau, track_img=True)
        oracle.run(ref, f_ref, L, P, 0.0, 0.005, (0.0, 0.0, -9.8), steps, drag=DRAG)
        ex, ev, px, pv = traj_errors(st["x"], st["img"], st["v"], st["ids"], ref, x)
        assert max(ex, ev, px, pv) < tol, (dtype, ex, ev, px, pv)


@pytest.mark.parametrize("cfg", [(256, 2, 0), (256, 1, 3), (128, 2, 3), (256, 2, 2)])
def test_nonlinear_drag_every_kernel_mode_agrees(lcs, cfg):
    field, x, v, tau = case(seed=122, n=9000)
    res = []
    for c in ((256, 2, 3), cfg):
        sim = lcs.Simulator(field, x, v, 0.005, tau=tau, sub=(3, 1, 2), drag="nonlinear",
                            nu=NU, kernel="df", sort_every=4)
        sim.set_step_config(*c)
        sim.step(9)
        res.append(gpu_state(sim))
        sim.close()
    for key in ("seg", "ids", "x", "v"):
        assert np.array_equal(res[0][key], res[1][key]), key


def test_nonlinear_drag_arguments(lcs):
    field, x, v, tau = case(n=100)
    for kw in (dict(nu=0.0), dict(nu=-1.0), dict(nu=NU, density_ratio=-2.0),
               dict(nu=NU, ckpt_every=5, track_images=True)):
        with pytest.raises(lcs.LcsError) as e:
            lcs.Simulator(field, x, v, 0.005, tau=tau, drag="nonlinear", **kw)
        assert e.value.status == lcs.LCS_ERR_ARG
    # density_ratio 0 selects the paper's 843
    a = lcs.Simulator(field, x, v, 0.005, tau=tau, drag="nonlinear", nu=NU)
    b = lcs.Simulator(field, x, v, 0.005, tau=tau, drag="nonlinear", nu=NU, density_ratio=843.0)
    a.step(3)
    b.step(3)
    assert np.array_equal(gpu_state(a)["v"], gpu_state(b)["v"])
