"""The hand-written adjoint (lcs_backward) against the oracle (needs a GPU).

* element by element against the oracle's adjoint on the same seeds;
* directional derivatives against central finite differences of the oracle's
  forward (h = 1e-6), with particles whose interpolation cells differ between
  the +h, -h and unperturbed runs masked out of the loss on both sides (the
  trilinear map is only piecewise linear);
* the differentiation workload (128^3, 2^20 particles, 200 steps, checkpoints
  every 20): sampled particles' gradients against the oracle run on just those
  particles, and the field gradient of a sampled seed.
Tolerance: 1e-6 relative (the stated bar for gradients); the adjoint's FP32
stencil arithmetic gives ~1e-7.
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import L

pytestmark = pytest.mark.gpu
TOL = 1e-6


@pytest.fixture(scope="module")
def lcs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2604_11008_gb300 as m
    from paper_2604_11008_gb300 import build
    build.build()
    return m


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def oracle_field_for(field, dtype):
    if dtype == "f32":
        return oracle.round_f32(field)
    if dtype == "bf16":
        return oracle.round_bf16(field)
    return field


@pytest.mark.parametrize("kernel,dtype", [("fp64", "f64"), ("df", "f64"), ("auto", "f32"),
                                          ("auto", "bf16")])
def test_adjoint_matches_oracle_adjoint(lcs, kernel, dtype):
    N, n, steps, K, dt = 16, 3000, 30, 7, 0.01
    field, _, x, v, tau = synth.small_case(300, N, 24, 4.0, n, 0.05, dt=dt)
    g = np.random.default_rng(301)
    v = g.standard_normal((3, n)) * 0.3
    gvec = (0.0, 0.0, -9.8)
    sim = lcs.Simulator(field, x, v, dt, tau=tau, g=gvec, sub=(2, 2, 2), sort_every=5,
                        sort_brick=4, ckpt_every=K, track_images=True, kernel=kernel,
                        field_dtype=dtype)
    sim.step(steps)
    gx = g.standard_normal((3, n))
    gv = g.standard_normal((3, n))
    gU, gx0, gv0 = sim.backward(gx, gv)
    f_ref = oracle_field_for(field, dtype)
    rx, rv, rU = oracle.adjoint(f_ref, L, x, v, tau, 0.0, dt, gvec, steps, gx, gv)
    ex, ev, eU = rel(gx0.cpu().numpy(), rx), rel(gv0.cpu().numpy(), rv), rel(gU.cpu().numpy(), rU)
    # FP32/BF16 storage interpolates in FP32 in the forward (rounding 2^-24 per
    # gather, amplified along the trajectory): 1e-5 there; FP64 kernels 1e-6
    tol = TOL if dtype == "f64" else 1e-5
    assert ex < tol and ev < tol and eU < tol, (ex, ev, eU)


def masked_fd(field, x0, v0, tau, tau_const, dt, gvec, steps, target, d, h=1e-6):
    """Central difference of the loss along d = (dU, dX0, dV0) with the
    oracle, and the mask of particles whose cell sequence is the same in the
    -h, 0, +h runs."""
    dU, dX, dV = d
    n = x0.shape[1]

    def run(f, xa, va):
        xx, vv = xa.copy(), va.copy()
        img = np.zeros((3, n), np.int32)
        hsh = np.zeros(n, np.uint64)
        oracle.advance(f, L, xx, vv, tau, tau_const, dt, gvec, steps, img=img, cellhash=hsh)
        return xx, img, hsh

    x0_, i0_, h0 = run(field, x0, v0)
    xp, ip, hp = run(field + h * dU, x0 + h * dX, v0 + h * dV)
    xm, im, hm = run(field - h * dU, x0 - h * dX, v0 - h * dV)
    mask = ((hp == h0) & (hm == h0)).astype(np.float64)
    # The same central difference [L(+h) - L(-h)] / 2h, subtracted term by
    # term: |a-t|^2 - |b-t|^2 = (a-b).(a+b-2t).  Subtracting the two summed
    # losses instead would lose ~1e-14 absolute to the summation rounding,
    # i.e. up to 1e-4 relative at h = 1e-6.
    up, um = xp + L * ip, xm + L * im
    fd = float(np.sum(mask * ((up - um) * (up + um - 2 * target)).sum(0)) / n) / (2 * h)
    return fd, mask, x0_ + L * i0_


def test_adjoint_directional_derivatives_vs_finite_differences(lcs):
    N, n, steps, K, dt = 32, 2048, 60, 10, 0.005
    field, _, x, v, _ = synth.small_case(310, N, 32, 6.0, n, None, dt=dt)
    g = np.random.default_rng(311)
    target = g.random((3, n)) * L
    gvec = np.zeros(3)
    sim = lcs.Simulator(field, x, v, dt, tau_const=0.1, sub=(2, 2, 2), ckpt_every=K,
                        track_images=True, sort_every=10)
    sim.step(steps)
    xt, _ = sim.final_state_by_id()
    xt = xt.cpu().numpy()
    worst = 0.0
    for k in range(16):
        d = (g.standard_normal(field.shape), g.standard_normal((3, n)), g.standard_normal((3, n)))
        fd, mask, x_ref = masked_fd(field, x, v, None, 0.1, dt, gvec, steps, target, d)
        gx = 2.0 / n * (xt - target) * mask[None, :]
        gU, gx0, gv0 = sim.backward(gx, np.zeros((3, n)))
        ad = float((gU.cpu().numpy() * d[0]).sum() + (gx0.cpu().numpy() * d[1]).sum()
                   + (gv0.cpu().numpy() * d[2]).sum())
        worst = max(worst, abs(ad - fd) / abs(fd))
    print(f"worst relative FD mismatch {worst:.3e}")
    assert worst < TOL, worst


def grad_workload():
    w = synth.WORKLOADS["grad_128"]
    field, _ = synth.make_field(w)
    dt = synth.cfl_dt(synth.max_speed(field), w.N)
    x, v, _ = synth.make_particles(w, dt)
    target = synth.positions(w.np_, synth.rng(w.number, synth.STREAM_TARGET))
    return w, field, dt, x, v, target


def test_grad_128_sampled_particles_against_oracle(lcs):
    """Full differentiation workload on the GPU; 4096 sampled particles'
    dL/dX0, dL/dV0 and their field gradient against the oracle run on those
    particles only (particles are independent; the field does not depend on
    them): norm-wise and in the max norm, every entry of the field gradient
    within 1e-6 of the largest."""
    import torch
    w, field, dt, x, v, target = grad_workload()
    n = w.np_
    sim = lcs.Simulator(field, x, v, dt, tau_const=w.tau_const, sub=w.sub, ckpt_every=20,
                        track_images=True, sort_every=10)
    sim.step(w.steps)
    xt, _ = sim.final_state_by_id()
    xt = xt.cpu().numpy()
    ns = 4096
    sample = np.random.default_rng(320).choice(n, ns, replace=False)
    gx = np.zeros((3, n))
    gx[:, sample] = 2.0 / n * (xt[:, sample] - target[:, sample])
    gU, gx0, gv0 = sim.backward(gx, np.zeros((3, n)))
    xs, vs = x[:, sample].copy(), v[:, sample].copy()
    rx, rv, rU = oracle.adjoint(field, L, xs, vs, None, w.tau_const, dt, w.g, w.steps,
                                gx[:, sample], np.zeros((3, ns)))
    gx0 = gx0.cpu().numpy()[:, sample]
    gv0 = gv0.cpu().numpy()[:, sample]
    gUn = gU.cpu().numpy()
    assert rel(gx0, rx) < TOL and rel(gv0, rv) < TOL, (rel(gx0, rx), rel(gv0, rv))
    assert rel(gUn, rU) < TOL, rel(gUn, rU)

    def maxnorm(a, b):
        return float(np.abs(a - b).max() / np.abs(b).max())
    mx, mv, mU = maxnorm(gx0, rx), maxnorm(gv0, rv), maxnorm(gUn, rU)
    print(f"grad_128, {ns} particles: max-norm errors dX0 {mx:.2e} dV0 {mv:.2e} dU {mU:.2e}")
    assert mx < TOL and mv < TOL and mU < TOL, (mx, mv, mU)
    # every other particle had a zero seed: its gradient is exactly zero
    others = np.setdiff1d(np.arange(n), sample)[:1000]
    g_all = sim.backward(gx, np.zeros((3, n)))[1].cpu().numpy()
    assert np.all(g_all[:, others] == 0.0)
    torch.cuda.synchronize()


def test_grad_128_subsample_finite_differences(lcs):
    """16 random directions (field, X0, V0) on 256 particles of the
    differentiation workload: GPU adjoint vs masked central differences."""
    w, field, dt, x, v, target = grad_workload()
    idx = np.random.default_rng(330).choice(w.np_, 256, replace=False)
    xs, vs, ts = x[:, idx].copy(), v[:, idx].copy(), target[:, idx].copy()
    n = 256
    sim = lcs.Simulator(field, xs, vs, dt, tau_const=w.tau_const, sub=w.sub, ckpt_every=20,
                        track_images=True)
    sim.step(w.steps)
    xt, _ = sim.final_state_by_id()
    xt = xt.cpu().numpy()
    g = np.random.default_rng(331)
    worst = 0.0
    for k in range(16):
        d = (g.standard_normal(field.shape), g.standard_normal((3, n)), g.standard_normal((3, n)))
        fd, mask, _ = masked_fd(field, xs, vs, None, w.tau_const, dt, np.zeros(3), w.steps, ts, d)
        gU, gx0, gv0 = sim.backward(2.0 / n * (xt - ts) * mask[None, :], np.zeros((3, n)))
        ad = float((gU.cpu().numpy() * d[0]).sum() + (gx0.cpu().numpy() * d[1]).sum()
                   + (gv0.cpu().numpy() * d[2]).sum())
        worst = max(worst, abs(ad - fd) / abs(fd))
    print(f"worst relative FD mismatch {worst:.3e}")
    assert worst < TOL, worst


def test_autograd_function_end_to_end(lcs):
    """torch.autograd through ParticleAdvect matches the oracle adjoint."""
    import torch
    N, n, steps, dt = 16, 500, 20, 0.01
    field, _, x, v, _ = synth.small_case(340, N, 16, 4.0, n, None, dt=dt)
    target = torch.from_numpy(np.random.default_rng(341).random((3, n)) * L).cuda()
    U = torch.from_numpy(field).cuda().requires_grad_(True)
    X0 = torch.from_numpy(x).cuda().requires_grad_(True)
    V0 = torch.from_numpy(v).cuda().requires_grad_(True)
    XT, VT = lcs.particle_advect(U, X0, V0, steps=steps, dt=dt, tau_const=0.1, sub=(2, 2, 1),
                                 ckpt_every=6)
    loss = ((XT - target) ** 2).sum(0).mean()
    loss.backward()
    xr, vr = x.copy(), v.copy()
    img = np.zeros((3, n), np.int32)
    oracle.advance(field, L, xr, vr, None, 0.1, dt, np.zeros(3), steps, img=img)
    xu = xr + L * img
    assert np.abs(XT.detach().cpu().numpy() - xu).max() < 1e-12
    seed = 2.0 / n * (xu - target.cpu().numpy())
    rx, rv, rU = oracle.adjoint(field, L, x, v, None, 0.1, dt, np.zeros(3), steps, seed,
                                np.zeros((3, n)))
    assert rel(X0.grad.cpu().numpy(), rx) < TOL
    assert rel(V0.grad.cpu().numpy(), rv) < TOL
    assert rel(U.grad.cpu().numpy(), rU) < TOL


def test_backward_requires_a_tape(lcs):
    field, _, x, v, _ = synth.small_case(350, 8, 4, 2.0, 50, None)
    sim = lcs.Simulator(field, x, v, 0.01, tau_const=0.1)
    sim.step(2)
    with pytest.raises(lcs.LcsError) as e:
        sim.backward(np.zeros((3, 50)), np.zeros((3, 50)))
    assert e.value.status == lcs.LCS_ERR_ARG
    sim.step(1)   # a refused call latches nothing
    sim.sync()
