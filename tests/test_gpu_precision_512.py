"""The precision workload at full size (needs a GPU, ~40 GB of device memory).

512^3 field (512 modes, k 1-64), 10^8 particles, log-normal tau (median
0.02, sigma 0.7), gravity, 8x8x8 subdomains, cell sort every 10 steps, 200
steps; field stored in FP64 (float-float kernel), FP32 and BF16.  Particles
do not interact (one-way coupling, Eqs. 5-6), so each of 10^5 sampled
particles is checked against the FP64 oracle run on those particles alone:
relative errors (norm-wise over the sample) within 1e-12 / 1e-5 / 1e-2.
The sampled ids also pin the migration: every sampled particle must sit in
the segment of the subdomain that contains it.
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import L, particle_errors

pytestmark = pytest.mark.gpu

BARS = {"f64": 1e-12, "f32": 1e-5, "bf16": 1e-2}


@pytest.fixture(scope="module")
def setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    free, _ = torch.cuda.mem_get_info()
    if free < 60e9:
        pytest.skip("needs ~60 GB of free device memory")
    import paper_2604_11008_gb300 as lcs
    from paper_2604_11008_gb300 import build
    build.build()
    w = synth.WORKLOADS["precision_512"]
    field, _ = synth.make_field(w, device="cuda")
    dt = synth.cfl_dt(synth.max_speed(field), w.N)
    x, v, tau = synth.make_particles(w, dt)
    sample = np.sort(np.random.default_rng(700).choice(w.np_, 100_000, replace=False))
    fcpu = field.cpu().numpy()
    xs, vs, ts = x[:, sample].copy(), v[:, sample].copy(), tau[sample].copy()
    img = np.zeros((3, len(sample)), np.int32)
    oracle.advance(fcpu, L, xs, vs, ts, 0.0, dt, w.g, w.steps, img=img)
    ref = (xs + L * img, vs)
    return lcs, w, field, dt, x, v, tau, sample, ref


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_precision_512_against_fp64_oracle(setup, dtype):
    import torch
    lcs, w, field, dt, x, v, tau, sample, (xr, vr) = setup
    sim = lcs.Simulator(field, x, v, dt, tau=tau, g=w.g, sub=w.sub, field_dtype=dtype,
                        sort_every=w.sort_every, track_images=True)
    sim.step(w.steps)
    st = sim.get_state()
    ids = st["ids"].long()
    pos = torch.empty_like(ids)
    pos[ids] = torch.arange(ids.numel(), device=ids.device)
    at = pos[torch.from_numpy(sample).cuda()]
    xg = (st["x"][:, at] + L * st["img"][:, at].double()).cpu().numpy()
    vg = st["v"][:, at].cpu().numpy()
    # segment membership of the sampled particles
    seg_of = torch.searchsorted(torch.from_numpy(st["seg"]).cuda(), at, right=True) - 1
    c = torch.clamp(torch.floor(st["x"][:, at] * (w.N / L)).long(), 0, w.N - 1)
    p = c // (w.N // torch.tensor(w.sub, device=c.device)[:, None])
    dest = p[0] + w.sub[0] * (p[1] + w.sub[1] * p[2])
    sim.close()
    del st
    assert torch.equal(seg_of, dest)
    x0 = x[:, sample]
    ex = np.linalg.norm(xg - xr) / np.linalg.norm(xr - x0)
    ev = np.linalg.norm(vg - vr) / np.linalg.norm(vr)
    px, pv = particle_errors(xg, xr, vg, vr, x0)
    print(f"{dtype}: e_x {ex:.3e}  e_v {ev:.3e}  per particle {px:.3e} {pv:.3e}")
    assert max(ex, ev, px, pv) < BARS[dtype], (ex, ev, px, pv)
