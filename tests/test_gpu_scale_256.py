"""The throughput workload at full size, as bench.py runs it (needs a GPU).

256^3 FP64 field (512 modes, k 1-32), 16,777,216 particles, log-normal tau
(median 0.05, sigma 0.5), gravity, 4x4x4 subdomains, cell sort every 10
steps, 1000 steps, step kernel autotuned as in bench.py.  Particles do not
interact (one-way coupling, Eqs. 5-6), so 20,000 sampled particles are
checked against the FP64 oracle run on those particles alone: norm-wise
relative errors within 1e-12 (positions compared modulo the period, as the
run does not track images).

Chaos horizon: a trajectory this long amplifies rounding differences, so
two more checks bound what the full-run comparison means.  (1) One step from
identical states every 10 steps: the sampled particles' GPU state after step
s (s = 29, 39, ..., 999) is advanced one step by the oracle and compared,
particle by particle, with the GPU's state after step s + 1 (a sort step):
the binding element-wise check of the long run, bar 1e-12.  (2) A shadow
run: the oracle against itself with every sampled initial position moved by
one unit in the last place, whose divergence is the intrinsic growth floor
of the full-run error.  Over 1000 steps the shadow run's own largest
per-particle errors exceed 1e-12 (a one-ulp start grows to a few 1e-12 for
the most sensitive particles), so the full-run per-particle errors are bounded
by ten times the shadow's, not by the one-step bar.

The whole final state is checked for what holds at any size: the id multiset
is unchanged, every particle sits in the segment of the subdomain that
contains it (migration, Sec. 2.3.3), and, the last step being a sort step,
the cell keys inside every segment are in order.
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import L, particle_errors

pytestmark = pytest.mark.gpu

N_SAMPLE = 20_000


@pytest.fixture(scope="module")
def final():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2604_11008_gb300 as lcs
    from paper_2604_11008_gb300 import build
    build.build()
    w = synth.WORKLOADS["scale_256"]
    field, _ = synth.make_field(w, device="cuda")
    dt = w.dt if w.dt is not None else synth.cfl_dt(synth.max_speed(field), w.N)
    x, v, tau = synth.make_particles(w, dt)
    sample = np.sort(np.random.default_rng(256).choice(w.np_, N_SAMPLE, replace=False))
    at = torch.from_numpy(sample).cuda()
    sim = lcs.Simulator(field, x, v, dt, tau=tau, tau_const=w.tau_const, g=w.g, sub=w.sub,
                        sort_every=w.sort_every)
    sim.tune(2)                        # advances 2 steps per tried configuration
    done = 2 * int((sim.tune_trials_ms > 0).sum())
    assert w.steps % w.sort_every == 0

    def sampled():
        xi, vi = sim.final_state_by_id()   # id order; ids are 0..np-1
        return xi[:, at].cpu().numpy(), vi[:, at].cpu().numpy()

    checks = []
    k = done
    while k < w.steps:
        s = k + (9 - k % 10) % 10          # next step count s with s + 1 a sort step
        sim.step(s - k)
        k = s
        before = sampled()
        sim.step(1)
        k += 1
        checks.append((s, before, sampled()))
    st = sim.get_state(device="cpu")
    sim.close()
    st = {kk: (a.numpy() if hasattr(a, "numpy") else a) for kk, a in st.items()}
    return w, field.cpu().numpy(), dt, x, v, tau, st, sample, checks


def test_sampled_trajectories_against_oracle(final):
    w, field, dt, x, v, tau, st, sample, _ = final
    xs, vs, ts = x[:, sample].copy(), v[:, sample].copy(), tau[sample].copy()
    img = np.zeros((3, len(sample)), np.int32)
    oracle.advance(field, L, xs, vs, ts, 0.0, dt, w.g, w.steps, img=img)
    pos = np.empty(w.np_, np.int64)
    pos[st["ids"].astype(np.int64)] = np.arange(w.np_)
    at = pos[sample]
    d = st["x"][:, at] - xs
    d -= L * np.round(d / L)           # the same point modulo the period
    xr = xs + L * img
    ex = np.linalg.norm(d) / np.linalg.norm(xr - x[:, sample])
    ev = np.linalg.norm(st["v"][:, at] - vs) / np.linalg.norm(vs)
    # element by element: the GPU position modulo the period, moved next to
    # the oracle's unwrapped one
    px, pv = particle_errors(xr + d, xr, st["v"][:, at], vs, x[:, sample])
    # shadow run: the oracle from initial positions one ulp away
    xh = np.ascontiguousarray(np.nextafter(x[:, sample], np.inf))
    vh = v[:, sample].copy()
    imh = np.zeros_like(img)
    oracle.advance(field, L, xh, vh, tau[sample].copy(), 0.0, dt, w.g, w.steps, img=imh)
    xhu = xh + L * imh
    sx = np.linalg.norm(xhu - xr) / np.linalg.norm(xr - x[:, sample])
    sv = np.linalg.norm(vh - vs) / np.linalg.norm(vs)
    spx, spv = particle_errors(xhu, xr, vh, vs, x[:, sample])
    print(f"scale_256 FP64 field, {w.steps} steps: GPU vs oracle e_x {ex:.3e} e_v {ev:.3e}, "
          f"per particle {px:.3e} {pv:.3e}; shadow (1 ulp in X0) e_x {sx:.3e} e_v {sv:.3e}, "
          f"per particle {spx:.3e} {spv:.3e}")
    assert max(ex, ev) < 1e-12, (ex, ev)
    # element by element against the intrinsic growth floor: the GPU's per-step
    # rounding (~2^-45 of the increments) against a single one-ulp start
    assert px < max(1e-12, 10 * spx) and pv < max(1e-12, 10 * spv), (px, pv, spx, spv)


def test_one_step_parity_every_10_steps(final):
    """One step from identical states (the GPU's own, exported), every 10
    steps of the run: per particle, the position within 1e-12 of a grid
    spacing (the FP64 positions carry ulp(L) ~ 1e-15 of rounding either way)
    and the velocity within 1e-12 of its own speed, floored at the rms speed
    of the sample (as in particle_errors)."""
    w, field, dt, x, v, tau, st, sample, checks = final
    assert len(checks) >= 90
    ts = tau[sample]
    worst_x = worst_v = 0.0
    for s, (x0, v0), (x1, v1) in checks:
        xo, vo = x0.copy(), v0.copy()
        oracle.advance(field, L, xo, vo, ts.copy(), 0.0, dt, w.g, 1)
        d = x1 - xo
        d -= L * np.round(d / L)
        ex = float(np.abs(d).max()) / (L / w.N)
        sp = np.linalg.norm(vo, axis=0)
        floor = np.sqrt(np.mean(sp ** 2))
        ev = float((np.linalg.norm(v1 - vo, axis=0) / np.maximum(sp, floor)).max())
        worst_x, worst_v = max(worst_x, ex), max(worst_v, ev)
        assert ex < 1e-12 and ev < 1e-12, (s, ex, ev)
    print(f"one-step parity at {len(checks)} steps: worst position error {worst_x:.3e} of a cell, "
          f"worst relative velocity error {worst_v:.3e}")


def test_ids_segments_and_cell_order(final):
    w, field, dt, x, v, tau, st, _, _ = final
    ids = st["ids"].astype(np.int64)
    assert np.array_equal(np.sort(ids), np.arange(w.np_))
    seg = st["seg"]
    assert seg[0] == 0 and seg[-1] == w.np_ and np.all(np.diff(seg) >= 0)
    dest, key = oracle.keys(w.N, L, w.sub, 8, st["x"])
    owner = np.repeat(np.arange(len(seg) - 1), np.diff(seg))
    assert np.array_equal(dest, owner)
    # keys non-decreasing inside every segment (drops only at segment starts)
    drops = np.nonzero(np.diff(key) < 0)[0] + 1
    assert np.isin(drops, seg[1:-1]).all()
