"""Parity of the CUDA path with the CPU oracle (needs a GPU).

Every comparison uses the same seeded inputs on both sides.  Integer work
(migration order, sort order, segment bounds) must match bit for bit;
FP64 trajectories within a relative 1e-12 (norm-wise, unwrapped positions
relative to the displacement, velocities relative to their norm)."""
import math

import numpy as np
import pytest

import oracle
import synth
from helpers import L, assert_same_storage, by_id, gpu_state, traj_errors

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-12


@pytest.fixture(scope="module")
def lcs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2604_11008_gb300 as m
    from paper_2604_11008_gb300 import build
    build.build()
    return m


# ---------------------------------------------------------------- partition (Sec. 2.3.3)

def test_partition_worked_example(lcs, worked_example):
    """mask 0,1,0,1,0: the mask-1 particles 2 and 4 land at 1-based buffer slots 1, 2."""
    mask = np.array([r[1] for r in worked_example], np.int32)
    scan = [r[2] for r in worked_example]
    perm, off, status = lcs.partition(mask, 2)
    perm, off = perm.cpu().numpy(), off.cpu().numpy()
    assert int(status.item()) == 0
    assert list(off) == [0, 3, 5]
    bin1 = perm[off[1]:off[2]]
    for slot, p in enumerate(bin1):
        assert scan[p] == slot + 1
    assert list(perm) == [0, 2, 4, 1, 3]


@pytest.mark.parametrize("n,nbins", [(0, 3), (1, 1), (5, 2), (4095, 7), (4097, 64), (70001, 3),
                                     (100000, 513), (250000, 65536)])
def test_partition_is_a_stable_counting_sort(lcs, n, nbins):
    g = np.random.default_rng(n + nbins)
    keys = g.integers(0, nbins, n).astype(np.int32)
    perm, off, status = lcs.partition(keys, nbins)
    ref = np.argsort(keys, kind="stable")
    assert np.array_equal(perm.cpu().numpy(), ref)
    assert np.array_equal(off.cpu().numpy(),
                          np.concatenate([[0], np.cumsum(np.bincount(keys, minlength=nbins))]))
    assert int(status.item()) == 0


def test_partition_flags_out_of_range_keys(lcs):
    keys = np.array([0, 5, 1, 9], np.int32)
    perm, off, status = lcs.partition(keys, 3)
    assert int(status.item()) == lcs.LCS_ERR_ARG
    assert list(perm.cpu().numpy()) == [0, 2, 1, 3]


# ---------------------------------------------------------------- placement and migration

KERNELS = ["fp64", "df"]


def make(lcs, field, x, v, dt, tau=None, tau_const=0.1, kernel="fp64", **kw):
    return lcs.Simulator(field, x, v, dt, tau=tau, tau_const=tau_const, kernel=kernel, **kw)


@pytest.mark.parametrize("P", [(1, 1, 1), (2, 2, 2), (3, 3, 3), (4, 2, 1)])
def test_initial_placement_matches_oracle(lcs, P):
    N = 12 if 3 in P else 16
    field, _, x, v, _ = synth.small_case(30, N, 8, 2.0, 9000, None)
    sim = make(lcs, field, x, v, 0.01, sub=P)
    st = gpu_state(sim)
    ref = oracle.initial_state(N, L, P, x, v, None)
    assert np.array_equal(st["seg"], ref.seg)
    assert np.array_equal(st["ids"].astype(np.uint32), ref.ids)
    # the library holds positions in fixed point (cell units, 52 fraction
    # bits) and velocities as float pairs (48 bits): read back within one
    # unit in the last place, and within 2^-47 relative
    assert np.all(np.abs(st["x"] - ref.x) <= np.spacing(L))
    assert np.all(np.abs(st["v"] - ref.v) <= np.abs(ref.v) * 2.0 ** -47)


def test_empty_and_single_particle(lcs):
    field, _, x, v, _ = synth.small_case(31, 8, 4, 2.0, 1, None)
    for n in (0, 1):
        sim = make(lcs, field, x[:, :n], v[:, :n], 0.01, sub=(2, 2, 2))
        sim.step(3)
        sim.sort()
        st = gpu_state(sim)
        assert st["seg"][-1] == n
        sim.close()


def test_migrate_pass_on_arbitrary_segments_bit_exact(lcs):
    """lcs_migrate on a state whose segments do not match positions equals the
    sequential-counter migration of the oracle on the same input."""
    N, P = 12, (3, 2, 2)
    field, _, x, v, _ = synth.small_case(32, N, 8, 2.0, 20000, None)
    sim = make(lcs, field, x, v, 0.01, sub=P)
    g = np.random.default_rng(33)
    cut = np.sort(g.integers(0, 20000, 11))
    seg = np.concatenate([[0], cut, [20000]]).astype(np.int64)
    ids = g.permutation(20000).astype(np.int32)
    sim.set_state(x[:, ids], v[:, ids], ids, seg)
    sim.migrate()
    st = gpu_state(sim)
    dest, _ = oracle.keys(N, L, P, 1, x[:, ids])
    perm, seg_out, _ = oracle.migrate(12, seg, dest)
    assert np.array_equal(st["seg"], seg_out)
    assert np.array_equal(st["ids"], ids[perm])
    # positions are held in fixed point (cell units, 52 fraction bits) and
    # read back rounded to FP64: within one unit in the last place
    assert np.all(np.abs(st["x"] - x[:, ids][:, perm]) <= np.spacing(L))


def one_step_identical_inputs(lcs, N, P, n, tau_median, g, seed, dt=0.01, steps_before=3,
                              kernel="fp64"):
    field, _, x, v, tau = synth.small_case(seed, N, 24, N / 4.0, n, tau_median, dt=dt)
    sim = make(lcs, field, x, v, dt, tau=tau, sub=P, g=g, track_images=True, kernel=kernel)
    sim.step(steps_before)
    s0 = gpu_state(sim)
    sim.step(1)
    s1 = gpu_state(sim)
    # oracle advance from the GPU's own state, then compare values by id
    xo, vo = s0["x"].copy(), s0["v"].copy()
    img = s0["img"].copy()
    tau_s = s0["tau"] if tau is not None else None
    oracle.advance(field, L, xo, vo, tau_s, 0.1, dt, g, 1, img=img)
    xg, vg, ig = by_id(s1["ids"], s1["x"], s1["v"], s1["img"])
    xr, vr, ir = by_id(s0["ids"], xo, vo, img)
    dx = np.abs((xg + L * ig) - (xr + L * ir)).max()
    dv = np.abs(vg - vr).max() / np.abs(vr).max()
    # one step from identical states: FP64 differs from the oracle only in
    # rounding order; the DF step carries ~48-bit intermediates
    assert dx < 1e-13 and dv < (1e-13 if kernel == "fp64" else 1e-12), (dx, dv)
    # bit-exact migration: the oracle's sequential-counter migration applied to
    # the GPU's post-step positions in the pre-step storage order
    pos_of = np.empty(n, np.int64)
    pos_of[s1["ids"]] = np.arange(n)
    x_pre = s1["x"][:, pos_of[s0["ids"]]]
    dest, _ = oracle.keys(N, L, P, 1, x_pre)
    perm, seg_out, _ = oracle.migrate(int(np.prod(P)), s0["seg"], dest)
    assert np.array_equal(s1["seg"], seg_out)
    assert np.array_equal(s1["ids"], s0["ids"][perm])
    moved = int((dest != np.repeat(np.arange(int(np.prod(P))), np.diff(s0["seg"]))).sum())
    return moved


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("N,P,n", [(16, (2, 2, 2), 5000), (24, (3, 3, 3), 30011),
                                   (32, (4, 2, 1), 70000), (16, (1, 1, 1), 1500),
                                   (20, (5, 1, 2), 12345), (12, (12, 4, 1), 6000)])
def test_one_step_identical_inputs(lcs, N, P, n, kernel):
    # (12, (12, 4, 1)): subdomains one cell wide along x
    moved = one_step_identical_inputs(lcs, N, P, n, 0.05, (0.0, 0.0, -9.8), seed=40 + n, dt=0.02,
                                      kernel=kernel)
    if int(np.prod(P)) > 1:
        assert moved > 0  # the case exercises migration


# ---------------------------------------------------------------- trajectories

def run_pair(lcs, N, M, kmax, n, P, dt, steps, tau_median=None, tau_const=0.1, g=(0, 0, 0),
             sort_every=0, brick=8, seed=50, kernel="fp64"):
    field, _, x, v, tau = synth.small_case(seed, N, M, kmax, n, tau_median, tau_const, dt=dt)
    sim = make(lcs, field, x, v, dt, tau=tau, tau_const=tau_const, sub=P, g=g,
               sort_every=sort_every, sort_brick=brick, track_images=True, kernel=kernel)
    sim.step(steps)
    st = gpu_state(sim)
    ref = oracle.initial_state(N, L, P, x, v, tau, track_img=True)
    oracle.run(ref, field, L, P, tau_const, dt, g, steps, sort_every=sort_every, brick=brick)
    return st, ref, x


@pytest.mark.parametrize("kernel", KERNELS)
def test_plain_32_full_trajectory(kernel):
    """The plain FP64 workload: 32^3, 64 modes k 1-4, 32768 particles, tau 0.1,
    dt 0.01, 100 steps, 2x2x2 subdomains with migration every step."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2604_11008_gb300 as lcs
    w = synth.WORKLOADS["plain_32"]
    field, modes = synth.make_field(w)
    x, v, _ = synth.make_particles(w, w.dt)
    sim = lcs.Simulator(field, x, v, w.dt, tau_const=w.tau_const, sub=w.sub, kernel=kernel,
                        track_images=True)
    sim.step(w.steps)
    st = gpu_state(sim)
    ref = oracle.initial_state(w.N, L, w.sub, x, v, None, track_img=True)
    oracle.run(ref, field, L, w.sub, w.tau_const, w.dt, w.g, w.steps)
    ex, ev, px, pv = traj_errors(st["x"], st["img"], st["v"], st["ids"], ref, x)
    assert max(ex, ev, px, pv) < TOL_FP64, (ex, ev, px, pv)
    assert_same_storage(st, ref, w.N, w.sub)
    assert np.array_equal(np.sort(st["ids"]), np.arange(w.np_))


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("P,sort_every,brick", [((2, 2, 2), 5, 4), ((3, 3, 3), 4, 8),
                                                ((1, 1, 1), 3, 1)])
def test_trajectory_with_gravity_and_sort(lcs, P, sort_every, brick, kernel):
    N = 24
    st, ref, x0 = run_pair(lcs, N, 32, 6.0, 20000, P, 0.005, 30, tau_median=0.05,
                           g=(0.0, 0.0, -9.8), sort_every=sort_every, brick=brick, seed=60,
                           kernel=kernel)
    ex, ev, px, pv = traj_errors(st["x"], st["img"], st["v"], st["ids"], ref, x0)
    assert max(ex, ev, px, pv) < TOL_FP64, (ex, ev, px, pv)
    assert_same_storage(st, ref, N, P, brick)


def test_sort_pass_bit_exact_on_identical_inputs(lcs):
    N, P, B = 24, (2, 3, 2), 4
    field, _, x, v, _ = synth.small_case(70, N, 16, 4.0, 40000, None)
    sim = make(lcs, field, x, v, 0.01, sub=P)
    sim.step(4)
    s0 = gpu_state(sim)
    sim2 = None
    sim.sort()  # default brick 8
    s1 = gpu_state(sim)
    _, key = oracle.keys(N, L, P, 8, s0["x"])
    perm = oracle.sort(12, s0["seg"], key)
    assert np.array_equal(s1["seg"], s0["seg"])
    assert np.array_equal(s1["ids"], s0["ids"][perm])
    assert np.array_equal(s1["x"], s0["x"][:, perm])
    # keys are sorted within segments
    _, key1 = oracle.keys(N, L, P, 8, s1["x"])
    for s in range(12):
        k = key1[s1["seg"][s]:s1["seg"][s + 1]]
        assert np.all(np.diff(k) >= 0)


@pytest.mark.parametrize("kernel", KERNELS)
def test_many_tiles_ragged_tail(lcs, kernel):
    """Several thousand scan tiles per step with a ragged last tile per segment."""
    N, P = 32, (2, 2, 2)
    moved = one_step_identical_inputs(lcs, N, P, 1_000_003, 0.05, (0.0, 0.0, -9.8), seed=80,
                                      dt=0.02, steps_before=1, kernel=kernel)
    assert moved > 1000


# ---------------------------------------------------------------- errors are latched, not faults

@pytest.mark.parametrize("kernel", KERNELS)
def test_nonfinite_state_is_reported(lcs, kernel):
    field, _, x, v, _ = synth.small_case(90, 8, 4, 2.0, 100, None)
    sim = make(lcs, field, x, v, 0.01, sub=(2, 1, 1), kernel=kernel)
    st = gpu_state(sim)
    vv = st["v"].copy()
    vv[0, 7] = np.nan
    sim.set_state(st["x"], vv, st["ids"], st["seg"])
    sim.step(1)
    with pytest.raises(lcs.LcsError) as e:
        sim.sync()
    assert e.value.status == lcs.LCS_ERR_NONFINITE
    with pytest.raises(lcs.LcsError) as e:
        sim.step(1)
    assert e.value.status == lcs.LCS_ERR_STATE


@pytest.mark.parametrize("kernel", KERNELS)
def test_displacement_beyond_neighbour_is_reported(lcs, kernel):
    field, _, x, v, _ = synth.small_case(91, 12, 4, 2.0, 100, None)
    sim = make(lcs, field, x, v, 0.01, sub=(4, 1, 1), kernel=kernel)
    st = gpu_state(sim)
    vv = st["v"].copy()
    vv[0, :] = 250.0   # 2.5 per step: more than one subdomain width (pi/2)
    sim.set_state(st["x"], vv, st["ids"], st["seg"])
    sim.step(1)
    with pytest.raises(lcs.LcsError) as e:
        sim.sync()
    assert e.value.status == lcs.LCS_ERR_DISPLACEMENT


def test_invalid_arguments(lcs):
    field, _, x, v, _ = synth.small_case(92, 12, 4, 2.0, 100, None)
    with pytest.raises(lcs.LcsError) as e:
        make(lcs, field, x, v, 0.01, sub=(5, 1, 1))      # 12 % 5 != 0
    assert e.value.status == lcs.LCS_ERR_ARG
    with pytest.raises(lcs.LcsError) as e:
        make(lcs, field, x, v, 0.5, tau_const=0.1)       # dt > tau
    assert e.value.status == lcs.LCS_ERR_ARG
    for bad in (np.nan, np.inf, -np.inf, 1e300):         # not a position in any image
        xb = x.copy()
        xb[1, 3] = bad
        with pytest.raises(lcs.LcsError) as e:
            make(lcs, field, xb, v, 0.01)
        assert e.value.status == lcs.LCS_ERR_ARG


def test_positions_outside_the_box_are_folded(lcs):
    """Initial positions given in other periodic images (Sec. 2.1) start the
    same trajectories as their images in [0, L); with images tracked, the
    id-ordered export returns them unwrapped relative to the positions given."""
    N, P, dt, steps = 16, (2, 2, 2), 0.01, 20
    field, _, x, v, _ = synth.small_case(95, N, 16, 4.0, 4000, None, dt=dt)
    shift = np.random.default_rng(96).integers(-3, 4, size=x.shape).astype(np.float64)
    xs = x + L * shift
    xs[0, 0], xs[1, 1], xs[2, 2] = L, -L, 2 * L   # exactly on images of 0
    x[0, 0], x[1, 1], x[2, 2] = 0.0, 0.0, 0.0
    shift[0, 0], shift[1, 1], shift[2, 2] = 1.0, -1.0, 2.0
    a = make(lcs, field, x, v, dt, sub=P, track_images=True, sort_every=5)
    b = make(lcs, field, xs, v, dt, sub=P, track_images=True, sort_every=5)
    # the fold x - k L is one FMA rounding away from the image in [0, L)
    xa0, _ = a.final_state_by_id(device="cpu")
    xb0, _ = b.final_state_by_id(device="cpu")
    assert np.abs(xb0.numpy() - xs).max() <= 8 * np.spacing(4 * L)
    assert np.abs(xa0.numpy() - x).max() <= np.spacing(L)
    a.step(steps)
    b.step(steps)
    xa, va, ia = a.final_state_by_id(device="cpu", ids=True)
    xb, vb, ib = b.final_state_by_id(device="cpu", ids=True)
    assert np.array_equal(ia.numpy(), np.arange(4000)) and np.array_equal(ib.numpy(), ia.numpy())
    dx = np.abs(xb.numpy() - L * shift - xa.numpy()).max()
    assert dx < 1e-12, dx
    assert np.abs(vb.numpy() - va.numpy()).max() < 1e-12
    # the oracle from the folded positions, unwrapped by its own image counts
    ref = oracle.initial_state(N, L, P, x, v, None, track_img=True)
    oracle.run(ref, field, L, P, 0.1, dt, (0.0, 0.0, 0.0), steps, sort_every=5, brick=8)
    xr, vr, ir = by_id(ref.ids, ref.x, ref.v, ref.img)
    assert np.abs(xa.numpy() - (xr + L * ir)).max() < 1e-12
    assert np.abs(va.numpy() - vr).max() < 1e-12


def test_state_by_id_without_images_and_with_custom_ids(lcs):
    """Without image tracking the id-ordered export returns the wrapped
    positions of lcs_get_state; custom ids come back in ascending order."""
    N, P = 12, (3, 2, 2)
    field, _, x, v, _ = synth.small_case(97, N, 8, 2.0, 3000, None)
    ids = np.random.default_rng(98).choice(10 ** 9, 3000, replace=False).astype(np.uint32)
    sim = lcs.Simulator(field, x, v, 0.01, tau_const=0.1, sub=P, ids=ids.astype(np.int32),
                        sort_every=2)
    sim.step(5)
    st = gpu_state(sim)
    xb, vb, ib = sim.final_state_by_id(device="cpu", ids=True)
    order = np.argsort(st["ids"].astype(np.uint32), kind="stable")
    assert np.array_equal(ib.numpy().astype(np.uint32), np.sort(ids))
    assert np.array_equal(xb.numpy(), st["x"][:, order])
    assert np.array_equal(vb.numpy(), st["v"][:, order])


# ---------------------------------------------------------------- precision variants

def test_field_storage_rounding_is_exact(lcs):
    """The stored field equals round-to-nearest-even FP32 / BF16 of the FP64
    field (oracle rounding), and the float pair of the DF kernel is
    hi = RN32(u), lo = RN32(u - hi)."""
    field, _, x, v, _ = synth.small_case(100, 16, 16, 4.0, 10, None)
    field[0, 0, 0, :4] = [1.0 + 2.0 ** -8, 1.0 + 2.0 ** -8 + 2.0 ** -40, 3 * 2.0 ** -134, -0.0]
    want = {"f32": oracle.round_f32(field), "bf16": oracle.round_bf16(field)}
    hi = field.astype(np.float32).astype(np.float64)
    lo = (field - hi).astype(np.float32).astype(np.float64)
    for dtype, kernel, ref in (("f32", "auto", want["f32"]), ("bf16", "auto", want["bf16"]),
                               ("f64", "df", hi + lo), ("f64", "fp64", field)):
        sim = lcs.Simulator(field, x, v, 0.01, tau_const=0.1, field_dtype=dtype, kernel=kernel)
        got = sim.get_field().cpu().numpy()
        assert np.array_equal(got, ref), dtype
        sim.close()


@pytest.mark.parametrize("dtype,tol_q,tol_64", [("f32", 1e-6, 1e-5), ("bf16", 1e-5, 1e-2)])
def test_precision_variant_trajectories(lcs, dtype, tol_q, tol_64):
    """FP32 / BF16 field storage with FP32 interpolation: against the oracle on
    the same rounded field (isolates the FP32 arithmetic) and against the FP64
    oracle on the original field (the stated bars 1e-5 / 1e-2)."""
    N, P, dt, steps = 32, (2, 2, 2), 0.01, 50
    field, _, x, v, tau = synth.small_case(101, N, 32, 6.0, 20000, 0.1, dt=dt)
    g = (0.0, 0.0, -9.8)
    sim = lcs.Simulator(field, x, v, dt, tau=tau, g=g, sub=P, field_dtype=dtype,
                        track_images=True)
    sim.step(steps)
    st = gpu_state(sim)
    fq = oracle.round_f32(field) if dtype == "f32" else oracle.round_bf16(field)
    for f_ref, tol in ((fq, tol_q), (field, tol_64)):
        ref = oracle.initial_state(N, L, P, x, v, tau, track_img=True)
        oracle.run(ref, f_ref, L, P, 0.0, dt, g, steps)
        ex, ev, px, pv = traj_errors(st["x"], st["img"], st["v"], st["ids"], ref, x)
        assert max(ex, ev, px, pv) < tol, (dtype, ex, ev, px, pv)


@pytest.mark.parametrize("kernel", KERNELS)
def test_positions_on_cell_faces_and_box_edges(lcs, kernel):
    # degenerate positions: exactly on cell faces (x = k dx), on cell centres,
    # at 0 and one ulp below L, on subdomain faces; the oracle decides cells
    # with the same floor(x N/L), so storage and trajectories must agree
    N, P, dt, steps = 16, (2, 2, 2), 0.005, 6
    dx = L / N
    rng = np.random.default_rng(77)
    pts = [0.0, np.nextafter(L, 0.0), dx, 8 * dx, (N - 1) * dx, 0.5 * dx, 7.5 * dx,
           np.nextafter(8 * dx, 0.0), np.nextafter(8 * dx, L)]
    x = np.ascontiguousarray(rng.choice(pts, size=(3, 3000)))
    field, _, _, _, _ = synth.small_case(78, N, 16, 3.0, 1, None)
    v = np.ascontiguousarray(rng.standard_normal(x.shape))
    sim = make(lcs, field, x, v, dt, sub=P, track_images=True, kernel=kernel, sort_every=3,
               sort_brick=4)
    st0 = gpu_state(sim)
    ref0 = oracle.initial_state(N, L, P, x, v, None, track_img=True)
    assert np.array_equal(st0["seg"], ref0.seg)
    assert np.array_equal(st0["ids"].astype(np.uint32), ref0.ids)
    sim.step(steps)
    st = gpu_state(sim)
    ref = oracle.initial_state(N, L, P, x, v, None, track_img=True)
    oracle.run(ref, field, L, P, 0.1, dt, (0.0, 0.0, 0.0), steps, sort_every=3, brick=4)
    ex, ev, px, pv = traj_errors(st["x"], st["img"], st["v"], st["ids"], ref, x)
    assert max(ex, ev, px, pv) < TOL_FP64, (ex, ev, px, pv)
    assert_same_storage(st, ref, N, P, 4)


def test_capacity_overflow_is_reported(lcs):
    # 6000 particles of subdomain 0 cross into subdomain 1 (200 particles,
    # room for 200 + 200/16 + 128) in one step: the arrivals cannot be
    # placed, which is reported instead of written out of range
    N, P, dt = 16, (2, 1, 1), 0.01
    dx = L / N
    rng = np.random.default_rng(79)
    xa = np.stack([rng.uniform(7.2 * dx, 7.9 * dx, 6000), rng.uniform(0, L, 6000),
                   rng.uniform(0, L, 6000)])
    xb = np.stack([rng.uniform(9 * dx, 15 * dx, 200), rng.uniform(0, L, 200),
                   rng.uniform(0, L, 200)])
    x = np.ascontiguousarray(np.concatenate([xa, xb], axis=1))
    v = np.zeros_like(x)
    v[0, :6000] = 1.2 * dx / dt
    field = np.zeros((3, N, N, N))
    sim = make(lcs, field, x, v, dt, tau_const=1.0, sub=P)
    with pytest.raises(lcs.LcsError) as e:
        sim.step(1)
        sim.sync()
    assert e.value.status == lcs.LCS_ERR_CAPACITY
