"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed
forms, invariants, a library routine for a special case, the paper's worked
example, or brute force on tiny inputs.  No GPU needed.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth

L = synth.L_BOX


def periodic_trilinear_scipy(field, pts):
    """Trilinear interpolation by scipy on a periodically padded cell-centre grid."""
    from scipy.interpolate import RegularGridInterpolator
    N = field.shape[-1]
    dx = L / N
    c = (np.arange(-1, N + 1) + 0.5) * dx
    out = []
    for comp in range(3):
        f = field[comp]                      # [k, j, i]
        f = np.pad(f, 1, mode="wrap")        # periodic copies on every side
        f = np.transpose(f, (2, 1, 0))       # -> [i, j, k] to match (x, y, z)
        rgi = RegularGridInterpolator((c, c, c), f, method="linear")
        out.append(rgi(pts.T))
    return np.array(out)


# ---------------------------------------------------------------- interpolation

def test_interp_constant_field_everywhere():
    N = 8
    field = np.empty((3, N, N, N))
    field[0], field[1], field[2] = 1.25, -0.5, 3.0
    g = np.random.default_rng(1)
    x = g.random((3, 500)) * L
    x[:, :4] = [[0.0, L * (1 - 1e-16), 1e-300, L / 2]] * 3
    u = oracle.interp(field, L, x)
    assert np.allclose(u[0], 1.25, rtol=0, atol=1e-15)
    assert np.allclose(u[1], -0.5, rtol=0, atol=1e-15)
    assert np.allclose(u[2], 3.0, rtol=0, atol=1e-15)


def test_interp_reproduces_multilinear_field():
    """Trilinear interpolation is exact for a + bx + cy + dz + exy + fyz + gxz + hxyz."""
    N = 16
    dx = L / N
    xc = synth.cell_centres(N)
    Z, Y, X = np.meshgrid(xc, xc, xc, indexing="ij")
    coef = np.array([[0.3, 1.1, -0.7, 0.2, 0.05, -0.03, 0.08, 0.011],
                     [-1.0, 0.2, 0.4, -0.9, -0.02, 0.07, 0.01, -0.004],
                     [0.5, -0.3, 0.6, 0.1, 0.04, 0.02, -0.06, 0.009]])

    def f(c, x, y, z):
        a = coef[c]
        return (a[0] + a[1] * x + a[2] * y + a[3] * z + a[4] * x * y + a[5] * y * z
                + a[6] * x * z + a[7] * x * y * z)
    field = np.array([f(c, X, Y, Z) for c in range(3)])
    g = np.random.default_rng(2)
    # stencils that do not cross the periodic seam: x in [dx/2, L - dx/2)
    pts = dx / 2 + g.random((3, 2000)) * (L - dx)
    u = oracle.interp(field, L, pts)
    for c in range(3):
        exact = f(c, pts[0], pts[1], pts[2])
        assert np.max(np.abs(u[c] - exact)) < 1e-12


def test_interp_matches_scipy_including_seam():
    """Against scipy's RegularGridInterpolator (linear) on a periodically padded grid."""
    field, _, _, _, _ = synth.small_case(11, 12, 16, 3.0, 4, None)
    g = np.random.default_rng(3)
    pts = g.random((3, 3000)) * L
    N = 12
    dx = L / N
    pts[:, :6] = [[0.0, dx / 4, L - dx / 4, dx / 2, L - 1e-12, 2 * dx]] * 3
    u = oracle.interp(field, L, pts)
    ref = periodic_trilinear_scipy(field, pts)
    assert np.max(np.abs(u - ref)) < 1e-13


def test_interp_single_mode_second_order():
    """A single Fourier mode is recovered with O((k dx)^2) error (halves of dx -> /4)."""
    errs = []
    g = np.random.default_rng(4)
    pts = g.random((3, 4000)) * L
    for N in (32, 64, 128):
        xc = synth.cell_centres(N)
        Z, Y, X = np.meshgrid(xc, xc, xc, indexing="ij")
        field = np.zeros((3, N, N, N))
        field[0] = np.cos(2 * Y + 0.3)        # u(y) is divergence free
        u = oracle.interp(field, L, pts)
        errs.append(np.max(np.abs(u[0] - np.cos(2 * pts[1] + 0.3))))
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


def test_interp_transpose_dot_product_and_jacobian():
    """<interp(U)(X), mu> = <U, interp^T(X) mu>, and J^T mu matches finite differences."""
    field, _, x, _, _ = synth.small_case(12, 8, 8, 2.0, 300, None)
    g = np.random.default_rng(5)
    mu = g.standard_normal((3, 300))
    u = oracle.interp(field, L, x)
    gf, jt = oracle.interp_transpose(field, L, x, mu)
    lhs = float(np.sum(u * mu))
    rhs = float(np.sum(field * gf))
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))
    # J^T mu by central differences along each axis (h small inside one cell)
    h = 1e-7
    N = field.shape[-1]
    for s in range(3):
        frac = (x[s] * N / L - 0.5) % 1.0
        ok = (frac > 1e-4) & (frac < 1 - 1e-4)
        xp, xm = x.copy(), x.copy()
        xp[s] += h
        xm[s] -= h
        fd = np.sum((oracle.interp(field, L, xp) - oracle.interp(field, L, xm)) * mu, 0) / (2 * h)
        assert np.max(np.abs(fd[ok] - jt[s][ok])) < 1e-6


# ---------------------------------------------------------------- Heun + drag

def uniform_field(N, U0):
    f = np.empty((3, N, N, N))
    for c in range(3):
        f[c] = U0[c]
    return f


def test_heun_uniform_flow_discrete_closed_form():
    """Uniform flow + gravity: V^n - Vinf = r^n (V0 - Vinf), r = 1 - h + h^2/2, and the
    matching closed form of X^n (exact discrete solution of Heun's method)."""
    N = 8
    U0 = np.array([0.7, -0.4, 0.25])
    gvec = np.array([0.1, -0.3, -9.8])
    field = uniform_field(N, U0)
    n = 64
    g = np.random.default_rng(6)
    x = g.random((3, n)) * L
    v = g.standard_normal((3, n))
    tau = np.exp(g.uniform(np.log(0.05), np.log(1.0), n))
    dt, steps = 0.01, 50
    x0, v0 = x.copy(), v.copy()
    img = np.zeros((3, n), np.int32)
    st = oracle.advance(field, L, x, v, tau, 0.0, dt, gvec, steps, img=img)
    assert st == oracle.ORC_OK
    h = dt / tau
    r = 1 - h + h * h / 2
    vinf = U0[:, None] + tau[None, :] * gvec[:, None]
    d0 = v0 - vinf
    v_ref = vinf + r ** steps * d0
    x_ref = x0 + steps * dt * vinf + dt * (1 - h / 2) * d0 * (1 - r ** steps) / (1 - r)
    xu = x + L * img
    assert np.max(np.abs(v - v_ref) / np.abs(vinf).max()) < 1e-13
    assert np.max(np.abs(xu - x_ref)) < 1e-12


def test_heun_converges_second_order_to_exponential_relaxation():
    """Continuous solution V = Vinf + (V0-Vinf) e^{-t/tau}: error falls 4x per halving of dt."""
    N = 8
    U0 = np.array([0.3, 0.2, -0.1])
    gvec = np.array([0.0, 0.0, -9.8])
    field = uniform_field(N, U0)
    tau, T = 0.2, 0.4
    x0 = np.full((3, 1), 1.0)
    v0 = np.array([[1.0], [-1.0], [0.5]])
    vinf = U0 + tau * gvec
    errs = []
    for dt in (0.02, 0.01, 0.005):
        x, v = x0.copy(), v0.copy()
        img = np.zeros((3, 1), np.int32)
        oracle.advance(field, L, x, v, None, tau, dt, gvec, int(round(T / dt)), img=img)
        e = math.exp(-T / tau)
        v_ex = vinf + (v0[:, 0] - vinf) * e
        x_ex = x0[:, 0] + vinf * T + tau * (v0[:, 0] - vinf) * (1 - e)
        errs.append(max(np.max(np.abs(v[:, 0] - v_ex)),
                        np.max(np.abs(x[:, 0] + L * img[:, 0] - x_ex))))
    assert 3.6 < errs[0] / errs[1] < 4.4 and 3.6 < errs[1] / errs[2] < 4.4


def _nonlinear_relaxation(w0, tau, nu, rr, t):
    """Exact speed relative to a uniform fluid under the drag factor of Eq. (7):
    dw/dt = -(1 + c w^a) w / tau with a = 0.687, c = 0.15 (2r/nu)^a and
    tau = (2/9) rr r^2 / nu.  Separating variables, y = w^a obeys
    y / (1 + c y) = K exp(-a t / tau) with K = y0 / (1 + c y0)."""
    a = 0.687
    r = math.sqrt(9.0 * nu * tau / (2.0 * rr))
    c = 0.15 * (2.0 * r / nu) ** a
    y0 = w0 ** a
    k = y0 / (1.0 + c * y0) * math.exp(-a * t / tau)
    return (k / (1.0 - c * k)) ** (1.0 / a)


def test_nonlinear_drag_converges_second_order_to_exact_relaxation():
    """Uniform flow, no gravity, relative speeds giving Re_p from about 0.5 to 5:
    the oracle's Heun steps with the drag of Eq. (7) approach the exact speed and
    displacement (the latter by quadrature) at second order."""
    from scipy.integrate import quad
    N, nu, rr, T = 4, 1e-3, 843.0, 0.4
    U0 = np.array([0.3, -0.2, 0.1])
    field = uniform_field(N, U0)
    cases = [(0.5, 0.05), (2.0, 0.05), (5.0, 0.2), (3.0, 0.1)]   # (w0, tau)
    e = np.array([[1.0, 0.0, 0.0], [0.0, 0.6, 0.8], [0.48, 0.6, 0.64], [0.0, 0.0, 1.0]]).T
    e = np.ascontiguousarray(e / np.linalg.norm(e, axis=0))
    w0 = np.array([c[0] for c in cases])
    tau = np.array([c[1] for c in cases])
    w_ref = np.array([_nonlinear_relaxation(w, tp, nu, rr, T) for w, tp in cases])
    d_ref = np.array([quad(lambda t, w=w, tp=tp: _nonlinear_relaxation(w, tp, nu, rr, t), 0, T,
                           epsabs=1e-14, epsrel=1e-13)[0] for w, tp in cases])
    errs = []
    for steps in (40, 80, 160, 320):
        x = np.full((3, len(cases)), 1.0)
        v = np.ascontiguousarray(U0[:, None] + w0[None, :] * e)
        img = np.zeros(x.shape, np.int32)
        st = oracle.advance(field, L, x, v, tau, 0.0, T / steps, np.zeros(3), steps, img=img,
                            drag=(1, nu, rr))
        assert st == oracle.ORC_OK
        wv = v - U0[:, None]
        xu = x + L * img - 1.0 - U0[:, None] * T
        errs.append(max(np.max(np.abs(wv - w_ref * e)), np.max(np.abs(xu - d_ref * e))))
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(3.6 < q < 4.4 for q in ratios), (errs, ratios)
    assert errs[-1] < 1e-5


def test_nonlinear_drag_rejects_bad_parameters():
    field = uniform_field(4, np.zeros(3))
    x = np.full((3, 2), 1.0)
    v = np.zeros((3, 2))
    for drag in ((1, 0.0, 843.0), (1, 1e-3, -1.0), (2, 1e-3, 843.0)):
        st = oracle.advance(field, L, x, v, None, 0.1, 0.01, np.zeros(3), 1, drag=drag)
        assert st == oracle.ORC_ERR_ARG


def test_evolving_field_converges_second_order_to_exact_solution():
    """Two uniform snapshots U_a at t_a and U_b at t_b: the fluid velocity is
    U(t) = c0 + c1 t, and dV/dt = (U(t) - V)/tau + g has the exact solution
    V = c0 + c1 t + tau g - tau c1 + (V0 - c0 - tau g + tau c1) e^{-t/tau}
    (and X by integration).  Heun with the stage times t and t + dt converges
    at second order; evaluating the second stage at the wrong time would
    leave a first-order error."""
    N, T = 4, 0.5
    Ua, Ub = np.array([0.4, -0.3, 0.2]), np.array([-0.6, 0.5, 1.1])
    ta, tb, t0 = -0.2, 0.8, 0.1
    fa, fb = uniform_field(N, Ua), uniform_field(N, Ub)
    gvec = np.array([0.0, 0.3, -1.0])
    c1 = (Ub - Ua) / (tb - ta)
    rng = np.random.default_rng(17)
    n = 6
    x0 = rng.random((3, n)) * L
    v0 = rng.standard_normal((3, n))
    tau = np.array([0.05, 0.1, 0.2, 0.3, 0.5, 1.0])

    def exact(t):  # time measured from t0
        c0 = Ua + (t0 - ta) * c1                 # U at the start time
        vinf0 = c0[:, None] + tau * gvec[:, None] - tau * c1[:, None]
        a = v0 - vinf0
        e = np.exp(-t / tau)
        v = vinf0 + c1[:, None] * t + a * e
        x = x0 + vinf0 * t + 0.5 * c1[:, None] * t * t + tau * a * (1 - e)
        return x, v

    xr, vr = exact(T)
    errs = []
    for steps in (50, 100, 200, 400):
        x, v = x0.copy(), v0.copy()
        img = np.zeros((3, n), np.int32)
        st = oracle.advance(fa, L, x, v, tau, 0.0, T / steps, gvec, steps, img=img, field_b=fb,
                            times=(t0, ta, tb))
        assert st == oracle.ORC_OK
        errs.append(max(np.max(np.abs(x + L * img - xr)), np.max(np.abs(v - vr))))
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(3.6 < q < 4.4 for q in ratios), (errs, ratios)


def test_evolving_field_with_equal_snapshots_is_the_frozen_field():
    field, _, x, v, tau = synth.small_case(18, 8, 8, 2.0, 50, 0.1)
    xa, va, xb, vb = x.copy(), v.copy(), x.copy(), v.copy()
    oracle.advance(field, L, xa, va, tau, 0.0, 0.01, np.zeros(3), 20)
    oracle.advance(field, L, xb, vb, tau, 0.0, 0.01, np.zeros(3), 20, field_b=field,
                   times=(0.3, 0.0, 1.0))
    assert np.abs(xa - xb).max() < 1e-14 and np.abs(va - vb).max() < 1e-14


def test_pair_histogram_of_a_cubic_lattice():
    """m^3 points of a simple cubic lattice filling the periodic box (spacing
    a = L/m): every point has 6 neighbours at a, 12 at a sqrt(2), 8 at
    a sqrt(3) and 6 at 2a, so the unordered pair counts are 3n, 6n, 4n, 3n
    (m >= 5 keeps 2a below L/2; the minimum image joins the faces)."""
    m = 6
    a = L / m
    g = np.arange(m) * a + 0.1 * a
    x = np.stack([c.ravel() for c in np.meshgrid(g, g, g, indexing="ij")])
    n = m ** 3
    r_max, nbins = 2.21 * a, 13         # bins of 0.17 a: 1, 1.414, 1.732, 2 lie inside bins
    c = oracle.pair_hist(x, L, r_max, nbins)
    want = np.zeros(nbins, np.int64)
    for k, mult in ((1.0, 3), (math.sqrt(2), 6), (math.sqrt(3), 4), (2.0, 3)):
        want[int(k / 0.17)] += mult * n
    assert np.array_equal(c, want), (c, want)


def test_pair_histogram_of_uniform_points_gives_g_near_one():
    """Uniform random points: counts / (n(n-1)/2 * shell volume / L^3) ~ 1."""
    rng = np.random.default_rng(9)
    n = 4000
    x = rng.random((3, n)) * L
    r_max, nbins = 0.6, 6
    c = oracle.pair_hist(x, L, r_max, nbins)
    edges = np.linspace(0, r_max, nbins + 1)
    shell = 4.0 / 3.0 * math.pi * (edges[1:] ** 3 - edges[:-1] ** 3)
    g = c / (n * (n - 1) / 2 * shell / L ** 3)
    assert np.all(np.abs(g[1:] - 1) < 0.15) and abs(g[0] - 1) < 0.6, g


def test_per_stage_migration_moves_particles_between_the_stages():
    """Migration after each Runge-Kutta stage (Sec. 3.2.2): the trajectories are
    those of the single-migration step bit for bit (same arithmetic, only the
    storage moves), every particle ends in the segment of its position, and
    particles whose predictor X* left the subdomain were moved before the second
    stage (their order differs from the single-migration order)."""
    N, P = 12, (3, 2, 2)
    field, _, x, v, tau = synth.small_case(41, N, 12, 3.0, 6000, 0.05, dt=0.02)
    v = np.ascontiguousarray(v + 3.0 * np.random.default_rng(5).standard_normal(v.shape))
    a = oracle.initial_state(N, L, P, x, v, tau, track_img=True)
    b = a.copy()
    g = (0.0, 0.0, -9.8)
    oracle.run(a, field, L, P, 0.0, 0.02, g, 6, sort_every=4, brick=2)
    oracle.run(b, field, L, P, 0.0, 0.02, g, 6, sort_every=4, brick=2, per_stage=True)
    oa, ob = np.argsort(a.ids), np.argsort(b.ids)
    assert np.array_equal(a.x[:, oa], b.x[:, ob]) and np.array_equal(a.v[:, oa], b.v[:, ob])
    assert np.array_equal(a.img[:, oa], b.img[:, ob])
    dest, _ = oracle.keys(N, L, P, 1, b.x)
    seg_of = np.repeat(np.arange(12), np.diff(b.seg))
    assert np.array_equal(dest, seg_of)
    assert np.array_equal(a.seg, b.seg) and not np.array_equal(a.ids, b.ids)


def test_heun_stage_structure_brute_force():
    """One step on a random field equals the Heun formulas evaluated with the
    independent scipy interpolator (catches a wrong stage, sign or weight)."""
    field, _, x, _, tau = synth.small_case(13, 10, 12, 3.0, 200, 0.3, sigma=0.3, dt=0.02)
    g = np.random.default_rng(7)
    v = g.standard_normal((3, 200)) * 0.5
    gvec = np.array([0.0, 0.5, -1.0])
    dt = 0.02
    x1, v1 = x.copy(), v.copy()
    img = np.zeros((3, 200), np.int32)
    oracle.advance(field, L, x1, v1, tau, 0.0, dt, gvec, 1, img=img)
    u1 = periodic_trilinear_scipy(field, x)
    a1 = (u1 - v) / tau + gvec[:, None]
    xs = x + dt * v
    vs = v + dt * a1
    u2 = periodic_trilinear_scipy(field, np.mod(xs, L))
    a2 = (u2 - vs) / tau + gvec[:, None]
    xr = x + 0.5 * dt * (v + vs)
    vr = v + 0.5 * dt * (a1 + a2)
    assert np.max(np.abs(v1 - vr)) < 1e-12
    assert np.max(np.abs(x1 + L * img - xr)) < 1e-12


# ---------------------------------------------------------------- wrap and keys

def test_wrap_keeps_positions_in_box_and_counts_images():
    N = 8
    field = uniform_field(N, [3.0, -3.0, 0.0])
    n = 6
    x = np.array([[L - 1e-3, 1e-3, L - 1e-15, 0.0, 5e-17, L / 2]] * 3)
    x[2] = 1.0
    v = np.array([[3.0] * n, [-3.0] * n, [0.0] * n])
    img = np.zeros((3, n), np.int32)
    xu0 = x.copy()
    for _ in range(20):
        oracle.advance(field, L, x, v, None, 1.0, 0.01, [0, 0, 0], 1, img=img)
        assert np.all(x >= 0.0) and np.all(x < L)
    # unwrapped displacement 20 * 0.01 * 3 = 0.6 along +x, -0.6 along y
    assert np.allclose(x[0] + L * img[0] - xu0[0], 0.6, atol=1e-12)
    assert np.allclose(x[1] + L * img[1] - xu0[1], -0.6, atol=1e-12)


def test_keys_brute_force_at_cell_faces():
    """dest and key vs Python integer arithmetic on positions at and next to cell faces."""
    N, P, B = 24, (2, 3, 4), 4
    inv = oracle.inv_dx(N, L)
    vals = [0.0, L - 2 * np.spacing(L), np.nextafter(L, 0)]
    for c in range(N + 1):
        face = c / inv
        vals += [face, np.nextafter(face, 0), np.nextafter(face, 10)]
    vals = np.array([v for v in vals if 0.0 <= v < L])
    g = np.random.default_rng(8)
    n = 3000
    x = np.stack([g.choice(vals, n) for _ in range(3)])
    dest, key = oracle.keys(N, L, P, B, x)
    for p in range(n):
        c = [min(math.floor(x[s, p] * inv), N - 1) for s in range(3)]
        W = [N // P[s] for s in range(3)]
        ps = [c[s] // W[s] for s in range(3)]
        assert dest[p] == ps[0] + P[0] * (ps[1] + P[1] * ps[2])
        loc = [c[s] - ps[s] * W[s] for s in range(3)]
        b = [loc[s] // B for s in range(3)]
        r = [loc[s] % B for s in range(3)]
        nb = [-(-W[s] // B) for s in range(3)]
        k = ((b[2] * nb[1] + b[1]) * nb[0] + b[0]) * B ** 3 + (r[2] * B + r[1]) * B + r[0]
        assert key[p] == k


def test_brick_one_is_plain_cell_order():
    N, P = 16, (1, 1, 1)
    g = np.random.default_rng(9)
    x = g.random((3, 1000)) * L
    _, key = oracle.keys(N, L, P, 1, x)
    c = np.minimum(np.floor(x * (N / L)).astype(np.int64), N - 1)
    assert np.array_equal(key, c[0] + N * (c[1] + N * c[2]))


# ---------------------------------------------------------------- migration

def test_migration_worked_example(worked_example):
    """Sec. 2.3.3 example: particles 2 and 4 go to send-buffer slots 1 and 2 (1-based)."""
    mask = [r[1] for r in worked_example]
    scan = [r[2] for r in worked_example]
    # five particles in subdomain 0 of P = 2; mask 1 means leaving to subdomain 1
    seg = np.array([0, 5, 5])
    dest = np.array(mask, np.int32)
    perm, seg_out, slot = oracle.migrate(2, seg, dest)
    for i, m in enumerate(mask):
        if m:
            assert slot[i] + 1 == scan[i]          # 0-based counter -> 1-based slot
    assert list(seg_out) == [0, 3, 5]
    assert list(perm) == [0, 2, 4, 1, 3]           # stayers 1,3,5 then packed 2,4


def brute_force_migration(P, seg, dest):
    src = np.repeat(np.arange(P), np.diff(seg))
    order = sorted(range(len(dest)), key=lambda i: (dest[i], dest[i] != src[i]))
    counts = np.bincount(dest, minlength=P)
    return np.array(order), np.concatenate([[0], np.cumsum(counts)])


@pytest.mark.parametrize("P", [1, 2, 3, 8, 27])
def test_migration_brute_force_tiny(P):
    g = np.random.default_rng(100 + P)
    for trial in range(200):
        n = int(g.integers(0, 65))
        cut = np.sort(g.integers(0, n + 1, P - 1))
        seg = np.concatenate([[0], cut, [n]]).astype(np.int64)
        src = np.repeat(np.arange(P), np.diff(seg))
        stay = g.random(n) < 0.6
        dest = np.where(stay, src, g.integers(0, P, n)).astype(np.int32)
        perm, seg_out, slot = oracle.migrate(P, seg, dest)
        ref_perm, ref_seg = brute_force_migration(P, seg, dest)
        assert np.array_equal(perm, ref_perm)
        assert np.array_equal(seg_out, ref_seg)
        # invariants: bijection, every particle lands in its destination segment
        assert np.array_equal(np.sort(perm), np.arange(n))
        new_seg_of = np.repeat(np.arange(P), np.diff(seg_out))
        assert np.array_equal(new_seg_of, dest[perm])
        # race-free pack: per (src, dest) pair the slots are exactly 0..count-1
        for s in range(P):
            for d in range(P):
                sel = (src == s) & (dest == d)
                assert np.array_equal(np.sort(slot[sel]), np.arange(sel.sum()))


def test_migration_conserves_ids_through_a_run():
    field, _, x, v, tau = synth.small_case(14, 16, 16, 3.0, 4000, 0.05, dt=0.01)
    P = (2, 2, 2)
    st = oracle.initial_state(16, L, P, x, v, tau)
    assert np.array_equal(np.sort(st.ids), np.arange(4000))
    oracle.run(st, field, L, P, 0.0, 0.01, (0, 0, -9.8), 30, sort_every=10, brick=4)
    assert np.array_equal(np.sort(st.ids), np.arange(4000))
    dest, _ = oracle.keys(16, L, P, 1, st.x)
    seg_of = np.repeat(np.arange(8), np.diff(st.seg))
    assert np.array_equal(seg_of, dest)


def test_initial_state_keeps_id_order_per_subdomain():
    g = np.random.default_rng(15)
    x = g.random((3, 500)) * L
    st = oracle.initial_state(8, L, (2, 2, 1), x, np.zeros_like(x), None)
    for s in range(4):
        ids = st.ids[st.seg[s]:st.seg[s + 1]]
        assert np.all(np.diff(ids.astype(np.int64)) > 0)


# ---------------------------------------------------------------- sort

def test_sort_is_stable_per_segment_brute_force():
    g = np.random.default_rng(16)
    for trial in range(50):
        P = int(g.integers(1, 6))
        n = int(g.integers(0, 200))
        cut = np.sort(g.integers(0, n + 1, P - 1))
        seg = np.concatenate([[0], cut, [n]]).astype(np.int64)
        key = g.integers(0, 7, n).astype(np.int64)
        perm = oracle.sort(P, seg, key)
        for s in range(P):
            a, b = seg[s], seg[s + 1]
            ref = sorted(range(a, b), key=lambda i: key[i])
            assert list(perm[a:b]) == ref


# ---------------------------------------------------------------- adjoint

def fd_grad_check(field, x0, v0, tau, dt, steps, target, seed):
    """Directional derivatives of the loss by central differences vs the adjoint."""
    n = x0.shape[1]
    gvec = np.zeros(3)

    def run(xa, va, fa):
        x, v = xa.copy(), va.copy()
        img = np.zeros((3, n), np.int32)
        hsh = np.zeros(n, np.uint64)
        oracle.advance(fa, L, x, v, tau, 0.1, dt, gvec, steps, img=img, cellhash=hsh)
        return x, img, hsh

    x, img, h0 = run(x0, v0, field)
    xu = x + L * img
    lx = 2.0 / n * (xu - target)
    gx, gv, gf = oracle.adjoint(field, L, x0, v0, tau, 0.1, dt, gvec, steps, lx,
                                np.zeros((3, n)))
    g = np.random.default_rng(seed)
    h = 1e-6
    worst = 0.0
    for trial in range(6):
        dxx, dvv, dff = (g.standard_normal(x0.shape), g.standard_normal(v0.shape),
                         g.standard_normal(field.shape))
        xp, ip, hp = run(x0 + h * dxx, v0 + h * dvv, field + h * dff)
        xm, im, hm = run(x0 - h * dxx, v0 - h * dvv, field - h * dff)
        mask = ((hp == h0) & (hm == h0)).astype(np.float64)
        # [L(+h) - L(-h)] / 2h subtracted term by term ((a-t)^2 - (b-t)^2 =
        # (a-b)(a+b-2t)) so that the summation rounding of L does not enter
        up, um = xp + L * ip, xm + L * im
        fd = float(np.sum(mask * ((up - um) * (up + um - 2 * target)).sum(0)) / n) / (2 * h)
        assert abs(fd - (oracle.loss(L, xp, ip, target, mask)
                         - oracle.loss(L, xm, im, target, mask)) / (2 * h)) < 1e-6 * abs(fd)
        # adjoint restricted to the same particles: rerun with masked seed
        lxm = lx * mask[None, :]
        gxm, gvm, gfm = oracle.adjoint(field, L, x0, v0, tau, 0.1, dt, gvec, steps, lxm,
                                       np.zeros((3, n)))
        ad = np.sum(gxm * dxx) + np.sum(gvm * dvv) + np.sum(gfm * dff)
        worst = max(worst, abs(fd - ad) / max(abs(ad), 1e-30))
    return worst


def test_adjoint_matches_finite_differences_one_step():
    field, _, x, v, _ = synth.small_case(17, 8, 12, 3.0, 64, None)
    g = np.random.default_rng(18)
    v = g.standard_normal(x.shape) * 0.3
    target = g.random((3, 64)) * L
    assert fd_grad_check(field, x, v, None, 0.02, 1, target, 19) < 1e-6


def test_adjoint_matches_finite_differences_many_steps():
    field, _, x, v, tau = synth.small_case(20, 8, 12, 3.0, 64, 0.1, sigma=0.4, dt=0.02)
    target = np.random.default_rng(21).random((3, 64)) * L
    assert fd_grad_check(field, x, v, tau, 0.02, 25, target, 22) < 1e-6


def test_adjoint_full_jacobian_tiny():
    """N = 4, 8 particles, 3 steps: every entry of d(x_T)/d(x0, v0) by FD vs adjoint rows."""
    field, _, x0, _, _ = synth.small_case(23, 4, 3, 1.5, 8, None)
    g = np.random.default_rng(24)
    v0 = g.standard_normal(x0.shape) * 0.2
    dt, steps, n, h = 0.05, 3, 8, 1e-6
    gvec = np.zeros(3)

    def fwd(xa, va):
        x, v = xa.copy(), va.copy()
        img = np.zeros((3, n), np.int32)
        oracle.advance(field, L, x, v, None, 0.1, dt, gvec, steps, img=img)
        return x + L * img
    for s_out in range(3):
        lx = np.zeros((3, n))
        lx[s_out] = 1.0            # rows d(sum_p x_T[s_out, p]) / d(inputs)
        gx, gv, _ = oracle.adjoint(field, L, x0, v0, None, 0.1, dt, gvec, steps, lx,
                                   np.zeros((3, n)), want_field=False)
        for s_in in range(3):
            for p in range(n):
                for which, grad in (("x", gx), ("v", gv)):
                    xp, xm, vp, vm = x0.copy(), x0.copy(), v0.copy(), v0.copy()
                    if which == "x":
                        xp[s_in, p] += h
                        xm[s_in, p] -= h
                    else:
                        vp[s_in, p] += h
                        vm[s_in, p] -= h
                    fd = (fwd(xp, vp)[s_out, p] - fwd(xm, vm)[s_out, p]) / (2 * h)
                    assert abs(fd - grad[s_in, p]) < 1e-6 * max(1.0, abs(fd))


# ---------------------------------------------------------------- rounding

def test_round_f32_matches_numpy():
    g = np.random.default_rng(25)
    a = g.standard_normal(10000) * 10.0 ** g.integers(-30, 30, 10000)
    assert np.array_equal(oracle.round_f32(a), a.astype(np.float32).astype(np.float64))


def test_round_bf16_direct_rne_cases():
    one = 1.0
    cases = {
        one + 2.0 ** -8: 1.0,                              # tie -> even (1.0)
        one + 3 * 2.0 ** -8: one + 2.0 ** -6,              # tie -> even (mantissa 2)
        one + 2.0 ** -8 + 2.0 ** -40: one + 2.0 ** -7,     # just above the tie: up
        -(one + 2.0 ** -8 + 2.0 ** -40): -(one + 2.0 ** -7),
        2.0 ** -130: 2.0 ** -130,                          # subnormal, representable
        3 * 2.0 ** -134: 2.0 ** -132,                      # subnormal tie 1.5 -> 2 (even)
        0.0: 0.0,
    }
    a = np.array(list(cases.keys()))
    assert np.array_equal(oracle.round_bf16(a), np.array(list(cases.values())))


def test_round_bf16_matches_torch_on_float_inputs():
    torch = pytest.importorskip("torch")
    g = np.random.default_rng(26)
    a = (g.standard_normal(20000) * 10.0 ** g.integers(-20, 20, 20000)).astype(np.float32)
    ref = torch.from_numpy(a).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(oracle.round_bf16(a.astype(np.float64)), ref)


def test_openmp_build_of_the_oracle_gives_identical_bits():
    """The all-cores build (OpenMP over particles, used only to time the CPU
    baseline) computes every particle with the same arithmetic: trajectories,
    image counts and the migration after them equal the plain build's bit
    for bit."""
    field, _, x, v, tau = synth.small_case(9, 16, 8, 3.0, 5000, 0.05, dt=0.01)
    out = []
    for threads in (None, 0):
        if oracle.use_threads(threads) is None:
            pytest.skip("no OpenMP build on this machine")
        st = oracle.initial_state(16, L, (2, 2, 2), x, v, tau, track_img=True)
        oracle.run(st, field, L, (2, 2, 2), 0.0, 0.01, (0.0, 0.0, -9.8), 12, sort_every=5,
                   brick=4)
        out.append(st)
    oracle.use_threads(None)
    a, b = out
    for k in ("x", "v", "img", "ids", "seg"):
        assert np.array_equal(getattr(a, k), getattr(b, k)), k


def test_loss_worked_example_and_image_invariance():
    """orc_loss, the adjoint's objective: the mean over all n particles of the
    (masked) squared distance between the unwrapped final position X + L img
    and the target.  Worked by hand on two particles with binary-exact
    values, so that a dropped image term, a dropped component or a mean over
    the masked count instead of n changes the result; and the same loss when
    a position moves by one box length while its image count moves back."""
    Lb = 2.0 * np.pi
    x = np.array([[1.0, 0.5], [2.0, 0.25], [3.0, 0.0]])
    img = np.array([[1, 0], [0, 0], [-1, 0]], np.int32)
    target = np.array([[1.0 + Lb, 0.0], [2.0, 0.0], [3.0 - Lb, 0.0]])
    # particle 0 sits on its target once unwrapped; particle 1 is
    # (0.5, 0.25, 0) away: 0.25 + 0.0625 = 0.3125; mean over n = 2
    assert oracle.loss(Lb, x, img, target) == 0.15625
    assert oracle.loss(Lb, x, img, target, mask=np.array([1.0, 2.0])) == 0.3125
    assert oracle.loss(Lb, x, img, target, mask=np.array([0.0, 1.0])) == 0.15625
    # without image counts particle 0 is one box length off in x and z
    assert oracle.loss(Lb, x, None, target) == pytest.approx((2 * Lb * Lb + 0.3125) / 2,
                                                             rel=1e-15)
    x2, img2 = x.copy(), img.copy()
    x2[1, 1] += Lb
    img2[1, 1] -= 1
    assert oracle.loss(Lb, x2, img2, target) == pytest.approx(0.15625, abs=1e-15)
