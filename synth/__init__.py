"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module holds none of the particle method's arithmetic (no interpolation,
no time integration, no wrap, no migration, no sort).  It only draws inputs:

* a frozen, divergence-free, periodic velocity field made of random Fourier
  modes, sampled at cell centres ((i+1/2)dx, (j+1/2)dx, (k+1/2)dx) of an N^3
  grid on the periodic cube of side L = 2*pi (the paper's domain, Sec. 2.1);
* uniform random particle positions, zero initial velocities, and log-normal
  particle relaxation times (tau_p of Sec. 2.2);
* loss targets and finite-difference directions for the gradient checks;
* the time step from the convective CFL rule of Eq. (3) with C1 = 0.3.

Every random stream is ``numpy.random.Generator(PCG64(1000*workload + stream))``
with streams 0 field modes, 1 positions, 2 tau_p, 3 targets, 4 FD directions,
5 ensemble sizes.  The field is synthesised with an inverse FFT of the exact
mode coefficients (integer wavevectors, half-cell phase shift), so it equals
the direct mode sum to rounding; ``direct_sum`` evaluates that sum at arbitrary
points for spot checks.

Arrays use the layouts of the library: field ``[3, N, N, N]`` indexed
``[component, k(z), j(y), i(x)]`` (x fastest), particles as SoA float64.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

L_BOX = 2.0 * math.pi
STREAM_FIELD, STREAM_POS, STREAM_TAU, STREAM_TARGET, STREAM_FD, STREAM_ENS = range(6)


def rng(workload: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(1000 * workload + stream))


@dataclasses.dataclass
class Modes:
    k: np.ndarray       # (M, 3) int64 integer wavevectors (k_x, k_y, k_z)
    amp: np.ndarray     # (M,) float64 amplitudes |k|^(-5/6)
    pol: np.ndarray     # (M, 3) float64 unit polarisation, pol . k = 0
    phase: np.ndarray   # (M,) float64 phases in [0, 2 pi)
    scale: float = 1.0  # overall factor S applied by field_from_modes


def draw_modes(M: int, kmin: float, kmax: float, g: np.random.Generator) -> Modes:
    """M distinct random integer wavevectors with |k| in [kmin, kmax].

    |k| is uniform in [kmin, kmax] and the direction uniform on the sphere;
    the vector is rounded to the nearest integer wavevector (needed for
    2*pi periodicity) and rejected if zero, out of range, or equal to +-k of
    an accepted mode.  Amplitude |k|^(-5/6): with |k| uniform this makes the
    shell-summed spectrum E(k) ~ k^(-5/3).  The polarisation is r x k for a
    random r, so every mode (and the field) is exactly divergence free.
    """
    ks, seen = [], set()
    draws = 0
    while len(ks) < M:
        draws += 1
        if draws > 10000 * M:  # the shell holds fewer than M distinct +-k pairs
            raise ValueError(f"cannot draw {M} distinct wavevectors with {kmin} <= |k| <= {kmax}")
        mag = g.uniform(kmin, kmax)
        d = g.standard_normal(3)
        d /= np.linalg.norm(d)
        kv = np.rint(mag * d).astype(np.int64)
        n = float(np.linalg.norm(kv))
        key, nkey = tuple(kv), tuple(-kv)
        if n == 0.0 or n < kmin or n > kmax or key in seen or nkey in seen:
            continue
        seen.add(key)
        ks.append(kv)
    k = np.array(ks, dtype=np.int64)
    amp = np.linalg.norm(k, axis=1) ** (-5.0 / 6.0)
    pol = np.empty((M, 3))
    for m in range(M):
        while True:
            r = g.standard_normal(3)
            a = np.cross(r, k[m].astype(np.float64))
            na = np.linalg.norm(a)
            if na > 1e-6 * np.linalg.norm(k[m]):
                pol[m] = a / na
                break
    phase = g.uniform(0.0, 2.0 * math.pi, size=M)
    return Modes(k=k, amp=amp, pol=pol, phase=phase)


def field_from_modes(modes: Modes, N: int, L: float = L_BOX, device: str = "cpu",
                     normalise: bool = True):
    """Sample u(x) = S * sum_m amp_m pol_m cos(2 pi k_m . x / L + phase_m) at cell centres.

    Returns a float64 array [3, N, N, N] (numpy on "cpu", torch tensor on a
    CUDA device).  With ``normalise`` the factor S makes the RMS over all
    components and cells equal to 1 (u_rms ~ 1 as in Table 1) and is stored
    in ``modes.scale``.
    """
    if np.abs(modes.k).max() >= N // 2:
        raise ValueError("wavevector aliases on this grid")
    if device == "cpu":
        out = np.empty((3, N, N, N), dtype=np.float64)
        for c in range(3):
            spec = np.zeros((N, N, N), dtype=np.complex128)
            _fill_spectrum(spec, modes, c, N)
            out[c] = np.fft.ifftn(spec).real
        s = 1.0 / math.sqrt(float(np.mean(out * out))) if normalise else modes.scale
        out *= s
        modes.scale = s
        return out
    import torch
    out = torch.empty((3, N, N, N), dtype=torch.float64, device=device)
    for c in range(3):
        spec = np.zeros((N, N, N), dtype=np.complex128) if N <= 128 else None
        if spec is not None:
            _fill_spectrum(spec, modes, c, N)
            t = torch.from_numpy(spec).to(device)
        else:
            t = torch.zeros((N, N, N), dtype=torch.complex128, device=device)
            idx, val = _spectrum_entries(modes, c, N)
            t[idx[:, 2], idx[:, 1], idx[:, 0]] += torch.from_numpy(val).to(device)
        out[c] = torch.fft.ifftn(t).real
        del t
    s = 1.0 / math.sqrt(float(torch.mean(out * out))) if normalise else modes.scale
    out *= s
    modes.scale = s
    return out


def _spectrum_entries(modes: Modes, c: int, N: int):
    """(index, value) pairs of the DFT coefficients of component c (before S)."""
    idx, val = [], []
    for m in range(len(modes.amp)):
        kv = modes.k[m]
        # cell centre n + 1/2 -> extra phase 2 pi k.(1/2,1/2,1/2)/N
        shift = math.pi * float(kv.sum()) / N
        coef = 0.5 * modes.amp[m] * modes.pol[m, c] * N ** 3
        for sgn in (1, -1):
            ph = sgn * (modes.phase[m] + shift)
            idx.append((sgn * kv) % N)
            val.append(coef * complex(math.cos(ph), math.sin(ph)))
    return np.array(idx, dtype=np.int64), np.array(val, dtype=np.complex128)


def _fill_spectrum(spec: np.ndarray, modes: Modes, c: int, N: int) -> None:
    idx, val = _spectrum_entries(modes, c, N)
    np.add.at(spec, (idx[:, 2], idx[:, 1], idx[:, 0]), val)


def direct_sum(modes: Modes, pts: np.ndarray, L: float = L_BOX) -> np.ndarray:
    """Evaluate the mode sum at points (P, 3) directly; returns (P, 3)."""
    ph = (2.0 * math.pi / L) * pts @ modes.k.T.astype(np.float64) + modes.phase[None, :]
    return modes.scale * (np.cos(ph) * modes.amp[None, :]) @ modes.pol


def cell_centres(N: int, L: float = L_BOX) -> np.ndarray:
    return (np.arange(N) + 0.5) * (L / N)


def cfl_dt(field_max_speed: float, N: int, C: float = 0.3, L: float = L_BOX) -> float:
    """Largest {1,2,5} x 10^k not above C * dx / max|U| (convective CFL, Eq. 3)."""
    raw = C * (L / N) / field_max_speed
    e = math.floor(math.log10(raw))
    best = 0.0
    for ee in (e - 1, e):
        for m in (1.0, 2.0, 5.0):
            v = m * 10.0 ** ee
            if v <= raw * (1 + 1e-12):
                best = max(best, v)
    return float(f"{best:.6g}")


def max_speed(field) -> float:
    try:
        import torch
        if isinstance(field, torch.Tensor):
            return float(torch.sqrt((field * field).sum(0)).max())
    except ImportError:
        pass
    return float(np.sqrt((field * field).sum(0)).max())


def positions(n: int, g: np.random.Generator, L: float = L_BOX) -> np.ndarray:
    """(3, n) float64 positions uniform in [0, L)^3."""
    x = g.random((3, n)) * L
    x[x >= L] = 0.0
    return x


def lognormal_tau(n: int, median: float, sigma: float, dt: float,
                  g: np.random.Generator) -> np.ndarray:
    """tau_p with ln tau ~ N(ln median, sigma), redrawn where tau < dt (so dt/tau <= 1)."""
    tau = np.exp(g.normal(math.log(median), sigma, size=n))
    bad = tau < dt
    while bad.any():
        tau[bad] = np.exp(g.normal(math.log(median), sigma, size=int(bad.sum())))
        bad = tau < dt
    return tau


@dataclasses.dataclass
class Workload:
    """One synthetic workload: grid, modes, particles, subdomains, step count."""
    name: str
    number: int
    N: int
    M: int
    kmax: float
    np_: int
    tau_median: float | None   # None -> constant tau_const
    tau_sigma: float
    tau_const: float
    g: tuple
    sub: tuple
    dt: float | None           # None -> CFL
    steps: int
    sort_every: int
    kmin: float = 1.0


WORKLOADS = {
    # 32^3, 64 modes k 1-4, 32768 particles, tau 0.1, dt 0.01, 100 steps, 2x2x2
    "plain_32": Workload("plain_32", 1, 32, 64, 4.0, 32768, None, 0.0, 0.1,
                         (0.0, 0.0, 0.0), (2, 2, 2), 0.01, 100, 0),
    # 256^3, 512 modes k 1-32, 16.8M particles, lognormal tau, gravity, 4x4x4
    "scale_256": Workload("scale_256", 2, 256, 512, 32.0, 16777216, 0.05, 0.5, 0.0,
                          (0.0, 0.0, -9.8), (4, 4, 4), None, 1000, 10),
    # 512^3, 512 modes k 1-64, 1e8 particles, gravity, 8x8x8
    "precision_512": Workload("precision_512", 3, 512, 512, 64.0, 100000000, 0.02, 0.7,
                              0.0, (0.0, 0.0, -9.8), (8, 8, 8), None, 200, 10),
    # 128^3, 512 modes k 1-16, 2^20 particles, tau 0.1, 200 steps
    "grad_128": Workload("grad_128", 4, 128, 512, 16.0, 1048576, None, 0.0, 0.1,
                         (0.0, 0.0, 0.0), (2, 2, 2), None, 200, 0),
}


def make_field(w: Workload, device: str = "cpu", N: int | None = None):
    """Field of workload w (optionally on another grid size N with the same modes)."""
    modes = draw_modes(w.M, w.kmin, w.kmax, rng(w.number, STREAM_FIELD))
    return field_from_modes(modes, N or w.N, device=device), modes


def make_particles(w: Workload, dt: float, n: int | None = None):
    """(x (3,n), v (3,n), tau (n,) or None) for workload w; the first n of the full draw."""
    n_all = w.np_
    n = n_all if n is None else n
    x = positions(n_all if n == n_all else n, rng(w.number, STREAM_POS))
    v = np.zeros_like(x)
    tau = None
    if w.tau_median is not None:
        tau = lognormal_tau(x.shape[1], w.tau_median, w.tau_sigma, dt, rng(w.number, STREAM_TAU))
    return x, v, tau


def small_case(seed: int, N: int, M: int, kmax: float, n: int, tau_median: float | None,
               tau_const: float = 0.1, sigma: float = 0.5, dt: float = 0.01):
    """Generic small seeded case for parity tests: (field, modes, x, v, tau)."""
    modes = draw_modes(M, 1.0, kmax, rng(seed, STREAM_FIELD))
    field = field_from_modes(modes, N)
    x = positions(n, rng(seed, STREAM_POS))
    v = np.zeros_like(x)
    tau = None if tau_median is None else lognormal_tau(n, tau_median, sigma, dt,
                                                         rng(seed, STREAM_TAU))
    return field, modes, x, v, tau


def batch_ensembles(n_ens: int = 48, number: int = 5, device: str = "cpu", scale: float = 1.0):
    """The batching workload: n_ens independent ensembles.

    Grid N uniform in {64, 96, 128, 256}; 256 modes with k in [1, N/8];
    particle count 10^clip(N(5.5, 0.5), 4, 7) (times `scale`); tau_p uniform
    in [0.01, 1]; no gravity; 2x2x2 subdomains; dt from the CFL rule per
    ensemble.  Returns a list of dicts with field, x0, v0, tau, dt, n."""
    g = rng(number, STREAM_ENS)
    sizes = g.choice([64, 96, 128, 256], size=n_ens)
    counts = 10.0 ** np.clip(g.normal(5.5, 0.5, size=n_ens), 4.0, 7.0)
    out = []
    for e in range(n_ens):
        N = int(sizes[e])
        gm = rng(number * 1000 + e, STREAM_FIELD)
        modes = draw_modes(256, 1.0, N / 8.0, gm)
        field = field_from_modes(modes, N, device=device)
        dt = cfl_dt(max_speed(field), N)
        n = max(1, int(counts[e] * scale))
        x = positions(n, rng(number * 1000 + e, STREAM_POS))
        tau = rng(number * 1000 + e, STREAM_TAU).uniform(0.01, 1.0, size=n)
        tau = np.maximum(tau, dt)
        out.append(dict(field=field, x0=x, v0=np.zeros_like(x), tau=tau, dt=dt, n=n, N=N))
    return out
