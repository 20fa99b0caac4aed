"""CPU oracle for the particle hot path -- TEST INFRASTRUCTURE ONLY.

A plain, slow, single-threaded FP64 restatement of the paper's particle
method (see ``lcs_oracle.c`` for the citations).  Only the tests, the smoke
check and the benchmark's CPU-baseline leg may import this package; the
library under ``paper_2604_11008_gb300`` never does, and this package never
imports the library.

The C source is compiled on first use with gcc (``-O2 -ffp-contract=off`` so
that x86 and Arm produce identical results) into ``oracle/_build``.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lcs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liblcs_oracle.so")
_SO_OMP = os.path.join(_BUILD, "liblcs_oracle_omp.so")
_lock = threading.Lock()
_lib = None
_omp = False  # load the OpenMP build (timed CPU baseline on all cores)

ORC_OK, ORC_ERR_DISPLACEMENT, ORC_ERR_ARG, ORC_ERR_NOMEM = 0, 1, 2, 3


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle shared library (idempotent); returns its path.
    openmp: the same source built with -fopenmp (the particle loop of
    orc_advance on all cores; identical arithmetic per particle)."""
    os.makedirs(_BUILD, exist_ok=True)
    so = _SO_OMP if openmp else _SO
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(_SRC):
        tmp = so + f".{os.getpid()}.tmp"
        extra = ["-fopenmp"] if openmp else []
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
                               *extra, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, so)
    return so


def use_threads(n: int | None):
    """Select the build the following calls use: n = None the plain
    single-threaded oracle, else the OpenMP build with n threads (0: all
    cores).  Returns the threads the particle loop uses, or None when the
    OpenMP build is not available on this machine."""
    global _lib, _omp
    with _lock:
        want = n is not None
        if want:
            try:
                build(openmp=True)
            except (OSError, subprocess.CalledProcessError):
                return None
        if want != _omp:
            _lib, _omp = None, want
    lib = _load()
    lib.orc_threads.argtypes = [C.c_int]
    lib.orc_threads.restype = C.c_int
    return int(lib.orc_threads(int(n or 0))) if want else 1


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build(openmp=_omp))
            P = C.c_void_p
            i64, i32, dbl = C.c_int64, C.c_int, C.c_double
            lib.orc_interp_many.argtypes = [P, i32, dbl, i64, P, P, P, P, P, P]
            lib.orc_advance.argtypes = [P, i32, dbl, dbl, i64, P, P, P, P, P, P, P, dbl, dbl, P,
                                        i32, P, P, i32, dbl, dbl, P, dbl, dbl, dbl]
            lib.orc_advance.restype = i32
            lib.orc_keys.argtypes = [i32, dbl, P, i32, i64, P, P, P, P, P]
            lib.orc_keys.restype = i32
            lib.orc_migrate.argtypes = [i32, i64, P, P, P, P, P]
            lib.orc_migrate.restype = i32
            lib.orc_sort.argtypes = [i32, P, P, P]
            lib.orc_sort.restype = i32
            lib.orc_loss.argtypes = [dbl, i64, P, P, P, P, P, P, P, P]
            lib.orc_loss.restype = dbl
            lib.orc_adjoint.argtypes = [P, i32, dbl, dbl, i64, P, P, P, P, P, P, P, dbl, dbl, P,
                                        i32, P, P, P]
            lib.orc_adjoint.restype = i32
            lib.orc_interp_transpose_many.argtypes = [P, i32, dbl, i64, P, P, P, P, P, P]
            lib.orc_round_f32.argtypes = [i64, P, P]
            lib.orc_round_bf16.argtypes = [i64, P, P]
            lib.orc_pair_hist.argtypes = [i64, P, P, P, dbl, dbl, i32, P]
            lib.orc_stage1.argtypes = [P, i32, dbl, dbl, i64, P, P, P, dbl, dbl, P, i32, dbl,
                                       dbl, P, dbl, dbl, dbl, P, P, P]
            lib.orc_stage1.restype = i32
            lib.orc_stage2.argtypes = [P, i32, dbl, dbl, i64, P, P, P, P, P, P, dbl, dbl, P,
                                       i32, dbl, dbl, P, dbl, dbl, dbl, P]
            lib.orc_stage2.restype = i32
            lib.orc_pair_hist.restype = None
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def inv_dx(N: int, L: float) -> float:
    """N / L as one correctly rounded FP64 division (the same value is passed to the GPU)."""
    return float(N) / float(L)


def interp(field: np.ndarray, L: float, x: np.ndarray) -> np.ndarray:
    """Trilinear interpolation of field [3,N,N,N] at positions x (3, n) -> (3, n)."""
    lib = _load()
    field = _c(field, np.float64)
    N = field.shape[-1]
    x = _c(x, np.float64)
    n = x.shape[1]
    out = np.empty((3, n))
    lib.orc_interp_many(_p(field), N, inv_dx(N, L), n, _p(x[0]), _p(x[1]), _p(x[2]),
                        _p(out[0]), _p(out[1]), _p(out[2]))
    return out


def interp_transpose(field, L, x, mu):
    """(interp^T(x) mu as a field [3,N,N,N], J(x)^T mu (3, n)) at positions x (3, n)."""
    lib = _load()
    field = _c(field, np.float64)
    N = field.shape[-1]
    x = _c(x, np.float64)
    mu = _c(mu, np.float64)
    n = x.shape[1]
    gf = np.zeros_like(field)
    jt = np.empty((3, n))
    lib.orc_interp_transpose_many(_p(field), N, inv_dx(N, L), n, _p(x[0]), _p(x[1]), _p(x[2]),
                                  _p(mu), _p(gf), _p(jt))
    return gf, jt


# Drag law: (0,) Stokes (f = 1); (1, nu, density_ratio) the factor of Eq. (7).
STOKES = (0, 0.0, 0.0)


def advance(field, L, x, v, tau, tau_const, dt, g, nsteps, img=None, cellhash=None,
            drag=STOKES, field_b=None, times=(0.0, 0.0, 1.0)):
    """Heun steps of Eqs. (5)-(6) with wrap, in place on x, v (3, n) float64 C arrays.
    With field_b, the field is linear in time between `field` at t_a and
    field_b at t_b; times = (t_start, t_a, t_b)."""
    lib = _load()
    field = _c(field, np.float64)
    N = field.shape[-1]
    assert x.flags.c_contiguous and v.flags.c_contiguous and x.dtype == np.float64
    n = x.shape[1]
    tau = None if tau is None else _c(tau, np.float64)
    gg = _c(g, np.float64)
    fb = None if field_b is None else _c(field_b, np.float64)
    return lib.orc_advance(_p(field), N, float(L), inv_dx(N, L), n, _p(x[0]), _p(x[1]),
                           _p(x[2]), _p(v[0]), _p(v[1]), _p(v[2]), _p(tau), float(tau_const),
                           float(dt), _p(gg), int(nsteps), _p(img), _p(cellhash),
                           int(drag[0]), float(drag[1]) if drag[0] else 0.0,
                           float(drag[2]) if drag[0] else 0.0, _p(fb), float(times[0]),
                           float(times[1]), float(times[2]))


def keys(N, L, P, brick, x):
    """(dest int32 (n,), key int64 (n,)) for positions x (3, n)."""
    lib = _load()
    x = _c(x, np.float64)
    n = x.shape[1]
    dest = np.empty(n, np.int32)
    key = np.empty(n, np.int64)
    PP = np.array(P, dtype=np.int32)
    st = lib.orc_keys(int(N), inv_dx(N, L), _p(PP), int(brick), n, _p(x[0]), _p(x[1]),
                      _p(x[2]), _p(dest), _p(key))
    if st != ORC_OK:
        raise ValueError(f"orc_keys failed ({st})")
    return dest, key


def migrate(P: int, seg, dest):
    """Sequential-counter migration: (perm new->old, seg_out (P+1,), slot (n,))."""
    lib = _load()
    seg = _c(seg, np.int64)
    dest = _c(dest, np.int32)
    n = dest.shape[0]
    perm = np.empty(n, np.int64)
    seg_out = np.empty(P + 1, np.int64)
    slot = np.empty(n, np.int64)
    st = lib.orc_migrate(int(P), n, _p(seg), _p(dest), _p(perm), _p(seg_out), _p(slot))
    if st != ORC_OK:
        raise ValueError(f"orc_migrate failed ({st})")
    return perm, seg_out, slot


def sort(P: int, seg, key):
    """Stable per-segment sort by key: perm new->old."""
    lib = _load()
    seg = _c(seg, np.int64)
    key = _c(key, np.int64)
    perm = np.empty(key.shape[0], np.int64)
    st = lib.orc_sort(int(P), _p(seg), _p(key), _p(perm))
    if st != ORC_OK:
        raise MemoryError("orc_sort")
    return perm


def pair_hist(x, L, r_max, nbins):
    """Counts (nbins,) of pair separations r < r_max (minimum image), all pairs."""
    lib = _load()
    x = _c(x, np.float64)
    counts = np.zeros(nbins, np.int64)
    lib.orc_pair_hist(x.shape[1], _p(x[0]), _p(x[1]), _p(x[2]), float(L), float(r_max),
                      int(nbins), _p(counts))
    return counts


def loss(L, x, img, target, mask=None):
    lib = _load()
    x = _c(x, np.float64)
    target = _c(target, np.float64)
    n = x.shape[1]
    img = None if img is None else _c(img, np.int32)
    mask = None if mask is None else _c(mask, np.float64)
    return lib.orc_loss(float(L), n, _p(x[0]), _p(x[1]), _p(x[2]), _p(img), _p(target[0]),
                        _p(target[1]), _p(target[2]), _p(mask))


def adjoint(field, L, x0, v0, tau, tau_const, dt, g, nsteps, lx, lv, want_field=True):
    """Reverse-mode derivative: returns (dL/dx0, dL/dv0, dL/dU or None) from final adjoints."""
    lib = _load()
    field = _c(field, np.float64)
    N = field.shape[-1]
    x0 = _c(x0, np.float64)
    v0 = _c(v0, np.float64)
    n = x0.shape[1]
    lx = np.array(lx, dtype=np.float64, order="C")
    lv = np.array(lv, dtype=np.float64, order="C")
    gf = np.zeros_like(field) if want_field else None
    tau = None if tau is None else _c(tau, np.float64)
    gg = _c(g, np.float64)
    st = lib.orc_adjoint(_p(field), N, float(L), inv_dx(N, L), n, _p(x0[0]), _p(x0[1]),
                         _p(x0[2]), _p(v0[0]), _p(v0[1]), _p(v0[2]), _p(tau), float(tau_const),
                         float(dt), _p(gg), int(nsteps), _p(lx), _p(lv), _p(gf))
    if st == ORC_ERR_NOMEM:
        raise MemoryError("orc_adjoint")
    return lx, lv, gf


def round_f32(a):
    lib = _load()
    a = _c(a, np.float64)
    out = np.empty_like(a)
    lib.orc_round_f32(a.size, _p(a), _p(out))
    return out


def round_bf16(a):
    lib = _load()
    a = _c(a, np.float64)
    out = np.empty_like(a)
    lib.orc_round_bf16(a.size, _p(a), _p(out))
    return out


class State:
    """Particle records in storage order plus the subdomain segments."""

    def __init__(self, x, v, tau, ids, seg, img=None):
        self.x, self.v, self.tau, self.ids, self.seg = x, v, tau, ids, seg
        self.img = img

    def permute(self, perm):
        self.x = np.ascontiguousarray(self.x[:, perm])
        self.v = np.ascontiguousarray(self.v[:, perm])
        if self.tau is not None:
            self.tau = np.ascontiguousarray(self.tau[perm])
        self.ids = np.ascontiguousarray(self.ids[perm])
        if self.img is not None:
            self.img = np.ascontiguousarray(self.img[:, perm])

    def copy(self):
        return State(self.x.copy(), self.v.copy(), None if self.tau is None else self.tau.copy(),
                     self.ids.copy(), self.seg.copy(),
                     None if self.img is None else self.img.copy())


def initial_state(N, L, P, x, v, tau, ids=None, track_img=False):
    """Particles in ID order, then one migration from a single source segment.

    Treating the whole array as one source gives every subdomain its particles
    in ID order (the stable initial placement)."""
    Ptot = int(np.prod(P))
    n = x.shape[1]
    ids = np.arange(n, dtype=np.uint32) if ids is None else np.asarray(ids, np.uint32)
    st = State(_c(x, np.float64).copy(), _c(v, np.float64).copy(),
               None if tau is None else _c(tau, np.float64).copy(), ids.copy(),
               np.array([0] + [n] * Ptot, np.int64),
               np.zeros((3, n), np.int32) if track_img else None)
    dest, _ = keys(N, L, P, 1, st.x)
    perm = np.argsort(dest, kind="stable")
    st.permute(perm)
    st.seg = np.concatenate([[0], np.cumsum(np.bincount(dest, minlength=Ptot))]).astype(np.int64)
    return st


def _wrapped(x, L):
    """Positions folded into [0, L) as the wrap of Sec. 2.1 does (x == L -> 0)."""
    w = np.where(x >= L, x - L, np.where(x < 0.0, x + L, x))
    return np.where(w == L, 0.0, w)


def step_per_stage(st: State, field, L, P, tau_const, dt, g, brick, do_sort: bool,
                   drag=STOKES, field_b=None, times=(0.0, 0.0, 1.0)):
    """One step with migration after each Runge-Kutta stage (Sec. 3.2.2): stage 1
    gives X*, V*, A1; the particles move to the subdomain of X* (folded into the
    box); stage 2 completes X', V' (wrapped); they move to the subdomain of X';
    then the optional cell sort.  The stage values travel with the particles."""
    lib = _load()
    field = _c(field, np.float64)
    N = field.shape[-1]
    n = st.x.shape[1]
    fb = None if field_b is None else _c(field_b, np.float64)
    tau = None if st.tau is None else _c(st.tau, np.float64)
    gg = _c(g, np.float64)
    dr = (int(drag[0]), float(drag[1]) if drag[0] else 0.0, float(drag[2]) if drag[0] else 0.0)
    xs, vs, a1 = np.empty((3, n)), np.empty((3, n)), np.empty((3, n))
    status = lib.orc_stage1(_p(field), N, float(L), inv_dx(N, L), n, _p(st.x), _p(st.v),
                            _p(tau), float(tau_const), float(dt), _p(gg), *dr, _p(fb),
                            float(times[0]), float(times[1]), float(times[2]), _p(xs), _p(vs),
                            _p(a1))
    dest, _ = keys(N, L, P, brick, _wrapped(xs, L))
    perm, seg_out, _ = migrate(int(np.prod(P)), st.seg, dest)
    st.permute(perm)
    st.seg = seg_out
    xs, vs, a1 = (np.ascontiguousarray(a[:, perm]) for a in (xs, vs, a1))
    tau = None if st.tau is None else _c(st.tau, np.float64)
    s2 = lib.orc_stage2(_p(field), N, float(L), inv_dx(N, L), n, _p(st.x), _p(st.v), _p(xs),
                        _p(vs), _p(a1), _p(tau), float(tau_const), float(dt), _p(gg), *dr,
                        _p(fb), float(times[0]), float(times[1]), float(times[2]),
                        _p(st.img))
    status = status or s2
    dest, key = keys(N, L, P, brick, st.x)
    perm, seg_out, _ = migrate(int(np.prod(P)), st.seg, dest)
    st.permute(perm)
    st.seg = seg_out
    if do_sort:
        _, key = keys(N, L, P, brick, st.x)
        perm = sort(int(np.prod(P)), st.seg, key)
        st.permute(perm)
    return status


def step(st: State, field, L, P, tau_const, dt, g, brick, do_sort: bool, drag=STOKES,
         field_b=None, times=(0.0, 0.0, 1.0)):
    """One step of the path: advance + wrap, migrate, and (if do_sort) the cell sort."""
    N = field.shape[-1]
    status = advance(field, L, st.x, st.v, st.tau, tau_const, dt, g, 1, img=st.img, drag=drag,
                     field_b=field_b, times=times)
    dest, key = keys(N, L, P, brick, st.x)
    perm, seg_out, _ = migrate(int(np.prod(P)), st.seg, dest)
    st.permute(perm)
    st.seg = seg_out
    if do_sort:
        _, key = keys(N, L, P, brick, st.x)
        perm = sort(int(np.prod(P)), st.seg, key)
        st.permute(perm)
    return status


def run(st: State, field, L, P, tau_const, dt, g, nsteps, sort_every=0, brick=8, step0=0,
        drag=STOKES, field_b=None, t_start=0.0, t_field=(0.0, 1.0), per_stage=False):
    """nsteps steps; the sort runs after steps whose 1-based index is a multiple of sort_every.
    With field_b the field is linear in time between `field` at t_field[0] and
    field_b at t_field[1]; step k (counted from step0) starts at t_start + k dt."""
    status = ORC_OK
    one = step_per_stage if per_stage else step
    for k in range(step0, step0 + nsteps):
        s = one(st, field, L, P, tau_const, dt, g, brick,
                sort_every > 0 and (k + 1) % sort_every == 0, drag=drag, field_b=field_b,
                times=(t_start + k * dt, t_field[0], t_field[1]))
        status = status or s
    return status
