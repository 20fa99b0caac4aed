"""GB300 particle library: thin Python binding over the C ABI of liblcs.so.

Everything that computes runs in the CUDA kernels behind ``include/lcs.h``;
this module only marshals arguments (torch CUDA tensors for device memory,
torch's current stream for ordering).  There is no CPU fallback: if the
compiled library is missing, importing the binding's entry points raises.

Method: Tominaga & Onishi, "LCS.jl" (arXiv 2604.11008) -- inertial particles
with Stokes drag (Eqs. 5-6, f = 1) and gravity, trilinear interpolation
from cell-centre values and two-stage RK2 (Sec. 2.2), periodic cube
(Sec. 2.1), and prefix-scan particle migration between subdomains
(Sec. 2.3.3), here between virtual subdomains in one GPU's memory.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblcs.so")

LCS_OK, LCS_ERR_ARG, LCS_ERR_CUDA, LCS_ERR_OOM, LCS_ERR_CAPACITY = 0, 1, 2, 3, 4
LCS_ERR_TIMEOUT, LCS_ERR_NONFINITE, LCS_ERR_DISPLACEMENT, LCS_ERR_STATE = 5, 6, 7, 8
LCS_TUNE_CONFIGS = 14  # step-kernel configurations lcs_tune tries
# step-kernel modes
STEP_PLAIN, STEP_STAGED_FIELD, STEP_PREFETCH, STEP_DEFERRED, STEP_OWNED_FIELD = 0, 1, 2, 3, 4
STATUS_NAMES = {0: "LCS_OK", 1: "LCS_ERR_ARG", 2: "LCS_ERR_CUDA", 3: "LCS_ERR_OOM",
                4: "LCS_ERR_CAPACITY", 5: "LCS_ERR_TIMEOUT", 6: "LCS_ERR_NONFINITE",
                7: "LCS_ERR_DISPLACEMENT", 8: "LCS_ERR_STATE"}
DTYPES = {"f64": 0, "f32": 1, "bf16": 2}
KERNELS = {"auto": 0, "fp64": 1, "df": 2}

# Every symbol declared in include/lcs.h.
EXPORTS = ("lcs_init", "lcs_step", "lcs_migrate", "lcs_sort", "lcs_set_state", "lcs_get_state",
           "lcs_get_field", "lcs_backward", "lcs_sync", "lcs_last_error", "lcs_destroy",
           "lcs_launch_count", "lcs_partition", "lcs_profile_steps", "lcs_partition_noalloc",
           "lcs_tune", "lcs_set_step_config", "lcs_staged_tiles", "lcs_set_field",
           "lcs_pair_histogram", "lcs_selftest_waits", "lcs_get_state_by_id",
           "lcs_step_config_of", "lcs_graph_launch_count", "lcs_pair_rdf")
PARTITION_NOALLOC_MAX_N = 1 << 20
DRAGS = {"stokes": 0, "nonlinear": 1}  # lcs_drag: f = 1, or the factor of Eq. (7)
PROF_CLASSES = ("step", "tail", "sort")


class LcsError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        self.status = status
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")


class Desc(C.Structure):
    _fields_ = [("n", C.c_int), ("box", C.c_double), ("sub", C.c_int * 3), ("np", C.c_int64),
                ("field_dtype", C.c_int), ("field_kernel", C.c_int), ("field", C.c_void_p),
                ("x0", C.c_void_p), ("v0", C.c_void_p), ("tau", C.c_void_p),
                ("tau_const", C.c_double), ("ids", C.c_void_p), ("dt", C.c_double),
                ("g", C.c_double * 3), ("sort_every", C.c_int), ("sort_brick", C.c_int),
                ("track_images", C.c_int), ("ckpt_every", C.c_int), ("drag", C.c_int),
                ("nu", C.c_double), ("density_ratio", C.c_double), ("field_next", C.c_void_p),
                ("t_start", C.c_double), ("t_field", C.c_double * 2),
                ("migrate_per_stage", C.c_int), ("owned_field", C.c_int)]


_lib = None


def lib():
    """Load liblcs.so (built by ``paper_2604_11008_gb300.build``); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"liblcs.so not built ({LIB_PATH}); run "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        P, i32, i64 = C.c_void_p, C.c_int, C.c_int64
        L.lcs_init.argtypes = [C.POINTER(Desc), i32, P, C.POINTER(P)]
        L.lcs_step.argtypes = [P, i64]
        L.lcs_migrate.argtypes = [P]
        L.lcs_sort.argtypes = [P]
        L.lcs_set_state.argtypes = [P, i32, P, P, P, P, P, P]
        L.lcs_get_state.argtypes = [P, i32, P, P, P, P, P, P]
        L.lcs_get_state_by_id.argtypes = [P, i32, P, P, P]
        L.lcs_step_config_of.argtypes = [P, i32, P, P, P]
        L.lcs_get_field.argtypes = [P, i32, P]
        L.lcs_backward.argtypes = [P, P, P, P, P, P]
        L.lcs_sync.argtypes = [P]
        L.lcs_last_error.argtypes = [P]
        L.lcs_last_error.restype = C.c_char_p
        L.lcs_destroy.argtypes = [P]
        L.lcs_destroy.restype = None
        L.lcs_launch_count.argtypes = [P]
        L.lcs_launch_count.restype = i64
        L.lcs_graph_launch_count.argtypes = [P]
        L.lcs_graph_launch_count.restype = i64
        L.lcs_partition.argtypes = [P, i64, i32, P, P, P, P]
        L.lcs_profile_steps.argtypes = [P, i64, P, P]
        L.lcs_partition_noalloc.argtypes = [P, i64, i32, P, P, P, P]
        L.lcs_tune.argtypes = [P, i32, P, P, P, P]
        L.lcs_set_step_config.argtypes = [P, i32, i32, i32]
        L.lcs_staged_tiles.argtypes = [P, P]
        L.lcs_set_field.argtypes = [P, i32, P, C.c_double]
        L.lcs_pair_histogram.argtypes = [P, i32, C.c_double, i32, P]
        L.lcs_pair_rdf.argtypes = [P, i32, C.c_double, i32, P, P, P]
        L.lcs_selftest_waits.argtypes = [P, P, P]
        for name in ("lcs_init", "lcs_step", "lcs_migrate", "lcs_sort", "lcs_set_state",
                     "lcs_get_state", "lcs_get_field", "lcs_backward", "lcs_sync",
                     "lcs_partition", "lcs_profile_steps", "lcs_partition_noalloc", "lcs_tune",
                     "lcs_set_step_config", "lcs_staged_tiles", "lcs_set_field",
                     "lcs_pair_histogram", "lcs_selftest_waits", "lcs_get_state_by_id",
                     "lcs_step_config_of", "lcs_pair_rdf"):
            getattr(L, name).restype = i32
        _lib = L
    return _lib


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(C.c_void_p)
    return C.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dev(t, dtype):
    import torch
    if not isinstance(t, torch.Tensor):
        t = torch.as_tensor(np.asarray(t))
    return t.to(device="cuda", dtype=dtype).contiguous()


def _dev_or_host(t, dtype):
    """A contiguous tensor of `dtype` where `t` already is: CUDA tensors stay
    on the device, host arrays stay on the host (the library copies them
    itself, at full speed from pinned memory)."""
    import torch
    if not isinstance(t, torch.Tensor):
        t = torch.as_tensor(np.asarray(t))
    return t.to(dtype=dtype).contiguous()


class Simulator:
    """Particles of one or more ensembles advancing in frozen periodic fields.

    Parameters mirror ``lcs_desc`` of include/lcs.h.  Arrays may be numpy or
    torch; they are copied to the current CUDA device.
    """

    def __init__(self, field, x0, v0, dt, tau=None, tau_const=0.0, g=(0.0, 0.0, 0.0),
                 sub=(1, 1, 1), box=2 * math.pi, field_dtype="f64", kernel="auto", ids=None,
                 sort_every=0, sort_brick=0, track_images=False, ckpt_every=0, stream=None,
                 ensembles=None, drag="stokes", nu=0.0, density_ratio=0.0, field_next=None,
                 t_start=0.0, t_field=(0.0, 1.0), migrate_per_stage=False, owned_field=False):
        import torch
        self._keep = []
        self._stream = stream
        specs = ensembles if ensembles is not None else [dict(
            field=field, x0=x0, v0=v0, dt=dt, tau=tau, tau_const=tau_const, g=g, sub=sub,
            box=box, field_dtype=field_dtype, kernel=kernel, ids=ids, sort_every=sort_every,
            sort_brick=sort_brick, track_images=track_images, ckpt_every=ckpt_every,
            drag=drag, nu=nu, density_ratio=density_ratio, field_next=field_next,
            t_start=t_start, t_field=t_field, migrate_per_stage=migrate_per_stage,
            owned_field=owned_field)]
        descs = (Desc * len(specs))()
        self.meta = []
        for k, sp in enumerate(specs):
            f = _dev(sp["field"], torch.float64)
            x = _dev(sp["x0"], torch.float64)
            v = _dev(sp["v0"], torch.float64)
            t = None if sp.get("tau") is None else _dev(sp["tau"], torch.float64)
            i = None if sp.get("ids") is None else _dev(sp["ids"], torch.int32)
            fn = None if sp.get("field_next") is None else _dev(sp["field_next"], torch.float64)
            self._keep += [f, x, v, t, i, fn]
            d = descs[k]
            d.n = int(f.shape[-1])
            d.box = float(sp.get("box", 2 * math.pi))
            d.sub[:] = [int(s) for s in sp.get("sub", (1, 1, 1))]
            d.np = int(x.shape[1])
            d.field_dtype = DTYPES[sp.get("field_dtype", "f64")]
            d.field_kernel = KERNELS[sp.get("kernel", "auto")]
            d.field, d.x0, d.v0 = f.data_ptr(), x.data_ptr(), v.data_ptr()
            d.tau = t.data_ptr() if t is not None else None
            d.tau_const = float(sp.get("tau_const", 0.0))
            d.ids = i.data_ptr() if i is not None else None
            d.dt = float(sp["dt"])
            d.g[:] = [float(a) for a in sp.get("g", (0.0, 0.0, 0.0))]
            d.sort_every = int(sp.get("sort_every", 0))
            d.sort_brick = int(sp.get("sort_brick", 0))
            d.track_images = int(bool(sp.get("track_images", False)))
            d.ckpt_every = int(sp.get("ckpt_every", 0))
            d.drag = DRAGS[sp.get("drag", "stokes")]
            d.nu = float(sp.get("nu", 0.0))
            d.density_ratio = float(sp.get("density_ratio", 0.0))
            d.field_next = fn.data_ptr() if fn is not None else None
            d.t_start = float(sp.get("t_start", 0.0))
            d.t_field[:] = [float(a) for a in sp.get("t_field", (0.0, 1.0))]
            d.migrate_per_stage = int(bool(sp.get("migrate_per_stage", False)))
            d.owned_field = int(bool(sp.get("owned_field", False)))
            self.meta.append(dict(n=d.n, np=d.np, P=int(np.prod(d.sub[:])), has_tau=t is not None,
                                  tau_const=d.tau_const, box=d.box))
        self._ctx = C.c_void_p()
        st = lib().lcs_init(descs, len(specs), _stream(stream), C.byref(self._ctx))
        self._keep = []  # inputs are read during lcs_init only
        if st != LCS_OK:
            raise LcsError(st, "lcs_init: " + lib().lcs_last_error(None).decode())

    # -- helpers
    def _check(self, st):
        if st != LCS_OK:
            msg = lib().lcs_last_error(self._ctx).decode()
            raise LcsError(st, msg)

    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            lib().lcs_destroy(self._ctx)
            self._ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- calls
    def step(self, nsteps: int = 1):
        self._check(lib().lcs_step(self._ctx, int(nsteps)))

    def migrate(self):
        self._check(lib().lcs_migrate(self._ctx))

    def sort(self):
        self._check(lib().lcs_sort(self._ctx))

    def sync(self):
        self._check(lib().lcs_sync(self._ctx))

    def profile_steps(self, nsteps: int):
        """Run nsteps un-graphed steps timing every kernel class with CUDA events.

        Returns {class: (total_ms, launches)} for the classes in PROF_CLASSES."""
        ms = np.zeros(len(PROF_CLASSES), dtype=np.float64)
        cnt = np.zeros(len(PROF_CLASSES), dtype=np.int64)
        self._check(lib().lcs_profile_steps(self._ctx, int(nsteps), _ptr(ms), _ptr(cnt)))
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(PROF_CLASSES)}

    def tune(self, steps_per_trial: int = 2):
        """Autotune the step kernel (scan tile and kernel mode); advances the
        simulation by steps_per_trial steps per tried configuration.  Returns
        (threads per block, items per thread, mode); the step-kernel
        milliseconds of every configuration are kept in tune_trials_ms (-1
        where skipped)."""
        b, it, md = C.c_int(), C.c_int(), C.c_int()
        ms = np.zeros(LCS_TUNE_CONFIGS, dtype=np.float64)
        self._check(lib().lcs_tune(self._ctx, int(steps_per_trial), C.byref(b), C.byref(it),
                                   C.byref(md), _ptr(ms)))
        self.tune_trials_ms = ms
        return b.value, it.value, md.value

    def set_field(self, field, t: float, ens: int = 0):
        """Evolving field: push the snapshot at time t (the current second
        snapshot becomes the first)."""
        import torch
        f = _dev(field, torch.float64)
        self._check(lib().lcs_set_field(self._ctx, int(ens), f.data_ptr(), float(t)))

    def pair_histogram(self, r_max: float, nbins: int, ens: int = 0) -> np.ndarray:
        """Counts of particle pairs by separation (r < r_max <= L/N, nbins bins)."""
        counts = np.zeros(int(nbins), dtype=np.int64)
        self._check(lib().lcs_pair_histogram(self._ctx, int(ens), float(r_max), int(nbins),
                                             _ptr(counts)))
        return counts

    def rdf(self, r_max: float, nbins: int, ens: int = 0):
        """Radial distribution function (lcs_pair_rdf): (bin centres, g, counts),
        g = counts / (np (np - 1) / 2 * shell volume / L^3)."""
        r = np.zeros(int(nbins), dtype=np.float64)
        g = np.zeros(int(nbins), dtype=np.float64)
        counts = np.zeros(int(nbins), dtype=np.int64)
        self._check(lib().lcs_pair_rdf(self._ctx, int(ens), float(r_max), int(nbins), _ptr(r),
                                       _ptr(g), _ptr(counts)))
        return r, g, counts

    def step_config_of(self, ens: int = 0):
        """(threads per block, particles per thread, mode) of ensemble `ens`."""
        b, it, md = C.c_int(), C.c_int(), C.c_int()
        self._check(lib().lcs_step_config_of(self._ctx, int(ens), C.byref(b), C.byref(it),
                                             C.byref(md)))
        return b.value, it.value, md.value

    def set_step_config(self, block: int, items: int, mode: int = STEP_PLAIN):
        """Pin one of the step-kernel configurations lcs_tune chooses among."""
        self._check(lib().lcs_set_step_config(self._ctx, int(block), int(items), int(mode)))

    @property
    def staged_tiles(self) -> int:
        """Step tiles so far whose field cells came from a shared-memory box."""
        n = C.c_int64()
        self._check(lib().lcs_staged_tiles(self._ctx, C.byref(n)))
        return n.value

    @property
    def launches(self) -> int:
        return int(lib().lcs_launch_count(self._ctx))

    @property
    def graph_launches(self) -> int:
        """CUDA graph launches issued by step() so far (one per recorded run of steps)."""
        return int(lib().lcs_graph_launch_count(self._ctx))

    def get_state(self, ens: int = 0, device: str = "cuda", out=None):
        """Current particles in storage order: dict of x, v (3, np), tau, ids, img, seg."""
        import torch
        m = self.meta[ens]
        n, P = m["np"], m["P"]
        if out is None:
            kw = dict(device=device)
            if device == "cpu":
                kw["pin_memory"] = torch.cuda.is_available()
            out = dict(x=torch.empty((3, n), dtype=torch.float64, **kw),
                       v=torch.empty((3, n), dtype=torch.float64, **kw),
                       tau=torch.empty(n, dtype=torch.float64, **kw),
                       ids=torch.empty(n, dtype=torch.int32, **kw),
                       img=torch.empty((3, n), dtype=torch.int32, **kw))
        seg = np.empty(P + 1, dtype=np.int64)
        self._check(lib().lcs_get_state(self._ctx, ens, _ptr(out["x"]), _ptr(out["v"]),
                                        _ptr(out.get("tau")), _ptr(out.get("ids")),
                                        _ptr(out.get("img")), _ptr(seg)))
        out["seg"] = seg
        return out

    def set_state(self, x, v, ids, seg, tau=None, img=None, ens: int = 0):
        import torch
        # host or device buffers, copied by lcs_set_state (synchronising)
        xs = _dev_or_host(x, torch.float64)
        vs = _dev_or_host(v, torch.float64)
        ii = _dev_or_host(ids, torch.int32)
        tt = None if tau is None else _dev_or_host(tau, torch.float64)
        im = None if img is None else _dev_or_host(img, torch.int32)
        seg = np.ascontiguousarray(seg, dtype=np.int64)
        self._check(lib().lcs_set_state(self._ctx, ens, _ptr(xs), _ptr(vs), _ptr(tt), _ptr(ii),
                                        _ptr(im), _ptr(seg)))

    def final_state_by_id(self, ens: int = 0, device: str = "cuda", ids: bool = False):
        """(X, V) as (3, np) tensors in particle-id order (lcs_get_state_by_id):
        X unwrapped across the periodic boundary when images are tracked.
        With ids=True also the sorted ids."""
        import torch
        n = self.meta[ens]["np"]
        kw = dict(device=device)
        if device == "cpu":
            kw["pin_memory"] = torch.cuda.is_available()
        x = torch.empty((3, n), dtype=torch.float64, **kw)
        v = torch.empty((3, n), dtype=torch.float64, **kw)
        i = torch.empty(n, dtype=torch.int32, **kw) if ids else None
        self._check(lib().lcs_get_state_by_id(self._ctx, ens, _ptr(x), _ptr(v), _ptr(i)))
        return (x, v, i) if ids else (x, v)

    def backward(self, gx, gv, gU=None):
        """Adjoint of the recorded steps (lcs_backward).

        gx, gv: dLoss/dX_T (unwrapped) and dLoss/dV_T, (3, np) in particle-id
        order.  Returns (dLoss/dU [3,N,N,N], dLoss/dX0, dLoss/dV0) as CUDA
        tensors; dLoss/dU is accumulated into gU when given."""
        import torch
        m = self.meta[0]
        n, N = m["np"], m["n"]
        gxd = _dev(gx, torch.float64)
        gvd = _dev(gv, torch.float64)
        if gU is None:
            gU = torch.zeros((3, N, N, N), dtype=torch.float64, device="cuda")
        gx0 = torch.empty((3, n), dtype=torch.float64, device="cuda")
        gv0 = torch.empty((3, n), dtype=torch.float64, device="cuda")
        self._check(lib().lcs_backward(self._ctx, _ptr(gxd), _ptr(gvd), _ptr(gU), _ptr(gx0),
                                       _ptr(gv0)))
        return gU, gx0, gv0

    def get_field(self, ens: int = 0):
        import torch
        n = self.meta[ens]["n"]
        out = torch.empty((3, n, n, n), dtype=torch.float64, device="cuda")
        self._check(lib().lcs_get_field(self._ctx, ens, _ptr(out)))
        return out


def partition(keys, nbins: int, stream=None):
    """Stable partition of uint32 keys into nbins bins (counting sort).

    Returns (perm, bin_off, status) as CUDA tensors; perm[r] = index of the
    key at rank r, bin_off the bin starts, status an int32 LCS_* code."""
    import torch
    k = _dev(keys, torch.int32)
    n = int(k.numel())
    perm = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    off = torch.empty(nbins + 1, dtype=torch.int64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = lib().lcs_partition(_ptr(k), n, int(nbins), _ptr(perm), _ptr(off), _ptr(status),
                             _stream(stream))
    if st != LCS_OK:
        raise LcsError(st, "lcs_partition failed")
    return perm[:n], off, status


def selftest_waits(stream=None):
    """Run the bounded-wait self-test (lcs_selftest_waits): the look-back and
    mbarrier waits of the step kernels against partners that never answer.
    Returns (lookback, mbarrier) statuses; LCS_ERR_TIMEOUT each when the
    wait gave up as designed."""
    a, b = C.c_int32(-1), C.c_int32(-1)
    st = lib().lcs_selftest_waits(_stream(stream), C.byref(a), C.byref(b))
    if st != LCS_OK:
        raise LcsError(st, "lcs_selftest_waits failed")
    return a.value, b.value


def _autograd_function():
    import torch

    class ParticleAdvect(torch.autograd.Function):
        """(U, X0, V0) -> (X_T unwrapped, V_T) after `steps` steps, differentiable.

        U: [3,N,N,N] FP64 field; X0, V0: (3, np) in particle-id order.  X0 may
        lie outside [0, L): the library folds it into the box and counts the
        folds as periodic images, so X_T comes back unwrapped relative to X0.
        The backward pass is the library's hand-written adjoint (lcs_backward)
        with checkpoints every `ckpt_every` steps."""

        @staticmethod
        def forward(ctx, U, X0, V0, opts):
            kw = {k: v for k, v in opts.items() if k not in ("steps",)}
            kw.setdefault("ckpt_every", 20)
            kw["track_images"] = True
            sim = Simulator(U.detach(), X0.detach(), V0.detach(), **kw)
            sim.step(int(opts["steps"]))
            xt, vt = sim.final_state_by_id()
            ctx.sim = sim
            return xt, vt

        @staticmethod
        def backward(ctx, gX, gV):
            sim = ctx.sim
            n = sim.meta[0]["np"]
            zeros = torch.zeros((3, n), dtype=torch.float64, device="cuda")
            gX = zeros if gX is None else gX
            gV = zeros if gV is None else gV
            gU, gx0, gv0 = sim.backward(gX.contiguous(), gV.contiguous())
            sim.close()
            ctx.sim = None
            return gU, gx0, gv0, None

    return ParticleAdvect


def particle_advect(U, X0, V0, **opts):
    """Differentiable advection: returns (X_T, V_T); see ParticleAdvect."""
    return _autograd_function().apply(U, X0, V0, opts)
