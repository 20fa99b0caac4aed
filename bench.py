"""Benchmark of the particle hot path: particle-updates/s including migration.

Workload (default ``scale_256``): 256^3 FP64 field of 512 random Fourier
modes (k 1-32, k^-5/3 spectrum), 16,777,216 particles uniform in the box,
tau_p log-normal (median 0.05, sigma 0.5), gravity (0, 0, -9.8), 4x4x4
virtual subdomains with migration every step and a cell sort every 10
steps, dt from the convective CFL rule.  One bench step = 10 time steps
(one sort period), so every timed step contains all passes of the path.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun, one process per GPU): every rank runs its own replica
of the workload (the virtual subdomains of one replica live in one GPU's
memory; no collective is on the data path); ``value`` sums all ranks' updates
over the slowest rank's time.  ``--impl reference`` times the CPU oracle on
this machine's host cores on a bounded sample of the same workload.
Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "particle-updates/s incl. prefix-scan migration; % HBM peak; adjoint/fwd ratio"
UNIT = "particle-updates/s"
STEPS_PER_BENCH_STEP = 10


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured", d
    return 6800.0, "fallback", {}


# ---------------------------------------------------------------- workload

def build_workload(name: str, device: str, n_override: int | None = None):
    w = synth.WORKLOADS[name]
    field, modes = synth.make_field(w, device=device)
    dt = w.dt if w.dt is not None else synth.cfl_dt(synth.max_speed(field), w.N)
    n = n_override or w.np_
    x, v, tau = synth.make_particles(w, dt, n=n)
    return w, field, modes, dt, x, v, tau


# ---------------------------------------------------------------- traffic

def library_source_hash() -> str:
    """SHA-256 over the code of the sources that define the step kernel (its
    templates, the physics and arithmetic headers, the per-storage
    instantiations), comments and whitespace removed."""
    import glob
    import hashlib
    root = os.path.dirname(os.path.abspath(__file__))
    csrc = os.path.join(root, "paper_2604_11008_gb300", "csrc")
    files = sorted(glob.glob(os.path.join(csrc, "lcs_step_*.cu")) +
                   glob.glob(os.path.join(csrc, "*.cuh")))
    import re
    h = hashlib.sha256()
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, encoding="utf-8") as fh:
            src = fh.read()
        # code only: comments and layout do not change the kernels
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()


def measured_counters(workload: str, field: str, kernel: str, n: int, cfg):
    """Counters of one step-kernel launch from the committed ncu captures
    (profiles/step_counters.json): DRAM bytes per launch, warp instructions
    and FP64-pipe warp instructions per particle update.  None when no
    capture matches this run or the step-kernel sources changed since."""
    path = os.path.join(ROOT, "profiles", "step_counters.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    if rec.get("source_sha256") != library_source_hash():
        return None
    for e in rec.get("entries", []):
        if (e["workload"], e["field"], e["kernel"], list(e["step_config"])) == \
                (workload, field, kernel, list(cfg)):
            out = dict(e)
            # DRAM bytes scale with the particle count of the run (the field
            # term is fixed): per-update and field parts as captured
            if e.get("particles") != n and "dram_bytes_per_update" not in e:
                out.pop("dram_bytes_per_launch", None)
            return out
    return None


def step_roofline(workload, field, kernel, n, N, has_tau, cfg, prof, hbm_peak, peak_kind, clk,
                  sms):
    """Roofline of the step kernel: algorithmic bytes per launch (every record
    read and written once, every field value read once) over its mean
    CUDA-event duration, against the measured HBM copy bandwidth; beside it
    the instruction-issue ceiling (warp instructions per update from the ncu
    capture, at the SM clock sampled during the timed region)."""
    step_ms, step_n = prof["step"]
    rec_bytes = 48 + (8 if has_tau else 0) + 4
    field_bytes_cell = {"f64": 24, "f32": 12, "bf16": 6}[field]
    alg = n * 2 * rec_bytes + field_bytes_cell * N ** 3
    t = step_ms / step_n * 1e-3
    achieved = alg / t / 1e9
    cnt = measured_counters(workload, field, kernel, n, cfg) or {}
    traffic = cnt.get("dram_bytes_per_launch")
    if traffic is None and "dram_bytes_per_update" in cnt:
        traffic = int(cnt["dram_bytes_per_update"] * n + cnt.get("dram_field_bytes", 0))
    r = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
         "frac": round(achieved / hbm_peak, 4), "traffic": traffic,
         "algorithmic_bytes": int(alg), "kernel": "k_step", "peak_source": peak_kind,
         "kernel_ms_per_launch": round(step_ms / step_n, 4),
         "kernel_share": round(step_ms / sum(p[0] for p in prof.values()), 3)}
    wipu = cnt.get("warp_inst_per_update")
    if wipu:
        mhz = (clk or {}).get("sm_mhz") or 2070.0
        peak_issue = sms * 4 * mhz * 1e6  # one warp instruction per scheduler per cycle
        ach = wipu * n / t
        r["issue"] = {"bound": "issue", "achieved": round(ach / 1e12, 4),
                      "peak": round(peak_issue / 1e12, 4), "unit": "T warp-instructions/s",
                      "frac": round(ach / peak_issue, 4), "warp_inst_per_update": wipu,
                      "peak_source": f"{sms} SMs x 4 schedulers x {mhz:.0f} MHz sampled"}
    f64pu = cnt.get("fp64_warp_inst_per_update")
    if f64pu:
        peak_f64 = 0.625e12 / 32  # nominal 1.25 TFLOP/s = 0.625 T FMA lanes/s, in warp instructions
        ach = f64pu * n / t
        r["fp64_pipe"] = {"bound": "alu", "achieved": round(ach * 32 / 1e12, 4),
                          "peak": 0.625, "unit": "T FP64 lane-instructions/s",
                          "frac": round(ach / peak_f64, 4),
                          "fp64_warp_inst_per_update": f64pu,
                          "peak_source": "nominal GB300 FP64 1.25 TFLOP/s (FMA = 2 FLOP)"}
    return r


# ---------------------------------------------------------------- ranks

def aggregate_over_ranks(ms: float, units: int, dist=None, device: str = "cpu"):
    """Whole-job (time, units) over the ranks of an initialised process group:
    the slowest rank's time and the sum of all ranks' particle updates (one
    rank, or dist None: the inputs unchanged).  Barrier first, so no rank
    reduces before every rank has stopped its clock."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms, units
    import torch
    dist.barrier()
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), int(u.item())


# ---------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- CPU oracle leg

def cpu_info():
    """(cores the OS reports, CPU model string) of this machine."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        import platform
        model = platform.processor() or platform.machine()
    return os.cpu_count(), model


def oracle_rate(w, field_np, dt, x, v, tau, n_sample: int, steps: int, threads=None,
                migrate=True):
    """Particle-updates/s of the CPU oracle on the first n_sample particles:
    threads None = the plain single-threaded oracle, else its OpenMP build
    (particle loop on `threads` cores, 0 = all; migration and sort stay
    sequential).  migrate=False times the particle advance alone (the
    sampled-ID form of the precision workload).  Returns (rate, seconds,
    threads used) or None when the OpenMP build is unavailable."""
    import oracle
    used = oracle.use_threads(threads)
    if used is None:
        return None
    try:
        L = synth.L_BOX
        xs, vs = x[:, :n_sample].copy(), v[:, :n_sample].copy()
        ts = None if tau is None else tau[:n_sample].copy()
        if migrate:
            st = oracle.initial_state(w.N, L, w.sub, xs, vs, ts)
            t0 = time.perf_counter()
            oracle.run(st, field_np, L, w.sub, w.tau_const, dt, w.g, steps,
                       sort_every=w.sort_every, brick=8)
        else:
            t0 = time.perf_counter()
            oracle.advance(field_np, L, xs, vs, ts, w.tau_const, dt, w.g, steps)
        t = time.perf_counter() - t0
    finally:
        oracle.use_threads(None)
    return n_sample * steps / t, t, used


def cpu_baseline_leg(w, field_np, dt, x, v, tau, n_sample, steps, migrate=True, what=""):
    """The oracle timed single-threaded (the baseline proper, as it stands)
    and on all host cores (OpenMP build), with the core count and CPU model."""
    nproc, model = cpu_info()
    one = oracle_rate(w, field_np, dt, x, v, tau, n_sample, steps, None, migrate)
    rate, secs, _ = one
    out = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{what}first {n_sample} particles of the workload, {steps} steps"
                     f"{' incl. migration and the cell sort' if migrate else ' (advance only)'}"
                     f", {secs:.1f} s", "nproc": nproc, "cpu_model": model}
    many = oracle_rate(w, field_np, dt, x, v, tau, n_sample, steps, 0, migrate)
    if many is not None:
        r2, s2, used = many
        out["all_cores"] = {"value": r2, "unit": UNIT, "cores": used,
                            "sample": f"same sample, OpenMP over particles, {s2:.1f} s"}
    else:
        out["all_cores"] = None
    return out


# ---------------------------------------------------------------- adjoint

def adjoint_ratio(lcs, torch, steps=None):
    """Forward (with checkpoints every 20 steps) and backward time of the
    differentiation workload: 128^3 field, 2^20 particles, 200 steps."""
    w = synth.WORKLOADS["grad_128"]
    field, _ = synth.make_field(w, device="cuda")
    dt = synth.cfl_dt(synth.max_speed(field), w.N)
    x, v, _ = synth.make_particles(w, dt)
    target = torch.from_numpy(synth.positions(w.np_, synth.rng(w.number,
                                                               synth.STREAM_TARGET))).cuda()
    steps = steps or w.steps
    res = {}
    for rep in range(2):  # first repetition warms up (graph capture, allocations)
        sim = lcs.Simulator(field, x, v, dt, tau_const=w.tau_const, sub=w.sub, ckpt_every=20,
                            track_images=True, sort_every=10)
        st = torch.cuda.current_stream()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        torch.cuda.synchronize()
        e0.record(st)
        sim.step(steps)
        e1.record(st)
        xt, _ = sim.final_state_by_id()
        gx = 2.0 / w.np_ * (xt - target)
        gv = torch.zeros_like(gx)
        torch.cuda.synchronize()
        e1b = torch.cuda.Event(enable_timing=True)
        e1b.record(st)
        sim.backward(gx, gv)
        e2.record(st)
        torch.cuda.synchronize()
        fwd, bwd = e0.elapsed_time(e1), e1b.elapsed_time(e2)
        res = {"workload": "grad_128 (128^3, 2^20 particles, 2x2x2, checkpoints every 20)",
               "steps": steps, "forward_ms": round(fwd, 3), "backward_ms": round(bwd, 3),
               "ratio": round(bwd / fwd, 3)}
        sim.close()
    return res


# ---------------------------------------------------------------- batching

def batch_throughput(lcs, torch, steps=500, n_ens=48):
    """The batching workload (48 ensembles, grids 64-256^3, 10^4-10^7
    particles, FP32 fields, 2x2x2, sort every 10, 500 steps): total
    particle-updates/s of all ensembles in one context (autotuned) against
    the same ensembles stepped one context at a time in FP64 and in FP32."""
    ens = synth.batch_ensembles(n_ens, device="cuda")
    total = sum(e["n"] for e in ens)
    st = torch.cuda.current_stream()

    def timed(sim, k):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        sim.step(k)
        e1.record(st)
        sim.sync()
        return e0.elapsed_time(e1)

    spec = lambda e, dtype: dict(field=e["field"], x0=e["x0"], v0=e["v0"], dt=e["dt"],
                                 tau=e["tau"], sub=(2, 2, 2), sort_every=10, field_dtype=dtype)
    sim = lcs.Simulator(None, None, None, None, ensembles=[spec(e, "f32") for e in ens])
    block, items, mode = sim.tune(2)  # 2 steps per tried configuration
    done = 2 * int((sim.tune_trials_ms > 0).sum())
    timed(sim, 10 - done % 10)  # graph capture; the timed steps start on a sort period
    g0 = sim.graph_launches
    ms_batch = timed(sim, steps)
    graph_launches = sim.graph_launches - g0
    configs = {}
    for k in range(len(ens)):
        key = "x".join(map(str, sim.step_config_of(k)))
        configs[key] = configs.get(key, 0) + 1
    launches = sim.launches
    sim.close()
    solo = {}
    for dtype in ("f64", "f32"):
        ms = 0.0
        for e in ens:
            s1 = lcs.Simulator(**spec(e, dtype))
            timed(s1, 10)  # warm-up: graph capture
            ms += timed(s1, steps)
            s1.close()
        solo[dtype] = ms
    rate = lambda ms_: total * steps / (ms_ * 1e-3)
    return {"workload": f"{n_ens} ensembles, grids 64-256^3, {total} particles, FP32 fields, "
                        f"2x2x2 each, sort every 10",
            "steps": steps, "value_batched_f32": rate(ms_batch),
            "value_one_by_one_f64": rate(solo["f64"]), "value_one_by_one_f32": rate(solo["f32"]),
            "speedup_vs_one_by_one_f64": round(solo["f64"] / ms_batch, 3),
            "speedup_vs_one_by_one_f32": round(solo["f32"] / ms_batch, 3),
            "tuned_block": block, "tuned_items": items, "tuned_mode": mode,
            "configs_per_ensemble": configs,
            "graph_launches_per_step": round(graph_launches / steps, 4), "unit": UNIT}


# ---------------------------------------------------------------- end to end

def e2e_leg(sim, torch, n, has_tau, steps, dist=None):
    """The same metric through the public API with host buffers: every bench
    step copies the state in from pinned host memory (lcs_set_state), runs 10
    time steps and copies it back (lcs_get_state)."""
    stream = torch.cuda.current_stream()
    st_host = sim.get_state(device="cpu")
    h2d = n * (24 + 24 + (8 if has_tau else 0) + 4) + 8 * (len(st_host["seg"]))
    d2h = h2d
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        sim.set_state(st_host["x"], st_host["v"], st_host["ids"], st_host["seg"],
                      tau=st_host["tau"] if has_tau else None)
        sim.step(STEPS_PER_BENCH_STEP)
        st_host = sim.get_state(device="cpu", out={k: st_host[k] for k in
                                                   ("x", "v", "tau", "ids")})
    e1.record(stream)
    torch.cuda.synchronize()
    e_ms, e_units = aggregate_over_ranks(e0.elapsed_time(e1), n * STEPS_PER_BENCH_STEP * steps,
                                         dist, "cuda")
    return {"value": e_units / (e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "steps": steps,
            "wall_s": round(time.perf_counter() - t0, 3)}


def timed_rate(sim, torch, n, steps):
    """Particle-updates/s over `steps` time steps (CUDA events on the stream)."""
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    sim.step(steps)
    e1.record(st)
    sim.sync()
    return n * steps / (e0.elapsed_time(e1) * 1e-3)


# ---------------------------------------------------------------- all-FP64 kernel

def fp64_kernel_leg(lcs, torch, args, w, field, dt, x, v, tau, hbm_peak, peak_kind, clk):
    """The bench workload with the all-FP64-arithmetic step kernel
    (LCS_KERNEL_FP64: the paper's arithmetic, every operation on the FP64
    pipe), deferred scatter with one particle per thread."""
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    sim = lcs.Simulator(field, x, v, dt, tau=tau, tau_const=w.tau_const, g=w.g, sub=w.sub,
                        field_dtype="f64", kernel="fp64", sort_every=w.sort_every)
    cfg = (256, 1, 3)
    sim.set_step_config(*cfg)
    sim.step(STEPS_PER_BENCH_STEP)
    sim.sync()
    n = x.shape[1]
    rate = timed_rate(sim, torch, n, 2 * STEPS_PER_BENCH_STEP)
    prof = sim.profile_steps(STEPS_PER_BENCH_STEP)
    sim.close()
    return {"value": rate, "unit": UNIT, "steps": 2 * STEPS_PER_BENCH_STEP,
            "config": f"{w.name}, LCS_KERNEL_FP64 (all arithmetic FP64), step config "
                      f"{list(cfg)}",
            "roofline": step_roofline(w.name, "f64", "fp64", n, w.N, tau is not None, cfg,
                                      prof, hbm_peak, peak_kind, clk, sms)}


# ---------------------------------------------------------------- precision variants

def precision_throughput(lcs, torch, hbm_peak, peak_kind, clk, steps=20, cpu=True):
    """The precision workload (512^3 field, 10^8 particles, 8x8x8, gravity,
    sort every 10): particle-updates/s with the field stored in FP64
    (float-float kernel), FP32 and BF16, the FP32-over-FP64 speedup, and for
    each the step kernel's roofline; for the FP64 field also the end-to-end
    rate through the API with host buffers and the CPU oracle on the 10^5-ID
    subsample of the precision test (advance only: particles are independent)."""
    w = synth.WORKLOADS["precision_512"]
    field, _ = synth.make_field(w, device="cuda")
    dt = synth.cfl_dt(synth.max_speed(field), w.N)
    x, v, tau = synth.make_particles(w, dt)
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    out = {"workload": "precision_512 (512^3, 1e8 particles, 8x8x8, sort every 10)",
           "steps": steps, "unit": UNIT}
    for dtype in ("f64", "f32", "bf16"):
        sim = lcs.Simulator(field, x, v, dt, tau=tau, g=w.g, sub=w.sub, field_dtype=dtype,
                            sort_every=w.sort_every)
        sim.step(10)
        sim.sync()
        out[dtype] = timed_rate(sim, torch, w.np_, steps)
        prof = sim.profile_steps(STEPS_PER_BENCH_STEP)
        cfg = (256, 1, 3) if dtype == "f64" else (256, 2, 3)
        out[f"{dtype}_roofline"] = step_roofline(w.name, dtype, "auto", w.np_, w.N, True, cfg,
                                                 prof, hbm_peak, peak_kind, clk, sms)
        if dtype == "f64":
            out["f64_e2e"] = e2e_leg(sim, torch, w.np_, True, 2)
        sim.close()
        torch.cuda.empty_cache()
    out["f32_speedup_vs_f64"] = round(out["f32"] / out["f64"], 3)
    out["bf16_speedup_vs_f64"] = round(out["bf16"] / out["f64"], 3)
    if cpu:
        sample = np.sort(np.random.default_rng(700).choice(w.np_, 100_000, replace=False))
        out["f64_cpu_baseline"] = cpu_baseline_leg(
            w, field.cpu().numpy(), dt, np.ascontiguousarray(x[:, sample]),
            np.ascontiguousarray(v[:, sample]), tau[sample].copy(), 100_000, 20, migrate=False,
            what="the 10^5 sampled ids of the precision test: ")
    del field
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------- model variants

def variants_throughput(lcs, torch, w, field, dt, x, v, tau, steps=20, nu=2e-3):
    """The bench workload with the drag factor of Eq. (7) (kinematic viscosity
    nu, density ratio 843) and with a field evolving linearly in time between
    two snapshots (the second a phase-shifted copy of the first), against the
    frozen field with Stokes drag, with migration after each Runge-Kutta
    stage, and with every subdomain reading its own field brick (owned-field
    mode, the multi-GPU memory pattern): particle-updates/s for the FP64 field (float-float kernel) and the
    FP32 field, deferred-scatter kernel; and the wall time of the
    pair-separation histogram (g(r)) on the bench state."""
    st = torch.cuda.current_stream()
    out = {"workload": f"{w.name}; drag of Eq. (7) with nu {nu}, rho_p/rho 843; evolving "
                       f"field between two snapshots", "steps": steps, "unit": UNIT}
    field2 = torch.roll(field, shifts=7, dims=-1)
    for dtype in ("f64", "f32"):
        for variant in ("stokes", "nonlinear_drag", "evolving_field", "migrate_per_stage",
                        "owned_field"):
            kw = dict(drag="nonlinear", nu=nu) if variant == "nonlinear_drag" else {}
            if variant == "evolving_field":
                kw = dict(field_next=field2, t_start=0.0, t_field=(0.0, 100.0 * dt))
            if variant == "migrate_per_stage":
                kw = dict(migrate_per_stage=True)
            if variant == "owned_field":
                kw = dict(owned_field=True)
            sim = lcs.Simulator(field, x, v, dt, tau=tau, tau_const=w.tau_const, g=w.g,
                                sub=w.sub, field_dtype=dtype, sort_every=w.sort_every, **kw)
            sim.step(10)
            sim.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            sim.step(steps)
            e1.record(st)
            sim.sync()
            out[f"{dtype}_{variant}"] = x.shape[1] * steps / (e0.elapsed_time(e1) * 1e-3)
            sim.close()
        for variant in ("nonlinear_drag", "evolving_field", "migrate_per_stage", "owned_field"):
            out[f"{dtype}_{variant}_over_stokes"] = round(out[f"{dtype}_{variant}"] /
                                                          out[f"{dtype}_stokes"], 3)
    del field2
    # particle statistics: the pair-separation histogram behind g(r) on the
    # bench state (pairs closer than one grid cell, 32 bins)
    sim = lcs.Simulator(field, x, v, dt, tau=tau, tau_const=w.tau_const, g=w.g, sub=w.sub,
                        sort_every=w.sort_every)
    sim.step(10)
    sim.sync()
    L = synth.L_BOX
    t0 = time.perf_counter()
    reps = 3
    for _ in range(reps):
        counts = sim.pair_histogram(L / w.N, 32)
    ms = (time.perf_counter() - t0) * 1e3 / reps
    sim.close()
    out["pair_histogram"] = {"ms": round(ms, 3), "pairs_below_one_cell": int(counts.sum()),
                             "particles_per_s": x.shape[1] / (ms * 1e-3)}
    return out


# ---------------------------------------------------------------- main

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="scale_256")
    ap.add_argument("--kernel", default="auto", choices=["auto", "fp64", "df"])
    ap.add_argument("--field", default="f64", choices=["f64", "f32", "bf16"])
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--variants", type=int, default=1,
                    help="also time the nonlinear drag of Eq. (7) and an evolving field")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=1 << 20)
    ap.add_argument("--precision", type=int, default=1,
                    help="also time FP64/FP32/BF16 field storage on precision_512")
    ap.add_argument("--batch", type=int, default=1,
                    help="also time the 48-ensemble batching workload")
    ap.add_argument("--adjoint", type=int, default=1,
                    help="also time forward (taped) vs backward on grad_128")
    ap.add_argument("--step-config", default="",
                    help="threads,items,mode of the step kernel instead of autotuning")
    ap.add_argument("--np", type=int, default=0,
                    help="particle count override (small profiling cases only)")
    ap.add_argument("--reps", type=int, default=5,
                    help="timed repetitions of K bench steps (the median is reported)")
    ap.add_argument("--fp64-kernel", type=int, default=1,
                    help="also time the all-FP64-arithmetic step kernel (LCS_KERNEL_FP64)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, world, rank)

    import torch
    import paper_2604_11008_gb300 as lcs

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    w, field, modes, dt, x, v, tau = build_workload(args.workload, "cuda", args.np or None)
    sim = lcs.Simulator(field, x, v, dt, tau=tau, tau_const=w.tau_const, g=w.g, sub=w.sub,
                        field_dtype=args.field, kernel=args.kernel, sort_every=w.sort_every)
    n = x.shape[1]
    K, W, R = args.steps, args.warmup, max(1, args.reps)
    if args.step_config:
        tuned = tuple(int(t) for t in args.step_config.split(","))
        sim.set_step_config(*tuned)
        sim.tune_trials_ms = []
    else:
        tuned = sim.tune(2)  # picks the step kernel; advances the state 2 steps per trial
    # the L2 (129 MB) is far smaller than the particle state (~1 GB) and the
    # field (537 MB): every timed step streams its inputs from HBM
    for _ in range(W):
        sim.step(STEPS_PER_BENCH_STEP)
    sim.sync()
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    l0 = sim.launches
    reps_ms = []
    for _ in range(R):  # R repetitions of exactly K bench steps; the median is reported
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(K):
            sim.step(STEPS_PER_BENCH_STEP)
        ev1.record(stream)
        ev1.synchronize()
        sim.sync()
        torch.cuda.synchronize()
        ms_r, updates = aggregate_over_ranks(ev0.elapsed_time(ev1), n * STEPS_PER_BENCH_STEP * K,
                                             dist, "cuda")
        reps_ms.append(ms_r)
    launches = (sim.launches - l0) // R
    clk = clocks.stop()
    ms = float(np.median(reps_ms))
    value = updates / (ms * 1e-3)

    # per-kernel device time (un-graphed replay of one sort period, events
    # around every kernel class on the launching stream)
    prof = sim.profile_steps(STEPS_PER_BENCH_STEP)
    hbm_peak, peak_kind, peaks = load_peaks()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    roofline = step_roofline(args.workload, args.field, args.kernel, n, w.N, tau is not None,
                             tuned, prof, hbm_peak, peak_kind, clk, sms)

    # end to end through the public API with host buffers
    e2e = None
    if args.e2e_steps > 0:
        e2e = e2e_leg(sim, torch, n, tau is not None, args.e2e_steps, dist)

    fp64_kernel = None
    if rank == 0 and args.fp64_kernel and args.field == "f64" and args.kernel == "auto":
        fp64_kernel = fp64_kernel_leg(lcs, torch, args, w, field, dt, x, v, tau, hbm_peak,
                                      peak_kind, clk)
    adjoint = None
    if rank == 0 and args.adjoint:
        adjoint = adjoint_ratio(lcs, torch)
    batch = None
    if rank == 0 and args.batch:
        batch = batch_throughput(lcs, torch)
    precision = None
    if rank == 0 and args.precision:
        precision = precision_throughput(lcs, torch, hbm_peak, peak_kind, clk,
                                         cpu=not args.no_cpu_baseline)
    variants = None
    if rank == 0 and args.variants:
        variants = variants_throughput(lcs, torch, w, field, dt, x, v, tau)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        field_np = field.cpu().numpy() if args.field == "f64" else None
        if field_np is not None:
            xs, vs = x, v
            cpu = cpu_baseline_leg(w, field_np, dt, xs, vs, tau, min(args.cpu_sample, n),
                                   STEPS_PER_BENCH_STEP)

    sim.close()
    if rank == 0:
        arith = {"f64": "float-float (FP32 pairs, 48-bit) on int64 fixed-point positions",
                 "f32": "FP32 field and increments on int64 fixed-point positions",
                 "bf16": "BF16 field, FP32 increments on int64 fixed-point positions"}
        if args.kernel == "fp64":
            arith["f64"] = "FP64"
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
               "warmup": W, "ms_per_step": ms / K, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None,
               "dtype": "f64" if args.kernel == "fp64" else
                        {"f64": "f32x2+i64", "f32": "f32+i64", "bf16": "bf16/f32+i64"}[args.field],
               "data": "synthetic",
               "config": {"workload": w.name, "grid": f"{w.N}^3", "modes": w.M,
                          "particles_per_gpu": n, "subdomains": "x".join(map(str, w.sub)),
                          "sort_every": w.sort_every, "dt": dt,
                          "time_steps_per_bench_step": STEPS_PER_BENCH_STEP,
                          "field_storage": args.field, "kernel": args.kernel,
                          "arithmetic": arith[args.field],
                          "tuned_block_items_mode": list(tuned),
                          "tune_trials_ms": [round(float(t), 3) for t in sim.tune_trials_ms],
                          "repetitions": R, "reps_ms": [round(t, 3) for t in reps_ms],
                          "l2": "inputs larger than L2 (state ~1 GB, field 0.54 GB)",
                          "parallelism": f"replicas{world}"},
               "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
               "fp64_kernel": fp64_kernel, "adjoint": adjoint, "batch": batch,
               "precision": precision, "model_variants": variants,
               "gpu_launches": int(launches), "clocks": clk,
               "kernel_profile_ms": {k: round(v_[0], 4) for k, v_ in prof.items()}}
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


def run_reference(args, world, rank):
    """The CPU oracle timed on this machine's host cores (rank 0 only)."""
    if rank != 0:
        return
    w, field, modes, dt, x, v, tau = build_workload(args.workload, "cpu",
                                                      n_override=args.cpu_sample)
    n = args.cpu_sample
    import oracle
    L = synth.L_BOX
    st = oracle.initial_state(w.N, L, w.sub, x, v, tau)
    for _ in range(args.warmup):
        oracle.run(st, field, L, w.sub, w.tau_const, dt, w.g, 1, sort_every=0)
    t0 = time.perf_counter()
    done = 0
    for k in range(args.steps):
        oracle.run(st, field, L, w.sub, w.tau_const, dt, w.g, STEPS_PER_BENCH_STEP,
                   sort_every=w.sort_every, brick=8)
        done += STEPS_PER_BENCH_STEP
    t = time.perf_counter() - t0
    value = n * done / t
    nproc, model = cpu_info()
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3 / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": w.name, "grid": f"{w.N}^3", "particles": n,
                      "subdomains": "x".join(map(str, w.sub)), "sort_every": w.sort_every,
                      "dt": dt, "time_steps_per_bench_step": STEPS_PER_BENCH_STEP},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": f"first {n} particles of the workload (bounded sample), "
                                      f"{done} time steps", "nproc": nproc,
                            "cpu_model": model},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
