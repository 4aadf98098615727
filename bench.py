#!/usr/bin/env python3
"""Benchmark of the fused FP64 RK4 ray tracer on the GRIN-fibre workload.

Workload (one "step"): 1,048,576 rays in a parabolic GRIN fibre (n0 = 1.5,
a = 2) with 16 Gaussian blobs, launched from x = -1 within 10 degrees of +x,
set on shell (gf_rays_onshell) and traced by 10,000 RK4 steps of dt = 5e-4
(gf_trace_rk4), FP64.  Metric: ray-steps/s (one RK4 step of one ray), counted
from the per-ray step counters the kernel writes.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gf|reference]

Multi-GPU (torchrun, one rank per GPU): every rank traces its own independent
batch of the same size (weak scaling, no data-path collective); timing is the
max over ranks.  `--impl reference` times the plain FP64 CPU oracle on the
host cores on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import inspect
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2508_15967_gb300 import workloads as W  # noqa: E402

METRIC = "ray-steps/s FP64 at 1M rays (GRIN fibre + 16 blobs, RK4)"
UNIT = "ray-steps/s"
SMS = 152


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gf", "reference"], default="gf")
    ap.add_argument("--rays", type=int, default=1 << 20,
                    help="rays of the headline trace (adjoint workload: at most its 65,536)")
    ap.add_argument("--nsteps", type=int, default=10000,
                    help="RK4 steps of the headline trace (aniso workload: at most its 4000)")
    ap.add_argument("--precision", choices=["f64", "f32", "f64x"], default="f64",
                    help="f64: IEEE double throughout (the headline); f32; f64x: double state and "
                         "integrator with double-float blob sums")
    ap.add_argument("--cpu-rays", type=int, default=4096,
                    help="rays of the oracle sample (x the full step count)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the secondary measurements (f64x, luneburg, cold, aniso, adjoint, batched)")
    ap.add_argument("--workload", choices=["grin", "luneburg", "cold", "batched", "aniso", "adjoint", "generated"],
                    default="grin", help="grin: the headline line; others print that measurement alone")
    ap.add_argument("--media", type=int, default=4096, help="batched: number of media")
    ap.add_argument("--tune-cache", default=None,
                    help="batched: autotuner cache file (written after tuning, reused when it holds the shape)")
    ap.add_argument("--scaling", choices=["weak", "strong"], default="weak",
                    help="N > 1: weak = every rank its own batch of the workload's size; strong = one "
                         "batch split across the ranks (grin, batched, adjoint)")
    ap.add_argument("--drawn-order", action="store_true",
                    help="batched, adjoint: rays in the order drawn, not sorted along a Morton curve of "
                         "their launch points")
    return ap.parse_args()


# --------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        rows = [l.split(",") for l in open(self.path).read().strip().splitlines() if l.count(",") >= 8]
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if "Active" == r[5 + j].strip()})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------------- oracle leg

def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:  # noqa: BLE001 -- a report field
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_throughput(wl, n_rays: int) -> dict:
    """Plain FP64 oracle on the first n_rays rays of the workload (host cores)."""
    import oracle as O
    m = O.medium(**wl.medium)
    k0, _ = O.onshell(m, wl.x0[:n_rays], wl.d[:n_rays])
    r = O.make_rays(wl.x0[:n_rays], k0)
    t0 = time.perf_counter()
    O.trace_rk4(m, r, wl.omega, wl.dt, wl.n_steps)
    el = time.perf_counter() - t0
    units = int(r.steps.astype(np.int64).sum())
    return {"value": units / el, "unit": UNIT, "cores": O.num_threads(), "cpu_model": cpu_model(),
            "kind": "oracle",
            "sample": f"{n_rays} rays x {wl.n_steps} RK4 steps of the same workload "
                      f"({units} ray-steps, {el:.1f} s)", "seconds": el}


def oracle_sample(name: str) -> dict:
    """The oracle as it stands on a bounded sample of one secondary workload
    (host cores), in the unit of that workload's GPU figure; a few seconds of
    CPU work each.  Inputs are prepared untimed (on-shell k, Newton on k_x)."""
    import oracle as O
    t0 = None
    reps = 1
    if name == "luneburg":
        wl = W.luneburg()
        n, reps = wl.n, 25          # one trace is ~10 ms of host time: repeat it
    elif name == "cold":
        wl, n = W.cold(n=32768), 32768
    elif name == "aniso":
        wl, n = W.aniso(n=1024), 1024
    elif name == "adjoint":
        wl, n = W.adjoint(n=256), 256
    elif name == "batched":
        wl = W.batched()
        off = wl.extra["offsets"]
        m_end = int(np.searchsorted(off, 65536, side="left"))
        m_end = max(1, min(m_end, len(off) - 1))
        n = int(off[m_end])
    else:
        raise ValueError(name)
    if name == "batched":
        blobs = wl.extra["blobs"]
        media = [O.medium(kind="luneburg", blobs=blobs[j]) for j in range(m_end)]
        k0 = np.empty_like(wl.x0[:n])
        for j in range(m_end):
            lo, hi = int(off[j]), int(off[j + 1])
            if hi > lo:
                k0[lo:hi], _ = O.onshell(media[j], wl.x0[lo:hi], wl.d[lo:hi])
        r = O.make_rays(wl.x0[:n], k0)
        e = wl.extra
        t0 = time.perf_counter()
        O.trace_dopri5(media, off[:m_end + 1], r, wl.omega, rtol=e["rtol"], atol=e["atol"], h0=e["h0"],
                       t_max=e["t_max"], radius=wl.radius, max_steps=e["max_steps"])
        el = time.perf_counter() - t0
        units = int(r.steps.astype(np.int64).sum())
        what = f"DOPRI5 over the first {m_end} media ({n} rays), accepted steps"
        unit = "accepted ray-steps/s"
    else:
        m = O.medium(**wl.medium)
        if name == "cold":
            k0, st, _ = O.newton_kx(m, wl.x0[:n], wl.extra["k_start"][:n], wl.omega)
        else:
            k0, st = O.onshell(m, wl.x0[:n], wl.d[:n], wl.omega)
        el, units = 0.0, 0
        for _ in range(reps):
            r = O.make_rays(wl.x0[:n], k0, status=st if name == "cold" else None)
            t0 = time.perf_counter()
            if name == "adjoint":
                O.tangent_rk4(m, r, wl.omega, wl.dt, wl.n_steps)
            else:
                O.trace_rk4(m, r, wl.omega, wl.dt, wl.n_steps)
            el += time.perf_counter() - t0
            units += n * wl.n_steps if name == "adjoint" else int(r.steps.astype(np.int64).sum())
        if name == "adjoint":
            what = (f"tangent-linear gradient (the oracle's adjoint) of {n} rays x {wl.n_steps} RK4 steps, "
                    f"{wl.medium['blobs'].shape[0]} parameters")
            unit = "gradient ray-steps/s"
        else:
            what = f"{n} rays x {wl.n_steps} RK4 steps" + (f", {reps} times" if reps > 1 else "")
            unit = UNIT
    return {"value": units / el, "unit": unit, "cores": O.num_threads(), "cpu_model": cpu_model(),
            "kind": "oracle",
            "sample": f"{what}: {units} units in {el:.2f} s (a sample of the same workload)"}


def _with_oracle(res: dict, name: str) -> dict:
    """Attach the oracle's figure on a sample of the same workload (never
    fails the measurement it is attached to)."""
    try:
        res["cpu_baseline"] = oracle_sample(name)
    except Exception as e:  # noqa: BLE001 -- a report field, not a result
        res["cpu_baseline"] = {"error": f"{type(e).__name__}: {e}"}
    return res


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = W.grin(n=max(a.cpu_rays, 1), n_steps=a.nsteps)
    for _ in range(a.warmup):
        oracle_throughput(wl, min(256, a.cpu_rays))
    vals, secs = [], 0.0
    for _ in range(a.steps):
        r = oracle_throughput(wl, a.cpu_rays)
        vals.append(r["value"])
        secs += r["seconds"]
    v = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * secs / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"grin_fibre_16_blobs rays={a.cpu_rays} (sample of {a.rays}) "
                                   f"rk4_steps={a.nsteps} dt=5e-4", "parallelism": "host cores"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": r["cores"], "cpu_model": r["cpu_model"],
                             "kind": "oracle", "sample": r["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- GPU leg

# Algorithmic FP64 flops (add/mul 1, fma 2) of the fused RK4 kernel, per unit
# of work; units are counted exactly by an untimed pass with work counters.
#   live blob term  18: x - c (3), |x - c|^2 (5), exponent (1), A e, n^2 +=,
#                       2 s A e (3), grad += (6); the base-2 table exp at FP64
#                       accuracy takes no FP64 operation in this kernel (its
#                       reduction and polynomial run on the FP32 pipes, the
#                       table product in integer arithmetic)
#   culled term      9: x - c, |x - c|^2 and the exponent, then skipped
#   evaluation      51: GRIN base n^2 and gradient (8), 1/n^2 as 8, the two
#                       prefactors (2), f (6), stage update and RK4 accumulate (24),
#                       D at one evaluation in four (5/4 rounded up to 3)
#   ray-step        18: final y + dt/6 (...) update
FLOPS_LIVE_TERM, FLOPS_CULLED_TERM, FLOPS_EVAL, FLOPS_STEP = 18, 9, 51, 18

# DRAM bytes (read + write) of one rk4_kernel<double, GRIN> launch over
# 1,048,576 rays, from an ncu capture of the same launch shape (the kernel
# loads and stores the ray state once, so the count does not depend on the
# number of steps).  Valid only for the FP64 GRIN kernel as captured.
TRAFFIC_BYTES_1M = 75_730_176 + 23_068_672


def algorithmic_flops(evals: int, live: int, n_blobs: int, ray_steps: int) -> int:
    culled = evals * n_blobs - live
    return FLOPS_LIVE_TERM * live + FLOPS_CULLED_TERM * culled + FLOPS_EVAL * evals + FLOPS_STEP * ray_steps


# Per-unit algorithmic counts from the workload descriptions (FP64 flops, fma = 2;
# exponentials and divisions are not counted, every blob term is charged whether
# or not the kernel culls it).  These give each roofline's primary fraction; the
# counted-work model above (live and culled terms from the kernel's counters)
# is reported beside the headline's.
#   GRIN + 16 blobs, per ray-step: 4 evaluations x (16 blob terms x 18 + index
#     law 6 + right-hand side 8) + RK4 combination 84
#   batched DOPRI5, 8 blobs, per attempted step (accepted or rejected):
#     6 evaluations x (8 x 18 + 13) + stage combination and error norm 150
#   adjoint medium, 64 blobs, per ray-step of a forward trace: 4 x (64 x 18 + 14) + 84
#   cold plasma, two species, per ray-step, counted from the evaluator: per
#     species 49 flops (and a reciprocal), D, its partials and f 83 (and a
#     reciprocal; D formed at every evaluation), stage update 24, RK4 18
MODEL_GRIN_RAY_STEP = 4 * (16 * 18 + 6 + 8) + 84
MODEL_DOPRI5_ATTEMPT = 6 * (8 * 18 + 13) + 150
MODEL_ADJ_FWD_RAY_STEP = 4 * (64 * 18 + 6 + 8) + 84
MODEL_COLD_RAY_STEP = 4 * (2 * 49 + 83 + 24) + 18
#   adjoint backward, per ray-step: the forward recomputation (as above) and the
#     vector-Jacobian product of each of the 4 stages: per blob term 27 (x - c 3,
#     (x - c).Kbar 5, the theta-bar update 5, the Hessian-vector term 14), per
#     stage 50 (Kbar, the quotient-rule scalar, base Hessian, ybar), lambda 6
MODEL_ADJ_BWD_RAY_STEP = MODEL_ADJ_FWD_RAY_STEP + 4 * (64 * 27 + 50) + 6
MODEL_TEXT = {
    "grin": f"{MODEL_GRIN_RAY_STEP} flops per ray-step: 4 evaluations x (16 blob terms x 18 + index law 6 + "
            "right-hand side 8) + RK4 combination 84; every blob term charged, also those the kernel skips as "
            "negligible (exponent below -58.5 in base 2), exponentials and divisions not counted",
    "dopri5": f"{MODEL_DOPRI5_ATTEMPT} flops per attempted step: 6 evaluations x (8 blob terms x 18 + 13) "
              "+ stage combination and error norm 150; exponentials and divisions not counted",
    "adj_fwd": f"{MODEL_ADJ_FWD_RAY_STEP} flops per ray-step: 4 evaluations x (64 blob terms x 18 + 14) + 84",
    "adj_bwd": f"{MODEL_ADJ_BWD_RAY_STEP} flops per ray-step: recomputation {MODEL_ADJ_FWD_RAY_STEP} + 4 stages x "
               "(64 blob terms x 27 + 50) + 6 for the vector-Jacobian products; exponentials not counted",
    "cold": f"{MODEL_COLD_RAY_STEP} flops per ray-step: 4 evaluations x (2 species x 49 + D and partials 83 + "
            "stage update 24) + 18; reciprocals not counted",
}


def fp64_peak_tflops(sm_mhz: float) -> float:
    """Non-tensor FP64 peak from unit counts and clock: 152 SMs x 2 DFMA/clk x 2 flops."""
    return SMS * 2 * 2 * sm_mhz * 1e6 / 1e12


def fp32_peak_tflops(sm_mhz: float) -> float:
    """Non-tensor FP32 peak: 152 SMs x 128 FFMA/clk x 2 flops."""
    return SMS * 128 * 2 * sm_mhz * 1e6 / 1e12


def roofline_of(flops: float, seconds: float, peak: float) -> dict:
    a = flops / seconds / 1e12
    return {"achieved_tflops": a, "frac": a / peak}


def _batch_rays(gf, torch, wl, media, off):
    """Device rays of a batch with k set on shell per medium (gf_rays_onshell)."""
    init = gf.Rays.from_numpy(wl.x0, None)
    dirs = torch.from_numpy(np.ascontiguousarray(wl.d.T)).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    for j, m in enumerate(media):
        lo, hi = int(off[j]), int(off[j + 1])
        if hi > lo:
            s = gf.GfRays(hi - lo, init.y.stride(0), init.y.data_ptr() + 8 * lo, init.t.data_ptr() + 8 * lo,
                          init.status.data_ptr() + 4 * lo, init.steps.data_ptr() + 4 * lo,
                          init.d_res.data_ptr() + 8 * lo, init.d_max.data_ptr() + 8 * lo)
            gf._check("gf_rays_onshell", gf.lib().gf_rays_onshell(m.handle, gf.GF_F64, gf.C.byref(s),
                                                                  dirs.data_ptr() + 8 * lo, 1.0, stream))
    return init


def measure_batched(gf, torch, tune_cache: str | None = None, n_media: int = 4096, peak: float | None = None,
                    morton: bool = True, shard: int = 0, media_range: tuple[int, int] | None = None,
                    full: bool = True, barrier=None) -> dict:
    """Batched DOPRI5 workload (4096 Luneburg + 8-blob media, ~12.56M rays,
    rtol = atol = 1e-9, exit at r = 1.5): persistent work-stealing graph launch
    vs one launch per medium (also a graph) and the persistent launch in
    GF_F64X, each timed once after a warm-up.  media_range = (m_lo, m_hi)
    traces only those media (a strong-scaling shard); full = False times the
    persistent launch alone."""
    peak = fp64_peak_tflops(2070.0) if peak is None else peak
    wl = W.batched(n_media=n_media, morton=morton, shard=shard)
    blobs, off = wl.extra["blobs"], wl.extra["offsets"]
    m_lo, m_hi = (0, len(off) - 1) if media_range is None else media_range
    sub_off = np.asarray(off[m_lo:m_hi + 1]) - int(off[m_lo])
    r_lo, r_hi = int(off[m_lo]), int(off[m_hi])
    wl.x0, wl.d = wl.x0[r_lo:r_hi], wl.d[r_lo:r_hi]
    media = [gf.gf_medium_create("luneburg", blobs=blobs[j]) for j in range(m_lo, m_hi)]
    batch = gf.gf_batch_create(media, sub_off)
    init = _batch_rays(gf, torch, wl, media, sub_off)
    e = wl.extra
    ctl = gf.step_ctl(rtol=e["rtol"], atol=e["atol"], h0=e["h0"], t_max=e["t_max"], radius=wl.radius,
                      max_steps=e["max_steps"])
    t0 = time.perf_counter()
    tune = gf.gf_dopri5_autotune(batch, init, 1.0, ctl, tune_cache)
    tune_s = time.perf_counter() - t0
    rays = init.clone()
    rej = torch.zeros(rays.n, dtype=torch.int32, device="cuda")

    def timed(sched):
        ms = []
        for it in range(2):                            # warm-up (graph capture), then timed
            for src, dst in zip((init.y, init.t, init.status, init.steps, init.d_max),
                                (rays.y, rays.t, rays.status, rays.steps, rays.d_max)):
                dst.copy_(src)
            if it == 1 and barrier is not None:
                barrier()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            gf.gf_trace_dopri5(batch, rays, rej, 1.0, ctl, sched, None)
            ev1.record()
            torch.cuda.synchronize()
            ms.append(ev0.elapsed_time(ev1))
        steps = int(rays.steps.to(torch.int64).sum().item())
        rejected = int(rej.to(torch.int64).sum().item())
        return {"ms": ms[-1], "accepted_ray_steps": steps, "rejected": rejected,
                "ray_steps_per_s": steps / (ms[-1] / 1e3),
                **roofline_of(MODEL_DOPRI5_ATTEMPT * (steps + rejected), ms[-1] / 1e3, peak)}

    out = {"persistent": timed(gf.GF_SCHED_PERSISTENT)}
    if full:
        out["per_medium"] = timed(gf.GF_SCHED_PER_MEDIUM)
        # the same batch with double-float blob sums (GF_F64X), tuned for that mode
        gf.gf_batch_set_precision(batch, gf.GF_F64X)
        gf.gf_dopri5_autotune(batch, init, 1.0, ctl, None)
        out["persistent_f64x"] = timed(gf.GF_SCHED_PERSISTENT)
        out["persistent_f64x"]["note"] = ("GF_F64X: double state and controller, double-float blob sums on "
                                          "the FP32 pipes; the fraction is of the FP64 peak")
        gf.gf_batch_set_precision(batch, gf.GF_F64)
        out["speedup_persistent_vs_per_medium"] = out["per_medium"]["ms"] / out["persistent"]["ms"]
    order = "Morton order per medium" if morton else "drawn order"
    return {"workload": f"{m_hi - m_lo} Luneburg+8-blob media, {wl.n} rays ({order}), DOPRI5 rtol=atol=1e-9, "
                        f"exit r=1.5",
            **out, "roofline_model": MODEL_TEXT["dopri5"], "peak_tflops": peak,
            "tune": {"block": tune.block, "rays_per_thread": tune.rays_per_thread,
                     "compaction": tune.compaction, "chunk": tune.chunk, "seconds": tune_s}}


# FP64 flops of one evaluation of the separable tricubic spline medium:
# 16 (y, z) rows x (4 nodes x 7 channels x 2 fma for value and d/dx, then
# 7 channels x 4 fma into value and the three gradients) = 1344 fma, weights
# of three axes (~60 flops), D and the right-hand side (~60 flops).
FLOPS_SPLINE_EVAL = 2 * 1344 + 60 + 60


def measure_aniso(gf, torch, peak_tflops: float, n_steps: int | None = None) -> dict:
    """Anisotropic tricubic B-spline workload (262,144 rays, 128^3 grid, RK4
    dt = 1e-3 x 4000, FP64; n_steps shortens the trace), one warm-up trace of
    up to 100 steps then one timed."""
    wl = W.aniso()
    n_steps = wl.n_steps if n_steps is None else n_steps
    m = gf.gf_medium_create(**wl.medium)
    init = gf.Rays.from_numpy(wl.x0, None)
    gf.gf_rays_onshell(m, init, torch.from_numpy(np.ascontiguousarray(wl.d.T)).cuda(), 1.0)
    rays = init.clone()
    gf.gf_trace_rk4(m, rays, 1.0, wl.dt, min(100, n_steps))
    rays = init.clone()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    gf.gf_trace_rk4(m, rays, 1.0, wl.dt, n_steps)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    units = int(rays.steps.to(torch.int64).sum().item())
    flops = (4 * units + wl.n) * FLOPS_SPLINE_EVAL
    return {"workload": f"{wl.n} rays, 128^3 tricubic spline grid (64 MiB FP32), RK4 dt=1e-3 x {n_steps}, FP64",
            "ms": ms, "ray_steps_per_s": units / (ms / 1e3),
            "achieved_tflops": flops / (ms / 1e3) / 1e12, "frac_fp64_peak": flops / (ms / 1e3) / 1e12 / peak_tflops,
            "max_abs_D": rays.d_max.max().item()}


def measure_luneburg(gf, torch) -> dict:
    """Luneburg lens workload (1,024 rays, RK4 dt = 1e-3 x 2000, FP64): far
    less than one wave of the GPU (152 SMs x 5 blocks of 128), so it is bound
    by the latency of one ray's 2000 sequential steps; time only.  Median of
    five traces after one warm-up."""
    wl = W.luneburg()
    m = gf.gf_medium_create(**wl.medium)
    init = gf.Rays.from_numpy(wl.x0, None)
    gf.gf_rays_onshell(m, init, torch.from_numpy(np.ascontiguousarray(wl.d.T)).cuda(), 1.0)
    ms = []
    for it in range(6):
        rays = init.clone()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        gf.gf_trace_rk4(m, rays, 1.0, wl.dt, wl.n_steps)
        e1.record()
        torch.cuda.synchronize()
        if it > 0:
            ms.append(e0.elapsed_time(e1))
    t = statistics.median(ms)
    return {"workload": f"{wl.n} rays, Luneburg lens, RK4 dt={wl.dt} x {wl.n_steps}, FP64",
            "ms": t, "ray_steps_per_s": wl.n * wl.n_steps / (t / 1e3), "us_per_step": 1e3 * t / wl.n_steps}


def measure_cold(gf, torch, peak: float | None = None, n: int | None = None, n_steps: int | None = None) -> dict:
    """Cold-plasma workload (1,048,576 rays in the magnetised slab of Sec. 4.1
    with the Eq. 4 density gradient, O branch, RK4 dt = 1e-2 x 1500, FP64),
    the counterpart of the paper's own benchmark (1e6 cold-plasma rays, timed
    without setup): Newton on k_x, then one warm-up and one timed trace.
    n and n_steps shorten it (profiling captures)."""
    d = inspect.signature(W.cold).parameters
    wl = W.cold(n=min(n or d["n"].default, d["n"].default),
                n_steps=min(n_steps or d["n_steps"].default, d["n_steps"].default))
    m = gf.gf_medium_create(**wl.medium)
    init = gf.Rays.from_numpy(wl.x0, wl.extra["k_start"])
    gf.gf_rays_newton_kx(m, init, wl.omega)
    torch.cuda.synchronize()
    ok = int((init.status == 0).sum().item())
    ms = []
    for _ in range(2):
        rays = init.clone()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        gf.gf_trace_rk4(m, rays, wl.omega, wl.dt, wl.n_steps)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    units = int(rays.steps.to(torch.int64).sum().item())
    peak = fp64_peak_tflops(2070.0) if peak is None else peak
    return {"workload": f"{wl.n} rays, cold plasma slab (electrons + ions, f = 1 + 0.1 x), O branch, "
                        f"RK4 dt={wl.dt} x {wl.n_steps}, FP64",
            "ms": ms[-1], "ray_steps_per_s": units / (ms[-1] / 1e3),
            **roofline_of(MODEL_COLD_RAY_STEP * units, ms[-1] / 1e3, peak),
            "roofline_model": MODEL_TEXT["cold"], "peak_tflops": peak, "newton_converged": ok,
            "reflected": int(((rays.y[3] < 0) & (init.status == 0)).sum().item()),
            "max_abs_D": rays.d_max[init.status == 0].max().item()}


def measure_f64x(gf, torch, wl, m, x0, dirs, rays) -> dict:
    """The headline workload in the GF_F64X mode (double state and integrator,
    double-float blob sums), one warm-up and one timed trace."""
    ms = []
    for _ in range(2):
        rays.y[:3].copy_(x0)
        for t in (rays.t, rays.status, rays.steps, rays.d_max):
            t.zero_()
        gf.gf_rays_onshell(m, rays, dirs, wl.omega)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        gf.gf_trace_rk4(m, rays, wl.omega, wl.dt, wl.n_steps, precision=gf.GF_F64X)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    units = int(rays.steps.to(torch.int64).sum().item())
    return {"ray_steps_per_s": units / (ms[-1] / 1e3), "ms": ms[-1], "max_abs_D": rays.d_max.max().item(),
            "dtype": "f64 state and integrator, f32x2 (double-float) blob sums",
            "parity": "<= 1e-9 relative to the FP64 oracle in tests/test_gpu_f64x.py"}


def measure_f32(gf, torch, wl, m, peak32: float) -> dict:
    """The headline workload on the FP32 path (FP32 state with Kahan-compensated
    updates, FP32 blob sums with the hardware base-2 exponential): one warm-up
    and one timed trace, then an untimed pass with work counters; rooflines
    against the FP32 non-tensor peak."""
    x0 = torch.from_numpy(np.ascontiguousarray(wl.x0.T)).to("cuda", torch.float32)
    dirs = torch.from_numpy(np.ascontiguousarray(wl.d.T)).to("cuda", torch.float32)
    rays = gf.Rays.empty(wl.n, torch.float32)

    def trace(counters=None):
        rays.y[:3].copy_(x0)
        for t in (rays.t, rays.status, rays.steps, rays.d_max):
            t.zero_()
        gf.gf_rays_onshell(m, rays, dirs, wl.omega)
        if counters is not None:
            gf.gf_bench_set_counters(counters)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        gf.gf_trace_rk4(m, rays, wl.omega, wl.dt, wl.n_steps)
        e1.record()
        torch.cuda.synchronize()
        if counters is not None:
            gf.gf_bench_set_counters(None)
        return e0.elapsed_time(e1)

    trace()
    ms = trace()
    units = int(rays.steps.to(torch.int64).sum().item())
    counters = torch.zeros(2, dtype=torch.int64, device="cuda")
    trace(counters)
    evals, live = (int(v) for v in counters.tolist())
    counted = algorithmic_flops(evals, live, wl.medium["blobs"].shape[0], units)
    return {"workload": f"grin_fibre_16_blobs rays={wl.n} rk4_steps={wl.n_steps} dt={wl.dt}, FP32",
            "dtype": "f32", "ms": ms, "ray_steps_per_s": units / (ms / 1e3),
            "roofline": {"bound": "alu", "unit": "TFLOP/s", "peak": peak32,
                         **roofline_of(MODEL_GRIN_RAY_STEP * units, ms / 1e3, peak32),
                         "model": MODEL_TEXT["grin"],
                         "counted_work": roofline_of(counted, ms / 1e3, peak32),
                         "peak_basis": "152 SM x 128 FFMA/clk x 2 flop at the sampled clock"},
            "max_abs_D": rays.d_max.max().item(),
            "parity": "<= 1e-4 relative to the FP64 oracle on the same FP32-rounded launch states "
                      "(tests/test_gpu_rk4.py)"}


def measure_generated(gf, torch, n_rays: int, n_steps: int) -> dict:
    """The GRIN + 16 blob medium written symbolically and compiled at run time
    (the paper's route: graph, df, reduce, generated kernel) against the
    hand-written FP64 kernel, same rays and steps."""
    from paper_2508_15967_gb300 import symbolic as S
    wl = W.grin(n=n_rays, n_steps=n_steps)
    D = S.isotropic(S.grin_n2(1.5, 2.0) + S.gaussian_blobs(wl.medium["blobs"]))
    t0 = time.perf_counter()
    mg = gf.gf_jit_medium_create(S.medium_source(D))
    jit_s = time.perf_counter() - t0
    mh = gf.gf_medium_create(**wl.medium)
    init = gf.Rays.from_numpy(wl.x0, None)
    gf.gf_rays_onshell(mh, init, torch.from_numpy(np.ascontiguousarray(wl.d.T)).cuda(), 1.0)
    out = {}
    for name, m in (("generated", mg), ("handwritten", mh)):
        for _ in range(2):
            rays = init.clone()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            gf.gf_trace_rk4(m, rays, 1.0, wl.dt, wl.n_steps)
            e1.record()
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out[name] = {"ms": ms, "ray_steps_per_s": wl.n * wl.n_steps / (ms / 1e3), "y": rays.y.clone()}
    dev = ((out["generated"].pop("y") - out["handwritten"].pop("y")).abs().max()).item()
    return {"workload": f"GRIN + 16 blobs, {wl.n} rays x {wl.n_steps} RK4 steps, FP64",
            "generated": out["generated"], "handwritten": out["handwritten"],
            "nvrtc_compile_s": jit_s, "graph_nodes": S.count_nodes(S.gradients(D)),
            "max_abs_state_difference": dev}


def measure_adjoint(gf, torch, n: int | None = None, n_steps: int | None = None, peak: float | None = None,
                    morton: bool = True, shard: int = 0, ray_range: tuple[int, int] | None = None,
                    allreduce=None, barrier=None) -> dict:
    """Adjoint workload (65,536 rays, Luneburg + 64 blobs, RK4 dt 1e-3 x 4000,
    checkpoints every 64; n and n_steps shrink it): forward with checkpoints
    and backward through the autograd Function, plus a plain forward, each
    timed after a warm-up.  ray_range = (lo, hi) traces only those rays (a
    strong-scaling shard); allreduce(grad) sums the parameter gradient over
    the ranks inside the timed backward."""
    peak = fp64_peak_tflops(2070.0) if peak is None else peak
    wl = W.adjoint(**({} if n is None else {"n": n}), **({} if n_steps is None else {"n_steps": n_steps}),
                   morton=morton, shard=shard)
    if ray_range is not None:
        wl.x0, wl.d = wl.x0[ray_range[0]:ray_range[1]], wl.d[ray_range[0]:ray_range[1]]
    m = gf.gf_medium_create(**wl.medium)
    init = gf.Rays.empty(wl.n)
    init.y[:3].copy_(torch.from_numpy(np.ascontiguousarray(wl.x0.T)).cuda())
    gf.gf_rays_onshell(m, init, torch.from_numpy(np.ascontiguousarray(wl.d.T)).cuda(), 1.0)
    y0 = init.y.clone()
    # targets: the same rays traced with the hidden amplitudes theta*
    gf.gf_medium_set_amplitudes(m, torch.tensor(wl.extra["theta_star"], device="cuda"))
    star = gf.Rays.empty(wl.n, diagnostics=False)
    star.y.copy_(y0)
    gf.gf_trace_rk4(m, star, 1.0, wl.dt, wl.n_steps)
    xstar = star.y[:3].clone()
    theta = torch.tensor(wl.extra["theta"], device="cuda", requires_grad=True)
    gf.gf_medium_set_amplitudes(m, theta.detach())
    every = wl.extra["checkpoint_every"]
    ev = lambda: torch.cuda.Event(enable_timing=True)
    res = {}
    for it in range(2):
        if it == 1 and barrier is not None:
            barrier()
        e0, e1, e2, e3, e4 = ev(), ev(), ev(), ev(), ev()
        e0.record()
        plain = gf.Rays.empty(wl.n, diagnostics=False)
        plain.y.copy_(y0)
        gf.gf_trace_rk4(m, plain, 1.0, wl.dt, wl.n_steps)
        e1.record()
        yN = gf.trace_rk4_autograd(m, theta, y0, 1.0, wl.dt, wl.n_steps, every)
        e2.record()
        loss = ((yN[:3] - xstar) ** 2).sum()
        e3.record()
        loss.backward()
        if allreduce is not None:
            allreduce(theta.grad)
        e4.record()
        torch.cuda.synchronize()
        res = {"plain_forward_ms": e0.elapsed_time(e1), "forward_ckpt_ms": e1.elapsed_time(e2),
               "backward_ms": e3.elapsed_time(e4)}
        grad = theta.grad.clone()
        theta.grad = None
    res["backward_over_forward"] = res["backward_ms"] / res["forward_ckpt_ms"]
    res["total_over_plain_forward"] = (res["forward_ckpt_ms"] + res["backward_ms"]) / res["plain_forward_ms"]
    # the gradient's throughput: ray-steps of the trace per second of forward + backward
    units = wl.n * wl.n_steps
    res["gradient_ray_steps_per_s"] = units / ((res["forward_ckpt_ms"] + res["backward_ms"]) / 1e3)
    res["roofline"] = {
        "forward": roofline_of(MODEL_ADJ_FWD_RAY_STEP * units, res["plain_forward_ms"] / 1e3, peak),
        "forward_ckpt": roofline_of(MODEL_ADJ_FWD_RAY_STEP * units, res["forward_ckpt_ms"] / 1e3, peak),
        # the backward's FP64 work is the recomputation (the forward's flops); its reverse sweep
        # (vector-Jacobian products, MODEL_ADJ_BWD_RAY_STEP - MODEL_ADJ_FWD_RAY_STEP flops per
        # ray-step algorithmically) runs in double-float on the FP32 pipes
        "backward_fp64_recomputation": roofline_of(MODEL_ADJ_FWD_RAY_STEP * units, res["backward_ms"] / 1e3, peak),
        "model": {"forward": MODEL_TEXT["adj_fwd"], "backward": MODEL_TEXT["adj_bwd"]},
        "peak_tflops": peak}
    # untimed backward with work counters: recomputed evaluations and blob terms, swept blob
    # terms, and recomputed segment ends that differ from the forward trace's checkpoints
    yN = gf.trace_rk4_autograd(m, theta, y0, 1.0, wl.dt, wl.n_steps, every)
    counters = torch.zeros(4, dtype=torch.int64, device="cuda")
    gf.gf_bench_set_counters(counters)
    try:
        ((yN[:3] - xstar) ** 2).sum().backward()
        torch.cuda.synchronize()
    finally:
        gf.gf_bench_set_counters(None)
    c = [int(v) for v in counters.tolist()]
    theta.grad = None
    res["backward_work"] = {"recomputed_evaluations": c[0], "recomputed_blob_terms": c[1],
                            "swept_blob_terms": c[2], "segment_ends_differing_from_checkpoints": c[3],
                            "note": "the sweep's blob terms run in double-float on the FP32 pipes"}
    res["scratch_bytes"] = gf.gf_adjoint_scratch_bytes(m, wl.n, every)
    res["loss"] = loss.item()
    res["grad_norm"] = float(grad.norm().item())
    order = "Morton order" if morton else "drawn order"
    res["workload"] = (f"{wl.n} rays ({order}), Luneburg + {len(wl.extra['theta'])} blobs, RK4 dt={wl.dt} x "
                       f"{wl.n_steps}, checkpoint every {every}")
    return res


def run_gpu(a):
    import torch
    import torch.distributed as dist
    import paper_2508_15967_gb300 as gf

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    dtype = torch.float32 if a.precision == "f32" else torch.float64
    prec = {"f64": gf.GF_F64, "f32": gf.GF_F32, "f64x": gf.GF_F64X}[a.precision]
    from paper_2508_15967_gb300.shard import ray_share
    seed_shard, r_lo, r_hi = ray_share(a.scaling, a.rays, rank, world)
    wl = W.grin(n=a.rays, n_steps=a.nsteps, shard=seed_shard)
    wl.x0, wl.d = wl.x0[r_lo:r_hi], wl.d[r_lo:r_hi]
    m = gf.gf_medium_create(**wl.medium)
    x0 = torch.from_numpy(np.ascontiguousarray(wl.x0.T)).to("cuda", dtype)
    dirs = torch.from_numpy(np.ascontiguousarray(wl.d.T)).to("cuda", dtype)
    rays = gf.Rays.empty(wl.n, dtype)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def reset():
        rays.y[:3].copy_(x0)
        rays.t.zero_()
        rays.status.zero_()
        rays.steps.zero_()
        rays.d_max.zero_()

    def step(k_ev=None):
        reset()
        gf.gf_rays_onshell(m, rays, dirs, wl.omega)
        if k_ev:
            k_ev[0].record(stream)
        gf.gf_trace_rk4(m, rays, wl.omega, wl.dt, wl.n_steps, precision=prec)
        if k_ev:
            k_ev[1].record(stream)

    # measured FMA peaks (informational; the roofline peak is derived below)
    fma64, _ = gf.gf_bench_fma_peak(gf.GF_F64, 1 << 15, 4)
    fma32, _ = gf.gf_bench_fma_peak(gf.GF_F32, 1 << 18, 8)

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    units_per_step = int(rays.steps.to(torch.int64).sum().item())

    clocks = ClockSampler(local)
    clocks.start()
    starts, ends, kev = [ev() for _ in range(a.steps)], [ev() for _ in range(a.steps)], []
    barrier()
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    for k in range(a.steps):
        flush.zero_()                                  # L2 flush between timed steps
        starts[k].record(stream)
        kk = (ev(), ev())
        step(kk)
        kev.append(kk)
        ends[k].record(stream)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - w0
    clk = clocks.stop()
    units = int(rays.steps.to(torch.int64).sum().item())
    assert units == units_per_step, "step counts changed between steps"
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    kern_ms = [s.elapsed_time(e) for s, e in kev]
    t_dev = sum(step_ms) / 1e3
    t_max = torch.tensor([t_dev], dtype=torch.float64, device="cuda")
    units_all = torch.tensor([units], dtype=torch.int64, device="cuda")   # ray-steps of one trace, all ranks
    if world > 1:
        dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
        dist.all_reduce(units_all, op=dist.ReduceOp.SUM)
    t_max = t_max.item()
    units_all = int(units_all.item())
    value = units_all * a.steps / t_max

    # end to end through the public API with host buffers (pinned), copies timed
    e2e = None
    if not a.no_e2e:
        x0_h = torch.from_numpy(np.ascontiguousarray(wl.x0.T)).to(dtype).pin_memory()
        d_h = torch.from_numpy(np.ascontiguousarray(wl.d.T)).to(dtype).pin_memory()
        out = {k: torch.empty_like(v, device="cpu").pin_memory() for k, v in
               dict(y=rays.y, t=rays.t, status=rays.status, steps=rays.steps,
                    d_res=rays.d_res, d_max=rays.d_max).items()}
        h2d = x0_h.numel() * x0_h.element_size() + d_h.numel() * d_h.element_size()
        d2h = sum(v.numel() * v.element_size() for v in out.values())
        barrier()
        torch.cuda.synchronize()
        e0 = time.perf_counter()
        for _ in range(a.steps):
            gf.trace_host(m, x0_h, d_h, wl.omega, wl.dt, wl.n_steps, rays, dirs, out, precision=prec)
        torch.cuda.synchronize()
        barrier()
        te = torch.tensor([time.perf_counter() - e0], dtype=torch.float64, device="cuda")
        if world > 1:
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
        e2e = {"value": units_all * a.steps / te.item(), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # exact work of one trace launch (untimed pass with counters)
    counters = torch.zeros(2, dtype=torch.int64, device="cuda")
    gf.gf_bench_set_counters(counters)
    step()
    torch.cuda.synchronize()
    gf.gf_bench_set_counters(None)
    evals, live = (int(v) for v in counters.tolist())
    n_blobs = wl.medium["blobs"].shape[0]
    flops = algorithmic_flops(evals, live, n_blobs, units)
    model_flops = MODEL_GRIN_RAY_STEP * units
    k_sec = statistics.mean(kern_ms) / 1e3
    achieved = model_flops / k_sec / 1e12
    achieved_counted = flops / k_sec / 1e12
    sm_mhz = (clk or {}).get("sm_mhz") or 2070.0
    # non-tensor peaks from unit counts and clock: 152 SMs x 2 DFMA/clk (FP64) or
    # 128 FFMA/clk (FP32) x 2 flops
    peak64 = fp64_peak_tflops(sm_mhz)
    peak32 = fp32_peak_tflops(sm_mhz)
    peak = peak64 if dtype == torch.float64 else peak32
    basis = (f"152 SM x 2 DFMA/clk x 2 flop x {sm_mhz:.0f} MHz (sampled)" if dtype == torch.float64
             else f"152 SM x 128 FFMA/clk x 2 flop x {sm_mhz:.0f} MHz (sampled)")
    kname = {"f64": "rk4_kernel<double, GRIN>", "f32": "rk4_kernel<float, GRIN>",
             "f64x": "rk4_kernel<double, GRIN, double-float blob sums>"}[a.precision]
    metric = {"f64": METRIC, "f32": METRIC.replace("FP64", "FP32"),
              "f64x": METRIC.replace("FP64", "FP64 state / double-float blob sums")}[a.precision]
    line = {
        "metric": metric, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": 1e3 * t_max / a.steps, "higher_is_better": True,
        "scaling": a.scaling, "vs_baseline": None,
        "dtype": {"f64": "f64", "f32": "f32", "f64x": "f64 state, f32x2 blob sums"}[a.precision],
        "data": "synthetic",
        "config": {"workload": f"grin_fibre_16_blobs rays={a.rays} rk4_steps={wl.n_steps} dt={wl.dt}",
                   "rays_per_gpu": wl.n, "rk4_steps": wl.n_steps,
                   "parallelism": f"ray shards x{world} ({a.scaling} scaling)",
                   "l2": "256 MiB buffer written between timed steps"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "model": MODEL_TEXT["grin"],
                     "flops_per_launch": model_flops,
                     "traffic": TRAFFIC_BYTES_1M if (wl.n == 1 << 20 and a.precision == "f64") else None,
                     "kernel": kname, "kernel_ms": 1e3 * k_sec,
                     "counted_work": {"achieved": achieved_counted, "frac": achieved_counted / peak,
                                      "flops_per_launch": flops,
                                      "model": "live blob term 18 (the table exponential takes no FP64 flop), culled term 9, "
                                               "evaluation 51, ray-step 18, from the kernel's work counters"},
                     "evaluations": evals, "blob_terms_live": live,
                     "blob_terms_total": evals * n_blobs,
                     "peak_basis": basis,
                     "fma_peak_measured_tflops": {"f64": fma64, "f32": fma32}},
        "clocks": clk, "gpu_launches": 2 * a.steps, "e2e": e2e, "wall_s": wall,
    }
    if a.precision == "f64":
        line["roofline"]["note"] = ("the FP64 pipe retires fewer operations than the model counts: the blob "
                                    "exponent |u|^2 (integer fixed point), the exponential (float pairs and "
                                    "integers), the negligible-term pre-test and the reciprocal seed run on the "
                                    "integer and FP32 pipes; ncu on this launch shape: FP64 pipe 92.6% busy, "
                                    "~471 FP64 instructions per ray-step in the first 20 steps")
    if a.precision == "f64x":
        line["roofline"]["note"] = ("the blob terms run in double-float on the FP32 pipes, so the FP64-flop "
                                    "count exceeds the FP64 peak; the mode is bound by instruction issue")
    if world == 1 and not a.no_extras:
        if a.precision == "f64":
            line["f64x"] = measure_f64x(gf, torch, wl, m, x0, dirs, rays)
            line["f32"] = measure_f32(gf, torch, wl, m, peak32)
        line["luneburg"] = measure_luneburg(gf, torch)
        line["cold"] = measure_cold(gf, torch, peak64)
        line["aniso"] = measure_aniso(gf, torch, peak64)
        line["adjoint"] = measure_adjoint(gf, torch, peak=peak64)
        line["batched"] = measure_batched(gf, torch, peak=peak64)
        if rank == 0 and not a.no_cpu_baseline:
            for name in ("luneburg", "cold", "aniso", "adjoint", "batched"):
                _with_oracle(line[name], name)
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cb = oracle_throughput(W.grin(n=a.cpu_rays, n_steps=a.nsteps), a.cpu_rays)
        cb.pop("seconds")
        line["cpu_baseline"] = cb
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_workload(a):
    """One secondary measurement as a JSON line.  batched and adjoint also run
    data-parallel under torchrun (one rank per GPU): weak scaling gives every
    rank its own batch of the workload's size, strong scaling splits one batch
    (media balanced on ray counts, or ray ranges); the adjoint's one exchange
    is the all-reduce of the parameter gradient (NCCL), inside the timed
    backward; the job's time is the slowest rank's."""
    import torch
    import torch.distributed as dist
    import paper_2508_15967_gb300 as gf
    from paper_2508_15967_gb300.shard import allreduce_gradient, max_over_ranks, media_share, ray_share

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    if world > 1:
        if a.workload not in ("batched", "adjoint"):
            raise SystemExit(f"--workload {a.workload} runs on one GPU; batched and adjoint run data-parallel")
        dist.init_process_group("nccl", device_id=torch.device("cuda", torch.cuda.current_device()))
    barrier = (lambda: dist.barrier()) if world > 1 else None
    peak = fp64_peak_tflops(2070.0)
    morton = not a.drawn_order
    if a.workload == "batched":
        off = W.batched(n_media=a.media).extra["offsets"]
        seed_shard, m_lo, m_hi = media_share(a.scaling, off, rank, world)
        res = measure_batched(gf, torch, tune_cache=a.tune_cache, n_media=a.media, peak=peak, morton=morton,
                              shard=seed_shard, media_range=(m_lo, m_hi), full=world == 1, barrier=barrier)
        if world > 1:
            p = res["persistent"]
            t = max_over_ranks(p["ms"] / 1e3, "cuda")
            tot = torch.tensor([p["accepted_ray_steps"], p["rejected"]], dtype=torch.int64, device="cuda")
            dist.all_reduce(tot)
            acc, rej = (int(v) for v in tot.tolist())
            res = {"metric": "accepted ray-steps/s, batched DOPRI5 (persistent launch)",
                   "value": acc / t, "unit": "accepted ray-steps/s", "n_gpus": world, "scaling": a.scaling,
                   "ms": 1e3 * t, "accepted_ray_steps": acc, "rejected": rej,
                   **roofline_of(MODEL_DOPRI5_ATTEMPT * (acc + rej), t, peak * world),
                   "roofline_model": MODEL_TEXT["dopri5"], "rank0": res}
    elif a.workload == "luneburg":
        res = measure_luneburg(gf, torch)
    elif a.workload == "cold":
        res = measure_cold(gf, torch, peak, a.rays, a.nsteps)
    elif a.workload == "aniso":
        full = inspect.signature(W.aniso).parameters["n_steps"].default
        res = measure_aniso(gf, torch, peak, min(a.nsteps, full))
    elif a.workload == "adjoint":
        d = inspect.signature(W.adjoint).parameters
        n = min(a.rays, d["n"].default)
        seed_shard, lo, hi = ray_share(a.scaling, n, rank, world)
        res = measure_adjoint(gf, torch, n, min(a.nsteps, d["n_steps"].default), peak=peak, morton=morton,
                              shard=seed_shard, ray_range=(lo, hi),
                              allreduce=allreduce_gradient if world > 1 else None, barrier=barrier)
        if world > 1:
            t = max_over_ranks((res["forward_ckpt_ms"] + res["backward_ms"]) / 1e3, "cuda")
            units = torch.tensor([(hi - lo) * min(a.nsteps, d["n_steps"].default)], dtype=torch.int64,
                                 device="cuda")
            dist.all_reduce(units)
            res = {"metric": "gradient ray-steps/s (forward with checkpoints + backward + gradient all-reduce)",
                   "value": int(units.item()) / t, "unit": "gradient ray-steps/s", "n_gpus": world,
                   "scaling": a.scaling, "ms": 1e3 * t, "rank0": res}
    else:
        res = measure_generated(gf, torch, min(a.rays, 1 << 18), min(a.nsteps, 2000))
    if world == 1 and a.workload in ("luneburg", "cold", "aniso", "adjoint", "batched") and not a.no_cpu_baseline:
        _with_oracle(res, a.workload)
    if rank == 0:
        print(json.dumps({"workload": a.workload, **res}), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload != "grin":
        run_workload(a)
    else:
        run_gpu(a)


if __name__ == "__main__":
    main()
