"""Benchmark of the WFP time march on GB300: scatterer-steps per second (M * steps / s).

Workload (headline): the million-spring clustered layout in the periodic box (16 Gaussian clusters
of width 0.05 plus 20 % uniform springs, stiffnesses uniform in [1, 10]), incident Gaussian of width
0.1 at x = -2, dt = 5e-4 (K = 6283 modes), tol = 1e-10 (W = 30), p = 8, four receivers; seeded
synthetic input (`workloads.config2`).  Its 1.3e10 pairs closer than delta and its 931,311-spring
block of pairs closer than dt fit no stored-weight plan, so the plan is the one without pair lists
(opts.local_weights = 1).  One step = one pass of the whole hot path: local sum, type-1 NUFFT, mode
update, type-2 NUFFT, implicit solve, receivers.

Timing: W untimed warm-up steps, then exactly K steps of one `wave1d_solve` call timed with CUDA
events on the caller's stream (the plan's work is stream-ordered on it).  Inputs are resident and
larger than the L2 (every step reads 3.6 GB of implicit-part weights and the 0.84 GB density rings).
Beside it: the per-stage times of K profiled steps (the roofline of the local sum), the end-to-end
rate through the public API with host buffers, the free-space M = 1e4 workload as a secondary
measurement, the forms beside FP64, and the CPU oracle on a bounded sample with the GPU's error
against it.  Under torchrun every rank marches its own replica; the timed region is bracketed by
barriers and the slowest rank's time is reported.

`--impl reference` times the plain CPU oracle of the same scheme (oracle/wfp.py) on the host
cores, on a bounded sample of the workload, one oracle time step per bench step.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "scatterer-steps/s (M*N_t/s) at stated error vs FP64 oracle; % of HBM roofline"
UNIT = "scatterer-steps/s"
L2_FLUSH_BYTES = 512 << 20
# DRAM bytes (read + write) of one k_step launch at this workload, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum), valid only for the kernel sources it was taken
# with: reported as roofline.traffic while their SHA-256 matches, else null
STEP_KERNEL_SOURCES = ["step.cu", "grid_sync.cuh", "phases.cuh", "device_common.cuh", "internal.h"]
STEP_TRAFFIC = {"sources_sha256": "0453b92af3711282c1935bfbfe99074ca9290f375d132ba9ff09e97526413ac9", "bytes_per_launch": 316612437 + 4545109}
L2_CLEAN_BYTES = 256 << 20
# DRAM bytes of one k_rs_local launch from one ncu capture of the clustered layout at M = 2e5 (its
# pairs below), for the kernel sources it was taken with (null once they change)
RS_LOCAL_SOURCES = ["range.cu", "range.cuh", "phases.cuh", "device_common.cuh", "internal.h"]
RS_LOCAL_TRAFFIC = {"sources_sha256": "3b8b29ccbe01c9db3548bd9b08fc635e68d5ec064449b29392f4d5ef30967b2e", "bytes_per_launch": 71751168.0, "pairs": 2935880666}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def max_over_ranks(value, device):
    """The largest of a per-rank number over the ranks of the default process group (the number
    itself when no group is initialised or it has one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(M, steps, world, ms):
    """Whole-job scatterer-steps/s: every rank marches M springs for `steps` steps; `ms` is the
    slowest rank's time."""
    return M * steps * world / (ms * 1e-3)


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        out_dir = os.path.join(ROOT, "paper_2507_07823_gb300", "_build")      # git-ignored
        os.makedirs(out_dir, exist_ok=True)
        self.path = os.path.join(out_dir, f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "10"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            # the timed region is short: start it only once the sampler is writing
            t_end = time.time() + 5.0
            while time.time() < t_end and os.path.getsize(self.path) == 0:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            return out
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [c.strip() for c in r]
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except Exception:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if sm:
            out.update(sm_mhz=float(np.median(sm)), sm_max_mhz=float(max(mx)), samples=len(sm))
        out["reasons"] = sorted(reasons)
        try:
            os.remove(self.path)
        except OSError:
            pass
        return out


def run_ours(args):
    import torch

    from paper_2507_07823_gb300 import build, wave1d, workloads

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    w = workloads.config2()
    K, Wm = args.steps, args.warmup
    assert Wm >= 3
    stream = torch.cuda.current_stream()
    t_plan = time.perf_counter()
    plan = wave1d.Plan.from_workload(w.with_(Nt=Wm + 3 * K + 8), stream=stream.cuda_stream, local_weights=1)
    t_plan = time.perf_counter() - t_plan
    info = plan.info
    for _ in range(Wm):
        plan.step()
    torch.cuda.synchronize()

    # --- device-timed march: exactly K steps of one wave1d_solve call (inputs resident; every step
    # reads the 3.6 GB of implicit-part weights and 0.84 GB of density rings, far more than L2) -----
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        e0.record(stream)
        wave1d._check(wave1d.wave1d_solve(plan.h, K, None, None, 1), "wave1d_solve")
        e1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    ms_total = max_over_ranks(e0.elapsed_time(e1), "cuda")
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    value = replica_throughput(w.M, K, world, ms_total)
    launches = K * range_launches_per_step(w)

    # --- per-stage device times (CUDA events between the stages, K steps): the local-sum stage is
    # exactly one launch of k_rs_local, which gives its per-launch time for the roofline ---------
    wave1d.wave1d_profile(plan.h, 1)
    for i in range(K):
        wave1d._check(wave1d.wave1d_step(plan.h), "wave1d_step")
    stage_ms, nprof = wave1d.wave1d_profile_read(plan.h)
    wave1d.wave1d_profile(plan.h, 0)
    per_step = {s: float(stage_ms[i] / nprof) for i, s in enumerate(wave1d.STAGES)}

    # --- end to end through the public API with host buffers: forcing g_j(t_{n+1}) from pinned host
    # memory every step, the densities back to pinned host memory every step ----------------------
    cur = wave1d.wave1d_get_info(plan.h).n
    g_host = torch.empty((K, w.M), dtype=torch.float64, pin_memory=True)
    tt = (cur + 1 + np.arange(K)) * w.dt
    g_host.numpy()[:] = w.beta[None, :] * periodic_gaussians(w, tt)
    out_host = torch.empty((K, w.M), dtype=torch.float64, pin_memory=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(K):
        wave1d._check(wave1d.wave1d_step(plan.h, g_host[i].numpy(), 0), "wave1d_step")
        wave1d._check(wave1d.wave1d_get_sigma(plan.h, out_host[i].numpy(), 0), "wave1d_get_sigma")
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_value = w.M * K * world / e2e_s
    plan.close()

    # --- roofline of the dominant kernel, k_rs_local: bound by FP32 issue, not by HBM.  Algorithmic
    # work per launch: the local sum's multiply-adds Q_m(d) sigma (info.local_terms, 2 flops each),
    # the work the method does whatever the arithmetic; peak: 152 SMs x 128 FP32 lanes x 2 flops x
    # the maximum SM clock.
    fp32_peak, clk_src = _fp32_peak()
    ms_local = per_step["local"]
    achieved = 2.0 * info.local_terms / (ms_local * 1e-3) / 1e12
    roof = {"kernel": "k_rs_local", "bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
            "frac": achieved / fp32_peak, "traffic": rs_local_traffic(info),
            "peak_source": f"derived: 152 SMs x 128 FP32 lanes x 2 flops x {clk_src}",
            "algorithmic_flops_per_launch": 2.0 * info.local_terms, "launch_ms": ms_local,
            "local_pairs": info.local_pairs, "local_terms": info.local_terms,
            "pairs_per_s": info.local_pairs / (ms_local * 1e-3),
            "timing": "CUDA events around the local-sum stage (one k_rs_local launch) of K profiled steps",
            "arithmetic": "compensated FP32 pairs (about 48 significant bits); 2 flops per term counts only the "
                          "multiply-add of the method, not the compensation or the weights' polynomials"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": Wm, "ms_per_step": ms_total / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32x2+f64", "data": "synthetic",
        "config": {"workload": f"{w.name}: {w.description}", "M": w.M, "dt": w.dt, "tol": w.tol, "p": w.p,
                   "K": info.K, "W": info.W, "nufft_w": info.nufft_w, "nf": info.nf,
                   "local_pairs": info.local_pairs, "nearby_pairs": info.nearby_pairs,
                   "plan": "local_weights = 1: no pair lists (local sum over sorted index windows with "
                           "weights from distance polynomials, implicit part by Jacobi sweeps)",
                   "arithmetic": "local sum in compensated FP32 pairs (k_rs_local); history part (NUFFTs, "
                                 "FFTs, mode recurrence), implicit solve and receivers in FP64",
                   "parallelism": f"replicas x{world}",
                   "l2": "not flushed: every step reads the 3.6 GB of implicit-part weights and the 0.84 GB "
                         "density rings, far more than the 126 MB L2",
                   "timed": f"one wave1d_solve of {K} steps after {Wm} warm-up steps",
                   "plan_seconds": t_plan},
        "stage_ms_per_step": per_step,
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * w.M,
                "d2h_bytes_per_step": 8 * w.M},
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "wall_s_timed_region": wall,
    }
    if world == 1 and not args.no_secondary:
        try:
            line["free_M1e4"] = free_space_secondary(torch, stream)
        except Exception as e:                               # recorded, never fatal to the line
            line["free_M1e4"] = {"error": repr(e)[:300]}
    if not args.no_spread_interp:
        hbm, _ = _peaks()
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        clean = torch.ones(L2_CLEAN_BYTES // 4, dtype=torch.float32, device="cuda")

        def flush_l2():
            flush.zero_()
            clean.sum()

        line["spread_interp_M1e6"] = spread_interp_million(torch, stream, flush_l2, hbm)
        line["spread_interp_batched"] = spread_interp_batched(torch, stream, flush_l2, hbm)
    if world == 1 and not args.no_forms:
        try:
            line["forms_beside_fp64"] = forms_beside_fp64(torch, w, K)
        except Exception as e:                               # recorded, never fatal to the line
            line["forms_beside_fp64"] = {"error": repr(e)[:300]}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_steps)
        line["error_vs_oracle"] = error_vs_oracle()
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def range_launches_per_step(w):
    """Kernel launches of one step of a plan without pair lists: the local sum, five history-part
    launches (spreading + FFT columns, FIR tail, FFT rows + mode update, inverse FFT columns,
    interpolation), the solve's set-up, its 40 Jacobi sweep launches (those after convergence return
    at once), the store, the receivers' local part (with receivers) and the finishing launch."""
    return 1 + 5 + 1 + 40 + 1 + (1 if len(w.xr) else 0) + 1


def periodic_gaussians(w, tt):
    """f(x_j - t) for times tt (rows), periodised over 2 pi (images |m| <= 2)."""
    f = np.zeros((len(tt), w.M))
    for a, c, wd in zip(w.amp, w.center, w.width):
        for mimg in range(-2, 3):
            f += a * np.exp(-0.5 * ((w.x[None, :] - tt[:, None] + 2 * math.pi * mimg - c) / wd) ** 2)
    return f


def _fp32_peak():
    """FP32 FMA peak (TFLOP/s) of 152 SMs x 128 lanes x 2 flops at the measured maximum SM clock."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f)["sm_max_mhz"])
        src = f"{mhz:.0f} MHz (MEASURED_PEAKS.json sm_max_mhz)"
    except Exception:
        mhz, src = 2070.0, "2070 MHz (nominal maximum)"
    return 152 * 128 * 2 * mhz * 1e6 / 1e12, src


def free_space_secondary(torch, stream):
    """The free-space workload (M = 1e4 uniform, beta log-uniform in [0.1, 100], three pulses,
    dt = 1e-3, tol = 1e-12) with stored weights: one chunk of rbc_period steps through wave1d_solve,
    from a chunk boundary, so the timed steps include one radiation projection step; and the
    one-launch step kernel's roofline (HBM: the stored weights it streams, L2 flushed before each
    single step)."""
    from paper_2507_07823_gb300 import wave1d, workloads
    w = workloads.config1()
    plan = wave1d.Plan.from_workload(w.with_(Nt=2000), stream=stream.cuda_stream)
    info = plan.info
    chunk = info.rbc_period
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    clean = torch.ones(L2_CLEAN_BYTES // 4, dtype=torch.float32, device="cuda")
    try:
        plan.solve(chunk, with_sigma=False)                  # warm-up, graph build, chunk-aligned
        torch.cuda.synchronize()
        reps = 3
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        wave1d._check(wave1d.wave1d_solve(plan.h, reps * chunk, None, None, 1), "wave1d_solve")
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / (reps * chunk)
        # the step kernel's per-launch time, L2 flushed before each single step (ordinary steps; the
        # first one untimed: it captures the single-step graph)
        wave1d._check(wave1d.wave1d_step(plan.h), "wave1d_step")
        torch.cuda.synchronize()
        ms_k = []
        for i in range(chunk - 2):
            flush.zero_()
            clean.sum()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            wave1d._check(wave1d.wave1d_step(plan.h), "wave1d_step")
            b.record(stream)
            torch.cuda.synchronize()
            ms_k.append(a.elapsed_time(b))
        hbm, peak_kind = _peaks()
        launch_ms = float(np.mean(ms_k))
        algo = 8 * info.local_terms
        achieved = algo / (launch_ms * 1e-3) / 1e9
    finally:
        plan.close()
    return {"workload": f"{w.name}: {w.description}", "value": w.M / (ms * 1e-3), "unit": UNIT,
            "ms_per_step": ms, "timed": f"{reps} chunks of {chunk} steps (each chunk: {chunk - 1} one-launch steps "
                                         "and one projection step of ten per-stage launches)",
            "roofline": {"kernel": "k_step", "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": step_traffic(),
                         "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                         "algorithmic_bytes_per_launch": algo,
                         "algorithmic": "8 B per stored weight Q_m (an FP32 pair), the stream the local sum must "
                                        "read once per step; padding, source lists and headers not counted",
                         "launch_ms": launch_ms, "launch_ms_median": float(np.median(ms_k)),
                         "launches_averaged": len(ms_k),
                         "timing": "single wave1d_step calls after one untimed, L2 flushed before each"}}


def rs_local_traffic(info):
    """DRAM bytes per k_rs_local launch at this workload, scaled by pairs from one ncu capture of a
    smaller clustered case (M = 2.5e5 in 4 clusters, the million-spring cluster density; the
    kernel's DRAM bytes are the window densities and positions it reads, which grow with the pairs),
    while the kernel sources match the ones it was taken with."""
    import hashlib
    h = hashlib.sha256()
    src = os.path.join(ROOT, "paper_2507_07823_gb300", "csrc")
    for f in RS_LOCAL_SOURCES:
        with open(os.path.join(src, f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest() != RS_LOCAL_TRAFFIC["sources_sha256"]:
        return None
    return RS_LOCAL_TRAFFIC["bytes_per_launch"] * info.local_pairs / RS_LOCAL_TRAFFIC["pairs"]


def spread_interp_million(torch, stream, flush_l2, hbm, reps=20):
    """A1 (spreading) and A6 (interpolation) alone at M = 1e6: the clustered periodic workload's
    positions, K = floor(pi / dt) = 6283, FP64 (tol 1e-10) and mixed (tol 1e-6).  Each pass is
    timed with events after an L2 flush (its inputs are smaller than L2).  Algorithmic bytes per
    step: 32 per spring (A1 reads a position and a density, A6 a position and writes u_H)."""
    from paper_2507_07823_gb300 import wave1d, workloads
    w2 = workloads.config2()
    K = int(np.floor(np.pi / w2.dt))
    out = {"workload": f"{w2.name}: {w2.description}", "M": w2.M, "K": K,
           "algorithmic_bytes": 32 * w2.M}
    for name, precision, tol in (("fp64", 0, 1e-10), ("mixed", 1, 1e-6)):
        nu = wave1d.Nufft(w2.x, K, tol, precision, stream=stream.cuda_stream)
        c = torch.rand(w2.M, dtype=torch.float64, device="cuda") + 0.5
        grid = torch.zeros(nu.nf, dtype=torch.float64, device="cuda")
        u = torch.zeros(w2.M, dtype=torch.float64, device="cuda")
        for _ in range(3):
            nu.spread(c, grid)
            nu.interp(grid, u)
        ts, ti = [], []
        for _ in range(reps):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            flush_l2()
            ev[0].record(stream)
            nu.spread(c, grid)
            ev[1].record(stream)
            flush_l2()
            ev[2].record(stream)
            nu.interp(grid, u)
            ev[3].record(stream)
            torch.cuda.synchronize()
            ts.append(ev[0].elapsed_time(ev[1]))
            ti.append(ev[2].elapsed_time(ev[3]))
        t_s, t_i = float(np.median(ts)), float(np.median(ti))
        achieved = 32 * w2.M / ((t_s + t_i) * 1e-3) / 1e9
        # bytes the implementation streams: cell index (4 B) and the density or u_H (8 B) per
        # point, plus 8 B per point and tap of FP64 weights, or a 4 B offset (mixed), per pass
        streamed = 2 * w2.M * (12 + (8 * nu.w if precision == 0 else 4))
        out[name] = {"tol": tol, "kernel_width": nu.w, "spread_us": 1e3 * t_s, "interp_us": 1e3 * t_i,
                     "achieved_GBps": achieved, "frac_of_hbm": achieved / hbm,
                     "streamed_bytes": streamed,
                     "streamed_GBps": streamed / ((t_s + t_i) * 1e-3) / 1e9,
                     "kernel": ("precomputed FP64 weights (8 B per point and tap read in each pass)"
                                if precision == 0 else
                                f"FP32 polynomials of degree {nu.degree} (max error {nu.kernel_err:.1e})")}
        nu.close()
    # Back-to-back passes, no flush: 12 point sets of the same recipe (other seeds) with their own
    # densities, spread one after another, then interpolated one after another; their inputs
    # (positions, offsets, densities, outputs: about 240 MB) exceed L2, so each pass reads its own
    # from DRAM, as the step's passes do between the local sum's weight streams.
    nsets = 12
    sets = [workloads.config2(seed=w2.seed + 1000 * (i + 1)) for i in range(nsets)]
    for name, precision, tol in (("fp64", 0, 1e-10), ("mixed", 1, 1e-6)):
        nus = [wave1d.Nufft(ws.x, K, tol, precision, stream=stream.cuda_stream) for ws in sets]
        cs = [torch.rand(w2.M, dtype=torch.float64, device="cuda") + 0.5 for _ in sets]
        grids = [torch.zeros(nus[0].nf, dtype=torch.float64, device="cuda") for _ in sets]
        us = [torch.zeros(w2.M, dtype=torch.float64, device="cuda") for _ in sets]
        for i in range(nsets):
            nus[i].spread(cs[i], grids[i])
            nus[i].interp(grids[i], us[i])
        best_s, best_i = [], []
        for _ in range(max(3, reps // 4)):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            flush_l2()
            ev[0].record(stream)
            for i in range(nsets):
                nus[i].spread(cs[i], grids[i])
            ev[1].record(stream)
            for i in range(nsets):
                nus[i].interp(grids[i], us[i])
            ev[2].record(stream)
            torch.cuda.synchronize()
            best_s.append(ev[0].elapsed_time(ev[1]) / nsets)
            best_i.append(ev[1].elapsed_time(ev[2]) / nsets)
        t_s, t_i = float(np.median(best_s)), float(np.median(best_i))
        achieved = 32 * w2.M / ((t_s + t_i) * 1e-3) / 1e9
        out[name]["back_to_back"] = {"point_sets": nsets, "spread_us": 1e3 * t_s, "interp_us": 1e3 * t_i,
                                     "achieved_GBps": achieved, "frac_of_hbm": achieved / hbm}
        for nu in nus:
            nu.close()
        del nus, cs, grids, us
    # the same event protocol around a plain device copy of 8 MB (16 MB of traffic, one pass's
    # algorithmic bytes): the ceiling of an isolated pass this small, launch and ramp included
    a = torch.rand(w2.M, dtype=torch.float64, device="cuda")
    b = torch.empty_like(a)
    tc = []
    for _ in range(reps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        flush_l2()
        ev[0].record(stream)
        b.copy_(a)
        ev[1].record(stream)
        torch.cuda.synchronize()
        tc.append(ev[0].elapsed_time(ev[1]))
    t_c = float(np.median(tc))
    out["copy_reference"] = {"bytes": 16 * w2.M, "us": 1e3 * t_c,
                             "frac_of_hbm": 16 * w2.M / (t_c * 1e-3) / 1e9 / hbm,
                             "what": "torch device copy of M doubles after the same L2 flush, one launch"}
    return out


def spread_interp_batched(torch, stream, flush_l2, hbm, reps=10):
    """A1 and A6 of the batched workload's instances (256 periodic instances, M log-uniform in
    [1e2, 1e5], dt = 1e-3: K = 3141) in one batched plan: one launch per pass over all instances,
    FP64 (tol 1e-12, as the workload) and mixed (tol 1e-6).  Each pass is timed with events after
    an L2 flush.  Algorithmic bytes: 32 per point (all instances)."""
    from paper_2507_07823_gb300 import wave1d, workloads
    inst = workloads.config3_instances()
    K = int(np.floor(np.pi / inst[0].dt))
    sets = [w.x for w in inst]
    Mtot = int(sum(v.size for v in sets))
    out = {"workload": f"{len(sets)} periodic instances, M log-uniform in [1e2, 1e5] (sum {Mtot}), K = {K}",
           "instances": len(sets), "M_total": Mtot, "K": K, "algorithmic_bytes": 32 * Mtot}
    for name, precision, tol in (("fp64", 0, 1e-12), ("mixed", 1, 1e-6)):
        t0 = time.perf_counter()
        nu = wave1d.Nufft(sets, K, tol, precision, stream=stream.cuda_stream)
        t_plan = time.perf_counter() - t0
        c = torch.rand(Mtot, dtype=torch.float64, device="cuda") + 0.5
        grid = torch.zeros(len(sets) * nu.nf, dtype=torch.float64, device="cuda")
        u = torch.zeros(Mtot, dtype=torch.float64, device="cuda")
        for _ in range(3):
            nu.spread(c, grid)
            nu.interp(grid, u)
        ts, ti = [], []
        for _ in range(reps):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            flush_l2()
            ev[0].record(stream)
            nu.spread(c, grid)
            ev[1].record(stream)
            flush_l2()
            ev[2].record(stream)
            nu.interp(grid, u)
            ev[3].record(stream)
            torch.cuda.synchronize()
            ts.append(ev[0].elapsed_time(ev[1]))
            ti.append(ev[2].elapsed_time(ev[3]))
        t_s, t_i = float(np.median(ts)), float(np.median(ti))
        achieved = 32 * Mtot / ((t_s + t_i) * 1e-3) / 1e9
        out[name] = {"tol": tol, "kernel_width": nu.w, "spread_us": 1e3 * t_s, "interp_us": 1e3 * t_i,
                     "achieved_GBps": achieved, "frac_of_hbm": achieved / hbm, "plan_seconds": t_plan}
        nu.close()
    return out


def forms_beside_fp64(torch, w, steps, warmup=3):
    """The forms beside the plain FP64 march, each timed with CUDA events on its own; a failure is
    recorded as a string, never fatal to the line.
      mixed_precision: the headline workload (a million clustered springs) with the history part's
        spreading and interpolation in FP32 (width-7 kernel, tol 1e-6), same plan otherwise; its
        error against the oracle is in error_vs_oracle.mixed.
      adjoint: the adjoint recipe at M = 1e4 with stored weights, both strategies and central
        differences on 8 stiffnesses (--adjoint-only adds M = 1e5 and 32 stiffnesses);
      batched: the batched workload's 256 instances (M up to 1e5), each instance's form chosen from
        its layout (joined in one launch per step, or its own plan without pair lists)."""
    from paper_2507_07823_gb300 import wave1d, workloads

    out = {}
    stream = torch.cuda.current_stream()

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    try:
        w6 = w.with_(tol=1e-6, Nt=warmup + steps)
        plan = wave1d.Plan.from_workload(w6, local_weights=1, precision=1)
        try:
            plan.solve(warmup, with_sigma=False)
            ms = timed(lambda: wave1d._check(wave1d.wave1d_solve(plan.h, steps, None, None, 1), "wave1d_solve"))
            out["mixed_precision"] = {"value": w.M * steps / (ms * 1e-3), "ms_per_step": ms / steps,
                                      "workload": f"{w.name} at tol 1e-6 (W = {plan.info.W}), FP32 spreading and "
                                                  f"interpolation, {steps} steps after {warmup}",
                                      "error_vs_oracle": "error_vs_oracle.mixed"}
        finally:
            plan.close()
    except Exception as e:
        out["mixed_precision"] = {"error": repr(e)[:300]}

    # adjoint: the adjoint workload's recipe at M = 1e4 (stored weights), 2000 steps, receivers at
    # the medium's entry and a seeded target trace; both strategies, and central differences of the
    # GPU march on 8 stiffnesses (32 in --adjoint-only)
    try:
        na = 2000
        wa = workloads.config4(M=10000, Nt=na)
        wa = wa.with_(xr=float(np.min(wa.x)) + 2 * wa.dt * np.arange(8))
        rng = np.random.default_rng(wa.seed)
        d = torch.from_numpy(0.01 * rng.standard_normal((na, len(wa.xr)))).cuda()
        holder = {}
        plan = wave1d.Plan.from_workload(wa)
        try:
            ms_f = timed(lambda: holder.update(zip(("sigma", "u"), plan.solve_device(na))))
            ms_a = timed(lambda: holder.update(g=plan.adjoint(holder["sigma"], holder["u"] - d)))
        finally:
            plan.close()
        del holder["sigma"]
        plan = wave1d.Plan.from_workload(wa)
        try:
            ms_cf = timed(lambda: holder.update(zip(("u2", "ck"), plan.solve_checkpointed(na, 100))))
            ms_ca = timed(lambda: holder.update(g2=plan.adjoint_checkpointed(holder["ck"], na, 100, holder["u2"] - d)))
        finally:
            plan.close()
        gh = holder["g"].cpu().numpy()
        fd_err = 0.0
        for j in np.random.default_rng(4).choice(wa.M, 8, replace=False):
            h = 1e-4 * wa.beta[j]
            Ls = []
            for sgn in (1.0, -1.0):
                bb = wa.beta.copy()
                bb[j] += sgn * h
                pl = wave1d.Plan.from_workload(wa.with_(beta=bb))
                try:
                    _, uu = pl.solve_device(na)
                    Ls.append(0.5 * float(torch.sum((uu - d) ** 2)))
                finally:
                    pl.close()
            fd_err = max(fd_err, abs((Ls[0] - Ls[1]) / (2 * h) - gh[j]))
        out["adjoint"] = {"forward_value": wa.M * na / (ms_f * 1e-3), "adjoint_value": wa.M * na / (ms_a * 1e-3),
                          "forward_ms_per_step": ms_f / na, "adjoint_ms_per_step": ms_a / na,
                          "checkpointed": {"interval": 100, "forward_ms_per_step": ms_cf / na,
                                           "adjoint_ms_per_step": ms_ca / na,
                                           "gradient_equal_bitwise": bool(torch.equal(holder["g"], holder["g2"]))},
                          "central_differences_8": {"max_abs_err_over_max_grad": fd_err / float(np.max(np.abs(gh)))},
                          "workload": f"{wa.name} recipe at M = 1e4 (stored weights), {na} steps, 8 receivers at the "
                                      "medium's entry, seeded target trace (M = 1e5 through the plan without pair "
                                      "lists: --adjoint-only)"}
    except Exception as e:
        out["adjoint"] = {"error": repr(e)[:300]}
    # batched: the batched workload's 256 instances (M up to 1e5), each instance's form chosen from
    # its layout: the small ones joined (one persistent launch), the large ones plans without pair
    # lists (concurrent branches of the step graph)
    try:
        nb = 10
        ws = workloads.config3_instances(Nt=3 + nb + 1)
        t0 = time.perf_counter()
        batch = wave1d.Batch(ws, local_weights=2)
        t_plan = time.perf_counter() - t0
        try:
            forms = batch.forms
            batch.solve(3, with_sigma=False)
            st = {}
            ms = timed(lambda: st.update(rc=wave1d.lib().wave1d_batch_solve(batch.h, nb, None, None, 1)))
            if st["rc"] != 0:
                raise RuntimeError(wave1d.lib().wave1d_batch_strerror().decode())
            out["batched"] = {"value": batch.M * nb / (ms * 1e-3), "ms_per_step": ms / nb, "M_total": batch.M,
                              "one_launch_joined": batch.one_launch, "plan_seconds": t_plan,
                              "instances_without_pair_lists": int(forms.sum()),
                              "workload": "256 periodic instances, M log-uniform in [1e2, 1e5], dt = 1e-3, tol 1e-12, "
                                          "p = 8, 10 steps after 3"}
        finally:
            batch.close()
    except Exception as e:
        out["batched"] = {"error": repr(e)[:300]}
    return out


def step_traffic():
    import hashlib
    h = hashlib.sha256()
    src = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2507_07823_gb300", "csrc")
    for f in STEP_KERNEL_SOURCES:
        with open(os.path.join(src, f), "rb") as fh:
            h.update(fh.read())
    return STEP_TRAFFIC["bytes_per_launch"] if h.hexdigest() == STEP_TRAFFIC["sources_sha256"] else None


def _oracle_sample():
    """A bounded sample of the million-spring workload for the CPU oracle: its 2000 springs of
    highest density (consecutive in position, inside one cluster, so every pair of them lies closer
    than delta), marched in the periodic box with the same dt, tol, p and pulse."""
    from paper_2507_07823_gb300 import workloads
    w = workloads.config2()
    xs = np.sort(w.x)
    n = 2000
    span = xs[n - 1:] - xs[:xs.size - n + 1]
    i = int(np.argmin(span))
    order = np.argsort(w.x, kind="stable")[i:i + n]
    return w.with_(x=w.x[order], beta=w.beta[order], xr=np.zeros(0), Nt=10_000), float(span[i])


def _cores():
    try:
        from threadpoolctl import threadpool_info
        return max([d.get("num_threads", 1) for d in threadpool_info()] + [1])
    except Exception:
        return os.cpu_count()


def cpu_baseline(nsteps):
    """The oracle of the same scheme (oracle/wfp.py, numpy/scipy FP64) timed on the host cores on a
    bounded sample of the workload (plan precompute excluded, as the paper excludes it)."""
    from oracle import wfp
    ws, span = _oracle_sample()
    o = wfp.from_workload(ws)
    for _ in range(3):
        o.step()
    t0 = time.perf_counter()
    for _ in range(nsteps):
        o.step()
    dt = time.perf_counter() - t0
    return {"value": ws.M * nsteps / dt, "unit": UNIT, "cores": _cores(), "kind": "oracle",
            "sample": f"{nsteps} time steps (after 3) of the {ws.M} most tightly packed springs of the "
                      f"million-spring workload (one cluster, span {span:.1e} < delta: every pair local), "
                      f"periodic, dt = {ws.dt}, tol = {ws.tol}, p = {ws.p}, oracle/wfp.py; plan excluded"}


def error_vs_oracle(nsteps=300):
    """Relative max error of the GPU march against the oracle over a whole march on a live sample of
    the workload's recipe: 3000 springs of the clustered layout (16 clusters of width 0.05 + 20 %
    uniform), dt = 5e-4, tol = 1e-10, p = 8, a pulse of width 0.005 that reaches springs within
    the first steps, receivers among them.  The FP64 plan without pair lists (the headline's) and
    the mixed form (tol 1e-6) against the oracle of each's tolerance."""
    from oracle import wfp
    from paper_2507_07823_gb300 import wave1d, workloads
    out = {"sample": f"clustered recipe at M = 3000, pulse width 0.005 at x = -2, {nsteps} steps, "
                     "receivers at -1.99, -1.97, -1.9, 2.5; relative max error over every step's densities "
                     "and receiver values"}
    for name, kw, tol in (("fp64", {}, 1e-10), ("mixed", {"precision": 1}, 1e-6)):
        w = workloads.config2(M=3000, Nt=nsteps, width=(0.005,), tol=tol).with_(xr=np.array([-1.99, -1.97, -1.9, 2.5]))
        plan = wave1d.Plan.from_workload(w, local_weights=1, **kw)
        try:
            s, u = plan.solve(nsteps)
        finally:
            plan.close()
        s_ref, u_ref = wfp.from_workload(w).run(nsteps)
        out[name] = {"tol": tol,
                     "sigma": float(np.max(np.abs(s - s_ref[1:])) / np.max(np.abs(s_ref))),
                     "u": float(np.max(np.abs(u - u_ref[1:])) / np.max(np.abs(u_ref))),
                     "max_abs_u": float(np.max(np.abs(u_ref)))}
    return out


def run_reference(args):
    rank, world, local = _dist()
    if rank != 0:
        return
    from oracle import wfp
    ws, span = _oracle_sample()
    o = wfp.from_workload(ws)
    for _ in range(args.warmup):
        o.step()
    K = min(args.steps, args.ref_max_steps)
    t0 = time.perf_counter()
    for _ in range(K):
        o.step()
    dt = time.perf_counter() - t0
    value = ws.M * K / dt
    from paper_2507_07823_gb300 import workloads
    w = workloads.config2()
    cb = {"value": value, "unit": UNIT, "cores": _cores(), "kind": "oracle",
          "sample": f"{K} oracle time steps (after {args.warmup}) of the {ws.M} most tightly packed springs "
                    f"of the million-spring workload (span {span:.1e} < delta), oracle/wfp.py, plan excluded"}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": K, "warmup": args.warmup, "ms_per_step": 1e3 * dt / K,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": f"{w.name}: {w.description}", "M": w.M,
                                            "sample_M": ws.M},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_spread_interp_only(args):
    """The M = 1e6 spreading / interpolation measurement alone (one JSON line), e.g. under ncu."""
    import torch

    from paper_2507_07823_gb300 import build

    build.build()
    hbm, _ = _peaks()
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    clean = torch.ones(L2_CLEAN_BYTES // 4, dtype=torch.float32, device="cuda")

    def flush_l2():
        flush.zero_()
        clean.sum()

    print(json.dumps({"spread_interp_M1e6": spread_interp_million(torch, stream, flush_l2, hbm,
                                                                   reps=args.spread_interp_reps),
                      "spread_interp_batched": spread_interp_batched(torch, stream, flush_l2, hbm,
                                                                     reps=args.spread_interp_reps)}))


def _adjoint_plan(wave1d, w, beta=None):
    b = w.beta if beta is None else beta
    return wave1d.Plan(w.x, b, w.bc, w.dt, w.Nt, w.tol, w.amp, w.center, w.width, w.xr, p=w.p,
                       max_local_bytes=64 << 30)


def adjoint_full_M(torch, wave1d, workloads, args):
    """The adjoint workload at its own M = 1e5 through the plan without pair lists (its one
    implicit block of every spring needs the iterative solve), over the stable horizon
    args.adjoint_full_steps (the scheme grows after about 2500 steps at this density): forward,
    reverse from the stored densities, and the checkpointed form (every args.adjoint_interval
    steps), which must give the same gradient bit for bit."""
    nsteps = args.adjoint_full_steps
    w = workloads.config4(Nt=nsteps)
    w = w.with_(xr=float(np.min(w.x)) + 2 * w.dt * np.arange(8))
    rng = np.random.default_rng(w.seed)
    d = torch.from_numpy(0.01 * rng.standard_normal((nsteps, len(w.xr)))).cuda()
    stream = torch.cuda.current_stream()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1)

    out = {"M": w.M, "steps": nsteps, "local_weights": "computed (plan without pair lists)"}
    try:
        plan = wave1d.Plan.from_workload(w, local_weights=1)
        (sigma, u), ms_f = timed(lambda: plan.solve_device(nsteps))
        g, ms_a = timed(lambda: plan.adjoint(sigma, u - d))
        plan.close()
        del sigma
        iv = args.adjoint_interval
        plan = wave1d.Plan.from_workload(w, local_weights=1)
        (u2, ck), ms_cf = timed(lambda: plan.solve_checkpointed(nsteps, iv))
        g2, ms_ca = timed(lambda: plan.adjoint_checkpointed(ck, nsteps, iv, u2 - d))
        plan.close()
        work = w.M * nsteps
        out.update({"forward_ms_per_step": ms_f / nsteps, "adjoint_ms_per_step": ms_a / nsteps,
                    "forward_value": work / (ms_f * 1e-3), "adjoint_value": work / (ms_a * 1e-3),
                    "checkpointed": {"interval": iv, "checkpoint_bytes": ck.numel(),
                                     "forward_ms_per_step": ms_cf / nsteps, "adjoint_ms_per_step": ms_ca / nsteps,
                                     "gradient_equal_bitwise": bool(torch.equal(g, g2))},
                    "grad_max": float(torch.max(torch.abs(g)))})
    except Exception as e:                                  # noqa: BLE001
        out["error"] = repr(e)[:300]
    return out


def run_adjoint_only(args):
    """The reverse-time march on the adjoint workload's recipe (free space, dt = 1e-3, tol = 1e-12,
    p = 8, beta ~ U[1, 10], 8 receivers): both strategies (stored densities, wave1d_adjoint; the
    march state checkpointed every `interval` steps and recomputed, wave1d_adjoint_checkpointed,
    which must give the same gradient bit for bit), and central differences of the loss
    L = 1/2 sum (u - d)^2 (d a seeded target trace) on 32 random stiffnesses, at --adjoint-M
    springs with stored weights; and, as `full_workload`, the workload's own M = 1e5 through the
    plan without pair lists over its stable horizon.  One JSON line; not part of the default
    benchmark line."""
    import torch

    from paper_2507_07823_gb300 import build, wave1d, workloads

    build.build()
    nsteps = args.adjoint_steps
    line = {"metric": "scatterer-steps/s of the reverse-time march (dL/dbeta)", "unit": "scatterer-steps/s",
            "dtype": "f64", "data": "synthetic"}
    line["full_workload"] = adjoint_full_M(torch, wave1d, workloads, args)
    w = workloads.config4(M=args.adjoint_M, Nt=nsteps)
    # the 8 receivers at the medium's entry, 2 dt apart: at this density the transmitted field is
    # localized within a few hundred springs, so receivers spread over the medium (the recipe's
    # default) see nothing within the march's stable horizon (about 2500 steps at M = 1e5)
    w = w.with_(xr=float(np.min(w.x)) + 2 * w.dt * np.arange(8))
    rng = np.random.default_rng(w.seed)
    d = torch.from_numpy(0.01 * rng.standard_normal((nsteps, len(w.xr)))).cuda()   # seeded target trace
    stream = torch.cuda.current_stream()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1)

    t0 = time.perf_counter()
    plan = _adjoint_plan(wave1d, w)
    t_plan = time.perf_counter() - t0
    info = plan.info
    (sigma, u), ms_fwd = timed(lambda: plan.solve_device(nsteps))
    ubar = u - d
    g, ms_adj = timed(lambda: plan.adjoint(sigma, ubar))
    loss = 0.5 * float(torch.sum(ubar ** 2))
    plan.close()
    del sigma
    interval = args.adjoint_interval
    plan = _adjoint_plan(wave1d, w)
    (u2, ckpt), ms_cfwd = timed(lambda: plan.solve_checkpointed(nsteps, interval))
    g2, ms_cadj = timed(lambda: plan.adjoint_checkpointed(ckpt, nsteps, interval, u2 - d))
    ckpt_bytes = ckpt.numel()
    plan.close()
    del ckpt
    # central differences of the forward march on 32 random stiffnesses (step 1e-4 beta_j)
    fd_rng = np.random.default_rng(4)
    idx = fd_rng.choice(w.M, args.adjoint_fd, replace=False)
    gh = g.cpu().numpy()
    fd_err = 0.0
    t0 = time.perf_counter()
    for j in idx:
        h = 1e-4 * w.beta[j]
        Ls = []
        for sgn in (1.0, -1.0):
            b = w.beta.copy()
            b[j] += sgn * h
            pl = _adjoint_plan(wave1d, w, b)
            _, uu = pl.solve_device(nsteps)
            Ls.append(0.5 * float(torch.sum((uu - d) ** 2)))
            pl.close()
        fd_err = max(fd_err, abs((Ls[0] - Ls[1]) / (2 * h) - gh[j]))
    t_fd = time.perf_counter() - t0
    work = w.M * nsteps
    line.update({
        "forward_value": work / (ms_fwd * 1e-3), "adjoint_value": work / (ms_adj * 1e-3),
        "forward_ms_per_step": ms_fwd / nsteps, "adjoint_ms_per_step": ms_adj / nsteps,
        "stored_density_bytes": 8 * w.M * nsteps,
        "checkpointed": {"interval": interval, "checkpoint_bytes": ckpt_bytes,
                         "segment_bytes": 8 * w.M * min(interval, nsteps),
                         "forward_value": work / (ms_cfwd * 1e-3), "adjoint_value": work / (ms_cadj * 1e-3),
                         "forward_ms_per_step": ms_cfwd / nsteps, "adjoint_ms_per_step": ms_cadj / nsteps,
                         "gradient_equal_bitwise": bool(torch.equal(g, g2)),
                         "receivers_equal_bitwise": bool(torch.equal(u, u2))},
        "central_differences": {"stiffnesses": int(args.adjoint_fd), "step": "1e-4 beta_j",
                                "max_abs_err_over_max_grad": fd_err / float(np.max(np.abs(gh))),
                                "wall_s": t_fd},
        "loss": loss, "plan_seconds": t_plan,
        "config": {"workload": f"{w.name} recipe at M = {w.M}: {w.description}", "M": w.M, "steps": nsteps,
                   "K": info.K, "W": info.W, "local_weights": info.local_weights, "R": len(w.xr),
                   "blocks": info.blocks, "max_block": info.max_block,
                   "timed": "CUDA events around one wave1d_solve (densities recorded on the device) and one "
                            "wave1d_adjoint call, then around wave1d_solve_checkpointed and "
                            "wave1d_adjoint_checkpointed on a fresh plan (work arrays included)"}})
    print(json.dumps(line))


def run_free_only(args):
    """The free-space M = 1e4 workload alone (the `free_M1e4` key of the benchmark line: stored
    weights, one-launch step kernel); the small case its kernel's profiles are taken on.  Not a
    benchmark line."""
    import torch

    from paper_2507_07823_gb300 import build

    build.build()
    print(json.dumps({"free_M1e4": free_space_secondary(torch, torch.cuda.current_stream())}))


def run_local_only(args):
    """The local sum of the plan without pair lists alone (k_rs_local) on the clustered recipe at
    --local-M springs in --local-clusters clusters (50,000 springs per cluster keeps the million-
    spring workload's cluster density), or with --local-uniform on a uniform instance of the
    batched workload's recipe: 2 steps, then 3 profiled steps.  The small cases the kernel's full
    profiles are taken on; not a benchmark line."""
    from paper_2507_07823_gb300 import build, wave1d, workloads

    build.build()
    if args.local_uniform:
        # the batched workload's largest instance: uniform, dt = 1e-3, tol 1e-12, p = 8
        w = workloads.make(f"uniform_M{args.local_M}", M=args.local_M, bc=workloads.PERIODIC, dt=1e-3, Nt=100,
                           tol=1e-12, p=8, seed=7823 + 3, amp=(1.0,), center=(-2.0,), width=(0.1,), R=4)
        label = f"uniform, M = {w.M}, dt = 1e-3, tol 1e-12, p = 8 (the batched workload's instance recipe)"
    else:
        w = workloads.config2(M=args.local_M, n_clusters=args.local_clusters, Nt=100)
        label = f"clustered recipe, M = {w.M}, {args.local_clusters} clusters"
    plan = wave1d.Plan.from_workload(w, local_weights=1)
    plan.solve(2, with_sigma=False)
    wave1d.wave1d_profile(plan.h, 1)
    for _ in range(3):
        wave1d._check(wave1d.wave1d_step(plan.h), "wave1d_step")
    ms, steps = wave1d.wave1d_profile_read(plan.h)
    info = plan.info
    plan.close()
    print(json.dumps({"workload": label, "M": w.M,
                      "local_pairs": info.local_pairs, "local_ms": float(ms[0] / steps),
                      "solve_ms": float(ms[wave1d.STAGES.index("solve")] / steps),
                      "pairs_per_s": info.local_pairs / (ms[0] / steps * 1e-3)}))


def run_mixed_only(args):
    """The benchmark workload marched in FP64 (the one-launch step) and in mixed precision (FP32
    spreading and interpolation, per-stage launches) for args.steps steps each after
    args.warmup warm-up steps: both rates and their relative difference in the densities and
    receiver fields.  Not part of the default benchmark line."""
    import torch

    from paper_2507_07823_gb300 import build, wave1d, workloads

    build.build()
    w = workloads.config1()
    K, Wm = args.steps, args.warmup
    out = {}
    fields = {}
    for name, kw in (("fp64", {}), ("mixed", {"precision": 1})):
        plan = wave1d.Plan.from_workload(w.with_(Nt=Wm + K), **kw)
        s_w, u_w = plan.solve(Wm)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream = torch.cuda.current_stream()
        e0.record(stream)
        wave1d._check(wave1d.wave1d_solve(plan.h, K, None, None, 1), "wave1d_solve")
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        fields[name] = (plan.sigma(), plan.receivers())
        out[name] = {"value": w.M * K / (ms * 1e-3), "ms_per_step": ms / K}
        plan.close()
    (s64, u64), (s32, u32) = fields["fp64"], fields["mixed"]
    out["rel_diff_sigma"] = float(np.max(np.abs(s32 - s64)) / np.max(np.abs(s64)))
    out["rel_diff_receivers"] = float(np.max(np.abs(u32 - u64)) / np.max(np.abs(u64)))
    print(json.dumps({"metric": METRIC, "unit": UNIT, "steps": K, "warmup": Wm, "dtype": "f64 / f32 history passes",
                      "config": {"workload": f"{w.name}: {w.description}"}, **out}))


def run_batched_only(args):
    """The batched workload's instances (256 periodic instances, M log-uniform up to
    args.batch_mmax) marched together through wave1d_batch_solve for args.steps steps after
    args.warmup: whole-batch scatterer-steps/s.  Forms: each instance's form chosen from its layout
    (local_weights = 2: the small ones joined, their step one persistent launch or one launch per
    pass; the large ones each a plan without pair lists, a branch of the step graph), and every
    instance without pair lists (local_weights = 1).  Not part of the default benchmark line."""
    import torch

    from paper_2507_07823_gb300 import build, wave1d, workloads

    build.build()
    ws = workloads.config3_instances(m_range=(1e2, args.batch_mmax), Nt=args.warmup + args.steps + 1)
    res = {}
    for name, kw in (("chosen_one_launch", dict(local_weights=2, step_kernel=1)),
                     ("chosen_per_pass", dict(local_weights=2, step_kernel=0)),
                     ("all_without_pair_lists", dict(local_weights=1))):
        t0 = time.perf_counter()
        batch = wave1d.Batch(ws, **kw)
        t_plan = time.perf_counter() - t0
        forms = batch.forms
        batch.solve(args.warmup, with_sigma=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream = torch.cuda.current_stream()
        e0.record(stream)
        st = wave1d.lib().wave1d_batch_solve(batch.h, args.steps, None, None, 1)
        e1.record(stream)
        torch.cuda.synchronize()
        if st != 0:
            raise RuntimeError(wave1d.lib().wave1d_batch_strerror().decode())
        ms = e0.elapsed_time(e1)
        Ms = np.array([w.M for w in ws])
        res[name] = {"value": batch.M * args.steps / (ms * 1e-3), "ms_per_step": ms / args.steps,
                     "one_launch": batch.one_launch, "plan_seconds": t_plan,
                     "instances_without_pair_lists": int(forms.sum()),
                     "smallest_M_without_pair_lists": int(Ms[forms == 1].min()) if forms.any() else None,
                     "largest_joined_M": int(Ms[forms == 0].max()) if (forms == 0).any() else None}
        M, R = batch.M, batch.R
        batch.close()
    best = res["chosen_one_launch"]
    print(json.dumps({"metric": METRIC, "unit": UNIT, "value": best["value"], "ms_per_step": best["ms_per_step"],
                      "steps": args.steps, "warmup": args.warmup, "dtype": "f64 / f32x2 local sums", "forms": res,
                      "config": {"workload": f"{len(ws)} periodic instances, M log-uniform in [1e2, {args.batch_mmax:g}], "
                                             f"dt = 1e-3, tol 1e-12, p = 8", "M_total": M, "R_total": R}}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-steps", type=int, default=10)
    ap.add_argument("--ref-max-steps", type=int, default=200)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true", help="skip the free-space M = 1e4 secondary measurement")
    ap.add_argument("--no-spread-interp", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the mixed / adjoint / batched forms beside FP64")
    ap.add_argument("--spread-interp-only", action="store_true",
                    help="only the M = 1e6 spreading / interpolation timings (not a benchmark line)")
    ap.add_argument("--spread-interp-reps", type=int, default=20)
    ap.add_argument("--adjoint-only", action="store_true",
                    help="only the forward and reverse-time march on the adjoint workload (not a benchmark line)")
    ap.add_argument("--adjoint-steps", type=int, default=2000)
    ap.add_argument("--adjoint-M", type=int, default=10000)
    ap.add_argument("--adjoint-interval", type=int, default=100, help="checkpoint interval (steps)")
    ap.add_argument("--adjoint-fd", type=int, default=32, help="stiffnesses checked by central differences")
    ap.add_argument("--adjoint-full-steps", type=int, default=1200,
                    help="steps of the M = 1e5 march through the plan without pair lists")
    ap.add_argument("--free-only", action="store_true",
                    help="only the free-space M = 1e4 workload with stored weights (not a benchmark line)")
    ap.add_argument("--local-only", action="store_true",
                    help="only the local sum of the plan without pair lists on a clustered case (not a benchmark line)")
    ap.add_argument("--local-M", type=int, default=250000)
    ap.add_argument("--local-clusters", type=int, default=4)
    ap.add_argument("--local-uniform", action="store_true",
                    help="--local-only on a uniform instance of the batched workload's recipe (--local-M springs)")
    ap.add_argument("--mixed-only", action="store_true",
                    help="only the FP64 and mixed-precision marches of the benchmark workload (not a benchmark line)")
    ap.add_argument("--batched-only", action="store_true",
                    help="only the batched march of the batched workload's instances (not a benchmark line)")
    ap.add_argument("--batch-mmax", type=float, default=1e5)
    args = ap.parse_args()
    if args.spread_interp_only:
        run_spread_interp_only(args)
    elif args.local_only:
        run_local_only(args)
    elif args.free_only:
        run_free_only(args)
    elif args.adjoint_only:
        run_adjoint_only(args)
    elif args.mixed_only:
        run_mixed_only(args)
    elif args.batched_only:
        run_batched_only(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
