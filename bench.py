#!/usr/bin/env python
"""Benchmark: point-iters/s of one trust-region-reflective fit on GB300.

Workload (the configuration the headline metric is quoted on): a rotated
elliptical 2D Gaussian (7 parameters: A, x0, y0, sx, sy, theta, c) fitted on a
1024 x 1024 pixel grid (1,048,576 points) of FP32 Poisson counts (peak 1000 on
background 20), sigma = sqrt(max(y, 1)), bounds sx, sy in [0.5, 500] and
theta in [-pi/2, pi/2]; FP32 model/Jacobian rows with FP64 reduction combine
and FP64 n x n solve (precision 'mixed'); ftol = xtol = gtol = 1e-10.

A step is one whole fit (gbfit_curve_fit) from p0 to termination.
  value      = sum over ranks of m * nfev / max over ranks of the summed step time
               (device time by CUDA events on the call's stream; inputs resident
               in HBM; L2 flushed by a 256 MiB write between steps).
  e2e        = the same metric through the C ABI with pinned HOST buffers: the
               host->device copy of y and sigma and the result read-back are
               inside the timed region (host wall clock around the call).
  roofline   = the persistent loop kernel (fit_loop_kernel<mixed>; one launch =
               one whole fit: every evaluation pass and trust-region step),
               timed per launch with CUDA events in the library's profiling
               mode, against the FP32 issue peak (the pass is bound by FP32
               arithmetic, not HBM).
  kernel_roofline = the fused evaluation pass alone (one gbfit_evaluate launch)
               for the 1D Gaussian at 1e6 / 1e7 / 5e7 points and the headline
               2D Gaussian, against the HBM copy peak and the FP32 peak.
  cpu_baseline = the FP64 oracle (test infrastructure) on the same workload,
               on rank 0 only.
--impl reference times that oracle as the reference arm.

Extra modes (not the headline line):
  --sweep     the 1D Gaussian size sweep, m = 1e3 ... 5e7, FP32 mixed and plain
              FP64 paths: one JSON line per (m, precision) with point-iters/s
  --batch     4,096 independent double-exponential fits of ragged m in one
              batched launch: fits/s and nfev distribution
  --no-extras only the timed fits of the headline workload (for ncu runs)
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "point-iters/s per TRF fit (% roofline); batched fits/s + p99 latency vs plain FP64"
UNIT = "point-iters/s"
W = H = 1024
M = W * H
TOL = dict(ftol=1e-10, xtol=1e-10, gtol=1e-10)
# Algorithmic work of one evaluation pass per point, rotated 2D Gaussian, mixed
# precision, implicit grid with sigma: bytes read (y, sigma: FP32) and FP32
# FLOPs (FFMA = 2, FADD / FMUL = 1, exp / rcp on the MUFU not counted).
# Difference form (trials near convergence): model value, cancellation-free
# difference and Jacobian row 86; weights, residuals and the Gram / gradient /
# cost / actual-reduction accumulation 90.  Direct form (a fit's first
# evaluation and wide trials): model value and Jacobian row at the trial
# point 40; weights and residual 10; Gram / gradient / cost / (w h)^2 sums 74.
BYTES_PER_POINT = 8
FLOPS_PER_POINT = 176
FLOPS_PER_POINT_DIRECT = 124
SM_COUNT, FP32_LANES_PER_SM, SM_MAX_MHZ = 152, 128, 2070.0
FP32_PEAK_TFLOPS = SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
L2_FLUSH_BYTES = 256 << 20


class L2Flush:
    """Evict the workload from L2 between timed steps (untimed): write a
    256 MiB buffer (twice the 129 MB L2)."""

    def __init__(self, device):
        import torch
        self.w = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=device)

    def zero_(self):
        self.w.zero_()
# DRAM bytes (read + write) per launch of the loop kernel (one whole fit of
# the headline workload, 5 passes) from the ncu capture summarised in
# profiles/fit_loop_mixed_gauss2d_1024.md (8.666 MB read + 3.3 KB written);
# None whenever the kernel has changed since the capture.
TRAFFIC_BYTES_PER_LAUNCH = 8.6697e6


def measured_peaks():
    """HBM copy bandwidth (GB/s) from MEASURED_PEAKS.json (driver-written),
    else the profiling recipe's fallback; and which one it is."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback (no MEASURED_PEAKS.json)"


# Algorithmic work per point of one fused evaluation pass at fixed p
# (gbfit_evaluate: a first evaluation, so the direct form): model value and
# Jacobian row, residual, Gram / gradient / cost / (w h)^2 sums; FMA = 2 FLOP,
# MUFU not counted.  1D Gaussian + offset on x, y FP32 (no sigma): 12 model +
# 28 residual and accumulation; rotated 2D Gaussian on the grid with sigma:
# 40 model + 10 weights and residual + 74 accumulation.
PASS_WORK = {"gauss1d_xy": (8, 40), "gauss2d_grid_sigma": (8, FLOPS_PER_POINT_DIRECT)}
# Plain FP64 pass (1D Gaussian on x, y FP64): 16 bytes per point; FP64
# instructions per point counted by ncu (profiles/eval_fp64_gauss1d_5e7.md).
FP64_PEAK_GFMA = 590.0        # FP64 FMA rate measured on this machine's GB300 (probe kernel, 1/62 of FP32)
# FP64 thread instructions per point of that pass (DFMA 25, DADD 8.1, DMUL 7 and the
# rest, ncu InstructionStats of the 5e7-point capture), each one FP64 pipe issue
FP64_INST_PER_POINT = 42.0


def kernel_roofline(dev, flush):
    """The fused Jacobian-reduction pass alone: one gbfit_evaluate launch (one
    evaluation pass over m points, its combine and an evaluation-only step),
    CUDA events around the launch (library profiling mode), L2 flushed before
    each launch; against the HBM copy peak and the FP32 issue peak."""
    import torch
    from paper_2208_12187_gb300 import gbfit, synth
    hbm, hbm_src = measured_peaks()
    out = []

    def timed(call, reps=5):
        call()
        gbfit.set_profiling(True)
        gbfit.stats_reset()
        for _ in range(reps):
            flush.zero_()
            call()
        st = gbfit.stats()
        gbfit.set_profiling(False)
        return st["eval_ms"] / max(st["eval_launches"], 1)

    def record(name, m, ms, bpp, fpp, extra):
        t = ms / 1e3
        gbs = m * bpp / t / 1e9
        tfs = m * fpp / t / 1e12
        t_roof = max(m * bpp / (hbm * 1e9), m * fpp / (FP32_PEAK_TFLOPS * 1e12))
        out.append({"workload": name, "m": m, "precision": "mixed", "us_per_launch": ms * 1e3,
                    "bytes_per_point": bpp, "flops_per_point": fpp, "achieved_gbs": gbs, "frac_hbm": gbs / hbm,
                    "achieved_tflops": tfs, "frac_fp32": tfs / FP32_PEAK_TFLOPS, "frac_roofline": t_roof / t,
                    **extra})

    for m in (1_000_000, 10_000_000, 50_000_000):
        pr = synth.gauss1d(m, seed=0, dtype=np.float32)
        x = torch.as_tensor(pr.x).to(dev)
        y = torch.as_tensor(pr.y).to(dev)
        ms = timed(lambda: gbfit.evaluate(pr.model, x, y, pr.p0, precision="mixed"))
        bpp, fpp = PASS_WORK["gauss1d_xy"]
        record("1D Gaussian + offset, x and y FP32", m, ms, bpp, fpp, {})
        if m == 50_000_000:
            x64, y64 = x.double(), y.double()
            ms64 = timed(lambda: gbfit.evaluate(pr.model, x64, y64, pr.p0, precision="fp64"), reps=3)
            pps = m / (ms64 / 1e3)
            out.append({"workload": "1D Gaussian + offset, x and y FP64, plain FP64 path", "m": m,
                        "precision": "fp64", "us_per_launch": ms64 * 1e3, "bytes_per_point": 16,
                        "achieved_gbs": m * 16 / (ms64 / 1e3) / 1e9, "frac_hbm": m * 16 / (ms64 / 1e3) / 1e9 / hbm,
                        "points_per_s": pps, "bound": "fp64 pipe",
                        "fp64_inst_per_point": FP64_INST_PER_POINT,
                        "frac_fp64_pipe": pps * FP64_INST_PER_POINT / (FP64_PEAK_GFMA * 1e9)})
            del x64, y64
        del x, y
    pr = make_problem(0)
    y = torch.as_tensor(pr.y).to(dev)
    sg = torch.as_tensor(pr.sigma).to(dev)
    ms = timed(lambda: gbfit.evaluate(pr.model, None, y, pr.p0, sigma=sg, grid_wh=(W, H), precision="mixed"))
    bpp, fpp = PASS_WORK["gauss2d_grid_sigma"]
    record("rotated 2D Gaussian, 1024 x 1024 grid, y and sigma FP32", M, ms, bpp, fpp, {})
    return {"records": out, "hbm_peak_gbs": hbm, "hbm_peak_source": hbm_src, "fp32_peak_tflops": FP32_PEAK_TFLOPS,
            "timing": "CUDA events around each gbfit_evaluate launch (profiling mode), L2 flushed before each"}


def workload_desc():
    return ("rotated 2D Gaussian (7 params) on a 1024x1024 pixel grid, 1,048,576 points, FP32 Poisson "
            "counts peak 1000 / background 20, sigma=sqrt(max(y,1)), bounds sx,sy in [0.5,500], "
            "theta in [-pi/2,pi/2]; FP32 model/Jacobian, FP64 combine and n x n solve")


def make_problem(rank: int):
    from paper_2208_12187_gb300 import synth
    return synth.gauss2d_grid(W, seed=rank, dtype=np.float32)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.device)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ distributed helpers
def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("gloo", rank=rank, world_size=world)
    return rank, local, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce(values, op, world):
    """All-reduce a list of floats over ranks (CPU, gloo): op 'max' or 'sum'."""
    if world == 1:
        return list(values)
    import torch
    import torch.distributed as dist
    t = torch.tensor(values, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return t.tolist()


# ------------------------------------------------------------------ CPU oracle timing
def oracle_rate(pr, budget_s: float = 12.0, max_fits: int = 8, want_result: bool = False):
    """Time whole oracle fits of the workload until the budget is spent."""
    from oracle import trf
    t_total, pts, fits, out = 0.0, 0.0, 0, None
    while fits < max_fits and (t_total < budget_s or fits == 0):
        t0 = time.perf_counter()
        out = trf.curve_fit_problem(pr, **TOL)
        t_total += time.perf_counter() - t0
        pts += pr.m * out["nfev"]
        fits += 1
    if want_result:
        return pts / t_total, fits, t_total, out
    return pts / t_total, fits, t_total


def oracle_rate_one_core(budget_s: float = 8.0):
    """The same oracle timing with one BLAS / OpenMP thread, in a child
    process (thread counts are fixed when numpy loads)."""
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-rate-only", str(budget_s)],
                             env=env, capture_output=True, text=True, timeout=budget_s * 10 + 60)
        return json.loads(out.stdout.strip().splitlines()[-1])
    except Exception as e:          # reported, never fatal for the bench line
        return {"error": str(e)[:200]}


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads") for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    return os.cpu_count()


# ------------------------------------------------------------------ arms
def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle on the host cores (rank 0 only)."""
    if rank != 0:
        return None
    pr = make_problem(0)
    for _ in range(args.warmup):
        pass  # the oracle has no warm-up state; W is accepted for the contract
    times, pts = [], 0.0
    from oracle import trf
    for _ in range(args.steps):
        t0 = time.perf_counter()
        out = trf.curve_fit_problem(pr, max_nfev=args.ref_nfev, **TOL)
        times.append(time.perf_counter() - t0)
        pts += pr.m * out["nfev"]
    total = sum(times)
    value = pts / total
    cores = blas_threads()
    sample = f"{args.steps} oracle fits of the workload, each capped at max_nfev={args.ref_nfev}"
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": workload_desc(), "m": M, "precision": "fp64 (oracle)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_ours(args, rank, local, world):
    import torch
    from paper_2208_12187_gb300 import build, gbfit
    torch.cuda.set_device(local)
    build.build()
    gbfit.load()
    pr = make_problem(rank)
    dev = torch.device("cuda", local)
    y = torch.as_tensor(pr.y).to(dev)
    sg = torch.as_tensor(pr.sigma).to(dev)
    flush = L2Flush(dev)
    stream = torch.cuda.current_stream()

    def fit(yy, ss):
        return gbfit.curve_fit(pr.model, None, yy, pr.p0, sigma=ss, lb=pr.lb, ub=pr.ub, grid_wh=(W, H),
                               precision="mixed", **TOL)

    for _ in range(max(args.warmup, 3)):
        fit(y, sg)
    torch.cuda.synchronize()
    gbfit.stats_reset()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    ms_total, pts, nfevs = 0.0, 0.0, []
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for _ in range(args.steps):
        flush.zero_()                       # L2 flush (untimed)
        torch.cuda.synchronize()
        e0.record(stream)
        out = fit(y, sg)
        e1.record(stream)
        e1.synchronize()
        ms_total += e0.elapsed_time(e1)
        pts += M * out["nfev"]
        nfevs.append(out["nfev"])
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    st = gbfit.stats()
    launches = int(st["kernel_launches"])
    ms_max, = allreduce([ms_total], "max", world)
    pts_sum, = allreduce([pts], "sum", world)
    value = pts_sum / (ms_max / 1e3)

    if args.no_extras:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "ms_per_step": ms_max / args.steps,
                              "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "note": "no extras"}))
        return None
    # ---- roofline: CUDA-event timing of the loop-kernel launch (one launch =
    # one whole fit: nfev evaluation passes plus the trust-region steps)
    gbfit.set_profiling(True)
    gbfit.stats_reset()
    passes = 0
    for _ in range(3):
        flush.zero_()
        passes += fit(y, sg)["nfev"]
    sp = gbfit.stats()
    gbfit.set_profiling(False)
    launches_p = max(sp["eval_launches"], 1)
    avg_ms = sp["eval_ms"] / launches_p
    # each fit's first evaluation and its wide trials run the direct form, the rest the difference form
    direct = launches_p + sp["phase_cycles"]["n_wide"]
    flops_per_launch = M * (FLOPS_PER_POINT_DIRECT * direct + FLOPS_PER_POINT * (passes - direct)) / launches_p
    achieved = flops_per_launch / (avg_ms / 1e3) / 1e12
    busy = sp["loop_busy_ms"] / max(sp["loop_busy_ms"] + sp["loop_wait_ms"], 1e-12)
    roof = {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP32_PEAK_TFLOPS, "traffic": TRAFFIC_BYTES_PER_LAUNCH,
            "kernel": "fit_loop_kernel<mixed> (rotated 2D Gaussian, grid, sigma; one launch per fit)",
            "flops_per_point": {"difference_form": FLOPS_PER_POINT, "direct_form": FLOPS_PER_POINT_DIRECT},
            "bytes_per_point": BYTES_PER_POINT, "passes_per_launch": passes / launches_p,
            "direct_form_passes_per_launch": direct / launches_p, "flops_per_launch": flops_per_launch,
            "avg_launch_us": avg_ms * 1e3,
            "cta_time_in_work_frac": busy,
            "peak_source": "152 SMs x 128 FP32 lanes x 2 FLOP x 2070 MHz (unit counts and max clock)"}
    if args.traffic is not None:
        roof["traffic"] = args.traffic

    kroof = kernel_roofline(dev, flush) if rank == 0 else None

    # ---- e2e: pinned host buffers through the C ABI, copies inside the timed region
    yh = torch.empty(M, dtype=torch.float32, pin_memory=True)
    sh = torch.empty(M, dtype=torch.float32, pin_memory=True)
    yh.copy_(torch.as_tensor(pr.y))
    sh.copy_(torch.as_tensor(pr.sigma))
    yn, sn = yh.numpy(), sh.numpy()
    for _ in range(2):
        fit(yn, sn)
    e2e_t, e2e_pts = 0.0, 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fit(yn, sn)                   # returns after the result read-back
        e2e_t += time.perf_counter() - t0
        e2e_pts += M * out["nfev"]
    e2e_t, = allreduce([e2e_t], "max", world)
    e2e_pts, = allreduce([e2e_pts], "sum", world)
    n = pr.n
    d2h = 8 * (n + n * n + 1) + 8        # popt, pcov, cost, nfev + status
    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": workload_desc(), "m": M, "precision": "mixed", "nfev_per_fit": nfevs[0],
                   "l2": "flushed between steps (256 MiB write, untimed)", "parallelism": f"{world} independent fits"},
        "roofline": roof,
        "kernel_roofline": kroof,
        "e2e": {"value": e2e_pts / e2e_t, "unit": UNIT, "h2d_bytes_per_step": 2 * 4 * M, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if rank == 0 and not args.no_cpu_baseline:
        rate, fits, secs, ref = oracle_rate(pr, want_result=True)
        one = oracle_rate_one_core()
        res["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
                               "sample": f"{fits} whole FP64 oracle fits of the same workload ({secs:.1f} s)",
                               "one_core": one}
        res["popt_rel_err_vs_oracle"] = float(np.max(np.abs(np.asarray(out["popt"]) - ref["popt"]) /
                                                     np.maximum(np.abs(ref["popt"]), 1.0)))
    return res


def run_compare(args):
    """The headline workload through explicit pixel coordinates and through
    the plain FP64 path; popt of the mixed forms against the plain FP64 GPU
    path (pinned to the oracle by the tests) (one JSON line)."""
    import torch
    from paper_2208_12187_gb300 import build, gbfit
    build.build()
    gbfit.load()
    pr = make_problem(0)
    dev = torch.device("cuda", 0)
    y = torch.as_tensor(pr.y).to(dev)
    sg = torch.as_tensor(pr.sigma).to(dev)
    flush = L2Flush(dev)
    res = layouts_and_fp64(args, pr, y, sg, flush, dev)
    ref = np.asarray(res["plain_fp64_grid"].pop("popt"))
    rel = lambda a: float(np.max(np.abs(np.asarray(a) - ref) / np.maximum(np.abs(ref), 1.0)))
    for k in ("mixed_grid", "mixed_explicit_soa2"):
        res[k]["popt_rel_err_vs_plain_fp64"] = rel(res[k].pop("popt"))
    print(json.dumps({"mode": "compare", "workload": workload_desc(), **res}))


def layouts_and_fp64(args, pr, y, sg, flush, dev):
    """Headline workload through explicit pixel coordinates (x, y rows FP32)
    and through the plain FP64 path (grid), a few timed fits each."""
    import torch
    from paper_2208_12187_gb300 import gbfit, synth
    Xc = torch.as_tensor(pr.coords().astype(np.float32)).to(dev)            # [2, m]
    out = {}
    for name, kw in (("mixed_grid", dict(xdata=None, grid_wh=(W, H), precision="mixed")),
                     ("mixed_explicit_soa2", dict(xdata=Xc, grid_wh=None, precision="mixed")),
                     ("plain_fp64_grid", dict(xdata=None, grid_wh=(W, H), precision="fp64"))):
        f = lambda: gbfit.curve_fit(pr.model, kw["xdata"], y, pr.p0, sigma=sg, lb=pr.lb, ub=pr.ub,
                                    grid_wh=kw["grid_wh"], precision=kw["precision"], **TOL)
        f()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms, pts, r = 0.0, 0.0, None
        for _ in range(3):
            flush.zero_()
            torch.cuda.synchronize()
            e0.record()
            r = f()
            e1.record()
            e1.synchronize()
            ms += e0.elapsed_time(e1)
            pts += M * r["nfev"]
        out[name] = {"value": pts / (ms / 1e3), "unit": UNIT, "ms_per_fit": ms / 3, "nfev": r["nfev"],
                     "popt": r["popt"]}
    return out


def run_eval_pass(args):
    """The fused evaluation pass alone (gbfit_evaluate) on the 1D Gaussian at
    the sizes of --sizes and the precisions of --precisions: --steps launches
    each after the L2 flush, CUDA-event time per launch (one JSON line per
    size and precision).  The capture target of the kernel-only ncu profiles."""
    import torch
    from paper_2208_12187_gb300 import build, gbfit, synth
    build.build()
    gbfit.load()
    dev = torch.device("cuda", 0)
    flush = L2Flush(dev)
    hbm, _ = measured_peaks()
    for m in [int(float(v)) for v in args.sizes.split(",")]:
        pr = synth.gauss1d(m, seed=0, dtype=np.float64)
        for prec in args.precisions.split(","):
            dt = torch.float32 if prec == "mixed" else torch.float64
            x = torch.as_tensor(pr.x).to(dt).to(dev)
            y = torch.as_tensor(pr.y).to(dt).to(dev)
            call = lambda: gbfit.evaluate(pr.model, x, y, pr.p0, precision=prec)
            call()
            gbfit.set_profiling(True)
            gbfit.stats_reset()
            for _ in range(args.steps):
                flush.zero_()
                call()
            st = gbfit.stats()
            gbfit.set_profiling(False)
            us = st["eval_ms"] / max(st["eval_launches"], 1) * 1e3
            bpp = 8 if prec == "mixed" else 16
            print(json.dumps({"mode": "eval_pass", "model": "gauss1d", "m": m, "precision": prec,
                              "us_per_launch": us, "gbs": m * bpp / us / 1e3, "frac_hbm": m * bpp / us / 1e3 / hbm,
                              "launches": int(st["eval_launches"])}), flush=True)
            del x, y


def run_phases(args):
    """Where one fit's launch spends its time: per-iteration cycle counters of
    the loop kernel's phases (owner CTA / stepping CTA, clock64) and the
    owner's global-timer figures, for the headline workload and three 1D
    workloads; warm L2 (no flush between fits), profiling on."""
    import torch
    from paper_2208_12187_gb300 import build, gbfit, synth
    build.build()
    gbfit.load()
    g2 = synth.gauss2d_grid(1024, seed=0, dtype=np.float32)
    y2, s2 = torch.as_tensor(g2.y).cuda(), torch.as_tensor(g2.sigma).cuda()
    work = [("rotated 2D Gaussian 1024x1024 grid + sigma, bounded", g2.m,
             lambda: gbfit.curve_fit(g2.model, None, y2, g2.p0, sigma=s2, lb=g2.lb, ub=g2.ub, grid_wh=g2.grid_wh,
                                     precision="mixed", **TOL))]
    for m in (1_000_000, 10_000_000):
        g1 = synth.gauss1d(m, seed=0)
        x1, y1 = torch.as_tensor(g1.x).float().cuda(), torch.as_tensor(g1.y).float().cuda()
        work.append((f"1D Gaussian, m={m:.0e}", m, lambda g1=g1, x1=x1, y1=y1: gbfit.curve_fit(
            g1.model, x1, y1, g1.p0, precision="mixed", **TOL)))
    d = synth.dexp(100_000, seed=21)
    xd, yd = torch.as_tensor(d.x).float().cuda(), torch.as_tensor(d.y).float().cuda()
    work.append(("double exponential, m=1e5, bounded", d.m, lambda: gbfit.curve_fit(
        d.model, xd, yd, d.p0, lb=d.lb, ub=d.ub, precision="mixed", **TOL)))
    for name, m, fit in work:
        for _ in range(3):
            fit()
        torch.cuda.synchronize()
        gbfit.set_profiling(True)
        gbfit.stats_reset()
        for _ in range(args.steps):
            out = fit()
        st = gbfit.stats()
        gbfit.set_profiling(False)
        pc, it, nfits = st["phase_cycles"], max(st["passes"], 1), args.steps
        timer_keys = ("start_ns", "round_ns", "owner_wait_ns", "barrier_ns")      # global timer, not cycles
        cycles = {k: round(v / it) for k, v in pc.items() if not k.startswith(("n_", "spare")) and k not in timer_keys}
        counts = {k: round(v / it, 3) for k, v in pc.items() if k.startswith("n_") or k in ("j32_sweeps", "refine_passes")}
        for k in counts:
            cycles.pop(k, None)
        timers = {k[:-3]: round(pc[k] / nfits / 1e3, 2) for k in timer_keys}
        print(json.dumps({"mode": "phases", "workload": name, "m": m, "precision": "mixed", "nfev": int(out["nfev"]),
                          "l2": "warm (no flush between fits)",
                          "launch_us": st["eval_ms"] / max(st["eval_launches"], 1) * 1e3,
                          "cycles_per_iteration": cycles, "events_per_iteration": counts,
                          "owner_global_timer_us_per_fit": timers}))


def run_sweep(args):
    """1D Gaussian + offset size sweep (config-0 generator), mixed and plain FP64."""
    import torch
    from paper_2208_12187_gb300 import build, gbfit, synth
    build.build()
    gbfit.load()
    flush = L2Flush("cuda")
    sizes = [int(v) for v in args.sizes.split(",")]
    for m in sizes:
        pr = synth.gauss1d(m, seed=0)
        for prec, dt in (("mixed", torch.float32), ("fp64", torch.float64)):
            if prec not in args.precisions.split(","):
                continue
            x = torch.as_tensor(pr.x).to(dt).cuda()
            y = torch.as_tensor(pr.y).to(dt).cuda()
            fit = lambda: gbfit.curve_fit(pr.model, x, y, pr.p0, precision=prec, **TOL)
            for _ in range(3):
                fit()
            gbfit.stats_reset()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ms, pts, nf = 0.0, 0.0, 0
            steps = max(1, min(args.steps, int(2e8 // m) + 1))
            for _ in range(steps):
                flush.zero_()
                torch.cuda.synchronize()
                e0.record()
                out = fit()
                e1.record()
                e1.synchronize()
                ms += e0.elapsed_time(e1)
                pts += m * out["nfev"]
                nf = out["nfev"]
            st = gbfit.stats()
            it = max(st["passes"], 1)
            cyc = st["phase_cycles"]
            bpp = 8 if prec == "mixed" else 16
            busy_ms = st["loop_busy_ms"] / max(st["loop_ctas"], 1)        # average CTA, per fit
            print(json.dumps({"mode": "sweep", "model": "gauss1d", "m": m, "precision": prec, "nfev": nf,
                              "fit_ms": ms / steps, "point_iters_per_s": pts / (ms / 1e3),
                              "bytes_per_point": 8 if prec == "mixed" else 16,
                              "hbm_gbs_equiv": pts * bpp / (ms / 1e3) / 1e9,
                              "hbm_frac_of_fit_time": pts * bpp / (ms / 1e3) / 1e9 / measured_peaks()[0],
                              "pass_gbs": m * nf * bpp / (busy_ms / 1e3) / 1e9,
                              "pass_hbm_frac": m * nf * bpp / (busy_ms / 1e3) / 1e9 / measured_peaks()[0],
                              "own_tile_cycles_per_iter": cyc["tile"] / it,
                              "step_cycles_per_iter": (cyc["logic"] + cyc["eigen"] + cyc["gn_path"] + cyc["step"] + cyc["prep"] + cyc["finish"]) / it,
                              "combine_cycles_per_iter": cyc["combine"] / it}))
            del x, y


# user-defined models as a user would write them (compiled at run time)
USER_GAUSS1D_SRC = r"""
template <class T, class S>
__device__ T model(const T* p, S x, S x2) {
    T d = x - p[1];
    return p[0] * exp(-square(d) / (2.0 * square(p[2]))) + p[3];
}
"""
USER_LORENTZ_SRC = r"""
template <class T, class S>
__device__ T model(const T* p, S x, S x2) {
    T u = (x - p[1]) / p[2];
    return p[0] / (1.0 + square(u)) + p[3];
}
"""


def run_user(args):
    """User-defined models: run-time compile time, and fit throughput of the
    built-in 1D Gaussian written as a user model against the built-in itself
    (same data, same fits), plus a Lorentzian peak."""
    import torch
    from paper_2208_12187_gb300 import build, gbfit, synth
    build.build()
    gbfit.load()
    t0 = time.perf_counter()
    gid = gbfit.register_model(USER_GAUSS1D_SRC, 4)
    t_compile = time.perf_counter() - t0
    lid = gbfit.register_model(USER_LORENTZ_SRC, 4)
    print(json.dumps({"mode": "user", "compile_s_per_model": t_compile, "nvrtc": "both precisions, one program"}))
    flush = L2Flush("cuda")

    def timed(fit, m):
        for _ in range(3):
            fit()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms, pts, out = 0.0, 0.0, None
        steps = max(3, min(args.steps, int(2e8 // m) + 1))
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0.record()
            out = fit()
            e1.record()
            e1.synchronize()
            ms += e0.elapsed_time(e1)
            pts += m * out["nfev"]
        return out, ms / steps, pts / (ms / 1e3)

    for m in [int(v) for v in args.sizes.split(",")]:
        for prec, dt in (("mixed", torch.float32), ("fp64", torch.float64)):
            if prec not in args.precisions.split(","):
                continue
            pr = synth.gauss1d(m, seed=0)
            x = torch.as_tensor(pr.x).to(dt).cuda()
            y = torch.as_tensor(pr.y).to(dt).cuda()
            ob, msb, rb = timed(lambda: gbfit.curve_fit(pr.model, x, y, pr.p0, precision=prec, **TOL), m)
            ou, msu, ru = timed(lambda: gbfit.curve_fit(gid, x, y, pr.p0, precision=prec, **TOL), m)
            lp = synth.user_family("lorentz1d", m, seed=0)
            lx = torch.as_tensor(lp.x).to(dt).cuda()
            ly = torch.as_tensor(lp.y).to(dt).cuda()
            ol, msl, rl = timed(lambda: gbfit.curve_fit(lid, lx, ly, lp.p0, precision=prec, **TOL), m)
            print(json.dumps({"mode": "user", "m": m, "precision": prec,
                              "builtin_gauss1d": {"fit_ms": msb, "point_iters_per_s": rb, "nfev": ob["nfev"]},
                              "user_gauss1d": {"fit_ms": msu, "point_iters_per_s": ru, "nfev": ou["nfev"],
                                               "rate_vs_builtin": ru / rb,
                                               "popt_rel_diff_vs_builtin": relerr_vec(ou["popt"], ob["popt"])},
                              "user_lorentz1d": {"fit_ms": msl, "point_iters_per_s": rl, "nfev": ol["nfev"],
                                                 "status": ol["status"]}}))
            del x, y, lx, ly


def run_cov(args):
    """Full-covariance fits (Appendix C): 1D Gaussian with AR(1)-correlated
    noise at several m; whole-call time (staging: copy of C, Cholesky, X =
    L^-1; then the fit) and the loop kernel's share from CUDA events."""
    import torch
    from paper_2208_12187_gb300 import build, gbfit, synth
    build.build()
    gbfit.load()
    for m in [int(v) for v in args.sizes.split(",")]:
        pr = synth.with_covariance(synth.gauss1d(m, seed=0), 0.5, 0.1, seed=1)
        C = torch.as_tensor(pr.sigma).cuda()
        for prec, dt in (("mixed", torch.float32), ("fp64", torch.float64)):
            if prec not in args.precisions.split(","):
                continue
            x = torch.as_tensor(pr.x).to(dt).cuda()
            y = torch.as_tensor(pr.y).to(dt).cuda()
            fit = lambda: gbfit.curve_fit(pr.model, x, y, pr.p0, sigma=C, precision=prec, **TOL)
            fit()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            steps = 3
            gbfit.set_profiling(True)
            gbfit.stats_reset()
            torch.cuda.synchronize()
            e0.record()
            for _ in range(steps):
                out = fit()
            e1.record()
            e1.synchronize()
            gbfit.set_profiling(False)
            st = gbfit.stats()
            call_ms = e0.elapsed_time(e1) / steps
            loop_ms = st["eval_ms"] / max(st["eval_launches"], 1)
            nf = out["nfev"]
            fma_per_pass = m * (m + 1) / 2 * (pr.n + (2 if prec == "mixed" else 1))
            print(json.dumps({"mode": "cov", "m": m, "precision": prec, "nfev": nf, "status": out["status"],
                              "call_ms": call_ms, "loop_ms": loop_ms, "staging_ms": call_ms - loop_ms,
                              "loop_ms_per_eval": loop_ms / nf,
                              "whitening_gflops_in_loop": 2 * fma_per_pass * nf / (loop_ms / 1e3) / 1e9}))
            del x, y
        del C


def run_batch(args):
    """4,096 ragged double-exponential fits in one batched launch, with tile
    shapes from the autotuner: the mixed form with its precision guard (the
    default), the guard's FP64 finish alone (guard_cond = inf), the guard off
    (every pass FP32), the plain FP64
    form in the same batched launch, and the plain FP64 path one fit at a
    time on a sample.  popt agreement of the mixed forms is stated against the
    plain FP64 batch (the FP64 GPU path is pinned to the oracle by the tests;
    the per-fit oracle criterion of the mixed forms is checked there too)."""
    import math
    import torch
    from paper_2208_12187_gb300 import build, gbfit, synth
    build.build()
    gbfit.load()
    t0 = time.perf_counter()
    bt = synth.dexp_batch(args.nfits, seed=7, dtype=np.float32)
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    tab = gbfit.autotune(bt.model, "mixed", m_max=200_000)
    tune_s = time.perf_counter() - t0
    shapes = {int(b): [int(tab["tile_points"][bt.model][gbfit.PREC_MIXED][b]),
                       int(tab["group_tiles"][bt.model][gbfit.PREC_MIXED][b])] for b in range(7, 18)}
    x = torch.as_tensor(bt.x).cuda()
    y = torch.as_tensor(bt.y).cuda()
    m = bt.offsets[1:] - bt.offsets[:-1]
    forms = {"mixed_guarded": dict(precision="mixed"),
             # the guard's FP64 finish alone (no escalation on the condition number)
             "mixed_guard_finish_only": dict(precision="mixed", guard_cond=math.inf),
             "mixed_guard_off": dict(precision="mixed", guard_cond=math.inf, guard_floor=math.inf),
             "fp64_batched": dict(precision="fp64")}
    res, outs = {}, {}
    for name, kw in forms.items():
        fit = lambda: gbfit.curve_fit_batch(bt.model, bt.offsets, x, y, bt.p0, lb=bt.lb, ub=bt.ub, **kw, **TOL)
        fit()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = 0.0
        gbfit.stats_reset()
        for _ in range(args.steps):
            torch.cuda.synchronize()
            e0.record()
            out = fit()
            e1.record()
            e1.synchronize()
            ms += e0.elapsed_time(e1)
        ms /= args.steps
        ph = gbfit.stats()["phase_cycles"]
        nfev = out["nfev"]
        res[name] = {"fits_per_s": bt.nfits / (ms / 1e3), "ms_per_batch": ms,
                     "point_iters_per_s": float(np.sum(m * nfev)) / (ms / 1e3),
                     "nfev_p50": float(np.median(nfev)), "nfev_max": int(nfev.max()),
                     "status_counts": {int(k): int(v) for k, v in zip(*np.unique(out["status"], return_counts=True))}}
        if name in ("mixed_guarded", "mixed_guard_finish_only"):
            res[name]["guard"] = {"fits_escalated": ph["n_guard_escalated"] / args.steps,
                                  "fits_fp64_finish": ph["n_guard_finished"] / args.steps,
                                  "fp64_evaluations": ph["n_eval64"] / args.steps}
        outs[name] = out
    # plain FP64, one fit at a time (same device data), on a sample
    S = min(args.serve_sample, bt.nfits)
    for k in range(4):
        a, b = int(bt.offsets[k]), int(bt.offsets[k + 1])
        gbfit.curve_fit(bt.model, x[a:b], y[a:b], bt.p0[k], lb=bt.lb[k], ub=bt.ub[k], precision="fp64", **TOL)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(S):
        a, b = int(bt.offsets[k]), int(bt.offsets[k + 1])
        gbfit.curve_fit(bt.model, x[a:b], y[a:b], bt.p0[k], lb=bt.lb[k], ub=bt.ub[k], precision="fp64", **TOL)
    torch.cuda.synchronize()
    plain_fps = S / (time.perf_counter() - t0)
    # the double exponential is symmetric under (a1, t1) <-> (a2, t2): compare with t1 <= t2 on both sides
    canon = lambda p: np.asarray(p)[[2, 3, 0, 1, 4]] if p[1] > p[3] else np.asarray(p)
    ref = outs["fp64_batched"]
    agree = {}
    for name in ("mixed_guarded", "mixed_guard_finish_only", "mixed_guard_off"):
        e = np.array([relerr_vec(canon(outs[name]["popt"][k]), canon(ref["popt"][k])) for k in range(bt.nfits)])
        agree[name] = {"frac_le_1e-6": float(np.mean(e <= 1e-6)), "frac_le_1e-5": float(np.mean(e <= 1e-5)),
                       "p50": float(np.median(e)), "p99": float(np.percentile(e, 99)), "max": float(e.max())}
    print(json.dumps({"mode": "batch", "model": "dexp", "nfits": bt.nfits, "total_points": int(bt.offsets[-1]),
                      "m": "log-uniform [200, 200000]", "data": "synthetic fp32", "generate_s": gen_s,
                      "autotune_s": tune_s, "tuned_shapes_log2m_to_tile_group": shapes, **res,
                      "plain_fp64_one_at_a_time": {"fits_per_s": plain_fps, "sample": S},
                      "guarded_over_plain_one_at_a_time_fits_per_s": res["mixed_guarded"]["fits_per_s"] / plain_fps,
                      "guarded_over_fp64_batched_fits_per_s": res["mixed_guarded"]["fits_per_s"] /
                      res["fp64_batched"]["fits_per_s"],
                      "finish_only_over_fp64_batched_fits_per_s": res["mixed_guard_finish_only"]["fits_per_s"] /
                      res["fp64_batched"]["fits_per_s"],
                      "popt_rel_err_vs_fp64_batched": agree}))


def relerr_vec(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1.0)))


def _serve_submit(srv, pr, k):
    x = None if pr.layout == 2 else pr.x
    return srv.submit(pr.model, x, pr.y, pr.p0, sigma=pr.sigma, lb=pr.lb, ub=pr.ub, grid_wh=pr.grid_wh, tag=k, **TOL)


def serve_open_loop(st, idx, t_arr, args, precision="mixed", trace=None):
    """Run the requests `idx` through one server, request j submitted once the
    wall clock passes t_arr[j].  Latency = arrival -> result retired on the
    host (includes queueing, the H2D copy of the request's data and every
    iteration).  Returns (fits/s over the whole stream, latencies, results)."""
    from paper_2208_12187_gb300 import gbfit
    srv = gbfit.Server(hbm_budget_bytes=int(args.serve_budget_gb * (1 << 30)), max_slots=args.serve_slots,
                       precision=precision, rounds_per_step=args.serve_rounds)
    n = len(idx)
    lat = np.zeros(n)
    late = np.zeros(n)
    res = [None] * n
    k = 0
    n_done = 0
    busy = 0
    T0 = time.perf_counter()
    while n_done < n:
        now = time.perf_counter() - T0
        while k < n and t_arr[k] <= now:
            _serve_submit(srv, st.request(int(idx[k])), k)
            late[k] = time.perf_counter() - T0 - t_arr[k]
            k += 1
        if busy or k > n_done:
            ts = time.perf_counter()
            a, q = srv.step()
            busy = a + q
            if trace is not None:
                trace.append((ts - T0, time.perf_counter() - ts, a, q))
        elif k < n:
            time.sleep(max(0.0, min(1e-3, t_arr[k] - (time.perf_counter() - T0))))
        for r in srv.poll():
            j = int(r["tag"])
            res[j] = r
            lat[j] = late[j] + (r["t_done"] - r["t_submit"])
            n_done += 1
    T = time.perf_counter() - T0
    srv.close()
    return n / T, lat, res


def run_serve(args):
    """Serving: open-loop Poisson stream of mixed-model, mixed-size requests
    (40% gauss1d, 40% dexp, 20% gauss2d; m log-uniform in [1e3, 4e6]),
    continuous batching under an HBM budget, against the plain
    one-fit-at-a-time FP64 path on a sample of the same stream."""
    import dataclasses
    import torch
    from paper_2208_12187_gb300 import build, gbfit, synth
    build.build()
    gbfit.load()
    t0 = time.perf_counter()
    for mdl in (synth.MODEL_GAUSS1D, synth.MODEL_DEXP, synth.MODEL_GAUSS2D):
        gbfit.autotune(mdl, "mixed", m_max=4_000_000)
    tune_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    st = synth.ServeStream(args.serve_requests, seed=11, n_data=2, dtype=np.float32)
    pin = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    for key, pr in list(st.data.items()):
        st.data[key] = dataclasses.replace(pr, x=pin(pr.x), y=pin(pr.y), sigma=pin(pr.sigma))
    gen_s = time.perf_counter() - t0
    N = len(st)
    idx = np.arange(N)
    base = {"mode": "serve", "requests": N, "mix": "40% gauss1d / 40% dexp / 20% gauss2d",
            "m": "log-uniform [1e3, 4e6] (2D: nearest W x W rung)", "mean_m": float(st.m.mean()),
            "budget_gb": args.serve_budget_gb, "slots": args.serve_slots, "rounds_per_step": args.serve_rounds,
            "data": "synthetic fp32, pinned host buffers", "generate_s": gen_s, "autotune_s": tune_s}
    pct = lambda lat: {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3)}
    # warm-up (builds, first-touch of the pool)
    serve_open_loop(st, idx[:64], np.zeros(64), args)
    # saturation: every request present at t = 0
    sat, lat, res = serve_open_loop(st, idx, np.zeros(N), args)
    pts = float(sum(int(st.m[j]) * r["nfev"] for j, r in enumerate(res)))
    bad = sum(r["status"] != 0 or r["fit_status"] < 1 for r in res)
    print(json.dumps({**base, "arm": "served-mixed", "arrival": "all at t=0", "fits_per_s": sat,
                      "point_iters_per_s": pts * sat / N, "not_converged": int(bad), **pct(lat)}), flush=True)
    # plain FP64, one fit at a time, on a sample of the stream
    S = min(args.serve_sample, N)
    def plain(t_arr):
        S = len(t_arr)
        lat = np.zeros(S)
        out = []
        T0 = time.perf_counter()
        for j in range(S):
            now = time.perf_counter() - T0
            if t_arr[j] > now:
                time.sleep(t_arr[j] - now)
            pr = st.request(j)
            x = None if pr.layout == 2 else pr.x
            out.append(gbfit.curve_fit(pr.model, x, pr.y, pr.p0, sigma=pr.sigma, lb=pr.lb, ub=pr.ub,
                                       grid_wh=pr.grid_wh, precision="fp64", **TOL))
            lat[j] = time.perf_counter() - T0 - t_arr[j]
        return S / (time.perf_counter() - T0), lat, out
    plain(np.zeros(min(S, 8)))
    psat, plat, pout = plain(np.zeros(S))
    err = []
    for j in range(S):
        a, b = res[j]["popt"], pout[j]["popt"]
        err.append(float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1.0))))
    err = np.array(err)
    print(json.dumps({**base, "arm": "plain-fp64-one-at-a-time", "sample": S, "arrival": "all at t=0",
                      "fits_per_s": psat, **pct(plat),
                      "served_mixed_vs_plain_fp64_popt_rel": {"max": float(err.max()), "p99": float(np.percentile(err, 99)),
                                                             "frac_le_1e-6": float(np.mean(err <= 1e-6))}}), flush=True)
    # open loop: a sweep of arrival rates up to saturation of the served form,
    # and the plain path at 80% of its own capacity (same rate for the served form)
    for frac in [float(f) for f in args.serve_rates.split(",")]:
        rate = frac * sat
        t_arr = synth.ServeStream.arrivals(N, rate, seed=3)
        thr, lat, _ = serve_open_loop(st, idx, t_arr, args)
        print(json.dumps({**base, "arm": "served-mixed", "arrival": "poisson", "rate_per_s": rate,
                          "rate_frac_of_saturation": frac, "fits_per_s": thr, **pct(lat)}), flush=True)
    rate = 0.8 * psat
    t_arr = synth.ServeStream.arrivals(S, rate, seed=4)
    _, plat, _ = plain(t_arr)
    _, slat, _ = serve_open_loop(st, idx[:S], t_arr, args)
    print(json.dumps({**base, "arm": "both-at-plain-rate", "sample": S, "arrival": "poisson", "rate_per_s": rate,
                      "plain_fp64": pct(plat), "served_mixed": pct(slat)}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-nfev", type=int, default=6)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per evaluation launch from an ncu capture of the current kernel")
    ap.add_argument("--sweep", action="store_true")
    ap.add_argument("--sizes", default="1000,10000,100000,1000000,10000000,50000000")
    ap.add_argument("--batch", action="store_true")
    ap.add_argument("--nfits", type=int, default=4096)
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--precisions", default="mixed,fp64")
    ap.add_argument("--oracle-sample", type=int, default=64)
    ap.add_argument("--serve", action="store_true")
    ap.add_argument("--user", action="store_true", help="user-defined models (run-time compiled) vs built-in")
    ap.add_argument("--cov", action="store_true", help="full-covariance fits (sizes from --sizes)")
    ap.add_argument("--eval-pass", action="store_true",
                    help="the fused evaluation pass alone (gbfit_evaluate), 1D Gaussian, --sizes x --precisions")
    ap.add_argument("--phases", action="store_true",
                    help="per-iteration phase cycles of the loop kernel (headline and 1D workloads, warm L2)")
    ap.add_argument("--compare", action="store_true",
                    help="headline workload: implicit grid vs explicit coordinates vs plain FP64, against the oracle")
    ap.add_argument("--serve-requests", type=int, default=20000)
    ap.add_argument("--serve-sample", type=int, default=200)
    ap.add_argument("--serve-budget-gb", type=float, default=16.0)
    ap.add_argument("--serve-slots", type=int, default=4096)
    ap.add_argument("--serve-rounds", type=int, default=4)
    ap.add_argument("--serve-rates", default="0.1,0.25,0.5,0.8,1.0,1.2")
    ap.add_argument("--oracle-rate-only", type=float, default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_rate_only is not None:
        rate, fits, secs = oracle_rate(make_problem(0), budget_s=args.oracle_rate_only, max_fits=4)
        print(json.dumps({"value": rate, "unit": UNIT, "cores": 1, "sample": f"{fits} fits ({secs:.1f} s)"}))
        return
    if args.sweep:
        return run_sweep(args)
    if args.batch:
        return run_batch(args)
    if args.serve:
        return run_serve(args)
    if args.user:
        return run_user(args)
    if args.cov:
        return run_cov(args)
    if args.compare:
        return run_compare(args)
    if args.phases:
        return run_phases(args)
    if args.eval_pass:
        return run_eval_pass(args)
    rank, local, world = dist_setup(args)
    if args.impl == "reference":
        res = run_reference(args, rank, world)
    else:
        res = run_ours(args, rank, local, world)
    if rank == 0 and res is not None:
        print(json.dumps(res))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
