#!/usr/bin/env python3
"""Throughput of the backward-Euler Richards step on GB300: DOF * Newton-steps / s.

A bench "step" is one backward-Euler time step of the workload (constitutive
evaluation, residual, Jacobian and diffusion-matrix assembly, AMG setup or
refresh, right-preconditioned Krylov solves with the AMG V-cycle, Newton-Armijo
line search) -- every stage of the path.  Default workload (configuration 2 of
the workload list): 128^3 cells (2.1M DOF), homogeneous Haverkamp soil,
upstream-mean K, Dirichlet top at -20.7 cm, no-flux elsewhere, p0 = -61.5 cm, dt
ramped linearly 1 -> 30 s over 20 steps, FGMRES(30) with an AMG V(2,2) l1-Jacobi
cycle, coarsest level (< 2000 unknowns) by dense inverse, Newton-Armijo to 1e-8
relative, FP64 throughout.  The larger mixed-precision workloads (256^3
harmonic, 512^3 sigma 2) do not converge with this method (see the design
notes), so this is the largest configuration of the list that runs.

Timing (independent of --warmup): W warm-up steps run on a context of their
own, which is then destroyed; the timed run is a fresh context stepping the
schedule from p0 (step m uses dt_{m mod 20}), AMG setup included, inputs
resident on the device, CUDA events around the K steps and nothing else in the
timed region but the nvidia-smi clock sampler (a separate process).

value   = sum over ranks of (DOF * Newton iterations in the timed steps) / max
          over ranks of the CUDA-event time of the timed steps.
e2e     = the same metric through rich_step_host on another fresh context: each
          step copies p from pinned host memory to the device and the result back.

Further passes, outside the timed region: the same schedule with the FP32 AMG
hierarchy (`fp32_amg`, speed-up and largest pressure deviation from FP64), a
per-kernel profile of the first steps (every launch timed with CUDA events)
that places the dominant kernel on its roofline (HBM bandwidth from
MEASURED_PEAKS.json, FP64 FMA throughput measured live by
rich_measure_fma_peak; the bound follows from the kernel's algorithmic
flops/byte against the balance point), the paper's own 24.2M-cell infiltration
grid in mixed precision (`paper_workload`), the oracle timed on the host cores
(`cpu_baseline`), a request stream through the request server (`serving`) and a
burst of same-shape requests served with and without batching (`serving_uniform`).

--impl reference times the CPU oracle (the plain FP64 numpy/scipy restatement)
on the host cores: each step is one Newton iteration of the workload's first
time step on a reduced grid of the same settings (a bounded sample).
With torchrun (N > 1) every rank runs an independent replica of the workload
(the path has no cross-rank exchange on one GPU each); rank 0 prints.
"""
import argparse
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FALLBACK_HBM_GBS = 6800.0
# ncu dram__bytes_read.sum + dram__bytes_write.sum per launch of a kernel on a
# workload, from the profiles/ summaries of the same kernel and workload (None:
# no capture of the current kernel).
# DRAM bytes per launch from ncu captures of the same workload: the finest FP64
# sweep measured whole; the batched dots measured over their first 60 launches
# (DRAM / algorithmic = 1.037) and scaled to the profile pass's 241.2 MB per launch
NCU_TRAFFIC_BYTES = {("richards128_fp64", "l1jacobi_l0"): 125.615616e6,
                     ("richards128_fp64", "multidot"): 1.037 * 241.2e6}
# the oracle's reduced grid for the host-core samples (cells per side)
CPU_SAMPLE_N = {"richards128_fp64": 48, "richards16_fp64": 16, "richards256_mixed": 32, "richards512_mixed": 32,
                "paper_infiltration": 96}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="richards128_fp64")
    ap.add_argument("--grid", type=int, default=None,
                    help="run the workload's settings on an n^3 grid instead (profiling captures); not a bench line")
    ap.add_argument("--amg-precision", default=None, choices=["fp64", "fp32"],
                    help="override the workload's AMG precision for the timed run")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the FP32-AMG comparison run")
    ap.add_argument("--no-profile", action="store_true", help="skip the per-kernel roofline pass")
    ap.add_argument("--profile-steps", type=int, default=3)
    ap.add_argument("--no-paper", action="store_true", help="skip the paper-grid mixed-precision run")
    ap.add_argument("--tune-file", default=None,
                    help="autotuner table: loaded at start if the file exists, written at the end (a profiled run "
                         "then runs the variants a plain run chose)")
    ap.add_argument("--paper-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--cpu-procs", type=int, default=0, help="oracle processes for the all-cores sample (0: min(16, cores))")
    ap.add_argument("--no-serving", action="store_true", help="skip the request-stream measurement")
    ap.add_argument("--serving-requests", type=int, default=512)
    ap.add_argument("--serving-slots", type=int, default=8)
    ap.add_argument("--serving-lists", type=int, default=1,
                    help="Galerkin product lists for served requests (0: searching refresh, whose shared-memory "
                         "atomics make results differ from run to run at rounding level)")
    ap.add_argument("--serving-only", action="store_true", help="print only the request-stream measurement")
    ap.add_argument("--serving-coarse-max", type=int, default=500)
    ap.add_argument("--serving-aggregation", type=int, default=0, help="0: MIS-2, 1: matching (SMATCH-style)")
    ap.add_argument("--serving-batch", type=int, default=8,
                    help="largest packed batch of same-shape requests (1: one request per slot)")
    ap.add_argument("--serving-stall", type=float, default=0.5,
                    help="serving requests' FGMRES gives up after a restart cycle that reduced the residual by less "
                         "than this fraction (0: off)")
    ap.add_argument("--serving-halvings", type=int, default=0,
                    help="time-step control of served requests (0: off; retries multiply the device time of the "
                         "failing requests, measured 3-10x on this stream)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            with open(path) as f:
                d = json.load(f)
            for k in ("hbm_gbs", "hbm_GBs", "hbm_copy_gbs"):
                if k in d:
                    return float(d[k]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def aggregate_over_ranks(dist, elapsed, work, device):
    """Whole-job numbers of an N-replica run: max elapsed time, summed work (DOF * Newton its)."""
    if dist is None:
        return elapsed, work
    import torch
    t = torch.tensor([elapsed], dtype=torch.float64, device=device)
    wk = torch.tensor([work], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(wk, op=dist.ReduceOp.SUM)
    return float(t[0]), float(wk[0])


def workload_setup(name, n=None):
    from paper_2112_05051_gb300 import synth
    w = synth.WORKLOADS[name]
    grid, soil, bc, ks, p0, dts = synth.workload_inputs(w, n)
    return w, grid, soil, bc, ks, p0, dts


def newton_opts(rb, w):
    return rb.default_newton_opts(kind=rb.KRYLOV_FGMRES if w.krylov == "fgmres" else rb.KRYLOV_FCG,
                                  restart=max(w.restart, 1), nu1=w.nu, nu2=w.nu, seed=w.amg_seed,
                                  coarse_max=w.coarse_max, amg_policy=rb.AMG_REFRESH, smooth_levels=w.smooth_levels)


def host_cpu():
    """Host CPU model and core count (the oracle's machine)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"model": model or platform.processor() or platform.machine(), "arch": platform.machine(),
            "os_cpu_count": os.cpu_count()}


def oracle_sample_main(workload, budget, n=None, steps=None, warmup=0):
    """Time oracle Newton iterations of the workload's first time step on an n^3 grid.

    Each timed unit is one Newton iteration (newton.step with max_newton = 1) from
    the state the previous one left; the AMG setup runs in an untimed first call."""
    from oracle import newton
    w, grid, soil, bc, ks, p0, dts = workload_setup(workload, n)
    prob = newton.Problem(grid, soil, bc, w.kmean, ks)
    opt = newton.NewtonOptions(krylov=w.krylov, restart=max(w.restart, 1), nu1=w.nu, nu2=w.nu,
                               amg_seed=w.amg_seed, coarse_max=min(w.coarse_max, max(50, grid.n // 50)),
                               max_newton=1, smooth_levels=w.smooth_levels)
    p = p0.copy()
    t0 = time.perf_counter()
    p, st = newton.step(prob, p, dts[0], opt)  # builds the hierarchy (not timed)
    setup_s = time.perf_counter() - t0
    for _ in range(warmup or 0):
        p, st = newton.step(prob, p, dts[0], opt)
    its, times = 0, []
    t0 = time.perf_counter()
    while True:
        t1 = time.perf_counter()
        p, st = newton.step(prob, p, dts[0], opt)
        times.append(time.perf_counter() - t1)
        its += st.newton_its
        if steps is not None:
            if len(times) >= steps:
                break
        elif time.perf_counter() - t0 >= budget:
            break
    el = time.perf_counter() - t0
    return {"dof": grid.n, "its": its, "seconds": el, "setup_s": setup_s, "step_times": times,
            "grid": [grid.nx, grid.ny, grid.nz]}


def _oracle_processes(workload, n, procs, budget=None, steps=None, warmup=0):
    """Run the oracle sample in `procs` concurrent one-thread processes; whole-host throughput."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample", workload, str(n),
           str(budget if budget is not None else 0.0), str(steps if steps is not None else 0), str(warmup)]
    t0 = time.perf_counter()
    ps = [subprocess.Popen(cmd, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
          for _ in range(procs)]
    res = []
    for pr in ps:
        out, err = pr.communicate(timeout=3600)
        if pr.returncode != 0:
            raise RuntimeError("oracle sample failed: " + (err.strip().splitlines() or ["?"])[-1])
        res.append(json.loads(out.strip().splitlines()[-1]))
    wall = time.perf_counter() - t0
    work = sum(r["dof"] * r["its"] for r in res)
    slowest = max(r["seconds"] for r in res)
    return {"value": work / slowest, "procs": procs, "its": sum(r["its"] for r in res), "seconds": slowest,
            "wall_s": wall, "grid": res[0]["grid"], "setup_s": max(r["setup_s"] for r in res)}


def cpu_baseline(workload, budget, procs):
    """The oracle on the host cores: one process, and `procs` concurrent processes."""
    n = CPU_SAMPLE_N.get(workload, 32)
    host = host_cpu()
    one = _oracle_processes(workload, n, 1, budget=budget)
    many = _oracle_processes(workload, n, procs, budget=budget) if procs > 1 else one
    return {"value": many["value"], "unit": "DOF*Newton-steps/s", "cores": many["procs"], "kind": "oracle",
            "one_core_value": one["value"], "host": host,
            "sample": "Newton iterations of the first time step of %s's settings on a reduced %s grid, each "
                      "process for about %g s (AMG setup excluded), plain numpy/scipy FP64, one thread per process; "
                      "%d processes at once: %d iterations; one process alone: %d iterations"
                      % (workload, "x".join(map(str, many["grid"])), budget, many["procs"], many["its"], one["its"])}


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    w, grid, soil, bc, ks, p0, dts = workload_setup(args.workload, args.grid)
    n = CPU_SAMPLE_N.get(args.workload, 32)
    procs = args.cpu_procs or min(16, os.cpu_count() or 1)
    res = _oracle_processes(args.workload, n, procs, steps=args.steps, warmup=args.warmup)
    value = res["value"]
    host = host_cpu()
    sample = ("%d Newton iterations (%d per process, %d one-thread processes at once) of the first time step "
              "of %s's settings on a reduced %s grid, plain numpy/scipy FP64; AMG setup and %d warm-up "
              "iterations untimed" % (res["its"], args.steps, procs, args.workload,
                                      "x".join(map(str, res["grid"])), args.warmup))
    line = {"metric": "DOF*Newton-steps/s", "value": value, "unit": "DOF*Newton-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * res["seconds"] / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": workload_config(w, grid),
            "cpu_baseline": {"value": value, "unit": "DOF*Newton-steps/s", "cores": procs, "kind": "oracle",
                             "sample": sample, "host": host},
            "e2e": {"value": value, "unit": "DOF*Newton-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def percentile(sorted_values, q):
    """The q-quantile of an ascending list by the nearest-rank rule: the smallest value
    with at least a fraction q of the values at or below it (None if empty)."""
    if not sorted_values:
        return None
    n = len(sorted_values)
    return sorted_values[min(n - 1, max(0, math.ceil(q * n) - 1))]


def _device_ms_split(results):
    """Device time of the requests' steps (ms_total), converged vs failed, with their mean
    Newton and Krylov iteration counts: where a stream's GPU time goes."""
    out = {}
    for name, sel in (("converged", lambda r: r["status"] == 0), ("failed", lambda r: r["status"] != 0)):
        rs = [r for r in results if sel(r)]
        out[name] = {"count": len(rs), "ms": sum(r["stats"].get("ms_total", 0.0) for r in rs),
                     "mean_newton": sum(r["stats"]["newton_its"] for r in rs) / len(rs) if rs else None,
                     "mean_linear": sum(r["stats"].get("linear_its", 0) for r in rs) / len(rs) if rs else None}
    return out


def stream_stats(results, dofs, seconds, error_names):
    """Latency percentiles (ms, submit -> done), converged work per second and failures by status name."""
    lat = sorted(1e3 * (r["t_done"] - r["t_submit"]) for r in results)
    lat_ok = sorted(1e3 * (r["t_done"] - r["t_submit"]) for r in results if r["status"] == 0)
    work = sum(n * r["stats"]["newton_its"] for n, r in zip(dofs, results) if r["status"] == 0)
    failed = {}
    for r in results:
        if r["status"] != 0:
            key = error_names.get(r["status"], str(r["status"]))
            failed[key] = failed.get(key, 0) + 1
    return {"latency_ms_converged": {"p50": percentile(lat_ok, 0.5), "p99": percentile(lat_ok, 0.99),
                                     "mean": sum(lat_ok) / len(lat_ok) if lat_ok else None,
                                     "max": lat_ok[-1] if lat_ok else None},
            "latency_ms_all": {"p50": percentile(lat, 0.5), "p99": percentile(lat, 0.99),
                               "mean": sum(lat) / len(lat) if lat else None, "max": lat[-1] if lat else None},
            "device_ms": _device_ms_split(results),
            "converged": len(lat_ok), "failure_rate": (len(lat) - len(lat_ok)) / len(lat) if lat else None,
            "converged_per_s": len(lat_ok) / seconds if seconds > 0 else None,
            "dof_newton_per_s": work / seconds if seconds > 0 else None, "failed": failed}


def serving_run(args, rb):
    """Request stream: one-step solves of mixed size and soil through the request server.

    Each request is one backward-Euler step (dt = 1 s) of an n^3 column, n drawn
    from {24, 32, 48, 64, 96}, with its own seeded log-normal K_s field (sigma
    uniform in [1, 2], field seed 1000 + id) and K-mean kind (arithmetic,
    upstream or harmonic), FP32 AMG (coarsest level < 500 unknowns) with FP64
    residual and outer FCG.  A closed
    burst of all requests measures the capacity mu (requests / s); then the same
    requests arrive as a Poisson stream at 0.8 mu (seed 5) and the latency
    submit -> result on the host is reported.  Finally one request of each size
    is rerun alone and compared with its result in the mix.
    """
    import numpy as np
    from paper_2112_05051_gb300 import synth
    rng = np.random.default_rng(5)
    n_req = args.serving_requests
    sizes = [24, 32, 48, 64, 96]
    soil = synth.Soil()
    bc = synth.infiltration_bc(synth.P_TOP)
    reqs = []
    p0s = {}
    for i in range(n_req):
        n = sizes[int(rng.integers(len(sizes)))]
        sigma = float(rng.uniform(1.0, 2.0))
        kmean = int(rng.integers(3))
        grid = synth.Grid(n, n, n)
        ks = synth.ks_field(grid, 1000 + i, sigma)
        p0s.setdefault(n, np.full(grid.n, synth.P_INITIAL))
        reqs.append((grid, ks, kmean, n))
    # coarsest level below 500 unknowns: its dense inverse is redone at every
    # refresh, and a short one-step request refreshes ~10 times
    # optional time-step control: a request whose step fails is retried in halves
    halvings = getattr(args, "serving_halvings", 0)
    opts = rb.default_newton_opts(kind=rb.KRYLOV_FCG, nu1=1, nu2=1, seed=3, smooth_levels=2,
                                  product_lists=args.serving_lists, coarse_max=args.serving_coarse_max,
                                  aggregation=args.serving_aggregation, max_dt_halvings=halvings,
                                  max_newton=20 if halvings else 50, stall=getattr(args, "serving_stall", 0.0))

    def submit(srv, q):
        grid, ks, kmean, n = q
        return srv.submit(grid, soil, bc, kmean, 1.0, p0=p0s[n], ks=ks, precision=rb.PREC_MIXED, opts=opts)

    batch_max = getattr(args, "serving_batch", 1)
    srv = rb.Server(slots=args.serving_slots, batch_max=batch_max) if batch_max > 1 else rb.Server(
        slots=args.serving_slots)
    # warm-up: one request of each size (library kernels loaded, memory pool primed)
    for n in sizes:
        k = next((j for j, q in enumerate(reqs) if q[3] == n), None)
        if k is not None:
            srv.wait(submit(srv, reqs[k]))
    t0 = time.perf_counter()
    ids = [submit(srv, q) for q in reqs]
    burst = [srv.wait(i) for i in ids]
    t_burst = time.perf_counter() - t0
    mu = n_req / t_burst
    lam = 0.8 * mu
    gaps = rng.exponential(1.0 / lam, n_req)
    t1 = time.perf_counter()
    due = t1
    ids = []
    for q, g in zip(reqs, gaps):
        due += g
        wait = due - time.perf_counter()
        if wait > 0:
            time.sleep(wait)
        ids.append(submit(srv, q))
    stream = [srv.wait(i) for i in ids]
    t_stream = time.perf_counter() - t1
    cnt = srv.counters()
    srv.close()
    st_b = stream_stats(burst, [q[0].n for q in reqs], t_burst, rb.ERRORS)
    st_s = stream_stats(stream, [q[0].n for q in reqs], t_stream, rb.ERRORS)
    # the same requests alone (one slot, nothing else in flight) against their results in the mix
    alone = rb.Server(slots=1)
    dev = 0.0
    checked = 0
    for n in sizes:
        k = next((j for j, q in enumerate(reqs) if q[3] == n and stream[j]["status"] == 0), None)
        if k is None:
            continue
        r = alone.wait(submit(alone, reqs[k]))
        if r["status"] == 0:
            dev = max(dev, float(np.abs(r["p"] - stream[k]["p"]).max() / np.abs(stream[k]["p"]).max()))
            checked += 1
    alone.close()
    return {"requests": n_req, "slots": args.serving_slots, "sizes": sizes, "sigma": [1.0, 2.0],
            "coarse_max": args.serving_coarse_max, "product_lists": args.serving_lists,
            "aggregation": "matching" if args.serving_aggregation else "MIS-2",
            "kmeans": ["arithmetic", "upstream", "harmonic"], "precision": "fp32 AMG, fp64 residual and FCG",
            "max_dt_halvings": halvings, "max_newton_per_attempt": 20 if halvings else 50,
            "fgmres_stall": getattr(args, "serving_stall", 0.0),
            "latency_ms_converged": st_s["latency_ms_converged"], "failure_rate": st_s["failure_rate"],
            "device_ms_burst": st_b["device_ms"],
            "converged_per_s": st_s["converged_per_s"], "stream_dof_newton_per_s": st_s["dof_newton_per_s"],
            "capacity_rps": mu, "capacity_converged_rps": st_b["converged_per_s"], "burst_s": t_burst,
            "burst_dof_newton_per_s": st_b["dof_newton_per_s"], "rate_rps": lam, "arrivals": "Poisson, seed 5",
            "stream_s": t_stream, "latency_ms_all": st_s["latency_ms_all"],
            "failed": st_s["failed"], "max_in_flight": cnt["max_in_flight"], "batch_max": batch_max,
            "batched_requests": sum(1 for r in stream if r.get("batch_size", 1) > 1),
            "batch_reruns": sum(1 for r in stream if r.get("batch_rerun", 0)),
            "mix_vs_alone_max_rel_dev": dev, "mix_vs_alone_checked": checked,
            "admission": "FIFO, a free slot and the request's device-memory estimate within 80% of free HBM"}


def serving_uniform(args, rb, n_req=256, n=32):
    """Where batching applies: a burst of same-shape requests (n^3 columns, sigma 0.5
    log-normal K_s fields, upstream mean, dt = 0.25 s, FP32 AMG, FCG) on which FCG
    needs no fallback, through the server with batch_max 1 and 8.  Capacity of the
    burst, failures, and the largest deviation of a batched result from the same
    request served alone."""
    import numpy as np
    from paper_2112_05051_gb300 import synth
    soil = synth.Soil()
    bc = synth.infiltration_bc(synth.P_TOP)
    grid = synth.Grid(n, n, n)
    p0 = np.full(grid.n, synth.P_INITIAL)
    fields = [synth.ks_field(grid, 5000 + i, 0.5, (4.0, 4.0, 2.0)) for i in range(n_req)]
    opts = rb.default_newton_opts(kind=rb.KRYLOV_FCG, nu1=1, nu2=1, seed=3, smooth_levels=2,
                                  coarse_max=args.serving_coarse_max)
    out = {"requests": n_req, "grid": [n, n, n], "sigma": 0.5, "kmean": "upstream", "dt": 0.25,
           "slots": args.serving_slots}
    results = {}
    for bm in (1, 8):
        srv = rb.Server(slots=args.serving_slots, batch_max=bm)
        srv.wait(srv.submit(grid, soil, bc, synth.KMEAN_UPSTREAM, 0.25, p0=p0, ks=fields[0], precision=rb.PREC_MIXED,
                            opts=opts))  # warm-up
        t0 = time.perf_counter()
        ids = [srv.submit(grid, soil, bc, synth.KMEAN_UPSTREAM, 0.25, p0=p0, ks=f, precision=rb.PREC_MIXED, opts=opts)
               for f in fields]
        res = [srv.wait(i) for i in ids]
        t = time.perf_counter() - t0
        srv.close()
        results[bm] = res
        out["batch%d" % bm] = {"capacity_rps": n_req / t, "burst_s": t,
                               "failed": sum(1 for r in res if r["status"] != 0),
                               "batched_requests": sum(1 for r in res if r.get("batch_size", 1) > 1),
                               "batch_reruns": sum(1 for r in res if r.get("batch_rerun", 0))}
    dev = 0.0
    for a, b in zip(results[1], results[8]):
        if a["status"] == 0 and b["status"] == 0:
            dev = max(dev, float(np.abs(a["p"] - b["p"]).max() / np.abs(a["p"]).max()))
    out["batched_vs_alone_max_rel_dev"] = dev
    out["speedup_batch8"] = out["batch8"]["capacity_rps"] / out["batch1"]["capacity_rps"]
    return out


def workload_config(w, grid):
    from paper_2112_05051_gb300 import synth
    return {"workload": w.name, "grid": [grid.nx, grid.ny, grid.nz], "dof": grid.n,
            "kmean": synth.kmean_name(w.kmean), "krylov": "%s(%d)" % (w.krylov, w.restart) if w.restart else w.krylov,
            "vcycle": "V(%d,%d) l1-Jacobi" % (w.nu, w.nu), "amg_precision": "fp32" if w.mixed else "fp64",
            "amg": "MIS-2 smoothed aggregation, P smoothed on the first %d levels, Galerkin refresh per Newton "
                   "iteration" % w.smooth_levels,
            "newton_rtol": 1e-8, "eta": 1e-7, "dt": w.dt, "schedule_steps": w.steps,
            "l2": "working set > 129 MB L2 (7-diagonal Jacobian alone 118 MB, FGMRES basis 1 GB)"}


class StepFailure(RuntimeError):
    def __init__(self, step, status, stats, done):
        super().__init__("step %d failed with status %d" % (step, status))
        self.step, self.status, self.stats, self.done = step, status, stats, done


def run_steps(ctx, pd, dts, count, opts, first=0, record=None):
    """Step the schedule count times (step m uses dt_{m mod len}); returns the per-step stats.

    record: a list of CUDA events, one recorded after each step on the current stream.
    A failing step raises StepFailure carrying its statistics and the steps done."""
    out = []
    for q in range(count):
        m = first + q
        s, st = ctx.step(pd, dts[m % len(dts)], opts, check_status=False)
        if record is not None:
            record[q].record()
        if s != 0:
            raise StepFailure(m, s, st, out)
        out.append(st)
    return out


def fp64_balance(peak_gbs, fp64_tflops):
    """Flops per byte where the FP64 FMA pipe and HBM take equal time."""
    return fp64_tflops * 1e12 / (peak_gbs * 1e9)


def roofline_of(name, ms, launches, nbytes, flops, fp64, peak_gbs, fp64_tflops, traffic):
    """A kernel placed on its roofline: HBM-bound when its algorithmic flops/byte lie
    below the FP64 balance point (FP32 kernels always), FP64-ALU-bound above it."""
    secs = ms / 1000.0
    gbs = nbytes / secs / 1e9 if secs > 0 else None
    tfl = flops / secs / 1e12 if secs > 0 else None
    intensity = flops / nbytes if nbytes > 0 else None
    bal = fp64_balance(peak_gbs, fp64_tflops)
    common = {"kernel": name, "launches": launches, "avg_launch_us": 1000.0 * ms / launches if launches else None,
              "algorithmic_bytes_per_launch": nbytes / launches if launches else None,
              "algorithmic_flops_per_launch": flops / launches if launches else None,
              "intensity_flop_per_byte": intensity, "fp64_balance_flop_per_byte": bal,
              "traffic": traffic, "hbm_frac": gbs / peak_gbs if gbs else None,
              "fp64_frac": tfl / fp64_tflops if (tfl and fp64) else None}
    if fp64 and intensity is not None and intensity > bal:
        return dict(common, bound="alu", achieved=tfl, peak=fp64_tflops, unit="TFLOP/s", frac=tfl / fp64_tflops,
                    peak_kind="measured FP64 FMA throughput (rich_measure_fma_peak, this run)")
    return dict(common, bound="hbm", achieved=gbs, peak=peak_gbs, unit="GB/s", frac=gbs / peak_gbs if gbs else None,
                peak_kind="measured (MEASURED_PEAKS.json hbm_gbs)")


# kernel name prefix -> (profile names that make it, runs in FP64 in the FP64 mode)
def _is_fp64_kernel(name, prec_fp64):
    if name in ("residual", "assemble", "stencil_spmv", "multidot", "orth_axpy", "orth_final", "fcg_update"):
        return True
    return prec_fp64


def profile_pass(rb, grid, soil, bc, w, ks, p0, dts, opts, prec, steps):
    """Every named launch of the first steps timed with CUDA events (an untimed pass of
    its own): per-kernel (launches, ms, algorithmic bytes, algorithmic flops)."""
    import torch
    lib = rb.load()
    ctx = rb.Context(grid, soil, bc, w.kmean, ks, precision=prec)
    pd = torch.tensor(p0, device="cuda")
    lib.rich_profile_stride(1)
    lib.rich_profile_kernel(b"*")
    run_steps(ctx, pd, dts, steps, opts)
    torch.cuda.synchronize()
    tab = rb.profile_table()
    lib.rich_profile_kernel(None)
    ctx.close()
    return tab


def run_ours(args):
    import ctypes
    import torch
    from paper_2112_05051_gb300 import richards as rb
    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    lib = rb.load()
    if args.tune_file and os.path.exists(args.tune_file):
        rb.autotune_load(open(args.tune_file).read())
    w, grid, soil, bc, ks, p0, dts = workload_setup(args.workload, args.grid)
    if args.amg_precision is not None:
        import dataclasses
        w = dataclasses.replace(w, mixed=args.amg_precision == "fp32")
    opts = newton_opts(rb, w)
    prec = rb.PREC_MIXED if w.mixed else rb.PREC_FP64
    K = args.steps

    # warm-up on a context of its own (kernels loaded, memory pool primed); destroyed after
    ctxw = rb.Context(grid, soil, bc, w.kmean, ks, precision=prec)
    pw = torch.tensor(p0, device="cuda")
    run_steps(ctxw, pw, dts, args.warmup, opts)
    torch.cuda.synchronize()
    ctxw.close()
    del pw

    # timed run: a fresh context from p0 over K steps of the schedule, AMG setup included
    rb.memory_peak(reset=True)
    torch.cuda.reset_peak_memory_stats()
    ctx = rb.Context(grid, soil, bc, w.kmean, ks, precision=prec)
    pd = torch.tensor(p0, device="cuda")
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    l0 = ctypes.c_longlong()
    l1 = ctypes.c_longlong()
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    lib.rich_kernel_launches(ctypes.byref(l0))
    e0.record()
    torch.cuda.nvtx.range_push("timed")  # profilers filter the timed steps by this range
    failure = None
    try:
        stats = run_steps(ctx, pd, dts, K, opts, record=marks)
    except StepFailure as f:  # a workload the method cannot solve: report where it stopped
        stats = f.done
        failure = {"step": f.step, "status": rb.ERRORS.get(f.status, str(f.status)),
                   "stats": {k: (round(v, 4) if isinstance(v, float) else v) for k, v in f.stats.as_dict().items()},
                   "p_range": [float(pd.min()), float(pd.max())]}
    torch.cuda.nvtx.range_pop()
    e1.record()
    torch.cuda.synchronize()
    if failure is not None:
        clk.stop()
        lib_used, _ = rb.memory_peak()
        ctx.close()
        print(json.dumps({"metric": "DOF*Newton-steps/s", "value": None, "unit": "DOF*Newton-steps/s",
                          "config": workload_config(w, grid), "failed": failure,
                          "steps_done": [x.newton_its for x in stats], "peak_device_memory_bytes": lib_used,
                          "amg_precision": "fp32" if prec == rb.PREC_MIXED else "fp64"}))
        return 1
    K = len(stats)
    lib.rich_kernel_launches(ctypes.byref(l1))
    if dist:
        dist.barrier()
    clocks = clk.stop()
    elapsed = e0.elapsed_time(e1) / 1000.0
    step_ms = [e0.elapsed_time(marks[0])] + [marks[q].elapsed_time(marks[q + 1]) for q in range(K - 1)]
    newton_its = sum(st.newton_its for st in stats)
    lin_its = sum(st.linear_its for st in stats)
    d = [st.as_dict() for st in stats]
    phases = {k: sum(x[k] for x in d) for k in ("ms_feval", "ms_jacobian", "ms_setup", "ms_linsol", "ms_total")}
    phases["ms_overhead"] = phases["ms_total"] - sum(phases[k] for k in ("ms_feval", "ms_jacobian", "ms_setup",
                                                                           "ms_linsol"))
    lib_used, lib_reserved = rb.memory_peak()
    peak_mem = {"library_pool_used_high_bytes": lib_used, "library_pool_reserved_high_bytes": lib_reserved,
                "torch_max_allocated_bytes": int(torch.cuda.max_memory_allocated())}
    p_fp64 = pd.clone() if prec == rb.PREC_FP64 else None
    ctx.close()
    work = float(grid.n) * newton_its
    elapsed, work = aggregate_over_ranks(dist, elapsed, work, "cuda")
    value = work / elapsed

    # end to end through the host-buffer entry point, a fresh context over the same steps
    e2e = None
    if not args.no_e2e:
        ctx2 = rb.Context(grid, soil, bc, w.kmean, ks, precision=prec)
        ph = torch.tensor(p0, dtype=torch.float64).pin_memory()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        its2 = 0
        for m in range(K):
            its2 += ctx2.step_host(ph, dts[m % len(dts)], opts).newton_its
        torch.cuda.synchronize()
        el2 = time.perf_counter() - t0
        work2, el2 = float(grid.n) * its2, el2
        el2, work2 = aggregate_over_ranks(dist, el2, work2, "cuda")
        e2e = {"value": work2 / el2, "unit": "DOF*Newton-steps/s", "h2d_bytes_per_step": 8 * grid.n,
               "d2h_bytes_per_step": 8 * grid.n, "newton_its": its2}
        ctx2.close()

    # the same steps with the FP32 AMG hierarchy and V-cycle (FP64 residual,
    # Jacobian, line search and outer Krylov): speed and deviation from FP64
    mixed = None
    if not args.no_mixed and prec == rb.PREC_FP64:
        ctx3 = rb.Context(grid, soil, bc, w.kmean, ks, precision=rb.PREC_MIXED)
        p3 = torch.tensor(p0, device="cuda")
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        f0.record()
        st3 = run_steps(ctx3, p3, dts, K, opts)
        f1.record()
        torch.cuda.synchronize()
        el3 = f0.elapsed_time(f1) / 1000.0
        its3 = sum(x.newton_its for x in st3)
        v3 = float(grid.n) * its3 / el3
        dev_end = float((p3 - p_fp64).abs().max() / p_fp64.abs().max())
        ctx3.close()
        # untimed lockstep replay: largest deviation of the mixed pressure from the FP64 one after any step
        ca = rb.Context(grid, soil, bc, w.kmean, ks, precision=rb.PREC_FP64)
        cb = rb.Context(grid, soil, bc, w.kmean, ks, precision=rb.PREC_MIXED)
        pa = torch.tensor(p0, device="cuda")
        pb = torch.tensor(p0, device="cuda")
        dev = 0.0
        for m in range(K):
            ca.step(pa, dts[m % len(dts)], opts)
            cb.step(pb, dts[m % len(dts)], opts)
            dev = max(dev, float((pb - pa).abs().max() / pa.abs().max()))
        ca.close()
        cb.close()
        mixed = {"value": v3, "unit": "DOF*Newton-steps/s", "speedup_vs_fp64": v3 / value if ws == 1 else None,
                 "newton_its": its3, "linear_its": sum(x.linear_its for x in st3), "fp64_newton_its": newton_its,
                 "fp64_linear_its": lin_its, "max_rel_dev_p_vs_fp64": dev, "rel_dev_p_at_end": dev_end,
                 "ms_per_step": 1000.0 * el3 / max(K, 1)}

    # per-kernel profile pass and the dominant kernel on its roofline
    peak_gbs, peak_kind = measured_peaks()
    fp64_tflops = rb.fma_peak_tflops(fp64=True)
    fp32_tflops = rb.fma_peak_tflops(fp64=False)
    roof, kernel_roofs = None, None
    if not args.no_profile:
        psteps = min(K, args.profile_steps)
        tab = profile_pass(rb, grid, soil, bc, w, ks, p0, dts, opts, prec, psteps)
        total = sum(v[1] for v in tab.values())
        rows = sorted(tab.items(), key=lambda kv: -kv[1][1])
        kernel_roofs = []
        for name, (cnt, kms, kb, kf) in rows[:12]:
            r = roofline_of(name, kms, cnt, kb, kf, _is_fp64_kernel(name, prec == rb.PREC_FP64), peak_gbs,
                            fp64_tflops, NCU_TRAFFIC_BYTES.get((w.name, name)))
            r["share_of_profiled_steps"] = kms / total if total else None
            r["profiled_steps"] = psteps
            kernel_roofs.append(r)
        roof = kernel_roofs[0] if kernel_roofs else None
        kernel_roofs = [{k: r[k] for k in ("kernel", "launches", "share_of_profiled_steps", "bound", "achieved",
                                           "peak", "unit",
                                           "frac", "intensity_flop_per_byte", "hbm_frac", "avg_launch_us")}
                        for r in kernel_roofs]
        if mixed is not None:  # the same pass on the FP32-AMG arm: its V-cycle kernels are FP32
            tab3 = profile_pass(rb, grid, soil, bc, w, ks, p0, dts, opts, rb.PREC_MIXED, psteps)
            tot3 = sum(v[1] for v in tab3.values())
            mixed["kernels_on_their_roofs"] = []
            for name, (cnt, kms, kb, kf) in sorted(tab3.items(), key=lambda kv: -kv[1][1])[:5]:
                r = roofline_of(name, kms, cnt, kb, kf, _is_fp64_kernel(name, False), peak_gbs, fp64_tflops, None)
                mixed["kernels_on_their_roofs"].append(
                    {"kernel": name, "share_of_profiled_steps": kms / tot3 if tot3 else None, "bound": r["bound"],
                     "frac": r["frac"], "hbm_frac": r["hbm_frac"], "avg_launch_us": r["avg_launch_us"]})

    # the paper's own problem (Sec. 6): 798 x 798 x 38 unknowns, mixed precision
    paper = None
    if not args.no_paper and ws == 1 and args.grid is None:
        try:
            paper = paper_run(rb, args.paper_steps)
        except Exception as e:
            paper = {"error": "%s: %s" % (type(e).__name__, e)}

    line = {"metric": "DOF*Newton-steps/s", "value": value, "unit": "DOF*Newton-steps/s", "n_gpus": ws,
            "steps": K, "warmup": args.warmup, "ms_per_step": 1000.0 * elapsed / max(K, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == rb.PREC_FP64 else "f64 outer, f32 AMG",
            "data": "synthetic", "config": workload_config(w, grid), "e2e": e2e,
            "gpu_launches": int(l1.value - l0.value), "clocks": clocks, "roofline": roof,
            "kernels_on_their_roofs": kernel_roofs,
            "measured_peaks": {"hbm_gbs": peak_gbs, "hbm_kind": peak_kind, "fp64_fma_tflops": fp64_tflops,
                               "fp32_fma_tflops": fp32_tflops,
                               "fp64_balance_flop_per_byte": fp64_balance(peak_gbs, fp64_tflops)},
            "autotuned_shapes": len(rb.autotune_table()),
            "autotune": [{"mode": m, "value_bytes": t, "rows_bin": nb, "mean_row": z, "sell_offered": so,
                          "choice": {rb.SELL_VARIANT8: "sell x8", rb.SELL_VARIANT2: "sell 2 lanes",
                                     rb.SELL_VARIANTP: "sell pipelined"}.get(g, "sell")
                          if g & rb.SELL_VARIANT else
                          ("%d lanes%s" % (g & 0xff, " x4" if g & rb.UNROLL else "")),
                          "us": us} for m, t, nb, z, so, g, us in rb.autotune_table()],
            "newton_its": newton_its, "linear_its": lin_its,
            "schedule_newton_its": [x.newton_its for x in stats],
            "latency_ms_per_time_step": {"p50": statistics.median(step_ms), "max": max(step_ms)},
            "fp32_amg": mixed, "paper_workload": paper,
            "peak_device_memory": peak_mem,
            "phase_ms": {k[3:]: round(v, 3) for k, v in phases.items()},
            "parallelism": "replicas" if ws > 1 else "single"}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = cpu_baseline(args.workload, args.cpu_budget,
                                                args.cpu_procs or min(16, os.cpu_count() or 1))
        except Exception as e:
            line["cpu_baseline"] = {"value": None, "error": "%s: %s" % (type(e).__name__, e)}
    if not args.no_serving and ws == 1:
        try:
            line["serving"] = serving_run(args, rb)
        except Exception as e:  # the main measurement stands on its own
            line["serving"] = {"error": "%s: %s" % (type(e).__name__, e)}
        try:
            line["serving_uniform"] = serving_uniform(args, rb)
        except Exception as e:
            line["serving_uniform"] = {"error": "%s: %s" % (type(e).__name__, e)}
    if rank == 0:
        print(json.dumps(line))
        if args.tune_file:
            with open(args.tune_file, "w") as f:
                f.write(rb.autotune_text())
    if dist:
        dist.destroy_process_group()
    return 0


def paper_run(rb, steps):
    """The paper's infiltration problem (Sec. 6) on its 800 x 800 x 40 node grid in mixed precision:
    DOF * Newton-steps / s over its first steps (CUDA events; setup included)."""
    import torch
    w, grid, soil, bc, ks, p0, dts = workload_setup("paper_infiltration")
    opts = newton_opts(rb, w)
    ctx = rb.Context(grid, soil, bc, w.kmean, ks, precision=rb.PREC_MIXED)
    pd = torch.tensor(p0, device="cuda")
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    st = run_steps(ctx, pd, dts, steps, opts)
    e1.record()
    torch.cuda.synchronize()
    el = e0.elapsed_time(e1) / 1000.0
    its = sum(x.newton_its for x in st)
    ctx.close()
    return {"workload": "paper_infiltration", "grid": [grid.nx, grid.ny, grid.nz], "dof": grid.n,
            "precision": "fp32 AMG, fp64 residual and FGMRES(10)", "steps": steps, "newton_its": its,
            "linear_its": sum(x.linear_its for x in st), "value": grid.n * its / el, "unit": "DOF*Newton-steps/s",
            "ms_per_step": 1000.0 * el / steps}


def main():
    if len(sys.argv) >= 2 and sys.argv[1] == "--oracle-sample":
        wl, n, budget, steps, warm = sys.argv[2], int(sys.argv[3]), float(sys.argv[4]), int(sys.argv[5]), int(sys.argv[6])
        res = oracle_sample_main(wl, budget, n=n, steps=steps or None, warmup=warm)
        res.pop("step_times", None)
        print(json.dumps(res))
        return 0
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.serving_only:
        from paper_2112_05051_gb300 import richards as rb
        rb.load()
        print(json.dumps({"serving": serving_run(args, rb), "serving_uniform": serving_uniform(args, rb)}))
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
