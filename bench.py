"""Throughput of the implicit theta-step on the adaptive polar mesh (one GB300 per rank).

Workload: the singular parabolic equation on the unit disk on the adaptive mesh --
m = 512 rings graded geometrically (ratio 1.03) toward r = 0 and r = 1, n = 1024
angles with node density 1 + 0.5 cos(theta - theta0), Crank-Nicolson, variable
dt_k = 1e-4 * 1.01^k over a 1000-level schedule (T ~ 209.6); manufactured solution
u = e^{-t}(1 - r^2)(1 + r cos theta).  Inputs are synthetic and seeded.

A bench step is one implicit theta-step (right-hand side, line factors, Krylov solve
to the FP64 tolerance, time-level update) of that schedule.  With K < 1000 the K steps
are spread evenly over the schedule, each starting from the manufactured solution at
its level (set outside the timed region); with K >= 1000 the schedule runs
consecutively.  L2 is flushed (a 512 MB write) before every timed step.

value  = grid-point updates (N per step) / device time of the K steps, summed over ranks
         (replicas: every rank advances its own copy; no collective on the data path);
         the headline path is the mixed one (FP32 inner solves, FP64 residual and update,
         same FP64 tolerance), the FP64 path is timed beside it on the same steps
e2e    = the same through the C ABI with the state copied in from pinned host memory
         and out to pinned host memory inside every timed step
roofline: the dominant kernel class's algorithmic bytes / its event-timed duration
cpu_baseline: the FP64 CPU oracle on a bounded sample of the same workload

--impl reference times the CPU oracle itself (the reference arm of this workload).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "grid-point-updates/s and HBM GB/s vs peak, mixed vs FP64 GPU at stated error"
UNIT = "grid-point-updates/s"
M_RINGS, N_ANGLES, K_SCHEDULE = 512, 1024, 1000
WORKLOAD = ("parabolic u_t = Lap u + f, adaptive polar mesh 512 x 1024 (r graded 1.03 "
            "to both ends, theta density 1 + 0.5 cos), Crank-Nicolson, dt_k = 1e-4 * 1.01^k, "
            "1000-level schedule")
FALLBACK_HBM_GBS = 6800.0

# ncu dram bytes (read + write) per launch of the dominant kernel class, from the
# capture summarised under profiles/; None until a capture of the current kernel exists
NCU_TRAFFIC = {}


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


# ------------------------------------------------------------------------- replicas
# With N ranks every rank advances its own replica (or its share of independent
# instances); nothing crosses ranks on the data path, only these scalar reductions of the
# timing and the update counts.
def shard(count, rank, world):
    """Independent instances of this rank: rank, rank + world, rank + 2 world, ..."""
    return list(range(rank, count, world))


def _reduce(dist, vals, op):
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(v) for v in vals], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=op)
    return [float(x) for x in t.tolist()]


def max_over_ranks(dist, v):
    """The slowest rank's time (v itself on one rank)."""
    return v if dist is None else _reduce(dist, [v], dist.ReduceOp.MAX)[0]


def sum_over_ranks(dist, vals):
    """Whole-job totals of per-rank counts."""
    return list(vals) if dist is None else _reduce(dist, vals, dist.ReduceOp.SUM)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms in the background."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        sm, smax, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.file.read().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.file.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": smax, "reasons": ["no samples"]}
        # median over the samples taken under load (clock above idle)
        hi = [s for s in sm if s >= 0.5 * max(sm)]
        return {"sm_mhz": statistics.median(hi), "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_problem(m=M_RINGS, n=N_ANGLES, K=K_SCHEDULE):
    import polar_inputs as pi
    return pi.config2(m=m, n=n, K=K)


def step_levels(K):
    """Schedule levels at which the K timed steps start."""
    if K >= K_SCHEDULE:
        return [k % K_SCHEDULE for k in range(K)], True
    return [int(math.floor(s * K_SCHEDULE / K)) for s in range(K)], False


# ------------------------------------------------------------------------- CPU oracle
def oracle_sample(budget_s=20.0, prob=None):
    """Times the FP64 CPU oracle on whole theta-steps of the workload (full mesh, steps
    spread over the schedule, each from the manufactured solution at its level) until
    about budget_s of CPU time has passed.  Returns (updates/s, steps, seconds)."""
    from oracle import polar_oracle as po
    prob = prob or make_problem()
    L, B = po.operator(prob)
    levels = [0, 500, 250, 750, 125, 625, 375, 875]
    done, t_used, upd = 0, 0.0, 0
    for k in levels:
        if done and t_used >= budget_s:
            break
        U = prob.exact(prob.t[k])
        dt = prob.t[k + 1] - prob.t[k]
        t0 = time.perf_counter()
        fo, go = po.source(prob, prob.t[k])
        fn, gn = po.source(prob, prob.t[k + 1])
        po.step(L, B, U, dt, prob.theta_w, fo, go, fn, gn)
        t_used += time.perf_counter() - t0
        upd += prob.N
        done += 1
    return upd / t_used, done, t_used


def run_reference(args):
    rank = env_int("RANK", 0)
    if rank != 0:
        return 0
    prob = make_problem()
    total = args.warmup + args.steps
    # each reference step is one oracle theta-step on a sample mesh whose size keeps
    # the whole run within about three minutes (one full-size step takes ~10-15 s)
    per_step = 150.0 / max(total, 1)
    scale = 1
    while scale < 8 and 13.0 / (scale * scale) > per_step:
        scale *= 2
    sample = make_problem(M_RINGS // scale, N_ANGLES // scale) if scale > 1 else prob
    from oracle import polar_oracle as po
    L, B = po.operator(sample)
    levels, _ = step_levels(args.steps)
    wl, _ = step_levels(max(args.warmup, 1))

    def one(k):
        U = sample.exact(sample.t[k])
        dt = sample.t[k + 1] - sample.t[k]
        fo, go = po.source(sample, sample.t[k])
        fn, gn = po.source(sample, sample.t[k + 1])
        po.step(L, B, U, dt, sample.theta_w, fo, go, fn, gn)

    for k in wl[:args.warmup]:
        one(k)
    t0 = time.perf_counter()
    for k in levels:
        one(k)
    el = time.perf_counter() - t0
    value = sample.N * len(levels) / el
    desc = (f"one FP64 oracle theta-step (sparse LU + one extended-precision refinement) per "
            f"bench step on the {sample.m} x {sample.n} version of the workload mesh, "
            f"levels spread over the schedule")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / len(levels),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "m": sample.m, "n": sample.n, "N": sample.N,
                       "sample_of": f"{M_RINGS} x {N_ANGLES}"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------- GPU arm
def run_native(args):
    import torch
    import paper_2509_15879_gb300 as P
    from paper_2509_15879_gb300 import driver

    world = env_int("WORLD_SIZE", 1)
    rank = env_int("RANK", 0)
    local = env_int("LOCAL_RANK", 0)
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU (the library has no CPU path)")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    prob = make_problem()
    stream = torch.cuda.current_stream()
    t_all = np.asarray(prob.t)
    W = prob.weight_table()
    exact = {}
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    levels, consecutive = step_levels(args.steps)

    def timed_run(precision, timers):
        """Warm-up, then the K timed steps; returns the measurements of this precision."""
        ctx = driver.create(prob, precision, stream=stream.cuda_stream)

        def set_level(k):
            if k not in exact:
                exact[k] = np.ascontiguousarray(prob.exact(t_all[k]))
            P.polar_set_state(ctx, exact[k], t_all[k])

        wl, _ = step_levels(max(args.warmup, 1))
        for k in wl[:args.warmup]:
            set_level(k)
            P.polar_advance(ctx, t_all[k:k + 2], prob.theta_w, W[k:k + 2])
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in levels]
        iters, refs, checkpoints = [], [], {}
        launches0 = P.polar_kernel_launches(ctx)
        if timers:
            P.polar_timing_enable(ctx, True)
            # the per-kernel pass runs the kernels eagerly (ncu cannot see kernels inside
            # conditional graph nodes); `ncu --profile-from-start off` captures this range
            torch.cuda.profiler.start()
        barrier()
        wall0 = time.perf_counter()
        for s, k in enumerate(levels):
            if not consecutive or k == 0:
                set_level(k)
            flush.fill_(float(s))
            ev[s][0].record(stream)
            st, _ = P.polar_advance(ctx, t_all[k:k + 2], prob.theta_w, W[k:k + 2])
            ev[s][1].record(stream)
            iters.append(st[0]["iters"])
            refs.append(st[0]["refinements"])
            if consecutive and not timers and (k + 1) % 100 == 0:
                checkpoints[k + 1] = P.polar_get_state(ctx)[0]
        barrier()
        if timers:
            torch.cuda.profiler.stop()
        wall = time.perf_counter() - wall0
        launches = P.polar_kernel_launches(ctx) - launches0
        kstats = P.polar_timing_query(ctx) if timers else {}
        P.polar_timing_enable(ctx, False)
        dev_ms = max_over_ranks(dist, sum(a.elapsed_time(b) for a, b in ev))
        U_last, t_last = P.polar_get_state(ctx)
        return dict(ctx=ctx, dev_ms=dev_ms, wall=wall, launches=launches, kstats=kstats,
                    iters=float(np.mean(iters)), refs=float(np.mean(refs)), U=U_last, t=t_last,
                    set_level=set_level, checkpoints=checkpoints)

    precision = P.POLAR_MIXED if args.precision == "mixed" else P.POLAR_FP64
    other = P.POLAR_FP64 if precision == P.POLAR_MIXED else P.POLAR_MIXED
    clocks = ClockSampler(local)
    clocks.start()
    main = timed_run(precision, False)
    clk = clocks.stop()
    # per-kernel CUDA events on a second pass over the same steps (kept out of the
    # headline run, whose launch rate the event records would perturb)
    prof = timed_run(precision, True)
    comp = timed_run(other, False) if args.compare else None
    ctx, dev_ms = main["ctx"], main["dev_ms"]
    kstats = prof["kstats"]
    set_level = main["set_level"]
    U_last, t_last = main["U"], main["t"]
    launches, wall = main["launches"], main["wall"]
    iters, refs = [main["iters"]], [main["refs"]]
    err_exact = float(np.max(np.abs(U_last - prob.exact(t_last))) /
                      np.max(np.abs(prob.exact(t_last))))
    err_cp = {k: float(np.max(np.abs(U - prob.exact(t_all[k]))) / np.max(np.abs(prob.exact(t_all[k]))))
              for k, U in sorted(main["checkpoints"].items())}
    updates = prob.N * len(levels) * world
    value = updates / (dev_ms * 1e-3)
    compare = None
    if comp is not None:
        diff = float(np.max(np.abs(main["U"] - comp["U"])) / np.max(np.abs(comp["U"])))
        # relative max-norm difference at the checkpoints t_100, t_200, ... (consecutive runs)
        cp = {k: float(np.max(np.abs(main["checkpoints"][k] - comp["checkpoints"][k])) /
                       np.max(np.abs(comp["checkpoints"][k])))
              for k in sorted(main["checkpoints"]) if k in comp["checkpoints"]}
        compare = {"precision": "fp64" if other == P.POLAR_FP64 else "mixed",
                   "value": updates / (comp["dev_ms"] * 1e-3), "ms_per_step": comp["dev_ms"] / len(levels),
                   "krylov_iters_per_step": comp["iters"], "refinements_per_step": comp["refs"],
                   "speedup_of_headline": comp["dev_ms"] / dev_ms,
                   "rel_max_diff_final_state": diff,
                   "rel_max_diff_at_checkpoints": cp}

    # ---- end to end: pinned host state in, pinned host state out, every step
    ke = sorted(set(levels))[:: max(1, len(set(levels)) // 20)][:20]
    host_in = {k: torch.from_numpy(np.ascontiguousarray(prob.exact(t_all[k]))).pin_memory()
               for k in ke}
    host_out = torch.empty(prob.N, dtype=torch.float64).pin_memory()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e_ms = 0.0
    for k in ke:
        flush.fill_(1.0)
        e0.record(stream)
        P.polar_set_state(ctx, host_in[k], t_all[k])
        P.polar_advance(ctx, t_all[k:k + 2], prob.theta_w, W[k:k + 2])
        P.polar_get_state(ctx, host_out)
        e1.record(stream)
        e1.synchronize()
        e_ms += e0.elapsed_time(e1)
    e_ms = max_over_ranks(dist, e_ms)
    e2e_value = prob.N * len(ke) * world / (e_ms * 1e-3)

    # ---- roofline of the dominant kernel class
    peak, peak_src = measured_peaks()
    dom = max(kstats.items(), key=lambda kv: kv[1]["ms"]) if kstats else None
    roof = None
    if dom is not None:
        name, d = dom
        achieved = d["bytes"] / (d["ms"] * 1e-3) / 1e9
        per_launch = d["bytes"] / max(d["launches"], 1)
        roof = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak,
                "peak_source": peak_src, "unit": "GB/s", "frac": achieved / peak,
                "traffic": NCU_TRAFFIC.get(name), "algorithmic_bytes_per_launch": per_launch,
                "avg_launch_us": 1e3 * d["ms"] / max(d["launches"], 1),
                "share_of_step": d["ms"] / prof["dev_ms"],
                "timing": "CUDA events around every launch, second pass over the same steps"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dev_ms / len(levels),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if precision == P.POLAR_FP64 else "f32+f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "m": prob.m, "n": prob.n, "N": prob.N,
                       "precision": args.precision,
                       "levels": "consecutive" if consecutive else
                                 f"{len(levels)} steps spread over the 1000-level schedule",
                       "l2": "flushed (512 MB write) before every timed step",
                       "parallelism": f"replicas x{world}"},
            "krylov_iters_per_step": float(np.mean(iters)),
            "refinements_per_step": float(np.mean(refs)),
            "rel_err_vs_manufactured_last_step": err_exact,
            "rel_err_vs_manufactured_at_checkpoints": err_cp,
            "compare": compare,
            "wall_s": wall,
            "gpu_launches": int(launches),
            "clocks": clk,
            "roofline": roof,
            "kernels": {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                            "GBps": round(v["bytes"] / max(v["ms"], 1e-9) / 1e6, 1)}
                        for k, v in sorted(kstats.items(), key=lambda kv: -kv[1]["ms"])},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": prob.N * 8,
                    "d2h_bytes_per_step": prob.N * 8, "steps": len(ke)}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, nsteps, secs = oracle_sample(args.cpu_budget, prob)
        line["cpu_baseline"] = {
            "value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{nsteps} full-size theta-steps of the workload ({secs:.1f} s; sparse LU "
                      f"+ one extended-precision refinement, single-threaded SuperLU)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------------- batch
def run_batch(args):
    """The 256-instance sweep: continuity equation on uneven adaptive meshes (m log-uniform
    in [64, 1024], n in [128, 2048], D amplitude in [0.2, 5], Peclet in [0.1, 20]), 500-level
    time stretch each, advanced together: one CUDA graph per step holds a step of every
    instance.  value = sum of N_i x steps / device time."""
    import torch
    import polar_inputs as pi
    import paper_2509_15879_gb300 as P
    from paper_2509_15879_gb300 import driver
    world = env_int("WORLD_SIZE", 1)
    rank = env_int("RANK", 0)
    local = env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    K_sched = 500
    count = args.instances
    # replicas: rank r takes instances r, r + world, ... (independent instances, no collective)
    mine = shard(count, rank, world)
    t0 = time.perf_counter()
    probs = [pi.config4_instance(i, K=K_sched) for i in mine]
    gen_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    precision = P.POLAR_MIXED if args.precision == "mixed" else P.POLAR_FP64

    def run(prec):
        ctxs = [driver.create(p, prec, stream=stream.cuda_stream) for p in probs]
        batch = P.polar_batch_create(ctxs, stream.cuda_stream)
        W = max(args.warmup, 1)
        driver.batch_advance(batch, probs, 0, W)
        for c, p in zip(ctxs, probs):  # back to the initial state for the timed steps
            P.polar_set_state(c, p.u0, p.t[0])
        K = min(args.steps, K_sched)
        clocks = ClockSampler(local)
        clocks.start()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        launches0 = sum(P.polar_kernel_launches(c) for c in ctxs)
        e0.record(stream)
        stats, _ = driver.batch_advance(batch, probs, 0, K, check=False)
        e1.record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        ms = max_over_ranks(dist, e0.elapsed_time(e1))
        states = [P.polar_get_state(c)[0] for c in ctxs]
        done = [sum(1 for s in row if s["status"] == 0) for row in stats]
        failed = [mine[i] for i, row in enumerate(stats) if any(s["status"] != 0 for s in row)]
        ok = [s for row in stats for s in row if s["status"] == 0]
        iters = float(np.mean([s["iters"] for s in ok])) if ok else 0.0
        # only the steps an instance completed count as updates (a failed step halts the
        # rest of that instance's schedule; its state stays at the last committed level)
        updates = sum_over_ranks(dist, [sum(p.N * d for p, d in zip(probs, done))])[0]
        launches = sum(P.polar_kernel_launches(c) for c in ctxs) - launches0
        return ms, K, states, iters, clk, launches, updates, failed

    ms, K, st_main, iters, clk, launches, updates, failed = run(precision)
    pts = sum_over_ranks(dist, [sum(p.N for p in probs)])[0]
    value = updates / (ms * 1e-3)
    compare = None
    if args.compare:
        other = P.POLAR_FP64 if precision == P.POLAR_MIXED else P.POLAR_MIXED
        ms2, _, st2, it2, _, _, up2, failed2 = run(other)
        bad = set(failed) | set(failed2)
        diff = max([float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
                    for i, a, b in zip(mine, st_main, st2) if i not in bad] or [0.0])
        compare = {"precision": "fp64" if other == P.POLAR_FP64 else "mixed",
                   "value": up2 / (ms2 * 1e-3), "ms_per_step": ms2 / K,
                   "krylov_iters_per_step": it2, "speedup_of_headline": ms2 / ms,
                   "failed_instances": failed2,
                   "max_rel_diff_final_states": diff}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": ms / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if precision == P.POLAR_FP64 else "f32+f64", "data": "synthetic",
            "config": {"workload": f"batched sweep: {count} continuity instances, m in [64, 1024], "
                                   f"n in [128, 2048], 500-level time stretch; one CUDA graph "
                                   f"per step for all instances", "instances": len(probs),
                       "sum_N": pts, "precision": args.precision,
                       "l2": "inputs larger than L2 (several GB of instance data)",
                       "parallelism": f"replicas x{world}"},
            "krylov_iters_per_step": iters, "failed_instances": failed, "compare": compare,
            "gpu_launches": int(launches),
            "clocks": clk, "setup_s": gen_s}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------------- profiling
def run_profile_step(args):
    """One eager theta-step of a named workload inside a CUDA profiler range, after the
    autotuner and a warm-up step, with per-kernel CUDA-event times (for
    `ncu --profile-from-start off`).  Workloads: c2 (the bench workload), c3 (continuity
    2048 x 4096, 2000-level time stretch), c5 (continuity 8192 x 16384 graded to r = 1,
    theta = 0.6, 200 levels).  The step is the third level of the schedule."""
    import torch
    import polar_inputs as pi
    import paper_2509_15879_gb300 as P
    from paper_2509_15879_gb300 import driver
    prob = {"c2": make_problem, "c3": pi.config3, "c5": pi.config5}[args.workload]()
    precision = P.POLAR_MIXED if args.precision == "mixed" else P.POLAR_FP64
    t = np.asarray(prob.t)
    W = prob.weight_table()
    ctx = driver.create(prob, precision)
    P.polar_advance(ctx, t[0:2], prob.theta_w, W[0:2])   # autotuner + graph
    P.polar_timing_enable(ctx, True)
    P.polar_advance(ctx, t[1:3], prob.theta_w, W[1:3])
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    st, _ = P.polar_advance(ctx, t[2:4], prob.theta_w, W[2:4])
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    q = P.polar_timing_query(ctx)
    print(json.dumps({"workload": args.workload, "m": prob.m, "n": prob.n,
                      "precision": args.precision, "step": st[0],
                      "kernels": {k: {"launches": v["launches"], "us_per_launch":
                                      round(1e3 * v["ms"] / max(v["launches"], 1), 2),
                                      "GBps": round(v["bytes"] / max(v["ms"], 1e-9) / 1e6, 1)}
                                  for k, v in sorted(q.items(), key=lambda kv: -kv[1]["ms"])}}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="mixed",
                    help="headline path; --compare 1 also times the other one")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--compare", type=int, default=1,
                    help="also time the other precision on the same steps")
    ap.add_argument("--workload", choices=["c2", "batch", "c3", "c5"], default="c2",
                    help="c2: the timed workload; batch: the 256-instance sweep; c3/c5: only "
                         "with --profile-step")
    ap.add_argument("--profile-step", action="store_true",
                    help="run one eager step of --workload inside a profiler range")
    ap.add_argument("--instances", type=int, default=256)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_step:
        return run_profile_step(args)
    if args.workload in ("c3", "c5"):
        ap.error("--workload c3/c5 needs --profile-step")
    if args.workload == "batch":
        return run_batch(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
