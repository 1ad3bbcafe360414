"""Throughput of the implicit theta-step on the adaptive polar mesh (one GB300 per rank).

Default workload (the largest single-GPU configuration of the benchmark): the continuity
(drift-diffusion) equation n_t = div(D grad n - v n) + G - n on the unit disk, m = 8192
rings graded geometrically (ratio 1.03, capped) toward r = 1, n = 16384 angles with node
density 1 + 0.5 cos(theta - theta0) (N = 134,217,729 unknowns, 1.07 GB per FP64 field),
D = exp(ln 2 * 8 seeded Fourier modes) in [0.5, 2], v = -grad(phi) scaled to cell Peclet 10,
manufactured solution with a sharp layer at r = 1, theta = 0.6 over the 200-level time
stretch t_k = sin((k/200)^1.5 pi/2).  Inputs are synthetic and seeded.  Other workloads
(--workload): c3 (continuity 2048 x 4096, Crank-Nicolson, 2000 levels), c2 (parabolic
512 x 1024, dt_k = 1e-4 * 1.01^k, 1000 levels), batch (the 256-instance sweep).

A bench step is one implicit theta-step (right-hand side, line factors, Krylov solves to
the FP64 tolerance, time-level update) at a level of the schedule; the K timed steps are
spread evenly over the schedule, each starting from the manufactured solution at its level
(set outside the timed region).  c2 with K >= 1000 runs the schedule consecutively.

value  = grid-point updates (N per step) / device time of the K steps, summed over ranks
         (replicas: every rank advances its own copy; no collective on the data path);
         the headline path is the mixed one (FP32 inner solves, FP64 residual and update,
         same FP64 tolerance), the FP64 path is timed beside it on the same steps
e2e    = the same through the C ABI with the state copied in from pinned host memory and
         out to pinned host memory inside every timed step
err_vs_oracle: per precision, against the FP64 CPU oracle on the same steps (element by
         element where the oracle can solve the workload's step, else the oracle's
         step equation on sampled rows)
roofline: the dominant kernel class's algorithmic bytes / its event-timed duration
cpu_baseline: the FP64 CPU oracle on a bounded sample of the same workload, on every
         host core (independent steps in parallel) and on one core

--impl reference times the CPU oracle itself (the reference arm of this workload).
"""
import argparse
import json
import math
import multiprocessing as mp
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
FALLBACK_HBM_GBS = 6800.0

# Workloads: generator (polar_inputs), schedule length, description, the mesh of the
# oracle's bounded sample, and how the oracle checks the GPU's steps ("full": the oracle
# solves the same step; "rows": the oracle's step equation on sampled rows).
WORKLOADS = {
    "c5": dict(gen="config5", K=200, sample=(256, 512), check="rows",
               desc="continuity n_t = div(D grad n - v n) + G - n, adaptive polar mesh "
                    "8192 x 16384 (r graded 1.03 toward r = 1, theta density 1 + 0.5 cos), "
                    "D in [0.5, 2] (8 Fourier modes), cell Peclet 10, theta = 0.6, "
                    "200-level time stretch"),
    "c3": dict(gen="config3", K=2000, sample=(256, 512), check="rows",
               desc="continuity, adaptive polar mesh 2048 x 4096 (r graded 1.03 to both "
                    "ends), D in [0.5, 2], cell Peclet 10, Crank-Nicolson, 2000-level time "
                    "stretch"),
    "c1": dict(gen="config1", K=100, sample=(None, None), check="full",
               desc="parabolic u_t = Lap u + f, uniform polar mesh 32 x 64, Crank-Nicolson, "
                    "dt = 0.01, 100 steps to T = 1 (separable: the direct FFT-in-theta solve)"),
    "c2": dict(gen="config2", K=1000, sample=(256, 512), check="full",
               desc="parabolic u_t = Lap u + f, adaptive polar mesh 512 x 1024 (r graded "
                    "1.03 to both ends, theta density 1 + 0.5 cos), Crank-Nicolson, "
                    "dt_k = 1e-4 * 1.01^k, 1000-level schedule"),
}

# ncu dram bytes (read + write) per launch of the dominant kernel class, from the capture
# summarised under profiles/, keyed by (workload, kernel class); absent until a capture of
# the current kernel exists.  The 8192 x 16384 entry: the FP64 level-0 even-ring
# post-smoothing captured on the same recipe at 2048 x 4096 (392.2 MB read + 34.3 MB
# written; algorithmic 403 MB), scaled by the 16x level-0 points of the full mesh.
NCU_TRAFFIC = {("c5", "ring_post_even@L0"): 426.5e6 * 16}

# FP64 arithmetic rate of the GB300s: 528 G FMA/s from a probe of independent FMA
# chains on every SM (the nominal figure is 1.25 TFLOP/s)
FP64_PEAK_TFLOPS = 1.056


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


def make_problem(workload, m=None, n=None):
    """The workload's problem (full size, or the same recipe on an m x n mesh)."""
    import polar_inputs as pi
    w = WORKLOADS[workload]
    gen = getattr(pi, w["gen"])
    return gen() if m is None else gen(m=m, n=n, K=w["K"])


def step_levels(K_sched, K):
    """Schedule levels at which K steps start (spread evenly), and whether they run the
    schedule consecutively (K >= the schedule length)."""
    if K >= K_sched:
        return [k % K_sched for k in range(K)], True
    return [int(math.floor(s * K_sched / K)) for s in range(K)], False


def rel_max(a, b):
    return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1e-300))


# ------------------------------------------------------------------------- CPU oracle
# The oracle runs in worker processes started with `spawn` (never forked from a process
# that holds a CUDA context).  A worker builds the sample problem and its operator once
# (initializer) and then times whole theta-steps: right-hand side, sparse LU of the step's
# matrix, solve and the extended-precision refinement.
_W = {}


def _oracle_init(workload, m, n):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle import polar_oracle as po
    prob = make_problem(workload, m, n) if m else make_problem(workload)
    _W.update(prob=prob, po=po, op=po.operator(prob))


def _oracle_step(k):
    """One oracle theta-step from the manufactured state at level k; returns
    (unknowns, seconds, new state or None)."""
    prob, po = _W["prob"], _W["po"]
    L, B = _W["op"]
    U = prob.exact(prob.t[k])
    dt = prob.t[k + 1] - prob.t[k]
    t0 = time.perf_counter()
    fo, go = po.source(prob, prob.t[k])
    fn, gn = po.source(prob, prob.t[k + 1])
    Un = po.step(L, B, U, dt, prob.theta_w, fo, go, fn, gn)
    return prob.N, time.perf_counter() - t0, Un


def _oracle_step_timing(k):
    N, sec, _ = _oracle_step(k)
    return N, sec


def _noop(_):
    return os.getpid()


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_pool(workload, m, n, cores):
    """A spawn pool of `cores` single-threaded oracle workers on the m x n sample
    (m = None: the full workload), initialised before it is returned."""
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(cores, initializer=_oracle_init, initargs=(workload, m, n))
    pool.map(_noop, range(4 * cores), chunksize=1)
    return pool


def oracle_sample(pool, cores, K_sched, budget_s, min_rounds=1):
    """Rounds of `cores` independent oracle steps (levels spread over the schedule), one
    per core, until about budget_s of wall time has passed.  Returns the all-cores rate,
    the single-core rate (updates / summed per-step seconds), the steps and the wall."""
    levels, _ = step_levels(K_sched, 8 * cores)
    done, upd, busy = 0, 0, 0.0
    t0 = time.perf_counter()
    rounds = 0
    while rounds < min_rounds or time.perf_counter() - t0 < budget_s:
        batch = [levels[(done + i) % len(levels)] for i in range(cores)]
        for N, sec in pool.map(_oracle_step_timing, batch, chunksize=1):
            upd += N
            busy += sec
        done += cores
        rounds += 1
    wall = time.perf_counter() - t0
    return upd / wall, upd / busy, done, wall


def run_reference(args):
    rank = env_int("RANK", 0)
    if rank != 0:
        return 0
    if args.workload not in WORKLOADS:
        print(json.dumps({"impl": "reference", "unavailable":
                          f"no oracle sample is defined for --workload {args.workload}"}))
        return 0
    w = WORKLOADS[args.workload]
    cores = host_cores()
    m, n = w["sample"]
    pool = oracle_pool(args.workload, m, n, cores)
    if m is None:  # the sample is the whole workload
        full = make_problem(args.workload)
        m, n = full.m, full.n
    levels, _ = step_levels(w["K"], 8 * cores)
    # one bench step = one oracle theta-step on every host core (levels spread over the
    # schedule) on the m x n sample of the workload
    rounds = args.warmup + args.steps
    t_steps, upd = [], 0
    for r in range(rounds):
        batch = [levels[(r * cores + i) % len(levels)] for i in range(cores)]
        t0 = time.perf_counter()
        res = pool.map(_oracle_step_timing, batch, chunksize=1)
        if r >= args.warmup:
            t_steps.append(time.perf_counter() - t0)
            upd += sum(N for N, _ in res)
    pool.close()
    pool.join()
    el = sum(t_steps)
    value = upd / el
    desc = (f"per bench step, one FP64 oracle theta-step (sparse LU + one extended-precision "
            f"refinement) on each of the {cores} host cores, on the {m} x {n} version of the "
            f"workload's mesh, levels spread over the schedule")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": w["desc"], "m": m, "n": n, "N": m * n + 1,
                       "sample_of": args.workload},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def sample_rows(prob, count=20000, seed=15879):
    """The origin, rings 1, 2, m-1 and m at 64 spread angles, and random cells."""
    m, n = prob.m, prob.n
    rng = np.random.default_rng(seed)
    js = np.linspace(0, n - 1, 64).astype(np.int64)
    special = [0]
    for i in (1, 2, m - 1, m):
        special.extend(1 + js * m + (i - 1))
    return np.unique(np.concatenate([special, rng.integers(1, prob.N, count)]))


def step_residual_rows(prob, rows, k, U_old, U_new):
    """max_i |(e - A U_new)_i| / A_ii / max|U_new| over `rows`, A and e of the oracle
    (its rows built from those cells' faces alone; extended-precision products)."""
    from oracle import polar_oracle as po
    L, B = po.conservative_operator(prob, rows)
    fo, go = po.source(prob, prob.t[k])
    fn, gn = po.source(prob, prob.t[k + 1])
    res = po.step_residual(L, B, U_old, U_new, prob.t[k + 1] - prob.t[k], prob.theta_w,
                           fo, go, fn, gn, rows)
    return float(np.max(np.abs(res)) / np.max(np.abs(U_new)))


# ------------------------------------------------------------------------- GPU arm
def run_native(args):
    import torch
    import paper_2509_15879_gb300 as P
    from paper_2509_15879_gb300 import driver

    world = env_int("WORLD_SIZE", 1)
    rank = env_int("RANK", 0)
    local = env_int("LOCAL_RANK", 0)
    w = WORKLOADS[args.workload]
    K_sched = w["K"]
    # the oracle's workers start (spawn) before this process touches the GPU
    cores = host_cores()
    pool = None
    want_cpu = rank == 0 and world == 1 and not args.no_cpu_baseline
    if want_cpu:
        pool = oracle_pool(args.workload, *w["sample"], cores)
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

    t_setup = time.perf_counter()
    prob = make_problem(args.workload)
    setup_s = time.perf_counter() - t_setup
    stream = torch.cuda.current_stream()
    t_all = np.asarray(prob.t)
    W = prob.weight_table()
    levels, consecutive = step_levels(K_sched, args.steps)
    big = prob.N * 8 > 256 * 1024 * 1024      # one FP64 field alone is larger than L2
    flush = None if big else torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32,
                                         device="cuda")
    host_u = torch.empty(prob.N, dtype=torch.float64).pin_memory()

    def exact_into(k, out):
        np.copyto(out.numpy(), prob.exact(t_all[k]))
        return out

    def timed_run(precision, timers, steps=None):
        """Warm-up, then the timed steps; returns the measurements of this precision."""
        ctx = driver.create(prob, precision, stream=stream.cuda_stream)

        def set_level(k):
            P.polar_set_state(ctx, exact_into(k, host_u), t_all[k])

        lv = levels if steps is None else levels[:steps]
        wl, _ = step_levels(K_sched, max(args.warmup, 1))
        for k in wl[:args.warmup]:
            set_level(k)
            P.polar_advance(ctx, t_all[k:k + 2], prob.theta_w, W[k:k + 2])
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in lv]
        stats = []
        launches0 = P.polar_kernel_launches(ctx)
        if timers:
            # the per-kernel pass runs the kernels eagerly (ncu does not see kernels inside
            # conditional graph nodes); `ncu --profile-from-start off` captures this range
            P.polar_timing_enable(ctx, True)
            torch.cuda.profiler.start()
        barrier()
        wall0 = time.perf_counter()
        for s, k in enumerate(lv):
            if not consecutive or k == 0:
                set_level(k)
            if flush is not None:
                flush.fill_(float(s))
            ev[s][0].record(stream)
            st, _ = P.polar_advance(ctx, t_all[k:k + 2], prob.theta_w, W[k:k + 2])
            ev[s][1].record(stream)
            stats.append(st[0])
        barrier()
        if timers:
            torch.cuda.profiler.stop()
        wall = time.perf_counter() - wall0
        launches = P.polar_kernel_launches(ctx) - launches0
        kstats = P.polar_timing_query(ctx) if timers else {}
        P.polar_timing_enable(ctx, False)
        dev_ms = max_over_ranks(dist, sum(a.elapsed_time(b) for a, b in ev))
        return dict(ctx=ctx, dev_ms=dev_ms, wall=wall, launches=launches, kstats=kstats,
                    stats=stats, steps=len(lv), set_level=set_level)

    def mean(stats, key):
        return float(np.mean([s[key] for s in stats]))

    def accuracy_states(run, acc_levels):
        """The state after one step from each accuracy level (host copies)."""
        out = {}
        for k in acc_levels:
            run["set_level"](k)
            st, _ = P.polar_advance(run["ctx"], t_all[k:k + 2], prob.theta_w, W[k:k + 2])
            assert st[0]["status"] == 0, st[0]
            out[k] = P.polar_get_state(run["ctx"])[0]
        return out

    precision = P.POLAR_MIXED if args.precision == "mixed" else P.POLAR_FP64
    other = P.POLAR_FP64 if precision == P.POLAR_MIXED else P.POLAR_MIXED
    name_of = {P.POLAR_MIXED: "mixed", P.POLAR_FP64: "fp64"}
    acc_levels = sorted(set(levels[:1] + levels[len(levels) // 2:len(levels) // 2 + 1]))
    # the oracle's full-size steps at the accuracy levels run on the host cores meanwhile
    full_oracle = None
    if w["check"] == "full" and want_cpu:
        pool_full = mp.get_context("spawn").Pool(len(acc_levels), initializer=_oracle_init,
                                                 initargs=(args.workload, None, None))
        full_oracle = (pool_full, pool_full.map_async(_oracle_step, acc_levels, chunksize=1))

    clocks = ClockSampler(local)
    clocks.start()
    main = timed_run(precision, False)
    clk = clocks.stop()
    acc = {name_of[precision]: accuracy_states(main, acc_levels)}
    # per-kernel CUDA events on a pass of its own over the first steps (kept out of the
    # headline run, whose launch rate the event records would perturb)
    prof = timed_run(precision, True, steps=min(len(levels), 4))
    del prof["ctx"]
    comp = None
    if args.compare:
        comp = timed_run(other, False)
        acc[name_of[other]] = accuracy_states(comp, acc_levels)
        del comp["ctx"]
    ctx, dev_ms = main["ctx"], main["dev_ms"]
    kstats = prof["kstats"]
    updates = prob.N * len(levels) * world
    value = updates / (dev_ms * 1e-3)
    compare = None
    if comp is not None:
        compare = {"precision": name_of[other],
                   "value": updates / (comp["dev_ms"] * 1e-3),
                   "ms_per_step": comp["dev_ms"] / len(levels),
                   "krylov_iters_per_step": mean(comp["stats"], "iters"),
                   "refinements_per_step": mean(comp["stats"], "refinements"),
                   "speedup_of_headline": comp["dev_ms"] / dev_ms,
                   "rel_max_diff_mixed_vs_fp64": {
                       str(k): rel_max(acc["mixed"][k], acc["fp64"][k]) for k in acc_levels}}

    # ---- accuracy against the oracle, per precision, on the steps from acc_levels
    err = {"levels": acc_levels}
    if w["check"] == "full" and full_oracle is not None:
        pool_full, res = full_oracle
        ref = {k: r[2] for k, r in zip(acc_levels, res.get())}
        pool_full.close()
        pool_full.join()
        err["kind"] = ("relative max-norm difference from the oracle's step (sparse LU + "
                       "extended-precision refinement) from the same state; v_weighted_l2: "
                       "the same difference in the L2 norm weighted by the control volumes")
        from oracle import polar_oracle as po
        V = po.Geometry(prob.r, prob.theta).V
        for nm, states in acc.items():
            err[nm] = {str(k): rel_max(states[k], ref[k]) for k in acc_levels}
            err[nm + "_v_weighted_l2"] = {
                str(k): float(np.sqrt(np.sum(V * (states[k] - ref[k]) ** 2) /
                                      np.sum(V * ref[k] ** 2))) for k in acc_levels}
    elif w["check"] == "rows":
        rows = sample_rows(prob)
        err["kind"] = (f"Jacobi-scaled residual max|(e - A U)_i| / A_ii / max|U| of the GPU's "
                       f"new level in the oracle's step equation, on {len(rows)} sampled rows "
                       f"(origin, rings 1, 2, m-1, m, random cells); bar 3e-14")
        for nm, states in acc.items():
            err[nm] = {str(k): step_residual_rows(prob, rows, k, prob.exact(t_all[k]), states[k])
                       for k in acc_levels}

    # ---- end to end: pinned host state in, pinned host state out, every step
    # eight of the timed levels, spread over them (the same mix of step costs)
    ke = [levels[(s * len(levels)) // min(len(levels), 8)] for s in range(min(len(levels), 8))]
    host_out = torch.empty(prob.N, dtype=torch.float64).pin_memory()
    host_in = [exact_into(k, torch.empty(prob.N, dtype=torch.float64).pin_memory())
               for k in ke[:2]]
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e_ms = 0.0
    for s, k in enumerate(ke):
        if s >= 2:
            exact_into(k, host_in[s % 2])
        if flush is not None:
            flush.fill_(1.0)
        e0.record(stream)
        P.polar_set_state(ctx, host_in[s % 2] if s >= 2 else host_in[s], t_all[k])
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
                "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src ==
                "measured" else peak_src, "unit": "GB/s", "frac": achieved / peak,
                "traffic": NCU_TRAFFIC.get((args.workload, name)),
                "algorithmic_bytes_per_launch": per_launch,
                "avg_launch_us": 1e3 * d["ms"] / max(d["launches"], 1),
                "share_of_step": d["ms"] / prof["dev_ms"],
                "timing": "CUDA events around every launch on the context's stream, eager "
                          "pass over the first timed steps"}
        if d.get("flops") and not name.endswith(".f32"):
            # the FP64 kernels are co-bound by GB300's FP64 pipe: their arithmetic rate
            # (flops per point as the kernel's source performs them, FMA = 2) against the
            # FP64 FMA rate measured on the GB300s
            tf = d["flops"] / (d["ms"] * 1e-3) / 1e12
            roof["fp64"] = {"achieved": tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                            "frac": tf / FP64_PEAK_TFLOPS,
                            "peak_source": "measured FP64 FMA probe, 528 G FMA/s (nominal "
                                           "1.25 TFLOP/s)",
                            "flops_per_launch": d["flops"] / max(d["launches"], 1)}

    stats = main["stats"]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dev_ms / len(levels),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if precision == P.POLAR_FP64 else "f32+f64",
            "data": "synthetic",
            "config": {"workload": w["desc"], "m": prob.m, "n": prob.n, "N": prob.N,
                       "precision": args.precision,
                       "levels": "consecutive" if consecutive else
                                 f"{len(levels)} steps spread over the {K_sched}-level schedule, "
                                 f"each from the manufactured state at its level",
                       "l2": ("inputs larger than L2 (1.07 GB per FP64 field)" if big else
                              "flushed (512 MB write) before every timed step"),
                       "parallelism": f"replicas x{world}"},
            "krylov_iters_per_step": mean(stats, "iters"),
            "fp64_krylov_iters_per_step": mean(stats, "fp64_iters"),
            "refinements_per_step": mean(stats, "refinements"),
            "compare": compare,
            "err_vs_oracle": err,
            "wall_s": main["wall"],
            "setup_s": setup_s,
            "gpu_launches": int(main["launches"]),
            "clocks": clk,
            "roofline": roof,
            "kernels": {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                            "GBps": round(v["bytes"] / max(v["ms"], 1e-9) / 1e6, 1),
                            "GFLOPs": (round(v["flops"] / max(v["ms"], 1e-9) / 1e6, 1)
                                       if v.get("flops") else None)}
                        for k, v in sorted(kstats.items(), key=lambda kv: -kv[1]["ms"])},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": prob.N * 8,
                    "d2h_bytes_per_step": prob.N * 8, "steps": len(ke)}}
    if pool is not None:
        v_all, v_one, nsteps, secs = oracle_sample(pool, cores, K_sched, args.cpu_budget)
        pool.close()
        pool.join()
        m_s, n_s = w["sample"]
        if m_s is None:  # the sample is the whole workload
            m_s, n_s = prob.m, prob.n
        line["cpu_baseline"] = {
            "value": v_all, "unit": UNIT, "cores": cores, "kind": "oracle",
            "single_core_value": v_one,
            "sample": f"{nsteps} FP64 oracle theta-steps (sparse LU + one extended-precision "
                      f"refinement each) on the {m_s} x {n_s} version of the workload's mesh, "
                      f"levels spread over the schedule, {cores} single-threaded workers in "
                      f"parallel for {secs:.1f} s; single_core_value = updates / summed "
                      f"per-step seconds"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------------- carrier pair
def _pair_oracle_step(args_):
    """One coupled oracle step of the pair recipe on an m x n mesh (timing sample)."""
    m, n = args_
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import polar_inputs as pi
    from oracle import coupled as oc
    cp = pi.coupled_pair(m=m, n=n, K=1)
    w = [np.array([1.0, 1.0]), np.array([1.0, 1.0])]
    t0 = time.perf_counter()
    _, _, iters, _, ok = oc.gummel_step(cp.phi, [cp.electrons, cp.holes],
                                        [cp.electrons.u0, cp.holes.u0], cp.t[0], cp.t[1],
                                        cp.theta_w, w, cp.w_phi, cp.mobility, cp.slots, 1e-10, 60,
                                        depth=3)
    return 2 * cp.electrons.N, time.perf_counter() - t0, iters


def run_pair(args):
    """The electron-hole pair with a self-consistent potential (Gummel's iteration with
    Anderson depth 3 per theta-step, stop at a potential change of 1e-10): the coupled-pair
    recipe on a 512 x 1024 mesh (or --mesh M N).  value = carrier updates (2 N per step) /
    device time."""
    import torch
    import polar_inputs as pi
    import paper_2509_15879_gb300 as P
    from paper_2509_15879_gb300 import driver
    rank = env_int("RANK", 0)
    if rank != 0:  # one pair per job: the other ranks have nothing to shard
        return 0
    m, n = args.mesh or (512, 1024)
    cores = host_cores()
    sample = (64, 128)
    pool = None
    if not args.no_cpu_baseline:  # spawn before this process touches the GPU
        pool = mp.get_context("spawn").Pool(cores)
        pool.map(_noop, range(cores), chunksize=1)
    torch.cuda.set_device(env_int("LOCAL_RANK", 0))
    K, W = args.steps, args.warmup
    cp = pi.coupled_pair(m=m, n=n, K=K + W)
    precision = P.POLAR_MIXED if args.precision == "mixed" else P.POLAR_FP64
    stream = torch.cuda.current_stream()
    ph = driver.create(cp.phi, precision, stream=stream.cuda_stream)
    el = driver.create(cp.electrons, precision, stream=stream.cuda_stream)
    ho = driver.create(cp.holes, precision, stream=stream.cuda_stream)
    P.polar_set_state(ph, np.zeros(cp.phi.N), 0.0)
    g = P.polar_gummel_create(ph, el, ho, cp.mobility, cp.slots[0], cp.slots[1], tol=1e-10,
                              max_iter=60, depth=3)
    w = [1.0, 1.0]
    for k in range(W):
        P.polar_gummel_step(g, cp.t[k], cp.t[k + 1], cp.theta_w, w, w, cp.w_phi)
    torch.cuda.synchronize()
    clocks = ClockSampler(env_int("LOCAL_RANK", 0))
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    iters = []
    e0.record(stream)
    for k in range(W, W + K):
        st, _ = P.polar_gummel_step(g, cp.t[k], cp.t[k + 1], cp.theta_w, w, w, cp.w_phi)
        iters.append(st["iters"])
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    updates = 2 * cp.electrons.N * K
    line = {"metric": METRIC, "value": updates / (ms * 1e-3), "unit": UNIT, "n_gpus": 1,
            "steps": K, "warmup": W, "ms_per_step": ms / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if precision == P.POLAR_FP64 else "f32+f64", "data": "synthetic",
            "config": {"workload": f"electron-hole pair with a Poisson potential, {m} x {n} "
                                   f"stretched adaptive mesh, Gummel's iteration "
                                   f"(Anderson depth 3) to a potential change of 1e-10 per "
                                   f"theta-step; updates = both carriers' unknowns per step",
                       "m": m, "n": n, "N": cp.electrons.N, "precision": args.precision},
            "potential_solves_per_step": float(np.mean(iters)), "clocks": clk}
    if pool is not None:
        t0 = time.perf_counter()
        res, rounds = [], 0
        while rounds == 0 or time.perf_counter() - t0 < args.cpu_budget:
            res += pool.map(_pair_oracle_step, [sample] * cores, chunksize=1)
            rounds += 1
        wall = time.perf_counter() - t0
        pool.close()
        pool.join()
        upd = sum(r[0] for r in res)
        line["cpu_baseline"] = {
            "value": upd / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "single_core_value": upd / sum(r[1] for r in res),
            "sample": f"{len(res)} coupled oracle steps (sparse LU per potential and carrier "
                      f"solve, {np.mean([r[2] for r in res]):.0f} potential solves each) on "
                      f"the {sample[0]} x {sample[1]} version of the recipe, {cores} workers"}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------- batch
def run_batch(args):
    """The 256-instance sweep: continuity equation on uneven adaptive meshes (m log-uniform
    in [64, 1024], n in [128, 2048], D amplitude in [0.2, 5], Peclet in [0.1, 20]), 500-level
    time stretch each, advanced together: one CUDA graph per step whose parallel branches
    are up to 8 size-sorted groups, in each of which a kernel class runs once per phase over
    the group's active instances.  value = sum of N_i x steps / device time."""
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
        K = min(args.steps, K_sched)
        # warm-up over the timed schedule's length: the autotuner runs, the schedule arrays
        # reach their size and the batch graph is captured outside the timed region
        driver.batch_advance(batch, probs, 0, K, check=False)
        for c, p in zip(ctxs, probs):  # back to the initial state for the timed steps
            P.polar_set_state(c, p.u0, p.t[0])
        clocks = ClockSampler(local)
        clocks.start()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        launches0 = P.polar_batch_kernel_launches(batch)
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
        # the batch's loops run as long as the slowest instance: mean over steps of the max
        imax = float(np.mean([max(row[k]["iters"] for row in stats) for k in range(K)]))
        # only the steps an instance completed count as updates (a failed step halts the
        # rest of that instance's schedule; its state stays at the last committed level)
        updates = sum_over_ranks(dist, [sum(p.N * d for p, d in zip(probs, done))])[0]
        launches = P.polar_batch_kernel_launches(batch) - launches0
        return ms, K, states, (iters, imax), clk, launches, updates, failed

    ms, K, st_main, (iters, imax), clk, launches, updates, failed = run(precision)
    pts = sum_over_ranks(dist, [sum(p.N for p in probs)])[0]
    value = updates / (ms * 1e-3)
    compare = None
    if args.compare:
        other = P.POLAR_FP64 if precision == P.POLAR_MIXED else P.POLAR_MIXED
        ms2, _, st2, (it2, _), _, _, up2, failed2 = run(other)
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
                                   f"per step of up to 8 size-sorted groups as parallel "
                                   f"branches, each kernel class launched once per phase over "
                                   f"a group's active instances", "instances": len(probs),
                       "sum_N": pts, "precision": args.precision,
                       "l2": "inputs larger than L2 (several GB of instance data)",
                       "parallelism": f"replicas x{world}"},
            "krylov_iters_per_step": iters, "krylov_iters_max_per_step": imax,
            "failed_instances": failed, "compare": compare,
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
    `ncu --profile-from-start off`) of one of WORKLOADS, at full size or, with --mesh
    M N, on the same recipe's M x N mesh.  The step is the third level of the schedule."""
    import torch
    import paper_2509_15879_gb300 as P
    from paper_2509_15879_gb300 import driver
    prob = make_problem(args.workload, *(args.mesh or (None, None)))
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
                                      "GBps": round(v["bytes"] / max(v["ms"], 1e-9) / 1e6, 1),
                                      "GFLOPs": (round(v["flops"] / max(v["ms"], 1e-9) / 1e6, 1)
                                                 if v.get("flops") else None)}
                                  for k, v in sorted(q.items(), key=lambda kv: -kv[1]["ms"])}}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=12)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="mixed",
                    help="headline path; --compare 1 also times the other one")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--compare", type=int, default=1,
                    help="also time the other precision on the same steps")
    ap.add_argument("--workload", choices=["c5", "c3", "c2", "c1", "batch", "pair"], default="c5",
                    help="c5 (default): continuity 8192 x 16384; c3: continuity 2048 x 4096; "
                         "c2: parabolic 512 x 1024; c1: parabolic 32 x 64 (direct solve); "
                         "batch: the 256-instance sweep; pair: the electron-hole pair "
                         "with a Poisson potential")
    ap.add_argument("--profile-step", action="store_true",
                    help="run one eager step of --workload inside a profiler range")
    ap.add_argument("--mesh", type=int, nargs=2, metavar=("M", "N"),
                    help="with --profile-step: the workload's recipe on an M x N mesh; with "
                         "--workload pair: the pair's mesh (default 512 x 1024)")
    ap.add_argument("--instances", type=int, default=256)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_step:
        return run_profile_step(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "pair":
        return run_pair(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
