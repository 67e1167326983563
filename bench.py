"""Benchmark: simulation steps per second, every step iterated to primal residual <= 1e-6,
on GB300 through libsubadmm (the C ABI in include/subadmm.h).

One benchmark step = one time step of every scene of the workload: assembly, beta,
factorisation, the ADMM loop to the stop rule, v-hat and the state update, all in the
library's kernels.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload batched|robots|fem_beam|chain] [--no-sub]

The headline line is the batched workload (4,096 uneven scenes in one launch per launch
class): the chosen form (mixed precision, batched, graph replay, autotuned variants) and
the plain FP64 form on the same scenes.  Every workload first runs an untimed pre-roll so
that the timed steps lie in its contact phase (the scenes start above the plane).  With a
single GPU the line also carries keyed sub-results for the other workloads: the 64 legged
robots after landing (with the learned warm start), the FEM beam, and the 8-link chain at a
fixed 100 iterations per step.

Under torchrun every rank simulates its own seeded batch (scenes are independent: weak
scaling, no data-path collective).  --impl reference times the FP64 CPU oracle on the host
cores on the same workload and segment instead.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import threading
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "sim steps/sec at primal residual ≤1e-6, chosen form vs plain FP64, 1 GB300"
FP64_NOMINAL_TFLOPS = 1.25     # GB300 nominal FP64 (non-tensor) rate
FP32_NOMINAL_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # 152 SMs x 128 FP32 lanes x FMA x clock
L2_FLUSH_BYTES = 512 << 20     # > 129 MB L2

# per workload: time step, untimed pre-roll (steps before warm-up, so that the timed segment
# lies in the contact phase), scene-sample size of the CPU oracle
WORKLOADS = {
    "batched": {"h": 1e-3, "preroll": 100, "cpu_scenes": 32},
    "robots": {"h": 2e-3, "preroll": 150, "cpu_scenes": 64},
    "fem_beam": {"h": 1e-3, "preroll": 0, "cpu_scenes": 1},
    "chain": {"h": 1e-3, "preroll": 0, "cpu_scenes": 1},
}


def workload_desc(workload: str, n_robots: int = 64, scenes: int = 4096) -> str:
    h = WORKLOADS[workload]["h"]
    if workload == "fem_beam":
        return (f"one linear-elastic tetrahedral beam 0.5 x 0.05 x 0.05 m (10 x 10 nodes x 137 "
                f"planes, Kuhn split, E=1e5 Pa, nu=0.45, rho=1000) cut into 64 slabs of 900/1200 "
                f"DOF joined by node-node equality (18,900 rows), 2,000 speculative ground "
                f"contacts mu=0.5, a 7-R arm (one rigid subsystem, PD drives) holding one end by "
                f"ball joints; h={h:g} s; each step iterated to r_p<=1e-6 with the previous "
                f"step's warm start")
    if workload == "batched":
        return (f"{scenes} independent uneven scenes of 2-32 subsystems each: floating rigid "
                f"chains of 1-40 bodies and 2x2xk spring-lattice blocks (a stand-in for small "
                f"FEM blocks) of 12-240 DOF, random tree + chord ball joints, 0-64 point "
                f"contacts per scene with the plane z=0, mu uniform in [0.3, 1.0]; h={h:g} s; "
                f"each step iterated to r_p<=1e-6 with the previous step's warm start")
    if workload == "chain":
        return ("serial chain of 8 rigid links (box 0.1x0.02x0.02 m, density 1000), ball "
                "joints, first link pinned, gravity; 4 subsystems of 2 links; h=1e-3 s, "
                "rho=1e3 fixed, exactly 100 ADMM iterations per step")
    return (f"{n_robots} independent legged robots (6-DOF trunk + 4 legs x 3 revolute joints, "
            f"one subsystem per leg and one for the trunk, PD drives as soft rows, 4 point-foot "
            f"plane contacts mu=0.8), dropped from 0.3-0.5 m; h={h:g} s; each step iterated to "
            f"r_p<=1e-6 with the previous step's warm start")


def make_problem(workload: str, rank: int = 0, n_robots: int = 64, scenes: int = 4096):
    """The scenes a rank simulates: an independent seeded batch per rank (weak scaling; the
    scenes never exchange data, so the ranks share no data-path collective)."""
    import scenegen as sg
    h = WORKLOADS[workload]["h"]
    if workload == "batched":
        return sg.batched(seed=rank, n_scenes=scenes, h=h, tol_primal=1e-6, max_iters=1000)
    if workload == "fem_beam":
        return sg.fem_beam(seed=rank, h=h, tol_primal=1e-6, max_iters=1000)
    if workload == "chain":
        return sg.chain(rank, max_iters=100, tol_primal=-1, rho=1e3)
    return sg.robots(seed=rank, n_robots=n_robots, h=h, tol_primal=1e-6, max_iters=1000)


def whole_job_rate(world: int, steps: int, t_ms_max: float) -> float:
    """Steps of every rank's batch per second over the slowest rank's time."""
    return world * steps / (t_ms_max / 1e3)


def algorithmic_work(problem):
    """Per-scene algorithmic FLOPs of the method (triangular-solve form of Eq. admm-1i):
    per iteration and subsystem 2 n^2 (two triangular solves) + 4 nnz(J_i) (J^T w and J v)
    + 20 m_i (projection, updates, residuals); per step and subsystem n^3/3 (Cholesky)
    + 2 sum_rows nnz(row)^2 (K = A + beta J^T J).  Also sum_i m_i^2 (entries of D)."""
    out = []
    for sc in problem.scenes:
        n = [s.n for s in sc.subs]
        m = [0] * len(n)
        nnz = [0] * len(n)
        rowsq = [0] * len(n)
        for itf in sc.ifs:
            if hasattr(itf, "J"):
                for s, Jm in zip(itf.subs, itf.J):
                    c = (np.asarray(Jm) != 0).sum(1)
                    m[s] += itf.rows
                    nnz[s] += int(c.sum())
                    rowsq[s] += int((c ** 2).sum())
                continue
            # nonzeros per row on one body side; a node side has one per row
            rows_cols = {1: [6, 6, 6], 2: [6, 6, 6, 3, 3], 3: [3], 4: [6, 6, 6]}[itf.kind]
            per_sub = {}
            for s, _ in [itf.a] + ([itf.b] if itf.b is not None else []):
                cols = [1] * len(rows_cols) if hasattr(sc.subs[s], "Ki") else rows_cols
                acc = per_sub.get(s, [0] * len(rows_cols))
                per_sub[s] = [x + c for x, c in zip(acc, cols)]
            for s, cols in per_sub.items():
                m[s] += len(cols)
                nnz[s] += sum(cols)
                rowsq[s] += sum(c * c for c in cols)
        it = sum(2 * ni * ni + 4 * zi + 20 * mi for ni, zi, mi in zip(n, nnz, m))
        # a linear block's K_i is constant: its factorisation is per run, not per step
        lin = [hasattr(s, "Ki") for s in sc.subs]
        st = sum((0.0 if li else ni ** 3 / 3.0) + 2 * q for ni, q, li in zip(n, rowsq, lin))
        out.append((it, st, sum(mi * mi for mi in m)))
    return out


def sub_sizes(scene):
    """(n_i, m_i) of every subsystem of a scene: DOF and side-rows (rows of J_ci)."""
    n = [s.n for s in scene.subs]
    m = [0] * len(n)
    for itf in scene.ifs:
        if hasattr(itf, "J"):
            for s in itf.subs:
                m[s] += itf.rows
            continue
        rows = {1: 3, 2: 5, 3: 1, 4: 3}[itf.kind]
        sides = {itf.a[0]} | ({itf.b[0]} if itf.b is not None else set())
        for s in sides:
            m[s] += rows
    return list(zip(n, m))


def gram_roofline(ctx, scene, reps: int = 20) -> dict:
    """The tcgen05 Gram kernel on the shapes of a scene's large blocks (W: n x (m + 1), the
    map's right-hand sides), timed standalone with CUDA events over ``reps`` runs.  Algorithmic
    work: the symmetric product, n (m + 1)(m + 2) flops per block; executed: three TF32 MMAs
    per product (split-TF32) over the padded upper-triangle tiles."""
    import torch
    jobs = [(n, m + 1) for n, m in sub_sizes(scene) if n >= 128 and m >= 16]
    if not jobs:
        return None
    g = torch.Generator(device="cuda").manual_seed(0)
    Ws = [torch.randn(n, (c + 3) // 4 * 4, device=ctx.dev, generator=g) for n, c in jobs]
    Gs = [torch.empty(c, c, device=ctx.dev) for _, c in jobs]
    ms = ctx.subadmm.sim_gram_tc(ctx.local, [w.data_ptr() for w in Ws], [n for n, _ in jobs],
                                 [c for _, c in jobs], [w.shape[1] for w in Ws],
                                 [x.data_ptr() for x in Gs], [c for _, c in jobs], reps=reps)
    alg = float(sum(n * c * (c + 1) for n, c in jobs))
    tiles = sum(((c + 127) // 128) * ((c + 127) // 128 + 1) // 2 for _, c in jobs)
    kpad = {n: (n + 31) // 32 * 32 for n, _ in jobs}
    exe = float(sum(3 * 2 * kpad[n] * 128 * 128 * (((c + 127) // 128) * ((c + 127) // 128 + 1) // 2)
                    for n, c in jobs))
    bf16 = measured_peaks().get("bf16_tflops")
    tf32 = (bf16 or 1900.0) / 2.0
    ach = alg / (ms / 1e3) / 1e12
    return {"bound": "tensor", "achieved": ach, "peak": tf32 / 3.0, "unit": "TFLOP/s",
            "frac": ach / (tf32 / 3.0), "traffic": None,
            "mma_tflops": exe / (ms / 1e3) / 1e12, "tf32_peak": tf32,
            "mma_frac": exe / (ms / 1e3) / 1e12 / tf32, "ms_per_launch": ms,
            "blocks": len(jobs), "tiles": tiles,
            "note": f"tcgen05 Gram kernel alone on the scene's {len(jobs)} blocks of >= 128 DOF "
                    f"(random W of their shapes), CUDA events over {reps - 1} launches; achieved = "
                    f"algorithmic flops n (m+1)(m+2) per block / time; peak = TF32 (measured bf16 "
                    f"{'burst' if bf16 else 'fallback'} x 1/2, the nominal ratio) / 3 (split-TF32 "
                    f"issues three MMAs per product); mma_* count every issued MMA flop"}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sms.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sms:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sms)}


KERNEL_SOURCES = ("layout.h", "rigid_model.cuh", "step_kernel.cuh", "grid_kernel.cuh", "subadmm.cu")


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2302_14344_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _recorded(name: str):
    """key: value lines of a committed ncu summary, or None when it is missing or the kernel
    sources changed since its capture."""
    try:
        txt = open(os.path.join(ROOT, "profiles", name)).read()
    except OSError:
        return None
    vals = {}
    for line in txt.splitlines():
        if ":" in line and not line.startswith(" "):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    return vals if vals.get("source_sha256") == kernel_source_hash() else None


def recorded_traffic(steps_per_launch: int):
    """DRAM bytes per launch of the step kernel (robots) from the committed ncu summary,
    scaled to this launch length (the per-step traffic is constant: descriptors and states
    are re-read every step), or None."""
    vals = _recorded("step_kernel_robots64_traffic.md")
    if not vals:
        return None
    return float(vals["traffic_bytes_per_launch"]) / float(vals["steps_per_launch"]) * steps_per_launch


def recorded_traffic_fem(iters_per_launch: float):
    """DRAM bytes per launch of the grid kernel (FEM beam): the summary's bytes per iteration
    (D streamed once per iteration dominates) times this run's iterations per launch, or
    None."""
    vals = _recorded("grid_step_kernel_fem_beam_traffic.md")
    if not vals:
        return None
    return float(vals["traffic_bytes_per_iteration"]) * iters_per_launch


def recorded_traffic_batched(steps_per_launch: int, scenes: int):
    """DRAM bytes per launch of the batched workload's step kernels from the committed ncu
    summary (a smaller batch of the same generator), scaled per scene and per step, or None."""
    vals = _recorded("step_kernel_batched_traffic.md")
    if not vals:
        return None
    return (float(vals["traffic_bytes_per_scene_step"]) * scenes * steps_per_launch)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def host_cpu() -> dict:
    """Host CPU model and core count (the oracle baselines' machine)."""
    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k = line.split(":", 1)
                if len(k) == 2 and k[0].strip() in ("model name", "Model name", "CPU part"):
                    model = k[1].strip()
                    if k[0].strip() != "CPU part":
                        break
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"model": model, "arch": platform.machine(), "nproc": os.cpu_count() or 1}


# ---------------------------------------------------------------------------------------------
# CPU oracle (test infrastructure; timed here as the reported baseline only)

def oracle_rate(workload: str, problem, preroll: int, warmup: int, steps: int,
                threads: int, seconds: float, n_scenes: int):
    """Time the FP64 CPU oracle, as it stands, on a bounded sample of the workload: the first
    ``n_scenes`` scenes (scenes are drawn independently, so a prefix is a random sample), run
    through the same pre-roll and warm-up as the GPU (untimed), then up to ``steps`` timed
    steps or ``seconds``.  Scenes run on ``threads`` host threads (ctypes releases the GIL);
    a single scene runs on the OpenMP build (subsystems and constraints over the threads).
    The rate is scaled to whole-workload steps per second."""
    import oracle
    n_all = len(problem.scenes)
    n = min(n_scenes, n_all)
    omp = n == 1 and threads > 1
    if omp:
        os.environ["OMP_NUM_THREADS"] = str(threads)
    scs = [oracle.OracleScene(sc, problem.options, openmp=omp) for sc in problem.scenes[:n]]
    pool = ThreadPoolExecutor(max_workers=threads) if (threads > 1 and n > 1) else None

    def step_all():
        if pool is None:
            for o in scs:
                o.step()
        else:
            list(pool.map(lambda o: o.step(), scs))
    for _ in range(preroll + warmup):
        step_all()
    t0 = time.perf_counter()
    k, iters = 0, 0
    while k < steps:
        step_all()
        k += 1
        iters += sum(o.residuals()["iters"] for o in scs)
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    if pool is not None:
        pool.shutdown()
    which = (f"all {n_all} scenes" if n == n_all else
             f"the first {n} of {n_all} scenes, rate scaled by {n}/{n_all}")
    how = (f"OpenMP build on {threads} threads (subsystems and constraints)" if omp else
           f"{threads} host threads over scenes" if pool is not None else "single thread")
    return {"value": k / dt * n / n_all, "unit": "steps/s", "cores": threads if (omp or pool) else 1,
            "kind": "oracle",
            "sample": f"steps {preroll + warmup}..{preroll + warmup + k} of {which} (whole sample "
                      f"per step, after an untimed pre-roll and warm-up like the GPU's); plain C "
                      f"-O2 FP64, {how}; {iters / max(k * n, 1):.1f} iterations per scene-step",
            "seconds": round(dt, 2), "cpu": host_cpu()}


def oracle_fem_rate(threads: int):
    """The FP64 CPU oracle on the FEM beam: one step takes minutes single-threaded, so the
    first step is timed at 1 and at 41 ADMM iterations on the OpenMP build (the shorter one
    twice, keeping the faster); their difference gives the time per iteration, the rest the
    per-step assembly and factorisation."""
    import oracle
    import scenegen as sg
    os.environ["OMP_NUM_THREADS"] = str(threads)
    times = {}
    for k, reps in ((1, 2), (41, 1)):
        p = sg.fem_beam(seed=0, h=1e-3, tol_primal=-1, max_iters=k)
        best = None
        for _ in range(reps):
            o = oracle.OracleScene(p.scenes[0], p.options, openmp=True)
            t0 = time.perf_counter()
            o.step()
            dt = time.perf_counter() - t0
            best = dt if best is None else min(best, dt)
        times[k] = best
    per_iter = max(times[41] - times[1], 0.0) / 40.0
    return {"setup_s": times[1] - per_iter, "per_iter_s": per_iter, "times": times}


def run_reference(args, rank: int, world: int):
    """The reference arm: the FP64 CPU oracle, as it stands, on the same workload, segment,
    metric and unit as this arm's line (rank 0 only)."""
    if rank != 0:
        return 0
    wl = WORKLOADS[args.workload]
    threads = os.cpu_count() or 1
    if args.workload == "fem_beam":
        r = oracle_fem_rate(threads)
        mean_iters = 600.0
        val = 1.0 / (r["setup_s"] + r["per_iter_s"] * mean_iters)
        cb = {"value": val, "unit": "steps/s", "cores": threads, "kind": "oracle",
              "sample": f"first step at 1 and 41 iterations: {r['setup_s']:.1f} s assembly and "
                        f"factorisation + {r['per_iter_s'] * 1e3:.0f} ms per iteration, "
                        f"extrapolated to {mean_iters:.0f} iterations per step; OpenMP build on "
                        f"{threads} threads", "cpu": host_cpu()}
        steps = 1
    else:
        p = make_problem(args.workload, 0, args.robots, args.scenes)
        cb = oracle_rate(args.workload, p, wl["preroll"] + 1, args.warmup, args.steps, threads,
                         args.reference_seconds, args.reference_scenes or wl["cpu_scenes"])
        val = cb["value"]
        steps = args.steps
    line = {"metric": METRIC, "value": val, "unit": "steps/s", "n_gpus": world, "steps": steps,
            "warmup": args.warmup, "ms_per_step": 1e3 / val, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": workload_desc(args.workload, args.robots, args.scenes),
                       "form": "FP64 CPU oracle", "preroll_steps": wl["preroll"]},
            "cpu_baseline": cb,
            "e2e": {"value": val, "unit": "steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------------------
# GPU timing

class Ctx:
    def __init__(self, subadmm, stream, dev, local, dist, flush):
        self.subadmm, self.stream, self.dev, self.local = subadmm, stream, dev, local
        self.dist, self.flush = dist, flush
        self.net, self.net_info = None, None


def time_form(ctx, p, precision, steps: int, warmup: int, preroll: int, spl: int,
              autotune: bool = True, graph: bool = True, sample_clocks: bool = False,
              keep_factors: bool = True, net=None, grid_rows=None, tc_factor: bool = True):
    """Pre-roll (untimed, so the timed segment lies in the contact phase), autotune the
    kernel variants on that state (restored afterwards), W warm-up steps, then K timed steps
    in launches of ``spl`` steps (the scenes are independent, so one launch advances every
    scene by that many steps without a device-wide wait per step).  The L2 is flushed before
    every timed launch; CUDA events on the launching stream; max over ranks.  With ``net``
    the warm-up and timed launches are learned ones (sim_step_learned: the network evaluated
    once per launch, its duals starting the launch's first step, its beta scales held)."""
    import torch
    sa = ctx.subadmm
    sim = sa.Simulation(p, stream=ctx.stream.cuda_stream, device=ctx.local, precision=precision,
                        grid_side_rows=grid_rows)

    def advance(n):
        if net is None:
            sim.step(n)
        else:
            sim.step_learned(net, n)
    if not keep_factors:
        sim.keep_factors(False)
    if not tc_factor:
        sim.tc_factor(False)
    sim.step(1)
    left = preroll
    while left > 0:
        n = min(left, 50)
        sim.step(n)
        left -= n
    tuned = sim.autotune(steps=3) if autotune else sim.launch_classes()
    if graph:
        sim.use_graph(True)
    for _ in range(warmup):
        advance(1)
    if net is not None and spl > 1:
        advance(spl)                       # the learned launch of the timed size, captured
    sim.sync()
    sim.iteration_stats()   # clear counters
    chunks = [spl] * (steps // spl) + ([steps % spl] if steps % spl else [])
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in chunks]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in chunks]
    if ctx.dist is not None:
        ctx.dist.barrier()
    torch.cuda.synchronize(ctx.dev)
    clk = ClockSampler(ctx.local) if sample_clocks else None
    if clk:
        clk.__enter__()
    torch.cuda.nvtx.range_push("timed")   # lets a profiler capture exactly these launches
    for k, n in enumerate(chunks):
        ctx.flush.zero_()                  # L2 flushed between timed launches
        ev0[k].record(ctx.stream)
        advance(n)
        ev1[k].record(ctx.stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize(ctx.dev)
    if clk:
        clk.__exit__()
    if ctx.dist is not None:
        ctx.dist.barrier()
    launch_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    t_ms = float(sum(launch_ms))
    if ctx.dist is not None:
        tt = torch.tensor([t_ms], device=ctx.dev)
        ctx.dist.all_reduce(tt, op=ctx.dist.ReduceOp.MAX)
        t_ms = float(tt.item())
    stats = sim.iteration_stats(per_scene=True)
    return {"sim": sim, "t_ms": t_ms, "launch_ms": launch_ms, "stats": stats, "classes": tuned,
            "clocks": clk.summary() if clk else None, "chunks": chunks}


def iter_summary(stats) -> dict:
    return {"mean_per_scene_step": stats["total_iters"] / max(stats["scene_steps"], 1),
            "max": stats["max_iters"], "not_converged": stats["not_converged"],
            "not_converged_frac": stats["not_converged"] / max(stats["scene_steps"], 1),
            "scene_steps": stats["scene_steps"]}


def alu_roofline(p, work, stats, t_ms, mixed: bool, steps: int, traffic=None):
    it_flops = np.array([w[0] for w in work])
    st_flops = float(sum(w[1] for w in work))
    flops = float(it_flops @ stats["per_scene"][:, 0]) + st_flops * steps
    achieved = flops / (t_ms / 1e3) / 1e12
    peak, pipe = (FP32_NOMINAL_TFLOPS, "FP32") if mixed else (FP64_NOMINAL_TFLOPS, "FP64")
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic,
            "note": f"{pipe} non-tensor pipe; peak nominal, derived from unit counts and clock "
                    f"({'152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz' if mixed else 'GB300 FP64 rate'});"
                    f" algorithmic flops of the triangular-solve form, {it_flops.mean():.0f} per "
                    f"scene-iteration (mean over scenes) and {st_flops / len(p.scenes):.0f} per "
                    f"scene-step, times the iterations each scene ran"}


def e2e_rate(ctx, sim, steps: int, world: int, net=None):
    """End to end through the C ABI with host buffers: the state in from pinned host memory,
    one step (a learned one with ``net``), the state out to pinned host memory, every step
    (host wall clock)."""
    import torch
    sa = ctx.subadmm
    sizes = sim.sizes()
    nstate = 13 * sizes["bodies"] + 6 * sizes["nodes"]
    hbuf = torch.empty(nstate, dtype=torch.float64).pin_memory()
    sa.sim_read_state(sim.h, hbuf.data_ptr())
    torch.cuda.synchronize(ctx.dev)
    t0 = time.perf_counter()
    for _ in range(steps):
        sa.sim_write_state(sim.h, hbuf.data_ptr())
        if net is None:
            sim.step(1)
        else:
            sim.step_learned(net, 1)
        sa.sim_read_state(sim.h, hbuf.data_ptr())
    dt = time.perf_counter() - t0
    if ctx.dist is not None:
        tt = torch.tensor([dt], device=ctx.dev)
        ctx.dist.all_reduce(tt, op=ctx.dist.ReduceOp.MAX)
        dt = float(tt.item())
    return {"value": world * steps / dt, "unit": "steps/s", "h2d_bytes_per_step": 8 * nstate,
            "d2h_bytes_per_step": 8 * nstate, "steps": steps, "timer": "host wall clock"}


def barrier_floor(ctx) -> dict:
    """Cycles of one __syncthreads_count round of a 256-thread block (one block per SM):
    the floor under one iteration of the block kernel, which has one such barrier."""
    return ctx.subadmm.sim_barrier_floor(ctx.local, 20000)


# ---------------------------------------------------------------------------------------------
# sub-results (single GPU only)

def sub_robots(ctx, args, threads: int) -> dict:
    """64 legged robots, timed after landing (pre-roll 150 steps: the feet touch down near
    step 120); mixed and plain FP64; the learned warm start against the previous-step start
    on the same segment; microseconds per iteration against the barrier floor."""
    import torch
    sa = ctx.subadmm
    wl = WORKLOADS["robots"]
    p = make_problem("robots", 0, args.robots)
    K = max(args.steps, 100)
    work = algorithmic_work(p)
    r = time_form(ctx, p, sa.SIM_MIXED, K, args.warmup, wl["preroll"], 50)
    f = time_form(ctx, p, sa.SIM_FP64, K, args.warmup, wl["preroll"], 50)
    out = {"workload": workload_desc("robots", args.robots),
           "timed_segment": f"steps {wl['preroll'] + 1 + args.warmup}..{wl['preroll'] + 1 + args.warmup + K} "
                            f"(after landing)",
           "value": K / (r["t_ms"] / 1e3), "unit": "steps/s", "form": "mixed",
           "iterations": iter_summary(r["stats"]),
           "plain_fp64": {"value": K / (f["t_ms"] / 1e3), "unit": "steps/s",
                          "iterations": iter_summary(f["stats"])},
           "roofline": alu_roofline(p, work, r["stats"], r["t_ms"], True, K,
                                    recorded_traffic(50) if K % 50 == 0 else None),
           "launch_classes": r["classes"]}
    out["chosen_over_plain"] = out["value"] / out["plain_fp64"]["value"]
    # the paper's full-system ADMM comparator (Sec. IV-B, FADMM): each robot merged into one
    # subsystem, the same solver and segment
    import scenegen as sg
    pm = sg.merged(p)
    fm = time_form(ctx, pm, sa.SIM_MIXED, K, args.warmup, wl["preroll"], 50)
    ff = time_form(ctx, pm, sa.SIM_FP64, K, args.warmup, wl["preroll"], 50)
    out["full_system_admm"] = {
        "value": K / (fm["t_ms"] / 1e3), "unit": "steps/s", "form": "mixed",
        "iterations": iter_summary(fm["stats"]),
        "plain_fp64": {"value": K / (ff["t_ms"] / 1e3), "unit": "steps/s",
                       "iterations": iter_summary(ff["stats"])},
        "subsystem_over_full": out["value"] / (K / (fm["t_ms"] / 1e3)),
        "note": "each robot merged into one subsystem of 78 DOF (every constraint its own "
                "z-variable, one factorisation per robot and step), same kernels and segment"}
    fm["sim"].close()
    ff["sim"].close()
    # cycles per iteration (phase tracer, a separate short run) against the barrier floor
    sim = r["sim"]
    sim.use_graph(False)
    sa.sim_phase_trace(sim.h, True)
    sim.step(20)
    sim.sync()
    ph = sa.sim_phase_trace(sim.h, False)
    fl = barrier_floor(ctx)
    per_it = (ph["v_step"] + ph["z_step"]) / max(ph["iterations"], 1)
    out["cycles_per_iteration"] = {"iteration": per_it, "barrier_floor": fl["cycles"],
                                   "ratio": per_it / max(fl["cycles"], 1e-9),
                                   "setup_and_recovery_per_scene_step":
                                       (ph["assemble"] + ph["factor"] + ph["recover"] + ph["exit"])
                                       / max(ph["scene_steps"], 1),
                                   "note": "SM cycles seen by each scene's first thread (phase "
                                           "tracer, 20 steps after the timed segment); floor = "
                                           "one __syncthreads_count round of a 256-thread block"}
    sim.close()
    f["sim"].close()
    if ctx.net is not None:
        try:
            out["learned_warm_start"] = learned_comparison(ctx.net, ctx.net_info, p, K,
                                                           wl["preroll"] + 1 + args.warmup, 50)
        except Exception as e:                       # reported, not fatal to the line
            out["learned_warm_start"] = {"error": repr(e)}
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = oracle_rate("robots", p, wl["preroll"] + 1, args.warmup, K,
                                          threads, 8.0, 64)
    return out


# the rho search labels a scene-step with the largest beta scale within 10% of its fewest
# iterations (learned.collect_rho)
RHO_LABEL_SLACK = 0.1


def train_warmstart(seed: int = 1) -> tuple:
    """The learned warm start's network, trained on the GPU by the library's own kernels on
    samples the plain simulator generates (config 5): the uneven batched scenes, the legged
    robots after landing, the FEM beam of the config-3 distribution and the 8-link chain,
    each through the rho search (every scene in seven copies with beta scaled 2^-3 .. 2^3;
    the fewest iterations label the seventh output).  Scenes of other seeds than the
    benchmark's."""
    import scenegen as sg
    import torch
    from paper_2302_14344_gb300 import learned as lr
    t0 = time.perf_counter()
    slack = RHO_LABEL_SLACK
    sources = [("batched", lambda: lr.collect_rho(sg.batched(101, n_scenes=512), steps=20,
                                                  warmup=100, slack=slack)),
               ("robots", lambda: lr.collect_rho(sg.robots(101, n_robots=64), steps=40,
                                                 warmup=150, slack=slack)),
               ("fem_beam", lambda: lr.collect_rho(sg.fem_beam(11, vary=True), steps=10,
                                                   warmup=3, slack=slack)),
               ("chain", lambda: lr.collect_rho(sg.chain(101, max_iters=1000, tol_primal=1e-6,
                                                         rho=1e3), steps=50, warmup=3,
                                                slack=slack))]
    parts, counts = [], {}
    for name, fn in sources:
        q = fn()
        parts.append(q)
        counts[name] = int(q[0].shape[0])
    X = torch.cat([q[0] for q in parts]); T = torch.cat([q[1] for q in parts])
    M = torch.cat([q[2] for q in parts])
    collect_s = time.perf_counter() - t0
    net = lr.init_network(seed=seed)
    losses = lr.train(net, X, T, M, epochs=6)
    return net, {"samples": int(X.shape[0]), "by_workload": counts, "epochs": 6,
                 "label": f"largest beta scale within {RHO_LABEL_SLACK:.0%} of the fewest iterations",
                 "loss_first_last": [losses[0], losses[-1]],
                 "collect_seconds": round(collect_s, 1),
                 "train_seconds": round(time.perf_counter() - t0 - collect_s, 1)}


def learned_comparison(net, info, p, steps: int, warmup: int, per_launch: int) -> dict:
    """The learned warm start (duals and beta scales) against the previous-step warm start on
    the same start and segment, both in launches of ``per_launch`` steps by graph replay (the
    network evaluated once per launch)."""
    from paper_2302_14344_gb300 import learned as lr
    res = lr.compare(p, net, steps=steps, warmup=warmup, per_launch=per_launch,
                     learned_warmup=1)
    pl, le = res["plain"], res["learned"]
    return {"value": 1e3 / le["ms_per_step"], "unit": "steps/s",
            "previous_step_start": 1e3 / pl["ms_per_step"],
            "learned_over_previous": pl["ms_per_step"] / le["ms_per_step"],
            "iterations_per_scene_step": {"learned": le["iters_per_scene_step"],
                                          "previous_step": pl["iters_per_scene_step"]},
            "not_converged": {"learned": le["not_converged"], "previous_step": pl["not_converged"]},
            "fallbacks": le["fallbacks"], "training": info,
            "note": f"mixed form, {per_launch} steps per launch by graph replay for both starts; "
                    f"the learned one evaluates the 32-256-256-256-7 network (fused tcgen05 "
                    f"kernel) once per launch: its duals start the launch's first step, its "
                    f"beta scales hold for the launch"}


def sub_fem_beam(ctx, args, threads: int) -> dict:
    """The FEM beam (one scene over the whole GPU): mixed, plain FP64, and plain FP64 with
    every block refactorised every step (Algorithm 1 literally)."""
    sa = ctx.subadmm
    p = make_problem("fem_beam")
    work = algorithmic_work(p)
    K = args.steps
    r = time_form(ctx, p, sa.SIM_MIXED, K, args.warmup, 0, 50, autotune=True, graph=False)
    f = time_form(ctx, p, sa.SIM_FP64, K, args.warmup, 0, 50, autotune=True, graph=False)
    rf = time_form(ctx, p, sa.SIM_FP64, min(K, 10), 2, 0, 1, autotune=False, graph=False,
                   keep_factors=False)
    rm = time_form(ctx, p, sa.SIM_MIXED, K, args.warmup, 0, 1, autotune=False, graph=False,
                   keep_factors=False)
    rw = time_form(ctx, p, sa.SIM_MIXED, K, args.warmup, 0, 1, autotune=False, graph=False,
                   keep_factors=False, tc_factor=False)
    d_bytes = float(sum(w[2] for w in work)) * 4
    hbm = measured_peaks().get("hbm_gbs")
    st = r["stats"]
    gbs = d_bytes * st["total_iters"] / (r["t_ms"] / 1e3) / 1e9
    launches = len(r["chunks"])
    out = {"workload": workload_desc("fem_beam"), "value": K / (r["t_ms"] / 1e3),
           "unit": "steps/s", "form": "mixed", "iterations": iter_summary(st),
           "timed_segment": f"steps {1 + args.warmup}..{1 + args.warmup + K}",
           "plain_fp64": {"value": K / (f["t_ms"] / 1e3), "unit": "steps/s",
                          "iterations": iter_summary(f["stats"])},
           "plain_fp64_refactor_every_step": {
               "value": len(rf["launch_ms"]) / (rf["t_ms"] / 1e3), "unit": "steps/s",
               "steps": len(rf["launch_ms"]), "iterations": iter_summary(rf["stats"]),
               "note": "every block refactorised every step (sim_keep_factors(0)), one launch "
                       "per step, L2 flushed before each"},
           "mixed_refactor_every_step": {
               "value": len(rm["launch_ms"]) / (rm["t_ms"] / 1e3), "unit": "steps/s",
               "steps": len(rm["launch_ms"]), "iterations": iter_summary(rm["stats"]),
               "note": "every block refactorised every step, as Algorithm 1 states it: per step "
                       "the grid kernel up to K = A + beta J^T J, the blocked factorisation "
                       "(per 128-column panel a CUDA-core panel kernel and a tcgen05 Schur "
                       "update), the grid kernel for W = L^-1 [J^T b], the tcgen05 Gram kernel "
                       "for D and c, the grid kernel's iterations; L2 flushed before each step",
               "one_warp_factor": {
                   "value": len(rw["launch_ms"]) / (rw["t_ms"] / 1e3), "unit": "steps/s",
                   "iterations": iter_summary(rw["stats"]),
                   "note": "the same with every factor formed inside the setup launch by one "
                           "warp per slab (sim_tc_factor(0))"}},
           "gram_tensor_roofline": gram_roofline(ctx, p.scenes[0]),
           "corotational": corotational_beam(ctx, args),
           "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm or 6800.0, "unit": "GB/s",
                        "frac": gbs / (hbm or 6800.0),
                        "traffic": recorded_traffic_fem(st["total_iters"] / launches),
                        "note": f"algorithmic bytes: D of every subsystem once per iteration "
                                f"({d_bytes / 1e6:.1f} MB, FP32) x iterations / whole-step time "
                                f"(setup and exit included: a lower bound on the stream rate); "
                                f"peak = {'measured copy bandwidth' if hbm else 'fallback'}"}}
    out["chosen_over_plain"] = out["value"] / out["plain_fp64"]["value"]
    for x in (r, f, rf, rm, rw):
        x["sim"].close()
    if ctx.net is not None:
        try:
            import scenegen as sg
            out["learned_warm_start"] = learned_comparison(
                ctx.net, ctx.net_info, sg.fem_beam(21, vary=True), K, 1 + args.warmup, K)
            out["learned_warm_start"]["workload"] = ("the beam of the config-3 distribution "
                                                     "drawn by seed 21 (held out)")
        except Exception as e:
            out["learned_warm_start"] = {"error": repr(e)}
    if not args.no_cpu_baseline:
        fr = oracle_fem_rate(threads)
        mi = out["iterations"]["mean_per_scene_step"]
        out["cpu_baseline"] = {
            "value": 1.0 / (fr["setup_s"] + fr["per_iter_s"] * mi), "unit": "steps/s",
            "cores": threads, "kind": "oracle",
            "sample": f"first step at 1 and 41 iterations on the OpenMP build ({threads} threads): "
                      f"{fr['setup_s']:.1f} s assembly and factorisation + "
                      f"{fr['per_iter_s'] * 1e3:.0f} ms per iteration, extrapolated to "
                      f"{mi:.0f} iterations per step", "cpu": host_cpu()}
    return out


def corotational_beam(ctx, args) -> dict:
    """The beam with co-rotational slabs (the paper's beam model): every step assembles the
    elements' rotations and refactorises every slab; the mixed form factorises the slabs by
    the blocked factorisation (tensor-core Schur updates) and forms their maps on the tensor
    cores, plain FP64 does both on the CUDA cores."""
    import scenegen as sg
    sa = ctx.subadmm
    p = sg.fem_beam(0, corotational=True, tol_primal=1e-6, max_iters=1000)
    K = min(args.steps, 10)
    out = {"workload": "the FEM beam with co-rotational slabs (66,096 elements rotated and "
                       "assembled every step, every slab refactorised every step)"}
    for name, prec, k in (("mixed", sa.SIM_MIXED, K), ("plain_fp64", sa.SIM_FP64, min(K, 5))):
        r = time_form(ctx, p, prec, k, 2, 0, 1, autotune=False, graph=False)
        out[name] = {"value": k / (r["t_ms"] / 1e3), "unit": "steps/s", "steps": k,
                     "iterations": iter_summary(r["stats"])}
        r["sim"].close()
    out["value"] = out["mixed"]["value"]
    out["unit"] = "steps/s"
    out["chosen_over_plain"] = out["mixed"]["value"] / out["plain_fp64"]["value"]
    return out


def sub_cable(ctx, args) -> dict:
    """The cable scene (640 segments as a discrete rod in 160 subsystems, two arms: 162
    subsystems) at a fixed 90 iterations per step, the paper's own protocol for its cable
    scene (Table I), mixed and FP64; one scene over the whole GPU (grid kernel)."""
    import scenegen as sg
    sa = ctx.subadmm
    p = sg.cable(0, tol_primal=-1, max_iters=90)
    K = args.steps
    out = {"workload": "cable: 640 rigid segments (1 cm, r 5 mm) joined by ball joints with PD "
                       "bending and twist rows (a discrete Cosserat rod), in 160 subsystems of 4, "
                       "plane contacts mu=0.5, two 7-R arm stand-ins holding the ends; h=1e-3 s; "
                       "exactly 90 ADMM iterations per step"}
    for name, prec in (("mixed", sa.SIM_MIXED), ("plain_fp64", sa.SIM_FP64)):
        r = time_form(ctx, p, prec, K, args.warmup, 0, 50, autotune=True, graph=False,
                      grid_rows=1)
        res = r["sim"].residuals(0)
        out[name] = {"value": K / (r["t_ms"] / 1e3), "unit": "steps/s",
                     "us_per_iteration": r["t_ms"] * 1e3 / (K * 90), "r_p_after_90": res["r_p"]}
        r["sim"].close()
    out["value"] = out["mixed"]["value"]
    out["unit"] = "steps/s"
    out["chosen_over_plain"] = out["mixed"]["value"] / out["plain_fp64"]["value"]
    return out


STIR_PAPER_MS = {30: 3.489, 60: 5.940, 90: 8.705}   # Table I, SubADMM, 4-core CPU
STIR_PAPER_PJ_MS = {30: 3.235, 60: 5.688, 90: 9.425}  # Table I, PJ, same machine
STIR_PJ_OMEGA = 0.3                                   # Projected Jacobi's relaxation here


def sub_stir(ctx, args) -> dict:
    """The granular stirring scene (216 spheres and a 7-R arm stand-in, 217 subsystems) at the
    paper's fixed 30 / 60 / 90 iterations per step (Table I), mixed and FP64, one scene over
    the whole GPU (grid kernel); the oracle's time per step on all host cores beside each,
    and the paper's own times (another machine, a CPU: context only)."""
    import scenegen as sg
    sa = ctx.subadmm
    K = args.steps
    out = {"workload": "stir: 216 spheres (r 1 cm, 4 g) on a 6x6x6 lattice in a box, one "
                       "subsystem each, sphere-sphere contacts between initial neighbours "
                       "(< 1.5 diameters), floor and wall contacts, a 7-R arm stand-in sweeping "
                       "a tool sphere through the top layers (217 subsystems, 1,338 DOF); "
                       "mu=0.5, h=1e-2 s; exactly 30 / 60 / 90 ADMM iterations per step",
           "paper_ms_per_step": {str(k): v for k, v in STIR_PAPER_MS.items()}}
    for iters in (30, 60, 90):
        p = sg.stir(0, tol_primal=-1, max_iters=iters)
        row = {}
        for name, prec in (("mixed", sa.SIM_MIXED), ("plain_fp64", sa.SIM_FP64)):
            r = time_form(ctx, p, prec, K, args.warmup, 0, 50, autotune=True, graph=False,
                          grid_rows=1)
            res = r["sim"].residuals(0)
            row[name] = {"ms_per_step": r["t_ms"] / K,
                         "us_per_iteration": r["t_ms"] * 1e3 / (K * iters),
                         "r_p_after": res["r_p"]}
            r["sim"].close()
        if not args.no_cpu_baseline:                 # sub-results run at N = 1 only
            row["oracle_ms_per_step"] = oracle_stir_ms(p, steps=5)
        row["paper_over_mixed"] = STIR_PAPER_MS[iters] / row["mixed"]["ms_per_step"]
        # the paper's Projected Jacobi comparison solver on the same scene (sim_set_solver)
        q = sg.stir(0, tol_primal=-1, max_iters=iters)
        q.options.solver, q.options.pj_omega = "pj", STIR_PJ_OMEGA
        r = time_form(ctx, q, sa.SIM_MIXED, K, args.warmup, 0, 50, autotune=True, graph=False,
                      grid_rows=1)
        row["projected_jacobi_mixed"] = {
            "ms_per_step": r["t_ms"] / K, "omega": STIR_PJ_OMEGA,
            "natural_residual_after": r["sim"].residuals(0)["r_p"],
            "paper_ms_per_step": STIR_PAPER_PJ_MS[iters]}
        r["sim"].close()
        out[str(iters)] = row
    out["value"] = 1e3 / out["90"]["mixed"]["ms_per_step"]
    out["unit"] = "steps/s at 90 iterations"
    return out


def oracle_stir_ms(p, steps: int) -> float:
    """The oracle (OpenMP build, all host cores) stepping the stir scene: ms per step."""
    import oracle
    o = oracle.OracleScene(p.scenes[0], p.options, openmp=True)
    o.step()
    t0 = time.perf_counter()
    for _ in range(steps):
        o.step()
    return (time.perf_counter() - t0) * 1e3 / steps


def sub_chain(ctx, args) -> dict:
    """The 8-link chain at exactly 100 iterations per step with rho = 1e3 (FP64 and mixed)."""
    sa = ctx.subadmm
    p = make_problem("chain")
    K = max(args.steps, 200)
    f = time_form(ctx, p, sa.SIM_FP64, K, args.warmup, 0, 50, autotune=False)
    r = time_form(ctx, p, sa.SIM_MIXED, K, args.warmup, 0, 50, autotune=False)
    out = {"workload": workload_desc("chain"), "value": K / (f["t_ms"] / 1e3),
           "unit": "steps/s", "form": "plain FP64", "iterations": iter_summary(f["stats"]),
           "mixed": {"value": K / (r["t_ms"] / 1e3), "unit": "steps/s"},
           "us_per_iteration_fp64": f["t_ms"] * 1e3 / (K * 100)}
    f["sim"].close()
    r["sim"].close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--robots", type=int, default=64)
    ap.add_argument("--workload", default="batched", choices=list(WORKLOADS),
                    help="batched: 4096 uneven scenes in one launch per class (the headline); "
                         "robots: 64 legged robots; fem_beam: one tetrahedral FEM beam of 64 "
                         "slabs held by a 7-R arm; chain: the 8-link chain at 100 iterations")
    ap.add_argument("--scenes", type=int, default=4096, help="scenes of the batched workload")
    ap.add_argument("--preroll", type=int, default=-1,
                    help="untimed steps before warm-up (default: per workload)")
    ap.add_argument("--reference-scenes", type=int, default=0,
                    help="scenes the CPU oracle steps (a prefix of the batch; 0: per workload)")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--reference-seconds", type=float, default=120.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--steps-per-launch", type=int, default=50)
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the heuristic kernel variants instead of timing them first")
    ap.add_argument("--no-graph", action="store_true", help="launch directly, not by graph replay")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned warm start")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip timing the plain FP64 form next to the chosen one")
    ap.add_argument("--no-sub", action="store_true", help="headline workload only")
    ap.add_argument("--refactor", action="store_true",
                    help="refactorise every block every step (sim_keep_factors(0), Algorithm 1 "
                         "as stated) in the headline workload's timing")
    ap.add_argument("--subs", default="robots,fem_beam,chain,cable,stir",
                    help="comma-separated sub-results to run (robots, fem_beam, chain, cable, "
                         "stir)")
    ap.add_argument("--sub-only", action="store_true",
                    help="skip the headline workload's GPU timing (sub-results only)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    from paper_2302_14344_gb300 import subadmm

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    ctx = Ctx(subadmm, stream, dev, local, dist, flush)
    wl = WORKLOADS[args.workload]
    preroll = wl["preroll"] if args.preroll < 0 else args.preroll
    threads = os.cpu_count() or 1

    p = make_problem(args.workload, rank, args.robots, args.scenes)
    work = algorithmic_work(p)
    K = args.steps
    spl = max(1, min(args.steps_per_launch, K))
    mixed_form = args.workload != "chain"
    prec = subadmm.SIM_MIXED if mixed_form else subadmm.SIM_FP64
    grid_scene = args.workload == "fem_beam"
    # the chosen form of the batched workload: the learned warm start (duals and beta scales,
    # network trained here on the GPU), batched, mixed precision
    learned = (not args.no_learned) and args.workload == "batched"
    if learned or (not args.no_learned and world == 1 and not args.no_sub):
        ctx.net, ctx.net_info = train_warmstart()
    prev = None
    if learned:
        rp = time_form(ctx, p, prec, K, args.warmup, preroll, spl, autotune=not args.no_autotune,
                       graph=not args.no_graph)
        prev = {"value": whole_job_rate(world, K, rp["t_ms"]), "unit": "steps/s",
                "ms_per_step": rp["t_ms"] / K, "iterations": iter_summary(rp["stats"]),
                "note": "mixed precision, batched, previous-step warm start (trace-rule beta), "
                        "same segment and launches"}
        rp["sim"].close()
    r = time_form(ctx, p, prec, K, args.warmup, preroll, spl, autotune=not args.no_autotune,
                  graph=not (args.no_graph or grid_scene), sample_clocks=True,
                  net=ctx.net if learned else None, keep_factors=not args.refactor)
    sim, t_ms, stats = r["sim"], r["t_ms"], r["stats"]
    sizes = sim.sizes()
    value = whole_job_rate(world, K, t_ms)
    if args.workload == "fem_beam":
        tsize = 4
        d_bytes = float(sum(w[2] for w in work)) * tsize
        hbm = measured_peaks().get("hbm_gbs")
        gbs = d_bytes * stats["total_iters"] / (t_ms / 1e3) / 1e9
        roofline = {"bound": "hbm", "achieved": gbs, "peak": hbm or 6800.0, "unit": "GB/s",
                    "frac": gbs / (hbm or 6800.0),
                    "traffic": recorded_traffic_fem(stats["total_iters"] / len(r["chunks"])),
                    "note": "D of every subsystem once per iteration x iterations / whole-step "
                            "time; peak = " + ("measured copy bandwidth" if hbm else "fallback")}
    else:
        traffic = None
        if args.workload == "robots" and args.robots == 64:
            traffic = recorded_traffic(spl)
        elif args.workload == "batched":
            traffic = recorded_traffic_batched(spl, len(p.scenes))
        roofline = alu_roofline(p, work, stats, t_ms, mixed_form, K, traffic)

    compare = None
    if not args.no_compare and mixed_form:
        f = time_form(ctx, p, subadmm.SIM_FP64, K, args.warmup, preroll, spl,
                      autotune=not args.no_autotune, graph=not (args.no_graph or grid_scene),
                      keep_factors=not args.refactor)
        compare = {"value": whole_job_rate(world, K, f["t_ms"]), "unit": "steps/s",
                   "ms_per_step": f["t_ms"] / K, "iterations": iter_summary(f["stats"])}
        compare["chosen_over_plain"] = value / compare["value"]
        f["sim"].close()

    if prev is not None:
        prev["learned_over_previous"] = value / prev["value"]
    e2e = e2e_rate(ctx, sim, min(K, 200), world, net=ctx.net if learned else None)
    e2e["segment"] = (f"steps {1 + preroll + args.warmup + K}.."
                      f"{1 + preroll + args.warmup + K + e2e['steps']} of the run")
    sim.close()

    subs = {}
    if not args.no_sub and world == 1:
        jobs = {"robots_after_landing": lambda: sub_robots(ctx, args, threads),
                "fem_beam": lambda: sub_fem_beam(ctx, args, threads),
                "chain_fixed_100_iterations": lambda: sub_chain(ctx, args),
                "cable_fixed_90_iterations": lambda: sub_cable(ctx, args),
                "stir_fixed_30_60_90_iterations": lambda: sub_stir(ctx, args)}
        wanted = [w.strip() for w in args.subs.split(",") if w.strip()]
        for name, fn in jobs.items():
            if name.startswith(args.workload) or not any(name.startswith(w) for w in wanted):
                continue
            try:
                subs[name] = fn()
            except Exception as e:                   # reported, not fatal to the line
                subs[name] = {"error": repr(e)}

    if rank == 0:
        n_if = sum(len(sc.ifs) for sc in p.scenes) / max(len(p.scenes), 1)
        line = {
            "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": t_ms / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if mixed_form else "f64", "data": "synthetic",
            "config": {"workload": workload_desc(args.workload, args.robots, args.scenes),
                       "form": (("chosen: learned warm start (a 32-256-256-256-7 network, "
                                 "trained here, proposes each interface's initial duals and a "
                                 "beta scale; evaluated once per launch) + " if learned else
                                 "chosen: ") +
                                "mixed precision (FP64 assembly, beta and final residual "
                                "check; FP32 factor for non-stiff blocks, FP64 for stiff ones; "
                                "FP32 iterations), batched, graph replay, autotuned")
                               if mixed_form else "plain FP64",
                       "scenes_per_gpu": sizes["scenes"],
                       "subsystems": sizes["subsystems"], "dof": sizes["dof"],
                       "interfaces": sizes["interfaces"], "rows": sizes["rows"],
                       "side_rows": sizes["side_rows"], "parallelism": f"scenes x{world}",
                       "l2": "flushed between timed launches (512 MiB write)",
                       "launch": f"{spl} steps per launch, one launch per class of scenes "
                                 f"(classes on forked streams)"
                                 + ("" if (args.no_graph or grid_scene) else
                                    ", replayed as a CUDA graph"),
                       "launch_classes": r["classes"],
                       "kernel_variants": "heuristic" if args.no_autotune else
                                          "autotuned on the pre-rolled state (sim_autotune, "
                                          "3 steps per variant, state restored)",
                       "factors": ("every block refactorised every step" if args.refactor
                                   else "constant blocks' factors kept across steps"),
                       "preroll_steps": preroll,
                       "timed_segment": f"steps {1 + preroll + args.warmup}.."
                                        f"{1 + preroll + args.warmup + K} of a run from rest "
                                        f"(1 first step, {preroll} untimed pre-roll, "
                                        f"{args.warmup} warm-up)"},
            "iterations": iter_summary(stats),
            "interface_updates_per_s": n_if * stats["total_iters"] * world / (t_ms / 1e3),
            "plain_fp64": compare,
            "mixed_previous_step_start": prev,
            "learned_training": ctx.net_info if learned else None,
            "roofline": roofline,
            "e2e": e2e,
            # kernels per timed launch: one per launch class, plus features, weight packing,
            # the fused network, learned duals and the two beta-scale kernels when learned
            # (a refactorising grid scene adds its blocked factorisation's and Gram kernel's
            # launches, which this count leaves out)
            "gpu_launches": len(r["launch_ms"]) * (len(r["classes"]) + (6 if learned else 0)),
            "clocks": r["clocks"],
            "launch_ms": {"mean": statistics.mean(r["launch_ms"]),
                          "median": statistics.median(r["launch_ms"]),
                          "min": min(r["launch_ms"]), "max": max(r["launch_ms"])},
        }
        if not args.no_cpu_baseline and world == 1:
            if args.workload == "fem_beam":
                fr = oracle_fem_rate(threads)
                mi = line["iterations"]["mean_per_scene_step"]
                line["cpu_baseline"] = {
                    "value": 1.0 / (fr["setup_s"] + fr["per_iter_s"] * mi), "unit": "steps/s",
                    "cores": threads, "kind": "oracle", "cpu": host_cpu(),
                    "sample": f"first step at 1 and 41 iterations, OpenMP build, extrapolated "
                              f"to {mi:.0f} iterations per step"}
            else:
                line["cpu_baseline"] = oracle_rate(args.workload, p, preroll + 1, args.warmup,
                                                   K, threads, args.cpu_seconds,
                                                   args.reference_scenes or wl["cpu_scenes"])
        line["sub_results"] = subs or None
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
