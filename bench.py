"""Benchmark: simulation steps per second of the 64-legged-robot batch, every step iterated
to primal residual <= 1e-6, on GB300 through libsubadmm (the C ABI in include/subadmm.h).

One benchmark step = one time step of the whole batch: assembly, beta, factorisation, the
ADMM loop to the stop rule, v-hat and the state update, all in the step kernel.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun every rank simulates its own seeded batch
(scenes are independent: weak scaling, no data-path collective).  --impl reference times
the FP64 CPU oracle on the host cores instead.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "sim steps/sec at primal residual ≤1e-6, chosen form vs plain FP64, 1 GB300"
FP64_NOMINAL_TFLOPS = 1.25     # GB300 nominal FP64 (non-tensor) rate
FP32_NOMINAL_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # 152 SMs x 128 FP32 lanes x FMA x clock
L2_FLUSH_BYTES = 512 << 20     # > 129 MB L2


def workload_desc(n_robots: int, h: float, workload: str = "robots", scenes: int = 0) -> str:
    if workload == "fem_beam":
        return (f"one linear-elastic tetrahedral beam 0.5 x 0.05 x 0.05 m (10 x 10 nodes x 137 "
                f"planes, Kuhn split, E=1e5 Pa, nu=0.45, rho=1000) cut into 64 slabs of 900/1200 "
                f"DOF joined by node-node equality (18,900 rows), 2,000 speculative ground "
                f"contacts mu=0.5, a 7-R arm (one rigid subsystem, PD drives) holding one end by "
                f"ball joints; h={h:g} s; each step iterated to r_p<=1e-6 with the previous "
                f"step's warm start")
    if workload == "batched":
        return (f"{scenes} independent uneven scenes of 2-32 subsystems each: rigid chains of "
                f"1-8 bodies and linear spring-lattice blocks of 6-240 DOF, tree + chord ball "
                f"joints, node plane contacts mu=0.5; h={h:g} s; each step iterated to "
                f"r_p<=1e-6 with the previous step's warm start")
    return (f"{n_robots} independent legged robots (6-DOF trunk + 4 legs x 3 revolute joints, "
            f"one subsystem per leg and one for the trunk, PD drives as soft rows, 4 point-foot "
            f"plane contacts mu=0.8), dropped from 0.3-0.5 m; h={h:g} s; each step iterated to "
            f"r_p<=1e-6 with the previous step's warm start")


def algorithmic_work(problem):
    """Per-scene algorithmic FLOPs of the method (triangular-solve form of Eq. admm-1i):
    per iteration and subsystem 2 n^2 (two triangular solves) + 4 nnz(J_i) (J^T w and J v)
    + 20 m_i (projection, updates, residuals); per step and subsystem n^3/3 (Cholesky)
    + 2 sum_rows nnz(row)^2 (K = A + beta J^T J)."""
    import numpy as np
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


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def cpu_baseline(problem, seconds: float, sample_scenes: int = 64):
    """Time the FP64 CPU oracle, as it stands, on a bounded sample of the same workload: the
    first steps of the first ``sample_scenes`` scenes of the batch (all of them when the batch
    is no larger; the scenes are drawn independently, so a prefix is a random sample), until
    ``seconds`` have elapsed.  The rate is scaled to whole-batch steps per second."""
    import oracle
    n_all = len(problem.scenes)
    scs = [oracle.OracleScene(sc, problem.options) for sc in problem.scenes[:sample_scenes]]
    t0 = time.perf_counter()
    steps = 0
    iters = 0
    while True:
        for o in scs:
            o.step()
            iters += o.residuals()["iters"]
        steps += 1
        if time.perf_counter() - t0 >= seconds or steps >= 500:
            break
    dt = time.perf_counter() - t0
    frac = len(scs) / n_all
    which = (f"all {n_all} scenes" if len(scs) == n_all else
             f"the first {len(scs)} of {n_all} scenes, rate scaled by {len(scs)}/{n_all}")
    return {"value": steps / dt * frac, "unit": "steps/s", "cores": 1, "kind": "oracle",
            "sample": f"first {steps} steps of {which} (whole sample per step), "
                      f"single-threaded plain C -O2, {iters / max(steps * len(scs), 1):.1f} "
                      f"iterations per scene-step",
            "seconds": dt}


def cpu_baseline_one_scene(args, h: float, mean_iters: float):
    """The FP64 CPU oracle, as it stands, on one large scene: one step takes minutes, so the
    first step is timed at 1 and at 4 ADMM iterations; their difference gives the time per
    iteration, the rest the per-step assembly and factorisation; the rate is extrapolated
    to the GPU run's mean iterations per step."""
    import oracle
    import scenegen as sg
    times = {}
    for k in (1, 4):
        p = sg.fem_beam(seed=0, h=h, tol_primal=-1, max_iters=k)
        o = oracle.OracleScene(p.scenes[0], p.options)
        t0 = time.perf_counter()
        o.step()
        times[k] = time.perf_counter() - t0
    per_iter = (times[4] - times[1]) / 3.0
    setup = times[1] - per_iter
    step_s = setup + per_iter * mean_iters
    return {"value": 1.0 / step_s, "unit": "steps/s", "cores": 1, "kind": "oracle",
            "sample": f"first step at 1 and 4 iterations ({times[1]:.1f} s, {times[4]:.1f} s): "
                      f"{setup:.1f} s assembly and factorisation + {per_iter * 1e3:.0f} ms per "
                      f"iteration, extrapolated to {mean_iters:.0f} iterations per step; "
                      f"single-threaded plain C -O2",
            "seconds": times[1] + times[4]}


def run_reference(args, rank: int, world: int):
    """The reference arm: the FP64 CPU oracle, as it stands, on the same workload (rank 0
    only); for a batch larger than ``--reference-scenes`` a prefix of that many scenes is
    stepped and the rate scaled to whole-batch steps."""
    if rank != 0:
        return 0
    import oracle
    h = 2e-3 if args.workload == "robots" else 1e-3
    if args.workload == "fem_beam":
        cb = cpu_baseline_one_scene(args, h, 500.0)
        line = {"metric": METRIC, "value": cb["value"], "unit": "steps/s", "n_gpus": world,
                "steps": 1, "warmup": 0, "ms_per_step": 1e3 / cb["value"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "impl": "reference",
                "config": {"workload": workload_desc(args.robots, h, args.workload),
                           "form": "FP64 CPU oracle"},
                "cpu_baseline": cb,
                "e2e": {"value": cb["value"], "unit": "steps/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0
    p = batch_for_rank(0, args.robots, h, args.workload, args.scenes)
    n_all = len(p.scenes)
    scs = [oracle.OracleScene(sc, p.options) for sc in p.scenes[:args.reference_scenes]]
    # warm-up steps, then time K steps bounded to a few minutes
    for _ in range(args.warmup):
        for o in scs:
            o.step()
    t0 = time.perf_counter()
    k = 0
    for k in range(1, args.steps + 1):
        for o in scs:
            o.step()
        if time.perf_counter() - t0 > args.reference_seconds:
            break
    dt = time.perf_counter() - t0
    frac = len(scs) / n_all
    val = k / dt * frac
    which = (f"all {n_all} scenes" if len(scs) == n_all else
             f"the first {len(scs)} of {n_all} scenes, rate scaled by {len(scs)}/{n_all}")
    line = {"metric": METRIC, "value": val, "unit": "steps/s", "n_gpus": world, "steps": k,
            "warmup": args.warmup, "ms_per_step": 1e3 / val, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": workload_desc(args.robots, h, args.workload, args.scenes),
                       "robots": args.robots, "form": "FP64 CPU oracle"},
            "cpu_baseline": {"value": val, "unit": "steps/s", "cores": 1, "kind": "oracle",
                             "sample": f"steps {args.warmup}..{args.warmup + k} of {which}"},
            "e2e": {"value": val, "unit": "steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def learned_comparison(args, p) -> dict:
    """The learned warm start against the previous-step warm start on this workload: the
    network is trained on robots of two other seeds after landing (steps 200-400), then
    both starts run the timed segment (mixed form, one launch per step, graph replay)."""
    import scenegen as sg
    import torch
    from paper_2302_14344_gb300 import learned as lr
    t0 = time.perf_counter()
    parts = [lr.collect(sg.robots(s, n_robots=args.robots), steps=200, warmup=200)
             for s in (101, 102)]
    X = torch.cat([q[0] for q in parts]); T = torch.cat([q[1] for q in parts])
    M = torch.cat([q[2] for q in parts])
    net = lr.init_network(seed=1)
    losses = lr.train(net, X, T, M, epochs=8)
    train_s = time.perf_counter() - t0
    res = lr.compare(p, net, steps=args.steps, warmup=args.warmup)
    pl, le = res["plain"], res["learned"]
    return {"value": 1e3 / le["ms_per_step"], "unit": "steps/s",
            "previous_step_start": 1e3 / pl["ms_per_step"],
            "learned_over_previous": pl["ms_per_step"] / le["ms_per_step"],
            "iterations_per_scene_step": {"learned": le["iters_per_scene_step"],
                                          "previous_step": pl["iters_per_scene_step"]},
            "fallbacks": le["fallbacks"], "scene_steps": args.steps * len(p.scenes),
            "training": {"samples": int(X.shape[0]), "epochs": 8,
                         "loss_first_last": [losses[0], losses[-1]],
                         "seconds": round(train_s, 1)},
            "note": "both starts stepped one launch per step (graph replay), timed segment "
                    "of this run; the network adds features + a 32-256-256-256-7 BF16 MLP "
                    "per step"}


def batch_for_rank(rank: int, n_robots: int, h: float, workload: str = "robots",
                   scenes: int = 4096):
    """The scenes a rank simulates: an independent seeded batch per rank (weak scaling; the
    scenes never exchange data, so the ranks share no data-path collective)."""
    import scenegen as sg
    if workload == "batched":
        return sg.batched(seed=rank, n_scenes=scenes, h=h, tol_primal=1e-6, max_iters=1000)
    if workload == "fem_beam":
        return sg.fem_beam(seed=rank, h=h, tol_primal=1e-6, max_iters=1000)
    return sg.robots(seed=rank, n_robots=n_robots, h=h, tol_primal=1e-6, max_iters=1000)


def whole_job_rate(world: int, steps: int, t_ms_max: float) -> float:
    """Steps of every rank's batch per second over the slowest rank's time."""
    return world * steps / (t_ms_max / 1e3)


def time_refactor_every_step(subadmm, p, stream, dev, local, flush, steps: int = 3):
    """The plain FP64 form with every block factorised again every step (Algorithm 1 as
    stated; by default a constant block's factor, the same matrix, is computed once):
    `steps` steps after one warm-up step, one launch each, L2 flushed before each."""
    import torch
    sim = subadmm.Simulation(p, stream=stream.cuda_stream, device=local,
                             precision=subadmm.SIM_FP64)
    sim.keep_factors(False)
    sim.step(1)
    sim.sync()
    sim.iteration_stats()   # clear counters
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    torch.cuda.synchronize(dev)
    for a, b in ev:
        flush.zero_()
        a.record(stream)
        sim.step(1)
        b.record(stream)
    torch.cuda.synchronize(dev)
    t = float(sum(a.elapsed_time(b) for a, b in ev))
    st = sim.iteration_stats()
    sim.close()
    return {"value": steps / (t / 1e3), "unit": "steps/s", "ms_per_step": t / steps,
            "steps": steps, "mean_iterations": st["total_iters"] / max(st["scene_steps"], 1),
            "note": "every block refactorised every step (sim_keep_factors(0)); timed segment "
                    "right after the first step, heuristic kernel variant, no graph"}


def time_form(subadmm, p, precision, args, stream, dev, local, dist, flush, sample_clocks):
    """Warm-up W steps, then K timed steps in launches of ``--steps-per-launch`` steps (the
    scenes are independent, so one launch advances every scene by that many steps without a
    device-wide wait per step).  The L2 is flushed before every timed launch."""
    import torch
    sim = subadmm.Simulation(p, stream=stream.cuda_stream, device=local, precision=precision)
    sim.step(1)
    tuned = sim.launch_classes() if args.no_autotune else sim.autotune(steps=3)
    if not args.no_graph:
        sim.use_graph(True)
    for _ in range(args.warmup - 1):
        sim.step(1)
    sim.sync()
    sim.iteration_stats()   # clear counters
    K = args.steps
    spl = max(1, min(args.steps_per_launch, K))
    chunks = [spl] * (K // spl) + ([K % spl] if K % spl else [])
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in chunks]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in chunks]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clk = ClockSampler(local) if sample_clocks else None
    if clk:
        clk.__enter__()
    for k, n in enumerate(chunks):
        flush.zero_()                      # L2 flushed between timed launches
        ev0[k].record(stream)
        sim.step(n)
        ev1[k].record(stream)
    torch.cuda.synchronize(dev)
    if clk:
        clk.__exit__()
    if dist is not None:
        dist.barrier()
    launch_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    t_ms = float(sum(launch_ms))
    if dist is not None:
        tt = torch.tensor([t_ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_ms = float(tt.item())
    stats = sim.iteration_stats(per_scene=True)
    stats["classes"] = tuned
    return sim, t_ms, launch_ms, stats, (clk.summary() if clk else None)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--robots", type=int, default=64)
    ap.add_argument("--workload", default="robots", choices=["robots", "batched", "fem_beam"],
                    help="robots: 64 legged robots (the headline workload); batched: many "
                         "uneven scenes of rigid chains and spring blocks in one launch; "
                         "fem_beam: one tetrahedral FEM beam of 64 slabs held by a 7-R arm")
    ap.add_argument("--scenes", type=int, default=4096, help="scenes of the batched workload")
    ap.add_argument("--reference-scenes", type=int, default=64,
                    help="scenes the reference arm steps (a prefix of the batch)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--reference-seconds", type=float, default=120.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--form", default="mixed", choices=["mixed", "fp64"],
                    help="mixed: FP32 iterations with FP64 setup and residual check (the "
                         "chosen form); fp64: the plain FP64 form")
    ap.add_argument("--steps-per-launch", type=int, default=50)
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the heuristic kernel variants instead of timing them first")
    ap.add_argument("--no-graph", action="store_true", help="launch directly, not by graph replay")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned warm start comparison (robots workload)")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip timing the plain FP64 form next to the chosen one")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import scenegen as sg
    from paper_2302_14344_gb300 import subadmm

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    h = 2e-3 if args.workload == "robots" else 1e-3
    p = batch_for_rank(rank, args.robots, h, args.workload, args.scenes)
    work = algorithmic_work(p)
    it_flops = np.array([w[0] for w in work])
    st_flops = float(sum(w[1] for w in work))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    forms = {"mixed": subadmm.SIM_MIXED, "fp64": subadmm.SIM_FP64}

    sim, t_ms, launch_ms, stats, clocks = time_form(subadmm, p, forms[args.form], args, stream,
                                                  dev, local, dist, flush, True)
    K = args.steps
    sizes = sim.sizes()
    value = whole_job_rate(world, K, t_ms)
    total_iters = stats["total_iters"]
    flops = float(it_flops @ stats["per_scene"][:, 0]) + st_flops * K
    achieved = flops / (t_ms / 1e3) / 1e12
    if args.form == "mixed":
        peak, pipe = FP32_NOMINAL_TFLOPS, "FP32"
    else:
        peak, pipe = FP64_NOMINAL_TFLOPS, "FP64"
    spl = max(1, min(args.steps_per_launch, K))
    if args.workload == "fem_beam":
        # one scene over the whole GPU: every iteration streams each subsystem's D (m_i x m_i)
        # from HBM (125 MB in FP32, more than L2 holds), so the bound is HBM bandwidth
        tsize = 4 if args.form == "mixed" else 8
        d_bytes = float(sum(w[2] for w in work)) * tsize
        hbm = measured_peaks().get("hbm_gbs")
        achieved_gbs = d_bytes * total_iters / (t_ms / 1e3) / 1e9
        launches = (K + spl - 1) // spl
        roofline = {"bound": "hbm", "achieved": achieved_gbs,
                    "peak": hbm if hbm else 6800.0, "unit": "GB/s",
                    "frac": achieved_gbs / (hbm if hbm else 6800.0),
                    "traffic": (recorded_traffic_fem(total_iters / launches)
                                if args.form == "mixed" else None),
                    "note": f"algorithmic bytes: D of every subsystem once per iteration "
                            f"({d_bytes / 1e6:.1f} MB) x iterations / whole-step time (setup and "
                            f"exit included, so a lower bound on the stream rate); peak = "
                            f"{'measured copy bandwidth' if hbm else 'fallback'}"}
    else:
        roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak,
                    # the recorded capture is of the 64-robot batch in the mixed form
                    "traffic": (recorded_traffic(spl) if args.workload == "robots" and
                                args.robots == 64 and args.form == "mixed" else None),
                    "note": f"{pipe} non-tensor pipe (iterations; the mixed form's per-step "
                            f"setup is FP64); peak = 152 SMs x lanes x 2 flops x 2.07 GHz; "
                            f"algorithmic flops of the triangular-solve form, "
                            f"{it_flops.mean():.0f} per scene-iteration (mean over scenes) and "
                            f"{st_flops / len(p.scenes):.0f} per scene-step"}

    compare = None
    if not args.no_compare and args.form != "fp64":
        sim2, t2, sm2, st2, _ = time_form(subadmm, p, subadmm.SIM_FP64, args, stream, dev, local,
                                          dist, flush, False)
        compare = {"value": world * K / (t2 / 1e3), "unit": "steps/s", "ms_per_step": t2 / K,
                   "mean_iterations": st2["total_iters"] / max(st2["scene_steps"], 1),
                   "not_converged": st2["not_converged"],
                   "chosen_over_plain": (world * K / (t_ms / 1e3)) / (world * K / (t2 / 1e3))}
        sim2.close()
    refactor = None
    if args.workload == "fem_beam" and not args.no_compare and world == 1:
        refactor = time_refactor_every_step(subadmm, p, stream, dev, local, flush)

    learned_line = None
    if args.workload == "robots" and not args.no_learned and world == 1:
        learned_line = learned_comparison(args, p)

    # end to end through the C ABI with host buffers: state in from pinned host memory,
    # one step, state out to pinned host memory, every step
    nstate = 13 * sizes["bodies"] + 6 * sizes["nodes"]
    hbuf = torch.empty(nstate, dtype=torch.float64).pin_memory()
    subadmm.sim_read_state(sim.h, hbuf.data_ptr())
    e2e_steps = min(K, 200)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        subadmm.sim_write_state(sim.h, hbuf.data_ptr())
        sim.step(1)
        subadmm.sim_read_state(sim.h, hbuf.data_ptr())
    e2e_dt = time.perf_counter() - t0
    if dist is not None:
        tt = torch.tensor([e2e_dt], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_dt = float(tt.item())
    e2e = {"value": world * e2e_steps / e2e_dt, "unit": "steps/s",
           "h2d_bytes_per_step": 8 * nstate, "d2h_bytes_per_step": 8 * nstate,
           "steps": e2e_steps, "timer": "host wall clock",
           "segment": f"steps {args.warmup + K}..{args.warmup + K + e2e_steps} of the run"}

    if rank == 0:
        n_if = sum(len(sc.ifs) for sc in p.scenes) / max(len(p.scenes), 1)
        line = {
            "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": t_ms / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.form == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": workload_desc(args.robots, h, args.workload, args.scenes),
                       "form": ("mixed: FP64 assembly, factorisation and residual check, "
                                "FP32 iterations") if args.form == "mixed" else "plain FP64",
                       "robots": args.robots, "scenes_per_gpu": sizes["scenes"],
                       "subsystems": sizes["subsystems"], "dof": sizes["dof"],
                       "interfaces": sizes["interfaces"], "rows": sizes["rows"],
                       "side_rows": sizes["side_rows"], "parallelism": f"scenes x{world}",
                       "l2": "flushed between timed steps (512 MiB write)",
                       "launch": f"step kernel, {min(args.steps_per_launch, K)} steps per launch, "
                                 f"one block of 256 threads per scene, one launch per class of "
                                 f"scenes (classes on forked streams)"
                                 + ("" if args.no_graph else ", replayed as a CUDA graph"),
                       "launch_classes": stats["classes"],
                       "kernel_variants": "heuristic" if args.no_autotune else
                                          "autotuned (sim_autotune, 3 steps per variant)",
                       "timed_segment": f"steps {args.warmup}..{args.warmup + K} of a run from "
                                        f"the drop"},
            "iterations": {"mean_per_scene_step": total_iters / max(stats["scene_steps"], 1),
                           "max": stats["max_iters"], "not_converged": stats["not_converged"],
                           "scene_steps": stats["scene_steps"]},
            "interface_updates_per_s": n_if * total_iters * world / (t_ms / 1e3),
            "plain_fp64": compare,
            "plain_fp64_refactor_every_step": refactor,
            "learned_warm_start": learned_line,
            "roofline": roofline,
            "e2e": e2e,
            "gpu_launches": len(launch_ms) * len(stats["classes"]),
            "clocks": clocks,
            "launch_ms": {"mean": statistics.mean(launch_ms),
                          "median": statistics.median(launch_ms),
                          "min": min(launch_ms), "max": max(launch_ms)},
        }
        if not args.no_cpu_baseline and world == 1:
            if args.workload == "fem_beam":
                line["cpu_baseline"] = cpu_baseline_one_scene(
                    args, h, total_iters / max(stats["scene_steps"], 1))
            else:
                line["cpu_baseline"] = cpu_baseline(batch_for_rank(0, args.robots, h,
                                                                   args.workload, args.scenes),
                                                    args.cpu_seconds)
        print(json.dumps(line), flush=True)
    sim.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
