"""The learned warm start, end to end: collect training samples from the plain simulator,
train the warm-start network on the GPU, and step with it.

Orchestration only: features, targets, the network's forward and backward passes and the
optimiser all run in the library's kernels (sim_interface_features, sim_interface_targets,
wsn_*); torch holds the device arrays and shuffles minibatches.
"""
from __future__ import annotations

from typing import Iterable, List, Tuple

import numpy as np

from . import subadmm as sa
from .warmstart import Network, join_params

FEATURES, OUTPUTS = 32, 7
SIZES = [FEATURES, 256, 256, 256, OUTPUTS]


def collect(problem, steps: int, warmup: int = 5, precision: int = sa.SIM_MIXED,
            device: int = 0):
    """Run the plain simulator (previous-step warm start) and record, for every interface
    of every step, the features at the step's start and the dual change the step made.
    Returns device tensors (X: n x 32, T: n x 7, M: n x 7)."""
    import torch
    sim = sa.Simulation(problem, device=device, precision=precision)
    sim.step(warmup)
    nif = sim.sizes()["interfaces"]
    xs, ts, ms = [], [], []
    for _ in range(steps):
        x = torch.empty((nif, FEATURES), device=f"cuda:{device}")
        t = torch.empty((nif, OUTPUTS), device=f"cuda:{device}")
        m = torch.empty((nif, OUTPUTS), device=f"cuda:{device}")
        sa.sim_interface_features(sim.h, x.data_ptr())
        sim.step(1)
        sa.sim_interface_targets(sim.h, x.data_ptr(), t.data_ptr(), m.data_ptr())
        xs.append(x); ts.append(t); ms.append(m)
    sim.sync()
    sim.close()
    return torch.cat(xs), torch.cat(ts), torch.cat(ms)


SCALES = [2.0 ** k for k in range(-3, 4)]    # candidate beta scales of the rho search
REF = 3                                       # index of scale 1 (the trace rule)


def _replicate(problem, copies: int):
    import scenegen as sg
    return sg.Problem([sc for _ in range(copies) for sc in problem.scenes], problem.options,
                      name=f"{problem.name}x{copies}")


def collect_rho(problem, steps: int, warmup: int = 5, precision: int = sa.SIM_MIXED,
                device: int = 0, slack: float = 0.0):
    """Samples from the plain simulator, with the best beta scale of each scene-step as the
    label of the network's seventh output.  Every scene runs in seven copies, copy k with
    every subsystem's beta scaled by 2^(k-3) (k = 3: the trace rule, Sec. III-D); after each
    step the copies' iteration counts give each scene's best scale (fewest iterations to the
    stop rule, ties to the scale nearest 1) and every copy is reset to the trace-rule copy's
    state, so that all copies start each step from the plain trajectory.  With ``slack`` > 0
    the label is the largest scale within (1 + slack) of the fewest iterations: too small a
    beta costs far more iterations than too large a one, so under an uncertain proposal the
    larger of near-equal scales is the safer label.  Features and dual targets are the
    trace-rule copy's.  Returns device tensors (X, T, M) like collect()."""
    import torch
    nsc = len(problem.scenes)
    rep = _replicate(problem, len(SCALES))
    sim = sa.Simulation(rep, device=device, precision=precision)
    nsub_copy = sum(len(sc.subs) for sc in problem.scenes)
    sim.set_beta_scale([SCALES[c] for c in range(len(SCALES)) for _ in range(nsub_copy)])
    sz = sim.sizes()
    nb = sz["bodies"] // len(SCALES)
    nn = sz["nodes"] // len(SCALES)
    state = torch.empty(13 * sz["bodies"] + 6 * sz["nodes"], dtype=torch.float64).pin_memory()

    def sync_copies():
        sa.sim_read_state(sim.h, state.data_ptr())
        bodies = state[: 13 * sz["bodies"]].view(len(SCALES), 13 * nb)
        nodes = state[13 * sz["bodies"]:].view(len(SCALES), 6 * nn)
        bodies[:] = bodies[REF].clone()
        nodes[:] = nodes[REF].clone()
        sa.sim_write_state(sim.h, state.data_ptr())

    for _ in range(warmup):
        sim.step(1)
        sync_copies()
    nif = sz["interfaces"]
    nif0 = nif // len(SCALES)
    per_scene_if = torch.tensor([len(sc.ifs) for sc in problem.scenes], device=f"cuda:{device}")
    order = sorted(range(len(SCALES)), key=lambda k: abs(k - REF))
    sim.iteration_stats()
    xs, ts, ms = [], [], []
    for _ in range(steps):
        x = torch.empty((nif, FEATURES), device=f"cuda:{device}")
        t = torch.empty((nif, OUTPUTS), device=f"cuda:{device}")
        m = torch.empty((nif, OUTPUTS), device=f"cuda:{device}")
        sa.sim_interface_features(sim.h, x.data_ptr())
        sim.step(1)
        sa.sim_interface_targets(sim.h, x.data_ptr(), t.data_ptr(), m.data_ptr())
        st = sim.iteration_stats(per_scene=True)["per_scene"]
        it = np.asarray(st[:, 0]).reshape(len(SCALES), nsc)
        nc = np.asarray(st[:, 2]).reshape(len(SCALES), nsc)
        best = np.zeros(nsc)
        for sc in range(nsc):
            cand = [k for k in order if nc[k, sc] == 0] or [REF]
            kb = min(cand, key=lambda k: (it[k, sc], abs(k - REF)))
            if slack > 0.0:
                kb = max(k for k in cand if it[k, sc] <= (1.0 + slack) * it[kb, sc])
            best[sc] = kb - REF
        lo, hi = REF * nif0, (REF + 1) * nif0
        label = torch.repeat_interleave(torch.tensor(best, dtype=torch.float32,
                                                     device=f"cuda:{device}"), per_scene_if)
        t_ref = t[lo:hi].clone()
        t_ref[:, OUTPUTS - 1] = label
        xs.append(x[lo:hi].clone()); ts.append(t_ref); ms.append(m[lo:hi].clone())
        sync_copies()
    sim.sync()
    sim.close()
    return torch.cat(xs), torch.cat(ts), torch.cat(ms)


def init_network(seed: int = 0, device: int = 0) -> Network:
    """He-initialised weights (drawn on the host from a seeded generator), zero biases."""
    rng = np.random.default_rng(seed)
    params = [(rng.standard_normal((a, b)) * np.sqrt(2.0 / a), np.zeros(b))
              for a, b in zip(SIZES[:-1], SIZES[1:])]
    net = Network(SIZES, device=device)
    net.set_params(join_params(params).astype(np.float32))
    return net


def train(net: Network, X, T, M, epochs: int = 3, batch: int = 4096, lr: float = 1e-3,
          seed: int = 0) -> List[float]:
    """Fit the normalisation on the data, then Adam over shuffled minibatches; returns the
    mean loss of each epoch."""
    import torch
    net.fit_normalization(X, T)
    g = torch.Generator(device=X.device)
    g.manual_seed(seed)
    n = X.shape[0]
    out = []
    for _ in range(epochs):
        perm = torch.randperm(n, device=X.device, generator=g)
        loss = torch.zeros(1, device=X.device)
        nb = 0
        for lo in range(0, n - batch + 1, batch):
            idx = perm[lo:lo + batch]
            net.train_step(X.index_select(0, idx).contiguous(), T.index_select(0, idx).contiguous(),
                           M.index_select(0, idx).contiguous(), lr, loss)
            nb += 1
        out.append(loss.item() / max(nb, 1))
    return out


def compare(problem, net: Network, steps: int, warmup: int = 5,
            precision: int = sa.SIM_MIXED, device: int = 0, learned_warmup: int = 0,
            per_launch: int = 1) -> dict:
    """The same start, stepped with the previous-step warm start and with the learned one,
    both in launches of ``per_launch`` steps (graph replay; the learned form evaluates the
    network once per launch): iterations per scene-step of each, fallbacks of the learned
    start, and the wall time of the device work (CUDA events).  ``learned_warmup`` launches
    of each form run untimed first (a changed beta scale refactorises kept blocks once)."""
    import torch
    if steps % per_launch:
        raise ValueError("steps must be a multiple of per_launch")
    res = {}
    for name in ("plain", "learned"):
        sim = sa.Simulation(problem, device=device, precision=precision)
        sim.step(warmup)
        sim.use_graph(True)
        for _ in range(1 + learned_warmup):     # the first call captures the graph
            if name == "learned":
                sim.step_learned(net, per_launch)
            else:
                sim.step(per_launch)
        sim.sync()
        sim.iteration_stats()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps // per_launch):
            if name == "plain":
                sim.step(per_launch)
            else:
                sim.step_learned(net, per_launch)
        e1.record()
        torch.cuda.synchronize()
        st = sim.iteration_stats()
        res[name] = {"iters_per_scene_step": st["total_iters"] / max(st["scene_steps"], 1),
                     "not_converged": st["not_converged"], "fallbacks": st["fallbacks"],
                     "ms_per_step": e0.elapsed_time(e1) / steps}
        sim.close()
    return res
