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
            precision: int = sa.SIM_MIXED, device: int = 0) -> dict:
    """The same start, stepped with the previous-step warm start and with the learned one:
    iterations per scene-step of each, fallbacks of the learned start, and the wall time
    of the device work (CUDA events)."""
    import torch
    res = {}
    for name in ("plain", "learned"):
        sim = sa.Simulation(problem, device=device, precision=precision)
        sim.step(warmup)
        sim.use_graph(True)
        if name == "learned":                   # first (direct) learned step and capture
            sim.step_learned(net, 1)
        else:
            sim.step(1)
        sim.sync()
        sim.iteration_stats()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        if name == "plain":
            for _ in range(steps):
                sim.step(1)
        else:
            sim.step_learned(net, steps)
        e1.record()
        torch.cuda.synchronize()
        st = sim.iteration_stats()
        res[name] = {"iters_per_scene_step": st["total_iters"] / max(st["scene_steps"], 1),
                     "not_converged": st["not_converged"], "fallbacks": st["fallbacks"],
                     "ms_per_step": e0.elapsed_time(e1) / steps}
        sim.close()
    return res
