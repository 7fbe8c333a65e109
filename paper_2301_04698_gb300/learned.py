"""Learned Poisson warm start: data, training and evaluation workflow.

The network and every kernel it runs are in libles.so (les_unet_*); this
module only sequences calls.  Pairs (b, psi) are produced by the solver itself:
each step of a seeded Taylor-Green run (32^3, FP64, K = 3, CG to 1e-10) is run
stage by stage and the right side and converged solution of every Poisson
solve are copied aside on the device.  Training minimises the mean squared
error of the network output against psi / rms(b) with Adam.  Evaluation runs
held-out seeds with zero, previous-step and learned first guesses, all to the
same relative residual, and reports CG iterations and solve time per step
(network inference included in the learned solve).
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import inputs, les


def generate_pairs(seeds, steps: int, n: int = 32, store=None, tol: float = 1e-10):
    """(b, psi) pairs from `steps` steps of each seeded run; FP32 tensors
    of shape (len(seeds) * steps * K, n, n, n) on the current device."""
    import torch
    store = store or torch.float32
    K = inputs.tgv(n).K
    total = len(seeds) * steps * K
    dev = torch.device("cuda", torch.cuda.current_device())
    B = torch.empty((total, n, n, n), dtype=store, device=dev)
    P = torch.empty((total, n, n, n), dtype=store, device=dev)
    i = 0
    for seed in seeds:
        case = inputs.tgv(n, seed=seed, steps_tol=tol)
        sim = les.Simulation(case)
        sim.set_state(inputs.initial_state(case))
        rhs, psi = sim.view("rhs"), None
        for _ in range(steps):
            sim.stage("begin")
            for _k in range(case.K):
                sim.stage("scalar")
                sim.stage("momentum")
                B[i].copy_(rhs - rhs.mean())
                sim.stage("solve")
                psi = sim.view("psi")
                P[i].copy_(psi)
                sim.stage("correct")
                i += 1
            sim.stage("end")
        sim.close()
    torch.cuda.synchronize()
    return B, P


def train(model, B, P, steps: int = 1500, batch: int = 16, lr: float = 2e-3, seed: int = 0,
          log_every: int = 100):
    """Adam on minibatches drawn from (B, P); cosine learning-rate decay."""
    import torch
    rng = np.random.default_rng(seed)
    n = B.shape[0]
    hist = []
    t0 = time.perf_counter()
    for s in range(steps):
        idx = torch.from_numpy(rng.choice(n, size=batch, replace=False)).to(B.device)
        lr_s = lr * 0.5 * (1.0 + math.cos(math.pi * s / steps))
        want = (s % log_every == 0) or s == steps - 1
        loss = model.train_step(B[idx].contiguous(), P[idx].contiguous(), lr_s, want_loss=want)
        if want:
            hist.append((s, loss))
    torch.cuda.synchronize()
    return hist, time.perf_counter() - t0


def relative_error(model, B, P, count: int = 64):
    """Mean relative L2 error of the network's psi_0 on `count` pairs."""
    errs = []
    for i in range(min(count, B.shape[0])):
        b = B[i].double().contiguous()
        p = P[i].double()
        q = model.forward(b)
        p = p - p.mean()
        errs.append(float((q - p).norm() / p.norm()))
    return float(np.mean(errs))


def evaluate(model, seeds, steps: int = 20, n: int = 32, tol: float = 1e-6, warmup: int = 2):
    """CG iterations and Poisson ms per step for zero / prev / learned first
    guesses on held-out seeds, every solve to the same relative residual."""
    import torch
    out = {}
    for mode in ("zero", "prev", "learned"):
        iters = 0
        ms = 0.0
        nsteps = 0
        for seed in seeds:
            case = inputs.tgv(n, seed=seed, steps_tol=tol, warm=mode)
            sim = les.Simulation(case)
            sim.set_state(inputs.initial_state(case))
            if mode == "learned":
                les.attach_model(sim, model)
            for s in range(warmup + steps):
                sim.stage("begin")
                for _k in range(case.K):
                    sim.stage("scalar")
                    sim.stage("momentum")
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    a.record(sim.stream)
                    st = sim.stage("solve")
                    b.record(sim.stream)
                    b.synchronize()
                    if s >= warmup:
                        iters += st["iters_total"]
                        ms += a.elapsed_time(b)
                    sim.stage("correct")
                sim.stage("end")
                if s >= warmup:
                    nsteps += 1
            sim.close()
        out[mode] = {"iters_per_step": iters / nsteps, "poisson_ms_per_step": ms / nsteps}
    out["speedup_vs_zero"] = out["zero"]["poisson_ms_per_step"] / out["learned"]["poisson_ms_per_step"]
    out["speedup_vs_prev"] = out["prev"]["poisson_ms_per_step"] / out["learned"]["poisson_ms_per_step"]
    out["tol"] = tol
    return out
