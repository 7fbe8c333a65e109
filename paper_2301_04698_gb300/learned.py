"""Learned Poisson warm start: data, training and evaluation workflow.

The network and every kernel it runs are in libles.so (les_unet_*); this
module only sequences calls.  Pairs (b, psi) are produced by the solver itself:
each step of a seeded Taylor-Green run (32^3, FP64, K = 3, CG to 1e-10) is run
stage by stage and the right side and converged solution of every Poisson
solve are copied aside on the device.  Training minimises the mean squared
error of the network output against psi / rms(b) with Adam, or the energy
norm of that error (the loss a CG solve from the guess pays for).  Evaluation runs
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


def train(model, B, P, steps: int = 1500, batch: int = 16, lr: float = 5e-4, seed: int = 0,
          log_every: int = 100, warmup: int = 100):
    """Adam on minibatches drawn from (B, P); linear warm-up, cosine decay."""
    import torch
    rng = np.random.default_rng(seed)
    n = B.shape[0]
    hist = []
    t0 = time.perf_counter()
    for s in range(steps):
        idx = torch.from_numpy(rng.choice(n, size=batch, replace=False)).to(B.device)
        lr_s = lr * min(1.0, (s + 1) / warmup) * 0.5 * (1.0 + math.cos(math.pi * s / steps))
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
        nc = 0
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
                    st = sim.stage("solve", allow_not_converged=True)
                    b.record(sim.stream)
                    b.synchronize()
                    if s >= warmup:
                        iters += st["iters_total"]
                        nc += st["not_converged"]
                        ms += a.elapsed_time(b)
                    sim.stage("correct")
                sim.stage("end")
                if s >= warmup:
                    nsteps += 1
            sim.close()
        out[mode] = {"iters_per_step": iters / nsteps, "poisson_ms_per_step": ms / nsteps,
                     "not_converged": nc}
    out["speedup_vs_zero"] = out["zero"]["poisson_ms_per_step"] / out["learned"]["poisson_ms_per_step"]
    out["speedup_vs_prev"] = out["prev"]["poisson_ms_per_step"] / out["learned"]["poisson_ms_per_step"]
    out["tol"] = tol
    return out


def init_weights(seed: int = 0) -> np.ndarray:
    """He-style uniform initial weights in the flat les_unet layout."""
    rng = np.random.default_rng(seed)
    layers = ((1, 16, 3), (16, 16, 3), (16, 32, 3), (32, 32, 3), (32, 64, 3), (64, 64, 3),
              (96, 32, 3), (32, 32, 3), (48, 16, 3), (16, 16, 3), (16, 1, 1))
    parts = []
    for li, (ci, co, k) in enumerate(layers):
        lim = np.sqrt(6.0 / (ci * k ** 3)) / np.sqrt(1.01)
        w = rng.uniform(-lim, lim, size=co * ci * k ** 3)
        if li == len(layers) - 1:
            w[:] = 0.0  # the untrained network predicts psi_0 = 0, the plain first guess
        parts.append(w)
        parts.append(np.zeros(co))
    return np.concatenate(parts).astype(np.float32)


def output_scale(B, P) -> float:
    """Typical rms(psi) / rms(b) over the data (the network's unit scale)."""
    rb = B.double().flatten(1).pow(2).mean(1).sqrt()
    rp = P.double().flatten(1).pow(2).mean(1).sqrt()
    ok = rb > 0
    return float((rp[ok] / rb[ok]).pow(2).mean().sqrt())


def main(argv=None):
    """Generate pairs, train, and compare first guesses; prints one JSON line."""
    import argparse
    import json

    import torch

    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=32)
    ap.add_argument("--train-seeds", type=int, default=67)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--train-steps", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=5e-4)
    ap.add_argument("--eval-seeds", type=int, default=4)
    ap.add_argument("--eval-steps", type=int, default=20)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--save", default="")
    ap.add_argument("--loss", default="energy", choices=("mse", "energy"))
    a = ap.parse_args(argv)
    les.load_library()
    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    seeds = list(range(100, 100 + a.train_seeds))
    B, P = generate_pairs(seeds, a.steps, n=a.n)
    t_gen = time.perf_counter() - t0
    nval = max(16, B.shape[0] // 50)
    model = les.UNet(a.n, max_batch=a.batch)
    model.set_weights(init_weights(0))
    model.set_loss(a.loss)
    model.out_scale = output_scale(B[nval:], P[nval:])
    hist, t_train = train(model, B[nval:], P[nval:], steps=a.train_steps, batch=a.batch, lr=a.lr)
    err_val = relative_error(model, B[:nval], P[:nval])
    ev = evaluate(model, list(range(1, 1 + a.eval_seeds)), steps=a.eval_steps, n=a.n, tol=a.tol)
    if a.save:
        np.save(a.save, model.get_weights())
    out = {"pairs": int(B.shape[0]), "loss": a.loss, "out_scale": model.out_scale, "gen_s": t_gen, "train_steps": a.train_steps, "train_s": t_train,
           "loss_first": hist[0][1], "loss_last": hist[-1][1], "loss_curve": hist, "val_rel_err": err_val,
           "eval": ev}
    print(json.dumps(out), flush=True)
    return out


if __name__ == "__main__":
    main()
