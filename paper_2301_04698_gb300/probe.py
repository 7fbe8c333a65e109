"""One Poisson solve through the public API, for timing and profiling a CG
kernel on a chosen grid (Sec. 2.4: L_c psi = b, CG to a relative residual).

    python -m paper_2301_04698_gb300.probe --grid 512x512x64 --variant 4 \\
        --iters 20 --repeat 2

The right side is a seeded uniform field on a grid with walls in z, FP32
unless --fp64; --resident 0 lets the on-chip CG run when the grid fits
there, --resident 1 forces a streaming kernel (--variant as in
les_tuning.cg_variant).  Prints one JSON line per solve: iterations, the
relative residual reached and the CUDA-event time.
"""
from __future__ import annotations

import argparse
import json

from . import inputs, les


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--grid", default="512x512x64", help="NXxNYxNZ")
    ap.add_argument("--variant", type=int, default=0, help="les_tuning.cg_variant")
    ap.add_argument("--resident", type=int, default=1, help="les_tuning.cg_resident (0: on chip when it fits)")
    ap.add_argument("--iters", type=int, default=20, help="CG iterations (the tolerance is unreachable)")
    ap.add_argument("--tol", type=float, default=1e-30)
    ap.add_argument("--repeat", type=int, default=2)
    ap.add_argument("--fp64", action="store_true")
    args = ap.parse_args(argv)
    import torch

    nx, ny, nz = (int(v) for v in args.grid.lower().split("x"))
    prec = 64 if args.fp64 else 32
    case = inputs.Case(name="probe", nx=nx, ny=ny, nz=nz, dx=35.0, dy=35.0, dz=10.0, walls=True,
                       precision=prec, init="zero", physics=())
    les.load_library()
    torch.cuda.set_device(0)
    sim = les.Simulation(case)
    sim.set_tuning(cg_variant=args.variant, cg_resident=args.resident)
    dt = torch.float64 if prec == 64 else torch.float32
    b = torch.from_numpy(inputs.uniform(1, 0, case.n, -1, 1).reshape(case.shape)).to("cuda", dt)
    for _ in range(args.repeat):
        x = torch.zeros_like(b)
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        rc, it, rel = sim.poisson_solve(b, x, args.tol, args.iters, allow_not_converged=True)
        t1.record()
        t1.synchronize()
        print(json.dumps({"grid": [nx, ny, nz], "precision": prec, "variant": args.variant, "iters": it,
                          "rel": rel, "ms": t0.elapsed_time(t1)}), flush=True)
    sim.close()


if __name__ == "__main__":
    main()
