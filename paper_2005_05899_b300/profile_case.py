"""Run one assembly case for profiling (e.g. under ncu).

    python -m paper_2005_05899_b300.profile_case --mesh airplane --n 100 \
        --plan chunk --threads 256 --chunk 512 --reps 3
    python -m paper_2005_05899_b300.profile_case --mesh channel --cells 269,134,135

Builds the seeded mesh and field, uploads them, sets the launch plan and runs
`--reps` mixed-precision assemblies (or RK3 graph steps with --rk3) with the
Vreman closure, or with `--closure mlp` a seeded random network scaled to
Vreman's mean eddy viscosity, then checks the device status word.
"""
from __future__ import annotations

import argparse
import sys
import time


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--mesh", choices=["airplane", "channel", "tgv"], default="airplane")
    ap.add_argument("--n", type=int, default=100, help="grid nodes per axis (airplane) or cells (tgv)")
    ap.add_argument("--cells", default="128,64,64",
                    help="channel cells nx,ny,nz (e.g. 269,134,135 for the 8M-element channel, inputs above L2)")
    ap.add_argument("--plan", choices=["chunk", "atomic"], default="chunk")
    ap.add_argument("--threads", type=int, default=256)
    ap.add_argument("--chunk", type=int, default=512)
    ap.add_argument("--acc", type=int, default=0)
    ap.add_argument("--prec", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--rk3", action="store_true")
    ap.add_argument("--time", type=int, default=0, help="then time this many assemblies per category")
    ap.add_argument("--closure", choices=["vreman", "mlp"], default="vreman")
    ap.add_argument("--project-iters", type=int, default=0,
                    help="instead of assemblies: Laplacian set-up, then projections of this many CG iterations")
    a = ap.parse_args(argv)
    import torch

    from . import fea
    from . import meshgen as mg
    if a.mesh == "airplane":
        m = mg.airplane_mesh(a.n, seed=4)
        f = mg.inflow_field(m, seed=5)
    elif a.mesh == "channel":
        nx, ny, nz = (int(v) for v in a.cells.split(","))
        m = mg.channel_mesh(nx, ny, nz)
        f = mg.channel_field(m)
    else:
        m = mg.tgv_mesh(a.n)
        f = mg.tgv_field(m)
    ctx = fea.Context(0)
    dm = ctx.upload_mesh(m)
    dm.set_plan(a.plan, a.threads, a.chunk, a.acc)
    dm.upload_field(f.u, f.p, f.nu, f.c_vreman)
    out = torch.empty((3, dm.n_nodes), dtype=torch.float64, device="cuda")
    if a.closure == "mlp":
        import numpy as np
        nut = torch.empty(dm.n_gauss_total, dtype=torch.float32, device="cuda")
        dm.assemble(out, prec=a.prec, closure="vreman", nut_out=nut)
        rng = np.random.default_rng(11)
        theta = (0.2 * rng.standard_normal(fea.MLP_NPARAM)).astype(np.float32)
        mean = np.array([1.0, 1.0, 0.5, -0.5, 1.0, -3.0], np.float32)
        ctx.mlp_load(theta, mean, np.ones(6, np.float32), float(nut.double().mean()) + 1e-12)
    t = time.time()
    if a.project_iters:
        dm.poisson_setup()
        for _ in range(a.reps):
            dm.project(1e-4, rtol=1e-30, max_iter=a.project_iters)
        torch.cuda.synchronize()
        ctx.sync_status()
        print(f"ok projection {a.reps} x {a.project_iters} CG iterations {time.time() - t:.3f}s", flush=True)
        return 0
    for _ in range(a.reps):
        if a.rk3:
            dm.rk_step_graph(1e-4, prec=a.prec, closure=a.closure)
        else:
            dm.assemble(out, prec=a.prec, closure=a.closure)
    torch.cuda.synchronize()
    ctx.sync_status()
    print(f"ok {m.counts()} {a.reps} reps {time.time() - t:.3f}s", flush=True)
    if a.time:
        # each category's kernels alone on the stream, timed with CUDA events
        ctx.profile(True)
        ctx.profile_read(0, 0, reset=True)
        for _ in range(a.time):
            dm.assemble(out, prec=a.prec, closure=a.closure)
        torch.cuda.synchronize()
        ctx.sync_status()
        for et, name in enumerate(("TET04", "PYR05", "PEN06", "HEX08")):
            for fj in (0, 1):
                ms, n = ctx.profile_read(et, fj, reset=False)
                if n:
                    print(f"time {name}{' fp64J' if fj else ''}: {ms / n:.4f} ms per launch ({n} launches, "
                          f"{m.counts()[name] / (ms / n) / 1e3:.0f} Melem/s of that type)", flush=True)
        ctx.profile(False)
    return 0


if __name__ == "__main__":
    sys.exit(main())
