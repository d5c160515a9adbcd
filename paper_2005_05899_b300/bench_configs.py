"""Secondary measurements: the channel mesh (mixed types) and the batch of
64 uneven meshes (one persistent launch vs one launch sequence per mesh).

    python -m paper_2005_05899_b300.bench_configs [--channel] [--batch] [--reps 20]

Prints one JSON line per measurement (CUDA-event times on the current stream,
after warm-up; inputs are larger than L2 for the channel and the batch).
"""
from __future__ import annotations

import argparse
import json
import sys
import time


def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def channel(reps: int):
    import torch
    from . import fea
    from . import meshgen as mg
    m = mg.channel_mesh()
    f = mg.channel_field(m)
    ctx = fea.Context(0)
    dm = ctx.upload_mesh(m)
    dm.upload_field(f.u, f.p, f.nu, f.c_vreman)
    plan = dm.autotune(prec="mixed", closure="vreman").as_dict()
    out = torch.empty((3, dm.n_nodes), dtype=torch.float64, device="cuda")
    for _ in range(3):
        dm.assemble(out)
    e0, e1 = _events()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        dm.assemble(out)
    e1.record()
    torch.cuda.synchronize()
    ctx.sync_status()
    ms = e0.elapsed_time(e1) / reps
    E = m.n_elem_total
    print(json.dumps({"workload": "channel 128x64x64 mixed (942,079 elements)", "counts": m.counts(),
                      "assemble_ms": ms, "melem_s": E / ms / 1e3, "plan": plan}), flush=True)


def batch(reps: int, count: int = 64):
    import torch
    from . import fea
    from . import meshgen as mg
    t = time.time()
    meshes = mg.batch_meshes(count=count, seed=7)
    gen_s = time.time() - t
    ctx = fea.Context(0)
    dms, outs = [], []
    E = 0
    for m, f in meshes:
        dm = ctx.upload_mesh(m)
        dm.upload_field(f.u, f.p, f.nu, f.c_vreman)
        dms.append(dm)
        outs.append(torch.empty((3, dm.n_nodes), dtype=torch.float64, device="cuda"))
        E += m.n_elem_total
    e0, e1 = _events()
    res = {}
    for mode in ("batched", "per_mesh"):
        def once():
            if mode == "batched":
                ctx.assemble_batched(dms, outs)
            else:
                for dm, o in zip(dms, outs):
                    dm.assemble(o)
        for _ in range(3):
            once()
        torch.cuda.synchronize()
        l0 = ctx.launch_count
        e0.record()
        for _ in range(reps):
            once()
        e1.record()
        torch.cuda.synchronize()
        ctx.sync_status()
        ms = e0.elapsed_time(e1) / reps
        res[mode] = {"ms": ms, "melem_s": E / ms / 1e3, "launches_per_call": (ctx.launch_count - l0) / reps}
    print(json.dumps({"workload": f"batch of {count} channel-like meshes, log-uniform 1e4-5e5 elements",
                      "elements": E, "generate_s": gen_s, **res}), flush=True)


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--channel", action="store_true")
    ap.add_argument("--batch", action="store_true")
    ap.add_argument("--reps", type=int, default=20)
    a = ap.parse_args(argv)
    if not (a.channel or a.batch):
        a.channel = a.batch = True
    if a.channel:
        channel(a.reps)
    if a.batch:
        batch(a.reps)
    return 0


if __name__ == "__main__":
    sys.exit(main())
