"""Secondary measurements: the channel mesh (mixed types), the batch of
64 uneven meshes (one persistent launch vs one launch sequence per mesh) and
the learned closure (trained on filtered fine Taylor-Green runs, then fused
into the assembly of an 8M-element mixed channel mesh against Vreman).

    python -m paper_2005_05899_b300.bench_configs [--channel] [--batch] [--closure] [--projection] [--balance]
        [--reps 20]

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
    # the batch autotuner's choice (persistent launch with its chunk size, or per-mesh scatter)
    best = ctx.autotune_batched(dms)
    for _ in range(3):
        ctx.assemble_batched(dms, outs)
    torch.cuda.synchronize()
    l0 = ctx.launch_count
    e0.record()
    for _ in range(reps):
        ctx.assemble_batched(dms, outs)
    e1.record()
    torch.cuda.synchronize()
    ctx.sync_status()
    ms = e0.elapsed_time(e1) / reps
    res["autotuned"] = {"plan": best.as_dict(), "ms": ms, "melem_s": E / ms / 1e3,
                        "launches_per_call": (ctx.launch_count - l0) / reps}
    print(json.dumps({"workload": f"batch of {count} channel-like meshes, log-uniform 1e4-5e5 elements",
                      "elements": E, "generate_s": gen_s, **res}), flush=True)


def _time_assemble(dm, out, reps: int, **kw) -> float:
    import torch
    for _ in range(3):
        dm.assemble(out, **kw)
    e0, e1 = _events()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        dm.assemble(out, **kw)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def closure(reps: int, n_f: int = 256, steps: int = 8000, dims=(269, 134, 135), save: str = ""):
    """Learned closure: GPU training on box-filtered n_f^3 Taylor-Green runs,
    a-priori errors on a held-out time, then the network fused at every Gauss
    point of a mixed channel mesh against the Vreman path: time per assembly,
    and relative L2 differences of nu_t and of the RHS (whole and subgrid part
    alone), plus the mixed-precision error of the learned path against its own
    FP64 assembly."""
    import numpy as np
    import torch
    from . import closure_data as cd
    from . import fea
    from . import meshgen as mg
    ctx = fea.Context(0)
    t = time.time()
    res = cd.run(n_f=n_f, ratios=(2, 4, 8), t_train=(3.0, 4.0, 5.0, 7.0, 8.0), t_test=(6.0,), steps=steps,
                 log=None, ctx=ctx, save=save)
    model = res.pop("model")
    train_total_s = time.time() - t
    m = mg.channel_mesh(*dims)
    f = mg.channel_field(m, nu=1.0 / 5600.0)
    dm = ctx.upload_mesh(m)
    dm.upload_field(f.u, f.p, f.nu, f.c_vreman)
    E = m.n_elem_total
    N, NG = dm.n_nodes, dm.n_gauss_total
    kinds = ("vreman", "mlp", "mlp_raw")   # mlp: with the training envelope; mlp_raw: without

    def closure_of(k):
        return "vreman" if k == "vreman" else "mlp"

    def envelope_for(k):
        if k == "mlp_raw":
            ctx.mlp_set_envelope(None, None)
        elif k == "mlp":
            ctx.mlp_set_envelope(model.env_lo, model.env_hi)

    rhs = {k: torch.empty((3, N), dtype=torch.float64, device="cuda") for k in kinds}
    sgs = {k: torch.empty((3, N), dtype=torch.float64, device="cuda") for k in kinds}
    nut = {k: torch.empty(NG, dtype=torch.float32, device="cuda") for k in kinds}
    plans, ms, fallback = {}, {}, {}
    for k in kinds:
        envelope_for(k)
        plans[k] = dm.autotune(prec="mixed", closure=closure_of(k)).as_dict()
        ms[k] = _time_assemble(dm, rhs[k], reps, prec="mixed", closure=closure_of(k))
        ctx.sync_status()
        if k != "vreman":
            ctx.mlp_fallback_read(reset=True)
        dm.assemble(rhs[k], prec="mixed", closure=closure_of(k), nut_out=nut[k])
        ctx.sync_status()
        if k != "vreman":
            fallback[k] = ctx.mlp_fallback_read(reset=True) / NG
        dm.assemble(sgs[k], prec="mixed", closure=closure_of(k), mask=fea.TERM_SGS)
    envelope_for("mlp")
    ref64 = torch.empty((3, N), dtype=torch.float64, device="cuda")
    dm.assemble(ref64, prec="fp64", closure="mlp", scatter="atomic")
    ctx.sync_status()

    def rel(a, b):
        return float(torch.linalg.norm((a - b).double()) / torch.linalg.norm(b.double()))

    nv = nut["vreman"]
    out = {"workload": f"learned closure: trained on box-filtered {n_f}^3 Taylor-Green runs, fused into "
                       f"channel {dims[0]}x{dims[1]}x{dims[2]} mixed ({E:,} elements)",
           "counts": m.counts(), "elements": E, "gauss_points": int(NG),
           "training": res, "train_total_s": train_total_s,
           "assemble_ms": ms, "melem_s": {k: E / v / 1e3 for k, v in ms.items()},
           "mlp_over_vreman_time": ms["mlp"] / ms["vreman"], "plans": plans,
           "fallback_frac": fallback,
           "nut_mean": {k: float(nut[k].double().mean()) for k in kinds},
           "nut_rel_l2_vs_vreman": {k: rel(nut[k], nv) for k in kinds if k != "vreman"},
           "rhs_rel_l2_vs_vreman": {k: rel(rhs[k], rhs["vreman"]) for k in kinds if k != "vreman"},
           "sgs_rel_l2_vs_vreman": {k: rel(sgs[k], sgs["vreman"]) for k in kinds if k != "vreman"},
           "mlp_mixed_vs_fp64_rel_l2": rel(rhs["mlp"], ref64)}
    print(json.dumps(out), flush=True)
    ctx.close()


def projection(n_axis: int = 170, dt: float = 2e-4, rtol: float = 1e-6, steps: int = 3):
    """Pressure projection on the airplane-like mesh: Laplacian set-up
    (host pattern + device values), then `steps` fractional steps (RK3 graph
    step + projection) with CG iteration counts and times; SpMV traffic per
    iteration = 12 B per stored entry + 8 B x 10 class vectors touched."""
    import torch
    from . import fea
    from . import meshgen as mg
    m = mg.airplane_mesh(n_axis, seed=4)
    f = mg.inflow_field(m, seed=5)
    ctx = fea.Context(0)
    dm = ctx.upload_mesh(m)
    dm.upload_field(f.u, f.p, f.nu, f.c_vreman)
    t = time.time()
    dm.poisson_setup()
    setup_s = time.time() - t
    res = []
    for k in range(steps):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record()
        dm.rk_step_graph(dt)
        e1.record()
        it, rr = dm.project(dt, rtol=rtol, max_iter=20000)
        e2.record()
        torch.cuda.synchronize()
        res.append({"rk3_ms": e0.elapsed_time(e1), "project_ms": e1.elapsed_time(e2), "cg_iters": it,
                    "rel_res": rr, "ms_per_cg_iter": e1.elapsed_time(e2) / max(it, 1)})
    ctx.sync_status()
    E = m.n_elem_total
    print(json.dumps({"workload": f"projection on the airplane-like mesh ({E:,} elements, {m.n_nodes:,} nodes)",
                      "setup_s": setup_s, "dt": dt, "rtol": rtol, "steps": res}), flush=True)


def wall(reps: int, n_axis: int = 170, dims=(269, 134, 135)):
    """Boundary assembly (wall model, FP64) timed with CUDA events: on the
    airplane-like mesh's wall (the innermost prism-layer triangles) against
    its RK stage with and without the term, and on the walls of a large
    channel (prism-layer triangles on both walls)."""
    import torch
    from . import fea
    from . import meshgen as mg
    ctx = fea.Context(0)
    out = {}
    m = mg.airplane_mesh(n_axis, seed=4)
    f = mg.inflow_field(m, seed=5)
    dm = ctx.upload_mesh(m)
    dm.upload_field(f.u, f.p, f.nu, f.c_vreman)
    rhs = torch.zeros((3, m.n_nodes), dtype=torch.float64, device="cuda")

    def timed(fn):
        for _ in range(3):
            fn()
        e0, e1 = _events()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    stage_plain = timed(lambda: dm.rk_stage(0, 1e-6))
    dm.wall_setup(**m.wall_faces)
    wall_ms = timed(lambda: dm.wall_assemble(rhs))
    stage_wall = timed(lambda: dm.rk_stage(0, 1e-6))
    ctx.sync_status()
    nf = int(m.wall_faces["tri"].shape[0])
    stage_wall64 = timed(lambda: dm.rk_stage(0, 1e-6, prec="fp64"))
    dm.wall_setup()
    stage_plain64 = timed(lambda: dm.rk_stage(0, 1e-6, prec="fp64"))
    ctx.sync_status()
    out["airplane"] = {"faces": nf, "elements": m.n_elem_total, "wall_fp64_ms": wall_ms,
                       "faces_per_s_fp64": nf / (wall_ms * 1e-3),
                       "mixed": {"rk_stage_ms": stage_plain, "rk_stage_with_wall_ms": stage_wall,
                                 "boundary_share": (stage_wall - stage_plain) / stage_wall},
                       "fp64": {"rk_stage_ms": stage_plain64, "rk_stage_with_wall_ms": stage_wall64,
                                "boundary_share": (stage_wall64 - stage_plain64) / stage_wall64}}
    del dm
    c = mg.channel_mesh(*dims, seed=2)
    cf = mg.channel_field(c, seed=3)
    dc = ctx.upload_mesh(c)
    dc.upload_field(cf.u, cf.p, cf.nu, cf.c_vreman)
    dc.wall_setup(**c.wall_faces)
    rc = torch.zeros((3, c.n_nodes), dtype=torch.float64, device="cuda")
    ms = timed(lambda: dc.wall_assemble(rc))
    ctx.sync_status()
    nf = int(c.wall_faces["tri"].shape[0])
    out["channel"] = {"faces": nf, "wall_fp64_ms": ms, "faces_per_s_fp64": nf / (ms * 1e-3)}
    print(json.dumps({"workload": "wall-model boundary assembly (Reichardt law, Newton for u_tau; "
                                  "FP32 root in the mixed stage, FP64 otherwise)",
                      **out}), flush=True)


def part_times(ctx, mesh, field, parts, reps: int):
    """Assembly time of every part (mixed precision, Vreman, autotuned plan
    of the first call), parts uploaded as meshes of their own, timed one
    after the other with CUDA events."""
    import torch
    times = []
    for part in parts:
        dm = ctx.upload_mesh(part.mesh)
        dm.upload_field(field.u[part.nodes], field.p[part.nodes], field.nu, field.c_vreman)
        out = torch.empty((3, dm.n_nodes), dtype=torch.float64, device="cuda")
        times.append(_time_assemble(dm, out, reps))
        del dm
    return times


def balance(reps: int, n_parts: int = 4, iters: int = 8, n_axis: int = 140):
    """The correction coefficients on measured times: the airplane-like mesh
    (tets everywhere, FP64-Jacobian prisms around the body) split into
    n_parts by the Gauss-point cost model, each part's assembly timed on the
    GPU, the partition corrected from the times, repeated."""
    from . import fea
    from . import meshgen as mg
    from . import partition as P
    m = mg.airplane_mesh(n_axis, seed=4)
    f = mg.inflow_field(m, seed=5)
    ctx = fea.Context(0)
    bal = P.Balancer(n_parts)
    hist = []
    for k in range(iters):
        parts = P.build_parts(m, n_parts, lam=bal.lam)
        t = part_times(ctx, m, f, parts, reps)
        hist.append({"iteration": k, "lambda": [round(x, 4) for x in bal.lam], "part_ms": [round(x, 4) for x in t],
                     "imbalance": round(P.Balancer.imbalance(t), 4),
                     "elements": [int(sum(v.size for v in p.elems.values())) for p in parts]})
        bal.update(t)
    ctx.sync_status()
    print(json.dumps({"workload": f"airplane-like {n_axis}^3 ({m.n_elem_total:,} elements: {m.counts()}) in "
                                  f"{n_parts} parts, Gauss-point weights corrected from measured part times",
                      "iterations": hist}), flush=True)


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--channel", action="store_true")
    ap.add_argument("--batch", action="store_true")
    ap.add_argument("--closure", action="store_true")
    ap.add_argument("--projection", action="store_true")
    ap.add_argument("--balance", action="store_true")
    ap.add_argument("--wall", action="store_true")
    ap.add_argument("--n-f", type=int, default=256, help="fine Taylor-Green grid of the closure's training runs")
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--save", default="", help="with --closure: write the trained network (npz) here")
    a = ap.parse_args(argv)
    if not (a.channel or a.batch or a.closure or a.projection or a.balance or a.wall):
        a.channel = a.batch = True
    if a.channel:
        channel(a.reps)
    if a.batch:
        batch(a.reps)
    if a.closure:
        closure(a.reps, n_f=a.n_f, save=a.save)
    if a.projection:
        projection()
    if a.balance:
        balance(a.reps)
    if a.wall:
        wall(a.reps)
    return 0


if __name__ == "__main__":
    sys.exit(main())
