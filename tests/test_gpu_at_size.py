"""Parity at the full sizes of the batched and the learned-closure workloads,
on sampled nodes: the oracle assembles only the elements incident to the
sampled nodes (whose RHS is then complete).

* the 64-mesh batch (8.1M elements in meshes of 1e4-5e5), one persistent
  launch with the batch autotuner's plan, mixed precision, Vreman: every mesh
  at 100 sampled nodes, gated like the other mixed-path parity tests;
* the network fused into the 8M-element mixed channel (the stored network,
  without the training envelope so that every Gauss point takes the network
  as in the oracle): 2,000 sampled nodes, gated like the fused-closure
  parity tests (relative to the subgrid term's norm: the network runs on
  BF16 weights and FP16 activations).
"""
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_2005_05899_b300 import fea
from paper_2005_05899_b300 import meshgen as mg

from test_gpu_mlp import gpu_rounded_theta

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def sub_oracle(mesh, field, pick, closure="vreman", mlp=None, mask=fea.TERM_ALL):
    mark = np.zeros(mesh.n_nodes, bool)
    mark[pick] = True
    sub = {t: c[mark[c].any(axis=1)] for t, c in mesh.conn.items()}
    used = np.unique(np.concatenate([c.ravel() for c in sub.values()]))
    remap = np.full(mesh.n_nodes, -1, np.int64)
    remap[used] = np.arange(used.size)
    om = O.OracleMesh(mesh.xyz[used], {t: remap[c].astype(np.int32) for t, c in sub.items()})
    return O.assemble_rhs(om, field.u[used], field.p[used], field.nu, field.c_vreman, closure, mask,
                          mlp=mlp)[remap[pick]]


def test_full_batch_sampled_parity():
    ctx = fea.Context(0)
    try:
        batch = mg.batch_meshes(count=64, seed=7)
        dms, outs = [], []
        for m, f in batch:
            dm = ctx.upload_mesh(m)
            dm.upload_field(f.u, f.p, f.nu, f.c_vreman)
            dms.append(dm)
            outs.append(torch.empty((3, dm.n_nodes), dtype=torch.float64, device="cuda"))
        plan = ctx.autotune_batched(dms)
        ctx.assemble_batched(dms, outs, prec="mixed", closure="vreman")
        ctx.sync_status()
        rng = np.random.default_rng(3)
        worst = 0.0
        for (m, f), o in zip(batch, outs):
            pick = np.sort(rng.choice(m.n_nodes, size=100, replace=False))
            ref = sub_oracle(m, f, pick)
            got = o[:, torch.from_numpy(pick).cuda()].cpu().numpy().T
            l2 = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            mx = np.abs(got - ref).max() / np.abs(ref).max()
            worst = max(worst, l2)
            assert l2 < 2e-5 and mx < 2e-4, (m.n_elem_total, l2, mx)
        print(f"batch of 64 ({sum(m.n_elem_total for m, _ in batch):,} elements), plan {plan.as_dict()}: "
              f"worst sampled rel-L2 {worst:.2e}")
    finally:
        ctx.close()


def test_fused_closure_on_the_8m_channel_sampled_parity():
    w = np.load(os.path.join(ROOT, "paper_2005_05899_b300", "closure_tgv256.npz"))
    ctx = fea.Context(0)
    try:
        ctx.mlp_load(w["theta"], w["mean"], w["std"], float(w["scale"]))
        ctx.mlp_set_envelope(None, None)
        m = mg.channel_mesh(269, 134, 135)
        f = mg.channel_field(m, nu=1.0 / 5600.0)
        dm = ctx.upload_mesh(m)
        dm.upload_field(f.u, f.p, f.nu, f.c_vreman)
        dm.autotune(prec="mixed", closure="mlp")
        out = torch.empty((3, dm.n_nodes), dtype=torch.float64, device="cuda")
        dm.assemble(out, prec="mixed", closure="mlp")
        ctx.sync_status()
        mlp = O.MLPParams(gpu_rounded_theta(w["theta"]), w["mean"].astype(np.float64), w["std"].astype(np.float64),
                          float(w["scale"]))
        rng = np.random.default_rng(4)
        pick = np.sort(rng.choice(m.n_nodes, size=2000, replace=False))
        ref = sub_oracle(m, f, pick, "mlp", mlp)
        ref_sgs = sub_oracle(m, f, pick, "mlp", mlp, mask=fea.TERM_SGS)
        got = out[:, torch.from_numpy(pick).cuda()].cpu().numpy().T
        err = np.linalg.norm(got - ref)
        print(f"fused closure, 8M channel, 2000 nodes: |d| / |R| {err / np.linalg.norm(ref):.2e}, "
              f"|d| / |R_sgs| {err / np.linalg.norm(ref_sgs):.2e}")
        assert err <= 3e-2 * np.linalg.norm(ref_sgs) + 2e-5 * np.linalg.norm(ref)
    finally:
        ctx.close()
