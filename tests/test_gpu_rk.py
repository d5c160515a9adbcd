"""GPU RK3 stages and the graph-replayed step against the oracle."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2005_05899_b300 import fea
from paper_2005_05899_b300 import meshgen as mg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = fea.Context(0)
    yield c
    c.close()


def state(dm):
    out = torch.empty((3, dm.n_nodes), dtype=torch.float64, device="cuda")
    dm.state(out)
    torch.cuda.synchronize()
    return out.cpu().numpy().T.copy()


def oracle_step(m, f, dt, steps=1):
    om = O.OracleMesh.of(m)
    u = f.u
    for _ in range(steps):
        u = O.rk3_step(om, m.periodic_master, m.dirichlet, u, f.p, f.nu, f.c_vreman, "vreman", dt)
    return u


def test_rk_stages_fp64_tgv(ctx):
    m = mg.tgv_mesh(16)
    f = mg.tgv_field(m)
    dm = ctx.upload_mesh(m)
    dm.upload_field(f.u, f.p, f.nu, f.c_vreman)
    dt = 0.05
    for k in range(3):
        dm.rk_stage(k, dt, prec="fp64")
    ctx.sync_status()
    ref = oracle_step(m, f, dt)
    got = state(dm)
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def test_graph_step_matches_stages_and_oracle(ctx):
    m = mg.channel_mesh(nx=10, ny=12, nz=8, seed=4, n_layers=2, split_frac=0.3)
    f = mg.channel_field(m, seed=2, nu=1e-2)
    dm = ctx.upload_mesh(m)
    dt = 2e-3
    dm.upload_field(f.u, f.p, f.nu, f.c_vreman)
    for s in range(2):
        dm.rk_step_graph(dt, prec="fp64")
    ctx.sync_status()
    g = state(dm)
    ref = oracle_step(m, f, dt, steps=2)
    assert np.abs(g - ref).max() < 1e-12 * np.abs(ref).max()
    d = m.dirichlet.astype(bool)
    assert np.array_equal(g[d], f.u[d])
    # mixed precision graph
    dm.upload_field(f.u, f.p, f.nu, f.c_vreman)
    dm.rk_step_graph(dt, prec="mixed")
    ctx.sync_status()
    gm = state(dm)
    ref1 = oracle_step(m, f, dt, steps=1)
    upd = np.abs(ref1 - f.u).max()
    assert np.abs(gm - ref1).max() < 2e-4 * upd


def test_stage_update_refreshes_the_fp32_field_exactly(ctx):
    """The stage update rewrites the FP32 copy of the field with its own
    round-to-nearest FP64 -> FP32 conversion.  A first stage with dt = 1e-300
    leaves the FP64 state unchanged bit for bit (and zeros stay zero), so the
    mixed assembly that follows must reproduce the one made right after the
    field upload, whose FP32 copy the hardware conversion wrote; one ulp of
    FP32 in u would move the RHS by ~1e-8."""
    m = mg.channel_mesh(nx=10, ny=12, nz=8, seed=21, n_layers=2, split_frac=0.3)
    f = mg.channel_field(m, seed=5, nu=1e-3)
    rng = np.random.default_rng(4)
    # values over six decades (the conversion's exponent handling), walls at 0
    u = f.u * (1.0 + rng.standard_normal(f.u.shape)) * 10.0 ** rng.uniform(-3.0, 3.0, (f.u.shape[0], 1))
    dm = ctx.upload_mesh(m)
    dm.set_plan("atomic", 128, 256, 0)
    dm.upload_field(u, f.p, f.nu, f.c_vreman)
    r0 = torch.empty((3, dm.n_nodes), dtype=torch.float64, device="cuda")
    dm.assemble(r0, prec="mixed")
    before = state(dm)
    dm.rk_stage(0, 1e-300, prec="mixed")
    after = state(dm)
    assert np.array_equal(before, after)
    r1 = torch.empty_like(r0)
    dm.assemble(r1, prec="mixed")
    ctx.sync_status()
    a, b = r0.cpu().numpy(), r1.cpu().numpy()
    assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()


def test_tail_order_mesh_graph_and_stages(ctx):
    """A mesh of one TET04 and one FP64-Jacobian PEN06 category (the
    airplane-like generator at 30^3): the PEN06 kernel runs as a
    programmatic dependent of the TET04 kernel.  Graph step and stage
    launches agree with each other and with the oracle within the mixed
    gates, and the assembly matches the oracle."""
    m = mg.airplane_mesh(30, seed=4)
    f = mg.inflow_field(m, seed=5)
    assert set(m.conn) == {mg.TET04, mg.PEN06}
    dt = 1e-3
    dm = ctx.upload_mesh(m)
    dm.set_plan("chunk", 128, 256, 0)
    dm.upload_field(f.u, f.p, f.nu, f.c_vreman)
    out = torch.empty((3, dm.n_nodes), dtype=torch.float64, device="cuda")
    dm.assemble(out)
    ctx.sync_status()
    ref_rhs = O.assemble_rhs(O.OracleMesh.of(m), f.u, f.p, f.nu, f.c_vreman, "vreman")
    got = out.cpu().numpy().T
    assert np.linalg.norm(got - ref_rhs) <= 2e-5 * np.linalg.norm(ref_rhs)
    for _ in range(2):
        dm.rk_step_graph(dt)
    ctx.sync_status()
    g = state(dm)
    dm.upload_field(f.u, f.p, f.nu, f.c_vreman)
    for _ in range(2):
        for k in range(3):
            dm.rk_stage(k, dt)
    ctx.sync_status()
    st = state(dm)
    ref = oracle_step(m, f, dt, steps=2)
    upd = np.abs(ref - f.u).max()
    assert np.abs(g - st).max() <= 1e-6 * upd
    assert np.abs(g - ref).max() < 2e-4 * upd
    # the allocation-free stage takes the same order
    un = torch.tensor(np.ascontiguousarray(f.u.T), dtype=torch.float64, device="cuda")
    p = torch.tensor(f.p, dtype=torch.float64, device="cuda")
    o1 = torch.empty_like(un)
    dm.rk_stage_noalloc(0, dt, un, un, p, o1, f.nu, f.c_vreman)
    dm.upload_field(f.u, f.p, f.nu, f.c_vreman)
    dm.rk_stage(0, dt)
    ctx.sync_status()
    s0 = state(dm)
    assert np.abs(o1.cpu().numpy().T - s0).max() <= 1e-6 * upd
