"""Edge cases of the GPU path: meshes without elements and with nodes no
element uses, non-finite input (reported, not faulting, and cleared), a
zero right-hand side and a zero iteration budget in the pressure solve, an
empty MLP batch, an RK stage on a mesh without elements, and chunk plans at
the limits of the validation."""
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


def rhs_of(ctx, dm, prec="mixed", **kw):
    out = torch.full((3, dm.n_nodes), 7.0, dtype=torch.float64, device="cuda")
    dm.assemble(out, prec=prec, **kw)
    ctx.sync_status()
    return out.cpu().numpy().T


def test_mesh_without_elements(ctx):
    m = mg.Mesh(xyz=np.random.default_rng(0).random((5, 3)), conn={})
    dm = ctx.upload_mesh(m)
    dm.upload_field(np.ones((5, 3)), np.ones(5), 0.1)
    assert np.array_equal(rhs_of(ctx, dm), np.zeros((5, 3)))
    ml = torch.full((5,), 3.0, dtype=torch.float64, device="cuda")
    dm.lumped_mass(ml)
    assert np.array_equal(ml.cpu().numpy(), np.zeros(5))
    dm.rk_stage(0, 0.1)
    out = torch.empty((3, 5), dtype=torch.float64, device="cuda")
    dm.state(out)
    ctx.sync_status()
    assert np.array_equal(out.cpu().numpy(), np.ones((3, 5)))


@pytest.mark.parametrize("prec,scatter", [("fp64", "atomic"), ("mixed", "chunk"), ("mixed", "atomic")])
def test_nodes_no_element_uses_get_zero(ctx, prec, scatter):
    m0 = mg.channel_mesh(nx=6, ny=8, nz=4, seed=3, n_layers=2, split_frac=0.3)
    extra = 7
    xyz = np.concatenate([m0.xyz, np.random.default_rng(1).random((extra, 3))])
    m = mg.Mesh(xyz=xyz, conn=m0.conn)
    f = mg.random_field(m, seed=2)
    dm = ctx.upload_mesh(m)
    dm.upload_field(f.u, f.p, f.nu, f.c_vreman)
    r = rhs_of(ctx, dm, prec=prec, scatter=scatter)
    assert np.array_equal(r[-extra:], np.zeros((extra, 3)))
    ref = O.assemble_rhs(O.OracleMesh.of(m), f.u, f.p, f.nu, f.c_vreman, "vreman")
    tol = 1e-12 if prec == "fp64" else 2e-5
    assert np.linalg.norm(r - ref) <= tol * np.linalg.norm(ref)


@pytest.mark.parametrize("plan", [("chunk", 256, 256, 0), ("atomic", 128, 256, 0)])
def test_non_finite_input_is_reported_then_cleared(ctx, plan):
    m = mg.channel_mesh(nx=6, ny=8, nz=4, seed=3, n_layers=2, split_frac=0.3)
    f = mg.random_field(m, seed=3)
    dm = ctx.upload_mesh(m)
    dm.set_plan(*plan)
    u = f.u.copy()
    u[m.conn[fea.HEX08][0, 0], 1] = np.nan
    dm.upload_field(u, f.p, f.nu, f.c_vreman)
    out = torch.empty((3, dm.n_nodes), dtype=torch.float64, device="cuda")
    dm.assemble(out)
    with pytest.raises(fea.FeaError) as ei:
        ctx.sync_status()
    assert ei.value.status == fea.ENUMERIC
    ctx.sync_status()   # the word was cleared by the read
    dm.upload_field(f.u, f.p, f.nu, f.c_vreman)
    r = rhs_of(ctx, dm)
    assert np.all(np.isfinite(r))


def test_pressure_solve_zero_rhs_and_zero_budget(ctx):
    m = mg.tgv_mesh(6)
    dm = ctx.upload_mesh(m)
    dm.poisson_setup()
    b = torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda")
    x = torch.ones(m.n_nodes, dtype=torch.float64, device="cuda")
    it, rr = dm.poisson_solve(b, x, rtol=1e-10, max_iter=100)
    assert it == 0 and rr == 0.0
    assert np.array_equal(x.cpu().numpy(), np.zeros(m.n_nodes))   # b = 0: x = 0 exactly
    b = torch.tensor(np.random.default_rng(5).standard_normal(m.n_nodes), device="cuda")
    x = torch.zeros_like(b)
    it, rr = dm.poisson_solve(b, x, rtol=1e-10, max_iter=0)
    assert it == 0 and rr > 0.0
    ctx.sync_status()


def test_empty_mlp_batch(ctx):
    rng = np.random.default_rng(0)
    ctx.mlp_load((0.1 * rng.standard_normal(fea.MLP_NPARAM)).astype(np.float32), np.zeros(6, np.float32),
                 np.ones(6, np.float32), 1e-3)
    x = torch.empty((0, 6), dtype=torch.float32, device="cuda")
    y = torch.empty(0, dtype=torch.float32, device="cuda")
    ctx.mlp_forward(x, y)
    ctx.sync_status()


def test_chunk_plans_at_the_validation_limits(ctx):
    m = mg.channel_mesh(nx=10, ny=8, nz=6, seed=3, n_layers=2, split_frac=0.3)
    f = mg.random_field(m, seed=6)
    dm = ctx.upload_mesh(m)
    dm.upload_field(f.u, f.p, f.nu, f.c_vreman)
    ref = O.assemble_rhs(O.OracleMesh.of(m), f.u, f.p, f.nu, f.c_vreman, "vreman")
    for plan in (("chunk", 32, 32, 0), ("chunk", 1024, 32, 0), ("chunk", 64, 4096, 1)):
        try:
            dm.set_plan(*plan)
        except fea.FeaError as e:
            assert e.status == fea.EINVAL      # a chunk whose shared memory does not fit is refused
            continue
        r = rhs_of(ctx, dm)
        assert np.linalg.norm(r - ref) <= 2e-5 * np.linalg.norm(ref), plan
