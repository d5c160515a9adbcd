"""The colour and warp-aggregated scatters against the oracle.

* FEA_SCATTER_COLOUR (greedy element colouring, one launch per colour, plain
  FP64 read-modify-write) and FEA_SCATTER_WARP (FP64 atomics after a
  match_any sum within the warp), each in FP64 (1e-12, the stated FP64
  tolerance) and mixed precision (the mixed gates of the parity tests), on
  the mixed channel mesh (all four element types, FP64-Jacobian prisms).
* The colour scatter fixes the summation order: two assemblies, and an RK
  stage run twice from the same state, agree bit for bit.  A colouring that
  let two elements of a colour share a node would race in the plain
  read-modify-writes and fail the 1e-12 parity.
* RK stages and the graph step under a colour plan match the oracle; the
  allocation-free stage works under it; the MLP closure keeps atomics.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2005_05899_b300 import fea
from paper_2005_05899_b300 import meshgen as mg
from test_gpu_parity import FP64_TOL, MIXED_L2, MIXED_MAX, errors, gpu_rhs, oracle_rhs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = fea.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def mixed_small():
    m = mg.channel_mesh(nx=12, ny=14, nz=10, seed=21, n_layers=2, split_frac=0.3)
    assert len(m.conn) == 4
    return m, mg.channel_field(m, seed=5, nu=1e-2)


@pytest.mark.parametrize("scatter", ["colour", "warp"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_scatter_matches_oracle(ctx, mixed_small, scatter, prec):
    m, f = mixed_small
    r, _ = gpu_rhs(ctx, m, f, prec, scatter=scatter)
    l2, mx = errors(r, oracle_rhs(m, f))
    if prec == "fp64":
        assert l2 < FP64_TOL and mx < FP64_TOL
    else:
        assert l2 < MIXED_L2 and mx < MIXED_MAX


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_colour_scatter_is_bitwise_reproducible(ctx, mixed_small, prec):
    m, f = mixed_small
    r1, dm = gpu_rhs(ctx, m, f, prec, scatter="colour")
    r2, _ = gpu_rhs(ctx, m, f, prec, scatter="colour", dm=dm)
    r3, _ = gpu_rhs(ctx, m, f, prec, scatter="colour")          # a fresh upload
    assert np.array_equal(r1, r2) and np.array_equal(r1, r3)


def _state(dm):
    out = torch.empty((3, dm.n_nodes), dtype=torch.float64, device="cuda")
    dm.state(out)
    torch.cuda.synchronize()
    return out.cpu().numpy().T.copy()


def test_rk_under_a_colour_plan(ctx, mixed_small):
    m, f = mixed_small
    dt = 2e-3
    dm = ctx.upload_mesh(m)
    dm.set_plan("colour", 128, 256, 0)
    assert dm.get_plan().scatter == 3
    dm.upload_field(f.u, f.p, f.nu, f.c_vreman)
    for k in range(3):
        dm.rk_stage(k, dt, prec="fp64")
    ctx.sync_status()
    ref = O.rk3_step(O.OracleMesh.of(m), m.periodic_master, m.dirichlet, f.u, f.p, f.nu, f.c_vreman, "vreman", dt)
    got = _state(dm)
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()
    # graph replay, mixed precision, twice from the same state: bitwise equal
    outs = []
    for _ in range(2):
        dm.upload_field(f.u, f.p, f.nu, f.c_vreman)
        dm.rk_step_graph(dt, prec="mixed")
        ctx.sync_status()
        outs.append(_state(dm))
    assert np.array_equal(outs[0], outs[1])
    upd = np.abs(ref - f.u).max()
    assert np.abs(outs[0] - ref).max() < 2e-4 * upd


def test_noalloc_stage_under_a_colour_plan(ctx, mixed_small):
    m, f = mixed_small
    dm = ctx.upload_mesh(m)
    dm.set_plan("colour", 128, 256, 0)
    dev = lambda a: torch.tensor(np.ascontiguousarray(a.T), dtype=torch.float64, device="cuda")
    un = dev(f.u)
    p = torch.tensor(f.p, dtype=torch.float64, device="cuda")
    out = torch.empty_like(un)
    dm.rk_stage_noalloc(0, 2e-3, un, un, p, out, f.nu, f.c_vreman, prec="fp64")
    ctx.sync_status()
    om = O.OracleMesh.of(m)
    mass = O.periodic_fold(m.periodic_master, O.lumped_mass(om))
    ref = O.rk_stage(om, m.periodic_master, m.dirichlet, mass, f.u, f.u, f.p, f.nu, f.c_vreman, "vreman", 0, 2e-3)
    assert np.abs(out.cpu().numpy().T - ref).max() < 1e-12 * np.abs(ref).max()


def test_batch_autotuner_picks_a_valid_mode(ctx):
    """fea_autotune_batched times the persistent launch (three chunk sizes)
    against per-mesh atomic / warp / colour launches; whatever it keeps, the
    batched assembly still matches the oracle."""
    batch = mg.batch_meshes(count=5, seed=9, e_min=2e3, e_max=2e4)
    dms, outs = [], []
    for m, f in batch:
        dm = ctx.upload_mesh(m)
        dm.upload_field(f.u, f.p, f.nu, f.c_vreman)
        dms.append(dm)
        outs.append(torch.full((3, dm.n_nodes), 7.0, dtype=torch.float64, device="cuda"))
    best = ctx.autotune_batched(dms, prec="mixed", closure="vreman")
    assert best.scatter in (1, 2, 3, 4)
    if best.scatter == 2:
        assert best.chunk_elems in (128, 256, 512)
    for dm in dms:
        assert dm.get_plan().scatter == best.scatter
    ctx.assemble_batched(dms, outs, prec="mixed", closure="vreman")
    ctx.sync_status()
    for (m, f), o in zip(batch, outs):
        l2, mx = errors(o.cpu().numpy().T, oracle_rhs(m, f))
        assert l2 < MIXED_L2 and mx < MIXED_MAX, (best.as_dict(), l2, mx)
