"""The allocation-free RK stage (fea_rk_stage_noalloc) against fea_rk_stage.

fea_rk_stage_noalloc serves callers that cannot allocate device memory at
call time (fixed, pre-reserved memory budgets): it reads and writes the
state in caller arrays and keeps its scratch in one static device array.
Two stages in a row through each entry point, and the three stages of a step
with the output written in place over u^(k) and over u^n, must agree within
the parity tolerances used elsewhere (FP64 path 1e-12; mixed path 2e-5 of the
update), and a mesh above the static limit must be rejected with a clear
error.

This file is collected last on purpose; it must pass alone in a fresh
process as well as after the other tests.
"""
import numpy as np
import pytest
import torch

from paper_2005_05899_b300 import fea
from paper_2005_05899_b300 import meshgen as mg

pytestmark = pytest.mark.gpu


def _state(dm):
    out = torch.empty((3, dm.n_nodes), dtype=torch.float64, device="cuda")
    dm.state(out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 2e-5)])
def test_noalloc_stage_matches_rk_stage_two_calls(prec, tol):
    ctx = fea.Context(0)
    m = mg.channel_mesh(nx=10, ny=12, nz=8, seed=4, n_layers=2, split_frac=0.3)
    f = mg.channel_field(m, seed=2, nu=1e-2)
    dm = ctx.upload_mesh(m)
    assert dm.n_nodes <= fea.NOALLOC_MAX_NODES
    dt = 2e-3
    # reference: the existing entry point on the library-owned state
    dm.upload_field(f.u, f.p, f.nu, f.c_vreman)
    dm.rk_stage(0, dt, prec=prec)
    ref1 = _state(dm)
    dm.rk_stage(1, dt, prec=prec)
    ref2 = _state(dm)
    # the allocation-free entry point on caller arrays, two calls in a row
    un = torch.tensor(np.ascontiguousarray(f.u.T), device="cuda")
    p = torch.tensor(f.p, device="cuda")
    out1 = torch.empty_like(un)
    out2 = torch.empty_like(un)
    dm.rk_stage_noalloc(0, dt, un, un, p, out1, f.nu, f.c_vreman, prec=prec)
    dm.rk_stage_noalloc(1, dt, un, out1, p, out2, f.nu, f.c_vreman, prec=prec)
    ctx.sync_status()
    got1, got2 = out1.cpu().numpy(), out2.cpu().numpy()
    u0 = f.u.T
    for got, ref in ((got1, ref1), (got2, ref2)):
        upd = np.abs(ref - u0).max()
        assert upd > 0
        if prec == "fp64":
            assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
        else:
            assert np.abs(got - ref).max() <= tol * upd
    ctx.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 2e-5)])
def test_noalloc_three_stages_with_aliased_outputs(prec, tol):
    """Stage 0 into a new array, stage 1 in place (uk_out is uk), stage 2
    written over u^n (uk_out is un): the three SSP-RK3 stages of one step."""
    ctx = fea.Context(0)
    m = mg.channel_mesh(nx=10, ny=12, nz=8, seed=4, n_layers=2, split_frac=0.3)
    f = mg.channel_field(m, seed=2, nu=1e-2)
    dm = ctx.upload_mesh(m)
    dt = 2e-3
    dm.upload_field(f.u, f.p, f.nu, f.c_vreman)
    refs = []
    for k in range(3):
        dm.rk_stage(k, dt, prec=prec)
        refs.append(_state(dm))
    un = torch.tensor(np.ascontiguousarray(f.u.T), device="cuda")
    p = torch.tensor(f.p, device="cuda")
    uk = torch.empty_like(un)
    dm.rk_stage_noalloc(0, dt, un, un, p, uk, f.nu, f.c_vreman, prec=prec)
    ctx.sync_status()
    got = [uk.cpu().numpy()]
    dm.rk_stage_noalloc(1, dt, un, uk, p, uk, f.nu, f.c_vreman, prec=prec)
    ctx.sync_status()
    got.append(uk.cpu().numpy())
    dm.rk_stage_noalloc(2, dt, un, uk, p, un, f.nu, f.c_vreman, prec=prec)
    ctx.sync_status()
    got.append(un.cpu().numpy())
    u0 = f.u.T
    for g, ref in zip(got, refs):
        upd = np.abs(ref - u0).max()
        assert upd > 0
        if prec == "fp64":
            assert np.abs(g - ref).max() <= tol * np.abs(ref).max()
        else:
            assert np.abs(g - ref).max() <= tol * upd
    ctx.close()


def test_noalloc_rejects_meshes_above_the_static_limit():
    ctx = fea.Context(0)
    m = mg.channel_mesh(nx=64, ny=64, nz=64, seed=1, n_layers=2, split_frac=0.0)
    assert m.n_nodes > fea.NOALLOC_MAX_NODES
    dm = ctx.upload_mesh(m)
    u = torch.zeros((3, dm.n_nodes), dtype=torch.float64, device="cuda")
    p = torch.zeros(dm.n_nodes, dtype=torch.float64, device="cuda")
    out = torch.empty_like(u)
    with pytest.raises(fea.FeaError) as ei:
        dm.rk_stage_noalloc(0, 1e-3, u, u, p, out, 1e-3)
    assert ei.value.status == fea.EINVAL
    assert "limit" in str(ei.value)
    ctx.close()
