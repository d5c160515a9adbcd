"""Wall-model boundary assembly on the GPU (FP64) against the oracle.

* The term alone (fea_wall_assemble): flat plates of quads and of triangles
  with jittered nodes and random exchange velocities, the channel's prism
  wall layers (triangles), the airplane mesh's wall (triangles); to 1e-12 of
  the largest entry (same FP64 formulas; exp / log1p differ by an ulp).
* In the time step: RK stages (FP64 and mixed) and the graph-replayed step
  with the walls released from the no-slip hold, against oracle stages with
  the boundary term; the mixed stage's wall contribution (its u_tau is the
  FP32 Newton root) to 2e-5; the allocation-free stage adds the same term.
* Errors: a face ordered into the fluid and out-of-range ids are rejected at
  setup (FEA_EMESH), bad constants with FEA_EINVAL; clearing the faces
  removes the term.
"""
import dataclasses

import numpy as np
import pytest
import torch

import oracle as O
from paper_2005_05899_b300 import fea
from paper_2005_05899_b300 import meshgen as mg
from test_oracle_wall import _plate

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = fea.Context(0)
    yield c
    c.close()


def _wall_gpu(ctx, m, u, nu, wall):
    dm = ctx.upload_mesh(m)
    dm.upload_field(u, np.zeros(m.n_nodes), nu, 0.07)
    dm.wall_setup(**wall)
    rhs = torch.zeros((3, m.n_nodes), dtype=torch.float64, device="cuda")
    dm.wall_assemble(rhs)
    ctx.sync_status()
    return rhs.cpu().numpy().T, dm


def _plate_mesh(quads, rng):
    xyz, hexes, wall = _plate(nx=7, ny=5, h=0.03, quads=quads, rng=rng)
    return mg.Mesh(xyz=xyz, conn={mg.HEX08: hexes}), wall


@pytest.mark.parametrize("quads", [True, False])
def test_plate_matches_oracle(ctx, quads):
    rng = np.random.default_rng(11 + quads)
    m, wall = _plate_mesh(quads, rng)
    u = rng.standard_normal((m.n_nodes, 3)) * 0.4 + [1.0, 0.3, 0.0]
    nu = 1.5e-5
    got, _ = _wall_gpu(ctx, m, u, nu, wall)
    ref = O.wall_rhs(O.OracleMesh.of(m), u, nu, **wall)
    assert np.abs(ref).max() > 0
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_channel_prism_walls_match_oracle(ctx):
    m = mg.channel_mesh(nx=12, ny=12, nz=8, seed=3, n_layers=2, split_frac=0.3)
    rng = np.random.default_rng(2)
    u = rng.standard_normal((m.n_nodes, 3)) * 0.2 + [1.0, 0.0, 0.0]
    wall = m.wall_faces
    assert wall["tri"].shape[0] == 2 * 2 * 12 * 8
    got, _ = _wall_gpu(ctx, m, u, 1e-4, wall)
    ref = O.wall_rhs(O.OracleMesh.of(m), u, 1e-4, **wall)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_airplane_wall_matches_oracle(ctx):
    m = mg.airplane_mesh(30, seed=4)
    f = mg.inflow_field(m, seed=5)
    u = f.u.copy()
    held = m.dirichlet.astype(bool)
    u[held] += 0.3            # the field holds the wall at zero; any exchange value will do
    got, _ = _wall_gpu(ctx, m, u, f.nu, m.wall_faces)
    ref = O.wall_rhs(O.OracleMesh.of(m), u, f.nu, **m.wall_faces)
    assert np.abs(ref).max() > 0
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def _released_channel():
    m = mg.channel_mesh(nx=10, ny=12, nz=8, seed=4, n_layers=2, split_frac=0.3)
    f = mg.channel_field(m, seed=2, nu=1e-2)
    wall = m.wall_faces
    rng = np.random.default_rng(7)
    u = (f.u + 0.2 * rng.standard_normal(f.u.shape))[m.periodic_master]
    m_free = dataclasses.replace(m, dirichlet=None)
    return m, m_free, dataclasses.replace(f, u=u), wall


def _oracle_steps(m_free, f, dt, wall, steps):
    om = O.OracleMesh.of(m_free)
    u = f.u
    for _ in range(steps):
        u = O.rk3_step(om, m_free.periodic_master, None, u, f.p, f.nu, f.c_vreman, "vreman", dt, wall=wall)
    return u


def _state(dm):
    out = torch.empty((3, dm.n_nodes), dtype=torch.float64, device="cuda")
    dm.state(out)
    torch.cuda.synchronize()
    return out.cpu().numpy().T.copy()


def test_rk_stages_and_graph_with_walls(ctx):
    m, m_free, f, wall = _released_channel()
    dt = 2e-3
    ref = _oracle_steps(m_free, f, dt, wall, 1)
    no_wall = _oracle_steps(m_free, f, dt, None, 1)
    dm = ctx.upload_mesh(m_free)
    dm.wall_setup(**wall)
    dm.upload_field(f.u, f.p, f.nu, f.c_vreman)
    for k in range(3):
        dm.rk_stage(k, dt, prec="fp64")
    ctx.sync_status()
    got = _state(dm)
    effect = np.abs(ref - no_wall).max()
    assert effect > 1e-6 * np.abs(ref).max()          # the wall term matters here
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()
    # graph replay (captured after the wall setup), two steps
    dm.upload_field(f.u, f.p, f.nu, f.c_vreman)
    for _ in range(2):
        dm.rk_step_graph(dt, prec="fp64")
    ctx.sync_status()
    ref2 = _oracle_steps(m_free, f, dt, wall, 2)
    assert np.abs(_state(dm) - ref2).max() < 1e-12 * np.abs(ref2).max()
    # mixed precision: the element part in FP32, u_tau the FP32 root
    dm.upload_field(f.u, f.p, f.nu, f.c_vreman)
    dm.rk_step_graph(dt, prec="mixed")
    ctx.sync_status()
    upd = np.abs(ref - f.u).max()
    assert np.abs(_state(dm) - ref).max() < 2e-4 * upd


def test_mixed_stage_wall_term_uses_the_fp32_root(ctx):
    """Mixed precision: u_tau is the FP32 Newton root, so the stage's wall
    contribution (stage with walls minus stage without, same FP32 element
    part) matches the oracle's to FP32 accuracy."""
    m, m_free, f, wall = _released_channel()
    dt = 2e-3
    outs = []
    for w in (wall, None):
        dm = ctx.upload_mesh(m_free)
        if w is not None:
            dm.wall_setup(**w)
        dm.upload_field(f.u, f.p, f.nu, f.c_vreman)
        dm.rk_stage(0, dt, prec="mixed")
        ctx.sync_status()
        outs.append(_state(dm))
    om = O.OracleMesh.of(m_free)
    mass = O.periodic_fold(m_free.periodic_master, O.lumped_mass(om))
    args = (om, m_free.periodic_master, None, mass, f.u, f.u, f.p, f.nu, f.c_vreman, "vreman", 0, dt)
    ref = O.rk_stage(*args, wall=wall) - O.rk_stage(*args)
    got = outs[0] - outs[1]
    assert np.abs(ref).max() > 0
    assert np.abs(got - ref).max() <= 2e-5 * np.abs(ref).max()


def test_noalloc_stage_adds_the_wall_term(ctx):
    m, m_free, f, wall = _released_channel()
    dt = 2e-3
    dm = ctx.upload_mesh(m_free)
    dm.wall_setup(**wall)
    dev = lambda a: torch.tensor(np.ascontiguousarray(a.T), dtype=torch.float64, device="cuda")
    un = dev(f.u)
    p = torch.tensor(f.p, dtype=torch.float64, device="cuda")
    out = torch.empty_like(un)
    dm.rk_stage_noalloc(0, dt, un, un, p, out, f.nu, f.c_vreman, prec="fp64")
    ctx.sync_status()
    om = O.OracleMesh.of(m_free)
    mass = O.periodic_fold(m_free.periodic_master, O.lumped_mass(om))
    ref = O.rk_stage(om, m_free.periodic_master, None, mass, f.u, f.u, f.p, f.nu, f.c_vreman, "vreman", 0, dt,
                     wall=wall)
    assert np.abs(out.cpu().numpy().T - ref).max() < 1e-12 * np.abs(ref).max()


def test_setup_errors_and_clearing(ctx):
    rng = np.random.default_rng(5)
    m, wall = _plate_mesh(True, rng)
    dm = ctx.upload_mesh(m)
    u = np.tile([1.0, 0.0, 0.0], (m.n_nodes, 1))
    dm.upload_field(u, np.zeros(m.n_nodes), 1e-5, 0.07)
    flipped = dict(quad=wall["quad"][:, ::-1].copy(), quad_exch=wall["quad_exch"][:, ::-1].copy())
    with pytest.raises(fea.FeaError) as e:
        dm.wall_setup(**flipped)
    assert e.value.status == fea.EMESH
    bad = dict(quad=wall["quad"].copy(), quad_exch=wall["quad_exch"].copy())
    bad["quad_exch"][0, 0] = m.n_nodes
    with pytest.raises(fea.FeaError) as e:
        dm.wall_setup(**bad)
    assert e.value.status == fea.EMESH
    with pytest.raises(fea.FeaError) as e:
        dm.wall_setup(**wall, kappa=0.0)
    assert e.value.status == fea.EINVAL
    rhs = torch.zeros((3, m.n_nodes), dtype=torch.float64, device="cuda")
    dm.wall_setup(**wall)
    dm.wall_assemble(rhs)
    ctx.sync_status()
    assert float(rhs.abs().max()) > 0
    dm.wall_setup()                      # clear
    rhs.zero_()
    dm.wall_assemble(rhs)
    ctx.sync_status()
    assert float(rhs.abs().max()) == 0.0
