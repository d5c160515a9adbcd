"""Pressure projection on the GPU against the FP64 oracle.

* B(u) and G(p) on the mixed mesh: FP64 element kernels against the oracle
  to 1e-12 of the largest entry.
* Jacobi-PCG on the periodic-class Laplacian: b = K x* (oracle K) for a
  known x* with x* = 0 on the pinned class; the solution at rtol 1e-12 must
  match x* to 1e-8 relative (the Laplacian's condition number times rtol).
* The projection step against the oracle's direct solve: periodic
  Taylor-Green mesh (u* = TG + a gradient) and the walled channel
  (velocity-Dirichlet nodes held), corrected velocity to 1e-8 of its norm.
"""
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


@pytest.fixture(scope="module")
def channel():
    m = mg.channel_mesh(nx=12, ny=10, nz=8, seed=3, n_layers=2, split_frac=0.3)
    f = mg.channel_field(m, seed=4, nu=1e-3)
    return m, f


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def test_divergence_and_gradient_match_oracle(ctx, channel):
    m, f = channel
    dm = ctx.upload_mesh(m)
    om = O.OracleMesh.of(m)
    rng = np.random.default_rng(1)
    p = rng.standard_normal(m.n_nodes)
    div = dm.divergence(dev(f.u.T), torch.empty(m.n_nodes, dtype=torch.float64, device="cuda"))
    grad = dm.gradient(dev(p), torch.empty((3, m.n_nodes), dtype=torch.float64, device="cuda"))
    ctx.sync_status()
    rb, rg = O.divergence(om, f.u), O.gradient(om, p)
    assert np.abs(div.cpu().numpy() - rb).max() <= 1e-12 * np.abs(rb).max()
    assert np.abs(grad.cpu().numpy().T - rg).max() <= 1e-12 * np.abs(rg).max()


def test_pcg_solves_the_class_laplacian(ctx, channel):
    m, _ = channel
    dm = ctx.upload_mesh(m)
    dm.poisson_setup()
    om = O.OracleMesh.of(m)
    P, cls, masters = O.fold_matrix(m.periodic_master)
    rng = np.random.default_rng(2)
    xc = rng.standard_normal(masters.size)
    xc[cls[0]] = 0.0                       # the pinned class
    x_nodes = xc[cls]
    b = O.assemble_laplacian(om) @ x_nodes   # fold(b) = K_folded x
    x = torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda")
    it, rr = dm.poisson_solve(dev(b), x, rtol=1e-12, max_iter=5000)
    ctx.sync_status()
    got = x.cpu().numpy()
    assert rr <= 1e-12 and 0 < it < 5000
    assert np.linalg.norm(got - x_nodes) <= 1e-8 * np.linalg.norm(x_nodes)
    assert np.all(got[cls == cls[0]] == 0.0)
    # a second solve from the solution converges at once
    it2, _ = dm.poisson_solve(dev(b), x, rtol=1e-10, max_iter=50)
    assert it2 <= 1


def _project_both(ctx, m, f, u_star, dt):
    om = O.OracleMesh.of(m)
    master = m.periodic_master if m.periodic_master is not None else np.arange(m.n_nodes)
    mass = O.periodic_fold(master, O.lumped_mass(om))
    dirichlet = m.dirichlet if m.dirichlet is not None else np.zeros(m.n_nodes, np.uint8)
    u_ref, p_ref, dp_ref = O.project(om, master, dirichlet, np.array([0]), mass, u_star, f.p, dt)
    dm = ctx.upload_mesh(m)
    dm.upload_field(u_star, f.p, f.nu, f.c_vreman)
    dm.poisson_setup()
    it, rr = dm.project(dt, rtol=1e-12, max_iter=5000)
    out = torch.empty((3, m.n_nodes), dtype=torch.float64, device="cuda")
    dm.state(out)
    ctx.sync_status()
    return out.cpu().numpy().T, u_ref, it, rr


def test_projection_matches_oracle_periodic_tgv(ctx):
    m = mg.tgv_mesh(12)
    f = mg.tgv_field(m)
    X = m.xyz[m.periodic_master]
    gphi = np.stack([np.cos(X[:, 0]) * np.sin(X[:, 1]) * np.cos(X[:, 2]),
                     np.sin(X[:, 0]) * np.cos(X[:, 1]) * np.cos(X[:, 2]),
                     -np.sin(X[:, 0]) * np.sin(X[:, 1]) * np.sin(X[:, 2])], axis=1)
    u_star = f.u + 0.05 * gphi
    got, ref, it, rr = _project_both(ctx, m, f, u_star, 0.01)
    assert rr <= 1e-12 and it > 0
    assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref)
    # the projection changed the field
    assert np.linalg.norm(got - u_star) > 0.01 * np.linalg.norm(0.05 * gphi)


def test_projection_matches_oracle_walled_channel(ctx, channel):
    m, f = channel
    got, ref, it, rr = _project_both(ctx, m, f, f.u, 0.005)
    assert rr <= 1e-12
    assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref)
    held = m.dirichlet.astype(bool)
    assert np.array_equal(got[held], f.u[held])
