"""Pins of the oracle's Runge-Kutta stage update and MLP closure pieces.

* RK3: for a linear operator L (viscous term only) three SSP-RK3 stages must
  reproduce the third-order Taylor polynomial u + dt L u + dt^2/2 L^2 u +
  dt^3/6 L^3 u exactly (up to round-off); Dirichlet nodes keep u^n.
* MLP: forward pass against PyTorch float64 layers (library), the gradient
  against PyTorch autograd and against central finite differences, one Adam
  step against torch.optim.Adam, and the invariant features against closed
  forms and rotation invariance.
"""
import math

import numpy as np
import torch

import oracle as O
from paper_2005_05899_b300 import meshgen as mg


def _L(om, master, mass, u, p, nu):
    R = O.assemble_rhs(om, u, p, nu, 0.0, "none", mask=O.TERM_VISC)
    R = O.periodic_fold(master, R)
    return R / mass[:, None]


def test_rk3_equals_taylor_polynomial_for_linear_operator():
    m = mg.tgv_mesh(6)
    f = mg.tgv_field(m)
    rng = np.random.default_rng(0)
    u = f.u + 0.1 * rng.standard_normal(f.u.shape)[m.periodic_master]
    p = np.zeros(m.n_nodes)
    om = O.OracleMesh.of(m)
    nu, dt = 0.5, 0.03
    mass = O.periodic_fold(m.periodic_master, O.lumped_mass(om))
    L1 = _L(om, m.periodic_master, mass, u, p, nu)
    L2 = _L(om, m.periodic_master, mass, L1, p, nu)
    L3 = _L(om, m.periodic_master, mass, L2, p, nu)
    taylor = u + dt * L1 + dt ** 2 / 2 * L2 + dt ** 3 / 6 * L3
    out = O.rk3_step(om, m.periodic_master, None, u, p, nu, 0.0, "none", dt, mask=O.TERM_VISC)
    assert np.abs(out - taylor).max() < 1e-13 * np.abs(u).max()
    # and it differs from a first-order update by a visible margin
    assert np.abs(out - (u + dt * L1)).max() > 1e-6


def test_rk_stages_compose_as_shu_osher_with_full_rhs():
    m = mg.channel_mesh(nx=6, ny=10, nz=4, seed=2, n_layers=2, split_frac=0.3)
    f = mg.channel_field(m, seed=1, nu=0.01)
    om = O.OracleMesh.of(m)
    master, dmask = m.periodic_master, m.dirichlet
    mass = O.periodic_fold(master, O.lumped_mass(om))
    dt = 1e-3

    def L(u):
        R = O.periodic_fold(master, O.assemble_rhs(om, u, f.p, f.nu, 0.07, "vreman"))
        return R / mass[:, None]

    un = f.u
    u1 = un + dt * L(un)
    u2 = 0.75 * un + 0.25 * (u1 + dt * L(u1))
    u3 = un / 3 + 2.0 / 3.0 * (u2 + dt * L(u2))
    d = dmask.astype(bool)
    assert d.any() and (~d).any()
    s1 = O.rk_stage(om, master, dmask, mass, un, un, f.p, f.nu, 0.07, "vreman", 0, dt)
    s2 = O.rk_stage(om, master, dmask, mass, un, s1, f.p, f.nu, 0.07, "vreman", 1, dt)
    s3 = O.rk_stage(om, master, dmask, mass, un, s2, f.p, f.nu, 0.07, "vreman", 2, dt)
    # every stage holds Dirichlet nodes at u^n
    for s in (s1, s2, s3):
        assert np.array_equal(s[d], un[d])
    # a held value reaches one element layer further per stage: nodes three
    # layers away from every Dirichlet node follow the unconstrained
    # Shu-Osher composition through all three stages
    near = d.copy()
    for _ in range(3):
        grow = near.copy()
        for c in m.conn.values():
            touch = near[c].any(axis=1)
            grow[c[touch].ravel()] = True
        near = grow
    free = ~near
    assert free.any()
    scale = np.abs(un).max()
    assert np.abs(s1[~d] - u1[~d]).max() < 1e-14 * scale
    assert np.abs(s3[free] - u3[free]).max() < 1e-14 * scale
    full = O.rk3_step(om, master, dmask, un, f.p, f.nu, 0.07, "vreman", dt)
    assert np.array_equal(full, s3)


# --------------------------------------------------------------------------
# MLP

def random_theta(rng, scale=0.4):
    return scale * rng.standard_normal(O.nparam())


def torch_model(theta):
    H, I = O.MLP_H, O.MLP_IN
    t = torch.tensor(theta, dtype=torch.float64)
    off = 0

    def take(n, shape):
        nonlocal off
        v = t[off:off + n].reshape(shape)
        off += n
        return v

    w1 = take(H * I, (H, I)); b1 = take(H, (H,))
    w2 = take(H * H, (H, H)); b2 = take(H, (H,))
    w3 = take(H * H, (H, H)); b3 = take(H, (H,))
    w4 = take(H, (1, H)); b4 = take(1, (1,))
    seq = torch.nn.Sequential(torch.nn.Linear(I, H), torch.nn.SiLU(), torch.nn.Linear(H, H), torch.nn.SiLU(),
                              torch.nn.Linear(H, H), torch.nn.SiLU(), torch.nn.Linear(H, 1)).double()
    with torch.no_grad():
        for lin, (w, b) in zip([seq[0], seq[2], seq[4], seq[6]], [(w1, b1), (w2, b2), (w3, b3), (w4, b4)]):
            lin.weight.copy_(w)
            lin.bias.copy_(b)
    return seq


def test_mlp_forward_matches_torch_layers():
    rng = np.random.default_rng(1)
    theta = random_theta(rng)
    mean = rng.standard_normal(6)
    std = rng.uniform(0.5, 2, 6)
    mlp = O.MLPParams(theta, mean, std, out_scale=3e-4)
    x = rng.standard_normal((33, 6)) * 2
    y = O.mlp_forward(mlp, x)
    seq = torch_model(theta)
    xt = (torch.tensor(x) - torch.tensor(mean)) / torch.tensor(std)
    ref = 3e-4 * torch.nn.functional.softplus(seq(xt), threshold=50.0).squeeze(1).detach().numpy()
    assert np.allclose(y, ref, rtol=1e-13, atol=0)


def test_mlp_gradient_matches_autograd_and_finite_differences():
    rng = np.random.default_rng(2)
    theta = random_theta(rng)
    x = rng.standard_normal((9, 6))
    y = rng.uniform(0, 2, 9)
    loss, g = O.mlp_loss_grad(theta, x, y)
    seq = torch_model(theta)
    pred = torch.nn.functional.softplus(seq(torch.tensor(x)), threshold=50.0).squeeze(1)
    tl = ((pred - torch.tensor(y)) ** 2).mean()
    tl.backward()
    gt = torch.cat([torch.cat([lin.weight.grad.reshape(-1), lin.bias.grad.reshape(-1)])
                    for lin in (seq[0], seq[2], seq[4], seq[6])]).numpy()
    assert math.isclose(loss, tl.item(), rel_tol=1e-13)
    assert np.linalg.norm(g - gt) <= 1e-11 * np.linalg.norm(gt)
    h = 1e-6
    idx = np.concatenate([rng.choice(g.size, 150, replace=False), np.arange(g.size - 65, g.size)])
    for k in idx:
        tp = theta.copy(); tp[k] += h
        tm = theta.copy(); tm[k] -= h
        fd = (O.mlp_loss_grad(tp, x, y, False)[0] - O.mlp_loss_grad(tm, x, y, False)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k])) + 1e-9, k


def test_adam_step_matches_torch_optim():
    rng = np.random.default_rng(3)
    n = 50
    theta = rng.standard_normal(n)
    m1 = np.zeros(n)
    m2 = np.zeros(n)
    pt = torch.tensor(theta.copy(), requires_grad=True)
    opt = torch.optim.Adam([pt], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    for t in range(1, 4):
        grad = rng.standard_normal(n)
        O.adam_step(theta, grad, m1, m2, 1e-2, 0.9, 0.999, 1e-8, t)
        pt.grad = torch.tensor(grad)
        opt.step()
    assert np.allclose(theta, pt.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_mlp_features_closed_forms_and_invariance():
    nu = 1e-3
    # solid rotation: no strain, |G|^2 = 2 w^2
    w = 1.3
    G = np.array([[0, -w, 0], [w, 0, 0], [0, 0, 0]], float)
    x = O.mlp_features(G, 0.5, nu)
    assert np.allclose(x, [0, -1, 0, 0, 0, math.log(0.25 * math.sqrt(2) * w / nu)], atol=1e-14)
    # axisymmetric strain diag(s, s, -2s): tr S^3 / |G|^3 = -6 s^3 / (6 s^2)^(3/2) = -1/sqrt(6)
    s_ = 0.7
    x = O.mlp_features(np.diag([s_, s_, -2 * s_]), 2.0, nu)
    assert np.allclose(x, [1, 0, -1 / math.sqrt(6), 0, 0, math.log(4.0 * math.sqrt(6) * s_ / nu)], atol=1e-14)
    # plane shear u = (gy, 0, 0): S and O share |G|^2 / 2; tr S O^2 = 0, tr S^2 O^2 = -|G|^4 / 8
    x = O.mlp_features(np.array([[0, 2.0, 0], [0, 0, 0], [0, 0, 0]]), 1.0, nu)
    assert np.allclose(x[:5], [0.5, -0.5, 0, 0, -0.125], atol=1e-14)
    rng = np.random.default_rng(4)
    G = rng.standard_normal((3, 3))
    q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    # rotation invariance, and scale invariance of the first five (the sixth shifts by log lambda)
    assert np.allclose(O.mlp_features(q @ G @ q.T, 0.3, nu), O.mlp_features(G, 0.3, nu), rtol=1e-12, atol=1e-13)
    lam = 37.0
    x1, x2 = O.mlp_features(G, 0.3, nu), O.mlp_features(lam * G, 0.3, nu)
    assert np.allclose(x2[:5], x1[:5], rtol=1e-12, atol=1e-14)
    assert abs(x2[5] - x1[5] - math.log(lam)) < 1e-12
    # a vanishing gradient has no direction
    assert np.all(O.mlp_features(np.zeros((3, 3)), 0.3, nu) == 0)


def test_mlp_closure_with_constant_output_is_a_viscosity():
    """With all weights zero the network's output is the constant C = s
    softplus(b4), so nu_t = C Delta^2 |G|.  A linear velocity field (one G
    everywhere) on a Kuhn-split grid of equal cubes (one element volume, so
    one Delta) makes that a constant viscosity: the MLP closure's subgrid
    term must equal the viscous term with nu replaced by C Delta^2 |G| (the
    2 eps form is linear in the viscosity)."""
    m = mg.tgv_mesh(4)
    rng = np.random.default_rng(6)
    B = rng.standard_normal((3, 3))
    u = m.xyz @ B.T + 0.3
    p = np.zeros(m.n_nodes)
    nu = 1e-3
    theta = np.zeros(O.nparam())
    theta[-1] = 0.3
    scale = 2e-2
    mlp = O.MLPParams(theta, np.zeros(6), np.ones(6), out_scale=scale)
    h = 2 * math.pi / 4
    delta = (h ** 3 / 6.0) ** (1.0 / 3.0)
    nut = scale * math.log1p(math.exp(0.3)) * delta ** 2 * np.linalg.norm(B)
    om = O.OracleMesh.of(m)
    sgs, nut_gp = O.assemble_rhs(om, u, p, nu, 0.07, "mlp", mask=O.TERM_SGS, mlp=mlp, want_nut=True)
    visc = O.assemble_rhs(om, u, p, nu, 0.07, "none", mask=O.TERM_VISC)
    assert all(np.allclose(v, nut, rtol=1e-12, atol=0) for v in nut_gp.values())
    assert np.abs(sgs - visc * (nut / nu)).max() <= 1e-11 * np.abs(visc * (nut / nu)).max()
