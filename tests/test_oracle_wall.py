"""Pins of the oracle's equilibrium wall model (the boundary assembly of
Algorithm 1; law of the wall = Reichardt's, sampled at exchange nodes).

* Reichardt's f: f(0) = 0 and f'(0) = 1 (viscous sublayer, u+ = y+), f(y+) =
  y+ to 1e-3 y+^2 near the wall; f(y+) - ln(y+)/kappa tends to the log-law
  intercept C + ln(kappa)/kappa; f' agrees with central differences of f.
* Newton for u_tau: the round trip U = u_tau f(y u_tau / nu) -> u_tau over
  y+ from 1e-3 to 1e5; in the sublayer u_tau^2 = nu U / y.
* Traction: on a flat wall with a uniform sample velocity every Gauss point
  has the same u_tau, so the nodal forces sum to -u_tau^2 |wall| t and each
  node receives its lumped share (a quarter of a parallelogram quad, a third
  of a triangle); the normal part of the sampled velocity and tangential
  offsets of the exchange nodes change nothing (the distance is the normal
  one); the force rotates with the geometry; a quad and its two triangles
  agree; a face ordered the wrong way round is an error.
* The RK stage with walls differs from the one without by
  b_k dt M^-1 (folded wall term) on the free nodes (the update is linear in R).
"""
import numpy as np
import pytest

import oracle as O
from paper_2005_05899_b300 import meshgen as mg

K, C = O.WALL_KAPPA, O.WALL_C


def test_reichardt_viscous_sublayer():
    f0, d0 = O.reichardt(0.0)
    assert f0 == 0.0 and d0 == pytest.approx(1.0, abs=1e-15)
    for yp in (1e-6, 1e-4, 1e-2, 0.1):
        f, _ = O.reichardt(yp)
        assert abs(f - yp) <= 1e-3 * yp * yp


def test_reichardt_log_law_limit():
    intercept = C + np.log(K) / K
    for yp in (1e6, 1e8, 1e10):
        f, d = O.reichardt(yp)
        assert abs(f - np.log(yp) / K - intercept) <= 2.0 / (K * K * yp)
        assert d == pytest.approx(1.0 / (K * yp), rel=1e-4)
    # the transition is monotone
    ys = np.logspace(-3, 6, 400)
    fs = [O.reichardt(y)[0] for y in ys]
    assert np.all(np.diff(fs) > 0)


def test_reichardt_derivative_matches_differences():
    for yp in (0.3, 2.0, 7.5, 11.0, 30.0, 250.0, 4000.0):
        h = 1e-5 * yp
        fd = (O.reichardt(yp + h)[0] - O.reichardt(yp - h)[0]) / (2 * h)
        assert O.reichardt(yp)[1] == pytest.approx(fd, rel=1e-8)


@pytest.mark.parametrize("yp_target", [1e-3, 0.5, 5.0, 11.0, 40.0, 300.0, 1e4, 1e5])
def test_newton_round_trip(yp_target):
    nu, y = 1.5e-5, 2e-3
    ut_true = yp_target * nu / y
    U = ut_true * O.reichardt(yp_target)[0]
    ut, it = O.wall_utau(U, y, nu)
    assert ut == pytest.approx(ut_true, rel=1e-13)
    assert 0 < it <= 30


def test_newton_converges_from_deep_sublayer_to_log_layer():
    """U y / nu from 1e-14 to 1e10: Newton converges in a few steps (the
    sublayer bracket is evaluated without cancellation) and the result
    satisfies its equation."""
    for nu in (1e-2, 1.0 / 5600, 1.0 / 1.93e6):
        for y in np.logspace(-7, 0, 12):
            for U in np.logspace(-10, 2, 16):
                ut, it = O.wall_utau(U, y, nu)
                assert it <= 8
                assert ut * O.reichardt(y * ut / nu)[0] == pytest.approx(U, rel=1e-13)


def test_newton_sublayer_closed_form_and_zero():
    nu, y, U = 1e-3, 1e-4, 1e-3          # y+ about 0.01
    ut, _ = O.wall_utau(U, y, nu)
    assert ut * ut == pytest.approx(nu * U / y, rel=1e-4)
    assert O.wall_utau(0.0, y, nu)[0] == 0.0
    with pytest.raises(O.OracleError):
        O.wall_utau(1.0, 0.0, nu)


def _plate(nx=4, ny=3, h=0.05, quads=True, shear=(0.0, 0.0), rng=None):
    """Structured wall z = 0 over [0,1]x[0,0.6] (nodes jittered in-plane), an
    exchange layer at z = h shifted tangentially by `shear`; one layer of
    hexes so that the oracle mesh is valid."""
    xs, ys = np.linspace(0, 1, nx + 1), np.linspace(0, 0.6, ny + 1)
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    base = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], axis=1)
    if rng is not None:
        inner = (X.ravel() > 0) & (X.ravel() < 1) & (Y.ravel() > 0) & (Y.ravel() < 0.6)
        base[inner, :2] += rng.uniform(-0.02, 0.02, (inner.sum(), 2))
    top = base + np.array([shear[0], shear[1], h])
    xyz = np.concatenate([base, top])
    nb = base.shape[0]
    nid = lambda i, j: i * (ny + 1) + j
    q = np.array([[nid(i, j), nid(i + 1, j), nid(i + 1, j + 1), nid(i, j + 1)]
                  for i in range(nx) for j in range(ny)], np.int32)
    hexes = np.concatenate([q, q + nb], axis=1)
    # wall faces: the fluid is above (z > 0), so the face normal must point to -z
    qw = q[:, [0, 3, 2, 1]]
    if quads:
        return xyz, hexes, dict(quad=qw, quad_exch=qw + nb)
    tri = np.concatenate([qw[:, [0, 1, 2]], qw[:, [0, 2, 3]]])
    return xyz, hexes, dict(tri=tri, tri_exch=tri + nb)


def _om(xyz, hexes):
    return O.OracleMesh(xyz, {O.HEX08: hexes})


@pytest.mark.parametrize("quads", [True, False])
def test_flat_wall_total_force_and_lumped_shares(quads):
    nu, h, U0 = 2e-5, 0.05, 1.3
    xyz, hexes, wall = _plate(h=h, quads=quads)
    nb = xyz.shape[0] // 2
    u = np.zeros_like(xyz)
    u[nb:] = [U0, 0.0, 0.0]
    R = O.wall_rhs(_om(xyz, hexes), u, nu, **wall)
    ut, _ = O.wall_utau(U0, h, nu)
    tau = ut * ut
    assert np.allclose(R.sum(axis=0), [-tau * 0.6, 0.0, 0.0], rtol=1e-13, atol=1e-18)
    assert np.all(R[nb:] == 0.0)
    # lumped shares: a corner node of the plate touches one face
    faces = wall["quad"] if quads else wall["tri"]
    share = np.zeros(nb)
    for f in faces:
        X = xyz[f]
        if quads:
            area = np.linalg.norm(np.cross(X[1] - X[0], X[3] - X[0]))
            share[f] += area / 4
        else:
            area = 0.5 * np.linalg.norm(np.cross(X[1] - X[0], X[2] - X[0]))
            share[f] += area / 3
    assert np.allclose(R[:nb, 0], -tau * share, rtol=1e-12)


def test_normal_velocity_and_tangential_offsets_change_nothing():
    nu, h = 2e-5, 0.04
    rng = np.random.default_rng(3)
    xyz, hexes, wall = _plate(h=h, rng=rng)
    nb = xyz.shape[0] // 2
    u = np.zeros_like(xyz)
    u[nb:] = rng.standard_normal((nb, 3)) * [1.0, 1.0, 0.0] + [1.0, 0.2, 0.0]
    R0 = O.wall_rhs(_om(xyz, hexes), u, nu, **wall)
    u2 = u.copy()
    u2[nb:, 2] = rng.standard_normal(nb)          # wall-normal velocity at the exchange nodes
    R1 = O.wall_rhs(_om(xyz, hexes), u2, nu, **wall)
    assert np.allclose(R1, R0, rtol=1e-13, atol=1e-16)
    xyz_s, hexes_s, wall_s = _plate(h=h, rng=np.random.default_rng(3), shear=(0.01, -0.007))
    R2 = O.wall_rhs(_om(xyz_s, hexes_s), u, nu, **wall_s)
    assert np.allclose(R2, R0, rtol=1e-13, atol=1e-16)


def test_force_rotates_with_the_geometry():
    nu, h = 2e-5, 0.05
    rng = np.random.default_rng(4)
    xyz, hexes, wall = _plate(h=h, rng=rng)
    nb = xyz.shape[0] // 2
    u = np.zeros_like(xyz)
    u[nb:] = rng.standard_normal((nb, 3)) * 0.3 + [1.0, -0.4, 0.0]
    R = O.wall_rhs(_om(xyz, hexes), u, nu, **wall)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    Rq = O.wall_rhs(_om(xyz @ Q.T + 0.3, hexes), u @ Q.T, nu, **wall)
    assert np.allclose(Rq, R @ Q.T, rtol=1e-12, atol=1e-12 * np.abs(R).max())


def test_quad_equals_its_two_triangles_for_uniform_sampling():
    nu, h = 1e-5, 0.02
    xyz, hexes, wq = _plate(h=h, quads=True)
    _, _, wt = _plate(h=h, quads=False)
    nb = xyz.shape[0] // 2
    u = np.zeros_like(xyz)
    u[nb:] = [0.8, 0.6, 0.0]
    Rq = O.wall_rhs(_om(xyz, hexes), u, nu, **wq)
    Rt = O.wall_rhs(_om(xyz, hexes), u, nu, **wt)
    assert np.allclose(Rq.sum(axis=0), Rt.sum(axis=0), rtol=1e-13)


def test_reversed_face_is_an_error():
    xyz, hexes, wall = _plate()
    u = np.ones_like(xyz)
    flipped = dict(quad=wall["quad"][:, ::-1].copy(), quad_exch=wall["quad_exch"][:, ::-1].copy())
    with pytest.raises(O.OracleError):
        O.wall_rhs(_om(xyz, hexes), u, 1e-5, **flipped)


def test_rk_stage_with_walls_is_linear_in_the_boundary_term():
    m = mg.channel_mesh(nx=6, ny=10, nz=4, seed=3, n_layers=2, split_frac=0.3)
    f = mg.channel_field(m, seed=4, nu=1e-3)
    wall = m.wall_faces
    assert wall["tri"].shape[0] > 0
    om = O.OracleMesh.of(m)
    mass = O.periodic_fold(m.periodic_master, O.lumped_mass(om))
    # the channel's walls are no-slip (held); release them so the term shows
    dirichlet = np.zeros(m.n_nodes, np.uint8)
    rng = np.random.default_rng(5)
    uk = f.u + 0.1 * rng.standard_normal(f.u.shape)
    uk = uk[m.periodic_master]
    dt, stage = 1e-3, 1
    a = O.rk_stage(om, m.periodic_master, dirichlet, mass, f.u, uk, f.p, f.nu, f.c_vreman, "vreman", stage, dt)
    b = O.rk_stage(om, m.periodic_master, dirichlet, mass, f.u, uk, f.p, f.nu, f.c_vreman, "vreman", stage, dt,
                   wall=wall)
    Rw = O.periodic_fold(m.periodic_master, O.wall_rhs(om, uk, f.nu, **wall))
    assert np.abs(Rw).max() > 0
    assert np.allclose(b - a, 0.25 * dt * Rw / mass[:, None], rtol=1e-10, atol=1e-15)
