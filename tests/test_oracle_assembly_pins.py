"""Pins of the oracle's assembly against what the mathematics fixes.

The paper prints no worked example of the assembly, so every expected value
here comes from a closed form, an invariant, a library routine or an
independent high-order evaluation:
  * patch test: a linear velocity gives exact gradients and a zero Galerkin
    viscous residual at interior nodes;
  * uniform field: zero RHS for every term;
  * lumped mass sums to the mesh volume; V/4 per node for a tetrahedron;
  * linear pressure: R_p = -M_L grad p at every node;
  * rigid rotation: R(Qx, Qu, p) = Q R(x, u, p), nu_t unchanged;
  * Vreman closed forms (pure shear, axisymmetric strain, solid rotation);
  * tetrahedron closed forms (consistent mass V(1 + delta_ab)/20);
  * global identity for a linear field on the mixed mesh;
  * independent high-order (Gauss-Legendre, collapsed) evaluation of the
    element residual on affinely mapped elements of every type;
  * Taylor-Green analytic RHS with O(h^2) convergence.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2005_05899_b300 import meshgen as mg

REF_NODES = {
    O.TET04: np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float),
    O.PYR05: np.array([[-1, -1, 0], [1, -1, 0], [1, 1, 0], [-1, 1, 0], [0, 0, 1]], float),
    O.PEN06: np.array([[0, 0, -1], [1, 0, -1], [0, 1, -1], [0, 0, 1], [1, 0, 1], [0, 1, 1]], float),
    O.HEX08: np.array([[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1],
                       [-1, -1, 1], [1, -1, 1], [1, 1, 1], [-1, 1, 1]], float),
}
ALL_TYPES = [O.TET04, O.PYR05, O.PEN06, O.HEX08]


@pytest.fixture(scope="module")
def small_mixed():
    m = mg.channel_mesh(nx=8, ny=12, nz=6, seed=11, n_layers=2, split_frac=0.35, sfc=True)
    for t in ALL_TYPES:
        assert m.n_elem(t) > 0
    return m


def box_boundary(m, lx=4 * math.pi, lz=2 * math.pi):
    x = m.xyz
    tol = 1e-12
    return ((np.abs(x[:, 0]) < tol) | (np.abs(x[:, 0] - lx) < tol) | (np.abs(x[:, 2]) < tol)
            | (np.abs(x[:, 2] - lz) < tol) | (np.abs(np.abs(x[:, 1]) - 1) < tol))


def rand_B(rng, scale=1.0):
    return scale * rng.standard_normal((3, 3))


# --------------------------------------------------------------------------

@pytest.mark.parametrize("etype", ALL_TYPES)
def test_patch_gradients_exact_on_distorted_elements(etype):
    rng = np.random.default_rng(etype)
    m = mg.single_element(etype, seed=10 + etype, distort=0.15)
    X = m.xyz[m.conn[etype][0]]
    B = rand_B(rng)
    a = rng.standard_normal(3)
    U = a + X @ B.T
    N, dNdx, W, det = O.element_geometry(etype, X)
    for g in range(N.shape[0]):
        G = U.T @ dNdx[g]
        assert np.allclose(G, B, atol=1e-12)
        assert np.allclose(X.T @ dNdx[g], np.eye(3), atol=1e-12)
        assert np.allclose(N[g] @ U, a + (N[g] @ X) @ B.T, atol=1e-13)
    assert np.all(det > 0)


def test_patch_viscous_residual_zero_at_interior_nodes(small_mixed):
    m = small_mixed
    rng = np.random.default_rng(3)
    B = rand_B(rng)
    u = rng.standard_normal(3) + m.xyz @ B.T
    p = np.zeros(m.n_nodes)
    om = O.OracleMesh.of(m)
    R = O.assemble_rhs(om, u, p, nu=0.37, c_vreman=0.0, closure="none", mask=O.TERM_VISC)
    inner = ~box_boundary(m)
    scale = np.abs(R).max()
    assert scale > 1e-3
    assert np.abs(R[inner]).max() < 1e-12 * max(1.0, scale)


def test_uniform_field_gives_zero_rhs(small_mixed):
    m = small_mixed
    u = np.tile([0.3, -1.2, 0.7], (m.n_nodes, 1))
    p = np.full(m.n_nodes, 2.5)
    om = O.OracleMesh.of(m)
    R, nut = O.assemble_rhs(om, u, p, nu=0.1, c_vreman=0.07, closure="vreman", want_nut=True)
    assert np.abs(R).max() < 1e-13
    for t in nut:   # gradients vanish up to round-off, so does nu_t
        assert np.abs(nut[t]).max() < 1e-15


def test_lumped_mass_sums_to_volume():
    m1 = mg.tgv_mesh(16)
    ml = O.lumped_mass(O.OracleMesh.of(m1))
    assert abs(ml.sum() - (2 * math.pi) ** 3) < 1e-11 * (2 * math.pi) ** 3
    m2 = mg.channel_mesh(nx=16, ny=16, nz=8, seed=5, n_layers=2, split_frac=0.3)
    ml2 = O.lumped_mass(O.OracleMesh.of(m2))
    vol = 4 * math.pi * 2 * 2 * math.pi
    assert abs(ml2.sum() - vol) < 1e-12 * vol
    assert np.all(ml2 > 0)


def test_lumped_mass_airplane_volume_is_box_minus_hole():
    m = mg.airplane_mesh(24, seed=4, sfc=True)
    ml = O.lumped_mass(O.OracleMesh.of(m))
    # hole volume by the divergence theorem over the innermost wall triangles
    tri = m.xyz[m.meta["inner_wall_faces"]]
    hole = abs(np.einsum("ij,ij->i", tri[:, 0], np.cross(tri[:, 1], tri[:, 2])).sum() / 6.0)
    assert hole > 1e-3
    assert abs(ml.sum() - (1.0 - hole)) < 1e-12


def test_tet_lumped_mass_is_quarter_volume():
    m = mg.single_element(O.TET04, seed=3)
    X = m.xyz[m.conn[O.TET04][0]]
    V = np.linalg.det(np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]])) / 6
    ml = O.lumped_mass(O.OracleMesh.of(m))
    assert np.allclose(ml[m.conn[O.TET04][0]], V / 4, rtol=1e-14)


def test_linear_pressure_identity(small_mixed):
    m = small_mixed
    rng = np.random.default_rng(4)
    gp = rng.standard_normal(3)
    p = 1.5 + m.xyz @ gp
    u = rng.standard_normal((m.n_nodes, 3))
    om = O.OracleMesh.of(m)
    R = O.assemble_rhs(om, u, p, nu=0.1, closure="none", mask=O.TERM_PRES)
    ml = O.lumped_mass(om)
    assert np.allclose(R, -ml[:, None] * gp[None, :], rtol=0, atol=1e-13 * np.abs(R).max())


def test_rotation_invariance(small_mixed):
    m = small_mixed
    rng = np.random.default_rng(5)
    q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    f = mg.random_field(m, seed=6, nu=0.02)
    om = O.OracleMesh.of(m)
    R, nut = O.assemble_rhs(om, f.u, f.p, f.nu, 0.07, "vreman", want_nut=True)
    omr = O.OracleMesh(m.xyz @ q.T, m.conn)
    Rr, nutr = O.assemble_rhs(omr, f.u @ q.T, f.p, f.nu, 0.07, "vreman", want_nut=True)
    err = np.linalg.norm(Rr - R @ q.T) / np.linalg.norm(R)
    assert err < 1e-13
    for t in nut:
        assert np.allclose(nutr[t], nut[t], rtol=1e-12, atol=1e-15)


def test_vreman_closed_forms():
    c, delta, gam = 0.07, 0.3, 1.7
    G = np.zeros((3, 3))
    G[0, 1] = gam                      # pure shear u = (gamma y, 0, 0)
    assert O.vreman(G, delta, c) == 0.0
    s = -0.8                            # axisymmetric strain diag(s, s, -2s)
    G = np.diag([s, s, -2 * s])
    assert math.isclose(O.vreman(G, delta, c), c * delta ** 2 * abs(s) * math.sqrt(1.5), rel_tol=1e-14)
    w = 2.3                             # solid rotation about z: u = w (-y, x, 0)
    G = np.array([[0, -w, 0], [w, 0, 0], [0, 0, 0]], float)
    assert math.isclose(O.vreman(G, delta, c), c * delta ** 2 * w / math.sqrt(2), rel_tol=1e-14)
    assert O.vreman(np.zeros((3, 3)), delta, c) == 0.0


def test_assembled_nut_uses_delta_cube_root_of_volume():
    # linear field: nu_t(element) = c Delta^2 |s| sqrt(3/2), Delta = V^(1/3)
    m = mg.tgv_mesh(4, sfc=False)
    s = 0.6
    u = m.xyz @ np.diag([s, s, -2 * s]).T
    om = O.OracleMesh.of(m)
    R, nut, vol = O.assemble_rhs(om, u, np.zeros(m.n_nodes), nu=0.0, c_vreman=0.07, closure="vreman",
                                 want_nut=True, want_vol=True)
    X = m.xyz[m.conn[O.TET04]]
    V = np.linalg.det(np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=1)) / 6
    assert np.allclose(vol[O.TET04], V, rtol=1e-14)
    expect = 0.07 * np.cbrt(V) ** 2 * s * math.sqrt(1.5)
    assert np.allclose(nut[O.TET04], expect[:, None], rtol=1e-13)


def test_sgs_term_is_nut_over_nu_times_viscous_for_linear_field(small_mixed):
    m = small_mixed
    rng = np.random.default_rng(8)
    for etype in ALL_TYPES:
        sub = mg.Mesh(xyz=m.xyz, conn={etype: m.conn[etype][:5]})
        om = O.OracleMesh.of(sub)
        B = rand_B(rng)
        u = m.xyz @ B.T
        p = np.zeros(m.n_nodes)
        for e in range(5):
            one = O.OracleMesh(m.xyz, {etype: m.conn[etype][e:e + 1]})
            Rs, nut = O.assemble_rhs(one, u, p, nu=0.0, c_vreman=0.07, closure="vreman", mask=O.TERM_SGS,
                                     want_nut=True)
            Rv = O.assemble_rhs(one, u, p, nu=1.0, closure="none", mask=O.TERM_VISC)
            nt = nut[etype][0]
            assert np.allclose(nt, nt[0], rtol=1e-12)
            assert np.allclose(Rs, nt[0] * Rv, rtol=1e-11, atol=1e-14)
        del om


# --------------------------------------------------------------------------
# tetrahedron closed forms

def tet_closed_form(X, U, P, nu, c_vreman, closure):
    E = np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]])
    V = np.linalg.det(E) / 6
    gr = np.linalg.inv(E).T                 # rows: grad of r, s, t
    dN = np.vstack([-gr.sum(axis=0), gr])   # (4, 3)
    G = U.T @ dN
    gp = dN.T @ P
    M = V / 20 * (np.ones((4, 4)) + np.eye(4))
    A = G + np.trace(G) * np.eye(3)
    eps = 0.5 * (G + G.T)
    nut = O.vreman(G, np.cbrt(V), c_vreman) if closure == "vreman" else 0.0
    R = -(M @ U) @ A.T - V / 4 * gp[None, :] - V * 2 * (nu + nut) * dN @ eps.T
    return R, M, nut


def test_tet_consistent_mass_closed_form():
    for seed in range(5):
        m = mg.single_element(O.TET04, seed=seed)
        X = m.xyz[m.conn[O.TET04][0]]
        V = np.linalg.det(np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]])) / 6
        Ae = O.element_mass(O.TET04, X)
        assert np.allclose(Ae, V / 20 * (np.ones((4, 4)) + np.eye(4)), rtol=1e-14, atol=0)


@pytest.mark.parametrize("closure", ["none", "vreman"])
def test_tet_element_residual_closed_form(closure):
    rng = np.random.default_rng(12)
    for seed in range(10):
        m = mg.single_element(O.TET04, seed=seed)
        c = m.conn[O.TET04][0]
        U = rng.standard_normal((4, 3))
        P = rng.standard_normal(4)
        u = np.zeros((4, 3))
        p = np.zeros(4)
        u[c] = U
        p[c] = P
        R = O.assemble_rhs(O.OracleMesh.of(m), u, p, nu=0.05, c_vreman=0.07, closure=closure)
        Rc, _, _ = tet_closed_form(m.xyz[c], U, P, 0.05, 0.07, closure)
        assert np.allclose(R[c], Rc, rtol=1e-13, atol=1e-14 * np.abs(Rc).max())


# --------------------------------------------------------------------------
# independent high-order evaluation on affinely mapped elements

def _leg01(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1), 0.5 * w


def high_order_rule(etype, n=6):
    """Collapsed tensor Gauss-Legendre rules (library nodes), exact for the
    polynomial integrands of affinely mapped linear elements."""
    a, wa = _leg01(n)
    s, ws = np.polynomial.legendre.leggauss(n)
    pts, w = [], []
    if etype == O.HEX08:
        for i in range(n):
            for j in range(n):
                for k in range(n):
                    pts.append((s[i], s[j], s[k]))
                    w.append(ws[i] * ws[j] * ws[k])
    elif etype == O.TET04:
        for i in range(n):
            for j in range(n):
                for k in range(n):
                    r = a[i]
                    q = a[j] * (1 - a[i])
                    t = a[k] * (1 - a[i]) * (1 - a[j])
                    pts.append((r, q, t))
                    w.append(wa[i] * wa[j] * wa[k] * (1 - a[i]) ** 2 * (1 - a[j]))
    elif etype == O.PEN06:
        for i in range(n):
            for j in range(n):
                for k in range(n):
                    pts.append((a[i], a[j] * (1 - a[i]), s[k]))
                    w.append(wa[i] * wa[j] * (1 - a[i]) * ws[k])
    elif etype == O.PYR05:
        for i in range(n):
            for j in range(n):
                for k in range(n):
                    t = a[k]
                    pts.append(((1 - t) * s[i], (1 - t) * s[j], t))
                    w.append(ws[i] * ws[j] * wa[k] * (1 - t) ** 2)
    return np.array(pts), np.array(w)


@pytest.mark.parametrize("etype", ALL_TYPES)
@pytest.mark.parametrize("linear_u", [False, True])
def test_element_residual_matches_high_order_evaluation(etype, linear_u):
    """On an affine prism the convective integrand N_a G u is cubic in the
    triangle coordinates, beyond the 3-point rule's degree 2: there the
    random-field case checks the viscous and pressure terms and the
    linear-field case (quadratic integrand) checks all terms."""
    rng = np.random.default_rng(20 + etype + 10 * linear_u)
    for trial in range(3):
        A = rng.standard_normal((3, 3)) + 2 * np.eye(3)
        if np.linalg.det(A) < 0:
            A[:, 0] *= -1
        X = REF_NODES[etype] @ A.T + rng.standard_normal(3)
        nen = X.shape[0]
        if linear_u:
            U = rng.standard_normal(3) + X @ rng.standard_normal((3, 3)).T
        else:
            U = rng.standard_normal((nen, 3))
        P = rng.standard_normal(nen)
        nu = 0.3
        conv = linear_u or etype != O.PEN06
        mask = O.TERM_ALL if conv else (O.TERM_VISC | O.TERM_PRES)
        conn = np.arange(nen, dtype=np.int32)[None]
        R = O.assemble_rhs(O.OracleMesh(X, {etype: conn}), U, P, nu=nu, closure="none", mask=mask)
        # independent evaluation: J = A (affine), grad N = A^-T grad_xi N
        pts, w = high_order_rule(etype)
        Ainv_T = np.linalg.inv(A).T
        detA = np.linalg.det(A)
        Rh = np.zeros((nen, 3))
        for xi, wg in zip(pts, w):
            N, dxi = O.shape(etype, xi)
            dN = dxi @ Ainv_T.T
            ug = N @ U
            G = U.T @ dN
            gp = dN.T @ P
            cvec = (G @ ug + np.trace(G) * ug) if conv else np.zeros(3)
            eps = 0.5 * (G + G.T)
            Rh -= wg * detA * (np.outer(N, cvec + gp) + 2 * nu * dN @ eps.T)
        assert np.allclose(R, Rh, rtol=1e-12, atol=1e-12 * np.abs(Rh).max())


def test_global_identity_linear_field_mixed_mesh(small_mixed):
    """sum_a R_a = -int (B + tr B I)(a + B x) dx - |Omega| grad p over the box."""
    m = small_mixed
    rng = np.random.default_rng(9)
    B = rand_B(rng)
    a = rng.standard_normal(3)
    gp = rng.standard_normal(3)
    u = a + m.xyz @ B.T
    p = m.xyz @ gp
    om = O.OracleMesh.of(m)
    R = O.assemble_rhs(om, u, p, nu=0.2, c_vreman=0.0, closure="none")
    lx, lz = 4 * math.pi, 2 * math.pi
    vol = lx * 2 * lz
    centre = np.array([lx / 2, 0.0, lz / 2])
    A = B + np.trace(B) * np.eye(3)
    expect = -vol * (A @ (a + B @ centre)) - vol * gp
    assert np.allclose(R.sum(axis=0), expect, rtol=1e-12, atol=1e-12 * np.abs(expect).max())


# --------------------------------------------------------------------------
# Taylor-Green vortex

def tgv_analytic_rhs(x, nu):
    X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
    rx = -np.sin(2 * X) * np.cos(2 * Z) / 8 - 3 * nu * np.sin(X) * np.cos(Y) * np.cos(Z)
    ry = -np.sin(2 * Y) * np.cos(2 * Z) / 8 + 3 * nu * np.cos(X) * np.sin(Y) * np.cos(Z)
    rz = (np.cos(2 * X) + np.cos(2 * Y)) * np.sin(2 * Z) / 8
    return np.stack([rx, ry, rz], axis=1)


def tgv_error(n, nu, mask=O.TERM_ALL):
    m = mg.tgv_mesh(n)
    f = mg.tgv_field(m, nu=nu)
    om = O.OracleMesh.of(m)
    R = O.periodic_fold(m.periodic_master, O.assemble_rhs(om, f.u, f.p, nu, 0.0, "none", mask=mask))
    ml = O.periodic_fold(m.periodic_master, O.lumped_mass(om))
    if mask == O.TERM_VISC:
        exact = -3 * nu * f.u
    else:
        exact = tgv_analytic_rhs(m.xyz[m.periodic_master], nu)
    approx = R / ml[:, None]
    return np.linalg.norm(approx - exact) / np.linalg.norm(exact)


def test_tgv_analytic_rhs_converges_second_order():
    nu = 1.0 / 1600.0
    # the sin 2x cos 2z terms have 8 nodes per wavelength at 16^3: rel-L2 0.187,
    # then 0.050 at 32^3 and 0.0128 at 64^3 (ratios 3.0, 3.7, 3.9 -> 4)
    e = [tgv_error(n, nu) for n in (8, 16, 32)]
    assert e[1] < 0.2
    assert e[0] / e[1] > 2.8 and e[1] / e[2] > 3.5, e


def test_tgv_viscous_term_converges_to_laplacian():
    e = [tgv_error(n, 1.0, mask=O.TERM_VISC) for n in (8, 16, 32)]
    assert e[0] / e[1] > 3.0 and e[1] / e[2] > 3.5, e
    assert e[2] < 0.01


# --------------------------------------------------------------------------

def test_openmp_variant_equals_serial(small_mixed):
    m = small_mixed
    f = mg.random_field(m, seed=4)
    om = O.OracleMesh.of(m)
    R = O.assemble_rhs(om, f.u, f.p, f.nu, 0.07)
    for nt in (1, 3, 0):
        R2 = O.assemble_rhs_omp(om, f.u, f.p, f.nu, 0.07, nthreads=nt)
        assert np.abs(R2 - R).max() <= 1e-13 * np.abs(R).max()


def test_periodic_fold():
    master = np.array([0, 1, 0, 3, 1], np.int32)
    v = np.array([[1.0, 2], [3, 4], [5, 6], [7, 8], [9, 10]])
    out = O.periodic_fold(master, v)
    expect = np.array([[6.0, 8], [12, 14], [6, 8], [7, 8], [12, 14]])
    assert np.array_equal(out, expect)


def test_bad_inputs_are_rejected():
    m = mg.single_element(O.TET04, seed=1)
    bad = m.conn[O.TET04][:, [0, 2, 1, 3]]    # inverted
    with pytest.raises(O.OracleError):
        O.assemble_rhs(O.OracleMesh(m.xyz, {O.TET04: bad}), np.zeros((4, 3)), np.zeros(4), 0.1)
    oob = m.conn[O.TET04].copy()
    oob[0, 0] = 7
    with pytest.raises(O.OracleError):
        O.assemble_rhs(O.OracleMesh(m.xyz, {O.TET04: oob}), np.zeros((4, 3)), np.zeros(4), 0.1)


def test_vreman_sum_of_squares_equals_printed_difference_form():
    """B_beta as the sum of principal 2x2 minors of beta (the printed form)
    equals the sum of squared cross products of the rows of G; both forms
    agree to round-off wherever B_beta is not near zero, and the oracle's
    sum-of-squares form stays non-negative where the printed form cancels."""
    rng = np.random.default_rng(31)
    c, delta = 0.07, 0.4
    for _ in range(200):
        G = rng.standard_normal((3, 3))
        al = G.T
        be = delta ** 2 * al.T @ al
        B = (be[0, 0] * be[1, 1] - be[0, 1] ** 2 + be[0, 0] * be[2, 2] - be[0, 2] ** 2
             + be[1, 1] * be[2, 2] - be[1, 2] ** 2)
        expect = c * math.sqrt(B / np.sum(al * al)) if B > 0 else 0.0
        assert math.isclose(O.vreman(G, delta, c), expect, rel_tol=1e-12)
    # nearly parallel rows: B_beta ~ 1e-20 relative, still >= 0 and tiny
    G = np.array([[1.0, 2.0, 3.0], [1.0, 2.0, 3.0 + 1e-10], [0, 0, 0]])
    v = O.vreman(G, delta, c)
    assert 0.0 <= v < 1e-9
