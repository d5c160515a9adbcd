"""Pins of the oracle's reference elements: quadrature rules and shape functions.

Each rule is checked against exact integrals of monomials over the reference
element (closed forms, not the rule's own formula), and the pyramid's axial
rule against SciPy's Gauss-Jacobi routine.  Shape functions are checked for
the Kronecker property, partition of unity, linear completeness and against
central finite differences of themselves.
"""
import math

import numpy as np
import pytest
from scipy.special import roots_jacobi

import oracle as O

REF_NODES = {
    O.TET04: np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float),
    O.PYR05: np.array([[-1, -1, 0], [1, -1, 0], [1, 1, 0], [-1, 1, 0], [0, 0, 1]], float),
    O.PEN06: np.array([[0, 0, -1], [1, 0, -1], [0, 1, -1], [0, 0, 1], [1, 0, 1], [0, 1, 1]], float),
    O.HEX08: np.array([[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1],
                       [-1, -1, 1], [1, -1, 1], [1, 1, 1], [-1, 1, 1]], float),
}
VOLUME = {O.TET04: 1 / 6, O.PYR05: 4 / 3, O.PEN06: 1.0, O.HEX08: 8.0}
f = math.factorial


def leg(k):  # int_{-1}^{1} x^k dx
    return 0.0 if k % 2 else 2.0 / (k + 1)


def exact_monomial(etype, a, b, c):
    """Exact integral of r^a s^b t^c over the reference element."""
    if etype == O.TET04:
        return f(a) * f(b) * f(c) / f(a + b + c + 3)
    if etype == O.PEN06:
        return f(a) * f(b) / f(a + b + 2) * leg(c)
    if etype == O.HEX08:
        return leg(a) * leg(b) * leg(c)
    if etype == O.PYR05:
        # xi = (1-t) x, eta = (1-t) y, zeta = t, Jacobian (1-t)^2
        m = a + b + 2
        return leg(a) * leg(b) * f(c) * f(m) / f(c + m + 1)
    raise ValueError


def exact_cases(etype):
    out = []
    for a in range(4):
        for b in range(4):
            for c in range(4):
                if etype == O.TET04 and a + b + c <= 2:
                    out.append((a, b, c))
                elif etype == O.PEN06 and a + b <= 2 and c <= 3:
                    out.append((a, b, c))
                elif etype == O.HEX08:
                    out.append((a, b, c))
                elif etype == O.PYR05 and a + b + c <= 3:
                    out.append((a, b, c))
    return out


@pytest.mark.parametrize("etype", [O.TET04, O.PYR05, O.PEN06, O.HEX08])
def test_weights_sum_to_reference_volume(etype):
    _, w = O.quadrature(etype)
    assert len(w) == O.NGAUSS[etype]
    assert abs(w.sum() - VOLUME[etype]) < 1e-15


@pytest.mark.parametrize("etype", [O.TET04, O.PYR05, O.PEN06, O.HEX08])
def test_quadrature_exact_for_monomials(etype):
    pts, w = O.quadrature(etype)
    for a, b, c in exact_cases(etype):
        q = np.sum(w * pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c)
        assert abs(q - exact_monomial(etype, a, b, c)) < 1e-14, (a, b, c)


def test_tet_rule_not_exact_beyond_degree_2():
    # the 4-point rule is degree 2 exactly: a cubic monomial must miss
    pts, w = O.quadrature(O.TET04)
    q = np.sum(w * pts[:, 0] ** 3)
    assert abs(q - exact_monomial(O.TET04, 3, 0, 0)) > 1e-6


def test_pyramid_axial_rule_matches_gauss_jacobi():
    # Gauss-Jacobi(alpha=2, beta=0) on [-1,1] mapped to t = (1+x)/2
    x, wj = roots_jacobi(2, 2.0, 0.0)
    t_ref = np.sort((1 + x) / 2)
    w_ref = (wj / 8.0)[np.argsort((1 + x) / 2)]
    pts, w = O.quadrature(O.PYR05)
    t = np.unique(np.round(pts[:, 2], 14))
    assert np.allclose(t, t_ref, atol=1e-14)
    for tk, wk in zip(t_ref, w_ref):
        sel = np.abs(pts[:, 2] - tk) < 1e-12
        assert abs(w[sel].sum() - 4.0 * wk) < 1e-14


@pytest.mark.parametrize("etype", [O.TET04, O.PYR05, O.PEN06, O.HEX08])
def test_shape_kronecker_and_partition(etype):
    nodes = REF_NODES[etype]
    for a, xi in enumerate(nodes):
        if etype == O.PYR05 and a == 4:
            xi = np.array([0, 0, 1 - 1e-9])
        N, _ = O.shape(etype, xi)
        e = np.zeros(len(nodes))
        e[a] = 1
        assert np.allclose(N, e, atol=1e-8)
    rng = np.random.default_rng(0)
    for _ in range(50):
        xi = random_point(etype, rng)
        N, dN = O.shape(etype, xi)
        assert abs(N.sum() - 1) < 1e-14
        assert np.abs(dN.sum(axis=0)).max() < 1e-14
        # linear completeness: sum_a N_a xi_a = xi
        assert np.allclose(N @ nodes, xi, atol=1e-14)


def random_point(etype, rng):
    while True:
        if etype == O.TET04:
            p = rng.uniform(0, 1, 3)
            if p.sum() < 1:
                return p
        elif etype == O.PEN06:
            p = rng.uniform(0, 1, 2)
            if p.sum() < 1:
                return np.array([p[0], p[1], rng.uniform(-1, 1)])
        elif etype == O.HEX08:
            return rng.uniform(-1, 1, 3)
        else:
            t = rng.uniform(0, 0.95)
            return np.array([(1 - t) * rng.uniform(-1, 1), (1 - t) * rng.uniform(-1, 1), t])


@pytest.mark.parametrize("etype", [O.TET04, O.PYR05, O.PEN06, O.HEX08])
def test_shape_derivatives_match_finite_differences(etype):
    rng = np.random.default_rng(1)
    h = 1e-6
    for _ in range(20):
        xi = random_point(etype, rng)
        _, dN = O.shape(etype, xi)
        for j in range(3):
            e = np.zeros(3)
            e[j] = h
            Np, _ = O.shape(etype, xi + e)
            Nm, _ = O.shape(etype, xi - e)
            assert np.allclose((Np - Nm) / (2 * h), dN[:, j], atol=1e-8)


def test_pyramid_triangle_faces_are_linear():
    # on the face eta = -(1 - zeta) only nodes 0, 1, 4 are non-zero and the
    # trace is linear: conformity with tetrahedra across triangular faces
    rng = np.random.default_rng(2)
    for _ in range(20):
        z = rng.uniform(0, 0.9)
        x = rng.uniform(-(1 - z), 1 - z)
        N, _ = O.shape(O.PYR05, [x, -(1 - z), z])
        assert abs(N[2]) < 1e-14 and abs(N[3]) < 1e-14
        assert abs(N[0] - 0.5 * (1 - z - x)) < 1e-14
        assert abs(N[1] - 0.5 * (1 - z + x)) < 1e-14
