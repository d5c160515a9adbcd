"""The structured PEN06 Jacobian of the element kernels, restated in NumPy,
against exact rational arithmetic and against the oracle (section 2.3.3:
J = sum_a x_a (x) grad_xi N_a).

The kernels form the columns at twice their value from five edge
differences per component (e1 = X1 - X0, e2 = X2 - X0, h_k = X_{k+3} - X_k):
  r-column   (2 e1 + Dr) + zeta Dr,   Dr = h1 - h0  (= f1 - e1, the twist),
  s-column   (2 e2 + Ds) + zeta Ds,   Ds = h2 - h0,
  zeta-column Q at the rule's triangle point (1/6, 1/6), Q + Dr/2 at
  (2/3, 1/6), Q + Ds/2 at (1/6, 2/3), with Q = h0 + (Dr + Ds)/6;
then J^-1 = 2 A / det and W = (w / 8) det for the adjugate A and determinant
det of those columns.

* Exact reference: J, det J and the Cartesian derivatives evaluated in
  rational arithmetic from the same FP64 coordinates and rule points.  The
  edge-difference form stays within a few ulps of it on thin prisms far from
  the origin, where the plain sum over nodes (the oracle's definition)
  loses digits to cancellation: about 5e-13 / 6e-11 / 5e-9 relative at
  thicknesses 1e-2 / 1e-4 / 1e-6 at a distance of 50.
* Oracle: on distorted prisms of unit size both agree to 1e-12.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_2005_05899_b300 import meshgen as mg

TRI = [(1 / 6, 1 / 6), (2 / 3, 1 / 6), (1 / 6, 2 / 3)]


def kernel_form(X, q, zeta, w):
    """det J, W and J^-1 at triangle point q, level zeta."""
    e1, e2 = X[1] - X[0], X[2] - X[0]
    h0, h1, h2 = X[3] - X[0], X[4] - X[1], X[5] - X[2]
    Dr, Ds = h1 - h0, h2 - h0
    Ar, As = 2 * e1 + Dr, 2 * e2 + Ds
    Q = h0 + (Dr + Ds) / 6
    c0, c1 = Ar + zeta * Dr, As + zeta * Ds
    c2 = Q if q == 0 else Q + 0.5 * (Dr if q == 1 else Ds)
    A = np.stack([np.cross(c1, c2), np.cross(c2, c0), np.cross(c0, c1)])   # rows: adjugate of the columns
    d8 = c2 @ np.cross(c0, c1)
    return d8 / 8, (w / 8) * d8, 2 * A / d8


def exact_form(X, xi, w):
    """The same quantities from the definition, in rational arithmetic."""
    Xf = [[Fraction(v) for v in row] for row in X]
    r, s, z = (Fraction(v) for v in xi)
    L = [1 - r - s, r, s]
    dL = [(-1, -1), (1, 0), (0, 1)]
    dN = [[Fraction(dL[k][0]) * (1 - z) / 2, Fraction(dL[k][1]) * (1 - z) / 2, -L[k] / 2] for k in range(3)]
    dN += [[Fraction(dL[k][0]) * (1 + z) / 2, Fraction(dL[k][1]) * (1 + z) / 2, L[k] / 2] for k in range(3)]
    J = [[sum(Xf[a][i] * dN[a][j] for a in range(6)) for j in range(3)] for i in range(3)]
    cof = lambda i, j: (J[(i + 1) % 3][(j + 1) % 3] * J[(i + 2) % 3][(j + 2) % 3]
                        - J[(i + 1) % 3][(j + 2) % 3] * J[(i + 2) % 3][(j + 1) % 3])
    det = sum(J[0][j] * cof(0, j) for j in range(3))
    Jinv = [[cof(j, i) / det for j in range(3)] for i in range(3)]       # adjugate / det
    grad = np.array([[float(sum(dN[a][k] * Jinv[k][j] for k in range(3))) for j in range(3)] for a in range(6)])
    return grad, float(det), float(Fraction(w) * det)


def points():
    pts, w = O.quadrature(O.PEN06)
    assert pts.shape[0] == 6
    out = []
    for xi, wg in zip(pts, w):
        q = [k for k, t in enumerate(TRI) if np.allclose(xi[:2], t, atol=1e-14)]
        assert len(q) == 1
        out.append((q[0], xi, wg))
    return out


def check_against_exact(X, tol):
    for q, xi, wg in points():
        _, dNxi = O.shape(O.PEN06, xi)
        det_k, W_k, Jinv_k = kernel_form(X, q, xi[2], wg)
        grad_e, det_e, W_e = exact_form(X, xi, wg)
        grad_k = dNxi @ Jinv_k
        assert det_k == pytest.approx(det_e, rel=tol)
        assert W_k == pytest.approx(W_e, rel=tol)
        assert np.abs(grad_k - grad_e).max() <= tol * np.abs(grad_e).max()


@pytest.mark.parametrize("seed", range(4))
def test_distorted_prisms_exact_and_oracle(seed):
    m = mg.single_element(O.PEN06, seed=seed, distort=0.15)
    X = m.xyz[m.conn[O.PEN06][0]]
    check_against_exact(X, 1e-14)
    _, dNx, W, det = O.element_geometry(O.PEN06, X)
    for g, (q, xi, wg) in enumerate(points()):
        _, dNxi = O.shape(O.PEN06, xi)
        det_k, W_k, Jinv_k = kernel_form(X, q, xi[2], wg)
        assert det_k == pytest.approx(det[g], rel=1e-12)
        assert W_k == pytest.approx(W[g], rel=1e-12)
        assert np.abs(dNxi @ Jinv_k - dNx[g]).max() <= 1e-12 * np.abs(dNx[g]).max()


@pytest.mark.parametrize("thickness", [1e-2, 1e-4, 1e-6])
def test_thin_boundary_layer_prisms_exact(thickness):
    """Prisms of a stretched wall layer: a triangle of size ~1 at a distance
    of 50 from the origin, extruded by a small thickness along a slightly
    tilted normal."""
    rng = np.random.default_rng(int(round(-np.log10(thickness))))
    base = np.array([[0.0, 0.0, 0.0], [1.0, 0.1, 0.0], [0.2, 0.9, 0.0]]) + 50.0
    nrm = np.array([0.02, -0.01, 1.0])
    top = base + thickness * (nrm + 0.05 * rng.standard_normal((3, 3)))
    check_against_exact(np.concatenate([base, top]), 1e-14)
