"""Pins of the oracle's model variants (the EMAC convective form and a
Vreman filter width per direction).

* Anisotropic Vreman: with equal widths h it equals the isotropic model with
  Delta = h (B_beta scales as h^4); with only two nonzero gradient columns
  c_m, c_n it is c Delta_m Delta_n |c_m x c_n| / |G| (Cauchy-Binet); the
  assembled nu_t of a stretched box element uses the box's edge lengths.
* EMAC: zero for a uniform field; the element residual of the EMAC
  convective form equals an independent high-order evaluation of
  -int N_a [(G + G^T + tr G) u - 1/2 grad (|u|^2)_h] on affinely mapped
  elements of every type, for a linear velocity field (where every rule is
  exact for the integrand).
"""
import numpy as np
import pytest

import oracle as O
from paper_2005_05899_b300 import meshgen as mg
from test_oracle_assembly_pins import ALL_TYPES, REF_NODES, high_order_rule


def test_aniso_vreman_equal_widths_is_isotropic():
    rng = np.random.default_rng(1)
    for _ in range(20):
        G = rng.standard_normal((3, 3))
        h = rng.uniform(0.01, 2.0)
        assert O.vreman_aniso(G, [h, h, h], 0.07) == pytest.approx(O.vreman(G, h, 0.07), rel=1e-13)


def test_aniso_vreman_two_columns_closed_form():
    rng = np.random.default_rng(2)
    for m, n in ((0, 1), (0, 2), (1, 2)):
        G = np.zeros((3, 3))
        G[:, m] = rng.standard_normal(3)
        G[:, n] = rng.standard_normal(3)
        d = rng.uniform(0.1, 3.0, 3)
        ref = 0.07 * d[m] * d[n] * np.linalg.norm(np.cross(G[:, m], G[:, n])) / np.linalg.norm(G)
        assert O.vreman_aniso(G, d, 0.07) == pytest.approx(ref, rel=1e-13)


def test_assembled_aniso_nut_uses_box_extents():
    hx, hy, hz = 0.8, 0.05, 0.3
    X = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0], [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]],
                 dtype=float) * [hx, hy, hz]
    B = np.array([[0.3, 1.2, -0.4], [0.5, -0.2, 0.9], [-1.1, 0.4, 0.2]])
    U = X @ B.T
    conn = np.arange(8, dtype=np.int32)[None]
    _, nut = O.assemble_rhs(O.OracleMesh(X, {O.HEX08: conn}), U, np.zeros(8), 1e-3, 0.07, "vreman", want_nut=True,
                            delta_form=1)
    ref = O.vreman_aniso(B, [hx, hy, hz], 0.07)
    assert np.allclose(nut[O.HEX08], ref, rtol=1e-13)
    _, nut_iso = O.assemble_rhs(O.OracleMesh(X, {O.HEX08: conn}), U, np.zeros(8), 1e-3, 0.07, "vreman",
                                want_nut=True)
    assert not np.allclose(nut_iso[O.HEX08], ref, rtol=1e-3)


def test_emac_uniform_field_gives_zero_convection():
    m = mg.channel_mesh(nx=6, ny=8, nz=4, seed=3, n_layers=2, split_frac=0.3)
    u = np.tile([0.7, -1.2, 0.4], (m.n_nodes, 1))
    r = O.assemble_rhs(O.OracleMesh.of(m), u, np.zeros(m.n_nodes), 1e-3, 0.07, "none", mask=O.TERM_CONV,
                       conv_form=1)
    assert np.abs(r).max() <= 1e-13


@pytest.mark.parametrize("etype", ALL_TYPES)
def test_emac_element_residual_matches_high_order_evaluation(etype):
    rng = np.random.default_rng(40 + etype)
    for _ in range(3):
        A = rng.standard_normal((3, 3)) + 2 * np.eye(3)
        if np.linalg.det(A) < 0:
            A[:, 0] *= -1
        X = REF_NODES[etype] @ A.T + rng.standard_normal(3)
        nen = X.shape[0]
        U = rng.standard_normal(3) + X @ rng.standard_normal((3, 3)).T
        conn = np.arange(nen, dtype=np.int32)[None]
        R = O.assemble_rhs(O.OracleMesh(X, {etype: conn}), U, np.zeros(nen), nu=0.0, closure="none",
                           mask=O.TERM_CONV, conv_form=1)
        pts, w = high_order_rule(etype)
        Ainv_T = np.linalg.inv(A).T
        detA = np.linalg.det(A)
        q = np.sum(U * U, axis=1)
        Rh = np.zeros((nen, 3))
        for xi, wg in zip(pts, w):
            N, dxi = O.shape(etype, xi)
            dN = dxi @ Ainv_T.T
            ug = N @ U
            G = U.T @ dN
            k = dN.T @ q
            c = G @ ug + G.T @ ug + np.trace(G) * ug - 0.5 * k
            Rh -= wg * detA * np.outer(N, c)
        assert np.allclose(R, Rh, rtol=1e-12, atol=1e-12 * np.abs(Rh).max()), etype
