"""FP64 CPU oracle of the momentum-RHS assembly: TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports, links or calls it, and shares no code with
it.  The C source ``fea_oracle.c`` states which passage of the paper (Borrell
et al. 2020, section 2.1 Eq. momentum, section 2.3.3 gather/compute/scatter
and the mass-matrix listing, Algorithm 1) each function follows.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests
(quadrature exactness, shape-function identities, patch test, uniform field,
lumped-mass volume, rotation invariance, linear-pressure identity, Vreman
closed forms, Taylor-Green analytic RHS with O(h^2) convergence, tetrahedron
closed-form integrals, NumPy brute force on single elements, finite-difference
MLP gradients, the wall law's limits and a flat plate's total force, the
projection's symmetry / null space / exact discrete integration by parts,
the balance iteration's fixed point and convergence, the model variants'
closed forms).  tests/golden/ holds regression fixtures of its results,
written by tests/golden/make_golden.py from this package alone.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Dict, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fea_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

TET04, PYR05, PEN06, HEX08 = 0, 1, 2, 3
NNODE = (4, 5, 6, 8)
NGAUSS = (4, 8, 6, 8)
TERM_CONV, TERM_VISC, TERM_SGS, TERM_PRES = 1, 2, 4, 8
TERM_ALL = 15
CLOSURE = {"none": 0, "vreman": 1, "mlp": 2}
MLP_IN, MLP_H = 6, 64


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain -O2, IEEE arithmetic, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-o", _LIB, _SRC, "-lm"]
        subprocess.check_call(cmd)
    return _LIB


class _Mesh(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("xyz", ctypes.POINTER(ctypes.c_double)),
                ("n_elem", ctypes.c_int64 * 4), ("conn", ctypes.POINTER(ctypes.c_int32) * 4)]


class _Mlp(ctypes.Structure):
    _fields_ = [(n, ctypes.POINTER(ctypes.c_double)) for n in
                ("w1", "b1", "w2", "b2", "w3", "b3", "w4", "b4", "feat_mean", "feat_std")] + \
               [("out_scale", ctypes.c_double)]


class _Params(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_double), ("c_vreman", ctypes.c_double), ("closure", ctypes.c_int),
                ("mask", ctypes.c_uint32), ("mlp", ctypes.POINTER(_Mlp)), ("conv_form", ctypes.c_int),
                ("delta_form", ctypes.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        _lib.orc_vreman.restype = ctypes.c_double
        _lib.orc_vreman_aniso.restype = ctypes.c_double
        _lib.orc_mlp_loss_grad.restype = ctypes.c_double
        _lib.orc_bad_element.restype = ctypes.c_int64
        _lib.orc_quadrature.argtypes = [ctypes.c_int, dp, dp]
        vp = ctypes.c_void_p
        _lib.orc_assemble_laplacian_coo.argtypes = [vp, vp, vp, dp]
        _lib.orc_assemble_divergence.argtypes = [vp, dp, dp]
        _lib.orc_assemble_gradient.argtypes = [vp, dp, dp]
        _lib.orc_shape.argtypes = [ctypes.c_int, dp, dp, dp]
        _lib.orc_reichardt.restype = ctypes.c_double
        _lib.orc_reichardt.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


class OracleError(RuntimeError):
    pass


class OracleMesh:
    """Keeps C-contiguous copies of a mesh alive for the C struct."""

    def __init__(self, xyz: np.ndarray, conn: Dict[int, np.ndarray]):
        self.xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        self.conn = {t: np.ascontiguousarray(c, dtype=np.int32) for t, c in conn.items()}
        self._empty = np.zeros((1,), np.int32)
        s = _Mesh()
        s.n_nodes = self.xyz.shape[0]
        s.xyz = _dp(self.xyz)
        for t in range(4):
            c = self.conn.get(t)
            if c is None or c.shape[0] == 0:
                s.n_elem[t] = 0
                s.conn[t] = _ip(self._empty)
            else:
                assert c.shape[1] == NNODE[t]
                s.n_elem[t] = c.shape[0]
                s.conn[t] = _ip(c)
        self.struct = s

    @classmethod
    def of(cls, mesh) -> "OracleMesh":
        return cls(mesh.xyz, mesh.conn)

    @property
    def n_nodes(self) -> int:
        return self.xyz.shape[0]


class MLPParams:
    """FP64 MLP weights (6 -> 64 -> 64 -> 64 -> 1) and input normalisation."""

    def __init__(self, theta: np.ndarray, feat_mean, feat_std, out_scale: float):
        self.theta = np.ascontiguousarray(theta, dtype=np.float64)
        assert self.theta.size == nparam()
        self.feat_mean = np.ascontiguousarray(feat_mean, dtype=np.float64)
        self.feat_std = np.ascontiguousarray(feat_std, dtype=np.float64)
        self.out_scale = float(out_scale)
        off = 0
        parts = {}
        for name, size in (("w1", MLP_H * MLP_IN), ("b1", MLP_H), ("w2", MLP_H * MLP_H), ("b2", MLP_H),
                           ("w3", MLP_H * MLP_H), ("b3", MLP_H), ("w4", MLP_H), ("b4", 1)):
            parts[name] = self.theta[off:off + size]
            off += size
        self.parts = parts
        s = _Mlp()
        base = self.theta.ctypes.data
        off = 0
        for name, size in (("w1", MLP_H * MLP_IN), ("b1", MLP_H), ("w2", MLP_H * MLP_H), ("b2", MLP_H),
                           ("w3", MLP_H * MLP_H), ("b3", MLP_H), ("w4", MLP_H), ("b4", 1)):
            setattr(s, name, ctypes.cast(base + 8 * off, ctypes.POINTER(ctypes.c_double)))
            off += size
        s.feat_mean = _dp(self.feat_mean)
        s.feat_std = _dp(self.feat_std)
        s.out_scale = self.out_scale
        self.struct = s


def nparam() -> int:
    return int(lib().orc_mlp_nparam())


def _params(nu, c_vreman, closure, mask, mlp: Optional[MLPParams], conv_form: int = 0, delta_form: int = 0):
    prm = _Params()
    prm.conv_form = int(conv_form)
    prm.delta_form = int(delta_form)
    prm.nu = float(nu)
    prm.c_vreman = float(c_vreman)
    prm.closure = CLOSURE[closure] if isinstance(closure, str) else int(closure)
    prm.mask = int(mask)
    prm.mlp = ctypes.pointer(mlp.struct) if mlp is not None else ctypes.POINTER(_Mlp)()
    return prm


def _check(status: int, what: str):
    if status != 0:
        t = ctypes.c_int(-1)
        e = lib().orc_bad_element(ctypes.byref(t))
        raise OracleError(f"{what}: status {status} (element {e} of type {t.value})")


def quadrature(etype: int):
    pts = np.zeros((8, 3))
    w = np.zeros(8)
    n = lib().orc_quadrature(etype, _dp(pts), _dp(w))
    return pts[:n].copy(), w[:n].copy()


def shape(etype: int, xi):
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    N = np.zeros(8)
    dN = np.zeros((8, 3))
    n = lib().orc_shape(etype, _dp(xi), _dp(N), _dp(dN))
    return N[:n].copy(), dN[:n].copy()


def element_geometry(etype: int, X: np.ndarray):
    """Per Gauss point: N (ng, nen), dN/dx (ng, nen, 3), W (ng,), det J (ng,)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    ng, nen = NGAUSS[etype], NNODE[etype]
    N = np.zeros((ng, nen))
    d = np.zeros((ng, nen, 3))
    W = np.zeros(ng)
    det = np.zeros(ng)
    st = lib().orc_element_geometry(ctypes.c_int(etype), _dp(X), _dp(N), _dp(d), _dp(W), _dp(det))
    if st != 0:
        raise OracleError(f"element_geometry status {st}; det J = {det}")
    return N, d, W, det


def element_mass(etype: int, X: np.ndarray) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.float64)
    nen = NNODE[etype]
    Ae = np.zeros((nen, nen))
    _check(lib().orc_element_mass(ctypes.c_int(etype), _dp(X), _dp(Ae)), "element_mass")
    return Ae


def vreman_aniso(G: np.ndarray, dm, c: float) -> float:
    G = np.ascontiguousarray(G, dtype=np.float64).reshape(9)
    d = np.ascontiguousarray(dm, dtype=np.float64)
    return float(lib().orc_vreman_aniso(_dp(G), _dp(d), ctypes.c_double(c)))


def vreman(G: np.ndarray, delta: float, c: float) -> float:
    G = np.ascontiguousarray(G, dtype=np.float64).reshape(9)
    return float(lib().orc_vreman(_dp(G), ctypes.c_double(delta), ctypes.c_double(c)))


def mlp_features(G: np.ndarray, delta: float, nu: float) -> np.ndarray:
    """The closure's six dimensionless inputs of one velocity gradient G (3x3),
    filter width delta and viscosity nu (see orc_mlp_features)."""
    G = np.ascontiguousarray(G, dtype=np.float64).reshape(9)
    x = np.zeros(6)
    lib().orc_mlp_features(_dp(G), ctypes.c_double(delta), ctypes.c_double(nu), _dp(x))
    return x


def mlp_forward(mlp: MLPParams, x: np.ndarray) -> np.ndarray:
    """nu_t for raw (un-normalised) feature rows x (B, 6)."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, MLP_IN)
    y = np.zeros(x.shape[0])
    lib().orc_mlp_forward(ctypes.byref(mlp.struct), _dp(x), ctypes.c_int64(x.shape[0]), _dp(y))
    return y


def mlp_loss_grad(theta: np.ndarray, x: np.ndarray, y: np.ndarray, want_grad: bool = True):
    """MSE loss of softplus(z) against y on normalised inputs x, and its gradient."""
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, MLP_IN)
    y = np.ascontiguousarray(y, dtype=np.float64)
    g = np.zeros(nparam()) if want_grad else None
    loss = lib().orc_mlp_loss_grad(_dp(theta), _dp(x), _dp(y), ctypes.c_int64(x.shape[0]),
                                   _dp(g) if g is not None else ctypes.POINTER(ctypes.c_double)())
    return float(loss), g


def adam_step(theta, grad, m1, m2, lr, beta1, beta2, eps, t):
    lib().orc_adam_step(_dp(theta), _dp(np.ascontiguousarray(grad, dtype=np.float64)), _dp(m1), _dp(m2),
                        ctypes.c_int64(theta.size), ctypes.c_double(lr), ctypes.c_double(beta1),
                        ctypes.c_double(beta2), ctypes.c_double(eps), ctypes.c_int64(t))


def assemble_rhs(om: OracleMesh, u: np.ndarray, p: np.ndarray, nu: float, c_vreman: float = 0.07,
                 closure="vreman", mask: int = TERM_ALL, mlp: Optional[MLPParams] = None,
                 want_nut: bool = False, want_vol: bool = False, conv_form: int = 0, delta_form: int = 0):
    """Serial FP64 assembly in natural element order.  Returns rhs (N, 3) and,
    on request, nu_t per type (E_t, ng) and element volumes per type (E_t,).
    conv_form 1: EMAC convective form; delta_form 1: per-direction Vreman widths."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    p = np.ascontiguousarray(p, dtype=np.float64)
    assert u.shape == (om.n_nodes, 3) and p.shape == (om.n_nodes,)
    rhs = np.zeros((om.n_nodes, 3))
    prm = _params(nu, c_vreman, closure, mask, mlp, conv_form, delta_form)
    nut = {t: np.zeros((c.shape[0], NGAUSS[t])) for t, c in om.conn.items()} if want_nut else {}
    vol = {t: np.zeros(c.shape[0]) for t, c in om.conn.items()} if want_vol else {}
    nut_arr = (ctypes.POINTER(ctypes.c_double) * 4)()
    vol_arr = (ctypes.POINTER(ctypes.c_double) * 4)()
    for t in range(4):
        if t in nut and nut[t].size:
            nut_arr[t] = _dp(nut[t])
        if t in vol and vol[t].size:
            vol_arr[t] = _dp(vol[t])
    st = lib().orc_assemble_rhs(ctypes.byref(om.struct), _dp(u), _dp(p), ctypes.byref(prm), _dp(rhs),
                                nut_arr if want_nut else None, vol_arr if want_vol else None)
    _check(st, "assemble_rhs")
    out = [rhs]
    if want_nut:
        out.append(nut)
    if want_vol:
        out.append(vol)
    return out[0] if len(out) == 1 else tuple(out)


def assemble_rhs_omp(om: OracleMesh, u, p, nu, c_vreman=0.07, closure="vreman", mask=TERM_ALL,
                     mlp: Optional[MLPParams] = None, nthreads: int = 0) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float64)
    p = np.ascontiguousarray(p, dtype=np.float64)
    rhs = np.zeros((om.n_nodes, 3))
    prm = _params(nu, c_vreman, closure, mask, mlp)
    st = lib().orc_assemble_rhs_omp(ctypes.byref(om.struct), _dp(u), _dp(p), ctypes.byref(prm), _dp(rhs),
                                    ctypes.c_int(nthreads))
    _check(st, "assemble_rhs_omp")
    return rhs


def max_threads() -> int:
    return int(lib().orc_max_threads())


def lumped_mass(om: OracleMesh) -> np.ndarray:
    m = np.zeros(om.n_nodes)
    _check(lib().orc_lumped_mass(ctypes.byref(om.struct), _dp(m)), "lumped_mass")
    return m


# ---- pressure projection (Algorithm 1: Laplacian, pressure equation, velocity
# correction; the reading of the step is documented with project()) ----------

def assemble_laplacian(om: OracleMesh):
    """K_ab = sum_e sum_g W_g grad N_a . grad N_b as a SciPy CSR matrix."""
    import scipy.sparse as sp
    nnz = sum(om.conn[t].shape[0] * NNODE[t] ** 2 for t in om.conn)
    rows = np.zeros(nnz, np.int64)
    cols = np.zeros(nnz, np.int64)
    vals = np.zeros(nnz)
    _check(lib().orc_assemble_laplacian_coo(ctypes.byref(om.struct), rows.ctypes.data_as(ctypes.c_void_p),
                                            cols.ctypes.data_as(ctypes.c_void_p), _dp(vals)), "laplacian")
    n = om.n_nodes
    return sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()


def divergence(om: OracleMesh, u: np.ndarray) -> np.ndarray:
    """B_a(u) = sum_e sum_g W_g N_a (div u)_g for u (N, 3)."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(om.n_nodes)
    _check(lib().orc_assemble_divergence(ctypes.byref(om.struct), _dp(u), _dp(out)), "divergence")
    return out


def gradient(om: OracleMesh, p: np.ndarray) -> np.ndarray:
    """G_a(p) = sum_e sum_g W_g N_a (grad p)_g, (N, 3)."""
    p = np.ascontiguousarray(p, dtype=np.float64)
    out = np.zeros((om.n_nodes, 3))
    _check(lib().orc_assemble_gradient(ctypes.byref(om.struct), _dp(p), _dp(out)), "gradient")
    return out


def fold_matrix(master: np.ndarray):
    """P (N x n_classes): P[i, class(i)] = 1, classes numbered by first master;
    returns (P, class index per node, the master node of each class)."""
    import scipy.sparse as sp
    masters, cls = np.unique(np.asarray(master, dtype=np.int64), return_inverse=True)
    n = cls.size
    return sp.csr_matrix((np.ones(n), (np.arange(n), cls)), shape=(n, masters.size)), cls, masters


def project(om: OracleMesh, master, vel_dirichlet, pinned, mass_folded, u_star, p, dt):
    """Incremental pressure projection after the Runge-Kutta stages (reading of
    Algorithm 1; the scheme's details are in a reference absent here):
      K dp = -(1/dt) B(u*)      on the periodic classes, dp = 0 at pinned nodes,
      u = u* - dt M_L^-1 G(dp)  (G folded; velocity-Dirichlet nodes keep u*),
      p = p + dp.
    Solved directly (SciPy sparse LU).  Returns (u, p, dp)."""
    import scipy.sparse.linalg as spla
    P, cls, _ = fold_matrix(master)
    K = (P.T @ assemble_laplacian(om) @ P).tocsr()
    b = P.T @ (-(1.0 / dt) * divergence(om, u_star))
    keep = np.ones(K.shape[0], bool)
    keep[np.unique(cls[np.asarray(pinned, dtype=np.int64)])] = False
    dpc = np.zeros(K.shape[0])
    dpc[keep] = spla.spsolve(K[keep][:, keep].tocsc(), b[keep])
    dp = dpc[cls]
    g = periodic_fold(master, gradient(om, dp))
    u = np.array(u_star, dtype=np.float64, copy=True)
    free = ~np.asarray(vel_dirichlet, dtype=bool)
    u[free] -= dt * g[free] / np.asarray(mass_folded)[free, None]
    return u, np.asarray(p, dtype=np.float64) + dp, dp


# ---- correction coefficients of the partition (the load-balancing section) ----

def balance_update(Lambda_hist, times_hist) -> np.ndarray:
    """New correction coefficients lambda [P] from the observations k of the
    cumulative coefficients Lambda^k [P+1] (Lambda_0 = 0, Lambda_P = P) and
    of the per-part times t^k [P], following the section's steps:
      t_bar^k = mean of t^k;  T_i^k = t_1 + ... + t_i;  Upsilon_i^k = T_i^k / t_bar^k;
      for every splitting point i: weighted linear regression y = alpha + beta x
      of the points (Lambda_i^k, Upsilon_i^k), weights 1.5^k, together with the
      origin (weight 1: no work takes no time); Lambda_i^new = (i - alpha)/beta;
      lambda_i = Lambda_i^new - Lambda_(i-1)^new.
    Readings: the section's normalisation sum(lambda) = 1 contradicts its
    Lambda_P = P and Gamma_i = lambda_i W / P; sum(lambda) = P is taken, and
    t_bar is the mean time.  Splitting points are kept ordered in [0, P]."""
    L = np.asarray(Lambda_hist, dtype=np.float64)
    T = np.asarray(times_hist, dtype=np.float64)
    K, P = T.shape
    new = np.zeros(P + 1)
    new[P] = P
    for i in range(1, P):
        x = [0.0] + [L[k, i] for k in range(K)]
        y = [0.0] + [T[k, :i].sum() / T[k].mean() for k in range(K)]
        w = np.array([1.0] + [1.5 ** k for k in range(K)])
        beta, alpha = np.polyfit(np.array(x), np.array(y), 1, w=np.sqrt(w))   # polyfit weighs the residuals
        new[i] = (i - alpha) / beta
    for i in range(1, P):
        new[i] = min(max(new[i], new[i - 1]), P)
    return np.diff(new)


def periodic_fold(master: np.ndarray, v: np.ndarray) -> np.ndarray:
    v = np.ascontiguousarray(v, dtype=np.float64).copy()
    ncomp = 1 if v.ndim == 1 else v.shape[1]
    master = np.ascontiguousarray(master, dtype=np.int32)
    lib().orc_periodic_fold(ctypes.c_int64(v.shape[0]), _ip(master), _dp(v), ctypes.c_int(ncomp))
    return v


def rk_stage(om: OracleMesh, master, dirichlet, mass_folded, un, uk, p, nu, c_vreman, closure, stage, dt,
             mask=TERM_ALL, mlp=None, wall=None) -> np.ndarray:
    """One SSP-RK3 stage; wall (optional) = wall-model faces (see wall_rhs), whose
    boundary term at u^(k) joins the element RHS (Algorithm 1)."""
    un = np.ascontiguousarray(un, dtype=np.float64)
    uk = np.ascontiguousarray(uk, dtype=np.float64)
    p = np.ascontiguousarray(p, dtype=np.float64)
    mass_folded = np.ascontiguousarray(mass_folded, dtype=np.float64)
    out = np.zeros_like(un)
    mp = _ip(np.ascontiguousarray(master, dtype=np.int32)) if master is not None else None
    dmask = None
    if dirichlet is not None:
        dmask = np.ascontiguousarray(dirichlet, dtype=np.uint8)
    prm = _params(nu, c_vreman, closure, mask, mlp)
    extra = None
    if wall is not None:
        extra = wall_rhs(om, uk, nu, **wall)
    st = lib().orc_rk_stage(ctypes.byref(om.struct), mp,
                            dmask.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)) if dmask is not None else None,
                            _dp(mass_folded), _dp(un), _dp(uk), _dp(p), ctypes.byref(prm), ctypes.c_int(stage),
                            ctypes.c_double(dt), _dp(extra) if extra is not None else None, _dp(out))
    _check(st, "rk_stage")
    return out


def rk3_step(om: OracleMesh, master, dirichlet, un, p, nu, c_vreman, closure, dt, mask=TERM_ALL, mlp=None,
             wall=None):
    """Three SSP-RK3 stages from u^n; returns u^(n+1)."""
    mass = lumped_mass(om)
    if master is not None:
        mass = periodic_fold(master, mass)
    uk = un
    for s in range(3):
        uk = rk_stage(om, master, dirichlet, mass, un, uk, p, nu, c_vreman, closure, s, dt, mask, mlp, wall)
    return uk


# ---- equilibrium wall model (the boundary assembly of Algorithm 1; the law of
# the wall and the sampling are readings, documented in fea_oracle.c) ---------

WALL_KAPPA, WALL_C = 0.41, 7.8


def reichardt(yp: float, kappa: float = WALL_KAPPA, c: float = WALL_C):
    """(f(y+), f'(y+)) of Reichardt's law of the wall."""
    d = ctypes.c_double(0.0)
    f = lib().orc_reichardt(ctypes.c_double(yp), ctypes.c_double(kappa), ctypes.c_double(c), ctypes.byref(d))
    return f, d.value


def wall_utau(U: float, y: float, nu: float, kappa: float = WALL_KAPPA, c: float = WALL_C):
    """(u_tau, Newton steps) with U = u_tau f(y u_tau / nu)."""
    v = ctypes.c_double(0.0)
    it = ctypes.c_int(0)
    st = lib().orc_wall_utau(ctypes.c_double(U), ctypes.c_double(y), ctypes.c_double(nu), ctypes.c_double(kappa),
                             ctypes.c_double(c), ctypes.byref(v), ctypes.byref(it))
    _check(st, "wall_utau")
    return v.value, it.value


def wall_rhs(om: OracleMesh, u: np.ndarray, nu: float, tri=None, tri_exch=None, quad=None, quad_exch=None,
             kappa: float = WALL_KAPPA, c: float = WALL_C) -> np.ndarray:
    """Wall-model boundary term (N, 3) of triangular and quadrilateral wall
    faces: tri / tri_exch (F, 3) and quad / quad_exch (F, 4) node ids, face
    nodes ordered so that x_xi x x_eta points out of the fluid."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    rhs = np.zeros((om.n_nodes, 3))
    for nv, f, x in ((3, tri, tri_exch), (4, quad, quad_exch)):
        if f is None or len(f) == 0:
            continue
        f = np.ascontiguousarray(f, dtype=np.int32)
        x = np.ascontiguousarray(x, dtype=np.int32)
        assert f.shape == x.shape and f.shape[1] == nv
        st = lib().orc_wall_rhs(ctypes.c_int64(om.n_nodes), _dp(om.xyz), _dp(u), ctypes.c_int(nv),
                                ctypes.c_int64(f.shape[0]), _ip(f), _ip(x), ctypes.c_double(nu),
                                ctypes.c_double(kappa), ctypes.c_double(c), _dp(rhs))
        _check(st, "wall_rhs")
    return rhs
