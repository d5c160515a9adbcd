"""Seeded synthetic meshes and fields for the momentum-RHS assembly.

This module only builds inputs: node coordinates, element connectivity per
element type, periodic master maps, Dirichlet masks, the per-element flag of
stretched boundary-layer prisms, and nodal velocity / pressure fields.  It
holds none of the finite-element arithmetic (no shape functions, no
quadrature, no Jacobians); the only geometry it evaluates is the sign of a
corner triple product, used to orient each element positively.  Both the FP64
oracle and the CUDA path consume what it produces.

Local node order per type follows the VTK convention:
  TET04  r=0,s=0,t=0 corner first, then the r, s and t vertices.
  PYR05  base quad (-1,-1),(1,-1),(1,1),(-1,1) at zeta=0, apex at zeta=1.
  PEN06  bottom triangle (zeta=-1), then the top triangle (zeta=+1).
  HEX08  bottom face counter-clockwise, then the top face.

The workloads mirror the paper's (section 2.2: linear hybrid meshes of
tetrahedra, prisms and pyramids with a boundary layer, 2M-32M elements per
node in section 5) with seeded stand-ins, because the JSM airplane meshes are
not available:
  tgv_mesh        16^3 periodic cube, Kuhn 6-tet split (Taylor-Green vortex).
  channel_mesh    stretched channel, prism wall layers, pyramid/tet splits.
  airplane_mesh   jittered tet grid with a carved ellipsoid and a prism layer.
  batch_meshes    many channel-like meshes of log-uniform size.
"""
from __future__ import annotations

import dataclasses
import itertools
import math
from typing import Dict, List, Optional

import numpy as np

TET04, PYR05, PEN06, HEX08 = 0, 1, 2, 3
ETYPES = (TET04, PYR05, PEN06, HEX08)
ETYPE_NAMES = ("TET04", "PYR05", "PEN06", "HEX08")
NODES_PER_ELEM = (4, 5, 6, 8)


@dataclasses.dataclass
class Mesh:
    """An unstructured mixed mesh, node arrays in the order given here."""

    xyz: np.ndarray                      # (N, 3) float64
    conn: Dict[int, np.ndarray]          # etype -> (E_t, n_en) int32
    periodic_master: Optional[np.ndarray] = None   # (N,) int32, master id or self
    dirichlet: Optional[np.ndarray] = None          # (N,) uint8
    fp64_flag: Dict[int, np.ndarray] = dataclasses.field(default_factory=dict)
    name: str = ""
    meta: dict = dataclasses.field(default_factory=dict)
    # wall-model faces: {"tri": (F,3), "tri_exch": (F,3)[, "quad", "quad_exch"]}
    # node ids, each face ordered so that its normal points out of the fluid
    wall_faces: Optional[Dict[str, np.ndarray]] = None

    @property
    def n_nodes(self) -> int:
        return int(self.xyz.shape[0])

    def n_elem(self, etype: int) -> int:
        c = self.conn.get(etype)
        return 0 if c is None else int(c.shape[0])

    @property
    def n_elem_total(self) -> int:
        return sum(self.n_elem(t) for t in ETYPES)

    def counts(self) -> dict:
        return {ETYPE_NAMES[t]: self.n_elem(t) for t in ETYPES}


@dataclasses.dataclass
class Field:
    """Nodal velocity (N, 3) and pressure (N,), float64."""

    u: np.ndarray
    p: np.ndarray
    nu: float
    c_vreman: float = 0.07


# --------------------------------------------------------------------------
# helpers

def _corner(dx: int, dy: int, dz: int) -> int:
    return dx + 2 * dy + 4 * dz


def _perm_parity(p) -> int:
    p = list(p)
    s = 1
    for i in range(len(p)):
        for j in range(i + 1, len(p)):
            if p[i] > p[j]:
                s = -s
    return s


def kuhn_local() -> np.ndarray:
    """(6, 4) corner indices (dx + 2dy + 4dz) of the Kuhn split of a cube.

    Every tetrahedron runs from corner 000 to corner 111 along one
    permutation of the axes, so neighbouring cubes split their shared faces
    along the same diagonal and the mesh is conforming (and periodic).
    """
    tets = []
    for perm in itertools.permutations((0, 1, 2)):
        v = [0, 0, 0]
        verts = [_corner(*v)]
        for ax in perm:
            v[ax] = 1
            verts.append(_corner(*v))
        if _perm_parity(perm) < 0:
            verts[1], verts[2] = verts[2], verts[1]
        tets.append(verts)
    return np.array(tets, dtype=np.int64)


HEX_LOCAL = np.array([_corner(0, 0, 0), _corner(1, 0, 0), _corner(1, 1, 0), _corner(0, 1, 0),
                      _corner(0, 0, 1), _corner(1, 0, 1), _corner(1, 1, 1), _corner(0, 1, 1)],
                     dtype=np.int64)


def _triple(a, b, c):
    return (a[:, 0] * (b[:, 1] * c[:, 2] - b[:, 2] * c[:, 1])
            - a[:, 1] * (b[:, 0] * c[:, 2] - b[:, 2] * c[:, 0])
            + a[:, 2] * (b[:, 0] * c[:, 1] - b[:, 1] * c[:, 0]))


def orientation(etype: int, conn: np.ndarray, xyz: np.ndarray) -> np.ndarray:
    """Sign-carrying corner triple product per element (positive = VTK-positive)."""
    x = xyz[conn]
    if etype == TET04:
        return _triple(x[:, 1] - x[:, 0], x[:, 2] - x[:, 0], x[:, 3] - x[:, 0])
    if etype == PYR05:
        centre = x[:, :4].mean(axis=1)
        a = 0.5 * ((x[:, 1] - x[:, 0]) + (x[:, 2] - x[:, 3]))
        b = 0.5 * ((x[:, 3] - x[:, 0]) + (x[:, 2] - x[:, 1]))
        return _triple(a, b, x[:, 4] - centre)
    if etype == PEN06:
        bot = x[:, :3].mean(axis=1)
        top = x[:, 3:].mean(axis=1)
        return _triple(x[:, 1] - x[:, 0], x[:, 2] - x[:, 0], top - bot)
    if etype == HEX08:
        a = 0.25 * ((x[:, 1] - x[:, 0]) + (x[:, 2] - x[:, 3]) + (x[:, 5] - x[:, 4]) + (x[:, 6] - x[:, 7]))
        b = 0.25 * ((x[:, 3] - x[:, 0]) + (x[:, 2] - x[:, 1]) + (x[:, 7] - x[:, 4]) + (x[:, 6] - x[:, 5]))
        c = 0.25 * ((x[:, 4] - x[:, 0]) + (x[:, 5] - x[:, 1]) + (x[:, 6] - x[:, 2]) + (x[:, 7] - x[:, 3]))
        return _triple(a, b, c)
    raise ValueError(etype)


_FLIP = {TET04: [0, 2, 1, 3], PYR05: [0, 3, 2, 1, 4], PEN06: [0, 2, 1, 3, 5, 4],
         HEX08: [0, 3, 2, 1, 4, 7, 6, 5]}


def orient_positive(etype: int, conn: np.ndarray, xyz: np.ndarray) -> np.ndarray:
    """Reorder the local nodes of negatively oriented elements (mirror flip)."""
    s = orientation(etype, conn, xyz)
    neg = s < 0
    if np.any(neg):
        conn = conn.copy()
        conn[neg] = conn[neg][:, _FLIP[etype]]
    return conn


def prism_wall_faces(mesh: Mesh) -> Dict[str, np.ndarray]:
    """Wall-model faces of a prism boundary layer: the triangle of every PEN06
    whose three nodes are wall (Dirichlet) nodes, with the opposite triangle's
    nodes as exchange nodes; faces are reordered so that their normal
    (x1 - x0) x (x2 - x0) points away from the exchange nodes (out of the
    fluid)."""
    pen = mesh.conn.get(PEN06)
    if pen is None or mesh.dirichlet is None:
        return {"tri": np.zeros((0, 3), np.int32), "tri_exch": np.zeros((0, 3), np.int32)}
    w = mesh.dirichlet.astype(bool)
    bot, top = w[pen[:, :3]].all(axis=1), w[pen[:, 3:]].all(axis=1)
    face = np.concatenate([pen[bot, :3], pen[top, 3:]]).astype(np.int32)
    exch = np.concatenate([pen[bot, 3:], pen[top, :3]]).astype(np.int32)
    X = mesh.xyz
    nrm = np.cross(X[face[:, 1]] - X[face[:, 0]], X[face[:, 2]] - X[face[:, 0]])
    into_fluid = np.einsum("ij,ij->i", nrm, X[exch].mean(axis=1) - X[face].mean(axis=1)) > 0
    face[into_fluid] = face[into_fluid][:, [0, 2, 1]]
    exch[into_fluid] = exch[into_fluid][:, [0, 2, 1]]
    return {"tri": face, "tri_exch": exch}


def morton_codes(xyz: np.ndarray, bits: int = 21) -> np.ndarray:
    """63-bit Morton (Z-order) keys of points quantised in their bounding box."""
    lo = xyz.min(axis=0)
    span = np.maximum(xyz.max(axis=0) - lo, 1e-300)
    q = np.floor((xyz - lo) / span * ((1 << bits) - 1)).astype(np.uint64)

    def split3(v):
        v = v & np.uint64(0x1FFFFF)
        v = (v | (v << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
        v = (v | (v << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
        v = (v | (v << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
        v = (v | (v << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
        v = (v | (v << np.uint64(2))) & np.uint64(0x1249249249249249)
        return v

    return split3(q[:, 0]) | (split3(q[:, 1]) << np.uint64(1)) | (split3(q[:, 2]) << np.uint64(2))


def renumber_nodes(mesh: Mesh, perm: np.ndarray) -> Mesh:
    """New node n is old node perm[n]; every node array and index is remapped."""
    perm = np.asarray(perm, dtype=np.int64)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(perm.size, dtype=np.int64)
    conn = {t: inv[c].astype(np.int32) for t, c in mesh.conn.items()}
    master = None
    if mesh.periodic_master is not None:
        master = inv[mesh.periodic_master[perm]].astype(np.int32)
    dirichlet = None if mesh.dirichlet is None else mesh.dirichlet[perm].copy()
    wall = None if mesh.wall_faces is None else {k: inv[v].astype(np.int32) for k, v in mesh.wall_faces.items()}
    out = dataclasses.replace(mesh, xyz=mesh.xyz[perm].copy(), conn=conn,
                              periodic_master=master, dirichlet=dirichlet,
                              meta=dict(mesh.meta), wall_faces=wall)
    out.meta["node_perm"] = perm
    return out


def sfc_sort_nodes(mesh: Mesh) -> Mesh:
    """Renumber nodes along a Morton curve (gather locality for every element)."""
    perm = np.argsort(morton_codes(mesh.xyz), kind="stable")
    return renumber_nodes(mesh, perm)


def _grid_ids(nx, ny, nz):
    return lambda i, j, k: i + (nx + 1) * (j + (ny + 1) * k)


def _cells(nx, ny, nz):
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return i.ravel(), j.ravel(), k.ravel()


def _cell_corners(i, j, k, nid):
    """(n_cells, 8) node ids of cell corners, corner index dx + 2dy + 4dz."""
    cols = []
    for c in range(8):
        dx, dy, dz = c & 1, (c >> 1) & 1, (c >> 2) & 1
        cols.append(nid(i + dx, j + dy, k + dz))
    return np.stack(cols, axis=1).astype(np.int64)


# --------------------------------------------------------------------------
# Taylor-Green vortex cube

def tgv_mesh(n: int = 16, sfc: bool = True) -> Mesh:
    """(2 pi)^3 periodic cube of n^3 cubes, each split into 6 TET04.

    (n+1)^3 geometric nodes are stored (4,913 for n=16); the nodes on the
    planes x, y or z = 2 pi are periodic slaves of the opposite planes.
    """
    L = 2.0 * math.pi
    nid = _grid_ids(n, n, n)
    g = np.arange(n + 1)
    kk, jj, ii = np.meshgrid(g, g, g, indexing="ij")
    ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()
    h = L / n
    xyz = np.stack([ii * h, jj * h, kk * h], axis=1).astype(np.float64)
    master = nid(ii % n, jj % n, kk % n).astype(np.int32)
    ci, cj, ck = _cells(n, n, n)
    corners = _cell_corners(ci, cj, ck, nid)
    tets = corners[:, kuhn_local()].reshape(-1, 4)
    tets = orient_positive(TET04, tets, xyz).astype(np.int32)
    mesh = Mesh(xyz=xyz, conn={TET04: tets}, periodic_master=master,
                dirichlet=np.zeros(xyz.shape[0], np.uint8), name=f"tgv{n}",
                meta={"n": n, "L": L})
    return sfc_sort_nodes(mesh) if sfc else mesh


def tgv_field(mesh: Mesh, nu: float = 1.0 / 1600.0, c_vreman: float = 0.07) -> Field:
    """Taylor-Green initial field, evaluated at each node's periodic master."""
    src = mesh.xyz if mesh.periodic_master is None else mesh.xyz[mesh.periodic_master]
    x, y, z = src[:, 0], src[:, 1], src[:, 2]
    u = np.stack([np.sin(x) * np.cos(y) * np.cos(z),
                  -np.cos(x) * np.sin(y) * np.cos(z),
                  np.zeros_like(x)], axis=1)
    p = (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0) / 16.0
    return Field(u=u, p=p, nu=nu, c_vreman=c_vreman)


# --------------------------------------------------------------------------
# channel with prism wall layers and pyramid / tet splits

def _stretched_y(ny: int, ratio: float) -> np.ndarray:
    half = ny // 2
    h1 = (ratio - 1.0) / (ratio ** half - 1.0) if ratio != 1.0 else 1.0 / half
    dy = h1 * ratio ** np.arange(half)
    yb = -1.0 + np.concatenate([[0.0], np.cumsum(dy)])
    yb[-1] = 0.0
    return np.concatenate([yb, -yb[-2::-1]])


# faces of a cube: 4 corners (dx + 2dy + 4dz), ordered around the face
_FACE_YM = [_corner(0, 0, 0), _corner(1, 0, 0), _corner(1, 0, 1), _corner(0, 0, 1)]
_FACE_YP = [_corner(0, 1, 0), _corner(1, 1, 0), _corner(1, 1, 1), _corner(0, 1, 1)]
_FACE_XM = [_corner(0, 0, 0), _corner(0, 1, 0), _corner(0, 1, 1), _corner(0, 0, 1)]
_FACE_XP = [_corner(1, 0, 0), _corner(1, 1, 0), _corner(1, 1, 1), _corner(1, 0, 1)]
_FACE_ZM = [_corner(0, 0, 0), _corner(1, 0, 0), _corner(1, 1, 0), _corner(0, 1, 0)]
_FACE_ZP = [_corner(0, 0, 1), _corner(1, 0, 1), _corner(1, 1, 1), _corner(0, 1, 1)]


def channel_mesh(nx: int = 128, ny: int = 64, nz: int = 64, seed: int = 2,
                 n_layers: int = 8, ratio: float = 1.08, split_frac: float = 0.10,
                 jitter: float = 0.15, lx: float = 4 * math.pi, lz: float = 2 * math.pi,
                 sfc: bool = True) -> Mesh:
    """Channel box lx x 2 x lz of nx x ny x nz hexahedral cells (y wall-normal).

    * y is geometrically stretched from each wall (ratio per cell).
    * The n_layers wall-adjacent cell layers on each side become 2 PEN06 each
      (prism axis wall-normal, one fixed wall-parallel diagonal).
    * The first hex layer above each prism stack (transition cells) and a
      seeded split_frac of the remaining interior cells get a centroid node;
      each of their six faces becomes one PYR05 on its quad, or two TET04
      (same diagonal as the prisms) on the face that borders a prism layer.
      The mesh is conforming.
    * Nodes are jittered by U(-jitter, jitter) x local spacing per axis,
      except normal to the walls and to the periodic planes, so the domain
      stays the exact box (volume lx * 2 * lz).
    * Periodic in x and z: nodes on x = lx or z = lz are slaves of x = 0 / z = 0.
    """
    assert ny % 2 == 0 and 2 * n_layers + 2 <= ny
    rng = np.random.default_rng(seed)
    nid = _grid_ids(nx, ny, nz)
    gx = np.linspace(0.0, lx, nx + 1)
    gy = _stretched_y(ny, ratio)
    gz = np.linspace(0.0, lz, nz + 1)
    gk, gj, gi = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    gi, gj, gk = gi.ravel(), gj.ravel(), gk.ravel()
    n_grid = gi.size
    xyz = np.stack([gx[gi], gy[gj], gz[gk]], axis=1)
    master = nid(gi % nx, gj, gk % nz).astype(np.int64)

    # jitter: drawn for every node, then masters' values copied to slaves
    hx = lx / nx
    hz = lz / nz
    dyc = np.diff(gy)
    hy = np.minimum(np.concatenate([[np.inf], dyc]), np.concatenate([dyc, [np.inf]]))
    jit = rng.uniform(-jitter, jitter, size=(n_grid, 3))
    jit[:, 0] *= hx
    jit[:, 1] *= hy[gj]
    jit[:, 2] *= hz
    jit[(gi == 0) | (gi == nx), 0] = 0.0
    jit[(gj == 0) | (gj == ny), 1] = 0.0
    jit[(gk == 0) | (gk == nz), 2] = 0.0
    jit = jit[master]
    xyz = xyz + jit

    ci, cj, ck = _cells(nx, ny, nz)
    corners = _cell_corners(ci, cj, ck, nid)
    n_cells = ci.size
    is_prism = (cj < n_layers) | (cj >= ny - n_layers)
    trans_lo = cj == n_layers
    trans_hi = cj == ny - n_layers - 1
    interior = ~is_prism & ~trans_lo & ~trans_hi
    n_pick = int(round(split_frac * int(interior.sum())))
    pick = rng.choice(np.flatnonzero(interior), size=n_pick, replace=False)
    is_split = trans_lo | trans_hi
    is_split[pick] = True
    is_hex = ~is_prism & ~is_split

    conn: Dict[int, List[np.ndarray]] = {t: [] for t in ETYPES}
    # hexes
    conn[HEX08].append(corners[is_hex][:, HEX_LOCAL])
    # prisms: triangles (a,b,c) and (a,c,d) of the x-z quad, extruded in y
    pc = corners[is_prism]
    a0, b0, c0, d0 = (pc[:, _corner(0, 0, 0)], pc[:, _corner(1, 0, 0)],
                      pc[:, _corner(1, 0, 1)], pc[:, _corner(0, 0, 1)])
    a1, b1, c1, d1 = (pc[:, _corner(0, 1, 0)], pc[:, _corner(1, 1, 0)],
                      pc[:, _corner(1, 1, 1)], pc[:, _corner(0, 1, 1)])
    conn[PEN06].append(np.stack([a0, b0, c0, a1, b1, c1], axis=1))
    conn[PEN06].append(np.stack([a0, c0, d0, a1, c1, d1], axis=1))
    # split cells: centroid node
    sc = corners[is_split]
    n_split = sc.shape[0]
    cent_ids = n_grid + np.arange(n_split)
    cent_xyz = xyz[sc].mean(axis=1)
    s_lo = trans_lo[is_split]
    s_hi = trans_hi[is_split]
    for face, tri_mask in ((_FACE_YM, s_lo), (_FACE_YP, s_hi), (_FACE_XM, None), (_FACE_XP, None),
                           (_FACE_ZM, None), (_FACE_ZP, None)):
        f = sc[:, face]
        pyr_mask = np.ones(n_split, bool) if tri_mask is None else ~tri_mask
        conn[PYR05].append(np.concatenate([f[pyr_mask], cent_ids[pyr_mask, None]], axis=1))
        if tri_mask is not None and np.any(tri_mask):
            ft = f[tri_mask]
            ct = cent_ids[tri_mask, None]
            # same diagonal as the prisms: corner a=(0,.,0) to c=(1,.,1)
            conn[TET04].append(np.concatenate([ft[:, [0, 1, 2]], ct], axis=1))
            conn[TET04].append(np.concatenate([ft[:, [0, 2, 3]], ct], axis=1))

    xyz = np.concatenate([xyz, cent_xyz], axis=0)
    master = np.concatenate([master, cent_ids]).astype(np.int32)
    dirichlet = np.zeros(xyz.shape[0], np.uint8)
    dirichlet[:n_grid][(gj == 0) | (gj == ny)] = 1

    out_conn = {}
    for t in ETYPES:
        if conn[t]:
            c = np.concatenate(conn[t], axis=0)
            if c.shape[0]:
                out_conn[t] = orient_positive(t, c, xyz).astype(np.int32)
    flags = {}
    if PEN06 in out_conn:
        flags[PEN06] = np.ones(out_conn[PEN06].shape[0], np.uint8)
    mesh = Mesh(xyz=xyz, conn=out_conn, periodic_master=master, dirichlet=dirichlet,
                fp64_flag=flags, name=f"channel{nx}x{ny}x{nz}",
                meta={"nx": nx, "ny": ny, "nz": nz, "seed": seed, "n_layers": n_layers,
                      "ratio": ratio, "split_frac": split_frac, "jitter": jitter,
                      "volume": lx * 2.0 * lz, "first_cell": float(gy[1] - gy[0])})
    mesh.wall_faces = prism_wall_faces(mesh)
    return sfc_sort_nodes(mesh) if sfc else mesh


def channel_field(mesh: Mesh, seed: int = 3, noise: float = 0.05,
                  nu: float = 1.0 / 5600.0, c_vreman: float = 0.07) -> Field:
    """Laminar parabola u_x = 1 - y^2 plus seeded N(0,1) noise x amplitude.

    Wall (Dirichlet) nodes are held at zero; periodic slaves copy masters.
    Pressure: seeded N(0,1) x amplitude.
    """
    rng = np.random.default_rng(seed)
    n = mesh.n_nodes
    y = mesh.xyz[:, 1]
    u = noise * rng.standard_normal((n, 3))
    u[:, 0] += 1.0 - y * y
    p = noise * rng.standard_normal(n)
    if mesh.dirichlet is not None:
        u[mesh.dirichlet.astype(bool)] = 0.0
    if mesh.periodic_master is not None:
        u = u[mesh.periodic_master]
        p = p[mesh.periodic_master]
    return Field(u=u, p=p, nu=nu, c_vreman=c_vreman)


def channel_dims_for(target_elems: float, aspect=(2.0, 1.0, 1.0)) -> tuple:
    """Channel cell counts whose mixed mesh has about target_elems elements.

    The config-style split yields about 1.8 elements per cell.
    """
    cells = target_elems / 1.8
    base = (cells / (aspect[0] * aspect[1] * aspect[2])) ** (1.0 / 3.0)
    ny = max(8, 2 * int(round(base * aspect[1] / 2.0)))
    nx = max(2, int(round(base * aspect[0])))
    nz = max(2, int(round(cells / (nx * ny))))
    return nx, ny, nz


# --------------------------------------------------------------------------
# airplane-like: jittered tet grid, carved ellipsoid, prism boundary layer

def _random_rotation(rng) -> np.ndarray:
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def prism_corner_products(conn: np.ndarray, xyz: np.ndarray) -> np.ndarray:
    """(E, 6) triple products at the corners of PEN06 elements: two triangle
    edges and the vertical edge at each corner (positive = valid corner)."""
    x = xyz[conn]
    out = []
    for (a, b, c), (top, bot) in (((0, 1, 2), (3, 0)), ((1, 2, 0), (4, 1)), ((2, 0, 1), (5, 2)),
                                  ((3, 4, 5), (3, 0)), ((4, 5, 3), (4, 1)), ((5, 3, 4), (5, 2))):
        out.append(_triple(x[:, b] - x[:, a], x[:, c] - x[:, a], x[:, top] - x[:, bot]))
    return np.stack(out, axis=1)


def airplane_mesh(n_nodes_axis: int = 170, seed: int = 4, n_bl: int = 5, bl_ratio: float = 1.2,
                  bl_thickness: float = 0.5,
                  jitter: float = 0.15, sfc: bool = True) -> Mesh:
    """Tet-dominant mesh of [0,1]^3 with a prism boundary layer on an ellipsoid.

    * An n^3-node grid is jittered by U(-jitter, jitter) x h per axis (not
      normal to the box faces) and every cube is split into 6 TET04.
    * A seeded ellipsoid (semi-axes U[0.10, 0.25], seeded rotation) at the
      centre is carved: cubes (all six tets) whose centroid lies inside are
      removed, so the wall is made of cube faces and is locally monotone.
    * The exposed staircase wall is extruded inward by n_bl PEN06 layers of
      geometric growth bl_ratio, along averaged
      wall normals (total thickness bl_thickness cells); these prisms carry
      the FP64-Jacobian flag.
    * Dirichlet nodes: the box faces and the innermost wall layer.
    """
    rng = np.random.default_rng(seed)
    n = n_nodes_axis - 1
    h = 1.0 / n
    nid = _grid_ids(n, n, n)
    g = np.arange(n + 1)
    coords = g * h
    # nodes
    kk, jj, ii = np.meshgrid(g, g, g, indexing="ij")
    ii, jj, kk = ii.ravel().astype(np.int32), jj.ravel().astype(np.int32), kk.ravel().astype(np.int32)
    xyz = np.stack([coords[ii], coords[jj], coords[kk]], axis=1)
    jit = rng.uniform(-jitter * h, jitter * h, size=xyz.shape)
    for ax, idx in enumerate((ii, jj, kk)):
        jit[(idx == 0) | (idx == n), ax] = 0.0
    xyz += jit
    del jit
    # ellipsoid
    semi = rng.uniform(0.10, 0.25, size=3)
    rot = _random_rotation(rng)
    centre = np.array([0.5, 0.5, 0.5])

    def inside(p):
        q = (p - centre) @ rot / semi
        return np.einsum("ij,ij->i", q, q) < 1.0

    # cells near the ellipsoid: only those can be carved
    r = semi.max() + 2 * h
    lo_c = max(0, int(math.floor((0.5 - r) / h)))
    hi_c = min(n, int(math.ceil((0.5 + r) / h)))
    kl = kuhn_local()
    # all tets, in cell order (cell index c = i + n*(j + n*k)), 6 per cell
    ci, cj, ck = _cells(n, n, n)
    corners = _cell_corners(ci, cj, ck, nid).astype(np.int32)
    del ci, cj, ck
    tets = corners[:, kl].reshape(-1, 4)
    del corners
    keep = np.ones(tets.shape[0], bool)
    # candidate tets in the bounding region
    rc = np.arange(lo_c, hi_c)
    k3, j3, i3 = np.meshgrid(rc, rc, rc, indexing="ij")
    cand_cells = (i3 + n * (j3 + n * k3)).ravel()
    cand = (cand_cells[:, None] * 6 + np.arange(6)[None, :]).ravel()
    ci3, cj3, ck3 = i3.ravel(), j3.ravel(), k3.ravel()
    cube_cent = xyz[_cell_corners(ci3, cj3, ck3, nid)].mean(axis=1)
    removed_cells = cand_cells[inside(cube_cent)]
    removed = (removed_cells[:, None] * 6 + np.arange(6)[None, :]).ravel()
    keep[removed] = False
    # wall faces: faces of kept tets whose opposite tet is removed
    faces_local = np.array([[1, 2, 3], [0, 3, 2], [0, 1, 3], [0, 2, 1]])  # outward for a positive tet

    def face_keys(f):
        s = np.sort(f, axis=1).astype(np.int64)
        return (s[:, 0] * (n + 1) ** 3 + s[:, 1]) * (n + 1) ** 3 + s[:, 2]

    near_kept = cand[keep[cand]]
    kf = tets[near_kept][:, faces_local].reshape(-1, 3)        # outward faces of kept tets
    rf = tets[removed][:, faces_local].reshape(-1, 3)
    kkeys = face_keys(kf)
    rkeys = np.unique(face_keys(rf))
    wall_mask = np.isin(kkeys, rkeys)
    wall = kf[wall_mask]              # outward from the fluid = pointing into the hole
    # extrusion direction per wall node, pointing into the hole: start from
    # the mean of the incident unit face normals, then push each direction
    # toward its least-aligned incident face until every face sees all of its
    # nodes' directions at a clear positive angle (staircase corners)
    xw = xyz[wall]
    fn = np.cross(xw[:, 1] - xw[:, 0], xw[:, 2] - xw[:, 0])
    fn /= np.linalg.norm(fn, axis=1, keepdims=True)
    wnodes, winv = np.unique(wall.ravel(), return_inverse=True)
    fv = winv.reshape(-1, 3)
    nrm = np.zeros((wnodes.size, 3))
    np.add.at(nrm, winv, np.repeat(fn, 3, axis=0))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    best, best_min = nrm.copy(), -np.inf
    fn3 = np.repeat(fn[:, None, :], 3, axis=1)
    for _ in range(40):
        dots = np.einsum("fk,fvk->fv", fn, nrm[fv])
        mn = np.full(wnodes.size, np.inf)
        np.minimum.at(mn, fv.ravel(), dots.ravel())
        if mn.min() > best_min:
            best, best_min = nrm.copy(), mn.min()
        worst = dots <= mn[fv] + 1e-12
        push = np.zeros_like(nrm)
        np.add.at(push, fv[worst], fn3[worst])
        nrm = nrm + 0.1 * push
        nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    nrm = best
    # layers: cumulative offsets of geometric growth; the total thickness
    # starts at bl_thickness cells and is halved until every prism has
    # positive corner triple products (its Jacobian sign at the six corners)
    n_grid = xyz.shape[0]
    layer_id = lambda l: (np.arange(wnodes.size) + n_grid + (l - 1) * wnodes.size) if l > 0 else wnodes
    wl = winv.reshape(-1, 3)
    grown = bl_thickness
    for _attempt in range(6):
        thick = bl_ratio ** np.arange(n_bl)
        thick = thick / thick.sum() * (grown * h)
        offs = np.concatenate([[0.0], np.cumsum(thick)])
        layer_xyz = [xyz[wnodes] + offs[l][None] * nrm for l in range(1, n_bl + 1)]
        new_xyz = np.concatenate(layer_xyz, axis=0)
        prisms = np.concatenate([np.concatenate([layer_id(l)[wl], layer_id(l + 1)[wl]], axis=1)
                                 for l in range(n_bl)], axis=0)
        if prism_corner_products(prisms, np.concatenate([xyz, new_xyz], axis=0)).min() > 0:
            break
        grown *= 0.5
    bl_total = grown * h
    xyz = np.concatenate([xyz, new_xyz], axis=0)
    tets = tets[keep]
    # drop grid nodes used by no element (inside the hole)
    used = np.zeros(xyz.shape[0], bool)
    used[tets.ravel()] = True
    used[prisms.ravel()] = True
    dirichlet = np.zeros(xyz.shape[0], np.uint8)
    box = np.zeros(n_grid, bool)
    for idx in (ii, jj, kk):
        box |= (idx == 0) | (idx == n)
    dirichlet[:n_grid][box] = 1
    dirichlet[layer_id(n_bl)] = 1
    remap = np.cumsum(used) - 1
    xyz = xyz[used]
    dirichlet = dirichlet[used]
    tets = remap[tets].astype(np.int32)
    prisms = remap[prisms].astype(np.int64)
    prisms = orient_positive(PEN06, prisms, xyz).astype(np.int32)
    tets = orient_positive(TET04, tets, xyz).astype(np.int32)
    wall_nodes = np.sort(remap[layer_id(n_bl)]).astype(np.int64)   # innermost layer = no-slip wall
    inner_faces = prisms[-wall.shape[0]:, 3:].copy()     # innermost layer: top triangles
    mesh = Mesh(xyz=xyz, conn={TET04: tets, PEN06: prisms}, periodic_master=None,
                dirichlet=dirichlet, fp64_flag={PEN06: np.ones(prisms.shape[0], np.uint8)},
                name=f"airplane{n_nodes_axis}",
                meta={"n_nodes_axis": n_nodes_axis, "seed": seed, "semi_axes": semi.tolist(),
                      "rotation": rot.tolist(), "n_bl": n_bl, "bl_ratio": bl_ratio,
                      "n_wall_faces": int(wall.shape[0]), "h": h, "bl_total": bl_total,
                      "wall_nodes": wall_nodes, "inner_wall_faces": inner_faces})
    mesh.wall_faces = prism_wall_faces(mesh)
    if sfc:
        mesh = sfc_sort_nodes(mesh)
        inv = np.empty_like(mesh.meta["node_perm"])
        inv[mesh.meta["node_perm"]] = np.arange(inv.size)
        mesh.meta["wall_nodes"] = np.sort(inv[wall_nodes]).astype(np.int64)
        mesh.meta["inner_wall_faces"] = inv[inner_faces].astype(np.int32)
    return mesh


def inflow_field(mesh: Mesh, seed: int = 5, noise: float = 0.02, nu: float = 1.0 / 1.93e6,
                 p_noise: float = 0.02, c_vreman: float = 0.07) -> Field:
    """Uniform inflow (1,0,0) plus seeded isotropic N(0,1) x noise; wall held at 0.

    Pressure: seeded N(0,1) x p_noise.  The innermost boundary-layer surface
    (no-slip wall) is set to zero velocity; the box faces keep the inflow.
    """
    rng = np.random.default_rng(seed)
    n = mesh.n_nodes
    u = noise * rng.standard_normal((n, 3))
    u[:, 0] += 1.0
    p = p_noise * rng.standard_normal(n)
    wall = mesh.meta.get("wall_nodes")
    if wall is not None:
        u[wall] = 0.0
    return Field(u=u, p=p, nu=nu, c_vreman=c_vreman)


# --------------------------------------------------------------------------
# batch of uneven mixed meshes

def batch_meshes(count: int = 64, seed: int = 7, e_min: float = 1e4, e_max: float = 5e5):
    """count channel-like mixed meshes of log-uniform size, each with its own field and nu."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(math.log(e_min), math.log(e_max), size=count))
    out = []
    for b, target in enumerate(sizes):
        nx, ny, nz = channel_dims_for(target)
        n_layers = max(1, ny // 8)
        m = channel_mesh(nx=nx, ny=ny, nz=nz, seed=int(rng.integers(1 << 30)), n_layers=n_layers)
        nu = float(np.exp(rng.uniform(math.log(1 / 5000), math.log(1 / 500))))
        f = channel_field(m, seed=int(rng.integers(1 << 30)), nu=nu)
        out.append((m, f))
    return out


# --------------------------------------------------------------------------
# single elements (tiny brute-force cases)

REFERENCE_NODES = {
    TET04: np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float),
    PYR05: np.array([[-1, -1, 0], [1, -1, 0], [1, 1, 0], [-1, 1, 0], [0, 0, 1]], float),
    PEN06: np.array([[0, 0, -1], [1, 0, -1], [0, 1, -1], [0, 0, 1], [1, 0, 1], [0, 1, 1]], float),
    HEX08: np.array([[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1],
                     [-1, -1, 1], [1, -1, 1], [1, 1, 1], [-1, 1, 1]], float),
}


def single_element(etype: int, seed: int = 0, distort: float = 0.1) -> Mesh:
    """One element: its reference-node coordinates, randomly scaled, rotated,
    translated and perturbed by U(-distort, distort)."""
    rng = np.random.default_rng(seed)
    ref = REFERENCE_NODES[etype]
    rot = _random_rotation(rng)
    scale = rng.uniform(0.5, 2.0)
    x = (ref + rng.uniform(-distort, distort, ref.shape)) * scale @ rot.T + rng.uniform(-1, 1, 3)
    conn = np.arange(ref.shape[0], dtype=np.int32)[None, :]
    conn = orient_positive(etype, conn, x).astype(np.int32)
    return Mesh(xyz=x, conn={etype: conn}, name=f"single_{ETYPE_NAMES[etype]}")


def random_field(mesh: Mesh, seed: int = 1, scale: float = 1.0, nu: float = 1e-2,
                 c_vreman: float = 0.07) -> Field:
    rng = np.random.default_rng(seed)
    n = mesh.n_nodes
    return Field(u=scale * rng.standard_normal((n, 3)), p=scale * rng.standard_normal(n),
                 nu=nu, c_vreman=c_vreman)
