"""A mesh partitioned over several devices (section 5 and section 2.3.1).

The elements are split along a space-filling curve into parts of nearly equal
cost (`fea.partition_sfc`: Gauss points as the cost model).  Each part is an
ordinary mesh of its own (its elements, the nodes they use renumbered
compactly; nodes on part boundaries are duplicated) that one device assembles
with the library.  Afterwards the contributions at duplicated nodes are summed
across parts: the per-stage exchange of section 2.3.1.

Periodic copies are handled by the same mechanism.  A *class* is the set of
node copies that must end with one value: a node and its periodic copies.  A
class whose copies all lie in one part is folded by that part's own periodic
map (`fea_periodic_fold`); a class that appears in two or more parts is
*shared*: each part packs the sum of its copies into a compact vector indexed
by the shared-class number (the same numbering on every part), the vectors are
summed over the parts (an all-reduce), and every copy receives the total.

Host logic only (NumPy): building the parts is set-up work, done once; the
exchange itself runs in the library's pack/unpack kernels and the
communication library's all-reduce.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, Dict, List, Optional

import numpy as np

from . import fea
from .meshgen import Mesh


@dataclasses.dataclass
class Part:
    index: int                       # part id in [0, n_parts)
    mesh: Mesh                       # the part as a mesh of its own
    nodes: np.ndarray                # local node -> global node (int64, increasing)
    elems: Dict[int, np.ndarray]     # etype -> global element ids of the part
    iface_loc: np.ndarray            # local nodes that are copies of shared classes (int64)
    iface_cls: np.ndarray            # their shared-class numbers (int64), common to all parts
    n_shared: int                    # number of shared classes (all parts)

    @property
    def n_nodes(self) -> int:
        return int(self.nodes.size)


def build_parts(mesh: Mesh, n_parts: int, level: int = 10,
                part_of: Optional[Dict[int, np.ndarray]] = None, lam=None) -> List[Part]:
    """Splits `mesh` into `n_parts` parts (SFC partition with correction
    coefficients `lam`, unless `part_of`, a part id per element and type, is
    given).  Every rank calls this with the same mesh and gets the same
    parts."""
    if part_of is None:
        part_of = fea.partition_sfc(mesh, n_parts, level, lam)
    N = mesh.n_nodes
    cls_of = (np.asarray(mesh.periodic_master, dtype=np.int64) if mesh.periodic_master is not None
              else np.arange(N, dtype=np.int64))
    if np.any(cls_of[cls_of] != cls_of):
        raise ValueError("periodic masters must be their own masters")
    used = []
    for p in range(n_parts):
        ids = [mesh.conn[t][part_of[t] == p].ravel() for t in mesh.conn if t in part_of]
        used.append(np.unique(np.concatenate(ids)) if ids else np.zeros(0, np.int64))
    # classes that appear in more than one part
    pairs = np.unique(np.concatenate([cls_of[u] * n_parts + p for p, u in enumerate(used)]))
    parts_per_class = np.bincount(pairs // n_parts, minlength=N)
    shared = np.flatnonzero(parts_per_class >= 2)
    shared_no = np.full(N, -1, np.int64)
    shared_no[shared] = np.arange(shared.size)
    # wall-model faces: each goes to the lowest-numbered part that holds all
    # of its nodes and exchange nodes (a prism-layer face goes with its prism
    # or a lower part), so that every face is assembled exactly once
    wall_owner = {}
    if mesh.wall_faces:
        member = np.zeros((n_parts, N), bool)
        for p in range(n_parts):
            member[p, used[p]] = True
        for kind, nv in (("tri", 3), ("quad", 4)):
            f = mesh.wall_faces.get(kind)
            if f is None or len(f) == 0:
                continue
            x = mesh.wall_faces[kind + "_exch"]
            ok = member[:, f].all(axis=2) & member[:, x].all(axis=2)      # (n_parts, F)
            if not ok.any(axis=0).all():
                raise ValueError(f"a wall face ({kind}) has nodes or exchange nodes in no single part")
            wall_owner[kind] = np.argmax(ok, axis=0)
    out = []
    g2l = np.full(N, -1, np.int64)
    for p in range(n_parts):
        nodes = used[p].astype(np.int64)
        g2l[:] = -1
        g2l[nodes] = np.arange(nodes.size)
        conn, elems, flags = {}, {}, {}
        for t, c in mesh.conn.items():
            sel = np.flatnonzero(part_of[t] == p)
            if sel.size == 0:
                continue
            elems[t] = sel
            conn[t] = g2l[c[sel]].astype(np.int32)
            if mesh.fp64_flag and t in mesh.fp64_flag:
                flags[t] = mesh.fp64_flag[t][sel]
        cls = cls_of[nodes]
        is_shared = shared_no[cls] >= 0
        # local fold for classes inside this part: every copy maps to the local
        # copy of the class's master (present: all copies are in this part)
        local_master = np.where(is_shared, np.arange(nodes.size), g2l[cls])
        if np.any(local_master < 0):
            raise ValueError("a class local to one part lost its master")
        iface_loc = np.flatnonzero(is_shared).astype(np.int64)
        wall = None
        if wall_owner:
            wall = {}
            for kind, owner in wall_owner.items():
                mine = owner == p
                wall[kind] = g2l[mesh.wall_faces[kind][mine]].astype(np.int32)
                wall[kind + "_exch"] = g2l[mesh.wall_faces[kind + "_exch"][mine]].astype(np.int32)
        sub = Mesh(xyz=mesh.xyz[nodes], conn=conn,
                   periodic_master=local_master.astype(np.int32) if mesh.periodic_master is not None else None,
                   dirichlet=mesh.dirichlet[nodes] if mesh.dirichlet is not None else None,
                   fp64_flag=flags, name=f"{mesh.name}.part{p}of{n_parts}", meta=dict(mesh.meta),
                   wall_faces=wall)
        out.append(Part(index=p, mesh=sub, nodes=nodes, elems=elems, iface_loc=iface_loc,
                        iface_cls=shared_no[cls[iface_loc]], n_shared=int(shared.size)))
    return out


class Balancer:
    """Correction coefficients of the partition from measured times (the
    load-balancing section): keeps the history of cumulative coefficients
    and per-part times and asks the library for the next coefficients."""

    def __init__(self, n_parts: int):
        self.n_parts = n_parts
        self.lam = np.ones(n_parts)
        self.Lambda_hist: List[np.ndarray] = []
        self.times_hist: List[np.ndarray] = []

    @staticmethod
    def imbalance(times) -> float:
        t = np.asarray(times, dtype=np.float64)
        return float(t.max() / t.mean())

    def update(self, times) -> np.ndarray:
        """Records the times measured with the current coefficients; returns
        the next coefficients (also kept in self.lam)."""
        self.Lambda_hist.append(np.concatenate([[0.0], np.cumsum(self.lam)]))
        self.times_hist.append(np.asarray(times, dtype=np.float64))
        self.lam = fea.balance_update(np.array(self.Lambda_hist), np.array(self.times_hist))
        return self.lam


class Exchange:
    """The per-stage interface sum of one part: pack (library kernel) ->
    all-reduce over the parts -> unpack (library kernel), in place on the
    part's folded RHS [3][n_local] (FP64, device).

    `allreduce(buf)` sums `buf` over the parts in place; by default
    torch.distributed.all_reduce on the default group.  `pack` / `unpack`
    default to the library's kernels on `ctx`."""

    def __init__(self, ctx, part: Part, device="cuda", allreduce: Optional[Callable] = None,
                 pack: Optional[Callable] = None, unpack: Optional[Callable] = None):
        import torch
        self.part = part
        self.loc = torch.as_tensor(part.iface_loc, dtype=torch.int64, device=device)
        self.cls = torch.as_tensor(part.iface_cls, dtype=torch.int64, device=device)
        self.buf = torch.zeros((3, part.n_shared), dtype=torch.float64, device=device)
        self._pack = pack or ctx.interface_pack
        self._unpack = unpack or ctx.interface_unpack
        if allreduce is None:
            import torch.distributed as dist
            allreduce = dist.all_reduce
        self._allreduce = allreduce

    def pack(self, rhs):
        """This part's class sums into self.buf."""
        return self._pack(rhs, self.loc, self.cls, self.buf)

    def unpack(self, rhs):
        """Every shared copy of rhs receives its class total from self.buf."""
        return self._unpack(self.buf, self.loc, self.cls, rhs)

    def __call__(self, rhs):
        self.pack(rhs)
        self._allreduce(self.buf)
        return self.unpack(rhs)
