"""SFC partition and the interface exchange of a partitioned mesh (CPU).

* The Hilbert order visits the cells of a 2^3 grid once each, consecutive
  cells being face neighbours (the defining property of the curve).
* The element partition is contiguous along that order and balanced in
  Gauss points to within one bin.
* Parts built from a periodic mixed mesh cover every element once, and
  their shared classes are numbered alike on every part.
* Distributed (gloo, world sizes 2 and 3, one process per part): each rank
  assembles its part with the oracle, folds its local periodic classes and
  runs the exchange (the library's `partition.Exchange`, with NumPy
  pack/unpack in place of the device kernels); every node must end with the
  single-process oracle's folded RHS.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
from paper_2005_05899_b300 import fea
from paper_2005_05899_b300 import meshgen as mg
from paper_2005_05899_b300 import partition as P

WEIGHT = {0: 4, 1: 8, 2: 6, 3: 8}


def small_mixed():
    m = mg.channel_mesh(nx=10, ny=10, nz=6, seed=3, n_layers=2, split_frac=0.3)
    f = mg.channel_field(m, seed=4, nu=1e-3)
    return m, f


def test_hilbert_order_visits_face_neighbours():
    g = np.arange(8) + 0.5
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    pts = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    rng = np.random.default_rng(0)
    perm = rng.permutation(pts.shape[0])
    pts = pts[perm]
    order = fea.sfc_order(pts, level=3)
    assert np.array_equal(np.sort(order), np.arange(512))
    cells = np.floor(pts[order]).astype(int)
    steps = np.abs(np.diff(cells, axis=0))
    assert np.all(steps.sum(axis=1) == 1), "consecutive cells must share a face"


def test_partition_is_contiguous_and_balanced():
    m, _ = small_mixed()
    cen = np.concatenate([m.xyz[m.conn[t]].mean(axis=1) for t in range(4)])
    w = np.concatenate([np.full(m.conn[t].shape[0], WEIGHT[t]) for t in range(4)])
    order = fea.sfc_order(cen, level=10)
    for n_parts in (1, 2, 3, 5):
        part = fea.partition_sfc(m, n_parts, level=10)
        ids = np.concatenate([part[t] for t in range(4)])
        assert ids.min() == 0 and ids.max() == n_parts - 1
        assert np.all(np.diff(ids[order]) >= 0), "parts must be contiguous along the curve"
        load = np.bincount(ids, weights=w, minlength=n_parts)
        assert np.abs(load - w.sum() / n_parts).max() <= w.max() * 4, load


def test_parts_cover_the_mesh_and_agree_on_shared_classes():
    m, _ = small_mixed()
    parts = P.build_parts(m, 3)
    for t in range(4):
        got = np.sort(np.concatenate([p.elems[t] for p in parts if t in p.elems]))
        assert np.array_equal(got, np.arange(m.conn[t].shape[0]))
    n_shared = {p.n_shared for p in parts}
    assert len(n_shared) == 1 and n_shared.pop() > 0
    # a shared class number means the same periodic class on every part
    cls_global = {}
    for p in parts:
        masters = m.periodic_master[p.nodes[p.iface_loc]]
        for c, g in zip(p.iface_cls, masters):
            assert cls_global.setdefault(int(c), int(g)) == int(g)
    # every shared class appears in at least two parts
    seen = np.zeros(parts[0].n_shared, int)
    for p in parts:
        seen[np.unique(p.iface_cls)] += 1
    assert np.all(seen >= 2)
    # local periodic maps point inside the part
    for p in parts:
        assert p.mesh.periodic_master.max() < p.n_nodes


def test_every_wall_face_goes_to_exactly_one_part():
    m, _ = small_mixed()
    assert m.wall_faces["tri"].shape[0] > 0
    parts = P.build_parts(m, 3)
    got = np.concatenate([p.nodes[p.mesh.wall_faces["tri"]] for p in parts])
    gx = np.concatenate([p.nodes[p.mesh.wall_faces["tri_exch"]] for p in parts])
    key = lambda f, x: np.sort([tuple(r) for r in np.concatenate([f, x], axis=1)], axis=0)
    assert got.shape == m.wall_faces["tri"].shape
    assert np.array_equal(key(got, gx), key(m.wall_faces["tri"], m.wall_faces["tri_exch"]))
    # the node order (and so the face orientation) is kept
    ref = {tuple(r) for r in np.concatenate([m.wall_faces["tri"], m.wall_faces["tri_exch"]], axis=1)}
    assert {tuple(r) for r in np.concatenate([got, gx], axis=1)} == ref


def _np_pack(v, loc, cls, out):
    out.zero_()
    for d in range(3):
        out[d].index_add_(0, cls, v[d, loc])
    return out


def _np_unpack(buf, loc, cls, v):
    v[:, loc] = buf[:, cls]
    return v


def _rank_main(rank, world, port, result_q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m, f = small_mixed()
        parts = P.build_parts(m, world)
        part = parts[rank]
        om = O.OracleMesh.of(part.mesh)
        u, p = f.u[part.nodes], f.p[part.nodes]
        r = O.assemble_rhs(om, u, p, f.nu, f.c_vreman, "vreman")
        r = O.periodic_fold(part.mesh.periodic_master, r)
        rhs = torch.from_numpy(np.ascontiguousarray(r.T))
        ex = P.Exchange(None, part, device="cpu", pack=_np_pack, unpack=_np_unpack)
        ex(rhs)
        ref = O.periodic_fold(m.periodic_master, O.assemble_rhs(O.OracleMesh.of(m), f.u, f.p, f.nu, f.c_vreman,
                                                                 "vreman"))[part.nodes]
        err = np.abs(rhs.numpy().T - ref).max() / np.abs(ref).max()
        result_q.put((rank, float(err), int(part.iface_loc.size)))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2, 3])
def test_distributed_exchange_equals_single_process_assembly(world):
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    mp.start_processes(_rank_main, args=(world, _free_port(), q), nprocs=world, join=True, start_method="spawn")
    res = sorted(q.get() for _ in range(world))
    for rank, err, n_iface in res:
        assert n_iface > 0
        assert err < 1e-13, (rank, err)
