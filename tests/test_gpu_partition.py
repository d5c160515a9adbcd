"""A partitioned mesh on the GPU: every part is assembled by the library,
folded over its own periodic classes, and the shared classes are completed
by the library's pack/unpack kernels.  On one GPU the all-reduce of the
parts' class vectors is a host-ordered sum of the parts' buffers (no kernel
waits on another).  Every node must end with the whole mesh's folded RHS:
FP64 path to 1e-12 of the whole-mesh FP64 assembly, mixed path within the
mixed-precision gates of the oracle."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2005_05899_b300 import fea
from paper_2005_05899_b300 import meshgen as mg
from paper_2005_05899_b300 import partition as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = fea.Context(0)
    yield c
    c.close()


def whole(ctx, m, f, prec):
    dm = ctx.upload_mesh(m)
    dm.upload_field(f.u, f.p, f.nu, f.c_vreman)
    out = torch.empty((3, dm.n_nodes), dtype=torch.float64, device="cuda")
    dm.assemble(out, prec=prec, scatter="atomic" if prec == "fp64" else "auto")
    dm.fold(out)
    ctx.sync_status()
    return out.cpu().numpy().T


@pytest.mark.parametrize("n_parts,prec", [(2, "fp64"), (3, "fp64"), (4, "mixed")])
def test_parts_with_exchange_equal_the_whole_mesh(ctx, n_parts, prec):
    m = mg.channel_mesh(nx=14, ny=12, nz=8, seed=3, n_layers=2, split_frac=0.3)
    f = mg.channel_field(m, seed=4, nu=1e-3)
    parts = P.build_parts(m, n_parts)
    rhs, ex = [], []
    for part in parts:
        dm = ctx.upload_mesh(part.mesh)
        dm.upload_field(f.u[part.nodes], f.p[part.nodes], f.nu, f.c_vreman)
        r = torch.empty((3, dm.n_nodes), dtype=torch.float64, device="cuda")
        dm.assemble(r, prec=prec, scatter="atomic" if prec == "fp64" else "auto")
        dm.fold(r)
        e = P.Exchange(ctx, part)
        e.pack(r)
        rhs.append(r)
        ex.append(e)
    total = sum(e.buf for e in ex)
    for e, r in zip(ex, rhs):
        e.buf.copy_(total)
        e.unpack(r)
    ctx.sync_status()
    ref = whole(ctx, m, f, prec)
    oref = O.periodic_fold(m.periodic_master, O.assemble_rhs(O.OracleMesh.of(m), f.u, f.p, f.nu, f.c_vreman,
                                                              "vreman"))
    scale = np.abs(oref).max()
    for part, r in zip(parts, rhs):
        got = r.cpu().numpy().T
        if prec == "fp64":
            assert np.abs(got - ref[part.nodes]).max() <= 1e-12 * scale
            assert np.abs(got - oref[part.nodes]).max() <= 1e-12 * scale
        else:
            assert np.linalg.norm(got - oref[part.nodes]) <= 2e-5 * np.linalg.norm(oref[part.nodes])
            assert np.abs(got - oref[part.nodes]).max() <= 2e-4 * scale


def test_interface_kernels_flag_bad_indices(ctx):
    v = torch.zeros((3, 10), dtype=torch.float64, device="cuda")
    buf = torch.zeros((3, 4), dtype=torch.float64, device="cuda")
    loc = torch.tensor([0, 11], dtype=torch.int64, device="cuda")
    cls = torch.tensor([1, 2], dtype=torch.int64, device="cuda")
    ctx.interface_pack(v, loc, cls, buf)
    with pytest.raises(fea.FeaError) as ei:
        ctx.sync_status()
    assert ei.value.status == fea.EMESH
    ctx.interface_unpack(buf, loc, cls, v)
    with pytest.raises(fea.FeaError):
        ctx.sync_status()
    ctx.sync_status()


def test_parts_with_wall_faces_equal_the_whole_mesh(ctx):
    """Wall faces split over the parts (each face with one owner) plus the
    exchange give the whole mesh's folded element + wall-model RHS."""
    m = mg.channel_mesh(nx=14, ny=12, nz=8, seed=3, n_layers=2, split_frac=0.3)
    f = mg.channel_field(m, seed=4, nu=1e-3)
    u = f.u + 0.1 * np.random.default_rng(6).standard_normal(f.u.shape)
    parts = P.build_parts(m, 3)
    rhs, ex = [], []
    for part in parts:
        dm = ctx.upload_mesh(part.mesh)
        dm.upload_field(u[part.nodes], f.p[part.nodes], f.nu, f.c_vreman)
        dm.wall_setup(**part.mesh.wall_faces)
        r = torch.empty((3, dm.n_nodes), dtype=torch.float64, device="cuda")
        dm.assemble(r, prec="fp64", scatter="atomic")
        dm.wall_assemble(r)
        dm.fold(r)
        e = P.Exchange(ctx, part)
        e.pack(r)
        rhs.append(r)
        ex.append(e)
    total = sum(e.buf for e in ex)
    for e, r in zip(ex, rhs):
        e.buf.copy_(total)
        e.unpack(r)
    ctx.sync_status()
    om = O.OracleMesh.of(m)
    ref = O.periodic_fold(m.periodic_master, O.assemble_rhs(om, u, f.p, f.nu, f.c_vreman, "vreman")
                          + O.wall_rhs(om, u, f.nu, **m.wall_faces))
    scale = np.abs(ref).max()
    for part, r in zip(parts, rhs):
        assert np.abs(r.cpu().numpy().T - ref[part.nodes]).max() <= 1e-12 * scale
