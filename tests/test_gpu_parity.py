"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (relative L2 over all nodes and components, and the max-norm of
the difference over the max-norm of the oracle's RHS):
  FP64 path:   1e-12 / 1e-12 (the stated FP64 tolerance);
  mixed path:  FP32 element arithmetic with FP32 coordinates whose rounding
               (2^-24 of the coordinate magnitude) relative to the element
               size sets the error: gates 2e-5 / 2e-4 here, the measured
               values are printed by the benchmark.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2005_05899_b300 import fea
from paper_2005_05899_b300 import meshgen as mg

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_L2 = 2e-5
MIXED_MAX = 2e-4


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    c = fea.Context(0)
    yield c
    c.close()


def errors(gpu, ref):
    d = gpu - ref
    return np.linalg.norm(d) / np.linalg.norm(ref), np.abs(d).max() / np.abs(ref).max()


def gpu_rhs(ctx, mesh, field, prec, closure="vreman", mask=fea.TERM_ALL, scatter="auto", want_nut=False,
            dm=None):
    dm = dm or ctx.upload_mesh(mesh)
    dm.upload_field(field.u, field.p, field.nu, field.c_vreman)
    out = torch.empty((3, dm.n_nodes), dtype=torch.float64, device="cuda")
    nut = torch.empty(dm.n_gauss_total, dtype=torch.float32, device="cuda") if want_nut else None
    dm.assemble(out, prec=prec, closure=closure, mask=mask, scatter=scatter, nut_out=nut)
    ctx.sync_status()
    r = out.cpu().numpy().T.copy()
    if want_nut:
        return r, nut.cpu().numpy(), dm
    return r, dm


def oracle_rhs(mesh, field, closure="vreman", mask=fea.TERM_ALL, want_nut=False):
    om = O.OracleMesh.of(mesh)
    return O.assemble_rhs(om, field.u, field.p, field.nu, field.c_vreman, closure, mask, want_nut=want_nut)


@pytest.fixture(scope="module")
def tgv():
    m = mg.tgv_mesh(16)
    return m, mg.tgv_field(m)


@pytest.fixture(scope="module")
def mixed_small():
    m = mg.channel_mesh(nx=12, ny=14, nz=10, seed=21, n_layers=2, split_frac=0.3)
    return m, mg.channel_field(m, seed=5, nu=1e-2)


def test_tgv_fp64_matches_oracle(ctx, tgv):
    m, f = tgv
    r, nut, _ = gpu_rhs(ctx, m, f, "fp64", want_nut=True)
    ref, nref = oracle_rhs(m, f, want_nut=True)
    l2, mx = errors(r, ref)
    assert l2 < FP64_TOL and mx < FP64_TOL, (l2, mx)
    assert np.allclose(nut, nref[0].ravel(), rtol=2e-7, atol=1e-12)


@pytest.mark.parametrize("mask", [fea.TERM_CONV, fea.TERM_VISC, fea.TERM_SGS, fea.TERM_PRES, fea.TERM_ALL])
def test_mixed_mesh_fp64_every_term(ctx, mixed_small, mask):
    m, f = mixed_small
    r, _ = gpu_rhs(ctx, m, f, "fp64", mask=mask)
    ref = oracle_rhs(m, f, mask=mask)
    l2, mx = errors(r, ref)
    assert l2 < FP64_TOL and mx < FP64_TOL, (mask, l2, mx)


def test_mixed_mesh_fp64_nut_per_gauss_point(ctx, mixed_small):
    m, f = mixed_small
    _, nut, _ = gpu_rhs(ctx, m, f, "fp64", want_nut=True)
    _, nref = oracle_rhs(m, f, want_nut=True)
    ref = np.concatenate([nref[t].ravel() for t in range(4) if t in nref])
    assert np.allclose(nut, ref, rtol=2e-7, atol=1e-30)


@pytest.mark.parametrize("closure", ["none", "vreman"])
def test_mixed_mesh_mixed_precision(ctx, mixed_small, closure):
    m, f = mixed_small
    r, _ = gpu_rhs(ctx, m, f, "mixed", closure=closure)
    ref = oracle_rhs(m, f, closure=closure)
    l2, mx = errors(r, ref)
    print(f"mixed {closure}: rel-L2 {l2:.3e} max {mx:.3e}")
    assert l2 < MIXED_L2 and mx < MIXED_MAX, (l2, mx)


@pytest.mark.parametrize("etype", [fea.TET04, fea.PYR05, fea.PEN06, fea.HEX08])
def test_single_elements(ctx, etype):
    m = mg.single_element(etype, seed=3 + etype)
    f = mg.random_field(m, seed=etype)
    r, _ = gpu_rhs(ctx, m, f, "fp64")
    ref = oracle_rhs(m, f)
    l2, mx = errors(r, ref)
    assert l2 < FP64_TOL and mx < FP64_TOL


def test_ragged_and_single_type_meshes(ctx):
    # sizes that are not multiples of any block size; one type only
    for nx, nz in ((3, 5), (7, 1), (1, 1)):
        m = mg.channel_mesh(nx=nx, ny=6, nz=nz, seed=1, n_layers=1, split_frac=0.0)
        only_hex = mg.Mesh(xyz=m.xyz, conn={fea.HEX08: m.conn[fea.HEX08]})
        f = mg.random_field(only_hex, seed=2)
        r, _ = gpu_rhs(ctx, only_hex, f, "fp64")
        ref = oracle_rhs(only_hex, f)
        assert errors(r, ref)[0] < FP64_TOL


def test_lumped_mass_and_fold(ctx, mixed_small):
    m, f = mixed_small
    dm = ctx.upload_mesh(m)
    ml = torch.empty(dm.n_nodes, dtype=torch.float64, device="cuda")
    dm.lumped_mass(ml)
    ref = O.lumped_mass(O.OracleMesh.of(m))
    assert np.abs(ml.cpu().numpy() - ref).max() < 1e-14 * ref.max()
    v = torch.tensor(np.stack([ref, 2 * ref]), device="cuda")
    dm.fold(v)
    fr = O.periodic_fold(m.periodic_master, np.stack([ref, 2 * ref], axis=1))
    assert np.abs(v.cpu().numpy().T - fr).max() < 1e-14 * fr.max()


def test_channel_full_size_mixed(ctx):
    m = mg.channel_mesh()
    f = mg.channel_field(m)
    r, _ = gpu_rhs(ctx, m, f, "mixed")
    ref = oracle_rhs(m, f)
    l2, mx = errors(r, ref)
    print(f"channel 128x64x64 mixed: rel-L2 {l2:.3e} max {mx:.3e}")
    assert l2 < MIXED_L2 and mx < MIXED_MAX


def test_upload_errors(ctx):
    m = mg.single_element(fea.TET04, seed=1)
    bad = mg.Mesh(xyz=m.xyz, conn={fea.TET04: m.conn[fea.TET04][:, [0, 2, 1, 3]]})
    with pytest.raises(fea.FeaError) as ei:
        ctx.upload_mesh(bad)
    assert ei.value.status == fea.EMESH
    oob = mg.Mesh(xyz=m.xyz, conn={fea.TET04: m.conn[fea.TET04] + 1})
    with pytest.raises(fea.FeaError) as ei:
        ctx.upload_mesh(oob)
    assert ei.value.status == fea.EMESH
    dm = ctx.upload_mesh(m)
    out = torch.empty((3, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(fea.FeaError) as ei:
        dm.assemble(out)
    assert ei.value.status == fea.ESTATE
    dm.upload_field(np.zeros((4, 3)), np.zeros(4), 0.1)
    with pytest.raises(fea.FeaError) as ei:
        dm.assemble(out, mask=99)
    assert ei.value.status == fea.EINVAL
    ctx.sync_status()
