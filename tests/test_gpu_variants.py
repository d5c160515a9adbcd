"""Model variants on the GPU against the oracle: EMAC convective form and
Vreman widths per direction, separately and together, on the mixed mesh
(generic kernels of every type) and on a tetrahedral mesh (the closed form
of TET04 outside the fused pipeline); FP64 to 1e-12, mixed precision within
the parity gates; nu_t per Gauss point."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2005_05899_b300 import fea
from paper_2005_05899_b300 import meshgen as mg

pytestmark = pytest.mark.gpu

FORMS = [("emac", "volume"), ("gu", "axes"), ("emac", "axes")]


@pytest.fixture(scope="module")
def ctx():
    c = fea.Context(0)
    yield c
    c.close()


def check(ctx, m, f, conv, delta, prec, scatter, closure="vreman"):
    dm = ctx.upload_mesh(m)
    dm.upload_field(f.u, f.p, f.nu, f.c_vreman)
    dm.set_model(conv, delta)
    out = torch.empty((3, dm.n_nodes), dtype=torch.float64, device="cuda")
    nut = torch.empty(dm.n_gauss_total, dtype=torch.float32, device="cuda")
    dm.assemble(out, prec=prec, scatter=scatter, closure=closure, nut_out=nut)
    ctx.sync_status()
    ref, nref = O.assemble_rhs(O.OracleMesh.of(m), f.u, f.p, f.nu, f.c_vreman, closure, want_nut=True,
                               conv_form=int(conv == "emac"), delta_form=int(delta == "axes"))
    got = out.cpu().numpy().T
    l2 = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    mx = np.abs(got - ref).max() / np.abs(ref).max()
    if prec == "fp64":
        assert l2 < 1e-12 and mx < 1e-12, (l2, mx)
    else:
        assert l2 < 2e-5 and mx < 2e-4, (l2, mx)
    nr = np.concatenate([nref[t].ravel() for t in range(4) if t in nref])
    assert np.allclose(nut.cpu().numpy(), nr, rtol=1e-4 if prec == "mixed" else 1e-6, atol=1e-7 * np.abs(nr).max())
    return got


@pytest.mark.parametrize("conv,delta", FORMS)
@pytest.mark.parametrize("prec,scatter", [("fp64", "atomic"), ("mixed", "chunk"), ("mixed", "atomic")])
def test_variants_mixed_mesh(ctx, conv, delta, prec, scatter):
    m = mg.channel_mesh(nx=10, ny=12, nz=8, seed=21, n_layers=2, split_frac=0.3)
    f = mg.random_field(m, seed=8)
    check(ctx, m, f, conv, delta, prec, scatter)


@pytest.mark.parametrize("conv,delta", FORMS)
def test_variants_tet_mesh_leave_the_pipeline(ctx, conv, delta):
    m = mg.tgv_mesh(10)
    f = mg.tgv_field(m)
    got = check(ctx, m, f, conv, delta, "mixed", "chunk")
    # the variant changes the result (it is not silently the default)
    base = check(ctx, m, f, "gu", "volume", "mixed", "chunk")
    assert np.linalg.norm(got - base) > 1e-6 * np.linalg.norm(base)


def test_set_model_rejects_unknown_forms(ctx):
    m = mg.tgv_mesh(4)
    dm = ctx.upload_mesh(m)
    with pytest.raises(fea.FeaError) as ei:
        ctx.check(dm._L().fea_set_model(ctx.handle, dm.id, 2, 0))
    assert ei.value.status == fea.EINVAL
    with pytest.raises(KeyError):
        dm.set_model("upwind", "volume")
