"""Bounded device waits: the TET04 assembly kernel's mbarrier waits give up
after a poll limit, leave their copies to land, and report FEA_ETIMEOUT; the
context stays usable and the next assembly at the default limit is exact.

The wait is made to run out by lowering the poll limit to one poll
(fea_set_wait_limit) - no fault, trap or endless loop is involved."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2005_05899_b300 import fea
from paper_2005_05899_b300 import meshgen as mg

pytestmark = pytest.mark.gpu


def test_wait_limit_gives_timeout_then_clean_assembly():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    m = mg.tgv_mesh(40)               # 384,000 TET04: several chunks per CTA
    f = mg.tgv_field(m)
    ctx = fea.Context(0)
    try:
        dm = ctx.upload_mesh(m)
        dm.upload_field(f.u, f.p, f.nu, f.c_vreman)
        dm.set_plan("chunk", 128, 256, 0)
        out = torch.zeros((3, dm.n_nodes), dtype=torch.float64, device="cuda")
        ctx.set_wait_limit(1)
        for _ in range(2):                       # twice: the abort path leaves the context usable
            dm.assemble(out, prec="mixed", closure="vreman")
            with pytest.raises(fea.FeaError) as ei:
                ctx.sync_status()
            assert ei.value.status == fea.ETIMEOUT
        ctx.set_wait_limit(0)
        dm.assemble(out, prec="mixed", closure="vreman")
        ctx.sync_status()
        got = out.cpu().numpy().T
        ref = O.assemble_rhs(O.OracleMesh.of(m), f.u, f.p, f.nu, f.c_vreman, "vreman")
        l2 = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert l2 < 2e-5, l2
    finally:
        ctx.close()

