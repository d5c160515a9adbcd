"""Learned closure, end to end on the GPU: fine Taylor-Green LES through the
library, box filtering, training with the library's training kernels, and an
a-priori comparison on a held-out time against Vreman and no model.

What is asserted is what the training objective targets: the least-squares
eddy viscosity nu_t* of the filtered field.  Measured on a 64^3 fine run
(held-out t = 6, coarse 16^3 and 8^3): relative nu_t error 0.79 / 0.69 for
the network against 0.82 / 0.80 for Vreman, correlation 0.46 / 0.56 against
0.38 / 0.29; the full-set fit explains about 40% of the target variance.  The
subgrid-force error of either eddy-viscosity model stays near that of no model
(0.9-1.1 of the true force's norm), so it is reported, not asserted.
"""
import pytest

pytestmark = pytest.mark.gpu


def test_learned_closure_beats_vreman_on_nut_a_priori():
    from paper_2005_05899_b300 import closure_data
    res = closure_data.run(n_f=64, ratios=(4, 8), t_train=(3.0, 4.0, 5.0, 7.0), t_test=(6.0,), steps=1500,
                           log=None)
    # the fit beats the best constant predictor by a clear margin
    assert res["fit_mse"] < 0.8 * res["target_var"], res
    assert len(res["test"]) == 2
    for e in res["test"]:
        assert e["mlp"]["nut"] < e["none"]["nut"], e
        assert e["mlp"]["nut"] < e["vreman"]["nut"], e
        assert e["mlp"]["nut_corr"] > e["vreman"]["nut_corr"] + 0.03, e


def test_library_projection_run_converges_to_the_spectral_one():
    """The fine runs of the training data keep the velocity divergence-free
    either by Algorithm 1 itself (the library's pressure projection after
    the RK3 stages) or by a spectral projection of every stage; the two are
    different discretisations of the same projection, so their difference
    shrinks at O(h^2): measured 1.28e-3 (16^3) and 5.9e-4 (24^3) relative L2
    at t = 1, a ratio of 0.46 against (16/24)^2 = 0.44."""
    import torch
    from paper_2005_05899_b300 import closure_data as cd
    from paper_2005_05899_b300 import fea
    ctx = fea.Context(0)
    diffs = []
    for n in (16, 24):
        a = cd.fine_tgv_run(ctx, n, (1.0,), projection="library")
        b = cd.fine_tgv_run(ctx, n, (1.0,), projection="spectral")
        diffs.append(float(torch.linalg.norm(a[0].u - b[0].u) / torch.linalg.norm(b[0].u)))
    ctx.close()
    assert diffs[0] < 3e-3 and diffs[1] < 1.5e-3, diffs
    assert diffs[1] < 0.6 * diffs[0], diffs
