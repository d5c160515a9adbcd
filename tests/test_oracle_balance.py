"""Pins of the oracle's partition correction coefficients (the
load-balancing section) and the library's implementation against it.

The section's setting: identical processors, element weights that misjudge
the cost, i.e. a cost density c(s) along the curve coordinate s in [0, P]
(s = Lambda).  Part i covers [Lambda_(i-1), Lambda_i], t_i is the integral
of c over it, the mean time is constant, and Upsilon_i = P C(Lambda_i) /
C(P) depends on Lambda_i alone; each splitting point must converge to the
root of C(Lambda_i) = i C(P) / P.  With heterogeneous processor speeds (the
co-execution case) Upsilon_i also depends on the other splitting points; the
iteration must still reduce the imbalance.
"""
import numpy as np
import pytest

import oracle as O
from paper_2005_05899_b300 import fea
from paper_2005_05899_b300 import partition as P


def cumulative_cost(P, density_breaks, density_values):
    """C(s) for a piecewise-constant cost density on [0, P]."""
    xs = np.concatenate([[0.0], density_breaks, [float(P)]])
    cs = np.concatenate([[0.0], np.cumsum(np.diff(xs) * density_values)])
    return lambda s: np.interp(s, xs, cs), xs, cs


def run_density(update, P, C, iters):
    lam = np.ones(P)
    Lh, Th, imb = [], [], []
    for _ in range(iters):
        Lam = np.concatenate([[0.0], np.cumsum(lam)])
        t = np.diff(C(Lam))
        imb.append(t.max() / t.mean())
        Lh.append(Lam)
        Th.append(t)
        lam = update(np.array(Lh), np.array(Th))
    return lam, imb


def run_speeds(update, speeds, iters):
    lam = np.ones(len(speeds))
    Lh, Th, imb = [], [], []
    for _ in range(iters):
        t = lam / speeds
        imb.append(t.max() / t.mean())
        Lh.append(np.concatenate([[0.0], np.cumsum(lam)]))
        Th.append(t)
        lam = update(np.array(Lh), np.array(Th))
    return lam, imb


def test_balanced_observation_is_a_fixed_point():
    lam = O.balance_update([np.arange(5.0)], [np.full(4, 2.5)])
    assert np.allclose(lam, 1.0, atol=1e-12)


@pytest.mark.parametrize("P,breaks,values", [(4, [1.3, 2.2], [1.0, 3.0, 0.7]),
                                             (8, [0.5, 3.0, 3.5, 6.0], [2.0, 1.0, 4.0, 1.0, 0.5])])
def test_splitting_points_converge_for_a_misjudged_cost(P, breaks, values):
    C, xs, cs = cumulative_cost(P, np.array(breaks), np.array(values))
    lam, imb = run_density(O.balance_update, P, C, 13)
    assert abs(lam.sum() - P) < 1e-12 and np.all(lam >= 0)
    # the regression over all (increasingly weighted) observations converges
    # steadily, not in one step: measured 1.83 -> 1.04 (P = 4) and
    # 2.22 -> 1.02 (P = 8) over 12 corrections
    assert imb[0] > 1.2 and imb[-1] < 1.06, imb
    assert all(b <= a + 1e-12 for a, b in zip(imb[2:], imb[3:])), imb
    Lam = np.concatenate([[0.0], np.cumsum(lam)])
    target = np.interp(np.arange(P + 1) * cs[-1] / P, cs, xs)   # the roots C(Lambda_i) = i C(P) / P
    assert np.abs(Lam - target).max() < 0.03 * P


def test_heterogeneous_speeds_reduce_the_imbalance():
    speeds = np.array([1.0, 1.0, 2.0, 1.0, 1.0, 1.0, 1.0, 1.5])
    lam, imb = run_speeds(O.balance_update, speeds, 12)
    assert imb[-1] < 1.01 and imb[-1] < imb[0] / 1.1, imb   # measured 1.116 -> 1.002


def test_library_matches_oracle():
    rng = np.random.default_rng(7)
    for P in (2, 3, 6):
        speeds = rng.uniform(0.3, 5.0, P)
        lam_o, _ = run_speeds(O.balance_update, speeds, 6)
        lam_l, _ = run_speeds(fea.balance_update, speeds, 6)
        assert np.allclose(lam_l, lam_o, rtol=1e-10, atol=1e-12)


def test_partition_follows_the_coefficients():
    from paper_2005_05899_b300 import meshgen as mg
    m = mg.channel_mesh(nx=12, ny=10, nz=8, seed=3, n_layers=2, split_frac=0.3)
    w = {0: 4, 1: 8, 2: 6, 3: 8}
    lam = np.array([0.5, 1.5, 1.0, 1.0])
    part = fea.partition_sfc(m, 4, lam=lam)
    load = np.zeros(4)
    for t, a in part.items():
        np.add.at(load, a, w[t])
    share = load / load.sum()
    assert np.allclose(share, lam / lam.sum(), atol=0.01), share
    b = P.Balancer(4)
    nxt = b.update([1.0, 2.0, 1.0, 1.0])
    assert abs(nxt.sum() - 4) < 1e-12 and nxt[1] < 1.0 and b.imbalance([1.0, 2.0, 1.0, 1.0]) == pytest.approx(1.6)
