"""Seeded input generators: counts, conformity, determinism, validity."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2005_05899_b300 import meshgen as mg

TRI_FACES = {
    mg.TET04: [[0, 1, 2], [0, 1, 3], [1, 2, 3], [0, 2, 3]],
    mg.PYR05: [[0, 1, 4], [1, 2, 4], [2, 3, 4], [3, 0, 4]],
    mg.PEN06: [[0, 1, 2], [3, 4, 5]],
    mg.HEX08: [],
}
QUAD_FACES = {
    mg.TET04: [],
    mg.PYR05: [[0, 1, 2, 3]],
    mg.PEN06: [[0, 1, 4, 3], [1, 2, 5, 4], [2, 0, 3, 5]],
    mg.HEX08: [[0, 1, 2, 3], [4, 5, 6, 7], [0, 1, 5, 4], [1, 2, 6, 5], [2, 3, 7, 6], [3, 0, 4, 7]],
}


def face_counts(m):
    keys = []
    for t, c in m.conn.items():
        for f in TRI_FACES[t]:
            s = np.sort(c[:, f], axis=1)
            keys.append(np.concatenate([s, np.full((s.shape[0], 1), -1)], axis=1))
        for f in QUAD_FACES[t]:
            keys.append(np.sort(c[:, f], axis=1))
    k = np.concatenate(keys)
    _, cnt = np.unique(k, axis=0, return_counts=True)
    uniq, inv = np.unique(k, axis=0, return_inverse=True)
    return k, cnt[inv.ravel()]


def test_tgv_counts_and_periodic_map():
    m = mg.tgv_mesh(16)
    assert m.n_elem(mg.TET04) == 24576 and m.n_nodes == 4913
    masters = np.unique(m.periodic_master)
    assert masters.size == 4096
    assert np.array_equal(m.periodic_master[masters], masters)
    # a slave sits at the master's position shifted by multiples of 2 pi
    d = m.xyz - m.xyz[m.periodic_master]
    assert np.allclose(np.round(d / (2 * math.pi)) * 2 * math.pi, d, atol=1e-12)


def test_channel_counts_full_size():
    m = mg.channel_mesh()
    assert m.counts() == {"TET04": 32768, "PYR05": 308018, "PEN06": 262144, "HEX08": 339149}
    assert m.meta["first_cell"] == pytest.approx(7.45e-3, rel=2e-3)
    assert m.dirichlet.sum() == 2 * 129 * 65
    assert np.all(m.fp64_flag[mg.PEN06] == 1)


@pytest.mark.parametrize("maker", [
    lambda: mg.channel_mesh(nx=10, ny=12, nz=8, seed=3, n_layers=2, split_frac=0.3),
    lambda: mg.airplane_mesh(20, seed=4),
    lambda: mg.tgv_mesh(5),
])
def test_meshes_are_conforming(maker):
    m = maker()
    k, cnt = face_counts(m)
    assert cnt.max() == 2                      # no face shared by three elements
    bnd = k[cnt == 1]
    x = m.xyz
    # a face seen once lies on the domain boundary: box planes or the inner wall
    lo, hi = x.min(axis=0), x.max(axis=0)
    nodes = bnd[bnd >= 0].reshape(-1) if False else None
    on_box = np.zeros(len(bnd), bool)
    for ax in range(3):
        for v in (lo[ax], hi[ax]):
            cols = [np.where(b >= 0, np.abs(x[np.maximum(b, 0), ax] - v) < 1e-12, True) for b in bnd.T]
            on_box |= np.all(np.stack(cols, axis=1), axis=1)
    if "inner_wall_faces" in m.meta:
        wall = {tuple(sorted(f)) + (-1,) for f in m.meta["inner_wall_faces"].tolist()}
        on_box |= np.array([tuple(sorted(f[f >= 0].tolist())) + (-1,) in wall if f[-1] == -1 else False
                            for f in np.sort(bnd, axis=1)[:, ::-1]]) | np.array(
            [tuple(f) in wall for f in bnd.tolist()])
    assert on_box.all(), int((~on_box).sum())


def test_generators_are_deterministic():
    a = mg.channel_mesh(nx=6, ny=8, nz=4, seed=9, n_layers=1)
    b = mg.channel_mesh(nx=6, ny=8, nz=4, seed=9, n_layers=1)
    assert np.array_equal(a.xyz, b.xyz)
    for t in a.conn:
        assert np.array_equal(a.conn[t], b.conn[t])
    fa, fb = mg.channel_field(a, seed=1), mg.channel_field(b, seed=1)
    assert np.array_equal(fa.u, fb.u) and np.array_equal(fa.p, fb.p)


def test_all_elements_valid_at_every_gauss_point():
    # the oracle rejects any element with det J <= 0 at a Gauss point
    for m in (mg.channel_mesh(nx=16, ny=16, nz=8, seed=2, n_layers=2, split_frac=0.2),
              mg.airplane_mesh(30, seed=4)):
        om = O.OracleMesh.of(m)
        ml = O.lumped_mass(om)
        assert np.all(ml[np.unique(np.concatenate([c.ravel() for c in m.conn.values()]))] > 0)


def test_batch_sizes_log_uniform():
    out = mg.batch_meshes(count=4, seed=7, e_min=2e3, e_max=2e4)
    assert len(out) == 4
    for m, f in out:
        assert 1e3 < m.n_elem_total < 4e4
        assert 1 / 5000 <= f.nu <= 1 / 500
        assert sum(m.n_elem(t) > 0 for t in mg.ETYPES) == 4
