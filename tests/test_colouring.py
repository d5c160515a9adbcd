"""Host greedy element colouring (fea_colour_elements), the one the colour
scatter launches colour by colour (no device needed).

* Validity: no two elements of one colour share a node, on Kuhn-split tets
  and on every category of the mixed channel mesh.
* Greedy: an element of colour c has, for every c' < c, an earlier element
  sharing a node with colour c' (brute force on a small mesh).
* Bounds: at least the largest node degree (the elements around a node
  need distinct colours), at most one more than the largest element
  neighbourhood.
* Edge cases: no elements; a node id out of range is FEA_EMESH.
"""
import numpy as np
import pytest

from paper_2005_05899_b300 import fea
from paper_2005_05899_b300 import meshgen as mg


def _check_valid(conn, col, nc):
    assert col.min() >= 0 and col.max() == nc - 1
    for c in range(nc):
        nodes = conn[col == c].ravel()
        assert np.unique(nodes).size == nodes.size, c


def _degree(conn, n):
    return np.bincount(conn.ravel(), minlength=n).max()


def test_kuhn_tets_valid_and_within_bounds():
    m = mg.tgv_mesh(8)
    conn = m.conn[mg.TET04]
    col, nc = fea.colour_elements(conn, m.n_nodes)
    _check_valid(conn, col, nc)
    deg = _degree(conn, m.n_nodes)
    # neighbours of an element: elements sharing one of its nodes
    nbr = max(np.unique(np.concatenate([np.flatnonzero((conn == v).any(axis=1)) for v in e])).size - 1
              for e in conn[:200])
    assert deg <= nc <= nbr + 1


def test_every_category_of_the_mixed_mesh():
    m = mg.channel_mesh(nx=8, ny=10, nz=6, seed=3, n_layers=2, split_frac=0.3)
    assert len(m.conn) == 4
    for t, conn in m.conn.items():
        col, nc = fea.colour_elements(conn, m.n_nodes)
        _check_valid(conn, col, nc)
        assert nc >= _degree(conn, m.n_nodes)


def test_greedy_choice_by_brute_force():
    m = mg.tgv_mesh(4)
    conn = m.conn[mg.TET04]
    col, nc = fea.colour_elements(conn, m.n_nodes)
    sets = [set(e) for e in conn]
    for e in range(conn.shape[0]):
        below = {col[f] for f in range(e) if sets[f] & sets[e]}
        assert set(range(col[e])) <= below, e          # every lower colour was taken by an earlier neighbour
        assert col[e] not in below


def test_empty_and_bad_ids():
    col, nc = fea.colour_elements(np.zeros((0, 4), np.int32), 10)
    assert nc == 0 and col.size == 0
    with pytest.raises(fea.FeaError) as e:
        fea.colour_elements(np.array([[0, 1, 2, 10]], np.int32), 10)
    assert e.value.status == fea.EMESH
