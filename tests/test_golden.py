"""The oracle against its stored regression fixtures (tests/golden/).

The fixtures were written by tests/golden/make_golden.py from the oracle
itself; they are not pins (those are the test_oracle_*.py files) but catch
any change of the oracle's arithmetic: the element residual of Eq. momentum
(section 2.1, assembled as in section 2.3.3) with each term alone, the
Vreman eddy viscosity and the element volume for one element of every type,
and the wall law with its Newton root.  Tolerance 1e-13 of each record's
largest value: the oracle is plain C at -O2 without contraction, so only the
C library's sqrt / cbrt / exp / log1p may differ between machines, by an ulp.
"""
import json
import os

import numpy as np
import pytest

import oracle as O

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
TYPES = {"TET04": O.TET04, "PYR05": O.PYR05, "PEN06": O.PEN06, "HEX08": O.HEX08}
MASKS = {"all": O.TERM_ALL, "conv": O.TERM_CONV, "visc": O.TERM_VISC, "sgs": O.TERM_SGS, "pres": O.TERM_PRES}
TOL = 1e-13


def _load(name):
    with open(os.path.join(HERE, name)) as fh:
        return json.load(fh)


def _close(got, want):
    got, want = np.asarray(got, dtype=np.float64), np.asarray(want, dtype=np.float64)
    assert got.shape == want.shape
    scale = max(np.abs(want).max(), 1e-300)
    return np.abs(got - want).max() <= TOL * scale


ELEMENTS = _load("single_elements.json")["elements"]


def test_fixture_covers_every_type_and_term():
    assert sorted(r["etype"] for r in ELEMENTS) == sorted(TYPES)
    for r in ELEMENTS:
        assert sorted(r["rhs"]) == sorted(MASKS)
        assert len(r["nut"]) == O.NGAUSS[TYPES[r["etype"]]]
        # the terms add up to the whole residual (a property of the stored values)
        parts = sum(np.asarray(r["rhs"][k]) for k in ("conv", "visc", "sgs", "pres"))
        assert _close(parts, r["rhs"]["all"])


@pytest.mark.parametrize("rec", ELEMENTS, ids=[r["etype"] for r in ELEMENTS])
def test_single_element_residuals(rec):
    t = TYPES[rec["etype"]]
    xyz = np.asarray(rec["xyz"], dtype=np.float64)
    conn = np.asarray(rec["conn"], dtype=np.int32)
    u = np.asarray(rec["u"], dtype=np.float64)
    p = np.asarray(rec["p"], dtype=np.float64)
    om = O.OracleMesh(xyz, {t: conn})
    for name, mask in MASKS.items():
        got = O.assemble_rhs(om, u, p, rec["nu"], rec["c_vreman"], "vreman", mask)
        assert _close(got, rec["rhs"][name]), (rec["etype"], name)
    _, nut, vol = O.assemble_rhs(om, u, p, rec["nu"], rec["c_vreman"], "vreman", O.TERM_ALL, want_nut=True,
                                 want_vol=True)
    assert _close(nut[t][0], rec["nut"])
    assert _close(vol[t][0], rec["volume"])


def test_wall_law_and_newton_root():
    data = _load("wall_law.json")
    assert data["kappa"] == O.WALL_KAPPA and data["C"] == O.WALL_C
    for r in data["law"]:
        f, d = O.reichardt(r["yplus"])
        assert _close([f, d], [r["uplus"], r["duplus"]]), r
    for r in data["utau"]:
        ut, _ = O.wall_utau(r["U"], r["y"], r["nu"])
        assert _close(ut, r["utau"]), r
