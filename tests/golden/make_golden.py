"""Writes the regression fixtures of this folder from the FP64 oracle.

    python tests/golden/make_golden.py

The paper prints no worked example of the assembly, so these files hold no
value of the paper's.  They store the oracle's own results on small inputs,
with the inputs, so that a change to the oracle's arithmetic shows up as a
changed fixture in review (tests/test_golden.py recomputes them).  They are
not pins: the pins, which tie the oracle to closed forms, invariants and
brute force, are the tests/test_oracle_*.py files.  Only ``oracle`` and the
seeded input generator ``meshgen`` are called here.

* single_elements.json - one distorted element of each type with a random
  nodal field: the element residual of Eq. momentum (section 2.1) assembled
  element by element (section 2.3.3), all terms and each term alone, with the
  Vreman eddy viscosity (section 2.1) at every Gauss point and the element
  volume.
* wall_law.json - Reichardt's law and the Newton root u_tau of the
  equilibrium wall model (the reading of the paper's wall model, boundary
  assembly of section 2.3.3) at points from the viscous sublayer to the log
  layer.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2005_05899_b300 import meshgen as mg  # noqa: E402

TYPE_NAMES = {O.TET04: "TET04", O.PYR05: "PYR05", O.PEN06: "PEN06", O.HEX08: "HEX08"}
MASKS = {"all": O.TERM_ALL, "conv": O.TERM_CONV, "visc": O.TERM_VISC, "sgs": O.TERM_SGS, "pres": O.TERM_PRES}
NU, C_VREMAN = 1e-2, 0.07
WALL_POINTS = [(1e-3, 2e-3, 1.5e-5), (0.3, 2e-3, 1.5e-5), (1.0, 1e-4, 1e-3), (2.0, 0.05, 1.0 / 5600),
               (1.0, 1e-2, 1.0 / 1.93e6)]
YPLUS = [0.0, 1e-3, 0.5, 5.0, 11.0, 30.0, 300.0, 1e4, 1e6]


def single_elements():
    out = []
    for t in (O.TET04, O.PYR05, O.PEN06, O.HEX08):
        m = mg.single_element(t, seed=40 + t)
        f = mg.random_field(m, seed=50 + t, nu=NU, c_vreman=C_VREMAN)
        om = O.OracleMesh(m.xyz, {t: m.conn[t]})
        rec = {"etype": TYPE_NAMES[t], "xyz": m.xyz.tolist(), "conn": m.conn[t].tolist(), "u": f.u.tolist(),
               "p": f.p.tolist(), "nu": NU, "c_vreman": C_VREMAN, "rhs": {}}
        for name, mask in MASKS.items():
            rec["rhs"][name] = O.assemble_rhs(om, f.u, f.p, NU, C_VREMAN, "vreman", mask).tolist()
        _, nut, vol = O.assemble_rhs(om, f.u, f.p, NU, C_VREMAN, "vreman", O.TERM_ALL, want_nut=True,
                                     want_vol=True)
        rec["nut"] = nut[t][0].tolist()
        rec["volume"] = float(vol[t][0])
        out.append(rec)
    return {"about": "oracle regression fixture (not a pin): element residual of Eq. momentum, section 2.1 / "
                     "2.3.3, Vreman closure; written by tests/golden/make_golden.py",
            "elements": out}


def wall_law():
    law = []
    for yp in YPLUS:
        f, d = O.reichardt(yp)
        law.append({"yplus": yp, "uplus": f, "duplus": d})
    roots = []
    for U, y, nu in WALL_POINTS:
        ut, _ = O.wall_utau(U, y, nu)
        roots.append({"U": U, "y": y, "nu": nu, "utau": ut})
    return {"about": "oracle regression fixture (not a pin): Reichardt's law (kappa = %g, C = %g) and the Newton "
                     "root of U = u_tau f(y u_tau / nu); written by tests/golden/make_golden.py"
                     % (O.WALL_KAPPA, O.WALL_C),
            "kappa": O.WALL_KAPPA, "C": O.WALL_C, "law": law, "utau": roots}


def main():
    for name, data in (("single_elements.json", single_elements()), ("wall_law.json", wall_law())):
        with open(os.path.join(HERE, name), "w") as fh:
            json.dump(data, fh, indent=1)
            fh.write("\n")
        print("wrote", name)


if __name__ == "__main__":
    main()
