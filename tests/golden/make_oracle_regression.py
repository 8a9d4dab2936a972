"""Writes oracle_regression.json: outputs of the oracle on three tiny cases, stored so that any
later change to the oracle's arithmetic shows up as a failing regression test and has to be
made on purpose.  Calls only oracle/ and synth/.  These are regression values, not pins: the
pins are the closed forms and invariants of tests/test_oracle_*.py.

    python tests/golden/make_oracle_regression.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import classify as OC  # noqa: E402
from oracle import forces as OF  # noqa: E402
from oracle import helmholtz as OH  # noqa: E402
from oracle import membrane as OM  # noqa: E402
from oracle import solve as OS  # noqa: E402
from oracle.grid import Grid  # noqa: E402

PROBE = [0, 777, 2345, 4096, 9999]


def compute():
    out = {}
    f = synth.faces_tanh(22, 2.0)
    grid = Grid(f, f, f)
    mesh = synth.octa_sphere(3, (0.5, 0.48, 0.52), 0.22)
    ib, G = OC.classify(grid, [mesh])
    b = synth.rhs_divergence(f, f, f, 1)
    p, lam = OS.solve_sparse(grid, ib, G, b)
    out["closed"] = {"nghost": int(len(G)), "nsolid": int(np.sum(ib == 1)),
                     "ghost_cells_sum": int(np.sum(G.cell)), "weights_sum": float(np.sum(G.w)),
                     "lambda": float(lam), "p_probe": [float(p.ravel()[q]) for q in PROBE]}
    ps, flags, F = OF.surface_forces(grid, ib, [mesh], p)
    out["closed"]["force_total"] = [float(x) for x in F.sum(axis=0)]
    ub = synth.counter_normal(9, 0, np.arange(len(G)))
    u = OH.solve_closed(grid, ib, G, 1e-4, synth.smooth_field(f, f, f, 3), ub)
    out["closed"]["helmholtz_probe"] = [float(u.ravel()[q]) for q in PROBE]
    plate = synth.plate(0.3, nq_x=6, nq_y=4)
    _, M = OM.classify(grid, [plate])
    pm, gm, lm = OM.solve_sparse(grid, M, b)
    out["membrane"] = {"nentries": int(len(M)), "entry_keys_sum": int(np.sum(2 * M.cell + M.side)),
                       "p_probe": [float(pm.ravel()[q]) for q in PROBE]}
    ps, flags, F = OF.surface_forces(grid, None, [plate], pm)
    out["membrane"]["force_total"] = [float(x) for x in F.sum(axis=0)]
    return out


if __name__ == "__main__":
    with open(os.path.join(HERE, "oracle_regression.json"), "w") as fh:
        json.dump(compute(), fh, indent=1)
