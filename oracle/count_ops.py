"""Floating-point operations per cell-update of one RK step, as the oracle performs them
(test infrastructure; writes profiles/oracle_opcounts.json, which the benchmark reads for its
FP32 roofline).

    python oracle/count_ops.py

The counting build (opcount.cpp) runs the oracle's own code with a counting number type, so
the figures are the oracle's evaluation of section 4.1 for one midpoint-RK step: the CFL
signal of the step's initial state, and for each of the two stages the primitive recovery on
interior and ghost cells, the MinBee interpolation of every cell on every axis, HLLC on every
face (both physical fluxes evaluated) and AddFlux.  The oracle's positivity check after the
step (primitive recovery and two compares per cell) is not part of the method and is taken
out exactly.  Counts depend slightly on the data (HLLC and MinBee branches), so the workload
is the benchmark's: the 3D periodic blast (rho = 1, p = 1e-3, p = 10 within 8 cells of the
centre, gamma = 1.4, CFL 0.4), here at 64^3.
"""
from __future__ import annotations

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1204_4779_gb300 import inputs  # noqa: E402

OUT = os.path.join(ROOT, "profiles", "oracle_opcounts.json")


def per_cell_update(V: np.ndarray, gamma: float, cfl: float, bc) -> dict:
    """Counts by kind per cell-update of one RK step on primitive data V."""
    U = oracle.prim_to_cons(V, gamma)
    ncell = int(np.prod(V.shape[1:]))
    with oracle.counting_ops() as counts:
        U1, _, steps, _ = oracle.run(U, gamma, cfl, 1, bc=bc, threads=1)
        step = counts()
    assert steps == 1
    with oracle.counting_ops() as counts:  # the positivity check's recovery, on the same state
        oracle.cons_to_prim(U1, gamma)
        check = counts()
    check["cmp"] += 2 * ncell
    out = {k: (step[k] - check[k]) / ncell for k in oracle.OP_KINDS}
    out["total"] = sum(out[k] for k in oracle.OP_KINDS)
    return out


def main():
    n = 64
    V = inputs.blast_3d(n, radius_cells=8.0)
    ops = per_cell_update(V, 1.4, 0.4, (0, 0, 0))
    rec = {
        "workload": f"3D periodic {n}^3 blast (radius 8 cells), gamma 1.4, CFL 0.4, one RK step",
        "unit": "floating-point operations per cell-update per RK step (add/sub, mul, div, sqrt,"
                " compare, min/max, abs, negate each count one)",
        "per_cell_update": {k: round(v, 3) for k, v in ops.items()},
        "excluded": "the oracle's positivity check after the step",
        "command": "python oracle/count_ops.py",
    }
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(json.dumps(rec, indent=1))


if __name__ == "__main__":
    main()
