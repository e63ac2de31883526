"""The operation-counting build of the oracle (oracle/opcount.cpp): it must compute exactly what
the plain build computes, and its counts must equal counts derived by hand from the oracle's
C source for single calls (MinBee interpolation, primitive recovery, one HLLC face).  The
counted figure per cell-update is the FP32 roofline's numerator in the benchmark."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1204_4779_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
Z = dict.fromkeys(oracle.OP_KINDS, 0)


def _expect(**kw):
    d = dict(Z)
    d.update(kw)
    return d


def test_interpolate_counts():
    # monotone: two differences, their product and its sign test, two magnitudes and their
    # comparison, then the two face values (half slope each)
    with oracle.counting_ops() as c:
        assert oracle.interpolate(0.0, 1.0, 2.0) == (0.5, 1.5)
        assert c() == _expect(add=4, mul=3, cmp=2, abs=2)
    # extremum: the sign test decides, no magnitudes compared
    with oracle.counting_ops() as c:
        assert oracle.interpolate(0.0, 1.0, 0.0) == (1.0, 1.0)
        assert c() == _expect(add=4, mul=3, cmp=1)


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_primitive_recovery_counts(dim):
    # per cell: dim divisions m_a / rho, dim products m_a v_a summed from 0 (dim adds), then
    # gamma - 1, E - kin/2 (two adds) and two products: (dim + 2) adds, (dim + 2) muls
    shape = (5, 4, 3)[:dim]
    U = oracle.prim_to_cons(inputs.smooth(shape, seed=dim), 1.4)
    n = int(np.prod(shape))
    with oracle.counting_ops() as c:
        oracle.cons_to_prim(U, 1.4)
        assert c() == _expect(add=(dim + 2) * n, mul=(dim + 2) * n, div=dim * n)


def test_hllc_star_face_counts():
    """1D face in the left star region, Davis speeds, counted from the source: both sides'
    conserved states (mul 4, add 3, div 1 each) and physical fluxes (which recompute the
    conserved state: mul 7, add 5, div 1 each), two sound speeds (mul, div, sqrt each), S_L and
    S_R (4 adds, 2 min/max), S* (add 8, mul 6, div 1), three branch tests, the star factor
    (add 2, mul 1, div 1), the star momentum (mul 1) and energy (add 4, mul 3, div 2), and
    F_K + S (U* - U_K) for three components (add 6, mul 3)."""
    VL, VR = np.array([1.0, 0.1, 1.0]), np.array([0.5, 0.0, 0.5])
    with oracle.counting_ops() as c:
        oracle.hllc(1, 0, 1.4, VL, VR)
        assert c() == _expect(add=40, mul=38, div=10, sqrt=2, cmp=3, minmax=2)


@pytest.mark.parametrize("riemann", [0, 1])
def test_counting_build_computes_the_same(riemann):
    for V, bc in ((inputs.blast_3d(10, radius_cells=3.0), (0, 0, 0)),
                  (inputs.kh_2d(24), (0, 1)), (inputs.sod_1d(64), (1,))):
        U = oracle.prim_to_cons(V, 1.4)
        A = oracle.run(U, 1.4, 0.4, 4, bc=bc, threads=1, riemann=riemann)
        with oracle.counting_ops():
            B = oracle.run(U, 1.4, 0.4, 4, bc=bc, threads=1, riemann=riemann)
        assert np.array_equal(A[0], B[0]) and A[1] == B[1] and A[2] == B[2]


def test_committed_counts_match_the_counting_script():
    import importlib.util
    spec = importlib.util.spec_from_file_location("count_ops", os.path.join(ROOT, "oracle", "count_ops.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    ops = mod.per_cell_update(inputs.blast_3d(64, radius_cells=8.0), 1.4, 0.4, (0, 0, 0))
    with open(os.path.join(ROOT, "profiles", "oracle_opcounts.json")) as f:
        rec = json.load(f)["per_cell_update"]
    for k, v in ops.items():
        assert abs(rec[k] - v) <= 1e-3 * max(1.0, v), k
    # a uniform state has no positivity-check or branch subtleties: the count per cell-update
    # is the same at any size up to the ghost-cell and extra-face terms, which shrink as 1/n
    per = []
    for n in (8, 16):
        per.append(mod.per_cell_update(inputs.uniform((n, n, n), rho=1.0, v=(0.1, 0.0, 0.0), p=1.0),
                                       1.4, 0.4, (0, 0, 0))["total"])
    assert per[1] < per[0] and (per[0] - per[1]) / per[1] < 0.5
