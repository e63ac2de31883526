"""Pins of the oracle's scheme options: first-order reconstruction (the order-1 branch of the
paper's interpolation listing) and the pressure-based HLLC wave speeds."""
import math

import numpy as np
import pytest

import exact_riemann as er
import oracle
from paper_1204_4779_gb300 import inputs

G = 1.4


def test_order1_on_a_moving_contact_is_the_upwind_recurrence():
    """Uniform u > 0 and p with any density profile: HLLC is exact upwinding of a contact and
    the order-1 faces are the cell values, so each RK stage is the first-order upwind update
    rho' = rho_base - c (u dt/dx) (rho - rho_left), c = 1/2 then 1 (the midpoint scheme)."""
    n = 40
    V = inputs.uniform((n,), rho=1.0, v=(0.6,), p=1.0)
    V[0] = 1.0 + 0.5 * np.sin(2 * np.pi * inputs.centres(n)) ** 2
    U = oracle.prim_to_cons(V, G)
    rho = V[0].copy()
    Ucur = U
    for _ in range(5):
        dt = oracle.cfl_dt(Ucur, G, 0.4)
        nu = 0.6 * dt * n
        r1 = rho - 0.5 * nu * (rho - np.roll(rho, 1))
        rho = rho - nu * (r1 - np.roll(r1, 1))
        Ucur, _, _, _ = oracle.run(Ucur, G, 0.4, 1, bc=(0,), order=1)
    assert np.max(np.abs(Ucur[0] - rho)) <= 1e-13
    assert np.max(np.abs(oracle.cons_to_prim(Ucur, G)[2] - 1.0)) <= 1e-13  # p stays uniform


def test_order1_converges_at_first_order():
    errs = []
    for n in (64, 128, 256):
        V = inputs.entropy_wave((n,))
        U2, *_ = oracle.run(oracle.prim_to_cons(V, G), G, 0.4, 10 ** 6, bc=(0,), t_end=1.0,
                            order=1)
        errs.append(np.mean(np.abs(oracle.cons_to_prim(U2, G)[0] - V[0])))
    orders = [math.log2(a / b) for a, b in zip(errs, errs[1:])]
    assert all(0.75 < o < 1.25 for o in orders), orders
    # and order 2 is far more accurate at the same resolution
    V = inputs.entropy_wave((128,))
    U2, *_ = oracle.run(oracle.prim_to_cons(V, G), G, 0.4, 10 ** 6, bc=(0,), t_end=1.0)
    assert np.mean(np.abs(oracle.cons_to_prim(U2, G)[0] - V[0])) < 0.2 * errs[1]


def _rand_state(rng, dim):
    return np.concatenate([[rng.uniform(0.2, 3.0)], rng.uniform(-1, 1, dim),
                           [rng.uniform(0.2, 3.0)]])


def test_pressure_based_speeds_special_cases():
    rng = np.random.default_rng(4)
    for _ in range(50):  # consistency: equal states give the Euler flux
        V = _rand_state(rng, 2)
        assert np.allclose(oracle.hllc(2, 0, G, V, V, riemann=1), oracle.euler_flux(2, 0, G, V),
                           rtol=1e-13, atol=1e-13)
    for u in (0.3, -0.4):  # an isolated contact is still resolved exactly
        VL = np.array([1.0, u, 0.2, 0.8])
        VR = np.array([0.3, u, -0.5, 0.8])
        up = VL if u > 0 else VR
        assert np.allclose(oracle.hllc(2, 0, G, VL, VR, riemann=1), oracle.euler_flux(2, 0, G, up),
                           rtol=1e-14, atol=1e-14)


def test_pressure_based_speeds_sod_against_exact_solution():
    n = 1024
    U = oracle.prim_to_cons(inputs.sod_1d(n), G)
    U2, t, _, _ = oracle.run(U, G, 0.4, 10 ** 6, bc=(1,), t_end=0.2, riemann=1)
    assert t == 0.2
    V2 = oracle.cons_to_prim(U2, G)
    ex = er.cell_averages((1, 0, 1), (0.125, 0, 0.1), G, n, 0.2, sub=8)
    e = float(np.mean(np.abs(V2[0] - ex[0])))
    assert e < 1.2e-3
    D, *_ = oracle.run(U, G, 0.4, 10 ** 6, bc=(1,), t_end=0.2)
    assert not np.array_equal(D, U2)  # the option changes the flux


def test_pressure_based_speeds_conserve_and_keep_symmetry():
    V = inputs.blast_3d(10, radius_cells=3.0)
    U = oracle.prim_to_cons(V, G)
    A, *_ = oracle.run(U, G, 0.4, 6, bc=(0, 0, 0), riemann=1, order=1)
    T0, T1 = oracle.totals(U), oracle.totals(A)
    assert abs(T1[0] - T0[0]) <= 1e-13 * T0[0] and abs(T1[4] - T0[4]) <= 1e-13 * T0[4]
    M = A[:, ::-1].copy()
    M[3] = -M[3]
    assert np.max(np.abs(A - M)) <= 1e-12 * np.max(np.abs(A))


def test_bad_options_are_rejected():
    U = oracle.prim_to_cons(inputs.sod_1d(16), G)
    with pytest.raises(oracle.OracleError):
        oracle.run(U, G, 0.4, 1, bc=(1,), order=3)
