"""Pins of the oracle's analytic-solution boundaries (the convergence tests of section 4.3: the
exact solution is substituted into the ghost layers at the time of each RK stage, so a wave can
cross a box that is not periodic along it, e.g. at 60 degrees to the x axis on the unit square).

The pins are independent of the oracle's own formulas: the order-1 scheme on a contact flow is
the first-order upwind recurrence, which a few lines of numpy run with the exact inflow values;
a uniform state equal to the boundary solution stays uniform; the second-order scheme converges
to the exact solution of inputs.oblique_wave."""
import math

import numpy as np
import pytest

import oracle
from paper_1204_4779_gb300 import inputs

G = 1.4
THETA60 = math.pi / 3


def _exact_rho(x, y, t, theta):
    """Density of the entropy wave at (x, y, t): 2 + sin(2 pi (s - t))."""
    s = (x - 0.5) * math.cos(theta) + (y - 0.5) * math.sin(theta) + 0.5
    return 2.0 + np.sin(2.0 * math.pi * (s - t))


def analytic_upwind_residual(n=(12, 10), theta=THETA60, steps=4):
    """Max |rho_oracle - rho_upwind| after `steps` order-1 steps of the entropy wave with analytic
    boundaries.  With uniform velocity (u, v) = (cos theta, sin theta) >= 0 and uniform pressure,
    HLLC is exact upwinding and each midpoint stage is
        rho' = rho_base - c dt (u (rho - rho_west) / dx + v (rho - rho_south) / dy),
    c = 1/2 at time t, then 1 at time t + dt/2; the west and south neighbours of the first
    column and row are the exact solution at the ghost-cell centres at the stage's time.  Works
    in 1D too (n of length 1: the line y = 1/2, no south term)."""
    dim = len(n)
    V = inputs.oblique_wave(n, "entropy", theta)
    U = oracle.prim_to_cons(V, G)
    nx = n[0]
    ny = n[1] if dim == 2 else 1
    dx, dy = 1.0 / nx, 1.0 / ny
    xc = (np.arange(nx) + 0.5) * dx
    yc = (np.arange(ny) + 0.5) * dy if dim == 2 else np.array([0.5])
    u, v = math.cos(theta), math.sin(theta)
    assert u >= 0 and v >= 0
    rho = V[0].reshape(ny, nx).copy()
    t = 0.0

    def rate(r, ts):
        west = np.concatenate([_exact_rho(-0.5 * dx, yc, ts, theta)[:, None], r[:, :-1]], axis=1)
        out = u * (r - west) / dx
        if dim == 2:
            south = np.concatenate([_exact_rho(xc, -0.5 * dy, ts, theta)[None, :], r[:-1, :]], axis=0)
            out = out + v * (r - south) / dy
        return out

    Ucur = U
    for _ in range(steps):
        dt = oracle.cfl_dt(Ucur, G, 0.4)
        r1 = rho - 0.5 * dt * rate(rho, t)
        rho = rho - dt * rate(r1, t + 0.5 * dt)
        Ucur, t2, _, _ = oracle.run(Ucur, G, 0.4, 1, bc=(2,) * dim, t0=t, order=1,
                                    analytic=(oracle.ANALYTIC_ENTROPY_WAVE, theta, 1.0),
                                    check=False)
        t = t + dt
        assert abs(t2 - t) <= 1e-15
    return float(np.max(np.abs(Ucur[0].reshape(ny, nx) - rho)))


@pytest.mark.parametrize("n,theta", [((16,), 0.0), ((12, 10), THETA60), ((9, 13), math.pi / 7),
                                     ((10, 10), 0.0)])
def test_order1_inflow_is_the_upwind_recurrence_with_exact_ghosts(n, theta):
    assert analytic_upwind_residual(n, theta) <= 1e-13


def test_uniform_state_equal_to_the_boundary_solution_stays_uniform():
    """The sound wave of amplitude 0 is rho = gamma, v = 0, p = 1 everywhere; a wrong field
    order or a wrong conversion in the ghost cells would disturb the first cells."""
    for n, bc in (((20,), (2,)), ((11, 7), (2, 2)), ((11, 7), (2, 0)), ((11, 7), (1, 2))):
        V = inputs.oblique_wave(n, "sound", 0.4, amp=0.0)
        U = oracle.prim_to_cons(V, G)
        U2, t, done, _ = oracle.run(U, G, 0.4, 5, bc=bc,
                                    analytic=(oracle.ANALYTIC_SOUND_WAVE, 0.4, 0.0))
        assert done == 5 and t > 0
        assert np.max(np.abs(U2 - U)) <= 1e-14


@pytest.mark.parametrize("kind,theta", [("entropy", 0.0), ("entropy", THETA60), ("sound", 0.0),
                                        ("sound", THETA60)])
def test_converges_to_the_exact_solution_at_second_order(kind, theta):
    """Mean |rho - rho_exact| / amp at t = 1/4 on 16^2, 32^2, 64^2 with analytic boundaries on
    both axes (measured orders 1.55-1.81: MinBee clips the extrema to first order)."""
    amp = 1.0 if kind == "entropy" else 1e-5
    ana = (oracle.ANALYTIC_ENTROPY_WAVE if kind == "entropy" else oracle.ANALYTIC_SOUND_WAVE,
           theta, amp)
    errs = []
    for n in (16, 32, 64):
        V = inputs.oblique_wave((n, n), kind, theta, amp=amp)
        U2, t, _, _ = oracle.run(oracle.prim_to_cons(V, G), G, 0.4, 10 ** 6, bc=(2, 2),
                                 t_end=0.25, analytic=ana, threads=4)
        assert t == 0.25
        E = inputs.oblique_wave((n, n), kind, theta, t=0.25, amp=amp)
        errs.append(float(np.mean(np.abs(oracle.cons_to_prim(U2, G)[0] - E[0]))) / amp)
    orders = [math.log2(a / b) for a, b in zip(errs, errs[1:])]
    assert errs[-1] < 6.5e-3, errs
    assert orders[0] > 1.45 and orders[1] > 1.7, orders


def test_coaxial_wave_matches_the_periodic_run_to_the_discretisation_error():
    """With theta = 0 the box is periodic along the wave, so the periodic run and the analytic
    run approximate the same solution; their difference is below the error of either."""
    n = 64
    V = inputs.oblique_wave((n,), "entropy", 0.0)
    U = oracle.prim_to_cons(V, G)
    A, *_ = oracle.run(U, G, 0.4, 10 ** 6, bc=(2,), t_end=0.5,
                       analytic=(oracle.ANALYTIC_ENTROPY_WAVE, 0.0, 1.0))
    P, *_ = oracle.run(U, G, 0.4, 10 ** 6, bc=(0,), t_end=0.5)
    E = inputs.oblique_wave((n,), "entropy", 0.0, t=0.5)[0]
    ea = np.mean(np.abs(A[0] - E))
    ep = np.mean(np.abs(P[0] - E))
    assert np.mean(np.abs(A[0] - P[0])) < 0.5 * max(ea, ep)
    assert ea < 2 * ep and ep < 2 * ea


def test_bad_boundary_options_are_rejected():
    U = oracle.prim_to_cons(inputs.oblique_wave((8, 8), "entropy", 0.0), G)
    with pytest.raises(oracle.OracleError):
        oracle.run(U, G, 0.4, 1, bc=(2, 0))  # analytic axis without a solution
    with pytest.raises(oracle.OracleError):
        oracle.run(U, G, 0.4, 1, bc=(2, 0), analytic=(4, 0.0, 1.0))
    with pytest.raises(oracle.OracleError):
        oracle.run(U, G, 0.4, 1, bc=(3, 0), analytic=(1, 0.0, 1.0))
    with pytest.raises(oracle.OracleError):
        oracle.fluxes(U, G, bc=(2, 0))


def sod_sample_deviation():
    """Max relative deviation of the oracle's exact Sod solution from the independent solver of
    exact_riemann.py over xi in [-3, 3] (every region: left state, fan, both star states,
    shocked state, right state)."""
    import exact_riemann as er
    worst = 0.0
    for xi in np.linspace(-3.0, 3.0, 1201):
        got, _ = oracle.sod_sample(G, xi)
        want = np.array(er.sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), G, xi))
        dev = float(np.max(np.abs(got - want) / np.maximum(1.0, np.abs(want))))
        worst = max(worst, dev if math.isfinite(dev) else math.inf)
    return worst


def test_shock_tube_solution_matches_the_independent_exact_solver():
    import exact_riemann as er
    assert sod_sample_deviation() <= 1e-13
    _, star = oracle.sod_sample(G, 0.0)
    ps, us, _, _ = er.star_state((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), G)
    assert abs(star[0] - ps) <= 1e-14 and abs(star[1] - us) <= 1e-14
    # Sod's star state for gamma = 1.4 (Toro, table 4.2 test 1): p* = 0.30313, u* = 0.92745
    assert abs(star[0] - 0.30313) < 5e-6 and abs(star[1] - 0.92745) < 5e-6


def _sod_exact_prim(n, theta, t):
    import exact_riemann as er
    xc = (np.arange(n) + 0.5) / n
    x, y = np.meshgrid(xc, xc)
    s = (x - 0.5) * math.cos(theta) + (y - 0.5) * math.sin(theta) + 0.5
    W = np.array([er.sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), G, xi)
                  for xi in ((s - 0.5) / t).ravel()]).T.reshape(3, n, n)
    return W


def test_oblique_shock_tube_with_analytic_boundaries():
    """Sod's tube at 60 degrees on the unit square to t = 0.125 (the section's test): the
    discontinuities cross the boundary at all times, so outflow boundaries disturb the solution
    there while the analytic ones do not; the analytic run converges at about first order (the
    rate of a solution with discontinuities) and is clearly closer to the exact solution."""
    th = THETA60
    ea, eo = [], []
    for n in (32, 64):
        U = oracle.prim_to_cons(inputs.oblique_wave((n, n), "shock_tube", th), G)
        A, t, _, _ = oracle.run(U, G, 0.4, 10 ** 6, bc=(2, 2), t_end=0.125,
                                analytic=(oracle.ANALYTIC_SHOCK_TUBE, th, 0.0), threads=4)
        O, *_ = oracle.run(U, G, 0.4, 10 ** 6, bc=(1, 1), t_end=0.125, threads=4)
        assert t == 0.125
        rho = _sod_exact_prim(n, th, 0.125)[0]
        ea.append(float(np.mean(np.abs(oracle.cons_to_prim(A, G)[0] - rho))))
        eo.append(float(np.mean(np.abs(oracle.cons_to_prim(O, G)[0] - rho))))
    assert ea[1] < 0.0115 and math.log2(ea[0] / ea[1]) > 0.7, ea
    assert ea[1] < 0.85 * eo[1], (ea, eo)
