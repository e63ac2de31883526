"""Plant plausible mistakes in a copy of the oracle's C source and check that the pins
catch every one of them (a dropped term, a wrong sign, a wrong index, a transposed operand).

The mutated copies are compiled into a temporary directory; the oracle under test is never
modified.
"""
import math
import os

import numpy as np
import pytest

import exact_riemann as er
import oracle
from paper_1204_4779_gb300 import inputs

SRC = os.path.join(os.path.dirname(oracle.__file__), "hydro_oracle.c")
G = 1.4

# (name, text in hydro_oracle.c, replacement)
MUTANTS = [
    ("addflux_sign", "sum += coef[a] * (fm - fp);", "sum += coef[a] * (fp - fm);"),
    ("energy_star_term_dropped", "(Ss - u) * (Ss + p / (r * (S - u)))", "(Ss - u) * Ss"),
    ("wave_speed_sign", "SL = fmin(ul - al, ur - ar);", "SL = fmin(ul - al, ur + ar);"),
    ("limiter_picks_larger", "else if (fabs(dy01) < fabs(dy12))", "else if (fabs(dy01) > fabs(dy12))"),
    ("limiter_no_extremum_clip", "if (dy01 * dy12 < 0.0)", "if (dy01 * dy12 < -1e300)"),
    ("face_values_swapped", "*left = y1 - 0.5 * dy;", "*left = y1 + 0.5 * dy;"),
    ("rk_stage2_from_U1", "add_flux(W, dt, U, U);", "add_flux(W, dt, U1, U);"),
    ("rk_stage1_full_dt", "add_flux(W, 0.5 * dt, U, U1);", "add_flux(W, dt, U, U1);"),
    ("pressure_kinetic_factor", "(U[dim + 1] - 0.5 * kin)", "(U[dim + 1] - kin)"),
    ("momentum_flux_no_pressure", "(b == a ? p : 0.0)", "0.0"),
    ("energy_flux_no_pressure", "F[dim + 1] = un * (U[dim + 1] + p);", "F[dim + 1] = un * U[dim + 1];"),
    ("tangential_star_momentum", "chi * (b == a ? Ss : V[1 + b])", "chi * Ss"),
    ("periodic_ghost_shift", "src[a] = wrap(ia, G->n[a]);", "src[a] = wrap(ia + 1, G->n[a]);"),
    ("cfl_no_sound_speed", "s += (fabs(v[1 + a]) + cs) / G->dr[a];", "s += (fabs(v[1 + a]) + 0.3 * cs) / G->dr[a];"),
    ("cell_size_wrong_axis", "coef[a] = dt / G->dr[a];", "coef[a] = dt / G->dr[0];"),
    ("star_contact_speed_sign", "(pr - pl + rl * ul * (SL - ul) - rr * ur * (SR - ur))",
     "(pl - pr + rl * ul * (SL - ul) - rr * ur * (SR - ur))"),
    ("hllc_side_choice", "int left = 0.0 <= Ss;", "int left = 0.0 <= -Ss;"),
    ("analytic_stage2_time", "flux_all_axes(W, U1, t + 0.5 * dt);", "flux_all_axes(W, U1, t);"),
    ("analytic_phase_sign", "sin(2.0 * pi * (s - t))", "sin(2.0 * pi * (s + t))"),
    ("analytic_rotation_sign", "(y - 0.5) * sn + 0.5", "(y - 0.5) * -sn + 0.5"),
    ("analytic_ghost_centre", "double x = (i0 + 0.5) * G->dr[0];", "double x = (i0 + 1.0) * G->dr[0];"),
    ("analytic_sound_pressure", "V[dim + 1] = 1.0 + G->gamma * A * w;", "V[dim + 1] = 1.0 + A * w;"),
    ("sod_fan_sound_speed", "double c = q * (xi - u);", "double c = q * (u - xi);"),
    ("sod_contact_side", "int right = xi > us;", "int right = xi > 0.0;"),
    ("sod_shock_density", "out[0] = K[0] * (r + m) / (m * r + 1.0)", "out[0] = K[0] * (r + m) / (r + 1.0)"),
    ("sod_rarefaction_tail", "double tail = us + q * astar;", "double tail = us + q * a;"),
    ("outflow_second_cell", "src[a] = ia < 0 ? 0 : G->n[a] - 1;", "src[a] = ia < 0 ? 1 : G->n[a] - 2;"),
    ("cons_energy_kinetic_factor", "V[dim + 1] / (gamma - 1.0) + 0.5 * rho * v2;",
     "V[dim + 1] / (gamma - 1.0) + rho * v2;"),
    ("clip_compares_t_end_with_dt", "if (t_end > 0.0 && dt >= t_end - t) {", "if (t_end > 0.0 && dt >= t_end) {"),
    ("totals_volume_axis", "vol *= dr[a];", "vol *= dr[0];"),
]


def _battery():
    """Quick pins; returns the names of those that fail."""
    fails = []

    def check(name, fn):
        try:
            ok = fn()
        except Exception:
            ok = False
        if not ok:
            fails.append(name)

    def sod():
        n = 256
        U = oracle.prim_to_cons(inputs.sod_1d(n), G)
        U2, t, _, rc = oracle.run(U, G, 0.4, 10 ** 6, bc=(1,), t_end=0.2, check=False)
        if rc:
            return False
        V2 = oracle.cons_to_prim(U2, G)
        ex = er.cell_averages((1, 0, 1), (0.125, 0, 0.1), G, n, 0.2, sub=4)
        return np.mean(np.abs(V2[0] - ex[0])) < 3.3e-3

    def entropy():
        errs = []
        for n in (32, 64):
            V = inputs.entropy_wave((n,))
            U2, *_ = oracle.run(oracle.prim_to_cons(V, G), G, 0.4, 10 ** 6, bc=(0,), t_end=1.0,
                                check=False)
            errs.append(np.mean(np.abs(oracle.cons_to_prim(U2, G)[0] - V[0])))
        return errs[1] < 2.2e-2 and math.log2(errs[0] / errs[1]) > 1.4

    def ywave():
        V = inputs.entropy_wave((8, 32), k=(0, 1), v=(0.0, 1.0))
        U2, *_ = oracle.run(oracle.prim_to_cons(V, G), G, 0.4, 10 ** 6, bc=(0, 0), t_end=1.0,
                            check=False)
        return np.mean(np.abs(oracle.cons_to_prim(U2, G)[0] - V[0])) < 0.12

    def contact():
        V = inputs.uniform((16, 16), rho=1.0, v=(0.0, 0.0), p=1.0)
        x = inputs.centres(16)
        V[0][:, x > 0.5] = 0.25
        V[2][:, x > 0.5] = 0.7
        U = oracle.prim_to_cons(V, G)
        U2, *_ = oracle.run(U, G, 0.4, 10, bc=(1, 0), check=False)
        return np.max(np.abs(U2 - U)) < 1e-14

    def consistency():
        rng = np.random.default_rng(0)
        for _ in range(20):
            V = np.concatenate([[rng.uniform(0.2, 3)], rng.uniform(-1, 1, 2), [rng.uniform(0.2, 3)]])
            for a in range(2):
                if not np.allclose(oracle.hllc(2, a, G, V, V), oracle.euler_flux(2, a, G, V),
                                   rtol=1e-13, atol=1e-13):
                    return False
        return True

    def moving_contact():
        VL = np.array([1.0, 0.3, 0.2, 0.8])
        VR = np.array([0.3, 0.3, -0.5, 0.8])
        return np.allclose(oracle.hllc(2, 0, G, VL, VR), oracle.euler_flux(2, 0, G, VL),
                           rtol=1e-14, atol=1e-14)

    def euler_def():
        V = np.array([2.0, 0.5, -0.25, 3.0])
        E = 3.0 / 0.4 + 0.5 * 2.0 * (0.25 + 0.0625)
        want = [1.0, 0.5 + 3.0, -0.25, 0.5 * (E + 3.0)]
        return np.allclose(oracle.euler_flux(2, 0, G, V), want, rtol=1e-15, atol=0)

    def star_rh():
        from test_oracle_pins import star_rh_residual
        rng = np.random.default_rng(5)
        for _ in range(40):
            VL = np.array([rng.uniform(0.2, 3), rng.uniform(-0.3, 0.5), rng.uniform(-1, 1),
                           rng.uniform(0.2, 3)])
            VR = np.array([rng.uniform(0.2, 3), rng.uniform(-0.5, 0.3), rng.uniform(-1, 1),
                           rng.uniform(0.2, 3)])
            res, Ss = star_rh_residual(VL, VR)
            if Ss >= 0 and res > 1e-12:
                return False
        return True

    def limiter():
        from test_oracle_pins import sawtooth_overshoot
        return (oracle.interpolate(1.0, 3.0, 2.0) == (3.0, 3.0)
                and oracle.interpolate(0.0, 1.0, 5.0) == (0.5, 1.5)
                and sawtooth_overshoot() <= 1e-14)

    def cfl():
        U = oracle.prim_to_cons(inputs.sod_1d(64), G)
        return abs(oracle.cfl_dt(U, G, 0.4) - 0.4 / (math.sqrt(1.4) * 64)) < 1e-15

    def conservation():
        U = oracle.prim_to_cons(inputs.smooth((13, 9), seed=1), G)
        U2, *_ = oracle.run(U, G, 0.4, 10, bc=(0, 0), check=False)
        T0, T1 = oracle.totals(U), oracle.totals(U2)
        return abs(T1[0] - T0[0]) < 1e-13 * T0[0] and abs(T1[4] - T0[4]) < 1e-13 * T0[4]

    def analytic():
        from test_oracle_analytic_bc import analytic_upwind_residual
        if analytic_upwind_residual((12, 10)) > 1e-13:
            return False
        # sound wave at 60 degrees: second-order accurate with exact inflow and outflow values
        n, A = 32, 1e-5
        V = inputs.oblique_wave((n, n), "sound", math.pi / 3, amp=A)
        U2, *_ = oracle.run(oracle.prim_to_cons(V, G), G, 0.4, 10 ** 6, bc=(2, 2), t_end=0.25,
                            analytic=(oracle.ANALYTIC_SOUND_WAVE, math.pi / 3, A), check=False)
        E = inputs.oblique_wave((n, n), "sound", math.pi / 3, t=0.25, amp=A)
        if np.mean(np.abs(oracle.cons_to_prim(U2, G)[0] - E[0])) >= 1.7e-2 * A:
            return False
        from test_oracle_analytic_bc import sod_sample_deviation
        return sod_sample_deviation() <= 1e-13

    def totals():
        from test_oracle_pins import test_totals_closed_form
        test_totals_closed_form()
        return True

    def bruteforce():
        # one RK step on tiny outflow grids against the 50-digit evaluation of the definitions
        from test_oracle_bruteforce import test_one_rk_step_matches_decimal_evaluation as t
        t((7,), (1,))
        t((3, 4), (1, 0))
        return True

    for name, fn in [("totals", totals), ("bruteforce", bruteforce), ("sod", sod), ("entropy", entropy), ("ywave", ywave), ("contact", contact),
                     ("consistency", consistency), ("moving_contact", moving_contact),
                     ("euler_def", euler_def), ("star_rh", star_rh), ("limiter", limiter), ("cfl", cfl), ("conservation", conservation),
                     ("analytic", analytic)]:
        check(name, fn)
    return fails


def test_unmutated_oracle_passes_the_battery():
    assert _battery() == []


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(name, old, new, tmp_path):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    mutated = tmp_path / "mutant.c"
    mutated.write_text(src.replace(old, new))
    lib = oracle.build(force=True, src=str(mutated), out=str(tmp_path / "libmutant.so"))
    with oracle.using_library(lib):
        fails = _battery()
    assert fails, f"mutant {name} survived every pin"
