"""Plant plausible mistakes in a copy of the linear-wave oracle's source and check that the pins
of test_wave_oracle.py (energy conservation, second-order convergence to d'Alembert's solution
with g at half steps, one step evaluated by hand) catch every one of them.  The oracle under
test is never modified: each mutated copy is executed as a module of its own."""
import math
import os
import types

import numpy as np
import pytest

import oracle

SRC = os.path.join(os.path.dirname(oracle.__file__), "wave_oracle.py")
C = 3.43

MUTANTS = [
    ("f_update_sign", "f1 = f + dt * g", "f1 = f - dt * g"),
    ("laplacian_of_old_f", "(fp + fm - 2.0 * f1)", "(fp + fm - 2.0 * f)"),
    ("coefficient_without_c", "(c * c * dt / (dx * dx))", "(c * dt / (dx * dx))"),
    ("energy_g_not_averaged", "gm = (g + g1) / 2.0", "gm = g1"),
    ("energy_one_sided_derivative", "dfdx = (fp - fm) / (2.0 * dx)", "dfdx = (fp - f1) / dx"),
    ("neighbour_index", "fp = np.roll(f1, -1)", "fp = np.roll(f1, 1)"),
]


def _module(src: str):
    m = types.ModuleType("wave_oracle_mutant")
    exec(compile(src, "wave_oracle_mutant", "exec"), m.__dict__)
    return m


def _battery(W) -> list:
    with np.errstate(all="ignore"):  # a mutant may overflow; that fails a pin below
        return _pins(W)


def _pins(W) -> list:
    fails = []
    # energy conserved to round-off
    n = 64
    f, g = W.initial(n)
    dx = 2 * math.pi / n
    _, _, E = W.run(f, g, C, 2 * math.pi, dx / C, 400)
    if not ((E.max() - E.min()) / E.mean() < 1e-12):
        fails.append("energy")
    # second order with g at half steps
    errs = []
    for n in (64, 128, 256):
        dx = 2 * math.pi / n
        dt = 0.5 * dx / C
        steps = int(round(0.5 / dt))
        x = np.arange(n) * dx
        f, g = W.initial(n)
        th = dt / 2
        g = -C * np.sin(x) * np.sin(C * th) + np.cos(3 * x) * np.cos(3 * C * th)
        f, g, _ = W.run(f, g, C, 2 * math.pi, dt, steps)
        t = steps * dt
        exact = np.sin(x) * np.cos(C * t) + np.cos(3 * x) * np.sin(3 * C * t) / (3 * C)
        errs.append(float(np.max(np.abs(f - exact))))
    orders = [math.log2(a / b) if b > 0 else 0.0 for a, b in zip(errs, errs[1:])]
    if not (min(orders) > 1.9 and errs[-1] < 1e-3):
        fails.append("convergence")
    # one step by hand: f1 = f + dt g; g1[1] = 0 + (4 * 0.1 / 0.25) (0 + 0.1 - 2)
    f1, g1, _ = W.step(np.array([0.0, 1.0, 0.0, 0.0]), np.array([1.0, 0.0, 0.0, -1.0]), 2.0,
                       0.5, 0.1)
    if not (np.allclose(f1, [0.1, 1.0, 0.0, -0.1]) and abs(g1[1] - 1.6 * (0.1 - 2.0)) < 1e-14):
        fails.append("by_hand")
    return fails


def test_unmutated_wave_oracle_passes_the_battery():
    assert _battery(_module(open(SRC).read())) == []


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    assert _battery(_module(src.replace(old, new))), f"mutant {name} survived every pin"
