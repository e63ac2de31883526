"""Plain FP64 CPU reference of the paper's linear-wave example (section 2.3): the wave
equation f_tt = c^2 f_xx written as f_t = g, g_t = c^2 f_xx, advanced by Eqs. eqLWDiscF and
eqLWDiscG on a periodic grid, with the discrete energy audited every step.

TEST INFRASTRUCTURE ONLY (tests/ and the CPU-baseline leg of bench.py): the CUDA path is checked
against it; it shares no code with it.

    f^{n+1}[i] = f^n[i] + dt g^n[i]
    g^{n+1}[i] = g^n[i] + (c^2 dt / dx^2) (f^{n+1}[i+1] + f^{n+1}[i-1] - 2 f^{n+1}[i])
    E^{n+1}    = sum_i (1/2) (c^2 ((f^{n+1}[i+1] - f^{n+1}[i-1]) / (2 dx))^2
                              + ((g^n[i] + g^{n+1}[i]) / 2)^2) dx

The energy is the form the paper's listing computes and the continuous energy
int (c^2 f_x^2 + g^2)/2 dx discretises (the printed Eq. eqLWDE puts c^2 inside the square and
drops the 1/2, which the scheme does not conserve).
"""
from __future__ import annotations

import numpy as np


def step(f, g, c: float, dx: float, dt: float):
    """One step; returns (f1, g1, E1)."""
    f = np.asarray(f, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    f1 = f + dt * g
    fp = np.roll(f1, -1)   # f1[i+1]
    fm = np.roll(f1, 1)    # f1[i-1]
    g1 = g + (c * c * dt / (dx * dx)) * (fp + fm - 2.0 * f1)
    dfdx = (fp - fm) / (2.0 * dx)
    gm = (g + g1) / 2.0
    E1 = float(np.sum(0.5 * (c * c * dfdx * dfdx + gm * gm) * dx))
    return f1, g1, E1


def run(f, g, c: float, length: float, dt: float, n_steps: int):
    """n_steps steps on n = len(f) cells of [0, length); returns (f, g, energies)."""
    n = len(f)
    dx = length / n
    energies = []
    for _ in range(n_steps):
        f, g, E = step(f, g, c, dx, dt)
        energies.append(E)
    return f, g, np.array(energies)


def initial(n: int, length: float = 2.0 * np.pi):
    """The paper's initial condition f = sin x, g = cos 3x on [0, 2 pi)."""
    x = np.arange(n, dtype=np.float64) * (length / n)
    return np.sin(x), np.cos(3.0 * x)
