"""Pins of the linear-wave oracle (paper section 2.3): the discrete energy is conserved to
round-off for N = 8 ... 3072 (the paper reports fluctuations of order 1e-13), and the scheme is
the second-order leap-frog when g is read at half steps: started from g(dt/2) it converges at
second order to d'Alembert's solution f = sin x cos ct + cos 3x sin 3ct / (3c); started from
g(0), as in the paper's initial condition, the half-step offset leaves a first-order error."""
import math

import numpy as np

from oracle import wave_oracle as W

C = 3.43


def test_energy_is_conserved_to_round_off():
    for n in (8, 64, 512, 3072):
        f, g = W.initial(n)
        dx = 2 * math.pi / n
        _, _, E = W.run(f, g, C, 2 * math.pi, dx / C, 400)
        assert (E.max() - E.min()) / E.mean() < 1e-12, n


def _errors(staggered):
    errs = []
    T = 0.5
    for n in (64, 128, 256):
        dx = 2 * math.pi / n
        dt = 0.5 * dx / C
        steps = int(round(T / dt))
        x = np.arange(n) * dx
        f, g = W.initial(n)
        if staggered:  # g_t of the exact solution at t = dt/2
            th = dt / 2
            g = -C * np.sin(x) * np.sin(C * th) + np.cos(3 * x) * np.cos(3 * C * th)
        f, g, _ = W.run(f, g, C, 2 * math.pi, dt, steps)
        t = steps * dt
        exact = np.sin(x) * np.cos(C * t) + np.cos(3 * x) * np.sin(3 * C * t) / (3 * C)
        errs.append(np.max(np.abs(f - exact)))
    return [math.log2(a / b) for a, b in zip(errs, errs[1:])]


def test_second_order_leap_frog_with_staggered_g():
    orders = _errors(True)
    assert min(orders) > 1.9, orders


def test_first_order_offset_with_g_at_t0():
    orders = _errors(False)
    assert all(0.9 < o < 1.2 for o in orders), orders


def test_one_step_by_hand():
    f = np.array([0.0, 1.0, 0.0, 0.0])
    g = np.array([1.0, 0.0, 0.0, -1.0])
    f1, g1, E = W.step(f, g, 2.0, 0.5, 0.1)
    assert np.allclose(f1, [0.1, 1.0, 0.0, -0.1])
    k = 4.0 * 0.1 / 0.25
    want_g = g + k * (np.roll(f1, -1) + np.roll(f1, 1) - 2 * f1)
    assert np.allclose(g1, want_g)
    assert abs(want_g[1] - (0.0 + 1.6 * (0.0 + 0.1 - 2.0))) < 1e-15
