"""Brute force on tiny grids: one midpoint-RK step evaluated in 50-digit decimal arithmetic,
straight from the definitions of section 4.1 (primitive recovery, MinBee faces, HLLC with
Davis wave speeds and the Toro-Spruce-Speares star state, AddFlux, the CFL dt), written here
independently of the oracle.  The oracle's FP64 step must agree to round-off; per-face fluxes
are compared too (oracle.fluxes).  The decimal evaluation shares nothing with the oracle but
the seeded input generator."""
import decimal
from decimal import Decimal as D

import numpy as np
import pytest

import oracle
from paper_1204_4779_gb300 import inputs

decimal.getcontext().prec = 50
GAMMA = D("1.4")


def dec(a):
    return np.vectorize(lambda x: D(float(x)), otypes=[object])(a)  # exact binary values


def prim_of_cons(u, dim):
    rho = u[0]
    v = [u[1 + a] / rho for a in range(dim)]
    kin = sum((u[1 + a] * v[a] for a in range(dim)), D(0))
    return [rho] + v + [(GAMMA - 1) * (u[dim + 1] - kin / 2)]


def cons_of_prim(w, dim):
    rho = w[0]
    v2 = sum((w[1 + a] * w[1 + a] for a in range(dim)), D(0))
    return [rho] + [rho * w[1 + a] for a in range(dim)] + [w[dim + 1] / (GAMMA - 1) + rho * v2 / 2]


def euler_flux(w, dim, ax):
    u = cons_of_prim(w, dim)
    un, p = w[1 + ax], w[dim + 1]
    return ([u[0] * un] + [u[1 + b] * un + (p if b == ax else D(0)) for b in range(dim)] +
            [un * (u[dim + 1] + p)])


def minbee(a, b):
    if a * b <= 0:
        return D(0)
    return a if abs(a) < abs(b) else b


def hllc(wl, wr, dim, ax):
    rl, ul, pl = wl[0], wl[1 + ax], wl[dim + 1]
    rr, ur, pr = wr[0], wr[1 + ax], wr[dim + 1]
    al, ar = (GAMMA * pl / rl).sqrt(), (GAMMA * pr / rr).sqrt()
    sl, sr = min(ul - al, ur - ar), max(ul + al, ur + ar)
    ss = (pr - pl + rl * ul * (sl - ul) - rr * ur * (sr - ur)) / (rl * (sl - ul) - rr * (sr - ur))
    fl, fr = euler_flux(wl, dim, ax), euler_flux(wr, dim, ax)
    if sl >= 0:
        return fl
    if ss < 0 and sr <= 0:
        return fr
    w, s = (wl, sl) if ss >= 0 else (wr, sr)
    r, u, p = w[0], w[1 + ax], w[dim + 1]
    uk, fk = cons_of_prim(w, dim), euler_flux(w, dim, ax)
    chi = r * (s - u) / (s - ss)
    star = ([chi] + [chi * (ss if b == ax else w[1 + b]) for b in range(dim)] +
            [chi * (uk[dim + 1] / r + (ss - u) * (ss + p / (r * (s - u))))])
    return [fk[k] + s * (star[k] - uk[k]) for k in range(dim + 2)]


def neighbour(idx, a, d, n, bc):
    j = list(idx)
    j[a] += d
    if bc[a] == 0:
        j[a] %= n[a]
    else:
        j[a] = min(max(j[a], 0), n[a] - 1)
    return tuple(j)


def fluxes(U, n, bc, dim):
    """F[a][idx] = flux through the low face of cell idx on axis a (idx may be n_a on axis a)."""
    cells = list(np.ndindex(*n))
    W = {c: prim_of_cons([U[k][c] for k in range(dim + 2)], dim) for c in cells}
    F = []
    for a in range(dim):
        def face_state(c, side):  # MinBee face value of cell c: side +1 upper, -1 lower
            wm, w0, wp = W[neighbour(c, a, -1, n, bc)], W[c], W[neighbour(c, a, +1, n, bc)]
            return [w0[k] + side * minbee(w0[k] - wm[k], wp[k] - w0[k]) / 2 for k in range(dim + 2)]
        Fa = {}
        for c in cells:
            for hi in (False, True):
                if hi and c[a] != n[a] - 1:
                    continue
                lo_cell = neighbour(c, a, -1, n, bc) if not hi else c
                up_cell = c if not hi else neighbour(c, a, +1, n, bc)
                key = c if not hi else tuple(c[b] + (1 if b == a else 0) for b in range(dim))
                Fa[key] = hllc(face_state(lo_cell, +1), face_state(up_cell, -1), dim, a)
        F.append(Fa)
    return F


def rk_step(U, n, bc, dim, cfl):
    cells = list(np.ndindex(*n))
    dr = [D(1) / D(m) for m in n]
    smax = D(0)
    for c in cells:
        w = prim_of_cons([U[k][c] for k in range(dim + 2)], dim)
        cs = (GAMMA * w[dim + 1] / w[0]).sqrt()
        smax = max(smax, sum(((abs(w[1 + a]) + cs) / dr[a] for a in range(dim)), D(0)))
    dt = D(cfl) / smax

    def add(Ub, F, c_dt):
        out = [np.empty(n, dtype=object) for _ in range(dim + 2)]
        for c in cells:
            for k in range(dim + 2):
                s = D(0)
                for a in range(dim):
                    up = tuple(c[b] + (1 if b == a else 0) for b in range(dim))
                    s += c_dt / dr[a] * (F[a][c][k] - F[a][up][k])
                out[k][c] = Ub[k][c] + s
        return out

    U1 = add(U, fluxes(U, n, bc, dim), dt / 2)
    return add(U, fluxes(U1, n, bc, dim), dt), dt


def _case(shape, bc, seed):
    V = inputs.smooth(shape, seed=seed)
    U = oracle.prim_to_cons(V, 1.4)
    dim = len(shape)
    n = tuple(reversed(U.shape[1:]))  # (nx, ny, ...) -> decimal arrays indexed (x, y, ...)
    Ud = [dec(U[k]).T for k in range(dim + 2)]
    return U, Ud, n, dim


@pytest.mark.parametrize("shape,bc", [((6,), (0,)), ((7,), (1,)), ((4, 3), (0, 1)), ((3, 4), (1, 0))])
def test_one_rk_step_matches_decimal_evaluation(shape, bc):
    U, Ud, n, dim = _case(shape, bc, seed=11)
    U2, t, steps, _ = oracle.run(U, 1.4, 0.4, 1, bc=bc, threads=1)
    Dd, dt = rk_step(Ud, n, bc, dim, "0.4")
    assert steps == 1 and abs(t - float(dt)) <= 1e-15 * float(dt)
    for k in range(dim + 2):
        ref = np.array([[float(x) for x in row] for row in np.atleast_2d(Dd[k].T)]).reshape(U2[k].shape)
        err = np.max(np.abs(U2[k] - ref)) / np.max(np.abs(ref))
        assert err <= 1e-13, (k, err)


@pytest.mark.parametrize("shape,bc", [((6,), (1,)), ((4, 3), (0, 0))])
def test_face_fluxes_match_decimal_evaluation(shape, bc):
    U, Ud, n, dim = _case(shape, bc, seed=12)
    F = oracle.fluxes(U, 1.4, bc=bc)
    Fd = fluxes(Ud, n, bc, dim)
    for a in range(dim):
        for key, fd in Fd[a].items():
            # oracle layout: (dim+2) planes of faces, face c - 1/2 of cell c, x fastest with the
            # face axis extended by one
            e = [n[b] + (1 if b == a else 0) for b in range(dim)]
            flat = 0
            for b in reversed(range(dim)):
                flat = flat * e[b] + key[b]
            got = [F[a][k].reshape(-1)[flat] for k in range(dim + 2)]
            for k in range(dim + 2):
                assert abs(got[k] - float(fd[k])) <= 1e-13 * max(1.0, abs(float(fd[k]))), (a, key, k)
