"""Grids at the library's size limits (2^31 - 1024 cells on an axis, fewer than 2^31 cells in
all): the index arithmetic of the stage,
CFL and totals kernels must not overflow.  A uniform periodic state with one perturbed cell at
the very end of the grid is stepped; the perturbation reaches at most a few cells in a few
steps (and wraps around the periodic ends), and every cell it reaches must hold exactly what
the same local problem gives on a small grid (the same kernels do the same arithmetic on the
same values; the dt of both runs comes from the same extreme cell), while the uniform rest of
the grid stays bitwise unchanged."""
import numpy as np
import pytest

from paper_1204_4779_gb300 import hydro

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
F32 = torch.float32
G = 1.4


def _uniform_with_bump(shape, bump_index):
    """Conserved FP32 planes: rho = 1, v = 0, p = 1 everywhere; rho = 1.5, p = 3 in one cell."""
    dim = len(shape)
    U = torch.zeros((dim + 2,) + tuple(reversed(shape)), dtype=F32, device="cuda")
    U[0].fill_(1.0)
    U[dim + 1].fill_(1.0 / (G - 1.0))
    flat0, flatE = U[0].view(-1), U[dim + 1].view(-1)
    flat0[bump_index] = 1.5
    flatE[bump_index] = 3.0 / (G - 1.0)
    return U


def _run(shape, bump_index, steps, dx):
    """Periodic run on a box of cell size dx on every axis (the same dx for the big and the small
    grid, so that both take the same dt)."""
    U = _uniform_with_bump(shape, bump_index)
    S = hydro.Solver(shape, G, bc="periodic", dtype=F32, cfl=0.4, lo=[0.0] * len(shape),
                     hi=[n * dx for n in shape])
    t, n = S.step(U, steps)
    T = S.totals(U)
    S.close()
    return U, t, n, T


def test_one_dimensional_grid_at_the_axis_limit():
    n = (1 << 31) - 1024
    big, tb, nb, Tb = _run((n,), n - 1, 3, 1.0 / 64)
    small, ts, ns, _ = _run((64,), 63, 3, 1.0 / 64)
    assert nb == ns == 3 and tb == ts
    w = 12  # cells the bump can reach in 3 steps (two per stage and side)
    for k in range(big.shape[0]):
        b, s = big[k], small[k]
        assert torch.equal(b[n - w:], s[64 - w:]), k
        assert torch.equal(b[:w], s[:w]), k
        mid = b[w:n - w]
        assert bool((mid == mid[0]).all()), k  # the rest is still the uniform state
    # the FP64 mass: n cells of density 1 and the bump's extra 0.5, times dx
    assert abs(Tb[0] - (n + 0.5) / 64) < 1e-6 * n / 64


def test_three_dimensional_grid_just_below_2_31_cells():
    m = 1290  # 1290^3 = 2,146,689,000 < 2^31
    last = m ** 3 - 1
    s = 24
    big, tb, nb, _ = _run((m, m, m), last, 2, 1.0 / s)
    small, ts, ns, _ = _run((s, s, s), s ** 3 - 1, 2, 1.0 / s)
    assert nb == ns == 2 and tb == ts
    w = 8  # cells the bump can reach in 2 steps
    idx_b = np.r_[0:w, m - w:m]
    idx_s = np.r_[0:w, s - w:s]
    ib = torch.as_tensor(idx_b, device="cuda")
    is_ = torch.as_tensor(idx_s, device="cuda")
    for k in range(5):
        cb = big[k].index_select(0, ib).index_select(1, ib).index_select(2, ib)
        cs = small[k].index_select(0, is_).index_select(1, is_).index_select(2, is_)
        assert torch.equal(cb, cs), k
        # far from the bump the state is untouched
        assert bool((big[k][m // 2, m // 3:m // 3 + 64, :] == big[k][m // 2, m // 3, 0]).all()), k
