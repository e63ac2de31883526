"""Batched path (hydro_batch_*): many independent 2D grids of uneven size in one persistent
launch per RK stage.  Every grid is checked against the CPU oracle run on that grid alone:
FP64 max relative error <= 1e-10, FP32 L1 density error <= 1e-4; the full configuration
(4096 grids, sides log-uniform on [32, 512], 50 steps) in FP32 and in FP64 on a seeded sample
of grids, which the oracle computes one by one (grids do not interact)."""
import numpy as np
import pytest

import oracle
from _helpers import l1_rel, max_rel_err
from paper_1204_4779_gb300 import hydro, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
F32, F64 = torch.float32, torch.float64
G = 1.4

SMALL = [(1, 1), (3, 2), (33, 9), (64, 64), (70, 45), (17, 100), (40, 8), (128, 3), (5, 31),
         (96, 80)]


def _packed(B, Vs, dtype):
    P = np.concatenate([V.reshape(4, -1) for V in Vs], axis=1)
    U64 = hydro.prim_to_cons(torch.from_numpy(P).cuda().view(4, 1, -1), G).view(4, -1)
    return U64.to(dtype).contiguous()


def _oracle(V, bc, n, t_end=0.0):
    U = oracle.prim_to_cons(V, G)
    return oracle.run(U, G, 0.4, n, bc=bc, t_end=t_end, threads=oracle.max_threads())


def _data(shapes, seed):
    return [inputs.batch_grid(nx, ny, seed, i) for i, (nx, ny) in enumerate(shapes)]


@pytest.mark.parametrize("bc", [("periodic", (0, 0)), ("outflow", (1, 1))])
def test_small_batch_fp64_matches_oracle_per_grid(bc):
    Vs = _data(SMALL, 7)
    B = hydro.BatchSolver(SMALL, G, bc=bc[0], dtype=F64, cfl=0.4)
    U = _packed(B, Vs, F64)
    t, steps = B.step(U, 25)
    assert steps == [25] * len(SMALL)
    for g, V in enumerate(Vs):
        O, to, so, _ = _oracle(V, bc[1], 25)
        Gg = B.grid_view(U, g).cpu().numpy()
        assert t[g] == to, (g, t[g], to)
        assert max_rel_err(Gg, O) <= 1e-10, g


def test_small_batch_fp32_l1():
    Vs = _data(SMALL, 8)
    for tile in ((32, 8), (16, 16)):
        B = hydro.BatchSolver(SMALL, G, dtype=F32, tile=tile)
        U = _packed(B, Vs, F32)
        t, steps = B.step(U, 40)
        for g, V in enumerate(Vs):
            O, to, _, _ = _oracle(V, (0, 0), 40)
            Gg = B.grid_view(U, g).double().cpu().numpy()
            assert l1_rel(Gg[0], O[0]) <= 1e-5, (tile, g)
            assert abs(t[g] - to) <= 1e-5 * to


def test_per_grid_time_clipping_and_start_times():
    shapes = [(20, 20), (64, 32), (9, 50)]
    Vs = _data(shapes, 9)
    B = hydro.BatchSolver(shapes, G, dtype=F64)
    U = _packed(B, Vs, F64)
    t0 = [0.0, 0.01, 0.02]
    t, steps = B.step(U, 100000, t_end=0.05, t=t0)
    for g, V in enumerate(Vs):
        O, to, so, _ = oracle.run(oracle.prim_to_cons(V, G), G, 0.4, 100000, bc=(0, 0),
                                  t_end=0.05, t0=t0[g])
        assert t[g] == to == 0.05 and steps[g] == so
        assert max_rel_err(B.grid_view(U, g).cpu().numpy(), O) <= 1e-10


def test_totals_per_grid_and_conservation():
    Vs = _data(SMALL, 10)
    B = hydro.BatchSolver(SMALL, G, dtype=F64)
    U = _packed(B, Vs, F64)
    T0 = np.array(B.totals(U))
    for g in range(len(SMALL)):
        To = oracle.totals(B.grid_view(U, g).cpu().numpy())
        assert np.allclose(T0[g], To, rtol=1e-13, atol=1e-13 * abs(To[4]))
    B.step(U, 30)
    T1 = np.array(B.totals(U))
    assert np.all(np.abs(T1[:, 0] - T0[:, 0]) <= 1e-13 * T0[:, 0])
    assert np.all(np.abs(T1[:, 4] - T0[:, 4]) <= 1e-13 * T0[:, 4])


def test_nonfinite_grid_stops_alone():
    Vs = _data(SMALL[:4], 11)
    B = hydro.BatchSolver(SMALL[:4], G, dtype=F64)
    U = _packed(B, Vs, F64)
    U[0, B.offsets[2] + 5] = float("nan")
    tt = [0.0] * 4
    with pytest.raises(hydro.HydroError) as ei:
        B.step(U, 10, t=tt)
    assert ei.value.status == hydro.HYDRO_ENONFINITE
    O, _, _, _ = _oracle(Vs[3], (0, 0), 10)
    assert max_rel_err(B.grid_view(U, 3).cpu().numpy(), O) <= 1e-10


def test_graph_and_direct_launches_agree():
    Vs = _data(SMALL, 12)
    A = hydro.BatchSolver(SMALL, G, dtype=F32)
    UA = _packed(A, Vs, F32)
    A.step(UA, 70)
    P = hydro.BatchSolver(SMALL, G, dtype=F32)
    P.set_profiling(True)
    UP = _packed(P, Vs, F32)
    P.step(UP, 70)
    assert torch.equal(UA, UP)
    kt = P.kernel_times()
    # the "cfl" slot holds the first CFL pass and the per-step dt finaliser
    assert kt["stage1"][1] == 70 and kt["stage2"][1] == 70 and kt["cfl"][1] == 71


@pytest.mark.slow
def test_full_batched_config_fp32():
    """4096 grids, sides log-uniform on [32, 512] (seed 1204477904), 50 steps, FP32 in one
    persistent launch per stage: a seeded sample of grids against the oracle, all grids'
    FP64 mass and energy audited."""
    shapes = [tuple(int(v) for v in s) for s in inputs.batch_shapes()]
    Vs = [inputs.batch_grid(nx, ny, 1204477904, i) for i, (nx, ny) in enumerate(shapes)]
    B = hydro.BatchSolver(shapes, G, dtype=F32)
    U = _packed(B, Vs, F32)
    T0 = np.array(B.totals(U))
    t, steps = B.step(U, 50)
    assert steps == [50] * len(shapes)
    T1 = np.array(B.totals(U))
    assert np.max(np.abs(T1[:, 0] - T0[:, 0]) / T0[:, 0]) <= 2e-6
    assert np.max(np.abs(T1[:, 4] - T0[:, 4]) / T0[:, 4]) <= 2e-6
    rng = np.random.default_rng(20)
    sample = sorted(set(rng.choice(len(shapes), 10, replace=False).tolist()) |
                    {int(np.argmax([a * b for a, b in shapes]))})
    worst = 0.0
    for g in sample:
        O, to, so, _ = _oracle(Vs[g], (0, 0), 50)
        e = l1_rel(B.grid_view(U, g)[0].double().cpu().numpy(), O[0])
        worst = max(worst, e)
        assert e <= 1e-4, (g, shapes[g], e)
        assert abs(t[g] - to) <= 1e-5 * to
    print(f"PARITY batched4096 fp32 worst_sampled_l1_rho={worst:.3e}")


@pytest.mark.slow
def test_full_batched_config_fp64():
    """The same 4096-grid configuration in FP64 (50 steps): a seeded sample of grids, and the
    largest, against the oracle run on each grid alone, max relative error <= 1e-10 and the same
    time."""
    shapes = [tuple(int(v) for v in s) for s in inputs.batch_shapes()]
    Vs = [inputs.batch_grid(nx, ny, 1204477904, i) for i, (nx, ny) in enumerate(shapes)]
    B = hydro.BatchSolver(shapes, G, dtype=F64)
    U = _packed(B, Vs, F64)
    t, steps = B.step(U, 50)
    assert steps == [50] * len(shapes)
    rng = np.random.default_rng(21)
    sample = sorted(set(rng.choice(len(shapes), 8, replace=False).tolist()) |
                    {int(np.argmax([a * b for a, b in shapes]))})
    worst = 0.0
    for g in sample:
        O, to, so, _ = _oracle(Vs[g], (0, 0), 50)
        e = max_rel_err(B.grid_view(U, g).cpu().numpy(), O)
        worst = max(worst, e)
        assert e <= 1e-10, (g, shapes[g], e)
        assert t[g] == to, (g, t[g], to)
    print(f"PARITY batched4096 fp64 worst_sampled_max_rel={worst:.3e}")


# ---- row tiles: a work item is a strip of x columns marching along y -----------------------

@pytest.mark.parametrize("march", [7, 32])
@pytest.mark.parametrize("bc", [("periodic", (0, 0)), ("outflow", (1, 1))])
def test_row_tiles_fp64_match_oracle_per_grid(bc, march):
    Vs = _data(SMALL, 9)
    B = hydro.BatchSolver(SMALL, G, bc=bc[0], dtype=F64, cfl=0.4, tile=(64, 1), march=march)
    U = _packed(B, Vs, F64)
    t, steps = B.step(U, 25)
    assert steps == [25] * len(SMALL)
    for g, V in enumerate(Vs):
        O, to, so, _ = _oracle(V, bc[1], 25)
        Gg = B.grid_view(U, g).cpu().numpy()
        assert t[g] == to, (g, t[g], to)
        assert max_rel_err(Gg, O) <= 1e-10, (g, march)


@pytest.mark.parametrize("tile", [(32, 1), (64, 1), (128, 1)])
def test_row_tiles_fp32_l1(tile):
    Vs = _data(SMALL, 10)
    B = hydro.BatchSolver(SMALL, G, dtype=F32, tile=tile, march=16)
    U = _packed(B, Vs, F32)
    t, steps = B.step(U, 40)
    for g, V in enumerate(Vs):
        O, to, _, _ = _oracle(V, (0, 0), 40)
        Gg = B.grid_view(U, g).double().cpu().numpy()
        assert l1_rel(Gg[0], O[0]) <= 1e-5, (tile, g)
        assert abs(t[g] - to) <= 1e-5 * to


def test_row_tiles_graph_and_direct_launches_agree():
    Vs = _data(SMALL, 13)
    A = hydro.BatchSolver(SMALL, G, dtype=F32, tile=(64, 1), march=16)
    UA = _packed(A, Vs, F32)
    A.step(UA, 30)
    P = hydro.BatchSolver(SMALL, G, dtype=F32, tile=(64, 1), march=16)
    P.set_profiling(True)
    UP = _packed(P, Vs, F32)
    P.step(UP, 30)
    assert torch.equal(UA, UP)


def test_row_tiles_reject_unsupported():
    from paper_1204_4779_gb300.hydro import HydroError
    with pytest.raises(HydroError):
        hydro.BatchSolver(SMALL, G, dtype=F64, tile=(128, 1))
    with pytest.raises(HydroError):
        hydro.BatchSolver(SMALL, G, dtype=F32, tile=(64, 1), march=-1)
