"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

FP64: max relative error <= 1e-10 after the run (density and energy element-wise, momenta
norm-wise).  FP32 (whole stencil in FP32 from the same FP64 initial data): L1 density error
relative to the FP64 oracle <= 1e-4 after 100 steps.  Sizes span several tiles with ragged
tails; the configs' full sizes are covered where the oracle finishes in seconds.
"""
import numpy as np
import pytest

import oracle
from _helpers import gpu_run, l1_rel, max_rel_err, oracle_run, shape_of
from paper_1204_4779_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
F32, F64 = torch.float32, torch.float64


def _compare64(V, gamma, bc, cfl, n, t_end=0.0, variant=None, tol=1e-10):
    G, tg, sg = gpu_run(V, gamma, bc, F64, cfl, n, t_end=t_end, variant=variant)
    O, to, so, _ = oracle_run(V, gamma, bc, cfl, n, t_end=t_end)
    assert sg == so and tg == to, (sg, so, tg, to)
    err = max_rel_err(G, O)
    assert err <= tol, err
    return err, G, O


def test_sod_1024_fp64_full_config():
    """1D Sod, 1024 cells, gamma 1.4, outflow, CFL 0.4, run to t = 0.2."""
    V = inputs.sod_1d(1024)
    err, G, O = _compare64(V, 1.4, (1,), 0.4, 100000, t_end=0.2)
    print(f"PARITY sod1024 fp64 max_rel={err:.3e}")
    assert not np.allclose(G, oracle.prim_to_cons(V, 1.4))


@pytest.mark.parametrize("bc", [(0, 0), (1, 0), (0, 1)])
def test_kh_ragged_fp64(bc):
    V = inputs.kh_2d(100, seed=1204477901, ny=77)
    _compare64(V, 5.0 / 3.0, bc, 0.4, 40)


def test_kh_1024_fp64_full_config():
    """2D 1024^2 shear layer, gamma 5/3, periodic, 100 steps, FP64."""
    V = inputs.kh_2d(1024, seed=1204477901)
    err, _, _ = _compare64(V, 5.0 / 3.0, (0, 0), 0.4, 100)
    print(f"PARITY kh1024 fp64 max_rel={err:.3e}")


@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 1, 1), (0, 1, 0)])
def test_blast_ragged_fp64(bc):
    V = inputs.blast_3d(shape=(37, 29, 23), radius_cells=5.0)
    _compare64(V, 1.4, bc, 0.4, 12, variant=dict(march=8))


def test_smooth_3d_march_chunks_fp64():
    """z-chunk boundaries (march 5 over 19 planes, a ragged last chunk) change nothing."""
    V = inputs.smooth((21, 18, 19), seed=4)
    _compare64(V, 1.4, (0, 0, 1), 0.4, 10, variant=dict(march=5))


# ------------------------------------------------------------------- FP32 ------------

def _l1_32(V, gamma, bc, n, variant=None):
    G, tg, sg = gpu_run(V, gamma, bc, F32, 0.4, n, variant=variant)
    O, to, so, _ = oracle_run(V, gamma, bc, 0.4, n)
    assert sg == so == n
    assert abs(tg - to) <= 1e-5 * to
    return l1_rel(G[0], O[0]), G, O


def test_kh_1024_fp32_full_config():
    V = inputs.kh_2d(1024, seed=1204477901)
    e, G, O = _l1_32(V, 5.0 / 3.0, (0, 0), 100)
    print(f"PARITY kh1024 fp32 l1_rho={e:.3e}")
    assert e <= 1e-4


def test_blast_fp32_l1():
    V = inputs.blast_3d(64, radius_cells=8.0)
    e, G, O = _l1_32(V, 1.4, (0, 0, 0), 100)
    print(f"blast 64^3 FP32 L1(rho) rel = {e:.3e}")
    assert e <= 1e-4


def test_sod_fp32_l1():
    V = inputs.sod_1d(1024)
    G, tg, sg = gpu_run(V, 1.4, (1,), F32, 0.4, 100000, t_end=0.2)
    O, to, so, _ = oracle_run(V, 1.4, (1,), 0.4, 100000, t_end=0.2)
    assert tg == to == 0.2
    assert abs(sg - so) <= 1
    e = l1_rel(G[0], O[0])
    print(f"PARITY sod1024 fp32 l1_rho={e:.3e}")
    assert e <= 1e-4


@pytest.mark.parametrize("tile", [(32, 8), (32, 4), (64, 4), (16, 16), (32, 16), (16, 8)])
@pytest.mark.parametrize("split,staging", [(2, 1), (1, 1), (2, 2), (1, 2)])
def test_every_fp32_3d_variant(tile, split, staging):
    """Every compiled tile with both fusion splits (2 fused, 1 separate CFL pass) and both
    staging depths, on the two-CTA register budget."""
    V = inputs.smooth((45, 38, 21), seed=11)
    e, _, _ = _l1_32(V, 1.4, (0, 1, 0), 10,
                     variant=dict(tile=tile, march=6, split=split, staging=staging, occupancy=2))
    assert e <= 2e-6


@pytest.mark.parametrize("tile", [(32, 8), (32, 4), (64, 4), (16, 16), (32, 16), (16, 8)])
@pytest.mark.parametrize("split,staging", [(2, 1), (1, 2)])
def test_fp32_3d_occupancy3_variant(tile, split, staging):
    """The kernels compiled for three resident CTAs per SM (about 80 registers a thread)."""
    V = inputs.smooth((45, 38, 21), seed=11)
    e, _, _ = _l1_32(V, 1.4, (0, 1, 0), 10,
                     variant=dict(tile=tile, march=6, split=split, staging=staging, occupancy=3))
    assert e <= 2e-6


@pytest.mark.parametrize("split", [1, 2])
@pytest.mark.parametrize("dim_shape", [(1, (300,)), (2, (70, 45)), (3, (37, 29, 23))])
def test_fp64_both_splits_match_oracle(dim_shape, split):
    """Fused and separate dt reductions compute the same step to 1e-10 in FP64."""
    dim, shape = dim_shape
    V = inputs.smooth(shape, seed=14)
    _compare64(V, 1.4, (0,) * dim, 0.4, 15, variant=dict(split=split, march=8))


@pytest.mark.parametrize("split", [1, 2])
def test_both_splits_time_clipping(split):
    V = inputs.sod_1d(256)
    _compare64(V, 1.4, (1,), 0.4, 100000, t_end=0.1, variant=dict(split=split))


@pytest.mark.parametrize("order,riemann", [(1, 0), (2, 1), (1, 1)])
@pytest.mark.parametrize("dim_shape", [(1, (300,)), (2, (70, 45)), (3, (37, 29, 23))])
def test_scheme_options_fp64_match_oracle(dim_shape, order, riemann):
    """First-order reconstruction and pressure-based wave speeds, FP64 <= 1e-10."""
    dim, shape = dim_shape
    V = inputs.smooth(shape, seed=15) if dim != 1 else inputs.sod_1d(300)
    bc = (1,) if dim == 1 else (0,) * dim
    G, tg, sg = gpu_run(V, 1.4, bc, F64, 0.4, 20, scheme=(order, riemann))
    O, to, so, _ = oracle_run(V, 1.4, bc, 0.4, 20, order=order, riemann=riemann)
    assert sg == so and tg == to
    assert max_rel_err(G, O) <= 1e-10


@pytest.mark.parametrize("order,riemann", [(1, 0), (2, 1)])
def test_scheme_options_fp32_blast(order, riemann):
    V = inputs.blast_3d(48, radius_cells=6.0)
    G, tg, sg = gpu_run(V, 1.4, (0, 0, 0), F32, 0.4, 30, scheme=(order, riemann))
    O, to, so, _ = oracle_run(V, 1.4, (0, 0, 0), 0.4, 30, order=order, riemann=riemann)
    assert l1_rel(G[0], O[0]) <= 1e-5


@pytest.mark.parametrize("tile", [(32, 8), (64, 4), (16, 16), (32, 16)])
def test_every_fp32_2d_tile(tile):
    V = inputs.smooth((70, 45), seed=12)
    e, _, _ = _l1_32(V, 1.4, (1, 0), 20, variant=dict(tile=tile))
    assert e <= 2e-6


@pytest.mark.parametrize("tile", [(128, 1), (256, 1)])
def test_every_fp32_1d_tile(tile):
    V = inputs.smooth((300,), seed=13)
    e, _, _ = _l1_32(V, 1.4, (0,), 50, variant=dict(tile=tile))
    assert e <= 2e-6


# ---- dim-2 row tiles: a row of x cells per CTA marching along y ---------------------------

@pytest.mark.parametrize("march", [5, 32])
@pytest.mark.parametrize("bc", [(0, 0), (1, 0), (0, 1)])
def test_row_tiles_fp64_ragged(bc, march):
    """Row tiles (128 x 1) marching along y: ragged x (100 = one partial tile) and ragged march
    chunks (77 rows), every boundary combination, FP64 <= 1e-10."""
    V = inputs.kh_2d(100, seed=1204477901, ny=77)
    _compare64(V, 5.0 / 3.0, bc, 0.4, 30, variant=dict(tile=(128, 1), march=march))


@pytest.mark.parametrize("split", [1, 2])
@pytest.mark.parametrize("shape", [(300, 7), (7, 300), (70, 1), (1, 45)])
def test_row_tiles_fp64_degenerate_shapes(shape, split):
    """Narrow, tall, one-row and one-column grids through row tiles, both dt reductions."""
    V = inputs.smooth(shape, seed=21)
    _compare64(V, 1.4, (0, 1), 0.4, 12, variant=dict(tile=(128, 1), march=16, split=split))


@pytest.mark.parametrize("order,riemann", [(1, 0), (2, 1)])
def test_row_tiles_scheme_options_fp64(order, riemann):
    V = inputs.smooth((70, 45), seed=22)
    G, tg, sg = gpu_run(V, 1.4, (0, 0), F64, 0.4, 20, variant=dict(tile=(128, 1), march=8),
                        scheme=(order, riemann))
    O, to, so, _ = oracle_run(V, 1.4, (0, 0), 0.4, 20, order=order, riemann=riemann)
    assert sg == so and tg == to
    assert max_rel_err(G, O) <= 1e-10


def test_row_tiles_fp64_kh_1024_full_config():
    """The 1024^2 shear layer (gamma 5/3, periodic, 100 steps) through FP64 row tiles."""
    V = inputs.kh_2d(1024, seed=1204477901)
    _compare64(V, 5.0 / 3.0, (0, 0), 0.4, 100, variant=dict(tile=(128, 1), march=32))


@pytest.mark.parametrize("occupancy", [2, 3])
@pytest.mark.parametrize("staging", [1, 2])
@pytest.mark.parametrize("split", [1, 2])
@pytest.mark.parametrize("tile", [(64, 1), (128, 1), (256, 1)])
def test_every_fp32_row_tile_variant(tile, split, staging, occupancy):
    V = inputs.smooth((300, 77), seed=23)
    e, _, _ = _l1_32(V, 1.4, (1, 0), 20, variant=dict(tile=tile, march=9, split=split,
                                                      staging=staging, occupancy=occupancy))
    assert e <= 2e-6


def test_row_tiles_fp32_kh_1024_full_config():
    V = inputs.kh_2d(1024, seed=1204477901)
    e, _, _ = _l1_32(V, 5.0 / 3.0, (0, 0), 100, variant=dict(tile=(128, 1), march=32))
    assert e <= 1e-4


# ---- the manifest forms (V or the face fluxes stored in HBM between the parts of a stage) ---

@pytest.mark.parametrize("manifest", [2, 3])
@pytest.mark.parametrize("split", [1, 2])
@pytest.mark.parametrize("dtype,tile", [(F32, (16, 8)), (F32, (32, 8)), (F32, (16, 16)),
                                        (F64, (32, 8))])
def test_manifest_forms_are_the_same_step(dtype, tile, split, manifest):
    """Storing V or the face fluxes changes where intermediates live, not the arithmetic: in
    FP64 (no contraction) the same step bit for bit; in FP32 the compiler may fuse a product
    of the recovery into its consumer when V stays in registers, so the forms agree to
    rounding (ragged x, y and march chunks, time clipping on the last step)."""
    V = inputs.blast_3d(shape=(37, 29, 23), radius_cells=5.0)
    base = dict(tile=tile, march=6, split=split)
    G0, t0, s0 = gpu_run(V, 1.4, (0, 1, 0), dtype, 0.4, 40, t_end=0.012, variant=base)
    G1, t1, s1 = gpu_run(V, 1.4, (0, 1, 0), dtype, 0.4, 40, t_end=0.012,
                         variant=dict(base, manifest=manifest))
    assert s0 == s1
    if dtype == F64:
        assert t0 == t1 and np.array_equal(G0, G1)
    else:
        assert abs(t0 - t1) <= 1e-6 * t0
        assert l1_rel(G1[0], G0[0]) <= 1e-6
        assert np.max(np.abs(G1 - G0)) <= 1e-4 * np.max(np.abs(G0))


@pytest.mark.parametrize("manifest", [2, 3])
def test_manifest_forms_fp64_match_oracle(manifest):
    V = inputs.smooth((21, 18, 19), seed=24)
    _compare64(V, 1.4, (1, 0, 1), 0.4, 10, variant=dict(march=5, manifest=manifest))


# ---- TMA plane staging (staging 3, 3D FP32 16 x 8) ------------------------------------------

@pytest.mark.parametrize("occupancy", [2, 3])
@pytest.mark.parametrize("shape,bc,march", [
    ((44, 38, 21), (0, 0, 0), 8),    # ragged x (44 = 2 x 16 + 12), y and z chunks
    ((44, 38, 21), (1, 0, 1), 64),   # outflow x and z, one z chunk
    ((48, 17, 9), (0, 1, 0), 4),     # ragged y, chunks of four planes (the last of one)
    ((16, 8, 1), (0, 0, 0), 64),     # one plane, one tile
    ((40, 24, 2), (1, 1, 1), 1),     # chunks of one plane (only the own box in flight)
    ((45, 38, 21), (0, 0, 0), 8),    # x extent not a multiple of 4: the look-ahead kernels run
])
def test_tma_staging_equals_look_ahead_staging(shape, bc, march, occupancy):
    """The planes come into shared memory by bulk tensor copies instead of per-thread loads;
    the arithmetic and its operands are the same, so the step is the same bit for bit."""
    V = inputs.smooth(shape, seed=31)
    base = dict(tile=(16, 8), march=march, split=2, occupancy=occupancy)
    G1, t1, s1 = gpu_run(V, 1.4, bc, F32, 0.4, 12, variant=dict(base, staging=1))
    G3, t3, s3 = gpu_run(V, 1.4, bc, F32, 0.4, 12, variant=dict(base, staging=3))
    assert s1 == s3 == 12 and t1 == t3
    assert np.array_equal(G1, G3)


def test_tma_staging_blast_fp32_vs_oracle():
    V = inputs.blast_3d(64, radius_cells=8.0)
    G, tg, sg = gpu_run(V, 1.4, (0, 0, 0), F32, 0.4, 100, variant=dict(staging=3))
    O, to, so, _ = oracle_run(V, 1.4, (0, 0, 0), 0.4, 100)
    assert sg == so == 100 and abs(tg - to) <= 1e-5 * to
    assert l1_rel(G[0], O[0]) <= 1e-4
