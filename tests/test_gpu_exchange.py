"""Ghost exchange through pack/unpack buffers (the kernels a slab decomposition over several
GPUs would put its transfers between), exercised on one GPU as the periodic wrap: every step
must equal the periodic boundary's bit for bit, in both precisions, with the exchange on either
axis or both, next to periodic or outflow axes, on ragged grids and with tiles as thin as two
cells along the exchange axis."""
import numpy as np
import pytest

from _helpers import gpu_state, max_rel_err, oracle_run
from paper_1204_4779_gb300 import hydro, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
F32, F64 = torch.float32, torch.float64


def _run(V, shape, bc, dtype, n, variant):
    U = gpu_state(V, 1.4, dtype)
    S = hydro.Solver(shape, 1.4, bc=list(bc), dtype=dtype, cfl=0.4, variant=variant)
    t, steps = S.step(U, n)
    var = S.variant()
    S.close()
    return U.cpu().numpy(), t, steps, var


CASES = [
    ((37, 29), (3, 3)),
    ((37, 29), (3, 0)),
    ((37, 29), (0, 3)),
    ((45, 21), (3, 1)),
    ((33, 40), (1, 3)),
    ((2, 19), (3, 3)),
    ((150,), (3,)),
    ((2,), (3,)),
]


@pytest.mark.parametrize("dtype", [F64, F32], ids=["f64", "f32"])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_exchange_equals_periodic_bitwise(case, dtype):
    shape, bc = CASES[case]
    V = inputs.smooth(shape, seed=17 + case)
    variant = {"tile": (32, 8)} if len(shape) == 2 else None
    periodic = tuple(0 if b == 3 else b for b in bc)
    E, te, se, var = _run(V, shape, bc, dtype, 25, variant)
    P, tp, sp, _ = _run(V, shape, periodic, dtype, 25, variant)
    assert se == sp == 25 and te == tp
    assert np.array_equal(E, P)
    if len(shape) == 2:
        assert var["tile"] == (32, 8)
    if dtype == F64:  # and the periodic run is the oracle's
        O, to, so, _ = oracle_run(V, 1.4, periodic, 0.4, 25)
        assert so == 25 and max_rel_err(E, O) <= 1e-10


def test_exchange_with_the_default_tile_and_unsupported_cases():
    V = inputs.smooth((64, 48), seed=3)
    E, _, _, var = _run(V, (64, 48), (3, 3), F32, 10, None)
    assert var["tile"][1] > 1  # a one-plane tile, as for analytic boundaries
    with pytest.raises(hydro.HydroError) as e:
        hydro.Solver((8, 8, 8), 1.4, bc="exchange", dtype=F32)
    assert e.value.status == hydro.HYDRO_EUNSUPPORTED
    with pytest.raises(hydro.HydroError) as e:
        hydro.Solver((1, 8), 1.4, bc=["exchange", "periodic"], dtype=F64)
    assert e.value.status == hydro.HYDRO_EUNSUPPORTED
