"""Out-of-bounds writes (no sanitizer on this pool): the state planes and the workspace are
placed between guard zones filled with a bit pattern; after steps, totals, CFL passes and
conversions on ragged grids, in every dimension, precision and kernel variant family, the
guards must be intact and nothing outside the planes written."""
import ctypes

import numpy as np
import pytest

from _helpers import gpu_state, shape_of
from paper_1204_4779_gb300 import hydro, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
GUARD = 1 << 16  # bytes on each side
PATTERN = 0x5A


def _guarded(nbytes, device="cuda"):
    buf = torch.full((GUARD + nbytes + GUARD,), PATTERN, dtype=torch.uint8, device=device)
    return buf


def _intact(buf, nbytes):
    lo = buf[:GUARD]
    hi = buf[GUARD + nbytes:]
    return bool((lo == PATTERN).all().item()) and bool((hi == PATTERN).all().item())


CASES = [
    ((37,), (1,), torch.float64, {}),
    ((300,), (0,), torch.float32, {"split": 2}),
    ((45, 29), (0, 1), torch.float32, {}),
    ((70, 33), (1, 0), torch.float64, {"split": 2}),
    ((37, 21, 19), (0, 1, 0), torch.float32, {"march": 5}),
    ((37, 21, 19), (1, 0, 1), torch.float32, {"march": 7, "split": 1, "staging": 2, "occupancy": 2}),
    ((33, 18, 11), (0, 0, 0), torch.float32, {"tile": (16, 16), "march": 4}),
    ((23, 29, 17), (0, 0, 1), torch.float64, {"march": 6, "split": 1}),
    # analytic boundaries: the ghost ring in the workspace is written before every stage
    ((45, 29), (2, 2), torch.float32, {}),
    ((37, 21), (2, 1), torch.float64, {}),
    ((150,), (2,), torch.float32, {}),
    # exchange boundaries: the pack buffers and the ring
    ((45, 29), (3, 2), torch.float64, {}),
    ((37, 21), (3, 3), torch.float32, {}),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_no_writes_outside_state_and_workspace(case):
    shape, bc, dtype, variant = CASES[case]
    V = inputs.smooth(shape, seed=case)
    U0 = gpu_state(V, 1.4, dtype)
    nbytes = U0.numel() * U0.element_size()
    sbuf = _guarded(nbytes)
    U = sbuf[GUARD:GUARD + nbytes].view(dtype).view(U0.shape)
    U.copy_(U0)
    S = hydro.Solver(shape, 1.4, bc=list(bc), dtype=dtype, variant=variant or None)
    wbytes = S.workspace.numel()
    wbuf = _guarded(wbytes + 256)
    # re-create the context on a guarded, 256-byte aligned workspace
    base = wbuf.data_ptr() + GUARD
    g = S.grid
    bcs = (ctypes.c_int32 * 3)(*(S.bc + [0] * (3 - S.dim)))
    var = None
    if variant:
        tile = variant.get("tile", (0, 0))
        var = hydro.Variant(tile[0], tile[1], variant.get("march", 0), variant.get("split", 0),
                            variant.get("staging", 0), variant.get("occupancy", 0))
    ctx = ctypes.c_void_p()
    lib = hydro.load_library()
    assert base % 256 == 0
    rc = lib.hydro_create(ctypes.byref(g), 1.4, bcs, hydro._prec(dtype), 0.4,
                          ctypes.byref(var) if var is not None else None, base, wbytes,
                          torch.cuda.current_stream().cuda_stream, ctypes.byref(ctx))
    assert rc == 0
    if 2 in bc:
        assert lib.hydro_set_analytic(ctx, hydro.HYDRO_ANALYTIC_SHOCK_TUBE, 0.9, 0.0) == 0
    st = hydro.state_struct(U, len(shape) + 2)
    t = ctypes.c_double(0.0)
    n = ctypes.c_int32()
    assert lib.hydro_step(ctx, ctypes.byref(st), 7, 0.0, ctypes.byref(t), ctypes.byref(n)) == 0
    out = (ctypes.c_double * 5)()
    assert lib.hydro_totals(ctx, ctypes.byref(st), out) == 0
    dt = ctypes.c_double()
    assert lib.hydro_cfl_dt(ctx, ctypes.byref(st), ctypes.byref(dt)) == 0
    lib.hydro_destroy(ctx)
    torch.cuda.synchronize()
    assert n.value == 7
    assert _intact(sbuf, nbytes), "write outside the state planes"
    assert _intact(wbuf, wbytes), "write outside the workspace"


def test_batched_and_conversion_guards():
    shapes = [(1, 1), (33, 9), (17, 40), (64, 3)]
    B = hydro.BatchSolver(shapes, 1.4, dtype=torch.float32)
    nb = 4 * B.total * 4
    sbuf = _guarded(nb)
    U = sbuf[GUARD:GUARD + nb].view(torch.float32).view(4, B.total)
    P = np.concatenate([inputs.batch_grid(a, b, 3, i).reshape(4, -1) for i, (a, b) in enumerate(shapes)], 1)
    U.copy_(hydro.prim_to_cons(torch.from_numpy(P).cuda().view(4, 1, -1), 1.4).view(4, -1).float())
    B.step(U, 9)
    B.totals(U)
    torch.cuda.synchronize()
    assert _intact(sbuf, nb)
    # element-wise conversion in place on a guarded buffer
    V = torch.from_numpy(inputs.smooth((13, 7, 5), seed=1)).cuda()
    n2 = V.numel() * 8
    cbuf = _guarded(n2)
    X = cbuf[GUARD:GUARD + n2].view(torch.float64).view(V.shape)
    X.copy_(V)
    st = hydro.state_struct(X, 5)
    assert hydro.load_library().hydro_prim_to_cons(3, 13 * 7 * 5, 1.4, hydro.HYDRO_F64,
                                                   ctypes.byref(st), ctypes.byref(st),
                                                   torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    assert _intact(cbuf, n2)


def test_bounded_mbarrier_wait_gives_up_and_the_context_stays_usable():
    """The bounded wait of the TMA-staged kernels, on an mbarrier phase that never completes (an
    arrival nobody makes): every thread gives up within the bound (2^16 tries or about a second
    of the global timer) instead of hanging, and the device runs a step afterwards."""
    from paper_1204_4779_gb300 import hydro, inputs
    gave_up, ms = hydro.wait_bound_check()
    assert gave_up == 32
    assert 0.0 < ms < 3000.0, ms
    V = inputs.blast_3d(shape=(32, 24, 16), radius_cells=4.0)
    U = hydro.prim_to_cons(torch.from_numpy(V).cuda(), 1.4).float().contiguous()
    S = hydro.Solver((32, 24, 16), 1.4, bc="periodic", dtype=torch.float32, cfl=0.4,
                     variant=dict(staging=3))
    t, n = S.step(U, 3)
    assert n == 3 and S.status() == hydro.HYDRO_OK and bool(torch.isfinite(U).all())
