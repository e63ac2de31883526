"""hydro_step_static: the step for callers that cannot allocate device memory.

Those callers (code inside a runtime that owns every allocation, embedded or real-time code
that must not allocate after start-up) cannot hand the library a workspace, so this entry point
keeps its RK stage buffer and control block in a fixed device array inside the library.  These
tests call it through the C ABI and check it against the regular hydro_step on the same input,
on two calls in a row (the second reuses the array the first left behind), in 1D, 2D and 3D and
both precisions; the 3D FP32 case also against the FP64 oracle, since the call runs one fixed
kernel variant (32 x 8 tiles, two-CTA budget) which hydro_step runs when asked for it; that a
warm call changes neither torch's allocated bytes nor the device's free memory; and that a grid
too large for the array is refused.  Collected last on purpose: it runs after every other test.
"""
import ctypes

import numpy as np
import pytest

from _helpers import gpu_state, l1_rel, max_rel_err, oracle_run
from paper_1204_4779_gb300 import hydro, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _grid(shape):
    g = hydro.Grid()
    g.dim = len(shape)
    for a in range(3):
        g.n[a] = shape[a] if a < len(shape) else 1
        g.lo[a] = 0.0
        g.hi[a] = 1.0
    return g


def _static_step(U, shape, gamma, bc, prec, cfl, n_steps, t_end=0.0, t0=0.0):
    lib = hydro.load_library()
    s = hydro.state_struct(U, len(shape) + 2)
    bcs = (ctypes.c_int32 * 3)(*(list(bc) + [0] * (3 - len(bc))))
    t = ctypes.c_double(t0)
    done = ctypes.c_int32()
    rc = lib.hydro_step_static(ctypes.byref(_grid(shape)), gamma, bcs, prec, cfl, ctypes.byref(s),
                               n_steps, t_end, ctypes.byref(t), ctypes.byref(done),
                               torch.cuda.current_stream().cuda_stream)
    return rc, t.value, done.value


# the fixed variant the call runs, as a hydro_step variant
FIXED_3D = dict(tile=(32, 8), march=64, split=2, staging=1, occupancy=2)

CASES = [
    # shape, gamma, bc, dtype, steps, t_end, initial data, hydro_step variant
    ((1024,), 1.4, (1,), torch.float64, 100000, 0.2, lambda: inputs.sod_1d(1024), None),
    ((300,), 1.4, (0,), torch.float32, 40, 0.0, lambda: inputs.smooth((300,), seed=31), None),
    ((70, 45), 5.0 / 3.0, (0, 1), torch.float32, 30, 0.0, lambda: inputs.kh_2d(70, seed=5, ny=45),
     None),
    ((70, 45), 5.0 / 3.0, (1, 0), torch.float64, 30, 0.0, lambda: inputs.kh_2d(70, seed=6, ny=45),
     None),
    ((30, 27, 21), 1.4, (0, 0, 1), torch.float64, 12, 0.0,
     lambda: inputs.blast_3d(shape=(30, 27, 21), radius_cells=5.0), None),
    ((40, 37, 33), 1.4, (0, 1, 0), torch.float32, 30, 0.0,
     lambda: inputs.blast_3d(shape=(40, 37, 33), radius_cells=6.0), FIXED_3D),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_static_step_matches_hydro_step_twice(case):
    shape, gamma, bc, dtype, steps, t_end, make, variant = CASES[case]
    V = make()
    prec = hydro.HYDRO_F32 if dtype == torch.float32 else hydro.HYDRO_F64
    U_ref = gpu_state(V, gamma, dtype)
    S = hydro.Solver(shape, gamma, bc=list(bc), dtype=dtype, cfl=0.4, variant=variant)
    t_ref, n_ref = S.step(U_ref, steps, t_end=t_end)
    ref = U_ref.double().cpu().numpy()
    tol = 1e-10 if dtype == torch.float64 else 1e-6
    for _ in range(2):  # two calls in a row share the library's array
        U = gpu_state(V, gamma, dtype)
        rc, t, n = _static_step(U, shape, gamma, bc, prec, 0.4, steps, t_end)
        assert rc == hydro.HYDRO_OK, hydro.load_library().hydro_strerror(rc)
        assert n == n_ref and t == t_ref
        got = U.double().cpu().numpy()
        assert max_rel_err(got, ref) <= tol
    if dtype == torch.float32 and len(shape) == 3:
        O, to, so, _ = oracle_run(V, gamma, bc, 0.4, steps)
        assert so == n and abs(t - to) <= 1e-5 * to
        assert l1_rel(got[0], O[0]) <= 1e-4


def test_static_step_allocates_nothing():
    """A warm call changes neither the bytes torch has allocated nor the device's free memory
    (the state planes are the caller's; the stage buffer is the library's fixed array)."""
    shape = (33, 31, 29)
    V = inputs.blast_3d(shape=shape, radius_cells=5.0)
    U = gpu_state(V, 1.4, torch.float32)
    for _ in range(2):  # warm: the first call's set-up and the kernels' first launches
        rc, _, _ = _static_step(U, shape, 1.4, (0, 0, 0), hydro.HYDRO_F32, 0.4, 3)
        assert rc == hydro.HYDRO_OK
    torch.cuda.synchronize()
    alloc0 = torch.cuda.memory_allocated()
    free0, _ = torch.cuda.mem_get_info()
    rc, _, n = _static_step(U, shape, 1.4, (0, 0, 0), hydro.HYDRO_F32, 0.4, 3)
    torch.cuda.synchronize()
    assert rc == hydro.HYDRO_OK and n == 3
    assert torch.cuda.memory_allocated() == alloc0
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_static_step_rejects_grids_larger_than_its_array():
    shape = (64, 64, 64)  # 5 FP32 planes of 64^3 cells need more than the 4 MiB array
    U = torch.ones((5, 64, 64, 64), dtype=torch.float32, device="cuda")
    U[4] = 2.5
    before = U.clone()
    rc, _, _ = _static_step(U, shape, 1.4, (0, 0, 0), hydro.HYDRO_F32, 0.4, 1)
    assert rc == hydro.HYDRO_EINVAL
    assert torch.equal(U, before)
    # the largest FP32 cube that fits, 59^3, is accepted
    V = inputs.blast_3d(shape=(59, 59, 59), radius_cells=6.0)
    U2 = gpu_state(V, 1.4, torch.float32)
    rc, t, n = _static_step(U2, (59, 59, 59), 1.4, (0, 0, 0), hydro.HYDRO_F32, 0.4, 4)
    assert rc == hydro.HYDRO_OK and n == 4
    U_ref = gpu_state(V, 1.4, torch.float32)
    S = hydro.Solver((59, 59, 59), 1.4, bc="periodic", dtype=torch.float32, cfl=0.4,
                     variant=FIXED_3D)
    t_ref, n_ref = S.step(U_ref, 4)
    assert n_ref == n and t_ref == t
    assert max_rel_err(U2.double().cpu().numpy(), U_ref.double().cpu().numpy()) <= 1e-6
