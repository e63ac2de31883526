"""hydro_step_static: the step for callers that cannot allocate device memory.

Those callers (code inside a runtime that owns every allocation, a stream capture in which
allocating is forbidden, embedded or real-time code that must not allocate after start-up)
cannot hand the library a workspace, so this entry point keeps its RK stage buffer and control
block in a fixed device array inside the library.  These tests call it through the C ABI and
check it against the regular hydro_step on the same input, on two calls in a row (the second
reuses the array the first left behind), and check that a grid too large for the array is
refused.  Collected last on purpose: it runs after every other test.
"""
import ctypes

import numpy as np
import pytest

from _helpers import gpu_state, max_rel_err
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


CASES = [
    # shape, gamma, bc, dtype, steps, t_end, initial data
    ((1024,), 1.4, (1,), torch.float64, 100000, 0.2, lambda: inputs.sod_1d(1024)),
    ((70, 45), 5.0 / 3.0, (0, 1), torch.float32, 30, 0.0, lambda: inputs.kh_2d(70, seed=5, ny=45)),
    ((30, 27, 21), 1.4, (0, 0, 1), torch.float64, 12, 0.0,
     lambda: inputs.blast_3d(shape=(30, 27, 21), radius_cells=5.0)),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_static_step_matches_hydro_step_twice(case):
    shape, gamma, bc, dtype, steps, t_end, make = CASES[case]
    V = make()
    prec = hydro.HYDRO_F32 if dtype == torch.float32 else hydro.HYDRO_F64
    U_ref = gpu_state(V, gamma, dtype)
    S = hydro.Solver(shape, gamma, bc=list(bc), dtype=dtype, cfl=0.4)
    t_ref, n_ref = S.step(U_ref, steps, t_end=t_end)
    ref = U_ref.double().cpu().numpy()
    tol = 1e-10 if dtype == torch.float64 else 1e-6
    for _ in range(2):  # two calls in a row share the library's array
        U = gpu_state(V, gamma, dtype)
        rc, t, n = _static_step(U, shape, gamma, bc, prec, 0.4, steps, t_end)
        assert rc == hydro.HYDRO_OK, hydro.load_library().hydro_strerror(rc)
        assert n == n_ref and t == t_ref
        assert max_rel_err(U.double().cpu().numpy(), ref) <= tol


def test_static_step_rejects_grids_larger_than_its_array():
    shape = (64, 64, 64)  # 5 FP32 planes of 64^3 cells need more than the 4 MiB array
    U = torch.ones((5, 64, 64, 64), dtype=torch.float32, device="cuda")
    U[4] = 2.5
    before = U.clone()
    rc, _, _ = _static_step(U, shape, 1.4, (0, 0, 0), hydro.HYDRO_F32, 0.4, 1)
    assert rc == hydro.HYDRO_EINVAL
    assert torch.equal(U, before)
    # the largest FP32 cube that fits, 59^3, is accepted
    V = inputs.uniform((59, 59, 59), rho=1.0, v=(0.1, 0.0, -0.1), p=1.0)
    U2 = gpu_state(V, 1.4, torch.float32)
    rc, _, n = _static_step(U2, (59, 59, 59), 1.4, (0, 0, 0), hydro.HYDRO_F32, 0.4, 2)
    assert rc == hydro.HYDRO_OK and n == 2
