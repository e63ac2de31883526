"""Behaviour of the C-ABI calls on the GPU: conversions, CFL dt, totals, time clipping,
error reporting, host-buffer stepping, graph vs. direct launches, determinism."""
import numpy as np
import pytest

import oracle
from _helpers import gpu_run, gpu_state, oracle_run, shape_of
from paper_1204_4779_gb300 import hydro, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
F32, F64 = torch.float32, torch.float64


@pytest.mark.parametrize("shape", [(33,), (20, 13), (9, 8, 7)])
def test_conversions_match_oracle_bitwise(shape):
    V = inputs.smooth(shape, seed=2)
    U = hydro.prim_to_cons(torch.from_numpy(V).cuda(), 1.4).cpu().numpy()
    Uo = oracle.prim_to_cons(V, 1.4)
    assert np.array_equal(U, Uo)
    V2 = hydro.cons_to_prim(torch.from_numpy(Uo).cuda(), 1.4).cpu().numpy()
    assert np.array_equal(V2, oracle.cons_to_prim(Uo, 1.4))


@pytest.mark.parametrize("shape", [(1024,), (64, 48), (20, 17, 9)])
def test_cfl_dt_matches_oracle(shape):
    V = inputs.smooth(shape, seed=3)
    S = hydro.Solver(shape, 1.4, dtype=F64, cfl=0.4)
    dt = S.cfl_dt(gpu_state(V, 1.4, F64))
    assert dt == oracle.cfl_dt(oracle.prim_to_cons(V, 1.4), 1.4, 0.4)
    S32 = hydro.Solver(shape, 1.4, dtype=F32, cfl=0.4)
    dt32 = S32.cfl_dt(gpu_state(V, 1.4, F32))
    assert abs(dt32 - dt) <= 2e-6 * dt


@pytest.mark.parametrize("dtype", [F32, F64])
def test_totals_match_oracle(dtype):
    V = inputs.smooth((40, 30, 20), seed=5)
    U = gpu_state(V, 1.4, dtype)
    S = hydro.Solver((40, 30, 20), 1.4, dtype=dtype)
    T = np.array(S.totals(U))
    To = oracle.totals(U.double().cpu().numpy())
    assert np.allclose(T, To, rtol=1e-13, atol=1e-13 * abs(To[4]))
    S2 = hydro.Solver((40, 30), 1.4, dtype=dtype)
    V2 = inputs.smooth((40, 30), seed=6)
    T2 = np.array(S2.totals(gpu_state(V2, 1.4, dtype)))
    assert T2[3] == 0.0


@pytest.mark.parametrize("dtype,tol", [(F64, 1e-13), (F32, 2e-6)])
def test_periodic_conservation(dtype, tol):
    V = inputs.blast_3d(shape=(40, 36, 33), radius_cells=6.0)
    U = gpu_state(V, 1.4, dtype)
    S = hydro.Solver((40, 36, 33), 1.4, dtype=dtype)
    T0 = np.array(S.totals(U))
    S.step(U, 60)
    T1 = np.array(S.totals(U))
    assert abs(T1[0] - T0[0]) <= tol * T0[0]
    assert abs(T1[4] - T0[4]) <= tol * T0[4]
    assert np.all(np.abs(T1[1:4] - T0[1:4]) <= tol * T0[4])


@pytest.mark.parametrize("dtype", [F32, F64])
def test_uniform_state_is_bitwise_unchanged(dtype):
    V = inputs.uniform((19, 12, 10), rho=1.3, v=(0.3, -0.2, 0.1), p=0.7)
    U = gpu_state(V, 1.4, dtype)
    U0 = U.clone()
    S = hydro.Solver((19, 12, 10), 1.4, bc=["periodic", "outflow", "periodic"], dtype=dtype)
    S.step(U, 5)
    assert torch.equal(U, U0)


def test_time_clipping_matches_oracle():
    V = inputs.sod_1d(64)
    G, t, steps = gpu_run(V, 1.4, (1,), F64, 0.4, 100000, t_end=0.05)
    O, to, so, _ = oracle_run(V, 1.4, (1,), 0.4, 100000, t_end=0.05)
    assert t == to == 0.05 and steps == so
    # more steps requested than needed: the rest are no-ops
    G2, t2, steps2 = gpu_run(V, 1.4, (1,), F64, 0.4, steps + 7, t_end=0.05)
    assert steps2 == steps and np.array_equal(G2, G)
    # t already at t_end: nothing happens
    U = gpu_state(V, 1.4, F64)
    S = hydro.Solver((64,), 1.4, bc="outflow", dtype=F64)
    t3, s3 = S.step(U, 5, t_end=0.05, t=0.05)
    assert s3 == 0 and t3 == 0.05


def test_generous_step_bound_stops_at_t_end():
    """A synchronous call stops launching graph chunks once t_end is reached: a bound of 10^6
    steps costs about as much as the steps actually taken (10^6 empty steps would take
    seconds)."""
    import time
    V = inputs.sod_1d(256)
    U = gpu_state(V, 1.4, F64)
    S = hydro.Solver((256,), 1.4, bc="outflow", dtype=F64)
    S.step(gpu_state(V, 1.4, F64), 64, t_end=0.01)  # graphs captured outside the timing
    t0 = time.perf_counter()
    t, steps = S.step(U, 10 ** 6, t_end=0.1)
    wall = time.perf_counter() - t0
    O, to, so, _ = oracle_run(V, 1.4, (1,), 0.4, 10 ** 6, t_end=0.1)
    assert t == to == 0.1 and steps == so
    assert wall < 1.0, wall
    # and the state is the one of the exact step count
    G, _, _ = gpu_run(V, 1.4, (1,), F64, 0.4, steps, t_end=0.1)
    assert np.array_equal(U.cpu().numpy(), G)


def test_profiled_stepping_stops_at_t_end():
    """Under profiling the steps run in batches of 64 with reused events, and the stepping stops
    after the batch in which t_end is reached."""
    V = inputs.sod_1d(256)
    U = gpu_state(V, 1.4, F64)
    S = hydro.Solver((256,), 1.4, bc="outflow", dtype=F64)
    S.set_profiling(True)
    t, steps = S.step(U, 10 ** 6, t_end=0.05)
    O, to, so, _ = oracle_run(V, 1.4, (1,), 0.4, 10 ** 6, t_end=0.05)
    assert t == to == 0.05 and steps == so
    kt = S.kernel_times()
    assert steps <= kt["stage1"][1] < steps + 64 and kt["stage2"][1] == kt["stage1"][1]
    G, _, _ = gpu_run(V, 1.4, (1,), F64, 0.4, steps, t_end=0.05)
    assert np.array_equal(U.cpu().numpy(), G)


def test_nonfinite_and_nonpositive_are_reported():
    V = inputs.uniform((32,), rho=1.0, v=(0.0,), p=1.0)
    for bad in ("nan", "negrho"):
        U = gpu_state(V, 1.4, F64)
        if bad == "nan":
            U[0, 5] = float("nan")
        else:
            U[0, 5] = -1.0
        S = hydro.Solver((32,), 1.4, dtype=F64)
        with pytest.raises(hydro.HydroError) as ei:
            S.step(U, 3)
        assert ei.value.status == hydro.HYDRO_ENONFINITE
        assert S.status() == hydro.HYDRO_ENONFINITE
    # a blow-up during the run: an absurd CFL number makes the scheme unstable
    V = inputs.smooth((64,), seed=1)
    U = gpu_state(V, 1.4, F64)
    S = hydro.Solver((64,), 1.4, dtype=F64, cfl=50.0)
    with pytest.raises(hydro.HydroError):
        S.step(U, 200)


def test_graph_and_direct_launches_agree_bitwise():
    V = inputs.kh_2d(96, seed=3, ny=80)
    A, ta, sa = gpu_run(V, 5.0 / 3.0, (0, 0), F32, 0.4, 70)
    B, tb, sb = gpu_run(V, 5.0 / 3.0, (0, 0), F32, 0.4, 70, profiling=True)
    assert np.array_equal(A, B) and ta == tb and sa == sb


def test_runs_are_deterministic():
    V = inputs.blast_3d(shape=(48, 40, 36), radius_cells=6.0)
    A, ta, _ = gpu_run(V, 1.4, (0, 0, 0), F32, 0.4, 30)
    B, tb, _ = gpu_run(V, 1.4, (0, 0, 0), F32, 0.4, 30)
    assert np.array_equal(A, B) and ta == tb


def test_step_split_across_calls_matches_one_call():
    V = inputs.smooth((50, 40), seed=8)
    A, ta, _ = gpu_run(V, 1.4, (0, 0), F64, 0.4, 20)
    U = gpu_state(V, 1.4, F64)
    S = hydro.Solver((50, 40), 1.4, dtype=F64)
    t = 0.0
    for n in (7, 1, 12):
        t, _ = S.step(U, n, t=t)
    assert np.array_equal(U.cpu().numpy(), A) and t == ta


def test_step_host_matches_device_step():
    V = inputs.smooth((64, 40), seed=9)
    A, ta, _ = gpu_run(V, 1.4, (0, 1), F32, 0.4, 15)
    U = gpu_state(V, 1.4, F32)
    host = U.cpu().pin_memory()
    out = torch.empty_like(host).pin_memory()
    dev = torch.empty_like(U)
    S = hydro.Solver((64, 40), 1.4, bc=["periodic", "outflow"], dtype=F32)
    t, n = S.step_host(dev, host, out, 15)
    assert n == 15 and t == ta
    assert np.array_equal(out.double().numpy(), A)


def test_kernel_times_are_recorded():
    V = inputs.smooth((64, 64, 32), seed=1)
    U = gpu_state(V, 1.4, F32)
    S = hydro.Solver((64, 64, 32), 1.4, dtype=F32)
    S.set_profiling(True)
    S.step(U, 4)
    kt = S.kernel_times(reset=True)
    assert kt["cfl"][1] == 1 and kt["stage1"][1] == 4 and kt["stage2"][1] == 4
    assert all(v[0] > 0 for v in kt.values())
    assert S.kernel_times()["stage1"] == (0.0, 0)


def test_single_cell_axes_and_tiny_grids():
    for shape, bc in (((1,), (0,)), ((2, 1), (0, 1)), ((3, 2, 1), (1, 0, 0)), ((5, 1, 4), (0, 0, 1))):
        V = inputs.smooth(shape, seed=4)
        G, tg, sg = gpu_run(V, 1.4, bc, F64, 0.3, 6)
        O, to, so, _ = oracle_run(V, 1.4, bc, 0.3, 6)
        assert sg == so and np.allclose(G, O, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("n_steps,t_end,shape,bc,staging", [
    (1, 0.0, (40, 36, 100), (0, 0, 0), 1), (3, 0.0, (40, 36, 100), (0, 0, 0), 1),
    (5, 0.002, (40, 36, 100), (0, 0, 0), 1),
    (1, 0.0, (40, 36, 100), (0, 1, 1), 1),   # outflow along z
    (2, 0.0, (24, 20, 57), (0, 0, 0), 1),    # a last slab of one plane: stage 1 whole first
    (1, 0.0, (24, 20, 11), (0, 0, 0), 1),    # two march chunks: two slabs
    # TMA plane staging: the slab launches start at march chunk zchunk0 > 0
    (3, 0.0, (40, 36, 100), (0, 0, 0), 3), (1, 0.0, (40, 36, 100), (0, 1, 1), 3),
    (2, 0.0, (24, 20, 57), (1, 0, 0), 3)])
def test_host_stepping_3d_overlapped_copy_back(n_steps, t_end, shape, bc, staging):
    """In 3D hydro_step_host copies the state in by z-slabs with the first CFL pass split over
    them, and runs the last step's two stages slab by slab, copying each slab back while later
    slabs compute (e.g. 13 march chunks of 8 planes, the last one ragged, in 8 slabs): the host
    result, time and step count equal stepping on the device, with either plane staging."""
    V = inputs.blast_3d(shape=shape, radius_cells=6.0)
    U = gpu_state(V, 1.4, F32)
    var = dict(march=8, staging=staging)
    S = hydro.Solver(shape, 1.4, bc=list(bc), dtype=F32, variant=var)
    Ud = U.clone()
    td, nd = S.step(Ud, n_steps, t_end=t_end)
    host = U.cpu().pin_memory()
    out = torch.empty_like(host).pin_memory()
    out.fill_(float("nan"))
    dev = torch.empty_like(U)
    th, nh = S.step_host(dev, host, out, n_steps, t_end=t_end)
    assert nh == nd and th == td
    assert torch.equal(out, Ud.cpu())
    assert torch.equal(dev, Ud)


@pytest.mark.parametrize("shape,bc", [((40, 36, 100), (0, 0, 0)), ((96, 70), (0, 1))])
def test_host_stepping_async_two_problems_in_flight(shape, bc):
    """hydro_step_host_async on two contexts with their own streams, calls interleaved
    (problem a's next copy in queued while b's step and copy back are in flight), each state
    copied in and back in place every call: after three calls each host state equals three
    one-step hydro_step calls on the device, bit for bit (3D: the overlapped slab path; 2D:
    whole-plane copies)."""
    Va = inputs.blast_3d(shape=shape, radius_cells=6.0) if len(shape) == 3 else \
        inputs.kh_2d(shape[0], seed=3)[:, :shape[1], :].copy()
    Vb = inputs.smooth(shape, seed=11)
    Ua, Ub = gpu_state(Va, 1.4, F32), gpu_state(Vb, 1.4, F32)
    var = dict(march=8) if len(shape) == 3 else None
    ref = hydro.Solver(shape, 1.4, bc=list(bc), dtype=F32, variant=var)
    Ra, Rb = Ua.clone(), Ub.clone()
    for _ in range(3):
        ref.step(Ra, 1)
        ref.step(Rb, 1)
    A = hydro.Solver(shape, 1.4, bc=list(bc), dtype=F32, variant=var)
    B = hydro.Solver(shape, 1.4, bc=list(bc), dtype=F32, variant=var)
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    ha, hb = Ua.cpu().pin_memory(), Ub.cpu().pin_memory()
    da, db = torch.empty_like(Ua), torch.empty_like(Ub)
    torch.cuda.synchronize()
    for _ in range(3):
        with torch.cuda.stream(sa):
            A.step_host_async(da, ha, ha, 1)
        with torch.cuda.stream(sb):
            B.step_host_async(db, hb, hb, 1)
    assert A.status() == 0 and B.status() == 0
    assert torch.equal(ha, Ra.cpu()) and torch.equal(hb, Rb.cpu())
    assert torch.equal(da, Ra) and torch.equal(db, Rb)


def test_host_stepping_async_reports_status_and_clips_at_t_end():
    """An asynchronous host step reports a failed step through the next synchronising call
    (hydro_status), and with t_end it launches every step but stops advancing at t_end, as
    hydro_step_host does."""
    V = inputs.uniform((40, 36, 24), rho=1.0, v=(0.1, 0.0, 0.0), p=1.0)
    U = gpu_state(V, 1.4, F32)
    U[4, 3, 7, 11] = float("nan")
    S = hydro.Solver((40, 36, 24), 1.4, dtype=F32, variant=dict(march=8))
    h = U.cpu().pin_memory()
    S.step_host_async(torch.empty_like(U), h, h, 2)
    assert S.status() == hydro.HYDRO_ENONFINITE
    Vb = inputs.blast_3d(shape=(40, 36, 24), radius_cells=5.0)
    Ub = gpu_state(Vb, 1.4, F32)
    Ud = Ub.clone()
    td, nd = S.step(Ud, 50, t_end=0.003)
    assert 1 < nd < 50
    hb = Ub.cpu().pin_memory()
    out = torch.full_like(hb, float("nan")).pin_memory()
    dev = torch.empty_like(Ub)
    S.step_host_async(dev, hb, out, 50, t_end=0.003)
    assert S.status() == 0
    assert torch.equal(out, Ud.cpu()) and torch.equal(dev, Ud)


def test_host_stepping_with_separate_host_planes():
    """Host planes in separate allocations (not one tensor): the copies go plane by plane
    instead of one strided copy per slab, with the same result."""
    import ctypes
    shape = (40, 36, 100)
    V = inputs.blast_3d(shape=shape, radius_cells=6.0)
    U = gpu_state(V, 1.4, F32)
    S = hydro.Solver(shape, 1.4, dtype=F32, variant=dict(march=8))
    Ud = U.clone()
    td, nd = S.step(Ud, 2)
    # planes at irregular offsets of pinned buffers, so that no single pitch fits them
    N = U[0].numel()
    offs = [k * N + 16 * k * k for k in range(5)]
    hin = torch.empty(5 * N + 1024, dtype=F32).pin_memory()
    hout = torch.full((5 * N + 1024,), float("nan"), dtype=F32).pin_memory()
    planes, outs = [], []
    for k in range(5):
        planes.append(hin[offs[k]:offs[k] + N].view(U[k].shape))
        planes[k].copy_(U[k].cpu())
        outs.append(hout[offs[k]:offs[k] + N].view(U[k].shape))
    dev = torch.empty_like(U)
    st = hydro.state_struct(dev, 5)
    pin = (ctypes.c_void_p * 5)(*[p.data_ptr() for p in planes])
    pout = (ctypes.c_void_p * 5)(*[o.data_ptr() for o in outs])
    t = ctypes.c_double(0.0)
    n = ctypes.c_int32()
    torch.cuda.synchronize()
    assert S.lib.hydro_step_host(S.ctx, ctypes.byref(st), pin, pout, 2, 0.0, ctypes.byref(t),
                                 ctypes.byref(n)) == 0
    assert n.value == nd and t.value == td
    for k in range(5):
        assert torch.equal(outs[k], Ud[k].cpu()), k


def test_resolved_default_variants():
    """hydro_get_variant: the library defaults per dimension and precision, and the defaults a
    variant that names another tile gets (that tile's march and register budget)."""
    cases = [
        ((40, 36, 30), F32, None, dict(tile=(16, 8), march=8, split=2, staging=1, occupancy=3)),
        ((40, 36, 100), F64, None, dict(tile=(32, 8), march=64, split=2, staging=1, occupancy=2)),
        ((300, 77), F32, None, dict(tile=(256, 1), march=16, split=2, staging=1, occupancy=3)),
        ((300, 77), F64, None, dict(tile=(32, 8), march=1, split=1, staging=1, occupancy=2)),
        ((300,), F32, None, dict(tile=(128, 1), march=1, split=1, staging=1, occupancy=2)),
        ((300, 77), F32, dict(tile=(32, 8)), dict(tile=(32, 8), march=1, split=1, staging=1,
                                                  occupancy=2)),
        ((300, 77), F32, dict(tile=(64, 1)), dict(tile=(64, 1), march=16, split=2, staging=1,
                                                  occupancy=2)),
        ((40, 36, 100), F32, dict(tile=(32, 8)), dict(tile=(32, 8), march=8, split=2, staging=1,
                                                      occupancy=3)),
        ((40, 36, 100), F32, dict(march=20), dict(tile=(16, 8), march=20, split=2, staging=1,
                                                  occupancy=3)),
    ]
    for shape, dt, var, want in cases:
        S = hydro.Solver(shape, 1.4, dtype=dt, variant=var)
        got = S.variant()
        S.close()
        assert got == dict(want, manifest=1), (shape, dt, var, got)


@pytest.mark.parametrize("n,march", [(512, 96), (448, 48), (384, 32), (256, 48), (192, 16),
                                     (128, 8)])
def test_default_march_follows_the_grid_size(n, march):
    """3D FP32 without a named march: among 8, 16, 32, ..., 128 the marches whose (tile, chunk)
    work items fill the GPU's resident CTAs (152 SMs x six 128-thread CTAs on GB300) three
    times, the one with the least 0.5 x chunks + 0.3 x (planes of the last chunk); else 8."""
    props = torch.cuda.get_device_properties(0)
    if props.multi_processor_count != 152:
        pytest.skip("the expected marches are those of a 152-SM GPU")
    S = hydro.Solver((n, n, n), 1.4, dtype=F32)
    got = S.variant()["march"]
    S.close()
    assert got == march


@pytest.mark.parametrize("n,march", [(4096, 64), (2048, 16), (1024, 16)])
def test_default_row_march_follows_the_grid_size(n, march):
    """2D FP32 row tiles without a named march: among 8, 16, 32, 64, 128 the marches whose work
    items fill the resident CTAs (152 SMs x three 256-thread CTAs) twice, the one with the
    least 0.5 x chunks + 0.3 x (rows of the last chunk); else 16."""
    props = torch.cuda.get_device_properties(0)
    if props.multi_processor_count != 152:
        pytest.skip("the expected marches are those of a 152-SM GPU")
    S = hydro.Solver((n, n), 5.0 / 3.0, dtype=F32)
    got = S.variant()
    S.close()
    assert got["tile"] == (256, 1) and got["march"] == march


def test_host_stepping_with_a_manifest_form():
    V = inputs.blast_3d(shape=(40, 36, 30), radius_cells=6.0)
    U = gpu_state(V, 1.4, F32)
    S = hydro.Solver((40, 36, 30), 1.4, dtype=F32, variant=dict(manifest=3, march=8))
    Ud = U.clone()
    td, nd = S.step(Ud, 3)
    host = U.cpu().pin_memory()
    out = torch.empty_like(host).pin_memory()
    dev = torch.empty_like(U)
    th, nh = S.step_host(dev, host, out, 3)
    assert (th, nh) == (td, nd) and torch.equal(out, Ud.cpu())
