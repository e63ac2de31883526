"""Python binding of libhydro.so (include/hydro.h): argument marshalling only.

PyTorch supplies device memory and the current CUDA stream; every step of the solver runs in
the library's kernels.  There is no CPU fallback: if libhydro.so cannot be loaded (or built
with nvcc) the constructor raises.

State tensors have shape (dim+2, [nz, [ny,]] nx), contiguous, planes (rho, m_x, [m_y, [m_z]],
E) for conserved or (rho, v_x, [v_y, [v_z]], p) for primitive variables, dtype float32 or
float64 on a CUDA device.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhydro.so")

HYDRO_OK, HYDRO_EINVAL, HYDRO_ECUDA, HYDRO_ENONFINITE, HYDRO_ETIMEOUT, HYDRO_EUNSUPPORTED = range(6)
HYDRO_BC_PERIODIC, HYDRO_BC_OUTFLOW, HYDRO_BC_ANALYTIC, HYDRO_BC_EXCHANGE = 0, 1, 2, 3
HYDRO_ANALYTIC_ENTROPY_WAVE, HYDRO_ANALYTIC_SOUND_WAVE, HYDRO_ANALYTIC_SHOCK_TUBE = 1, 2, 3
ANALYTIC_KINDS = {"entropy": 1, "sound": 2, "shock_tube": 3}
HYDRO_F64, HYDRO_F32 = 0, 1

# every symbol include/hydro.h declares
EXPORTS = (
    "hydro_version", "hydro_strerror", "hydro_last_cuda_error", "hydro_variant_supported",
    "hydro_workspace_bytes", "hydro_workspace_bytes_variant", "hydro_create", "hydro_get_variant",
    "hydro_destroy", "hydro_set_stream",
    "hydro_step",
    "hydro_step_host", "hydro_step_host_async", "hydro_set_scheme", "hydro_set_analytic", "hydro_analytic_state", "hydro_cfl_dt", "hydro_totals", "hydro_status", "hydro_prim_to_cons",
    "hydro_cons_to_prim", "hydro_set_profiling", "hydro_kernel_times", "hydro_step_static",
    "hydro_batch_workspace_bytes", "hydro_batch_create", "hydro_batch_destroy",
    "hydro_batch_offsets", "hydro_batch_set_stream", "hydro_batch_step", "hydro_batch_totals",
    "hydro_batch_set_profiling", "hydro_batch_kernel_times",
    "hydro_mlp_sizes", "hydro_mlp_forward", "hydro_mlp_gradient", "hydro_mlp_adam", "hydro_mlp_train",
    "hydro_wave_workspace_bytes", "hydro_wave_run", "hydro_fma_rate", "hydro_wait_bound_check",
)


class HydroError(RuntimeError):
    def __init__(self, status: int, what: str):
        lib = _lib
        msg = lib.hydro_strerror(status).decode() if lib else str(status)
        if status == HYDRO_ECUDA and lib:
            msg += ": " + lib.hydro_last_cuda_error().decode()
        super().__init__(f"{what}: {msg}")
        self.status = status


class Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("n", ctypes.c_int64 * 3), ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3)]


class State(ctypes.Structure):
    _fields_ = [("plane", ctypes.c_void_p * 5)]


class Variant(ctypes.Structure):
    _fields_ = [("tile_x", ctypes.c_int32), ("tile_y", ctypes.c_int32),
                ("march", ctypes.c_int32), ("split", ctypes.c_int32), ("staging", ctypes.c_int32),
                ("occupancy", ctypes.c_int32), ("manifest", ctypes.c_int32)]


_lib = None
_lock = threading.Lock()


def load_library(path: str = LIB_PATH, build_if_missing: bool = True):
    """Load libhydro.so (building it with nvcc first if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path) and build_if_missing:
            from . import _build
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libhydro.so not found at {path}; build it with "
                               "`python -m paper_1204_4779_gb300._build`")
        lib = ctypes.CDLL(path)
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        P = ctypes.POINTER
        sig = {
            "hydro_version": ([], ctypes.c_int),
            "hydro_strerror": ([ctypes.c_int], ctypes.c_char_p),
            "hydro_last_cuda_error": ([], ctypes.c_char_p),
            "hydro_variant_supported": ([i32, i32, P(Variant)], ctypes.c_int),
            "hydro_workspace_bytes": ([P(Grid), i32, P(ctypes.c_size_t)], ctypes.c_int),
            "hydro_workspace_bytes_variant": ([P(Grid), i32, P(Variant), P(ctypes.c_size_t)],
                                              ctypes.c_int),
            "hydro_create": ([P(Grid), dbl, P(i32), i32, dbl, P(Variant), vp, ctypes.c_size_t, vp,
                              P(vp)], ctypes.c_int),
            "hydro_destroy": ([vp], ctypes.c_int),
            "hydro_get_variant": ([vp, P(Variant)], ctypes.c_int),
            "hydro_set_stream": ([vp, vp], ctypes.c_int),
            "hydro_set_scheme": ([vp, i32, i32], ctypes.c_int),
            "hydro_set_analytic": ([vp, i32, dbl, dbl], ctypes.c_int),
            "hydro_analytic_state": ([P(Grid), dbl, i32, i32, dbl, dbl, dbl, P(State), vp],
                                     ctypes.c_int),
            "hydro_step": ([vp, P(State), i32, dbl, P(dbl), P(i32)], ctypes.c_int),
            "hydro_step_host": ([vp, P(State), P(vp), P(vp), i32, dbl, P(dbl), P(i32)], ctypes.c_int),
            "hydro_step_host_async": ([vp, P(State), P(vp), P(vp), i32, dbl, dbl], ctypes.c_int),
            "hydro_cfl_dt": ([vp, P(State), P(dbl)], ctypes.c_int),
            "hydro_totals": ([vp, P(State), P(dbl)], ctypes.c_int),
            "hydro_status": ([vp], ctypes.c_int),
            "hydro_prim_to_cons": ([i32, i64, dbl, i32, P(State), P(State), vp], ctypes.c_int),
            "hydro_cons_to_prim": ([i32, i64, dbl, i32, P(State), P(State), vp], ctypes.c_int),
            "hydro_set_profiling": ([vp, i32], ctypes.c_int),
            "hydro_kernel_times": ([vp, P(dbl), P(i64), i32, i32], ctypes.c_int),
            "hydro_step_static": ([P(Grid), dbl, P(i32), i32, dbl, P(State), i32, dbl, P(dbl), P(i32),
                                   vp], ctypes.c_int),
            "hydro_batch_workspace_bytes": ([i32, P(i64), P(i64), i32, P(Variant), P(ctypes.c_size_t)],
                                            ctypes.c_int),
            "hydro_batch_create": ([i32, P(i64), P(i64), dbl, P(i32), i32, dbl, P(Variant), vp,
                                    ctypes.c_size_t, vp, P(vp)], ctypes.c_int),
            "hydro_batch_destroy": ([vp], ctypes.c_int),
            "hydro_batch_offsets": ([vp, P(i64)], ctypes.c_int),
            "hydro_batch_set_stream": ([vp, vp], ctypes.c_int),
            "hydro_batch_step": ([vp, P(State), i32, dbl, P(dbl), P(i32)], ctypes.c_int),
            "hydro_batch_totals": ([vp, P(State), P(dbl)], ctypes.c_int),
            "hydro_batch_set_profiling": ([vp, i32], ctypes.c_int),
            "hydro_batch_kernel_times": ([vp, P(dbl), P(i64), i32, i32], ctypes.c_int),
            "hydro_mlp_sizes": ([i32, i32, i64, P(i64), P(ctypes.c_size_t)], ctypes.c_int),
            "hydro_fma_rate": ([i32, vp, P(dbl)], ctypes.c_int),
            "hydro_wait_bound_check": ([vp, vp, P(i32), P(dbl)], ctypes.c_int),
            "hydro_wave_workspace_bytes": ([i64, i32, i32, P(ctypes.c_size_t)], ctypes.c_int),
            "hydro_wave_run": ([i32, i64, dbl, dbl, dbl, vp, vp, i32, P(dbl), vp, ctypes.c_size_t, vp],
                               ctypes.c_int),
            "hydro_mlp_forward": ([vp, i32, i32, vp, i64, vp, vp, vp], ctypes.c_int),
            "hydro_mlp_gradient": ([vp, i32, i32, vp, vp, i64, vp, vp, vp, vp], ctypes.c_int),
            "hydro_mlp_adam": ([vp, vp, vp, vp, i64, i32, ctypes.c_float, ctypes.c_float,
                                ctypes.c_float, ctypes.c_float, vp], ctypes.c_int),
            "hydro_mlp_train": ([vp, vp, vp, i32, i32, vp, vp, i64, i32, i32, ctypes.c_float, vp, vp,
                                 vp], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _check(rc: int, what: str):
    if rc != HYDRO_OK:
        raise HydroError(rc, what)


def _prec(dtype) -> int:
    if dtype == torch.float32:
        return HYDRO_F32
    if dtype == torch.float64:
        return HYDRO_F64
    raise ValueError(f"unsupported dtype {dtype}")


def _stream_ptr(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def state_struct(t: torch.Tensor, nv: int) -> State:
    """Plane pointers of a contiguous (nv, ...) tensor."""
    if not t.is_contiguous():
        raise ValueError("state tensors must be contiguous")
    s = State()
    plane_bytes = t[0].numel() * t.element_size()
    base = t.data_ptr()
    for k in range(nv):
        s.plane[k] = base + k * plane_bytes
    return s


def variant_supported(dtype, dim: int, tile=(0, 0), march: int = 0, split: int = 0,
                      staging: int = 0, occupancy: int = 0, manifest: int = 0) -> bool:
    lib = load_library()
    v = Variant(int(tile[0]), int(tile[1]), int(march), int(split), int(staging), int(occupancy),
                int(manifest))
    return bool(lib.hydro_variant_supported(_prec(dtype), dim, ctypes.byref(v)))


def _convert(x: torch.Tensor, gamma: float, to_cons: bool) -> torch.Tensor:
    lib = load_library()
    dim = x.dim() - 1
    out = torch.empty_like(x)
    si, so = state_struct(x, dim + 2), state_struct(out, dim + 2)
    fn = lib.hydro_prim_to_cons if to_cons else lib.hydro_cons_to_prim
    _check(fn(dim, x[0].numel(), float(gamma), _prec(x.dtype), ctypes.byref(si), ctypes.byref(so),
              _stream_ptr(x.device)), "convert")
    return out


def prim_to_cons(V: torch.Tensor, gamma: float) -> torch.Tensor:
    """Conserved planes from primitive planes on the GPU (m = rho v, E = p/(g-1) + rho v^2/2)."""
    return _convert(V.contiguous(), gamma, True)


def cons_to_prim(U: torch.Tensor, gamma: float) -> torch.Tensor:
    return _convert(U.contiguous(), gamma, False)


def analytic_state(shape, gamma: float, kind, theta: float = 0.0, amplitude: float = 1.0,
                   t: float = 0.0, dtype=torch.float64, device=None) -> torch.Tensor:
    """Conserved planes of an exact solution of the convergence tests (kind "entropy", "sound",
    "shock_tube" or 1-3) at the cell centres of the unit box (dim 1 or 2) at time t."""
    lib = load_library()
    dim = len(shape)
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    U = torch.empty((dim + 2,) + tuple(reversed([int(n) for n in shape])), dtype=dtype, device=dev)
    g = Grid()
    g.dim = dim
    for a in range(3):
        g.n[a] = int(shape[a]) if a < dim else 1
        g.lo[a], g.hi[a] = 0.0, 1.0
    k = ANALYTIC_KINDS[kind] if isinstance(kind, str) else int(kind)
    st = state_struct(U, dim + 2)
    with torch.cuda.device(dev):
        _check(lib.hydro_analytic_state(ctypes.byref(g), float(gamma), _prec(dtype), k,
                                        float(theta), float(amplitude), float(t), ctypes.byref(st),
                                        _stream_ptr(dev)), "hydro_analytic_state")
    return U


class Solver:
    """One context of libhydro.so on the current CUDA device.

    shape: cells per axis (nx, [ny, [nz]]); bc: per-axis "periodic"/"outflow"/"analytic"/
    "exchange" (or 0-3; analytic boundaries take their solution from set_analytic; exchange
    boundaries wrap through the ghost pack/unpack kernels);
    variant: dict(tile=(bx, by), march=m, split=0|1|2, staging=0|1|2|3, occupancy=0|2|3,
    manifest=0|1|2|3) or None for the default (staging 3: TMA plane staging, 3D FP32 tiles).
    """

    def __init__(self, shape, gamma: float, bc="periodic", dtype=torch.float32, cfl: float = 0.4,
                 variant=None, lo=None, hi=None, device=None):
        self.lib = load_library()
        self.dim = len(shape)
        self.shape = tuple(int(s) for s in shape)
        self.nv = self.dim + 2
        self.gamma = float(gamma)
        self.cfl = float(cfl)
        self.dtype = dtype
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        if isinstance(bc, (str, int)):
            bc = [bc] * self.dim
        names = {"periodic": HYDRO_BC_PERIODIC, "outflow": HYDRO_BC_OUTFLOW,
                 "analytic": HYDRO_BC_ANALYTIC, "exchange": HYDRO_BC_EXCHANGE}
        self.bc = [names[b] if isinstance(b, str) else int(b) for b in bc]
        g = Grid()
        g.dim = self.dim
        for a in range(3):
            g.n[a] = self.shape[a] if a < self.dim else 1
            g.lo[a] = 0.0 if lo is None else float(lo[a]) if a < self.dim else 0.0
            g.hi[a] = 1.0 if hi is None else float(hi[a]) if a < self.dim else 1.0
        self.grid = g
        var = None
        if variant:
            tile = variant.get("tile", (0, 0))
            var = Variant(int(tile[0]), int(tile[1]), int(variant.get("march", 0)),
                          int(variant.get("split", 0)), int(variant.get("staging", 0)),
                          int(variant.get("occupancy", 0)), int(variant.get("manifest", 0)))
        nbytes = ctypes.c_size_t()
        _check(self.lib.hydro_workspace_bytes_variant(ctypes.byref(g), _prec(dtype),
                                                      ctypes.byref(var) if var is not None else None,
                                                      ctypes.byref(nbytes)),
               "hydro_workspace_bytes_variant")
        self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device=self.device)
        bcs = (ctypes.c_int32 * 3)(*(self.bc + [0] * (3 - self.dim)))
        ctx = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(self.lib.hydro_create(ctypes.byref(g), self.gamma, bcs, _prec(dtype), self.cfl,
                                         ctypes.byref(var) if var is not None else None,
                                         self.workspace.data_ptr(), int(nbytes.value),
                                         _stream_ptr(self.device), ctypes.byref(ctx)), "hydro_create")
        self.ctx = ctx

    # -- lifetime --------------------------------------------------------------------------
    def close(self):
        if getattr(self, "ctx", None):
            self.lib.hydro_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def variant(self) -> dict:
        """The variant this context runs, defaults filled in (hydro_get_variant)."""
        v = Variant()
        _check(self.lib.hydro_get_variant(self.ctx, ctypes.byref(v)), "hydro_get_variant")
        return {"tile": (v.tile_x, v.tile_y), "march": v.march, "split": v.split,
                "staging": v.staging, "occupancy": v.occupancy, "manifest": v.manifest}

    # -- helpers ---------------------------------------------------------------------------
    def empty_state(self) -> torch.Tensor:
        return torch.empty((self.nv,) + tuple(reversed(self.shape)), dtype=self.dtype,
                           device=self.device)

    def _state(self, U: torch.Tensor) -> State:
        if U.dtype != self.dtype or U.device != self.device:
            raise ValueError("state dtype/device does not match the solver")
        if tuple(U.shape) != (self.nv,) + tuple(reversed(self.shape)):
            raise ValueError(f"state shape {tuple(U.shape)} does not match the grid")
        return state_struct(U, self.nv)

    def _sync_stream(self):
        self.lib.hydro_set_stream(self.ctx, _stream_ptr(self.device))

    # -- the C ABI -------------------------------------------------------------------------
    def step(self, U: torch.Tensor, n_steps: int, t_end: float = 0.0, t: float = 0.0,
             sync: bool = True):
        """Advance U in place; returns (t, steps_done) (None, None when sync=False)."""
        self._sync_stream()
        s = self._state(U)
        if not sync:
            _check(self.lib.hydro_step(self.ctx, ctypes.byref(s), int(n_steps), float(t_end), None,
                                       None), "hydro_step")
            return None, None
        tt = ctypes.c_double(t)
        done = ctypes.c_int32()
        _check(self.lib.hydro_step(self.ctx, ctypes.byref(s), int(n_steps), float(t_end),
                                   ctypes.byref(tt), ctypes.byref(done)), "hydro_step")
        return tt.value, done.value

    def step_host(self, U_dev: torch.Tensor, host_in: torch.Tensor, host_out: torch.Tensor,
                  n_steps: int, t_end: float = 0.0, t: float = 0.0):
        """Copy host_in -> U_dev, advance, copy U_dev -> host_out, in one library call."""
        self._sync_stream()
        s = self._state(U_dev)
        hi = state_struct(host_in, self.nv)
        ho = state_struct(host_out, self.nv)
        pin = (ctypes.c_void_p * 5)(*hi.plane)
        pout = (ctypes.c_void_p * 5)(*ho.plane)
        tt = ctypes.c_double(t)
        done = ctypes.c_int32()
        _check(self.lib.hydro_step_host(self.ctx, ctypes.byref(s), pin, pout, int(n_steps),
                                        float(t_end), ctypes.byref(tt), ctypes.byref(done)),
               "hydro_step_host")
        return tt.value, done.value

    def step_host_async(self, U_dev: torch.Tensor, host_in: torch.Tensor, host_out: torch.Tensor,
                        n_steps: int, t_end: float = 0.0, t: float = 0.0):
        """hydro_step_host_async: enqueue the copy in, the steps and the copy back on the current
        torch stream and return; host_in and host_out stay untouched until that stream has
        finished (status() waits for it)."""
        self._sync_stream()
        s = self._state(U_dev)
        hi = state_struct(host_in, self.nv)
        ho = state_struct(host_out, self.nv)
        pin = (ctypes.c_void_p * 5)(*hi.plane)
        pout = (ctypes.c_void_p * 5)(*ho.plane)
        _check(self.lib.hydro_step_host_async(self.ctx, ctypes.byref(s), pin, pout, int(n_steps),
                                              float(t_end), float(t)), "hydro_step_host_async")

    def cfl_dt(self, U: torch.Tensor) -> float:
        self._sync_stream()
        s = self._state(U)
        dt = ctypes.c_double()
        _check(self.lib.hydro_cfl_dt(self.ctx, ctypes.byref(s), ctypes.byref(dt)), "hydro_cfl_dt")
        return dt.value

    def totals(self, U: torch.Tensor):
        self._sync_stream()
        s = self._state(U)
        out = (ctypes.c_double * 5)()
        _check(self.lib.hydro_totals(self.ctx, ctypes.byref(s), out), "hydro_totals")
        return list(out)

    def status(self) -> int:
        return self.lib.hydro_status(self.ctx)

    def set_profiling(self, on: bool):
        _check(self.lib.hydro_set_profiling(self.ctx, 1 if on else 0), "hydro_set_profiling")

    def set_scheme(self, order: int = 2, riemann: int = 0):
        """Reconstruction order (2 MinBee, 1 first order) and HLLC wave speeds (0 Davis, 1
        pressure-based) of later steps."""
        _check(self.lib.hydro_set_scheme(self.ctx, int(order), int(riemann)), "hydro_set_scheme")

    def set_analytic(self, kind, theta: float = 0.0, amplitude: float = 1.0):
        """Exact solution of the analytic boundaries (kind "entropy", "sound", "shock_tube" or
        1-3), travelling at angle theta (radians) from the x axis; amplitude of the sound wave."""
        k = ANALYTIC_KINDS[kind] if isinstance(kind, str) else int(kind)
        _check(self.lib.hydro_set_analytic(self.ctx, k, float(theta), float(amplitude)),
               "hydro_set_analytic")

    def kernel_times(self, reset: bool = False):
        """{kind: (total_ms, launches)} for kinds 'cfl', 'stage1', 'stage2'."""
        ms = (ctypes.c_double * 3)()
        n = (ctypes.c_int64 * 3)()
        _check(self.lib.hydro_kernel_times(self.ctx, ms, n, 3, 1 if reset else 0),
               "hydro_kernel_times")
        return {k: (ms[i], n[i]) for i, k in enumerate(("cfl", "stage1", "stage2"))}


class BatchSolver:
    """Many independent 2D grids of uneven size advanced together (hydro_batch_* of the C ABI).

    shapes: sequence of (nx, ny); every grid is its own unit square with its own CFL dt.
    tile: (bx, by) of the batch kernels, default (32, 8); (bx, 1) selects row tiles, which march
    along y through `march` rows per work item (default 32).
    The packed state is a tensor of shape (4, total_cells): plane k holds grid g's cells at
    [offsets[g], offsets[g+1]), x fastest.
    """

    def __init__(self, shapes, gamma: float, bc="periodic", dtype=torch.float32, cfl: float = 0.4,
                 tile=None, march: int = 0, device=None):
        self.lib = load_library()
        self.shapes = [(int(a), int(b)) for a, b in shapes]
        self.n = len(self.shapes)
        self.gamma, self.cfl, self.dtype = float(gamma), float(cfl), dtype
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        if isinstance(bc, (str, int)):
            bc = [bc, bc]
        bcs = (ctypes.c_int32 * 2)(*[HYDRO_BC_PERIODIC if b in ("periodic", 0) else HYDRO_BC_OUTFLOW
                                     for b in bc])
        nx = (ctypes.c_int64 * self.n)(*[s[0] for s in self.shapes])
        ny = (ctypes.c_int64 * self.n)(*[s[1] for s in self.shapes])
        var = Variant(int(tile[0]), int(tile[1]), int(march), 0, 0, 0) if tile else None
        nbytes = ctypes.c_size_t()
        _check(self.lib.hydro_batch_workspace_bytes(self.n, nx, ny, _prec(dtype),
                                                    ctypes.byref(var) if var else None,
                                                    ctypes.byref(nbytes)), "hydro_batch_workspace_bytes")
        self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device=self.device)
        ctx = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(self.lib.hydro_batch_create(self.n, nx, ny, self.gamma, bcs, _prec(dtype), self.cfl,
                                               ctypes.byref(var) if var else None,
                                               self.workspace.data_ptr(), int(nbytes.value),
                                               _stream_ptr(self.device), ctypes.byref(ctx)),
                   "hydro_batch_create")
        self.ctx = ctx
        offs = (ctypes.c_int64 * (self.n + 1))()
        _check(self.lib.hydro_batch_offsets(self.ctx, offs), "hydro_batch_offsets")
        self.offsets = list(offs)
        self.total = self.offsets[-1]

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.hydro_batch_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def empty_state(self) -> torch.Tensor:
        return torch.empty((4, self.total), dtype=self.dtype, device=self.device)

    def grid_view(self, packed: torch.Tensor, g: int) -> torch.Tensor:
        """(4, ny, nx) view of grid g inside a packed tensor."""
        nx, ny = self.shapes[g]
        return packed[:, self.offsets[g]:self.offsets[g + 1]].view(4, ny, nx)

    def _state(self, U: torch.Tensor) -> State:
        if U.dtype != self.dtype or tuple(U.shape) != (4, self.total):
            raise ValueError("packed state must be (4, total_cells) of the batch dtype")
        return state_struct(U, 4)

    def step(self, U: torch.Tensor, n_steps: int, t_end: float = 0.0, t=None, sync: bool = True):
        """Advance every grid in place; returns (t per grid, steps per grid)."""
        self.lib.hydro_batch_set_stream(self.ctx, _stream_ptr(self.device))
        s = self._state(U)
        if not sync:
            _check(self.lib.hydro_batch_step(self.ctx, ctypes.byref(s), int(n_steps), float(t_end),
                                             None, None), "hydro_batch_step")
            return None, None
        tt = (ctypes.c_double * self.n)(*(t if t is not None else [0.0] * self.n))
        done = (ctypes.c_int32 * self.n)()
        _check(self.lib.hydro_batch_step(self.ctx, ctypes.byref(s), int(n_steps), float(t_end), tt,
                                         done), "hydro_batch_step")
        return list(tt), list(done)

    def totals(self, U: torch.Tensor):
        self.lib.hydro_batch_set_stream(self.ctx, _stream_ptr(self.device))
        s = self._state(U)
        out = (ctypes.c_double * (5 * self.n))()
        _check(self.lib.hydro_batch_totals(self.ctx, ctypes.byref(s), out), "hydro_batch_totals")
        return [list(out[5 * g:5 * g + 5]) for g in range(self.n)]

    def set_profiling(self, on: bool):
        _check(self.lib.hydro_batch_set_profiling(self.ctx, 1 if on else 0), "hydro_batch_set_profiling")

    def kernel_times(self, reset: bool = False):
        ms = (ctypes.c_double * 3)()
        n = (ctypes.c_int64 * 3)()
        _check(self.lib.hydro_batch_kernel_times(self.ctx, ms, n, 3, 1 if reset else 0),
               "hydro_batch_kernel_times")
        return {k: (ms[i], n[i]) for i, k in enumerate(("cfl", "stage1", "stage2"))}


def fma_rate(dtype=torch.float32, device=None) -> float:
    """Measured FMA throughput of the device (hydro_fma_rate), in lane operations per second."""
    lib = load_library()
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    out = ctypes.c_double()
    with torch.cuda.device(dev):
        _check(lib.hydro_fma_rate(_prec(dtype), _stream_ptr(dev), ctypes.byref(out)), "hydro_fma_rate")
    return out.value


def wait_bound_check(device=None):
    """hydro_wait_bound_check: (threads of 32 that gave up waiting on an mbarrier phase that never
    completes, the kernel's milliseconds)."""
    lib = load_library()
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    buf = torch.zeros(1, dtype=torch.int32, device=dev)
    n, ms = ctypes.c_int32(), ctypes.c_double()
    with torch.cuda.device(dev):
        _check(lib.hydro_wait_bound_check(ctypes.c_void_p(buf.data_ptr()), _stream_ptr(dev),
                                          ctypes.byref(n), ctypes.byref(ms)), "hydro_wait_bound_check")
    return n.value, ms.value


def wave_run(f: torch.Tensor, g: torch.Tensor, c: float, length: float, dt: float, n_steps: int):
    """The paper's linear-wave example (hydro_wave_run): advance f, g (1D device tensors, float32
    or float64) in place by n_steps steps; returns the FP64 energy after each step."""
    lib = load_library()
    if f.shape != g.shape or f.dim() != 1 or f.dtype != g.dtype:
        raise ValueError("f and g must be 1D tensors of one shape and dtype")
    n = f.numel()
    nbytes = ctypes.c_size_t()
    _check(lib.hydro_wave_workspace_bytes(n, _prec(f.dtype), int(n_steps), ctypes.byref(nbytes)),
           "hydro_wave_workspace_bytes")
    ws = torch.empty(int(nbytes.value), dtype=torch.uint8, device=f.device)
    energy = (ctypes.c_double * max(int(n_steps), 1))()
    _check(lib.hydro_wave_run(_prec(f.dtype), n, float(c), float(length), float(dt), f.data_ptr(),
                              g.data_ptr(), int(n_steps), energy, ws.data_ptr(), int(nbytes.value),
                              _stream_ptr(f.device)), "hydro_wave_run")
    return list(energy)[:int(n_steps)]
