"""Plain FP64 CPU oracle of the Paraiso compressible-Euler step (arXiv:1204.4779, section 4.1).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` are the only callers.  The solver package never imports this module, and this module
imports nothing from the solver package.

The arithmetic lives in ``hydro_oracle.c`` (plain C, ``-O2 -ffp-contract=off``, no fast-math).  This
wrapper only builds it with gcc, loads it with ctypes and marshals numpy arrays.

Arrays are numpy float64 of shape ``(dim+2, nz, ny, nx)`` (trailing axes dropped for dim < 3):
structure of arrays, x fastest.  Conserved planes are (rho, m_x, [m_y, [m_z]], E); primitive planes are
(rho, v_x, [v_y, [v_z]], p).
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hydro_oracle.c")
_LIB = os.path.join(_HERE, "libhydro_oracle.so")
_lock = threading.Lock()
_lib = None

ORC_OK, ORC_EINVAL, ORC_ENOMEM, ORC_ENONFINITE = 0, 1, 2, 3


class OracleError(RuntimeError):
    pass


def build(force: bool = False, src: str = _SRC, out: str = _LIB) -> str:
    """Compile hydro_oracle.c into libhydro_oracle.so (OpenMP when the compiler has it)."""
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-shared", "-fPIC"]
    tmp = out + f".tmp{os.getpid()}"
    try:
        subprocess.run(base + ["-fopenmp", "-o", tmp, src, "-lm"], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-o", tmp, src, "-lm"], check=True, capture_output=True, text=True)
    os.replace(tmp, out)
    return out


_OPC_SRC = os.path.join(_HERE, "opcount.cpp")
_OPC_LIB = os.path.join(_HERE, "libhydro_oracle_opcount.so")
OP_KINDS = ("add", "mul", "div", "sqrt", "cmp", "minmax", "abs", "neg")


def build_opcount(force: bool = False, out: str = _OPC_LIB) -> str:
    """Compile the operation-counting build (opcount.cpp: hydro_oracle.c as C++ with a counting
    number type in place of double), single-threaded."""
    newest = max(os.path.getmtime(_OPC_SRC), os.path.getmtime(_SRC))
    if not force and os.path.exists(out) and os.path.getmtime(out) >= newest:
        return out
    tmp = out + f".tmp{os.getpid()}"
    subprocess.run(["g++", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c++17",
                    "-Wno-unknown-pragmas", "-shared", "-fPIC", "-o", tmp, _OPC_SRC, "-lm"],
                   check=True, capture_output=True, text=True)
    os.replace(tmp, out)
    return out


@contextlib.contextmanager
def counting_ops():
    """Route every oracle call through the counting build.  Yields `counts()`, which returns the
    floating-point operations performed since entry, by kind (OP_KINDS), as a dict."""
    path = build_opcount()
    raw = ctypes.CDLL(path)
    n = raw.oracle_opcount_kinds()
    buf = (ctypes.c_ulonglong * n)()

    def counts():
        raw.oracle_opcount_get(buf)
        return dict(zip(OP_KINDS, (int(v) for v in buf)))

    with using_library(path):
        raw.oracle_opcount_reset()
        yield counts


@contextlib.contextmanager
def using_library(path: str):
    """Temporarily route every call through another build of the oracle (used by the tests
    that plant mistakes in a copy of the source and check that a pin catches them)."""
    global _lib
    with _lock:
        saved = _lib
        _lib = _bind(ctypes.CDLL(path))
    try:
        yield
    finally:
        with _lock:
            _lib = saved


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        _lib = _bind(ctypes.CDLL(_LIB))
        return _lib


def _bind(lib):
    """Declare the C signatures of the oracle entry points on a loaded library."""
    dp = ctypes.POINTER(ctypes.c_double)
    lp = ctypes.POINTER(ctypes.c_long)
    ip = ctypes.POINTER(ctypes.c_int)
    c_int, c_double = ctypes.c_int, ctypes.c_double
    lib.oracle_interpolate.argtypes = [c_double, c_double, c_double, dp, dp]
    lib.oracle_interpolate.restype = None
    lib.oracle_hllc.argtypes = [c_int, c_int, c_double, dp, dp, dp]
    lib.oracle_hllc.restype = None
    lib.oracle_euler_flux.argtypes = [c_int, c_int, c_double, dp, dp]
    lib.oracle_euler_flux.restype = None
    lib.oracle_prim_to_cons.argtypes = [c_int, lp, c_double, dp, dp]
    lib.oracle_cons_to_prim.argtypes = [c_int, lp, c_double, dp, dp]
    lib.oracle_cfl_dt.argtypes = [c_int, lp, dp, c_double, dp, c_double, dp]
    lib.oracle_fluxes.argtypes = [c_int, lp, dp, c_double, ip, dp, ctypes.POINTER(dp)]
    lib.oracle_run.argtypes = [c_int, lp, dp, c_double, ip, c_double, dp, c_int, c_double,
                               dp, ip, c_int]
    lib.oracle_run_opt.argtypes = [c_int, lp, dp, c_double, ip, c_double, c_int, c_int, dp, c_int,
                                   c_double, dp, ip, c_int, c_int, c_double, c_double]
    lib.oracle_run_opt.restype = c_int
    lib.oracle_hllc_opt.argtypes = [c_int, c_int, c_double, c_int, dp, dp, dp]
    lib.oracle_hllc_opt.restype = None
    lib.oracle_sod_sample.argtypes = [c_double, c_double, dp, dp]
    lib.oracle_sod_sample.restype = None
    lib.oracle_totals.argtypes = [c_int, lp, dp, dp, dp]
    for f in ("oracle_prim_to_cons", "oracle_cons_to_prim", "oracle_cfl_dt", "oracle_fluxes",
              "oracle_run", "oracle_totals", "oracle_has_openmp", "oracle_max_threads"):
        getattr(lib, f).restype = c_int
    return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _shape_info(q: np.ndarray):
    """(dim, n[3]) from an SoA array of shape (dim+2, [nz, [ny,]] nx)."""
    dim = q.ndim - 1
    if dim < 1 or dim > 3 or q.shape[0] != dim + 2:
        raise ValueError(f"expected shape (dim+2, ..., nx), got {q.shape}")
    n = list(reversed(q.shape[1:])) + [1] * (3 - dim)
    return dim, (ctypes.c_long * 3)(*n)


def _c64(q) -> np.ndarray:
    return np.ascontiguousarray(q, dtype=np.float64)


def has_openmp() -> bool:
    return bool(_load().oracle_has_openmp())


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def interpolate(y0: float, y1: float, y2: float):
    """Eq. eqInterpolateSingle: returns (value at the lower face, value at the upper face)."""
    lo, hi = ctypes.c_double(), ctypes.c_double()
    _load().oracle_interpolate(y0, y1, y2, ctypes.byref(lo), ctypes.byref(hi))
    return lo.value, hi.value


def hllc(dim: int, axis: int, gamma: float, VL, VR, riemann: int = 0) -> np.ndarray:
    """HLLC flux through a face with normal `axis` from primitive states VL (lower) and VR
    (upper); riemann: wave-speed estimate, 0 Davis (default), 1 pressure-based."""
    vl, vr = _c64(VL), _c64(VR)
    out = np.zeros(dim + 2)
    if riemann == 0:
        _load().oracle_hllc(dim, axis, gamma, _dp(vl), _dp(vr), _dp(out))
    else:
        _load().oracle_hllc_opt(dim, axis, gamma, riemann, _dp(vl), _dp(vr), _dp(out))
    return out


def euler_flux(dim: int, axis: int, gamma: float, V) -> np.ndarray:
    v = _c64(V)
    out = np.zeros(dim + 2)
    _load().oracle_euler_flux(dim, axis, gamma, _dp(v), _dp(out))
    return out


def prim_to_cons(V, gamma: float) -> np.ndarray:
    v = _c64(V)
    dim, n = _shape_info(v)
    u = np.empty_like(v)
    _load().oracle_prim_to_cons(dim, n, gamma, _dp(v), _dp(u))
    return u


def cons_to_prim(U, gamma: float) -> np.ndarray:
    u = _c64(U)
    dim, n = _shape_info(u)
    v = np.empty_like(u)
    _load().oracle_cons_to_prim(dim, n, gamma, _dp(u), _dp(v))
    return v


def _dr(dim, n, dr):
    if dr is None:
        dr = [1.0 / n[a] for a in range(dim)]
    dr = list(dr) + [1.0] * (3 - len(dr))
    return (ctypes.c_double * 3)(*dr)


def cfl_dt(U, gamma: float, cfl: float, dr=None) -> float:
    u = _c64(U)
    dim, n = _shape_info(u)
    out = ctypes.c_double()
    rc = _load().oracle_cfl_dt(dim, n, _dr(dim, n, dr), gamma, _dp(u), cfl, ctypes.byref(out))
    if rc:
        raise OracleError(f"oracle_cfl_dt rc={rc}")
    return out.value


def fluxes(U, gamma: float, bc=(0, 0, 0), dr=None):
    """Face fluxes of every axis; element a has shape (dim+2, face counts) with face i-1/2 at index i."""
    u = _c64(U)
    dim, n = _shape_info(u)
    outs = []
    for a in range(dim):
        shape = [n[b] + (1 if b == a else 0) for b in range(3)]
        outs.append(np.zeros((dim + 2, shape[2], shape[1], shape[0])))
    ptrs = (ctypes.POINTER(ctypes.c_double) * 3)(*([_dp(o) for o in outs] + [None] * (3 - dim)))
    bcs = (ctypes.c_int * 3)(*(list(bc) + [0] * (3 - len(bc))))
    rc = _load().oracle_fluxes(dim, n, _dr(dim, n, dr), gamma, bcs, _dp(u), ptrs)
    if rc:
        raise OracleError(f"oracle_fluxes rc={rc}")
    return [o.reshape((dim + 2,) + tuple(reversed(
        [n[b] + (1 if b == a else 0) for b in range(dim)]))) for a, o in enumerate(outs)]


ANALYTIC_ENTROPY_WAVE, ANALYTIC_SOUND_WAVE, ANALYTIC_SHOCK_TUBE = 1, 2, 3


def sod_sample(gamma: float, xi: float):
    """Exact solution of Sod's shock tube (1, 0, 1) | (0.125, 0, 0.1) at xi = (x - x0) / t:
    ((rho, u, p), (p*, u*))."""
    out = np.zeros(3)
    star = np.zeros(2)
    _load().oracle_sod_sample(float(gamma), float(xi), _dp(out), _dp(star))
    return out, star


def run(U, gamma: float, cfl: float, n_steps: int, bc=(0, 0, 0), t_end: float = 0.0,
        t0: float = 0.0, dr=None, threads: int = 1, check: bool = True, order: int = 2,
        riemann: int = 0, analytic=None):
    """Advance a copy of U by up to n_steps midpoint-RK steps (order: reconstruction order 1
    or 2; riemann: HLLC wave speeds, 0 Davis, 1 pressure-based).  bc per axis: 0 periodic,
    1 outflow, 2 the analytic solution analytic = (kind, theta, amplitude) substituted into the
    ghost cells at each stage's time (kind: ANALYTIC_ENTROPY_WAVE, ANALYTIC_SOUND_WAVE or
    ANALYTIC_SHOCK_TUBE, the solution rotated by theta about (1/2, 1/2); section 4.3's
    convergence tests).

    Returns (U_new, t, steps_done, rc).  With t_end > 0 the last step is clipped onto t_end.
    """
    u = _c64(U).copy()
    dim, n = _shape_info(u)
    bcs = (ctypes.c_int * 3)(*(list(bc) + [0] * (3 - len(bc))))
    t = ctypes.c_double(t0)
    done = ctypes.c_int()
    ana = analytic or (0, 0.0, 0.0)
    if order == 2 and riemann == 0 and analytic is None:
        rc = _load().oracle_run(dim, n, _dr(dim, n, dr), gamma, bcs, cfl, _dp(u), int(n_steps),
                                float(t_end), ctypes.byref(t), ctypes.byref(done), int(threads))
    else:
        rc = _load().oracle_run_opt(dim, n, _dr(dim, n, dr), gamma, bcs, cfl, int(order),
                                    int(riemann), _dp(u), int(n_steps), float(t_end),
                                    ctypes.byref(t), ctypes.byref(done), int(threads),
                                    int(ana[0]), float(ana[1]), float(ana[2]))
    if check and rc not in (ORC_OK,):
        raise OracleError(f"oracle_run rc={rc}")
    return u, t.value, done.value, rc


def totals(U, dr=None) -> np.ndarray:
    """(mass, m_x, m_y, m_z, E) integrated over the box: fixed-order pairwise FP64 sums x cell volume."""
    u = _c64(U)
    dim, n = _shape_info(u)
    out = np.zeros(5)
    _load().oracle_totals(dim, n, _dr(dim, n, dr), _dp(u), _dp(out))
    return out
