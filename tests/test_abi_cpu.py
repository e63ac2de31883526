"""The C-ABI library loads without a GPU and exports every symbol include/hydro.h declares;
argument checking that needs no device."""
import ctypes
import os
import re

import pytest

from paper_1204_4779_gb300 import hydro

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "hydro.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hydro_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = hydro.load_library()
    syms = declared_symbols()
    assert len(syms) >= 17
    for s in syms:
        assert hasattr(lib, s), s
    assert set(syms) == set(hydro.EXPORTS)


def test_version_and_strerror():
    lib = hydro.load_library()
    assert lib.hydro_version() == 1
    for code in range(7):
        assert lib.hydro_strerror(code)


def _grid(dim, n, lo=0.0, hi=1.0):
    g = hydro.Grid()
    g.dim = dim
    for a in range(3):
        g.n[a] = n[a] if a < len(n) else 1
        g.lo[a] = lo
        g.hi[a] = hi
    return g


def test_workspace_bytes_and_bad_grids():
    lib = hydro.load_library()
    b = ctypes.c_size_t()
    assert lib.hydro_workspace_bytes(ctypes.byref(_grid(3, (512, 512, 512))), hydro.HYDRO_F32,
                                     ctypes.byref(b)) == 0
    assert b.value >= 5 * 512 ** 3 * 4
    for g in (_grid(0, (4,)), _grid(4, (4,)), _grid(2, (0, 4)), _grid(1, (8,), lo=1.0, hi=1.0),
              _grid(3, (2048, 2048, 1024))):
        assert lib.hydro_workspace_bytes(ctypes.byref(g), hydro.HYDRO_F32, ctypes.byref(b)) == \
            hydro.HYDRO_EINVAL
    assert lib.hydro_workspace_bytes(ctypes.byref(_grid(1, (8,))), 7, ctypes.byref(b)) == \
        hydro.HYDRO_EINVAL
    assert lib.hydro_workspace_bytes(None, 0, ctypes.byref(b)) == hydro.HYDRO_EINVAL
    # the per-axis limit: 2^31 - 1024 cells (a tile plus its halo stays below 2^31), and the
    # 1D ghost ring of analytic and exchange boundaries is four cells, not a row
    top = (1 << 31) - 1024
    assert lib.hydro_workspace_bytes(ctypes.byref(_grid(1, (top + 1,))), hydro.HYDRO_F32,
                                     ctypes.byref(b)) == hydro.HYDRO_EINVAL
    assert lib.hydro_workspace_bytes(ctypes.byref(_grid(1, (top,))), hydro.HYDRO_F32,
                                     ctypes.byref(b)) == 0
    assert b.value < 3 * top * 4 + (1 << 20)  # the stage buffer U1 and a few small blocks


def test_create_rejects_bad_arguments_before_touching_the_device():
    lib = hydro.load_library()
    g = _grid(2, (16, 16))
    bc = (ctypes.c_int32 * 3)(0, 0, 0)
    ctx = ctypes.c_void_p()
    ws = ctypes.c_void_p(1 << 20)  # never dereferenced: every call below fails validation
    E = hydro.HYDRO_EINVAL
    assert lib.hydro_create(ctypes.byref(g), 1.0, bc, 1, 0.4, None, ws, 1 << 30, None, ctypes.byref(ctx)) == E
    assert lib.hydro_create(ctypes.byref(g), 1.4, bc, 1, 0.0, None, ws, 1 << 30, None, ctypes.byref(ctx)) == E
    assert lib.hydro_create(ctypes.byref(g), 1.4, bc, 1, 0.4, None, ws, 16, None, ctypes.byref(ctx)) == E
    assert lib.hydro_create(ctypes.byref(g), 1.4, bc, 1, 0.4, None, ctypes.c_void_p((1 << 20) + 8),
                            1 << 30, None, ctypes.byref(ctx)) == E
    assert lib.hydro_create(ctypes.byref(g), 1.4, bc, 1, 0.4, None, None, 1 << 30, None, ctypes.byref(ctx)) == E
    bad_bc = (ctypes.c_int32 * 3)(0, 5, 0)
    assert lib.hydro_create(ctypes.byref(g), 1.4, bad_bc, 1, 0.4, None, ws, 1 << 30, None, ctypes.byref(ctx)) == E
    v = hydro.Variant(7, 7, 0, 0, 0, 0)
    assert lib.hydro_create(ctypes.byref(g), 1.4, bc, 1, 0.4, ctypes.byref(v), ws, 1 << 30, None,
                            ctypes.byref(ctx)) == hydro.HYDRO_EUNSUPPORTED
    assert lib.hydro_create(ctypes.byref(g), 1.4, bc, 1, 0.4, None, ws, 1 << 30, None, None) == E
    assert not ctx.value


def test_null_context_calls_fail_cleanly():
    lib = hydro.load_library()
    E = hydro.HYDRO_EINVAL
    assert lib.hydro_step(None, None, 1, 0.0, None, None) == E
    assert lib.hydro_step_host(None, None, None, None, 1, 0.0, None, None) == E
    assert lib.hydro_step_host_async(None, None, None, None, 1, 0.0, 0.0) == E
    assert lib.hydro_cfl_dt(None, None, None) == E
    assert lib.hydro_totals(None, None, None) == E
    assert lib.hydro_destroy(None) == E
    assert lib.hydro_status(None) == E
    assert lib.hydro_set_profiling(None, 1) == E
    assert lib.hydro_prim_to_cons(4, 10, 1.4, 0, None, None, None) == E


def test_variant_table():
    import torch
    assert hydro.variant_supported(torch.float32, 3)
    assert hydro.variant_supported(torch.float32, 3, (32, 8), 64)
    assert hydro.variant_supported(torch.float64, 2, (32, 8))
    assert not hydro.variant_supported(torch.float32, 3, (8, 8))
    # row tiles (2D)
    assert hydro.variant_supported(torch.float32, 2, (256, 1), 16, occupancy=3)
    assert hydro.variant_supported(torch.float64, 2, (128, 1), 8)
    assert not hydro.variant_supported(torch.float64, 2, (256, 1))
    assert not hydro.variant_supported(torch.float32, 2, (32, 8), occupancy=3)
    # the manifest forms: dim 3, compiled tiles, look-ahead staging, default budget
    for m in (1, 2, 3):
        assert hydro.variant_supported(torch.float32, 3, (16, 8), manifest=m)
        assert hydro.variant_supported(torch.float64, 3, (32, 8), manifest=m)
    assert not hydro.variant_supported(torch.float32, 3, (32, 4), manifest=2)
    assert not hydro.variant_supported(torch.float32, 2, (256, 1), manifest=2)
    assert not hydro.variant_supported(torch.float32, 3, (16, 8), staging=2, manifest=3)
    assert not hydro.variant_supported(torch.float32, 3, (16, 8), occupancy=2, manifest=2)
    assert not hydro.variant_supported(torch.float32, 3, (16, 8), manifest=4)
    assert not hydro.variant_supported(torch.float32, 4)
    assert hydro.variant_supported(torch.float32, 3, (16, 8), 32, split=1, staging=2)
    assert hydro.variant_supported(torch.float64, 3, (32, 8), 32, split=1)
    assert not hydro.variant_supported(torch.float64, 3, (32, 8), 32, staging=2)
    assert hydro.variant_supported(torch.float32, 3, (32, 8), 32, split=2)
    assert not hydro.variant_supported(torch.float32, 3, (32, 8), 32, split=3)
    assert hydro.variant_supported(torch.float32, 2, (32, 8), staging=2)  # one plane: ignored
    assert hydro.variant_supported(torch.float32, 3, (32, 8), 64, occupancy=3)
    assert not hydro.variant_supported(torch.float64, 3, (32, 8), 64, occupancy=3)
    assert not hydro.variant_supported(torch.float32, 2, (32, 8), occupancy=3)
    # the manifest forms: dim 3, compiled tiles, look-ahead staging, default budget
    for m in (1, 2, 3):
        assert hydro.variant_supported(torch.float32, 3, (16, 8), manifest=m)
        assert hydro.variant_supported(torch.float64, 3, (32, 8), manifest=m)
    assert not hydro.variant_supported(torch.float32, 3, (32, 4), manifest=2)
    assert not hydro.variant_supported(torch.float32, 2, (256, 1), manifest=2)
    assert not hydro.variant_supported(torch.float32, 3, (16, 8), staging=2, manifest=3)
    assert not hydro.variant_supported(torch.float32, 3, (16, 8), occupancy=2, manifest=2)
    assert not hydro.variant_supported(torch.float32, 3, (16, 8), manifest=4)
    # TMA plane staging: 3D FP32 16 x 8, either budget, nothing stored between the parts
    assert hydro.variant_supported(torch.float32, 3, (16, 8), staging=3)
    assert hydro.variant_supported(torch.float32, 3, (16, 8), 32, split=1, staging=3, occupancy=2)
    assert not hydro.variant_supported(torch.float32, 3, (32, 8), staging=3)
    assert not hydro.variant_supported(torch.float64, 3, (32, 8), staging=3)
    assert not hydro.variant_supported(torch.float32, 2, (256, 1), staging=3)
    assert not hydro.variant_supported(torch.float32, 3, (16, 8), staging=3, manifest=2)
    assert not hydro.variant_supported(torch.float32, 3, (16, 8), staging=4)


def test_workspace_bytes_of_the_manifest_forms():
    lib = hydro.load_library()
    g = hydro.Grid()
    g.dim = 3
    for a, n in enumerate((40, 36, 30)):
        g.n[a], g.lo[a], g.hi[a] = n, 0.0, 1.0
    sizes = {}
    for m in (1, 2, 3):
        v = hydro.Variant(0, 0, 0, 0, 0, 0, m)
        b = ctypes.c_size_t()
        assert lib.hydro_workspace_bytes_variant(ctypes.byref(g), hydro.HYDRO_F32, ctypes.byref(v),
                                                 ctypes.byref(b)) == 0
        sizes[m] = b.value
    base = ctypes.c_size_t()
    assert lib.hydro_workspace_bytes(ctypes.byref(g), hydro.HYDRO_F32, ctypes.byref(base)) == 0
    ncell = 40 * 36 * 30
    assert sizes[1] == base.value
    assert sizes[2] - sizes[1] >= 5 * ncell * 4                       # the V planes
    faces = 41 * 36 * 30 + 40 * 37 * 30 + 40 * 36 * 31
    assert sizes[3] - sizes[1] >= 5 * faces * 4                       # the face-flux planes
    bad = hydro.Variant(32, 4, 0, 0, 0, 0, 2)
    assert lib.hydro_workspace_bytes_variant(ctypes.byref(g), hydro.HYDRO_F32, ctypes.byref(bad),
                                             ctypes.byref(base)) == hydro.HYDRO_EUNSUPPORTED


def test_header_is_plain_c(tmp_path):
    """include/hydro.h is a C header: it compiles as C99 with -pedantic, warning-free, and every
    type a signature uses is a plain C type."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_header.c"
    src.write_text('#include "hydro.h"\n'
                   "int main(void) {\n"
                   "    hydro_variant_t v = {0, 0, 0, 0, 0, 0, 0};\n"
                   "    hydro_grid_t g;\n"
                   "    (void)v; (void)g;\n"
                   "    return hydro_version() > 0 ? 0 : 1;\n"
                   "}\n")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", inc,
                        "-c", str(src), "-o", str(tmp_path / "use_header.o")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
