"""Oracle parity on the benchmark configurations at their full sizes, one result per
configuration (section 4.1's step through the C ABI against the FP64 CPU oracle):

  * the 512^3 periodic blast (radius 8 cells, gamma 1.4, CFL 0.4, 100 RK steps) in FP32, the
    launch configuration the benchmark times, and in FP64.  The oracle computes it on the
    centred 80^3 sub-box with the full grid's cell size (_helpers.blast_subbox_oracle proves
    at every step that the wrap of the sub-box changes nothing); the GPU run is the whole
    512^3 grid, every cell outside the sub-box must still hold the background bit for bit, and
    the L1 density error is stated over the whole grid (the embedded oracle result) and over
    the sub-box alone;
  * the tuning targets' other grids: the 2048^2 shear layer (gamma 5/3) and the 128^3 blast,
    100 steps, FP32 and FP64.

Gates: FP64 max relative error <= 1e-10 (density and energy element-wise, momenta norm-wise),
FP32 L1(rho) <= 1e-4 relative.  Each test prints one PARITY line with the measured values."""
import numpy as np
import pytest

from _helpers import blast_subbox_oracle, gpu_run, l1_rel, max_rel_err, oracle_run
from paper_1204_4779_gb300 import hydro, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
F32, F64 = torch.float32, torch.float64

N_BLAST, M_BOX, STEPS = 512, 80, 100
LO_BOX = (N_BLAST - M_BOX) // 2


@pytest.fixture(scope="module")
def blast512_oracle():
    return blast_subbox_oracle(N_BLAST, LO_BOX, M_BOX, STEPS, radius=8.0)


def _blast512_gpu(dtype):
    """The whole 512^3 grid on the GPU from the library's FP64 conversion of the blast (cast for
    FP32); returns the state tensor, the initial background values (a corner cell), t and the
    steps taken."""
    n = N_BLAST
    V = inputs.blast_3d_torch(n, 8.0, device="cuda")
    U = hydro.prim_to_cons(V, 1.4).to(dtype).contiguous()
    del V
    bg = U[:, 0, 0, 0].clone()
    S = hydro.Solver((n, n, n), 1.4, bc="periodic", dtype=dtype, cfl=0.4)
    t, steps = S.step(U, STEPS)
    S.close()
    return U, bg, t, steps


def _outside_is_background(U, bg):
    """Every cell outside the sub-box holds the background values bit for bit."""
    lo, hi = LO_BOX, LO_BOX + M_BOX
    for k in range(U.shape[0]):
        same = U[k] == bg[k]
        same[lo:hi, lo:hi, lo:hi] = True
        if not bool(same.all()):
            return False
    return True


def test_blast_512_fp32_full_config_vs_oracle(blast512_oracle):
    O, to = blast512_oracle
    U, bg, tg, steps = _blast512_gpu(F32)
    assert steps == STEPS
    assert abs(tg - to) <= 1e-5 * to, (tg, to)
    assert _outside_is_background(U, bg)
    lo, hi = LO_BOX, LO_BOX + M_BOX
    G = U[:, lo:hi, lo:hi, lo:hi].double().cpu().numpy()
    del U
    diff = float(np.sum(np.abs(G[0] - O[0])))
    total = float(np.sum(np.abs(O[0]))) + (N_BLAST ** 3 - M_BOX ** 3) * 1.0
    l1_full = diff / total
    l1_box = diff / float(np.sum(np.abs(O[0])))
    print(f"PARITY blast512 fp32 l1_rho_full={l1_full:.3e} l1_rho_subbox={l1_box:.3e} "
          f"t_gpu={tg!r} t_oracle={to!r}")
    assert l1_full <= 1e-4 and l1_box <= 1e-4


@pytest.mark.slow
def test_blast_512_fp64_full_config_vs_oracle(blast512_oracle):
    O, to = blast512_oracle
    U, bg, tg, steps = _blast512_gpu(F64)
    assert steps == STEPS
    assert abs(tg - to) <= 1e-14 * to, (tg, to)
    assert _outside_is_background(U, bg)
    lo, hi = LO_BOX, LO_BOX + M_BOX
    G = U[:, lo:hi, lo:hi, lo:hi].cpu().numpy()
    del U
    err = max_rel_err(G, O)
    print(f"PARITY blast512 fp64 max_rel={err:.3e} t_gpu={tg!r} t_oracle={to!r}")
    assert err <= 1e-10


# ---- the other grids of the tuning configuration ---------------------------------------

@pytest.fixture(scope="module")
def kh2048_oracle():
    V = inputs.kh_2d(2048, seed=1204477905)
    O, to, so, _ = oracle_run(V, 5.0 / 3.0, (0, 0), 0.4, STEPS)
    return V, O, to, so


@pytest.fixture(scope="module")
def blast128_oracle():
    V = inputs.blast_3d(128, radius_cells=8.0)
    O, to, so, _ = oracle_run(V, 1.4, (0, 0, 0), 0.4, STEPS)
    return V, O, to, so


def test_kh_2048_fp32_vs_oracle(kh2048_oracle):
    V, O, to, so = kh2048_oracle
    G, tg, sg = gpu_run(V, 5.0 / 3.0, (0, 0), F32, 0.4, STEPS)
    assert sg == so == STEPS and abs(tg - to) <= 1e-5 * to
    e = l1_rel(G[0], O[0])
    print(f"PARITY kh2048 fp32 l1_rho={e:.3e}")
    assert e <= 1e-4


def test_kh_2048_fp64_vs_oracle(kh2048_oracle):
    V, O, to, so = kh2048_oracle
    G, tg, sg = gpu_run(V, 5.0 / 3.0, (0, 0), F64, 0.4, STEPS)
    assert sg == so and tg == to
    err = max_rel_err(G, O)
    print(f"PARITY kh2048 fp64 max_rel={err:.3e}")
    assert err <= 1e-10


def test_blast_128_fp32_vs_oracle(blast128_oracle):
    V, O, to, so = blast128_oracle
    G, tg, sg = gpu_run(V, 1.4, (0, 0, 0), F32, 0.4, STEPS)
    assert sg == so == STEPS and abs(tg - to) <= 1e-5 * to
    e = l1_rel(G[0], O[0])
    print(f"PARITY blast128 fp32 l1_rho={e:.3e}")
    assert e <= 1e-4


def test_blast_128_fp64_vs_oracle(blast128_oracle):
    V, O, to, so = blast128_oracle
    G, tg, sg = gpu_run(V, 1.4, (0, 0, 0), F64, 0.4, STEPS)
    assert sg == so and tg == to
    err = max_rel_err(G, O)
    print(f"PARITY blast128 fp64 max_rel={err:.3e}")
    assert err <= 1e-10
