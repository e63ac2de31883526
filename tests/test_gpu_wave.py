"""The linear-wave example on the GPU (hydro_wave_run) against the FP64 oracle: states and
per-step energies for N = 8 ... 3072 (the paper's range, FP64), energy conservation at a large
size, and the FP32 form."""
import math

import numpy as np
import pytest

from oracle import wave_oracle as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
C = 3.43


@pytest.mark.parametrize("n", [8, 9, 256, 257, 3072])
def test_fp64_matches_oracle(n):
    from paper_1204_4779_gb300 import hydro
    f0, g0 = W.initial(n)
    dx = 2 * math.pi / n
    dt = dx / C
    steps = 301
    fo, go, Eo = W.run(f0, g0, C, 2 * math.pi, dt, steps)
    f = torch.from_numpy(f0.copy()).cuda()
    g = torch.from_numpy(g0.copy()).cuda()
    E = np.array(hydro.wave_run(f, g, C, 2 * math.pi, dt, steps))
    assert np.max(np.abs(f.cpu().numpy() - fo)) <= 1e-12 * np.max(np.abs(fo))
    assert np.max(np.abs(g.cpu().numpy() - go)) <= 1e-12 * np.max(np.abs(go))
    assert np.max(np.abs(E - Eo)) <= 1e-13 * Eo.mean()
    assert (E.max() - E.min()) / E.mean() < 1e-12


def test_energy_conserved_at_large_size():
    from paper_1204_4779_gb300 import hydro
    n = 1 << 22
    x = torch.arange(n, dtype=torch.float64, device="cuda") * (2 * math.pi / n)
    f, g = torch.sin(x), torch.cos(3 * x)
    dt = (2 * math.pi / n) / C
    E = np.array(hydro.wave_run(f, g, C, 2 * math.pi, dt, 200))
    assert (E.max() - E.min()) / E.mean() < 1e-12


def test_fp32_energy_and_state():
    from paper_1204_4779_gb300 import hydro
    n = 1024
    f0, g0 = W.initial(n)
    dt = (2 * math.pi / n) / C
    fo, go, Eo = W.run(f0, g0, C, 2 * math.pi, dt, 200)
    f = torch.from_numpy(f0).float().cuda()
    g = torch.from_numpy(g0).float().cuda()
    E = np.array(hydro.wave_run(f, g, C, 2 * math.pi, dt, 200))
    assert np.max(np.abs(f.double().cpu().numpy() - fo)) <= 1e-4
    assert np.max(np.abs(E - Eo)) / Eo.mean() <= 1e-5
