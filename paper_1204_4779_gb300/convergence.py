"""The convergence tests of section 4.3 on the GPU: the entropy wave and the sound wave (to
t = 1) and Sod's shock tube (to t = 0.125) on the unit square at resolutions N x N, coaxial
(along x) and oblique (rotated by 60 degrees about (1/2, 1/2)), with the exact solution
substituted outside the square at every RK stage (analytic boundaries).  Each run starts from
the exact solution at t = 0 and is compared with it at the end time.

Errors: the mean absolute density error over the cells (the L1 norm of the density error
vector divided by the cell count), and the same summed over all conserved fields; for the sound
wave both are divided by the amplitude A = 1e-5.

    python -m paper_1204_4779_gb300.convergence --sizes 16 32 64 128 256 512 1024 --dtype f64
"""
from __future__ import annotations

import argparse
import json
import math
import time

import torch

from . import hydro

GAMMA = 1.4
CFL = 0.4
TESTS = {  # kind: (end time, amplitude)
    "entropy": (1.0, 1.0),
    "sound": (1.0, 1e-5),
    "shock_tube": (0.125, 0.0),
}
ANGLES = {"coaxial": 0.0, "oblique": math.pi / 3}


def run(kind: str, theta: float, n: int, dtype=torch.float64, device=None) -> dict:
    """One test at N x N: errors against the exact solution at the end time, steps, seconds."""
    t_end, amp = TESTS[kind]
    U = hydro.analytic_state((n, n), GAMMA, kind, theta, amp, 0.0, dtype=dtype, device=device)
    S = hydro.Solver((n, n), GAMMA, bc="analytic", dtype=dtype, cfl=CFL, device=device)
    S.set_analytic(kind, theta, amp)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    t, steps = S.step(U, 1 << 30, t_end=t_end)
    seconds = time.perf_counter() - t0
    S.close()
    E = hydro.analytic_state((n, n), GAMMA, kind, theta, amp, t_end, dtype=torch.float64,
                             device=device)
    D = (U.double() - E).abs()
    scale = amp if kind == "sound" else 1.0
    return {"kind": kind, "theta": theta, "n": n, "t": t, "steps": steps,
            "l1_rho": float(D[0].mean()) / scale,
            "l1_all": float(D.mean(dim=(1, 2)).sum()) / scale,
            "seconds": seconds}


def orders(errs):
    return [math.log2(a / b) if a > 0 and b > 0 else float("nan") for a, b in zip(errs, errs[1:])]


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--sizes", type=int, nargs="+", default=[16, 32, 64, 128, 256, 512, 1024])
    ap.add_argument("--dtype", choices=["f32", "f64"], default="f64")
    ap.add_argument("--kinds", nargs="+", default=list(TESTS))
    ap.add_argument("--angles", nargs="+", default=list(ANGLES))
    ap.add_argument("--out", default=None, help="write the results as JSON")
    a = ap.parse_args(argv)
    dtype = torch.float32 if a.dtype == "f32" else torch.float64
    results = []
    for kind in a.kinds:
        for name in a.angles:
            rows = [run(kind, ANGLES[name], n, dtype) for n in a.sizes]
            o = orders([r["l1_rho"] for r in rows])
            for r, od in zip(rows, [None] + o):
                r["angle"] = name
                r["order_rho"] = od
                results.append(r)
                print(f"{kind:10s} {name:7s} N={r['n']:5d} steps={r['steps']:6d} "
                      f"L1(rho)={r['l1_rho']:.4e} L1(U)={r['l1_all']:.4e} "
                      f"order={'' if od is None else f'{od:.2f}'} {r['seconds']:.2f}s", flush=True)
    if a.out:
        with open(a.out, "w") as f:
            json.dump({"dtype": a.dtype, "gamma": GAMMA, "cfl": CFL, "results": results}, f,
                      indent=1)


if __name__ == "__main__":
    main()
