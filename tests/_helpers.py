"""Shared helpers of the parity tests: run the same seeded primitive initial data through the
CUDA path (via the C ABI) and through the CPU oracle, and measure their difference."""
import numpy as np

import oracle


def shape_of(V):
    return tuple(reversed(V.shape[1:]))


def oracle_run(V, gamma, bc, cfl, n_steps, t_end=0.0, threads=None, order=2, riemann=0):
    U = oracle.prim_to_cons(V, gamma)
    th = oracle.max_threads() if threads is None else threads
    return oracle.run(U, gamma, cfl, n_steps, bc=bc, t_end=t_end, threads=th, order=order,
                      riemann=riemann)


def gpu_state(V, gamma, dtype):
    """Conserved state on the GPU: FP64 conversion by the library, then cast (plumbing)."""
    import torch
    from paper_1204_4779_gb300 import hydro
    V64 = torch.from_numpy(np.ascontiguousarray(V)).to("cuda")
    U64 = hydro.prim_to_cons(V64, gamma)
    return U64.to(dtype).contiguous()


def gpu_run(V, gamma, bc, dtype, cfl, n_steps, t_end=0.0, variant=None, profiling=False,
            scheme=None):
    import torch
    from paper_1204_4779_gb300 import hydro
    U = gpu_state(V, gamma, dtype)
    S = hydro.Solver(shape_of(V), gamma, bc=list(bc), dtype=dtype, cfl=cfl, variant=variant)
    if profiling:
        S.set_profiling(True)
    if scheme is not None:
        S.set_scheme(*scheme)
    t, steps = S.step(U, n_steps, t_end=t_end)
    out = U.to(torch.float64).cpu().numpy()
    S.close()
    return out, t, steps


def max_rel_err(G, O):
    """Largest relative error over fields: density and energy element-wise |g-o|/|o|,
    momenta norm-wise max|g-o| / max|o| (absolute where the reference field is all zero)."""
    nv = O.shape[0]
    errs = []
    for k in range(nv):
        g, o = G[k], O[k]
        if k in (0, nv - 1):
            errs.append(float(np.max(np.abs(g - o) / np.abs(o))))
        else:
            scale = float(np.max(np.abs(o)))
            errs.append(float(np.max(np.abs(g - o))) / (scale if scale > 0 else 1.0))
    return max(errs)


def l1_rel(g, o):
    return float(np.sum(np.abs(g - o)) / np.sum(np.abs(o)))
