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


def outer_layers_equal(U, bg, w):
    """True if every cell within w cells of a face of the box holds exactly the values bg
    (one value per field)."""
    dim = U.ndim - 1
    for ax in range(1, dim + 1):
        for sl in (slice(0, w), slice(U.shape[ax] - w, U.shape[ax])):
            idx = [slice(None)] * (dim + 1)
            idx[ax] = sl
            part = U[tuple(idx)]
            if not np.all(part == bg.reshape((-1,) + (1,) * dim)):
                return False
    return True


def blast_subbox_oracle(n, lo, m, steps, radius=8.0, gamma=1.4, cfl=0.4, threads=None):
    """The oracle's result for the n^3 periodic blast after `steps` RK steps, restricted to the
    cells [lo, lo + m)^3, computed on that sub-box alone (cell size 1/n, periodic wrap).

    The wrap is exact while the disturbance stays away from the sub-box faces: if the four
    outer cell layers hold the uniform background at the start of a step, stage 1 leaves the
    two outer layers of U1 at the background (a uniform neighbourhood of two cells gives equal
    fluxes), so every ghost cell of either stage reads background values, as on the full grid,
    where everything outside the sub-box is still background; and dt, the maximum of the CFL
    signal, is the same, because the background's signal is below the blast's.  The check is
    made before every step and after the last one; a failure raises.  Returns (U, t)."""
    from paper_1204_4779_gb300 import inputs
    V = inputs.blast_3d_box(n, lo, m, radius)
    U = oracle.prim_to_cons(V, gamma)
    bg = U[:, 0, 0, 0].copy()
    th = oracle.max_threads() if threads is None else threads
    t = 0.0
    for s in range(steps):
        if not outer_layers_equal(U, bg, 4):
            raise AssertionError(f"the disturbance reached the sub-box faces before step {s}")
        U, t, done, _ = oracle.run(U, gamma, cfl, 1, bc=(0, 0, 0), t0=t, dr=[1.0 / n] * 3,
                                   threads=th)
        assert done == 1
    if not outer_layers_equal(U, bg, 4):
        raise AssertionError("the disturbance reached the sub-box faces")
    return U, t
