"""Seeded synthetic initial data for the compressible-Euler step.

This module holds no part of the numerical method: it only lays out PRIMITIVE fields
(rho, v_x, [v_y, [v_z]], p) on cell centres of the unit box, as float64 numpy arrays of shape
(dim+2, [nz, [ny,]] nx) with x fastest.  Both the CUDA path and the CPU oracle start from these
arrays and convert them to conserved variables with their own code.

Workloads (section 4 of arXiv:1204.4779 gives the Sod, entropy-wave and sound-wave problems;
the others are synthetic stand-ins with the shapes and value ranges of the benchmark configs):
  sod_1d        Sod shock tube, left (1, 0, 1), right (0.125, 0, 0.1), interface at x = 1/2
  kh_2d         two-state shear layer (Kelvin-Helmholtz type), seeded sinusoidal v_y perturbation
  blast_3d      uniform rho = 1, p = 1e-3 with p = 10 inside a sphere around the box centre
  smooth_2d     seeded random smooth periodic data (rho, p in [0.5, 2], |v| < 0.3)
  entropy_wave  rho = 2 + sin(2 pi k.x), v = const, p = 1   (section 4.3 convergence test)
  sound_wave    linear acoustic wave of amplitude A          (section 4.3 convergence test)
  batch_shapes  log-uniform side lengths for the batched configuration
"""
from __future__ import annotations

import math

import numpy as np


def centres(n: int) -> np.ndarray:
    """Cell-centre coordinates of n cells on [0, 1]."""
    return (np.arange(n, dtype=np.float64) + 0.5) / n


def _mesh(shape_xyz):
    """Coordinate arrays (x, [y, [z]]) broadcast to shape (nz, ny, nx) order."""
    axes = [centres(n) for n in shape_xyz]
    grids = np.meshgrid(*reversed(axes), indexing="ij")
    return list(reversed(grids))  # x first


def sod_1d(n: int = 1024, mirrored: bool = False, x0: float = 0.5) -> np.ndarray:
    """Sod shock tube on [0,1]; `mirrored` swaps the sides (x -> 1-x)."""
    x = centres(n)
    left = (x > 1.0 - x0) if mirrored else (x < x0)
    V = np.empty((3, n))
    V[0] = np.where(left, 1.0, 0.125)
    V[1] = 0.0
    V[2] = np.where(left, 1.0, 0.1)
    return V


def kh_2d(n: int = 1024, seed: int = 1204477901, ny: int | None = None) -> np.ndarray:
    """Shear layer: rho = 2, v_x = +0.5 for |y - 1/2| < 1/4; rho = 1, v_x = -0.5 elsewhere;
    v_y = 0.01 sin(4 pi x + phi) with phi ~ U[0, 2pi) drawn from `seed`; p = 2.5."""
    ny = n if ny is None else ny
    rng = np.random.default_rng(seed)
    phi = rng.uniform(0.0, 2.0 * math.pi)
    x, y = _mesh((n, ny))
    inner = np.abs(y - 0.5) < 0.25
    V = np.empty((4, ny, n))
    V[0] = np.where(inner, 2.0, 1.0)
    V[1] = np.where(inner, 0.5, -0.5)
    V[2] = 0.01 * np.sin(4.0 * math.pi * x + phi)
    V[3] = 2.5
    return V


def blast_3d(n: int = 512, radius_cells: float = 8.0, p_in: float = 10.0,
             p_out: float = 1e-3, shape=None) -> np.ndarray:
    """Uniform rho = 1, v = 0, p = p_out, with p = p_in where the cell centre lies within
    radius_cells * (1/n) of the box centre (1/2, 1/2, 1/2)."""
    nx, ny, nz = shape if shape is not None else (n, n, n)
    x, y, z = _mesh((nx, ny, nz))
    h = 1.0 / max(nx, ny, nz)
    r2 = (x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2
    inside = r2 <= (radius_cells * h) ** 2
    V = np.zeros((5, nz, ny, nx))
    V[0] = 1.0
    V[4] = np.where(inside, p_in, p_out)
    return V


def blast_3d_box(n: int, lo: int, m: int, radius_cells: float = 8.0, p_in: float = 10.0,
                 p_out: float = 1e-3) -> np.ndarray:
    """The cells [lo, lo + m) on every axis of the n^3 field of blast_3d, computed directly
    (the same cell-centre coordinates, so the same values as slicing the full field)."""
    c = (np.arange(lo, lo + m, dtype=np.float64) + 0.5) / n
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    h = 1.0 / n
    r2 = (x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2
    inside = r2 <= (radius_cells * h) ** 2
    V = np.zeros((5, m, m, m))
    V[0] = 1.0
    V[4] = np.where(inside, p_in, p_out)
    return V


def smooth(shape_xyz, seed: int, rho=(0.5, 2.0), p=(0.5, 2.0), vmax: float = 0.2) -> np.ndarray:
    """Seeded smooth periodic data: each field is mid + amp * sin(2 pi (k . x) + phi) with
    integer wave numbers k in {1, 2}^dim and phi ~ U[0, 2pi).  rho and p stay inside the given
    ranges and each velocity component inside [-vmax, vmax]."""
    dim = len(shape_xyz)
    rng = np.random.default_rng(seed)
    X = _mesh(tuple(shape_xyz))
    V = np.empty((dim + 2,) + tuple(reversed(shape_xyz)))

    def field():
        k = rng.integers(1, 3, size=dim)
        phase = rng.uniform(0.0, 2.0 * math.pi)
        arg = sum(2.0 * math.pi * k[a] * X[a] for a in range(dim))
        return np.sin(arg + phase)

    V[0] = 0.5 * (rho[0] + rho[1]) + 0.5 * (rho[1] - rho[0]) * field()
    for a in range(dim):
        V[1 + a] = vmax * field()
    V[dim + 1] = 0.5 * (p[0] + p[1]) + 0.5 * (p[1] - p[0]) * field()
    return V


def entropy_wave(shape_xyz, k=(1,), v=(1.0,), amp: float = 1.0) -> np.ndarray:
    """rho = 2 + amp sin(2 pi k.x), constant velocity v, p = 1 (paper, section 4.3)."""
    dim = len(shape_xyz)
    X = _mesh(tuple(shape_xyz))
    kk = list(k) + [0] * (dim - len(k))
    vv = list(v) + [0.0] * (dim - len(v))
    arg = sum(2.0 * math.pi * kk[a] * X[a] for a in range(dim))
    V = np.empty((dim + 2,) + tuple(reversed(shape_xyz)))
    V[0] = 2.0 + amp * np.sin(arg)
    for a in range(dim):
        V[1 + a] = vv[a]
    V[dim + 1] = 1.0
    return V


def sound_wave(shape_xyz, gamma: float = 1.4, amp: float = 1e-5, k=(1,)) -> np.ndarray:
    """rho = gamma (1 + A s), v = A s along k/|k|, p = 1 + gamma A s, s = sin(2 pi k.x)
    (paper, section 4.3; with k = (1,) this is the printed coaxial wave)."""
    dim = len(shape_xyz)
    X = _mesh(tuple(shape_xyz))
    kk = np.array(list(k) + [0] * (dim - len(k)), dtype=np.float64)
    khat = kk / np.linalg.norm(kk)
    s = np.sin(sum(2.0 * math.pi * kk[a] * X[a] for a in range(dim)))
    V = np.empty((dim + 2,) + tuple(reversed(shape_xyz)))
    V[0] = gamma * (1.0 + amp * s)
    for a in range(dim):
        V[1 + a] = amp * s * khat[a]
    V[dim + 1] = 1.0 + gamma * amp * s
    return V


def oblique_wave(shape_xyz, kind: str, theta: float, t: float = 0.0, amp: float = 1.0,
                 gamma: float = 1.4) -> np.ndarray:
    """The convergence-test waves of section 4.3 on the unit square (1D: the line y = 1/2),
    travelling at angle theta from the x axis, at time t: with the coordinate along the wave
    s = (x - 1/2) cos theta + (y - 1/2) sin theta + 1/2 and w = sin(2 pi (s - t)),
    kind "entropy": rho = 2 + amp w, v = (cos theta, sin theta), p = 1;
    kind "sound":   rho = gamma (1 + amp w), v = amp w (cos theta, sin theta), p = 1 + gamma amp w;
    kind "shock_tube" (t = 0 only): Sod's states (rho, v, p) = (1, 0, 1) where s < 1/2, else
    (0.125, 0, 0.1).  Unlike entropy_wave / sound_wave the grid need not be periodic along the
    wave."""
    dim = len(shape_xyz)
    X = _mesh(tuple(shape_xyz))
    x = X[0]
    y = X[1] if dim >= 2 else np.full_like(x, 0.5)
    d = (math.cos(theta), math.sin(theta))
    w = np.sin(2.0 * math.pi * ((x - 0.5) * d[0] + (y - 0.5) * d[1] + 0.5 - t))
    V = np.empty((dim + 2,) + tuple(reversed(shape_xyz)))
    if kind == "shock_tube":
        if t != 0.0:
            raise ValueError("the shock tube's initial states only")
        left = (x - 0.5) * d[0] + (y - 0.5) * d[1] < 0.0
        V[0] = np.where(left, 1.0, 0.125)
        V[1:dim + 1] = 0.0
        V[dim + 1] = np.where(left, 1.0, 0.1)
        return V
    if kind == "entropy":
        V[0] = 2.0 + amp * w
        for a in range(dim):
            V[1 + a] = d[a]
        V[dim + 1] = 1.0
    elif kind == "sound":
        V[0] = gamma * (1.0 + amp * w)
        for a in range(dim):
            V[1 + a] = amp * w * d[a]
        V[dim + 1] = 1.0 + gamma * amp * w
    else:
        raise ValueError(kind)
    return V


def uniform(shape_xyz, rho: float = 1.0, v=(0.0, 0.0, 0.0), p: float = 1.0) -> np.ndarray:
    dim = len(shape_xyz)
    V = np.empty((dim + 2,) + tuple(reversed(shape_xyz)))
    V[0] = rho
    for a in range(dim):
        V[1 + a] = v[a]
    V[dim + 1] = p
    return V


def batch_shapes(n_grids: int = 4096, seed: int = 1204477904, lo: int = 32, hi: int = 512):
    """Side lengths (nx, ny) drawn independently and log-uniformly on [lo, hi], rounded."""
    rng = np.random.default_rng(seed)
    s = np.exp(rng.uniform(math.log(lo), math.log(hi), size=(n_grids, 2)))
    return np.clip(np.rint(s).astype(np.int64), lo, hi)


def batch_grid(nx: int, ny: int, seed: int, index: int) -> np.ndarray:
    """Initial data of grid `index` of a batch: seeded smooth data with rho, p in [0.5, 2],
    |v| <= 0.2 per component (so |v| < 0.3)."""
    return smooth((int(nx), int(ny)), seed=seed * 7919 + index, rho=(0.5, 2.0),
                  p=(0.5, 2.0), vmax=0.2)


def blast_3d_torch(n: int = 512, radius_cells: float = 8.0, p_in: float = 10.0,
                   p_out: float = 1e-3, device="cuda", dtype=None):
    """Same field as blast_3d, laid out directly in device memory by torch (for grids too large
    to stage through host numpy arrays)."""
    import torch
    dtype = dtype or torch.float64
    c = (torch.arange(n, device=device, dtype=torch.float64) + 0.5) / n - 0.5
    h = 1.0 / n
    r2 = c.view(1, 1, n) ** 2 + c.view(1, n, 1) ** 2 + c.view(n, 1, 1) ** 2  # x, y, z order
    V = torch.zeros((5, n, n, n), device=device, dtype=dtype)
    V[0] = 1.0
    inside = r2 <= (radius_cells * h) ** 2
    V[4] = p_out
    V[4][inside] = p_in
    return V
