"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module holds no finite-element arithmetic: it only draws numbers.  Both the
library side and the oracle receive the arrays produced here and build their own
meshes, numberings and operators from them.

Mesh: the unit cube split into nx*ny*nz hexahedra.  Vertices sit on a structured
(nx+1)x(ny+1)x(nz+1) grid, numbered lexicographically with x fastest.  Each vertex
is moved by a uniform random offset in [-amp*h_d, amp*h_d] along direction d
(h_d = 1/n_d), except along directions normal to a boundary plane the vertex lies
on, so that the domain stays exactly the unit cube and its faces stay planar.  The
random stream does not depend on which components are kept: three draws are taken
per vertex, in vertex order, and the unused ones are discarded.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "perturbed_cube_vertices",
    "uniform_vector",
    "problem_mix",
    "serve_requests",
]


def perturbed_cube_vertices(nx: int, ny: int, nz: int, seed: int = 0, amp: float = 0.1) -> np.ndarray:
    """Vertex coordinates, shape ((nx+1)*(ny+1)*(nz+1), 3), float64, x index fastest."""
    if min(nx, ny, nz) < 1:
        raise ValueError("need at least one element per direction")
    n = (nx, ny, nz)
    h = np.array([1.0 / nx, 1.0 / ny, 1.0 / nz])
    # index grids in (z, y, x) storage order so that the flattened order is x-fastest
    kz, ky, kx = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    idx = np.stack([kx.ravel(), ky.ravel(), kz.ravel()], axis=1)          # (nv, 3) integer grid coords
    xyz = idx * h[None, :]
    rng = np.random.default_rng(seed)
    delta = rng.uniform(-1.0, 1.0, size=xyz.shape) * (amp * h)[None, :]
    interior = np.stack([(idx[:, d] > 0) & (idx[:, d] < n[d]) for d in range(3)], axis=1)
    xyz = xyz + np.where(interior, delta, 0.0)
    # boundary coordinates are set exactly (0 or 1), interior ones carry the offset
    return np.ascontiguousarray(xyz, dtype=np.float64)


def uniform_vector(n: int, seed: int = 0, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """n i.i.d. uniform draws in [lo, hi], float64."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=n).astype(np.float64)


def problem_mix(count: int, seed: int = 0, p_range=(1, 6), n_range=(2, 24)) -> list[dict]:
    """A seeded list of independent problems: form (mass/diffusion, prob. 0.5 each),
    order p uniform in p_range, element counts per direction uniform in n_range, and
    per-problem mesh/rhs seeds."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        form = "mass" if rng.uniform() < 0.5 else "diffusion"
        p = int(rng.integers(p_range[0], p_range[1] + 1))
        nx, ny, nz = (int(v) for v in rng.integers(n_range[0], n_range[1] + 1, size=3))
        out.append({"form": form, "p": p, "n": (nx, ny, nz),
                    "mesh_seed": int(rng.integers(0, 2**31 - 1)),
                    "rhs_seed": int(rng.integers(0, 2**31 - 1))})
    return out


def serve_requests(count: int, seed: int = 0, p_range=(1, 8), dofs_range=(1e3, 5e6), mixed_fraction: float = 0.5):
    """A seeded stream of solve requests: form mass/diffusion with probability 1/2, order p
    uniform in p_range, global DOF count log-uniform in dofs_range (a cube with
    round((N^(1/3) - 1) / p) elements per direction, at least 1), precision 'mixed' with
    probability mixed_fraction else 'fp64', and a mesh seed."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        form = "mass" if rng.uniform() < 0.5 else "diffusion"
        p = int(rng.integers(p_range[0], p_range[1] + 1))
        target = float(np.exp(rng.uniform(np.log(dofs_range[0]), np.log(dofs_range[1]))))
        ne = max(1, int(round((target ** (1.0 / 3.0) - 1.0) / p)))
        precision = "mixed" if rng.uniform() < mixed_fraction else "fp64"
        out.append({"form": form, "p": p, "n": (ne, ne, ne), "precision": precision,
                    "mesh_seed": int(rng.integers(0, 2**31 - 1))})
    return out
