"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module holds no finite-element arithmetic: it only draws numbers.  Both the
library side and the oracle receive the arrays produced here and build their own
meshes, numberings and operators from them.

Meshes: the unit cube split into nx*ny*nz hexahedra (structured vertex grid, or the same
mesh as vertices + element connectivity with its structure hidden), and an unstructured
hexahedral mesh of the unit cube (tiles of five quadrilaterals, extruded).

Structured mesh: the unit cube split into nx*ny*nz hexahedra.  Vertices sit on a structured
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
    "grid_connectivity",
    "scrambled_hex_mesh",
    "tiled_unstructured_cube",
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


def grid_connectivity(nx: int, ny: int, nz: int) -> np.ndarray:
    """(nx*ny*nz, 8) int32 vertex ids of the structured grid's elements, element
    ex + nx*(ey + ny*ez), corner (i, j, k) at column i + 2j + 4k (vertex ids as in
    perturbed_cube_vertices)."""
    ez, ey, ex = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ex, ey, ez = ex.ravel(), ey.ravel(), ez.ravel()
    out = np.empty((nx * ny * nz, 8), dtype=np.int32)
    for c in range(8):
        i, j, k = c & 1, (c >> 1) & 1, (c >> 2) & 1
        out[:, c] = (ex + i) + (nx + 1) * ((ey + j) + (ny + 1) * (ez + k))
    return out


def _cube_rotations() -> list:
    """The 24 rotations of the cube as permutations of its corners: rot[c'] = c means the
    corner at position c' after the rotation is the one that was at c."""
    import itertools
    rots = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            R = np.zeros((3, 3), dtype=int)
            for r in range(3):
                R[r, perm[r]] = signs[r]
            if round(np.linalg.det(R)) != 1:
                continue
            table = []
            for cn in range(8):   # new corner cn at centred position s' = R s
                sp = np.array([2 * ((cn >> d) & 1) - 1 for d in range(3)])
                so = R.T @ sp
                table.append(int(sum(((so[d] + 1) // 2) << d for d in range(3))))
            rots.append(table)
    return rots


def scrambled_hex_mesh(nx: int, ny: int, nz: int, seed: int = 0, amp: float = 0.1):
    """The perturbed cube mesh of perturbed_cube_vertices as (vertices, conn) with its
    structure hidden: vertex ids randomly permuted, elements in random order, and each
    element's corners listed in one of the 24 rotated tensor-product orders (orientation
    kept, so det J stays positive)."""
    verts = perturbed_cube_vertices(nx, ny, nz, seed=seed, amp=amp)
    conn = grid_connectivity(nx, ny, nz)
    rng = np.random.default_rng(seed + 7919)
    vperm = rng.permutation(len(verts))          # old id -> new id
    new_verts = np.empty_like(verts)
    new_verts[vperm] = verts
    conn = vperm[conn]
    conn = conn[rng.permutation(len(conn))]
    rots = _cube_rotations()
    pick = rng.integers(0, len(rots), size=len(conn))
    out = np.empty_like(conn)
    for e in range(len(conn)):
        out[e] = conn[e][rots[pick[e]]]
    return np.ascontiguousarray(new_verts), np.ascontiguousarray(out.astype(np.int32))


def tiled_unstructured_cube(m: int, nz: int, seed: int = 0, inner: float = 0.3, jitter: float = 0.05,
                            scramble: bool = True):
    """An unstructured hexahedral mesh of the unit cube: the unit square is cut into m x m
    tiles, each tile into 5 quadrilaterals (an inner square with corners at `inner` and
    1 - `inner` of the tile, jittered by +-jitter of the tile size, and the 4 trapezoids
    between it and the tile's sides), and that 2D mesh is extruded through nz layers.  The
    inner corners have 3 quadrilaterals around them (edges of 3 hexahedra), which a
    structured grid never has.  With scramble, vertex ids, element order and each element's
    corner order are randomised as in scrambled_hex_mesh.  Returns (vertices, conn)."""
    rng = np.random.default_rng(seed)
    h = 1.0 / m
    pts = [(i * h, j * h) for j in range(m + 1) for i in range(m + 1)]   # tile corners
    quads = []
    for ty in range(m):
        for tx in range(m):
            o = [tx + (m + 1) * ty, tx + 1 + (m + 1) * ty, tx + 1 + (m + 1) * (ty + 1), tx + (m + 1) * (ty + 1)]
            base = len(pts)
            for (a, b) in ((inner, inner), (1 - inner, inner), (1 - inner, 1 - inner), (inner, 1 - inner)):
                da, db = rng.uniform(-jitter, jitter, size=2)
                pts.append(((tx + a + da) * h, (ty + b + db) * h))
            i0, i1, i2, i3 = base, base + 1, base + 2, base + 3
            # counter-clockwise quadrilaterals
            quads += [[i0, i1, i2, i3], [o[0], o[1], i1, i0], [o[1], o[2], i2, i1], [o[2], o[3], i3, i2],
                      [o[3], o[0], i0, i3]]
    pts = np.asarray(pts)
    n2 = len(pts)
    z = np.linspace(0.0, 1.0, nz + 1)
    verts = np.concatenate([np.column_stack([pts, np.full(n2, zk)]) for zk in z])
    conn = []
    for k in range(nz):
        for q0, q1, q2, q3 in quads:
            lo, hi = k * n2, (k + 1) * n2
            # tensor order: (0,0)=q0, (1,0)=q1, (0,1)=q3, (1,1)=q2, then the upper layer
            conn.append([lo + q0, lo + q1, lo + q3, lo + q2, hi + q0, hi + q1, hi + q3, hi + q2])
    conn = np.asarray(conn, dtype=np.int32)
    if not scramble:
        return verts, conn
    vperm = rng.permutation(len(verts))
    new_verts = np.empty_like(verts)
    new_verts[vperm] = verts
    conn = vperm[conn]
    conn = conn[rng.permutation(len(conn))]
    rots = _cube_rotations()
    pick = rng.integers(0, len(rots), size=len(conn))
    out = np.array([conn[e][rots[pick[e]]] for e in range(len(conn))], dtype=np.int32)
    return np.ascontiguousarray(new_verts), np.ascontiguousarray(out)


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
