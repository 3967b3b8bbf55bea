"""CPU FP64 oracle for high-order H1 mass / diffusion on trilinear hexahedral meshes.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or call this
module: only the tests, the smoke check and the benchmark's CPU-baseline leg do.
It shares no code with the CUDA library (different language, different
algorithm: explicit 3D basis products and full sparse assembly instead of sum
factorisation and partial assembly).

What it computes (arXiv 2402.15940):
  * the finite element operator A = P^T G^T B^T D B G P of Fig. "fig_feod" (Sec. 3.5),
    here with P = I (one subdomain, conforming mesh);
  * partial assembly only reorders the sums of the classical Galerkin matrix built
    with the same quadrature (Sec. 2.2, "assembly levels"), so the oracle builds that
    matrix by its plain definition, element by element, and assembles it into CSR
    ("sparse matrix assembly", Sec. 2.2);
  * the bake-off problems BP1 (mass) and BP3 (diffusion) named in Sec. 2.2;
  * a Krylov solve with a diagonal (Jacobi) preconditioner (Sec. 2.1: iterative
    method plus preconditioner; diagonal-based smoothing), here preconditioned CG.

Readings where the paper is silent (each also listed in the design notes):
  R1 basis: Lagrange polynomials on the Gauss-Lobatto-Legendre (GLL) nodes of order p;
  R2 reference element [0,1]^3, quadrature weights summing to 1;
  R3 global DOF numbering lexicographic over the (p*nx+1)(p*ny+1)(p*nz+1) node grid,
     x fastest; element-local numbering lexicographic (a + n*(b + n*c));
  R5 geometry: the trilinear map from the 8 element corners;
  R6 quadrature: tensor Gauss-Legendre with q points per direction (default p+2);
  R7 coefficient 1;
  R8 Dirichlet: diffusion fixes all boundary DOFs, mass fixes none;
  R9 CG stops when ||r_k||_2 <= rtol * ||b||_2 (unpreconditioned residual), x0 = 0.

All floating point is float64.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

MASS = "mass"
DIFFUSION = "diffusion"


# ----------------------------------------------------------------------------
# 1D rules and bases (sum factorisation, Sec. 2.1, relies on these 1D tables;
# here they only serve to build the explicit 3D basis)
# ----------------------------------------------------------------------------

def gauss_legendre(q: int):
    """q-point Gauss-Legendre rule on [0,1]: points (ascending) and weights (sum 1)."""
    t, w = np.polynomial.legendre.leggauss(q)
    return 0.5 * (t + 1.0), 0.5 * w


def _legendre_and_derivs(n: int, t):
    """P_n(t), P_n'(t), P_n''(t) by the three-term recurrence, in long double."""
    t = np.asarray(t, dtype=np.longdouble)
    p0 = np.ones_like(t)
    if n == 0:
        return p0, np.zeros_like(t), np.zeros_like(t)
    p1 = t.copy()
    for k in range(2, n + 1):
        p0, p1 = p1, ((2 * k - 1) * t * p1 - (k - 1) * p0) / k
    # derivatives from the Legendre ODE: (1-t^2) P'' - 2 t P' + n(n+1) P = 0,
    # and P_n' = n (t P_n - P_{n-1}) / (t^2 - 1)
    d1 = n * (t * p1 - p0) / (t * t - 1.0)
    d2 = (2.0 * t * d1 - n * (n + 1) * p1) / (1.0 - t * t)
    return p1, d1, d2


def gll_points(p: int) -> np.ndarray:
    """The p+1 Gauss-Lobatto-Legendre nodes on [0,1]: the endpoints and the p-1
    roots of P_p' (reading R1)."""
    if p < 1:
        raise ValueError("order must be >= 1")
    if p == 1:
        return np.array([0.0, 1.0])
    # initial guesses: Chebyshev-Gauss-Lobatto points, then Newton on P_p'
    k = np.arange(1, p)
    t = -np.cos(np.pi * k / p).astype(np.longdouble)
    for _ in range(100):
        _, d1, d2 = _legendre_and_derivs(p, t)
        step = d1 / d2
        t = t - step
        if np.max(np.abs(step)) < 1e-30:
            break
    nodes = np.concatenate([[-1.0], np.sort(t.astype(np.float64)), [1.0]])
    return 0.5 * (nodes + 1.0)


def lagrange(nodes: np.ndarray, t: np.ndarray):
    """Values and first derivatives of the Lagrange polynomials on `nodes` at points t.
    Returns V[len(t), n] and dV[len(t), n], from the product formula
    phi_j(t) = prod_{m!=j} (t - t_m)/(t_j - t_m)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    n = len(nodes)
    V = np.ones((len(t), n))
    dV = np.zeros((len(t), n))
    for j in range(n):
        others = [m for m in range(n) if m != j]
        denom = np.prod([nodes[j] - nodes[m] for m in others])
        V[:, j] = np.prod([t - nodes[m] for m in others], axis=0) / denom if others else 1.0
        for l in others:
            rest = [m for m in others if m != l]
            term = np.prod([t - nodes[m] for m in rest], axis=0) if rest else np.ones_like(t)
            dV[:, j] += term / denom
    return V, dV


# ----------------------------------------------------------------------------
# Mesh and numbering (the L-vector / E-vector levels of Fig. fig_feod)
# ----------------------------------------------------------------------------

class HexGridMesh:
    """Structured hexahedral mesh whose (nx+1)(ny+1)(nz+1) vertices may sit anywhere.
    Element e = ex + nx*(ey + ny*ez); its corner c = i + 2j + 4k is vertex
    (ex+i, ey+j, ez+k)."""

    def __init__(self, nx: int, ny: int, nz: int, vertices: np.ndarray):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        v = np.asarray(vertices, dtype=np.float64)
        if v.shape != ((nx + 1) * (ny + 1) * (nz + 1), 3):
            raise ValueError("vertex array has the wrong shape")
        self.vertices = v

    @property
    def num_elements(self) -> int:
        return self.nx * self.ny * self.nz

    def vertex_id(self, i, j, k):
        return i + (self.nx + 1) * (j + (self.ny + 1) * k)

    def element_corners(self) -> np.ndarray:
        """(E, 8, 3) corner coordinates."""
        ez, ey, ex = np.meshgrid(np.arange(self.nz), np.arange(self.ny), np.arange(self.nx), indexing="ij")
        ex, ey, ez = ex.ravel(), ey.ravel(), ez.ravel()
        out = np.empty((self.num_elements, 8, 3))
        for c in range(8):
            i, j, k = c & 1, (c >> 1) & 1, (c >> 2) & 1
            out[:, c, :] = self.vertices[self.vertex_id(ex + i, ey + j, ez + k)]
        return out


class HexMesh:
    """Conforming hexahedral mesh given by its vertices (nverts, 3) and element connectivity
    (E, 8): the vertex ids of each element, corner (i, j, k) of the reference cube at column
    i + 2j + 4k.  The global DOF numbering is hex_numbering's (reading R3 for this input)."""

    def __init__(self, vertices: np.ndarray, conn: np.ndarray):
        self.vertices = np.asarray(vertices, dtype=np.float64)
        self.conn = np.asarray(conn, dtype=np.int64)
        if self.vertices.ndim != 2 or self.vertices.shape[1] != 3 or self.conn.ndim != 2 or self.conn.shape[1] != 8:
            raise ValueError("vertices must be (nverts, 3) and conn (E, 8)")
        self._numbering = {}

    @property
    def num_elements(self) -> int:
        return self.conn.shape[0]

    def element_corners(self) -> np.ndarray:
        """(E, 8, 3) corner coordinates."""
        return self.vertices[self.conn]


def _face_nodes(p: int, d0: int, side: int):
    """Element-local indices of the nodes on the local face where coordinate d0 is side*p."""
    n = p + 1
    return [a + n * (b + n * c) for c in range(n) for b in range(n) for a in range(n)
            if (a, b, c)[d0] == side * p]


def hex_numbering(mesh: HexMesh, p: int):
    """Global DOFs of order p on a connectivity mesh, built from a node's place in the mesh
    rather than from any element's frame: local node (a, b, c) of an element is the point whose
    trilinear weight on corner (i, j, k) is proportional to the integer
    (a or p-a) * (b or p-b) * (c or p-c) (a if i = 1 else p - a, and so on), and the node's key is
    the set of (global vertex id, weight) pairs with nonzero weight.  Elements that share a
    vertex, edge or face give the shared GLL nodes the same key (the GLL points are symmetric, so
    index t from one end is index p - t from the other); interior nodes carry all 8 vertices of
    their element.  DOFs are numbered in sorted key order.  Boundary DOFs: the nodes of every face
    held by one element.  Returns (elem_dofs (E, (p+1)^3), N, boundary DOFs sorted)."""
    if p in mesh._numbering:
        return mesh._numbering[p]
    n = p + 1
    loc = [(a, b, c) for c in range(n) for b in range(n) for a in range(n)]
    wts = np.array([[(a if (cr & 1) else p - a) * (b if (cr >> 1) & 1 else p - b) * (c if (cr >> 2) & 1 else p - c)
                     for cr in range(8)] for (a, b, c) in loc], dtype=np.int64)
    keys = []
    for e in range(mesh.num_elements):
        vid = mesh.conn[e]
        for l in range(len(loc)):
            nz = wts[l] != 0
            keys.append(tuple(sorted(zip(vid[nz].tolist(), wts[l][nz].tolist()))))
    uniq = sorted(set(keys))
    index = {k: i for i, k in enumerate(uniq)}
    dofs = np.array([index[k] for k in keys], dtype=np.int64).reshape(mesh.num_elements, len(loc))
    count = {}
    for e in range(mesh.num_elements):
        for d0 in range(3):
            for side in (0, 1):
                fv = tuple(sorted(mesh.conn[e][[cr for cr in range(8) if ((cr >> d0) & 1) == side]].tolist()))
                count.setdefault(fv, []).append((e, d0, side))
    bdr = set()
    for fv, holders in count.items():
        if len(holders) == 1:
            e, d0, side = holders[0]
            bdr.update(dofs[e, _face_nodes(p, d0, side)].tolist())
    out = (dofs, len(uniq), np.array(sorted(bdr), dtype=np.int64))
    mesh._numbering[p] = out
    return out


def num_dofs(mesh, p: int) -> int:
    if isinstance(mesh, HexMesh):
        return hex_numbering(mesh, p)[1]
    return (p * mesh.nx + 1) * (p * mesh.ny + 1) * (p * mesh.nz + 1)


def elem_dofs(mesh, p: int) -> np.ndarray:
    """(E, (p+1)^3) global DOF of each element-local node (reading R3): the map G."""
    if isinstance(mesh, HexMesh):
        return hex_numbering(mesh, p)[0]
    n = p + 1
    Nx, Ny = p * mesh.nx + 1, p * mesh.ny + 1
    ez, ey, ex = np.meshgrid(np.arange(mesh.nz), np.arange(mesh.ny), np.arange(mesh.nx), indexing="ij")
    ex, ey, ez = ex.ravel(), ey.ravel(), ez.ravel()
    c, b, a = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    a, b, c = a.ravel(), b.ravel(), c.ravel()          # local index a + n*(b + n*c)
    gx = p * ex[:, None] + a[None, :]
    gy = p * ey[:, None] + b[None, :]
    gz = p * ez[:, None] + c[None, :]
    return (gx + Nx * (gy + Ny * gz)).astype(np.int64)


def boundary_dofs(mesh, p: int) -> np.ndarray:
    """Sorted global DOFs on the boundary of the node grid (connectivity mesh: on the faces
    held by one element)."""
    if isinstance(mesh, HexMesh):
        return hex_numbering(mesh, p)[2]
    Nx, Ny, Nz = p * mesh.nx + 1, p * mesh.ny + 1, p * mesh.nz + 1
    gz, gy, gx = np.meshgrid(np.arange(Nz), np.arange(Ny), np.arange(Nx), indexing="ij")
    on = (gx == 0) | (gx == Nx - 1) | (gy == 0) | (gy == Ny - 1) | (gz == 0) | (gz == Nz - 1)
    return np.nonzero(on.ravel())[0].astype(np.int64)


def node_coords(mesh: HexGridMesh, p: int) -> np.ndarray:
    """(N, 3) physical coordinates of every global node (the GLL points mapped by
    the trilinear map of an element that owns them)."""
    n = p + 1
    X = mesh.element_corners()
    r = gll_points(p)
    xi = np.array([[r[a], r[b], r[c]] for c in range(n) for b in range(n) for a in range(n)])
    xs, _ = trilinear(X, xi)
    out = np.empty((num_dofs(mesh, p), 3))
    out[elem_dofs(mesh, p).ravel()] = xs.reshape(-1, 3)
    return out


# ----------------------------------------------------------------------------
# Geometry (what D carries, Sec. 3.5: physical coordinates enter only through D)
# ----------------------------------------------------------------------------

def trilinear(X: np.ndarray, xi: np.ndarray):
    """Trilinear map of elements with corners X (E, 8, 3) at reference points xi (m, 3).
    Returns physical points (E, m, 3) and Jacobians J (E, m, 3, 3), J[d, r] = dx_d/dxi_r."""
    m = xi.shape[0]
    N = np.empty((m, 8))
    dN = np.empty((m, 8, 3))
    for c in range(8):
        bits = [(c >> d) & 1 for d in range(3)]
        f = [xi[:, d] if bits[d] else 1.0 - xi[:, d] for d in range(3)]
        df = [np.ones(m) if bits[d] else -np.ones(m) for d in range(3)]
        N[:, c] = f[0] * f[1] * f[2]
        dN[:, c, 0] = df[0] * f[1] * f[2]
        dN[:, c, 1] = f[0] * df[1] * f[2]
        dN[:, c, 2] = f[0] * f[1] * df[2]
    x = np.einsum("mc,ecd->emd", N, X)
    J = np.einsum("mcr,ecd->emdr", dN, X)
    return x, J


class Rule3D:
    """Tensor quadrature points in [0,1]^3 with point index i + q*(j + q*k), and the
    explicit 3D Lagrange basis tables (no sum factorisation):
    Phi[pt, a] = phi_a0(x) phi_a1(y) phi_a2(z), dPhi[pt, a, r] = d/dxi_r of it."""

    def __init__(self, p: int, q: int):
        self.p, self.q, self.n = p, q, p + 1
        pts, wts = gauss_legendre(q)
        V, dV = lagrange(gll_points(p), pts)
        self.xi = np.array([[pts[i], pts[j], pts[k]] for k in range(q) for j in range(q) for i in range(q)])
        self.w = np.array([wts[i] * wts[j] * wts[k] for k in range(q) for j in range(q) for i in range(q)])
        n = self.n
        lid = [(a, b, c) for c in range(n) for b in range(n) for a in range(n)]
        qid = [(i, j, k) for k in range(q) for j in range(q) for i in range(q)]
        Phi = np.empty((q ** 3, n ** 3))
        dPhi = np.empty((q ** 3, n ** 3, 3))
        for s, (i, j, k) in enumerate(qid):
            for t, (a, b, c) in enumerate(lid):
                Phi[s, t] = V[i, a] * V[j, b] * V[k, c]
                dPhi[s, t, 0] = dV[i, a] * V[j, b] * V[k, c]
                dPhi[s, t, 1] = V[i, a] * dV[j, b] * V[k, c]
                dPhi[s, t, 2] = V[i, a] * V[j, b] * dV[k, c]
        self.Phi, self.dPhi = Phi, dPhi


_rule_cache: dict = {}


def rule(p: int, q: int) -> Rule3D:
    key = (p, q)
    if key not in _rule_cache:
        _rule_cache[key] = Rule3D(p, q)
    return _rule_cache[key]


def _chunks(E: int, per_elem_bytes: int, budget=256 << 20):
    step = max(1, budget // max(per_elem_bytes, 1))
    for s in range(0, E, step):
        yield s, min(E, s + step)


def qp_factors(X: np.ndarray, R: Rule3D, form: str):
    """Per element and quadrature point: w*detJ (mass) or w*detJ*J^{-1}J^{-T} (diffusion),
    computed with a general 3x3 inverse."""
    _, J = trilinear(X, R.xi)
    det = np.linalg.det(J)
    if np.any(det <= 0):
        raise ValueError("non-positive Jacobian determinant (inverted element)")
    wdet = R.w[None, :] * det
    if form == MASS:
        return wdet
    Jinv = np.linalg.inv(J)
    return wdet[..., None, None] * np.einsum("emrd,emsd->emrs", Jinv, Jinv)


# ----------------------------------------------------------------------------
# Element matrices, assembly, action
# ----------------------------------------------------------------------------

def element_matrices(X: np.ndarray, p: int, q: int, form: str) -> np.ndarray:
    """(E, n^3, n^3) element matrices by quadrature:
    mass  Me[a,b] = sum_pt w detJ Phi_a Phi_b,
    diff. Ke[a,b] = sum_pt w detJ (J^{-T} grad Phi_a) . (J^{-T} grad Phi_b)."""
    R = rule(p, q)
    F = qp_factors(X, R, form)
    if form == MASS:
        return np.matmul(R.Phi.T[None, :, :] * F[:, None, :], R.Phi[None, :, :])
    # Ke[a,b] = sum_{pt,r} dPhi[pt,a,r] V[pt,r,b] with V[pt,r,b] = sum_s F[pt,r,s] dPhi[pt,b,s]
    m, n3 = R.dPhi.shape[0], R.dPhi.shape[1]
    V = np.einsum("emrs,mbs->emrb", F, R.dPhi, optimize=True).reshape(X.shape[0], m * 3, n3)
    Pt = R.dPhi.transpose(1, 0, 2).reshape(n3, m * 3)
    return np.matmul(Pt[None, :, :], V)


def assemble_csr(mesh: HexGridMesh, p: int, q: int, form: str) -> sp.csr_matrix:
    """Global sparse matrix: sum over elements of G_e^T A_e G_e (sparse matrix
    assembly level, Sec. 2.2)."""
    n3 = (p + 1) ** 3
    dofs = elem_dofs(mesh, p)
    X = mesh.element_corners()
    N = num_dofs(mesh, p)
    rows, cols, vals = [], [], []
    for s, e in _chunks(mesh.num_elements, n3 * n3 * 8 * 4 + (q ** 3) * n3 * 8 * 6):
        Ae = element_matrices(X[s:e], p, q, form)
        d = dofs[s:e]
        rows.append(np.repeat(d, n3, axis=1).ravel())
        cols.append(np.tile(d, (1, n3)).ravel())
        vals.append(Ae.reshape(e - s, -1).ravel())
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))
    return A.tocsr()


def constrain(A: sp.spmatrix, ess) -> sp.csr_matrix:
    """Constrained operator (I-E) A (I-E) + E for the essential DOF set E."""
    N = A.shape[0]
    keep = np.ones(N)
    keep[np.asarray(ess, dtype=np.int64)] = 0.0
    Kd = sp.diags(keep)
    return (Kd @ A @ Kd + sp.diags(1.0 - keep)).tocsr()


def action_elementwise(mesh: HexGridMesh, p: int, q: int, form: str, x: np.ndarray, ess=None) -> np.ndarray:
    """y = A x without forming any matrix: for each element, evaluate u (or grad u) at
    every quadrature point with the explicit 3D basis, weight, and test against every
    basis function.  With `ess`, returns the constrained product (I-E)A(I-E)x + Ex."""
    x = np.asarray(x, dtype=np.float64)
    xin = x.copy()
    if ess is not None:
        xin[np.asarray(ess, dtype=np.int64)] = 0.0
    R = rule(p, q)
    dofs = elem_dofs(mesh, p)
    X = mesh.element_corners()
    y = np.zeros_like(x)
    for s, e in _chunks(mesh.num_elements, (q ** 3) * 8 * 40):
        F = qp_factors(X[s:e], R, form)
        xe = xin[dofs[s:e]]
        if form == MASS:
            u = xe @ R.Phi.T                                   # (e, m)
            ye = (F * u) @ R.Phi
        else:
            g = np.einsum("mar,ea->emr", R.dPhi, xe, optimize=True)
            v = np.einsum("emrs,ems->emr", F, g)
            ye = np.einsum("mar,emr->ea", R.dPhi, v, optimize=True)
        np.add.at(y, dofs[s:e].ravel(), ye.ravel())
    if ess is not None:
        ess = np.asarray(ess, dtype=np.int64)
        y[ess] = x[ess]
    return y


def elements_of_dof(mesh: HexGridMesh, p: int, dof: int):
    """Elements that contain global node `dof`, with its local index in each."""
    Nx, Ny = p * mesh.nx + 1, p * mesh.ny + 1
    gx, gy, gz = dof % Nx, (dof // Nx) % Ny, dof // (Nx * Ny)
    n = p + 1
    out = []
    def cands(g, ne):
        e0 = g // p
        res = []
        for e in (e0 - 1, e0):
            if 0 <= e < ne and 0 <= g - p * e <= p:
                res.append((e, g - p * e))
        return res
    for ez, c in cands(gz, mesh.nz):
        for ey, b in cands(gy, mesh.ny):
            for ex, a in cands(gx, mesh.nx):
                out.append((ex + mesh.nx * (ey + mesh.ny * ez), a + n * (b + n * c)))
    return out


def action_rows(mesh: HexGridMesh, p: int, q: int, form: str, x: np.ndarray, rows, ess=None) -> np.ndarray:
    """Selected entries y[rows] of y = A x (or of the constrained product), each computed
    from the element rows that touch it.  Cost is independent of the mesh size, so it
    checks full-size results by sampling."""
    x = np.asarray(x, dtype=np.float64)
    ess_set = None
    if ess is not None:
        ess_set = np.zeros(len(x), dtype=bool)
        ess_set[np.asarray(ess, dtype=np.int64)] = True
    R = rule(p, q)
    dofs_all = None
    out = np.empty(len(rows))
    for t, i in enumerate(rows):
        i = int(i)
        if ess_set is not None and ess_set[i]:
            out[t] = x[i]
            continue
        acc = 0.0
        for e, l in elements_of_dof(mesh, p, i):
            ex, ey, ez = e % mesh.nx, (e // mesh.nx) % mesh.ny, e // (mesh.nx * mesh.ny)
            sub = HexGridMesh(1, 1, 1, np.array([mesh.vertices[mesh.vertex_id(ex + (c & 1), ey + ((c >> 1) & 1), ez + ((c >> 2) & 1))]
                                                 for c in range(8)]))
            X = sub.element_corners()
            F = qp_factors(X, R, form)[0]
            d = _element_global_dofs(mesh, p, e)
            xe = x[d].copy()
            if ess_set is not None:
                xe[ess_set[d]] = 0.0
            if form == MASS:
                row = (R.Phi[:, l] * F) @ R.Phi
            else:
                row = np.einsum("mr,mrs,mbs->b", R.dPhi[:, l, :], F, R.dPhi, optimize=True)
            acc += row @ xe
        out[t] = acc
    return out


def _element_global_dofs(mesh: HexGridMesh, p: int, e: int) -> np.ndarray:
    n = p + 1
    ex, ey, ez = e % mesh.nx, (e // mesh.nx) % mesh.ny, e // (mesh.nx * mesh.ny)
    Nx, Ny = p * mesh.nx + 1, p * mesh.ny + 1
    c, b, a = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    return ((p * ex + a.ravel()) + Nx * ((p * ey + b.ravel()) + Ny * (p * ez + c.ravel()))).astype(np.int64)


def diagonal_elementwise(mesh: HexGridMesh, p: int, q: int, form: str, ess=None) -> np.ndarray:
    """diag(A) = sum_e diag(A_e) scattered, with each diagonal entry computed as the
    quadrature of phi_a^2 (mass) or |J^{-T} grad phi_a|^2 (diffusion) times w detJ.
    Essential rows get 1 (the constrained operator)."""
    R = rule(p, q)
    dofs = elem_dofs(mesh, p)
    X = mesh.element_corners()
    dg = np.zeros(num_dofs(mesh, p))
    for s, e in _chunks(mesh.num_elements, (q ** 3) * 8 * 40 + (q ** 3) * ((p + 1) ** 3) * 8 * 4):
        F = qp_factors(X[s:e], R, form)
        if form == MASS:
            de = F @ (R.Phi ** 2)
        else:
            de = np.einsum("mar,emrs,mas->ea", R.dPhi, F, R.dPhi, optimize=True)
        np.add.at(dg, dofs[s:e].ravel(), de.ravel())
    if ess is not None:
        dg[np.asarray(ess, dtype=np.int64)] = 1.0
    return dg


def qp_coords(mesh: HexGridMesh, p: int, q: int) -> np.ndarray:
    """(E, q^3, 3) physical quadrature point coordinates."""
    x, _ = trilinear(mesh.element_corners(), rule(p, q).xi)
    return x


def rhs_from_qp(mesh: HexGridMesh, p: int, q: int, fq: np.ndarray) -> np.ndarray:
    """b_i = sum_e sum_pt w detJ f(x_pt) phi_i(xi_pt): the load vector for f given at the
    physical quadrature points (E, q^3)."""
    R = rule(p, q)
    F = qp_factors(mesh.element_corners(), R, MASS)
    be = (F * np.asarray(fq).reshape(F.shape)) @ R.Phi
    b = np.zeros(num_dofs(mesh, p))
    np.add.at(b, elem_dofs(mesh, p).ravel(), be.ravel())
    return b


def sine_solution(xyz: np.ndarray) -> np.ndarray:
    return np.sin(np.pi * xyz[..., 0]) * np.sin(np.pi * xyz[..., 1]) * np.sin(np.pi * xyz[..., 2])


def sine_source(form: str, xyz: np.ndarray) -> np.ndarray:
    """f with u = sin(pi x) sin(pi y) sin(pi z): -lap u = 3 pi^2 u (diffusion), u (mass)."""
    u = sine_solution(xyz)
    return 3.0 * np.pi ** 2 * u if form == DIFFUSION else u


# ----------------------------------------------------------------------------
# Solver
# ----------------------------------------------------------------------------

def jacobi_pcg(apply, b: np.ndarray, diag: np.ndarray, rtol: float = 1e-10, maxit: int = 10000, x0=None):
    """Jacobi-preconditioned conjugate gradients (reading R9 for the stopping rule).
    Iteration k: h = A d; alpha = (z,r)/(d,h); x += alpha d; r -= alpha h; stop if
    ||r|| <= rtol ||b||; z = r/diag; beta = (z_new,r_new)/(z,r); d = z + beta d.
    Returns (x, iterations, final ||r||/||b||)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - apply(x) if x0 is not None else b.copy()
    nb = math.sqrt(float(b @ b))
    if nb == 0.0:
        return x, 0, 0.0
    if math.sqrt(float(r @ r)) <= rtol * nb:
        return x, 0, math.sqrt(float(r @ r)) / nb
    z = r / diag
    d = z.copy()
    rho = float(z @ r)
    it = 0
    while it < maxit:
        h = apply(d)
        alpha = rho / float(d @ h)
        x += alpha * d
        r -= alpha * h
        it += 1
        rr = math.sqrt(float(r @ r))
        if rr <= rtol * nb:
            break
        z = r / diag
        rho_new = float(z @ r)
        d = z + (rho_new / rho) * d
        rho = rho_new
    return x, it, math.sqrt(float(r @ r)) / nb


# ----------------------------------------------------------------------------
# Problem setup helpers
# ----------------------------------------------------------------------------

class Problem:
    """A mass or diffusion problem on a HexGridMesh with its CSR matrix (small and
    medium sizes) and the constrained system of reading R8."""

    def __init__(self, mesh: HexGridMesh, p: int, q: int | None, form: str, assemble: bool = True):
        self.mesh, self.p, self.q, self.form = mesh, p, (p + 2 if q is None else q), form
        self.N = num_dofs(mesh, p)
        self.ess = boundary_dofs(mesh, p) if form == DIFFUSION else np.zeros(0, dtype=np.int64)
        self.A = assemble_csr(mesh, p, self.q, form) if assemble else None
        self.Ac = constrain(self.A, self.ess) if assemble else None

    def apply(self, x, constrained=False):
        if self.A is None:
            return action_elementwise(self.mesh, self.p, self.q, self.form, x,
                                      ess=self.ess if constrained else None)
        return (self.Ac if constrained else self.A) @ x

    def diagonal(self, constrained=True):
        if self.A is None:
            return diagonal_elementwise(self.mesh, self.p, self.q, self.form,
                                        ess=self.ess if constrained else None)
        return (self.Ac if constrained else self.A).diagonal()

    def sine_rhs(self):
        """Load vector of the manufactured sine problem, with the homogeneous Dirichlet
        rows (diffusion) set to the boundary value 0."""
        f = sine_source(self.form, qp_coords(self.mesh, self.p, self.q))
        b = rhs_from_qp(self.mesh, self.p, self.q, f)
        b[self.ess] = 0.0
        return b

    def solve(self, b, rtol=1e-10, maxit=10000):
        diag = self.diagonal(constrained=True)
        return jacobi_pcg(lambda v: self.apply(v, constrained=True), b, diag, rtol=rtol, maxit=maxit)


def l2_error(mesh: HexGridMesh, p: int, uh: np.ndarray, exact, q_err: int | None = None) -> float:
    """||u_h - u||_{L2(Omega)} with a separate rule of q_err = p+5 points per direction."""
    qe = p + 5 if q_err is None else q_err
    R = rule(p, qe)
    F = qp_factors(mesh.element_corners(), R, MASS)
    x, _ = trilinear(mesh.element_corners(), R.xi)
    uq = uh[elem_dofs(mesh, p)] @ R.Phi.T
    return math.sqrt(float(np.sum(F * (uq - exact(x)) ** 2)))


# ----------------------------------------------------------------------------
# Brute force (tiny meshes): scalar loops only, no numpy linear algebra, used to
# pin the vectorised assembly above
# ----------------------------------------------------------------------------

def _lagrange_scalar(nodes, j, t):
    v = 1.0
    for m in range(len(nodes)):
        if m != j:
            v *= (t - nodes[m]) / (nodes[j] - nodes[m])
    return v


def _lagrange_deriv_scalar(nodes, j, t):
    s = 0.0
    for l in range(len(nodes)):
        if l == j:
            continue
        term = 1.0 / (nodes[j] - nodes[l])
        for m in range(len(nodes)):
            if m != j and m != l:
                term *= (t - nodes[m]) / (nodes[j] - nodes[m])
        s += term
    return s


def dense_bruteforce(mesh: HexGridMesh, p: int, q: int, form: str) -> np.ndarray:
    """Dense global matrix by explicit scalar loops over elements, quadrature points
    and basis pairs, with the 3x3 inverse written out by cofactors."""
    if mesh.num_elements > 8:
        raise ValueError("brute force is for at most 8 elements")
    n = p + 1
    N = num_dofs(mesh, p)
    A = np.zeros((N, N))
    nodes = [float(v) for v in gll_points(p)]
    pts, wts = gauss_legendre(q)
    dofs = elem_dofs(mesh, p)
    Xall = mesh.element_corners()
    for e in range(mesh.num_elements):
        X = [[float(Xall[e, c, d]) for d in range(3)] for c in range(8)]
        for k in range(q):
            for j in range(q):
                for i in range(q):
                    xi = (float(pts[i]), float(pts[j]), float(pts[k]))
                    w = float(wts[i] * wts[j] * wts[k])
                    J = [[0.0] * 3 for _ in range(3)]
                    for c in range(8):
                        b = [(c >> d) & 1 for d in range(3)]
                        f = [xi[d] if b[d] else 1.0 - xi[d] for d in range(3)]
                        df = [1.0 if b[d] else -1.0 for d in range(3)]
                        g = (df[0] * f[1] * f[2], f[0] * df[1] * f[2], f[0] * f[1] * df[2])
                        for d in range(3):
                            for r in range(3):
                                J[d][r] += X[c][d] * g[r]
                    det = (J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1])
                           - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0])
                           + J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]))
                    # inverse transpose by cofactors: (J^{-T})[d][r] = cof(J)[d][r] / det
                    cof = [[0.0] * 3 for _ in range(3)]
                    for d in range(3):
                        for r in range(3):
                            rows = [x for x in range(3) if x != d]
                            cols = [x for x in range(3) if x != r]
                            minor = (J[rows[0]][cols[0]] * J[rows[1]][cols[1]]
                                     - J[rows[0]][cols[1]] * J[rows[1]][cols[0]])
                            cof[d][r] = (-1.0) ** (d + r) * minor
                    val, grad = [], []
                    for c in range(n):
                        for bb in range(n):
                            for a in range(n):
                                la, lb, lc = (_lagrange_scalar(nodes, a, xi[0]), _lagrange_scalar(nodes, bb, xi[1]),
                                              _lagrange_scalar(nodes, c, xi[2]))
                                da, db, dc = (_lagrange_deriv_scalar(nodes, a, xi[0]),
                                              _lagrange_deriv_scalar(nodes, bb, xi[1]),
                                              _lagrange_deriv_scalar(nodes, c, xi[2]))
                                val.append(la * lb * lc)
                                gr = (da * lb * lc, la * db * lc, la * lb * dc)
                                grad.append([sum(cof[d][r] * gr[r] for r in range(3)) / det for d in range(3)])
                    for s in range(n ** 3):
                        for t in range(n ** 3):
                            if form == MASS:
                                v = val[s] * val[t]
                            else:
                                v = grad[s][0] * grad[t][0] + grad[s][1] * grad[t][1] + grad[s][2] * grad[t][2]
                            A[dofs[e, s], dofs[e, t]] += w * det * v
    return A


# ----------------------------------------------------------------------------
# p-multigrid pieces (Sec. 2.1: order hierarchy on one mesh, transfers between
# orders, diagonal-based smoothing with Chebyshev acceleration)
# ----------------------------------------------------------------------------

def order_prolongation(mesh: HexGridMesh, pc: int, pf: int) -> sp.csr_matrix:
    """P with P[i, j] = phi_j^{pc}(x_i): the coarse (order pc) nodal basis function j
    evaluated at fine (order pf) node i, element by element on the reference element
    (the map is the same for both orders, so this is the natural injection Q_pc into Q_pf)."""
    nf, nc = pf + 1, pc + 1
    Vc, _ = lagrange(gll_points(pc), gll_points(pf))           # (nf, nc) 1D
    I3 = np.zeros((nf ** 3, nc ** 3))
    for c in range(nf):
        for b in range(nf):
            for a in range(nf):
                row = a + nf * (b + nf * c)
                for k in range(nc):
                    for j in range(nc):
                        for i in range(nc):
                            I3[row, i + nc * (j + nc * k)] = Vc[a, i] * Vc[b, j] * Vc[c, k]
    df, dc = elem_dofs(mesh, pf), elem_dofs(mesh, pc)
    P = sp.lil_matrix((num_dofs(mesh, pf), num_dofs(mesh, pc)))
    for e in range(mesh.num_elements):
        for r in range(nf ** 3):
            for s in range(nc ** 3):
                if I3[r, s] != 0.0:
                    P[df[e, r], dc[e, s]] = I3[r, s]     # equal from every element sharing the node
    return P.tocsr()


def chebyshev_smoother(apply, diag: np.ndarray, b: np.ndarray, lmin: float, lmax: float, k: int) -> np.ndarray:
    """k steps of Chebyshev acceleration of Jacobi for A x = b from x0 = 0, for the
    eigenvalues of D^{-1}A assumed in [lmin, lmax] (the classical three-term recurrence:
    theta, delta the centre and half-width of the interval, sigma = theta/delta)."""
    theta, delta = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
    sigma = theta / delta
    rho = 1.0 / sigma
    x = np.zeros_like(b)
    r = b.copy()
    d = r / diag / theta
    for _ in range(k):
        x = x + d
        r = r - apply(d)
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * (r / diag)
        rho = rho_new
    return x


def pmg_vcycle(As, diags, Ps, lmax, degree, coarse_degree, b, smooth=(0.25, 1.1), coarse=(0.003, 1.2), ess=None):
    """One symmetric V-cycle over levels 0 (finest) .. L (coarsest): Chebyshev-Jacobi
    pre-smoothing from 0, residual, restriction by P^T (essential rows of the coarser level
    set to 0), recursion, prolongation by P, residual, post-smoothing, correction; the
    coarsest level applies a higher-degree Chebyshev polynomial.  As[l] are the (constrained)
    level matrices, Ps[l] maps level l+1 to level l, ess[l] the essential rows of level l."""
    def rec(l, rhs):
        A = As[l]
        app = lambda v: A @ v  # noqa: E731
        if l == len(As) - 1:
            return chebyshev_smoother(app, diags[l], rhs, coarse[0] * lmax[l], coarse[1] * lmax[l], coarse_degree)
        x = chebyshev_smoother(app, diags[l], rhs, smooth[0] * lmax[l], smooth[1] * lmax[l], degree)
        r = rhs - A @ x
        rc = Ps[l].T @ (r if ess is None or ess[l] is None else np.where(np.isin(np.arange(len(r)), ess[l]), 0.0, r))
        if ess is not None and ess[l + 1] is not None:
            rc[ess[l + 1]] = 0.0
        x = x + Ps[l] @ rec(l + 1, rc)
        r = rhs - A @ x
        return x + chebyshev_smoother(app, diags[l], r, smooth[0] * lmax[l], smooth[1] * lmax[l], degree)
    return rec(0, np.asarray(b, dtype=np.float64))
