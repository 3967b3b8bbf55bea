"""Meshes given by element connectivity, on the CPU: the oracle's numbering of such a mesh
(built from each node's trilinear weights on the global vertices) is pinned against the
structured grid it may come from and against invariants on a genuinely unstructured mesh,
and the library's host numbering (fepa_hex_numbering, no GPU needed) is checked to identify
exactly the same shared nodes as the oracle's, on scrambled and unstructured meshes."""
import numpy as np
import pytest

import fem_inputs as FI
import oracle as O


def structured(shape, seed):
    return O.HexGridMesh(*shape, FI.perturbed_cube_vertices(*shape, seed=seed))


def perm_from_maps(d_from, d_to, N):
    """pi with pi[d_from[e, l]] = d_to[e, l] for every slot; asserts it is a bijection."""
    pi = np.full(N, -1, dtype=np.int64)
    a, b = d_from.ravel(), d_to.ravel()
    pi[a] = b
    assert (pi >= 0).all()
    assert np.array_equal(pi[a], b), "one node maps to two"
    assert len(np.unique(pi)) == N, "two nodes map to one"
    return pi


def perm_from_coords(x_from, x_to):
    """pi with x_to[pi[i]] = x_from[i] (distinct points, matched to 1e-9)."""
    key = lambda X: np.round(X * 1e9).astype(np.int64)  # noqa: E731
    kf, kt = key(x_from), key(x_to)
    order_t = np.lexsort(kt.T[::-1])
    order_f = np.lexsort(kf.T[::-1])
    assert np.array_equal(kf[order_f], kt[order_t])
    pi = np.empty(len(x_from), dtype=np.int64)
    pi[order_f] = order_t
    return pi


@pytest.mark.parametrize("form", [O.MASS, O.DIFFUSION])
@pytest.mark.parametrize("p", [1, 2, 3])
def test_grid_as_connectivity_is_the_same_operator(p, form):
    shape = (3, 2, 2)
    g = structured(shape, seed=5)
    h = O.HexMesh(g.vertices, FI.grid_connectivity(*shape))
    N = O.num_dofs(g, p)
    assert O.num_dofs(h, p) == N
    pi = perm_from_maps(O.elem_dofs(g, p), O.elem_dofs(h, p), N)
    Ag = O.assemble_csr(g, p, p + 2, form).toarray()
    Ah = O.assemble_csr(h, p, p + 2, form).toarray()
    np.testing.assert_allclose(Ah[np.ix_(pi, pi)], Ag, atol=1e-15 * np.abs(Ag).max())
    np.testing.assert_array_equal(np.sort(pi[O.boundary_dofs(g, p)]), O.boundary_dofs(h, p))


@pytest.mark.parametrize("form", [O.MASS, O.DIFFUSION])
@pytest.mark.parametrize("p", [1, 2, 4])
def test_scrambled_mesh_is_the_same_operator(p, form):
    # vertex ids permuted, elements reordered, every element's corners listed in a rotated
    # order: the same discrete operator up to the renumbering of the nodes
    shape, seed = (3, 2, 2), 8
    g = structured(shape, seed)
    h = O.HexMesh(*FI.scrambled_hex_mesh(*shape, seed=seed))
    pi = perm_from_coords(O.node_coords(g, p), O.node_coords(h, p))
    Ag = O.assemble_csr(g, p, p + 2, form).toarray()
    Ah = O.assemble_csr(h, p, p + 2, form).toarray()
    np.testing.assert_allclose(Ah[np.ix_(pi, pi)], Ag, atol=1e-13 * np.abs(Ag).max())
    np.testing.assert_array_equal(np.sort(pi[O.boundary_dofs(g, p)]), O.boundary_dofs(h, p))


@pytest.mark.parametrize("p", [1, 2, 3])
def test_unstructured_mesh_invariants(p):
    # tiles of five quadrilaterals, extruded: edges held by 3 elements (never in a grid)
    h = O.HexMesh(*FI.tiled_unstructured_cube(2, 2, seed=3))
    N = O.num_dofs(h, p)
    M = O.assemble_csr(h, p, p + 2, O.MASS)
    K = O.assemble_csr(h, p, p + 2, O.DIFFUSION)
    one = np.ones(N)
    assert abs(one @ M @ one - 1.0) < 1e-13                 # |unit cube|
    assert np.abs(K @ one).max() < 1e-12 * abs(K).max()     # constants in the kernel
    assert abs(K - K.T).max() < 1e-14 * abs(K).max()
    xyz = O.node_coords(h, p)
    bd = O.boundary_dofs(h, p)
    on = np.nonzero(np.any((np.abs(xyz) < 1e-12) | (np.abs(xyz - 1.0) < 1e-12), axis=1))[0]
    np.testing.assert_array_equal(bd, on)                   # boundary = nodes on the cube's faces
    interior = np.setdiff1d(np.arange(N), bd)
    u = 0.3 + 1.1 * xyz[:, 0] - 0.7 * xyz[:, 1] + 2.3 * xyz[:, 2]
    assert np.abs((K @ u)[interior]).max() < 1e-12 * np.abs(K).max()   # linear patch test
    # the mass projection reproduces polynomials of total degree <= p (in the space on trilinear maps)
    f = lambda X: (0.2 + X[..., 0] - 0.5 * X[..., 1] + 0.7 * X[..., 2]) ** p  # noqa: E731
    b = O.rhs_from_qp(h, p, p + 2, f(O.qp_coords(h, p, p + 2)))
    import scipy.sparse.linalg as spla
    c = spla.spsolve(M.tocsc(), b)
    np.testing.assert_allclose(c, f(xyz), atol=1e-11)


@pytest.mark.parametrize("form", [O.MASS, O.DIFFUSION])
def test_unstructured_bruteforce(form):
    h = O.HexMesh(*FI.tiled_unstructured_cube(1, 1, seed=4))   # 5 elements
    A = O.assemble_csr(h, 2, 4, form).toarray()
    np.testing.assert_allclose(O.dense_bruteforce(h, 2, 4, form), A, atol=1e-13 * np.abs(A).max())


# ---------------------------------------------------------------- the library's host numbering

@pytest.fixture(scope="module")
def F():
    from paper_2402_15940_b300 import build
    build.build()
    import paper_2402_15940_b300 as mod
    mod.load_library()
    return mod


MESHES = {
    "scrambled": lambda: FI.scrambled_hex_mesh(3, 2, 2, seed=9),
    "unstructured": lambda: FI.tiled_unstructured_cube(2, 2, seed=10),
    "grid": lambda: (FI.perturbed_cube_vertices(2, 3, 2, seed=11), FI.grid_connectivity(2, 3, 2)),
}


@pytest.mark.parametrize("name", sorted(MESHES))
@pytest.mark.parametrize("p", [1, 2, 3, 4, 6, 8])
def test_library_numbering_identifies_the_same_nodes(F, name, p):
    verts, conn = MESHES[name]()
    lib_dofs, N = F.hex_numbering(len(verts), conn, p)
    ora_dofs, No, _ = O.hex_numbering(O.HexMesh(verts, conn), p)
    assert N == No
    perm_from_maps(lib_dofs.astype(np.int64), ora_dofs, N)


def test_library_numbering_rejects_invalid_meshes(F):
    from paper_2402_15940_b300 import fepa
    verts, conn = FI.scrambled_hex_mesh(2, 2, 1, seed=12)
    def code(c, p=2, nv=len(verts)):
        with pytest.raises(fepa.FepaError) as ei:
            F.hex_numbering(nv, c, p)
        return ei.value.code
    bad = conn.copy(); bad[1, 3] = len(verts)               # vertex id out of range
    assert code(bad) == fepa.ERR_MESH
    bad = conn.copy(); bad[2, 5] = bad[2, 0]                # repeated vertex
    assert code(bad) == fepa.ERR_MESH
    assert code(np.concatenate([conn, conn[:1]])) == fepa.ERR_MESH   # a face held by three elements
    bad = conn.copy(); bad[0, [2, 3]] = bad[0, [3, 2]]      # a face's quadrilateral twisted
    assert code(bad) == fepa.ERR_MESH
    assert code(conn, p=9) == fepa.ERR_UNSUPPORTED
