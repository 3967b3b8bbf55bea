"""GPU parity on meshes given by element connectivity (fepa_op_create_hex): the same kernels
reach every element's DOFs through the map G built from the connectivity.  Compared with the
oracle on scrambled grids (vertex ids permuted, elements reordered, each element's corners
listed in a rotated order) and on an unstructured mesh (tiles of five quadrilaterals,
extruded, with edges held by three elements), for p = 1..8 and both forms: the FP64 action
to 1e-12 and the FP32 action to 1e-5 (the tolerances of the structured tests), the diagonal,
the load vector, the quadrature-point coordinates, the boundary, and CG, mixed-precision and
p-multigrid solves.  The library and the oracle number the DOFs independently; the vectors
are compared through the permutation their element maps define, which must be a bijection.
At the benchmark's size the connectivity op of the grid equals the structured op."""
import math

import numpy as np
import pytest

import fem_inputs as FI
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-12, 1e-5


def F():
    import paper_2402_15940_b300 as mod
    return mod


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def perm(d_lib, d_ora, N):
    """pi[ora dof] = lib dof, checked to be a bijection."""
    pi = np.full(N, -1, dtype=np.int64)
    pi[d_ora.ravel()] = d_lib.ravel()
    assert (pi >= 0).all() and np.array_equal(pi[d_ora.ravel()], d_lib.ravel())
    assert len(np.unique(pi)) == N
    return pi


SCR_SHAPES = {1: (4, 3, 3), 2: (3, 3, 2), 3: (3, 2, 2), 4: (2, 2, 2), 5: (2, 2, 1), 6: (2, 1, 1), 7: (2, 1, 1),
              8: (1, 1, 2)}


def mesh_for(kind, p, seed):
    if kind == "scrambled":
        return FI.scrambled_hex_mesh(*SCR_SHAPES[p], seed=seed)
    return FI.tiled_unstructured_cube(1 if p >= 5 else 2, 1 if p >= 4 else 2, seed=seed)


def setup(kind, p, form, seed):
    verts, conn = mesh_for(kind, p, seed)
    op = F().Operator.from_hex(verts, conn, p, form=form)
    mesh = O.HexMesh(verts, conn)
    dl = op.elem_dofs().cpu().numpy().astype(np.int64)
    do, N, bd = O.hex_numbering(mesh, p)
    assert op.N == N
    return op, mesh, perm(dl, do, N), bd


@pytest.mark.parametrize("form", ["mass", "diffusion"])
@pytest.mark.parametrize("p", list(range(1, 9)))
@pytest.mark.parametrize("kind", ["scrambled", "unstructured"])
def test_hex_actions_diag_rhs_match_oracle(kind, p, form):
    op, mesh, pi, bd = setup(kind, p, form, seed=20 + p)
    prob = O.Problem(mesh, p, None, form, assemble=p <= 5)
    # boundary: the same node set
    np.testing.assert_array_equal(np.sort(op.boundary_dofs()), np.sort(pi[bd]))
    x = FI.uniform_vector(op.N, seed=p)
    xl = np.empty_like(x)
    xl[pi] = x                                   # library numbering of the same vector
    y = op.apply(torch.from_numpy(xl).cuda()).cpu().numpy()[pi]
    assert rel(y, prob.apply(x)) <= TOL64
    y32 = op.apply_f32(torch.from_numpy(xl.astype(np.float32)).cuda()).cpu().numpy()[pi]
    assert rel(y32, prob.apply(x.astype(np.float32).astype(np.float64))) <= TOL32
    qx = op.qp_coords().cpu().numpy()
    np.testing.assert_allclose(qx, O.qp_coords(mesh, p, p + 2), atol=1e-14)
    fq = O.sine_source(form, O.qp_coords(mesh, p, p + 2))
    b = op.rhs(torch.from_numpy(np.ascontiguousarray(fq)).cuda()).cpu().numpy()[pi]
    assert rel(b, O.rhs_from_qp(mesh, p, p + 2, fq)) <= TOL64
    if form == "diffusion":
        op.set_essential(op.boundary_dofs())
        y = op.apply(torch.from_numpy(xl).cuda()).cpu().numpy()[pi]
        assert rel(y, prob.apply(x, constrained=True)) <= TOL64
    dg = op.diagonal().cpu().numpy()[pi]
    assert rel(dg, prob.diagonal(constrained=form == "diffusion")) <= TOL64


@pytest.mark.parametrize("kind", ["scrambled", "unstructured"])
@pytest.mark.parametrize("p", [2, 3])
def test_hex_solves_match_oracle(kind, p):
    op, mesh, pi, bd = setup(kind, p, "diffusion", seed=40 + p)
    op.set_essential(op.boundary_dofs())
    prob = O.Problem(mesh, p, None, O.DIFFUSION)
    b = op.rhs_sine(3 * math.pi ** 2)
    bo = prob.sine_rhs()
    assert rel(b.cpu().numpy()[pi], bo) <= TOL64
    xo, it_o, _ = prob.solve(bo, rtol=1e-10)
    x, st = op.solve(b, rtol=1e-10)
    assert abs(st["iterations"] - it_o) <= 1
    assert rel(x.cpu().numpy()[pi], xo) <= 1e-9
    xt, _, _ = prob.solve(bo, rtol=1e-14)
    xr, sr = op.solve_refined(b, rtol=1e-12)
    assert sr["status"] == 0 and rel(xr.cpu().numpy()[pi], xt) <= 1e-10
    mg = F().Multigrid(op, precision="fp32")
    xm, sm = mg.solve(b, rtol=1e-12, maxit=200)
    assert sm["status"] == 0 and rel(xm.cpu().numpy()[pi], xt) <= 1e-10


def test_hex_mass_solve_and_moved_vertices():
    verts, conn = FI.tiled_unstructured_cube(2, 2, seed=50)
    op = F().Operator.from_hex(verts, conn, 3, form="mass")
    v2 = verts.copy()
    interior = np.all((verts > 1e-12) & (verts < 1 - 1e-12), axis=1)
    v2[interior] += 0.01 * np.sin(7.0 * verts[interior])        # move the interior vertices
    op.set_vertices(v2)
    mesh = O.HexMesh(v2, conn)
    dl = op.elem_dofs().cpu().numpy().astype(np.int64)
    do, N, _ = O.hex_numbering(mesh, 3)
    pi = perm(dl, do, N)
    prob = O.Problem(mesh, 3, None, O.MASS)
    x = FI.uniform_vector(N, seed=51)
    xl = np.empty_like(x)
    xl[pi] = x
    assert rel(op.apply(torch.from_numpy(xl).cuda()).cpu().numpy()[pi], prob.apply(x)) <= TOL64
    b = op.rhs_sine(1.0)
    xs, st = op.solve(b, rtol=1e-10)
    xo, it_o, _ = prob.solve(prob.sine_rhs(), rtol=1e-10)
    assert abs(st["iterations"] - it_o) <= 1 and rel(xs.cpu().numpy()[pi], xo) <= 1e-9


def test_hex_rejects_inverted_and_invalid():
    from paper_2402_15940_b300 import fepa
    verts, conn = FI.scrambled_hex_mesh(2, 2, 2, seed=60)
    bad = conn.copy()
    bad[3] = bad[3][[1, 0, 3, 2, 5, 4, 7, 6]]    # mirrored corner order: det J < 0
    with pytest.raises(fepa.FepaError) as ei:
        F().Operator.from_hex(verts, bad, 2)
    assert ei.value.code == fepa.ERR_MESH
    bad = conn.copy()
    bad[0, 0] = -1
    with pytest.raises(fepa.FepaError) as ei:
        F().Operator.from_hex(verts, bad, 2)
    assert ei.value.code == fepa.ERR_MESH


@pytest.mark.parametrize("form", ["diffusion", "mass"])
def test_hex_grid_equals_structured_at_benchmark_size(form):
    """The benchmark's mesh (p = 4, 64^3 elements, 257^3 DOFs) passed as connectivity: the
    element maps give the permutation between the two numberings (same element order and
    frames), and both FP64 and FP32 actions and the diagonal agree through it."""
    n, p = 64, 4
    verts = FI.perturbed_cube_vertices(n, n, n, seed=0)
    st = F().Operator(n, n, n, verts, p, form=form)
    hx = F().Operator.from_hex(verts, FI.grid_connectivity(n, n, n), p, form=form)
    ds, dh = st.elem_dofs().long().flatten(), hx.elem_dofs().long().flatten()
    pi = torch.full((st.N,), -1, dtype=torch.long, device="cuda")
    pi[ds] = dh                                   # structured dof -> connectivity dof
    assert bool((pi >= 0).all()) and bool((pi[ds] == dh).all())
    if form == "diffusion":
        st.set_essential(st.boundary_dofs())
        hx.set_essential(hx.boundary_dofs())
        bs = torch.from_numpy(st.boundary_dofs().astype(np.int64)).cuda()
        bh = torch.from_numpy(np.sort(hx.boundary_dofs()).astype(np.int64)).cuda()
        assert torch.equal(torch.sort(pi[bs]).values, bh)
    x = torch.from_numpy(FI.uniform_vector(st.N, seed=3)).cuda()
    xh = torch.empty_like(x)
    xh[pi] = x
    ys, yh = st.apply(x), hx.apply(xh)[pi]
    assert float(torch.linalg.norm(yh - ys) / torch.linalg.norm(ys)) <= 1e-14
    y32s, y32h = st.apply_f32(x.float()), hx.apply_f32(xh.float())[pi]
    assert float(torch.linalg.norm((y32h - y32s).double()) / torch.linalg.norm(y32s.double())) <= 1e-6
    d_s, d_h = st.diagonal(), hx.diagonal()[pi]
    assert float(torch.linalg.norm(d_h - d_s) / torch.linalg.norm(d_s)) <= 1e-14


@pytest.mark.parametrize("p", [2, 4, 7])
def test_hex_every_action_variant_matches_oracle(p):
    """Every compiled FP64 action (DFMA, double-float in full- and half-size blocks) and every
    FP32 launch shape on the unstructured mesh, diffusion with the boundary fixed."""
    op, mesh, pi, bd = setup("unstructured", p, "diffusion", seed=60 + p)
    op.set_essential(op.boundary_dofs())
    prob = O.Problem(mesh, p, None, O.DIFFUSION, assemble=p <= 5)
    x = FI.uniform_vector(op.N, seed=61)
    xl = np.empty_like(x)
    xl[pi] = x
    ref = prob.apply(x, constrained=True)
    for v in (0, 1, 2):
        op.set_f64_variant(v)
        y = op.apply(torch.from_numpy(xl).cuda()).cpu().numpy()[pi]
        assert rel(y, ref) <= TOL64, v
    ref32 = prob.apply(x.astype(np.float32).astype(np.float64), constrained=True)
    for v in range(4):
        op.set_f32_variant(v)
        y32 = op.apply_f32(torch.from_numpy(xl.astype(np.float32)).cuda()).cpu().numpy()[pi]
        assert rel(y32, ref32) <= TOL32, v


def test_hex_resumable_multigrid_solve_matches_oracle():
    """The resumable multigrid-preconditioned CG on the unstructured mesh: the blocking solve's
    iterations and solution, and the oracle's tightly solved solution."""
    op, mesh, pi, bd = setup("unstructured", 4, "diffusion", seed=64)
    op.set_essential(op.boundary_dofs())
    b = op.rhs_sine(3 * math.pi ** 2)
    mg = F().Multigrid(op, precision="fp64")
    x1, s1 = mg.solve(b, rtol=1e-11)
    x2 = torch.zeros_like(b)
    mg.solver_start(b, x2, rtol=1e-11)
    st = mg.solver_poll(blocking=True)
    while not st["done"]:
        mg.solver_advance(3)
        st = mg.solver_poll(blocking=True)
    assert st["status"] == 0 and st["iterations"] == s1["iterations"]
    assert rel(x2.cpu().numpy(), x1.cpu().numpy()) <= 1e-12
    prob = O.Problem(mesh, 4, None, O.DIFFUSION)
    xt, _, _ = prob.solve(prob.sine_rhs(), rtol=1e-14)
    assert rel(x2.cpu().numpy()[pi], xt) <= 1e-9
    mg.close()
