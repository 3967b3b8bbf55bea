"""GPU parity of the double-float FP64 action (variant 1: every value split into two
floats, contractions by exact FMA products and TwoSum accumulation on the FP32 pipe)
against the oracle, at the FP64 action's tolerance (relative l2 <= 1e-12), and against
the DFMA kernel; CG and multigrid solves on it; the full-size sampled rows."""
import math

import numpy as np
import pytest

import fem_inputs as FI
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12
# elements per block is 256 // (q*q): several blocks and a ragged tail for each p
SHAPES = {1: (5, 4, 3), 2: (4, 3, 3), 3: (3, 3, 3), 4: (3, 3, 2), 5: (3, 2, 2), 6: (3, 2, 1), 7: (2, 2, 2),
          8: (3, 1, 1)}


def F():
    import paper_2402_15940_b300 as mod
    return mod


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def make(shape, p, form, seed=0, q=None, variant=1):
    verts = FI.perturbed_cube_vertices(*shape, seed=seed)
    op = F().Operator(*shape, verts, p, form=form, q=0 if q is None else q)
    op.set_f64_variant(variant)
    return op, O.HexGridMesh(*shape, verts)


def oracle_action(mesh, p, q, form, x, ess=None):
    if p <= 5:
        A = O.assemble_csr(mesh, p, q, form)
        if ess is not None:
            A = O.constrain(A, ess)
        return A @ x
    return O.action_elementwise(mesh, p, q, form, x, ess=ess)


@pytest.mark.parametrize("form", ["mass", "diffusion"])
@pytest.mark.parametrize("p", list(range(1, 9)))
def test_df_apply_matches_oracle(p, form):
    op, mesh = make(SHAPES[p], p, form, seed=p)
    assert op.f64_variant()[0] == 1
    x = FI.uniform_vector(op.N, seed=100 + p)
    y = host(op.apply(dev(x)))
    ref = oracle_action(mesh, p, p + 2, form, x)
    assert rel(y, ref) <= TOL
    assert np.max(np.abs(y - ref)) <= 10 * TOL * np.max(np.abs(ref))


@pytest.mark.parametrize("form", ["mass", "diffusion"])
@pytest.mark.parametrize("p", [1, 3, 5, 8])
def test_df_apply_q_equals_p_plus_1(p, form):
    op, mesh = make(SHAPES[p], p, form, seed=p, q=p + 1)
    x = FI.uniform_vector(op.N, seed=7)
    assert rel(host(op.apply(dev(x))), oracle_action(mesh, p, p + 1, form, x)) <= TOL


@pytest.mark.parametrize("form", ["mass", "diffusion"])
@pytest.mark.parametrize("p", [2, 4, 7])
def test_df_apply_constrained_matches_oracle(p, form):
    op, mesh = make(SHAPES[p], p, form, seed=11)
    ess = op.boundary_dofs()
    op.set_essential(ess)
    x = FI.uniform_vector(op.N, seed=12)
    y = host(op.apply(dev(x)))
    assert rel(y, oracle_action(mesh, p, p + 2, form, x, ess=ess.astype(np.int64))) <= TOL
    # essential rows return x exactly (the owner occurrence adds x in FP64)
    assert np.array_equal(y[ess], x[ess])


@pytest.mark.parametrize("form", ["mass", "diffusion"])
@pytest.mark.parametrize("p", [2, 4, 6])
def test_df_agrees_with_dfma_kernel(p, form):
    shape = (5, 4, 4)
    op64, _ = make(shape, p, form, seed=5, variant=0)
    opdf, _ = make(shape, p, form, seed=5, variant=1)
    x = dev(FI.uniform_vector(op64.N, seed=6))
    y64, ydf = host(op64.apply(x)), host(opdf.apply(x))
    e = rel(ydf, y64)
    assert e <= TOL
    # far from FP32 (~1e-7): the low words carry the extra 24 bits
    assert e <= 1e-13


@pytest.mark.parametrize("form", ["mass", "diffusion"])
@pytest.mark.parametrize("p", list(range(1, 9)))
def test_df_half_block_matches_oracle_and_full_block(p, form):
    """Variant 2 (the double-float kernel in blocks of half as many elements; the meshes of
    SHAPES leave a ragged last block in both shapes) against the oracle, and against variant 1:
    the same per-element arithmetic, only the order of the FP64 atomic additions differs."""
    op, mesh = make(SHAPES[p], p, form, seed=p, variant=2)
    assert op.f64_variant()[0] == 2
    x = FI.uniform_vector(op.N, seed=300 + p)
    y2 = host(op.apply(dev(x)))
    assert rel(y2, oracle_action(mesh, p, p + 2, form, x)) <= TOL
    op.set_f64_variant(1)
    y1 = host(op.apply(dev(x)))
    assert rel(y2, y1) <= 1e-15


def test_df_half_block_cg_solve_matches_oracle():
    op, mesh = make((6, 5, 4), 2, "diffusion", seed=23, variant=2)
    prob = O.Problem(mesh, 2, None, "diffusion")
    op.set_essential(prob.ess.astype(np.int32))
    b = FI.uniform_vector(op.N, seed=24)
    b[prob.ess] = 0.0
    x, st = op.solve(dev(b), rtol=1e-10, maxit=5000)
    xo, it_o, _ = prob.solve(b, rtol=1e-10)
    assert abs(st["iterations"] - it_o) <= 1
    assert rel(host(x), xo) <= 1e-8


def test_df_scale_and_linearity():
    """A(a x + b z) = a A x + b A z to double-float accuracy, and A(2^k x) = 2^k A x
    for moderate k (scaling by a power of two is exact in both words; only the order
    of the FP64 atomic sums differs between launches)."""
    op, _ = make((4, 3, 3), 3, "diffusion", seed=8)
    x = FI.uniform_vector(op.N, seed=1)
    z = FI.uniform_vector(op.N, seed=2)
    Ax, Az = host(op.apply(dev(x))), host(op.apply(dev(z)))
    lin = host(op.apply(dev(0.75 * x - 1.5 * z)))
    assert rel(lin, 0.75 * Ax - 1.5 * Az) <= 1e-13
    for k in (-20, 17):
        assert rel(host(op.apply(dev(np.ldexp(x, k)))), np.ldexp(Ax, k)) <= 1e-15


@pytest.mark.parametrize("form,p,shape", [("mass", 3, (3, 3, 2)), ("diffusion", 5, (2, 3, 2)),
                                          ("diffusion", 8, (2, 1, 2)), ("diffusion", 2, (6, 5, 4))])
def test_df_cg_solve_matches_oracle(form, p, shape):
    op, mesh = make(shape, p, form, seed=23)
    prob = O.Problem(mesh, p, None, form, assemble=p <= 5)
    if form == "diffusion":
        op.set_essential(prob.ess.astype(np.int32))
    b = FI.uniform_vector(op.N, seed=24)
    b[prob.ess] = 0.0
    x, st = op.solve(dev(b), rtol=1e-10, maxit=5000)
    xo, it_o, _ = prob.solve(b, rtol=1e-10)
    assert abs(st["iterations"] - it_o) <= 1
    assert rel(host(x), xo) <= 1e-8


def test_variant_switch_rebuilds_graph_and_autotune_picks_one():
    op, _ = make((4, 4, 4), 4, "diffusion", seed=3, variant=0)
    op.set_essential(op.boundary_dofs())
    b = op.rhs_sine(3 * math.pi ** 2)
    x0, s0 = op.solve(b, rtol=1e-10)
    op.set_f64_variant(1)
    x1, s1 = op.solve(b, rtol=1e-10)
    assert op.f64_variant()[0] == 1
    assert abs(s0["iterations"] - s1["iterations"]) <= 1
    assert rel(host(x1), host(x0)) <= 1e-9
    op.set_f64_variant(-1)
    x2, s2 = op.solve(b, rtol=1e-10)
    assert op.f64_variant()[0] in (0, 1, 2)
    assert rel(host(x2), host(x0)) <= 1e-9


def test_df_multigrid_solve():
    shape, p = (4, 4, 4), 4
    op, mesh = make(shape, p, "diffusion", seed=5)
    op.set_essential(op.boundary_dofs())
    mg = F().Multigrid(op, precision="fp32")
    b = op.rhs_sine(3 * math.pi ** 2)
    x, st = mg.solve(b, rtol=1e-10)
    prob = O.Problem(mesh, p, None, "diffusion")
    xo, _, _ = prob.solve(host(b), rtol=1e-13)
    assert st["status"] == 0 and st["rel_residual"] <= 1e-10
    assert rel(host(x), xo) <= 1e-9


def test_df_full_size_bp3_p4_sampled():
    """Diffusion, p=4 on 64^3 perturbed hexes (257^3 DOFs): sampled rows of the
    constrained double-float action against the oracle, one by one."""
    shape, p = (64, 64, 64), 4
    op, mesh = make(shape, p, "diffusion", seed=0)
    ess = op.boundary_dofs()
    op.set_essential(ess)
    x = FI.uniform_vector(op.N, seed=0)
    y = host(op.apply(dev(x)))
    rng = np.random.default_rng(42)
    rows = np.concatenate([rng.choice(op.N, 48, replace=False), ess[rng.choice(len(ess), 8, replace=False)],
                           [0, op.N - 1, op.N // 2]])
    ref = O.action_rows(mesh, p, p + 2, O.DIFFUSION, x, rows, ess=ess.astype(np.int64))
    assert np.max(np.abs(y[rows] - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("form", ["mass", "diffusion"])
@pytest.mark.parametrize("p", [1, 2, 3, 5, 8])
def test_diagonal_both_kernels_match_oracle(p, form, variant):
    """diag(A) by the FP64 kernel (variant 0) and by the double-float kernel (variant 1)."""
    op, mesh = make(SHAPES[p], p, form, seed=13, variant=variant)
    d = host(op.diagonal())
    ref = O.diagonal_elementwise(mesh, p, p + 2, form)
    assert rel(d, ref) <= TOL and np.max(np.abs(d - ref)) <= 10 * TOL * np.max(np.abs(ref))
    ess = op.boundary_dofs()
    op.set_essential(ess)
    d = host(op.diagonal())
    assert rel(d, O.diagonal_elementwise(mesh, p, p + 2, form, ess=ess.astype(np.int64))) <= TOL
    assert np.all(d[ess] == 1.0)


@pytest.mark.parametrize("form", ["mass", "diffusion"])
@pytest.mark.parametrize("p,q", [(1, 2), (2, 3), (3, 5), (4, 6), (6, 7), (8, 10)])
def test_geometry_matches_oracle_every_q(p, q, form):
    """D from the double-float geometry kernel for every compiled quadrature size."""
    shape = SHAPES[p]
    verts = FI.perturbed_cube_vertices(*shape, seed=p + q)
    op = F().Operator(*shape, verts, p, form=form, q=q)
    mesh = O.HexGridMesh(*shape, verts)
    qd = host(op.qdata())
    Fq = O.qp_factors(mesh.element_corners(), O.rule(p, q), form)
    if form == "mass":
        assert rel(qd[:, 0, :], Fq) <= TOL
    else:
        comps = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
        assert rel(qd, np.stack([Fq[:, :, r, s] for r, s in comps], axis=1)) <= TOL


@pytest.mark.parametrize("p", [1, 2, 3, 4, 6, 8])
def test_load_vector_matches_oracle(p):
    """b = G^T B^T (w det J f), double-float kernel: f given per point, and the sine
    manufactured source (the sine evaluated in double-float: reduction to |r| <= 1/4,
    Taylor series of sin and cos)."""
    shape = SHAPES[p]
    op, mesh = make(shape, p, "diffusion", seed=17)
    f = FI.uniform_vector(op.E * op.q ** 3, seed=18)
    ref = O.rhs_from_qp(mesh, p, p + 2, f.reshape(op.E, -1))
    assert rel(host(op.rhs(dev(f))), ref) <= TOL
    prob = O.Problem(mesh, p, None, O.DIFFUSION, assemble=False)
    op.set_essential(op.boundary_dofs())
    for scale in (3 * math.pi ** 2, -0.5):
        got = host(op.rhs_sine(scale))
        ref = prob.sine_rhs() * scale / (3 * math.pi ** 2)
        assert rel(got, ref) <= TOL
        assert np.max(np.abs(got - ref)) <= 10 * TOL * np.max(np.abs(ref))


def test_load_vector_on_a_shifted_mesh():
    """Coordinates outside [0, 1] (several periods of the sine, negative values): the
    reduction x = k/2 + r covers every quadrant."""
    shape, p = (3, 3, 2), 3
    verts = FI.perturbed_cube_vertices(*shape, seed=4) * 3.0 - 1.3
    op = F().Operator(*shape, verts, p, form="mass")
    mesh = O.HexGridMesh(*shape, verts)
    prob = O.Problem(mesh, p, None, O.MASS, assemble=False)
    assert rel(host(op.rhs_sine(1.0)), prob.sine_rhs()) <= TOL   # mass: f = u, scale 1
