"""GPU parity: the CUDA path (through the C ABI) against the CPU FP64 oracle.

Tolerance: relative l2 error <= 1e-12 for the FP64 operator action, the stored
quadrature data, the diagonal and the load vector (the two sides sum the same terms
in different orders, so only rounding differs); bit-exact for the element->DOF map.
Mesh shapes are chosen so that every kernel covers several thread blocks and a
ragged last block (E not a multiple of the elements per block).
"""
import math

import numpy as np
import pytest

import fem_inputs as FI
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12

# elements per block of the apply kernel is 256 // (q*q); shapes give a ragged tail
SHAPES = {1: (5, 4, 3), 2: (4, 3, 3), 3: (3, 3, 3), 4: (3, 3, 2), 5: (3, 2, 2), 6: (3, 2, 1), 7: (2, 2, 2),
          8: (3, 1, 1)}


def fepa():
    import paper_2402_15940_b300 as F
    return F


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def assert_close(a, b, tol=TOL):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    assert rel_err(a, b) <= tol, rel_err(a, b)
    assert np.max(np.abs(a - b)) <= 10 * tol * max(np.max(np.abs(b)), 1e-300)


def make(shape, p, form, seed=0, q=None):
    verts = FI.perturbed_cube_vertices(*shape, seed=seed)
    op = fepa().Operator(*shape, verts, p, form=form, q=0 if q is None else q)
    mesh = O.HexGridMesh(*shape, verts)
    return op, mesh


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def oracle_action(mesh, p, q, form, x, ess=None):
    if p <= 5:
        A = O.assemble_csr(mesh, p, q, form)
        if ess is not None:
            A = O.constrain(A, ess)
        return A @ x
    return O.action_elementwise(mesh, p, q, form, x, ess=ess)


# ---------------------------------------------------------------- a1, a3: D and G

@pytest.mark.parametrize("form", ["mass", "diffusion"])
@pytest.mark.parametrize("p", [1, 2, 4, 8])
def test_qdata_matches_oracle(p, form):
    shape = SHAPES[p]
    op, mesh = make(shape, p, form, seed=3)
    qd = host(op.qdata())
    R = O.rule(p, p + 2)
    F = O.qp_factors(mesh.element_corners(), R, form)
    if form == "mass":
        assert_close(qd[:, 0, :], F)
    else:
        # compared as one tensor: on meshes one element thick some off-diagonal components
        # vanish exactly and only rounding noise remains in them
        comps = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
        ref = np.stack([F[:, :, r, s] for r, s in comps], axis=1)
        assert_close(qd, ref)


@pytest.mark.parametrize("p", [1, 3, 6, 8])
def test_elem_dofs_bit_exact(p):
    op, mesh = make(SHAPES[p], p, "mass")
    g = host(op.elem_dofs())
    assert np.array_equal(g.astype(np.int64), O.elem_dofs(mesh, p))
    # still unflagged after essential DOFs are set
    op.set_essential(op.boundary_dofs())
    assert np.array_equal(host(op.elem_dofs()).astype(np.int64), O.elem_dofs(mesh, p))


def test_boundary_dofs_match_oracle():
    for p in (1, 2, 5):
        op, mesh = make((3, 2, 4), p, "diffusion")
        assert np.array_equal(op.boundary_dofs().astype(np.int64), O.boundary_dofs(mesh, p))


@pytest.mark.parametrize("p", [1, 4, 7])
def test_qp_coords_match_oracle(p):
    op, mesh = make(SHAPES[p], p, "mass", seed=5)
    assert_close(host(op.qp_coords()), O.qp_coords(mesh, p, p + 2))


# ---------------------------------------------------------------- a2-a7: the fused action

@pytest.mark.parametrize("form", ["mass", "diffusion"])
@pytest.mark.parametrize("p", list(range(1, 9)))
def test_apply_matches_oracle(p, form):
    shape = SHAPES[p]
    op, mesh = make(shape, p, form, seed=p)
    x = FI.uniform_vector(op.N, seed=100 + p)
    y = host(op.apply(dev(x)))
    assert_close(y, oracle_action(mesh, p, p + 2, form, x))


@pytest.mark.parametrize("form", ["mass", "diffusion"])
@pytest.mark.parametrize("p", [1, 2, 3, 5, 8])
def test_apply_q_equals_p_plus_1(p, form):
    shape = SHAPES[p]
    op, mesh = make(shape, p, form, seed=p, q=p + 1)
    assert op.q == p + 1
    x = FI.uniform_vector(op.N, seed=7)
    assert_close(host(op.apply(dev(x))), oracle_action(mesh, p, p + 1, form, x))


# ---------------------------------------------------------------- a8: Dirichlet

@pytest.mark.parametrize("form", ["mass", "diffusion"])
@pytest.mark.parametrize("p", [1, 2, 4, 6, 8])
def test_apply_constrained_matches_oracle(p, form):
    shape = SHAPES[p]
    op, mesh = make(shape, p, form, seed=11)
    ess = op.boundary_dofs()
    op.set_essential(ess)
    x = FI.uniform_vector(op.N, seed=12)
    y = host(op.apply(dev(x)))
    assert_close(y, oracle_action(mesh, p, p + 2, form, x, ess=ess.astype(np.int64)))
    # an arbitrary (non-boundary) essential set, then clearing it
    rng = np.random.default_rng(3)
    ess2 = np.sort(rng.choice(op.N, size=max(1, op.N // 7), replace=False)).astype(np.int32)
    op.set_essential(ess2)
    assert_close(host(op.apply(dev(x))), oracle_action(mesh, p, p + 2, form, x, ess=ess2.astype(np.int64)))
    op.set_essential([])
    assert_close(host(op.apply(dev(x))), oracle_action(mesh, p, p + 2, form, x))


# ---------------------------------------------------------------- a10: diagonal

@pytest.mark.parametrize("form", ["mass", "diffusion"])
@pytest.mark.parametrize("p", [1, 2, 3, 5, 8])
def test_diagonal_matches_oracle(p, form):
    shape = SHAPES[p]
    op, mesh = make(shape, p, form, seed=13)
    assert_close(host(op.diagonal()), O.diagonal_elementwise(mesh, p, p + 2, form))
    ess = op.boundary_dofs()
    op.set_essential(ess)
    assert_close(host(op.diagonal()), O.diagonal_elementwise(mesh, p, p + 2, form, ess=ess.astype(np.int64)))


# ---------------------------------------------------------------- a11: load vector

@pytest.mark.parametrize("p", [1, 2, 4, 8])
def test_rhs_matches_oracle(p):
    shape = SHAPES[p]
    op, mesh = make(shape, p, "diffusion", seed=17)
    f = FI.uniform_vector(op.E * op.q ** 3, seed=18)
    assert_close(host(op.rhs(dev(f))), O.rhs_from_qp(mesh, p, p + 2, f.reshape(op.E, -1)))
    op.set_essential(op.boundary_dofs())
    prob = O.Problem(mesh, p, None, O.DIFFUSION, assemble=False)
    assert_close(host(op.rhs_sine(3 * math.pi ** 2)), prob.sine_rhs())


# ---------------------------------------------------------------- invariants on the GPU

@pytest.mark.parametrize("p", [1, 3, 6])
def test_gpu_invariants(p):
    shape = (3, 2, 3)
    opm, _ = make(shape, p, "mass", seed=19)
    opk, _ = make(shape, p, "diffusion", seed=19)
    one = torch.ones(opm.N, dtype=torch.float64, device="cuda")
    assert abs(float(opm.apply(one).sum()) - 1.0) < 1e-13          # 1^T M 1 = |Omega|
    assert float(opk.apply(one).abs().max()) < 1e-11               # K 1 = 0
    u = dev(FI.uniform_vector(opk.N, seed=1))
    v = dev(FI.uniform_vector(opk.N, seed=2))
    for op in (opm, opk):
        a, b = float(torch.dot(u, op.apply(v))), float(torch.dot(v, op.apply(u)))
        assert abs(a - b) <= 1e-12 * max(abs(a), 1.0)


# ---------------------------------------------------------------- a9: CG solve

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_poisson_4x4x4_p2_solve(seed):
    """The plain FP64 Poisson problem: 4x4x4 perturbed hexes, p=2 (729 DOFs), q=4,
    sine manufactured solution, homogeneous Dirichlet, Jacobi PCG to 1e-10."""
    shape, p = (4, 4, 4), 2
    op, mesh = make(shape, p, "diffusion", seed=seed)
    assert op.N == 729
    op.set_essential(op.boundary_dofs())
    b = op.rhs_sine(3 * math.pi ** 2)
    x, st = op.solve(b, rtol=1e-10, maxit=1000)
    prob = O.Problem(mesh, p, None, O.DIFFUSION)
    bo = prob.sine_rhs()
    assert_close(host(b), bo)
    xo, it_o, res_o = prob.solve(bo, rtol=1e-10)
    assert st["status"] == 0 and st["rel_residual"] <= 1e-10
    assert abs(st["iterations"] - it_o) <= 1
    assert rel_err(host(x), xo) <= 1e-9
    xt, _, _ = prob.solve(bo, rtol=1e-14)
    assert rel_err(host(x), xt) <= 1e-8
    # discretisation error of the solution is that of the oracle's
    e_gpu = O.l2_error(mesh, p, host(x), O.sine_solution)
    e_orc = O.l2_error(mesh, p, xo, O.sine_solution)
    assert abs(e_gpu - e_orc) <= 1e-8 * e_orc


@pytest.mark.parametrize("form,p,shape", [("mass", 3, (3, 3, 2)), ("diffusion", 5, (2, 3, 2)),
                                          ("diffusion", 8, (2, 1, 2)), ("mass", 1, (7, 5, 6))])
def test_solve_matches_oracle(form, p, shape):
    op, mesh = make(shape, p, form, seed=23)
    prob = O.Problem(mesh, p, None, form, assemble=p <= 5)
    if form == "diffusion":
        op.set_essential(prob.ess.astype(np.int32))
    b = FI.uniform_vector(op.N, seed=24)
    b[prob.ess] = 0.0
    x, st = op.solve(dev(b), rtol=1e-10, maxit=5000)
    xo, it_o, _ = prob.solve(b, rtol=1e-10)
    assert abs(st["iterations"] - it_o) <= 1
    assert rel_err(host(x), xo) <= 1e-8


def test_solve_host_buffers_equals_device():
    op, _ = make((3, 3, 3), 3, "diffusion", seed=29)
    op.set_essential(op.boundary_dofs())
    b = op.rhs_sine(1.0)
    xd, st_d = op.solve(b, rtol=1e-10)
    xh, st_h = op.solve_host(host(b), rtol=1e-10)
    assert st_d["iterations"] == st_h["iterations"]
    assert rel_err(xh, host(xd)) <= 1e-14


def test_unpreconditioned_and_fixed_iterations():
    op, mesh = make((3, 3, 3), 2, "diffusion", seed=31)
    op.set_essential(op.boundary_dofs())
    b = op.rhs_sine(1.0)
    x, st = op.solve(b, rtol=1e-10, precond="none")
    prob = O.Problem(mesh, 2, None, O.DIFFUSION)
    xo, it_o, _ = O.jacobi_pcg(lambda v: prob.Ac @ v, host(b), np.ones(prob.N), rtol=1e-10)
    assert abs(st["iterations"] - it_o) <= 1
    x2 = torch.zeros_like(b)
    st2 = op.iterations(b, x2, 5)
    assert st2["iterations"] == 5
    _, _, res5 = O.jacobi_pcg(lambda v: prob.Ac @ v, host(b), prob.Ac.diagonal(), rtol=0.0, maxit=5)
    assert abs(st2["rel_residual"] - res5) <= 1e-10 * max(res5, 1e-30) + 1e-14


def test_noconv_status():
    F = fepa()
    op, _ = make((4, 4, 4), 3, "diffusion", seed=1)
    op.set_essential(op.boundary_dofs())
    b = op.rhs_sine(1.0)
    with pytest.raises(F.FepaError) as ei:
        op.solve(b, rtol=1e-12, maxit=3)
    assert ei.value.code == -5
    x, st = op.solve(b, rtol=1e-12, maxit=3, raise_on_noconv=False)
    assert st["iterations"] == 3 and st["status"] == -5


# ---------------------------------------------------------------- edge cases

@pytest.mark.parametrize("p", [1, 4, 8])
def test_single_element(p):
    for form in ("mass", "diffusion"):
        op, mesh = make((1, 1, 1), p, form, seed=37)
        x = FI.uniform_vector(op.N, seed=38)
        assert_close(host(op.apply(dev(x))), O.assemble_csr(mesh, p, p + 2, form) @ x)


def test_inverted_element_rejected():
    F = fepa()
    verts = FI.perturbed_cube_vertices(2, 2, 2, seed=0)
    verts[13] = [0.95, 0.95, 0.95]   # the interior vertex pushed past its neighbours -> det J < 0
    with pytest.raises(ValueError):  # the oracle agrees that the mesh is inverted
        O.qp_factors(O.HexGridMesh(2, 2, 2, verts).element_corners(), O.rule(2, 4), O.DIFFUSION)
    with pytest.raises(F.FepaError) as ei:
        F.Operator(2, 2, 2, verts, 2, form="diffusion")
    assert ei.value.code == -4


def test_argument_errors():
    F = fepa()
    op, _ = make((2, 2, 2), 2, "mass")
    with pytest.raises(F.FepaError):
        op.set_essential([op.N])
    with pytest.raises(F.FepaError):
        op.set_essential([-1])
    x = torch.zeros(op.N, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        op.apply(torch.zeros(op.N + 1, dtype=torch.float64, device="cuda"))
    with pytest.raises(TypeError):
        op.apply(x.float())
    with pytest.raises(F.FepaError):
        op.solve(x, rtol=-1.0)


def test_launches_are_counted():
    F = fepa()
    op, _ = make((2, 2, 2), 2, "mass")
    one = torch.ones(op.N, dtype=torch.float64, device="cuda")
    op.apply(one)   # the first FP64 use may time the kernel variants (counted launches)
    c0 = F.launch_count()
    op.apply(one)
    assert F.launch_count() == c0 + 1


# ---------------------------------------------------------------- full size, sampled

def test_full_size_bp3_p4_sampled():
    """Diffusion, p=4 on 64^3 perturbed hexes (257^3 DOFs), constrained action, sampled
    rows checked one by one against the oracle; plus global invariants."""
    shape, p = (64, 64, 64), 4
    op, mesh = make(shape, p, "diffusion", seed=0)
    assert op.N == 257 ** 3
    ess = op.boundary_dofs()
    op.set_essential(ess)
    x = FI.uniform_vector(op.N, seed=0)
    y = host(op.apply(dev(x)))
    rng = np.random.default_rng(42)
    rows = np.concatenate([rng.choice(op.N, 48, replace=False), ess[rng.choice(len(ess), 8, replace=False)],
                           [0, op.N - 1, op.N // 2]])
    ref = O.action_rows(mesh, p, p + 2, O.DIFFUSION, x, rows, ess=ess.astype(np.int64))
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(y[rows] - ref)) <= 1e-12 * scale
    # unconstrained K 1 = 0 at full size
    op.set_essential([])
    one = torch.ones(op.N, dtype=torch.float64, device="cuda")
    assert float(op.apply(one).abs().max()) < 1e-10
