"""GPU parity of the mixed-precision path: the FP32 operator and FP64 iterative
refinement around an FP32 Jacobi-PCG, against the CPU FP64 oracle.

FP32 action tolerance: every output is a sum through 3 forward contractions (n terms
each), the 3x3 D product, 3 transposed contractions (q terms each) and at most 8
element contributions, all rounded to binary32 (unit roundoff u = 2^-24 ~ 6e-8), plus
the rounding of D and of the 1D tables.  The standard bound gives about
(3n + 3q + 14) u ~ 3e-6 of |B^T| |D| |B| |x| per entry at p = 8; for the random x used
here ||A x|| is within a small factor of that, so relative l2 error <= 1e-5 is the
bound asserted (measured values are near 1e-7).

Refined solve: the FP64 residual decides when to stop, so the solution is checked
against the oracle's FP64 solution to 1e-10 relative error.
"""
import math

import numpy as np
import pytest

import fem_inputs as FI
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = 1e-5
SHAPES = {1: (5, 4, 3), 2: (4, 3, 3), 3: (3, 3, 3), 4: (3, 3, 2), 5: (3, 2, 2), 6: (3, 2, 1), 7: (2, 2, 2),
          8: (3, 1, 1)}


def F():
    import paper_2402_15940_b300 as mod
    return mod


def make(shape, p, form, seed=0):
    verts = FI.perturbed_cube_vertices(*shape, seed=seed)
    return F().Operator(*shape, verts, p, form=form), O.HexGridMesh(*shape, verts)


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def oracle_action(mesh, p, form, x, ess=None, q=None):
    q = p + 2 if q is None else q
    if p <= 5:
        A = O.assemble_csr(mesh, p, q, form)
        if ess is not None:
            A = O.constrain(A, ess)
        return A @ x
    return O.action_elementwise(mesh, p, q, form, x, ess=ess)


@pytest.mark.parametrize("form", ["mass", "diffusion"])
@pytest.mark.parametrize("p", list(range(1, 9)))
def test_apply_f32_matches_oracle(p, form):
    op, mesh = make(SHAPES[p], p, form, seed=p)
    x32 = FI.uniform_vector(op.N, seed=200 + p).astype(np.float32)
    y = op.apply_f32(torch.from_numpy(x32).cuda()).cpu().numpy()
    ref = oracle_action(mesh, p, form, x32.astype(np.float64))
    e = rel(y, ref)
    assert e <= TOL32, e


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("form,p", [("diffusion", 1), ("diffusion", 4), ("mass", 3), ("diffusion", 8),
                                    ("mass", 6)])
def test_every_f32_variant_matches_oracle(form, p, variant):
    op, mesh = make(SHAPES[p], p, form, seed=11 + p)
    op.set_f32_variant(variant)
    ess = op.boundary_dofs()
    op.set_essential(ess)
    x32 = FI.uniform_vector(op.N, seed=13).astype(np.float32)
    y = op.apply_f32(torch.from_numpy(x32).cuda()).cpu().numpy()
    assert op.f32_variant()[0] == variant
    assert rel(y, oracle_action(mesh, p, form, x32.astype(np.float64), ess=ess.astype(np.int64))) <= TOL32


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("form", ["mass", "diffusion"])
@pytest.mark.parametrize("p", list(range(1, 9)))
def test_f32_variants_with_q_p_plus_1(p, form, variant):
    """Every variant at q = p + 1 (each (p, q, form) has its own shared-memory layout) on a
    mesh of several blocks of elements with a ragged last block."""
    shape = (5, 3, 2) if p <= 4 else (3, 2, 2)
    op, mesh = make_q(shape, p, form, p + 1, seed=40 + p)
    op.set_f32_variant(variant)
    ess = op.boundary_dofs()
    op.set_essential(ess)
    x32 = FI.uniform_vector(op.N, seed=41 + p).astype(np.float32)
    y = op.apply_f32(torch.from_numpy(x32).cuda()).cpu().numpy()
    ref = oracle_action(mesh, p, form, x32.astype(np.float64), ess=ess.astype(np.int64), q=p + 1)
    assert rel(y, ref) <= TOL32


def make_q(shape, p, form, q, seed=0):
    verts = FI.perturbed_cube_vertices(*shape, seed=seed)
    return F().Operator(*shape, verts, p, form=form, q=q), O.HexGridMesh(*shape, verts)


def test_autotuned_variant_is_recorded():
    op, _ = make((4, 4, 4), 3, "diffusion", seed=3)
    x32 = torch.zeros(op.N, dtype=torch.float32, device="cuda")
    assert op.f32_variant()[0] == -1
    op.apply_f32(x32)
    v, name = op.f32_variant()
    assert 0 <= v <= 3 and name != "unknown"


@pytest.mark.parametrize("p", [2, 5, 8])
def test_apply_f32_constrained(p):
    op, mesh = make(SHAPES[p], p, "diffusion", seed=3)
    ess = op.boundary_dofs()
    op.set_essential(ess)
    x32 = FI.uniform_vector(op.N, seed=5).astype(np.float32)
    y = op.apply_f32(torch.from_numpy(x32).cuda()).cpu().numpy()
    assert rel(y, oracle_action(mesh, p, "diffusion", x32.astype(np.float64), ess=ess.astype(np.int64))) <= TOL32


def test_apply_f32_follows_new_vertices():
    op, _ = make((3, 3, 3), 3, "diffusion", seed=1)
    x32 = torch.from_numpy(FI.uniform_vector(op.N, seed=1).astype(np.float32)).cuda()
    op.apply_f32(x32)
    verts2 = FI.perturbed_cube_vertices(3, 3, 3, seed=2)
    op.set_vertices(verts2)
    y = op.apply_f32(x32).cpu().numpy()
    mesh2 = O.HexGridMesh(3, 3, 3, verts2)
    assert rel(y, oracle_action(mesh2, 3, "diffusion", x32.cpu().numpy().astype(np.float64))) <= TOL32


@pytest.mark.parametrize("form,p,shape", [("diffusion", 2, (4, 4, 4)), ("diffusion", 4, (3, 3, 3)),
                                          ("diffusion", 6, (2, 2, 2)), ("mass", 3, (3, 4, 2)),
                                          ("diffusion", 8, (2, 1, 2))])
def test_refined_solution_matches_oracle(form, p, shape):
    op, mesh = make(shape, p, form, seed=41)
    prob = O.Problem(mesh, p, None, form, assemble=p <= 5)
    if form == "diffusion":
        op.set_essential(prob.ess.astype(np.int32))
        b = op.rhs_sine(3 * math.pi ** 2)
        bo = prob.sine_rhs()
    else:
        bo = FI.uniform_vector(op.N, seed=42)
        b = torch.from_numpy(bo).cuda()
    x, st = op.solve_refined(b, rtol=1e-12, inner_rtol=1e-4)
    assert st["status"] == 0 and st["rel_residual"] <= 1e-12 and st["outer_iterations"] >= 1
    xo, _, _ = prob.solve(bo, rtol=1e-14)
    assert rel(x.cpu().numpy(), xo) <= 1e-10


def test_refined_counts_and_host_buffers():
    op, mesh = make((4, 4, 4), 3, "diffusion", seed=43)
    op.set_essential(op.boundary_dofs())
    b = op.rhs_sine(1.0)
    xd, sd = op.solve_refined(b, rtol=1e-10)
    xh, sh = op.solve_refined_host(b.cpu().numpy(), rtol=1e-10)
    # FP32 atomic summation order varies between runs: counts may move a little
    assert abs(sd["outer_iterations"] - sh["outer_iterations"]) <= 1
    assert abs(sd["inner_iterations"] - sh["inner_iterations"]) <= max(4, 0.1 * sd["inner_iterations"])
    assert rel(xh, xd.cpu().numpy()) <= 1e-9
    # the plain FP64 solve reaches the same solution
    x64, _ = op.solve(b, rtol=1e-10)
    assert rel(xd.cpu().numpy(), x64.cpu().numpy()) <= 1e-8


def test_refined_noconv():
    op, _ = make((4, 4, 4), 2, "diffusion", seed=44)
    op.set_essential(op.boundary_dofs())
    b = op.rhs_sine(1.0)
    x, st = op.solve_refined(b, rtol=1e-14, max_outer=1, raise_on_noconv=False)
    assert st["status"] == -5 and st["outer_iterations"] == 1


FIRST_STEP_CASES = [("diffusion", 3, (5, 4, 3), v) for v in (0, 1, 2)] + \
    [("diffusion", 4, (5, 4, 3), v) for v in (0, 1, 2)] + \
    [("mass", 4, (4, 3, 3), 1), ("diffusion", 5, (3, 3, 2), 2), ("diffusion", 6, (3, 2, 2), 1),
     ("mass", 8, (2, 1, 2), 0)]


@pytest.mark.parametrize("form,p,shape,variant", [("diffusion", 4, (5, 4, 3), 0), ("diffusion", 4, (5, 4, 3), 1),
                                                  ("diffusion", 3, (5, 4, 3), 2), ("diffusion", 5, (3, 3, 2), 1),
                                                  ("diffusion", 2, (4, 4, 3), 1), ("diffusion", 6, (3, 2, 2), 3),
                                                  ("mass", 5, (3, 3, 2), 2), ("mass", 8, (2, 1, 2), 1)])
def test_apply_f32_dot_matches_oracle(form, p, shape, variant):
    """y = A x and (x, A x) from one call: the fused kernel for p >= 3 and variants 0-2,
    a separate pass elsewhere (p = 2, variant 3); x is not zero at essential DOFs."""
    op, mesh = make(shape, p, form, seed=50)
    prob = O.Problem(mesh, p, None, form, assemble=p <= 5)
    if form == "diffusion":
        op.set_essential(prob.ess.astype(np.int32))
    op.set_f32_variant(variant)
    x32 = torch.from_numpy(FI.uniform_vector(op.N, seed=51).astype(np.float32)).cuda()
    y, xax = op.apply_f32_dot(x32)
    xd = x32.cpu().numpy().astype(np.float64)
    ya = prob.apply(xd, constrained=True)
    assert rel(y.cpu().numpy(), ya) <= TOL32
    assert abs(float(xax.item()) - xd @ ya) <= TOL32 * abs(xd @ ya)
    y2, xax2 = op.apply_f32_dot(x32)  # the slots were cleared for the next call
    assert abs(float(xax2.item()) - float(xax.item())) <= 1e-6 * abs(xd @ ya)


@pytest.mark.parametrize("field", ["sine_solution", "interior_one"])
def test_apply_f32_dot_on_smooth_low_energy_vectors(field):
    """(x, A x) from the fused FP32 kernel at BP3 p = 4 on smooth, low-energy x, where the
    diffusion form's terms cancel most: the discrete solution of the sine problem, and a field
    that is 1 at every free DOF and 0 on the boundary (A_e x_e is rounding noise on every
    interior element).  The fused FP32 sum is compared with the exact (x, A x) of the same
    FP32 x, and with the product formed from the kernel's FP32 y in FP64 (what the separate
    dot pass computes)."""
    op, mesh = make((6, 5, 4), 4, "diffusion", seed=52)
    prob = O.Problem(mesh, 4, None, "diffusion")
    op.set_essential(prob.ess.astype(np.int32))
    op.set_f32_variant(1)
    if field == "sine_solution":
        xd, _, _ = prob.solve(prob.sine_rhs(), rtol=1e-12)
    else:
        xd = np.ones(op.N)
        xd[prob.ess] = 0.0
    x32 = torch.from_numpy(xd.astype(np.float32)).cuda()
    xr = x32.cpu().numpy().astype(np.float64)
    exact = xr @ prob.apply(xr, constrained=True)
    y, xax = op.apply_f32_dot(x32)
    e_fused = abs(float(xax.item()) - exact) / abs(exact)
    e_sep = abs(xr @ y.cpu().numpy().astype(np.float64) - exact) / abs(exact)
    print(f"{field}: (x, A x) relative error fused {e_fused:.2e}, from FP32 y {e_sep:.2e}")
    assert e_fused <= 1e-5 and e_sep <= 1e-5


@pytest.mark.parametrize("fused", [True, False])
@pytest.mark.parametrize("form,p,shape,variant", FIRST_STEP_CASES)
def test_first_cg_step_matches_oracle(form, p, shape, variant, fused):
    """One FP32 Jacobi-PCG step from x = 0 is x = alpha z with z = b / diag(A) and
    alpha = (z, b) / (z, A z).  With the fused build (z, A z) comes out of the action kernel
    (per-element sums over blocks with a ragged last group, plus the identity rows of the
    essential DOFs, where b is not zero here); without it from a separate pass over z and A z."""
    op, mesh = make(shape, p, form, seed=47)
    prob = O.Problem(mesh, p, None, form, assemble=p <= 5)
    if form == "diffusion":
        op.set_essential(prob.ess.astype(np.int32))
    op.set_f32_variant(variant)
    op.set_fused_dot(fused)
    bo = FI.uniform_vector(op.N, seed=48)
    x, st = op.solve_refined(torch.from_numpy(bo).cuda(), rtol=1e-14, max_outer=1, inner_maxit=1,
                             raise_on_noconv=False)
    op.set_fused_dot(True)
    assert st["inner_iterations"] == 1 and st["outer_iterations"] == 1
    z = bo / prob.diagonal()
    alpha = (z @ bo) / (z @ prob.apply(z, constrained=True))
    assert rel(x.cpu().numpy(), alpha * z) <= TOL32


@pytest.mark.parametrize("form,p,shape", [("diffusion", 4, (6, 5, 4)), ("mass", 3, (5, 4, 4))])
def test_fused_dot_solve_equals_separate_pass(form, p, shape):
    """The refined solve with (d, A d) from the action kernel reaches the solution of the one
    with a separate (d, h) pass, in about as many FP32 iterations."""
    op, mesh = make(shape, p, form, seed=49)
    if form == "diffusion":
        op.set_essential(op.boundary_dofs())
    b = op.rhs_sine(1.0)
    xf, sf = op.solve_refined(b, rtol=1e-10)
    op.set_fused_dot(False)
    xs, ss = op.solve_refined(b, rtol=1e-10)
    op.set_fused_dot(True)
    assert sf["status"] == 0 and ss["status"] == 0
    assert abs(sf["inner_iterations"] - ss["inner_iterations"]) <= max(4, 0.1 * ss["inner_iterations"])
    assert rel(xf.cpu().numpy(), xs.cpu().numpy()) <= 1e-9


@pytest.mark.parametrize("mode", ["graph", "stream"])
def test_refined_single_step_corrections(mode):
    """Inner solves of one FP32 CG step each: every correction is that step's alpha d, which
    the loop's last (flushed) x update must deliver, so the FP64 refinement still converges,
    in graph and stream mode alike."""
    op, mesh = make((3, 3, 3), 2, "mass", seed=46)
    op.set_cg_mode(mode)
    b = op.rhs_sine(1.0)
    x, st = op.solve_refined(b, rtol=1e-8, max_outer=400, inner_maxit=1)
    op.set_cg_mode("graph")
    assert st["status"] == 0 and st["rel_residual"] <= 1e-8
    assert st["outer_iterations"] > 3 and st["inner_iterations"] == st["outer_iterations"]
    xo, _, _ = O.Problem(mesh, 2, None, "mass").solve(b.cpu().numpy(), rtol=1e-12)
    assert rel(x.cpu().numpy(), xo) <= 1e-6


@pytest.mark.parametrize("solver", ["cg", "refined"])
def test_stream_mode_equals_graph_mode(solver):
    op, _ = make((5, 4, 4), 3, "diffusion", seed=45)
    op.set_essential(op.boundary_dofs())
    b = op.rhs_sine(1.0)
    run = (lambda: op.solve(b, rtol=1e-10)) if solver == "cg" else (lambda: op.solve_refined(b, rtol=1e-10))
    xg, sg = run()
    op.set_cg_mode("stream")
    xs, ss = run()
    op.set_cg_mode("graph")
    key = "iterations" if solver == "cg" else "inner_iterations"
    # FP64 CG: within one iteration; FP32 inner counts may move a little (atomic order)
    assert abs(sg[key] - ss[key]) <= (1 if solver == "cg" else max(4, 0.1 * sg[key]))
    assert rel(xs.cpu().numpy(), xg.cpu().numpy()) <= 1e-9


@pytest.mark.parametrize("p,n", [(4, 64), (6, 32)])
def test_refined_full_size_sampled(p, n):
    """The refined solve at the sizes of the mixed-precision configuration (diffusion,
    p=4 on 64^3 and p=6 on 32^3 perturbed hexes, sine RHS): sampled rows of the FP64
    residual checked one by one by the oracle, and agreement with the plain FP64 solve."""
    op, mesh = make((n, n, n), p, "diffusion", seed=0)
    ess = op.boundary_dofs()
    op.set_essential(ess)
    b = op.rhs_sine(3 * math.pi ** 2)
    x, st = op.solve_refined(b, rtol=1e-10)
    assert st["status"] == 0 and st["rel_residual"] <= 1e-10
    xh, bh = x.cpu().numpy(), b.cpu().numpy()
    rng = np.random.default_rng(7)
    rows = rng.choice(op.N, 40, replace=False)
    Ax = O.action_rows(mesh, p, p + 2, O.DIFFUSION, xh, rows, ess=ess.astype(np.int64))
    assert np.max(np.abs(bh[rows] - Ax)) <= 1e-10 * np.linalg.norm(bh)
    x64, s64 = op.solve(b, rtol=1e-12, maxit=20000)
    assert rel(xh, x64.cpu().numpy()) <= 1e-9


# ---------------------------------------------------------------- reliable updates

@pytest.mark.parametrize("form,p,shape", [("diffusion", 2, (4, 4, 4)), ("diffusion", 4, (3, 3, 3)),
                                          ("diffusion", 6, (2, 2, 2)), ("mass", 3, (3, 4, 2)),
                                          ("diffusion", 8, (2, 1, 2))])
def test_reliable_solution_matches_oracle(form, p, shape):
    op, mesh = make(shape, p, form, seed=41)
    prob = O.Problem(mesh, p, None, form, assemble=p <= 5)
    if form == "diffusion":
        op.set_essential(prob.ess.astype(np.int32))
        b = op.rhs_sine(3 * math.pi ** 2)
        bo = prob.sine_rhs()
    else:
        bo = FI.uniform_vector(op.N, seed=42)
        b = torch.from_numpy(bo).cuda()
    x, st = op.solve_reliable(b, rtol=1e-12, delta=0.1)
    assert st["status"] == 0 and st["rel_residual"] <= 1e-12
    xo, _, _ = prob.solve(bo, rtol=1e-14)
    assert rel(x.cpu().numpy(), xo) <= 1e-10


@pytest.mark.parametrize("delta", [0.3, 0.1, 0.01])
def test_reliable_keeps_the_krylov_space(delta):
    """With the direction carried over each replacement, the FP32 iteration count stays
    near the FP64 CG's (the restarted refinement needs several times more here)."""
    op, _ = make((8, 8, 8), 3, "diffusion", seed=46)
    op.set_essential(op.boundary_dofs())
    b = op.rhs_sine(3 * math.pi ** 2)
    x64, s64 = op.solve(b, rtol=1e-10)
    x, st = op.solve_reliable(b, rtol=1e-10, delta=delta)
    assert st["status"] == 0 and st["rel_residual"] <= 1e-10 and st["outer_iterations"] >= 1
    assert st["inner_iterations"] <= 1.3 * s64["iterations"] + 10
    assert rel(x.cpu().numpy(), x64.cpu().numpy()) <= 1e-8
    xh, sh = op.solve_reliable_host(b.cpu().numpy(), rtol=1e-10, delta=delta)
    assert abs(sh["inner_iterations"] - st["inner_iterations"]) <= max(4, 0.1 * st["inner_iterations"])
    assert rel(xh, x.cpu().numpy()) <= 1e-9


def test_reliable_noconv_and_arguments():
    op, _ = make((4, 4, 4), 2, "diffusion", seed=44)
    op.set_essential(op.boundary_dofs())
    b = op.rhs_sine(1.0)
    x, st = op.solve_reliable(b, rtol=1e-14, maxit=5, raise_on_noconv=False)
    assert st["status"] == -5 and st["inner_iterations"] >= 5
    for bad in (0.0, 1.0, -0.5):
        with pytest.raises(Exception):
            op.solve_reliable(b, delta=bad)


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_fused_dot_on_a_smooth_vector(variant):
    """(x, A x) from the fused FP32 action on a smooth, low-energy x (the sine interpolant,
    zero on the boundary): per element the terms x_l (A_e x)_l nearly cancel, the case where
    summing them in FP32 loses the most.  Compared with the FP64 oracle's x . A x and with the
    separate pass (the persistent variant has no fused build, so there (x, A x) is a
    double-float dot of x and the FP32 y)."""
    shape, p = (6, 5, 4), 4
    op, mesh = make(shape, p, "diffusion", seed=52)
    prob = O.Problem(mesh, p, None, O.DIFFUSION)
    op.set_essential(prob.ess.astype(np.int32))
    xd = O.sine_solution(O.node_coords(mesh, p)).astype(np.float32).astype(np.float64)
    x32 = torch.from_numpy(xd.astype(np.float32)).cuda()
    exact = xd @ prob.apply(xd, constrained=True)
    op.set_f32_variant(variant)
    _, fused = op.apply_f32_dot(x32)
    op.set_f32_variant(3)
    _, sep = op.apply_f32_dot(x32)
    e_fused = abs(float(fused.item()) - exact) / exact
    e_sep = abs(float(sep.item()) - exact) / exact
    print(f"smooth x: (x, A x) rel. error fused {e_fused:.2e}, separate pass {e_sep:.2e}")
    assert e_fused <= 1e-5 and e_sep <= 1e-5
