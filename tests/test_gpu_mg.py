"""GPU parity of the p-multigrid pieces against the oracle: order transfers (P, P^T),
the Chebyshev-Jacobi smoother, the lambda_max estimate, the symmetric V-cycle, and the
V-cycle-preconditioned CG solve.  FP64 tolerance 1e-12 (same sums in another order)
for transfers and smoothers; solutions within 1e-9 of the oracle at the 1e-10 stop."""
import math

import numpy as np
import pytest

import fem_inputs as FI
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SMOOTH_LO, SMOOTH_HI, COARSE_LO, COARSE_HI = 0.245, 1.08, 0.003, 1.18


def F():
    import paper_2402_15940_b300 as mod
    return mod


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nd, nb = np.linalg.norm(a - b), np.linalg.norm(b)
    if nb == 0.0:        # e.g. a coarse level whose DOFs are all essential
        return nd
    return nd / nb


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def setup(shape, p, form, seed=0, degree=2, coarse=24):
    verts = FI.perturbed_cube_vertices(*shape, seed=seed)
    op = F().Operator(*shape, verts, p, form=form)
    if form == "diffusion":
        op.set_essential(op.boundary_dofs())
    mg = F().Multigrid(op, smooth_degree=degree, coarse_degree=coarse)
    return op, mg, O.HexGridMesh(*shape, verts)


@pytest.mark.parametrize("form,p,shape", [("diffusion", 4, (3, 2, 2)), ("mass", 3, (2, 3, 2)),
                                          ("diffusion", 8, (2, 1, 2)), ("diffusion", 5, (2, 2, 2))])
def test_levels_and_transfers_match_oracle(form, p, shape):
    op, mg, mesh = setup(shape, p, form)
    orders = [lv["order"] for lv in mg.levels]
    expect = [p]
    while expect[-1] > 1:
        expect.append(max(1, expect[-1] // 2))
    assert orders == expect
    for l in range(len(orders) - 1):
        pf, pc = orders[l], orders[l + 1]
        P = O.order_prolongation(mesh, pc, pf)
        xc = FI.uniform_vector(P.shape[1], seed=l)
        assert rel(mg.prolong(l, dev(xc)).cpu().numpy(), P @ xc) <= 1e-12
        rf = FI.uniform_vector(P.shape[0], seed=10 + l)
        if form == "diffusion":
            rf_in = rf.copy()
            rf_in[O.boundary_dofs(mesh, pf)] = 0.0
            ref = P.T @ rf_in
            ref[O.boundary_dofs(mesh, pc)] = 0.0
        else:
            ref = P.T @ rf
        assert rel(mg.restrict(l, dev(rf)).cpu().numpy(), ref) <= 1e-12


@pytest.mark.parametrize("form,p", [("diffusion", 4), ("mass", 2), ("diffusion", 6)])
def test_smoothers_match_oracle_chebyshev(form, p):
    shape = (2, 2, 3)
    op, mg, mesh = setup(shape, p, form, degree=3, coarse=17)
    for l, lv in enumerate(mg.levels):
        prob = O.Problem(mesh, lv["order"], None, form)
        Ac = prob.Ac
        b = FI.uniform_vector(prob.N, seed=l)
        if form == "diffusion":
            b[prob.ess] = 0.0
        last = l == len(mg.levels) - 1
        lo, hi, k = (COARSE_LO, COARSE_HI, 17) if last else (SMOOTH_LO, SMOOTH_HI, 3)
        ref = O.chebyshev_smoother(lambda v: Ac @ v, Ac.diagonal(), b, lo * lv["lambda_max"], hi * lv["lambda_max"], k)
        assert rel(mg.smooth(l, dev(b)).cpu().numpy(), ref) <= 1e-12


def test_lambda_max_estimate():
    op, mg, mesh = setup((2, 2, 2), 3, "diffusion")
    for lv in mg.levels:
        prob = O.Problem(mesh, lv["order"], None, O.DIFFUSION)
        A = prob.Ac.toarray()
        lam = np.linalg.eigvals(A / np.diag(A)[:, None]).real.max()
        assert 0.95 * lam <= lv["lambda_max"] <= lam * (1 + 1e-9)   # largest Ritz value: from below


@pytest.mark.parametrize("form", ["diffusion", "mass"])
def test_vcycle_symmetric_positive(form):
    op, mg, _ = setup((3, 3, 2), 4, form, seed=2)
    u = dev(FI.uniform_vector(op.N, seed=1))
    v = dev(FI.uniform_vector(op.N, seed=2))
    if form == "diffusion":
        ess = torch.from_numpy(op.boundary_dofs().astype(np.int64)).cuda()
        u[ess] = 0.0
        v[ess] = 0.0
    Mu, Mv = mg.vcycle(u), mg.vcycle(v)
    a, b = float(torch.dot(v, Mu)), float(torch.dot(u, Mv))
    assert abs(a - b) <= 1e-11 * max(abs(a), abs(b))
    assert float(torch.dot(u, Mu)) > 0 and float(torch.dot(v, Mv)) > 0


@pytest.mark.parametrize("form,p,shape", [("diffusion", 4, (4, 4, 4)), ("diffusion", 2, (6, 6, 5)),
                                          ("mass", 3, (3, 3, 3)), ("diffusion", 6, (2, 3, 2))])
def test_mg_solve_matches_oracle_and_needs_fewer_iterations(form, p, shape):
    op, mg, mesh = setup(shape, p, form, seed=5)
    b = op.rhs_sine(3 * math.pi ** 2 if form == "diffusion" else 1.0)
    x, st = mg.solve(b, rtol=1e-10)
    xj, sj = op.solve(b, rtol=1e-10)
    prob = O.Problem(mesh, p, None, form, assemble=p <= 5)
    xo, it_o, _ = prob.solve(b.cpu().numpy(), rtol=1e-13)
    assert st["status"] == 0 and st["rel_residual"] <= 1e-10
    assert rel(x.cpu().numpy(), xo) <= 1e-9
    assert st["iterations"] < sj["iterations"]


@pytest.mark.parametrize("form,p,shape", [("diffusion", 4, (4, 4, 4)), ("diffusion", 8, (2, 2, 2)),
                                          ("mass", 2, (5, 4, 4))])
def test_fp32_vcycle_solve_matches_oracle(form, p, shape):
    """FP32 V-cycle inside the FP64 CG: the preconditioner is FP32, the operator action,
    dot products and scalars FP64, so the solution meets the FP64 tolerance."""
    verts = FI.perturbed_cube_vertices(*shape, seed=6)
    op = F().Operator(*shape, verts, p, form=form)
    if form == "diffusion":
        op.set_essential(op.boundary_dofs())
    b = op.rhs_sine(1.0)
    mg64 = F().Multigrid(op, precision="fp64")
    x64, s64 = mg64.solve(b, rtol=1e-10)
    mg32 = F().Multigrid(op, precision="fp32")
    x32, s32 = mg32.solve(b, rtol=1e-10)
    prob = O.Problem(O.HexGridMesh(*shape, verts), p, None, form, assemble=p <= 5)
    xo, _, _ = prob.solve(b.cpu().numpy(), rtol=1e-13)
    assert s32["status"] == 0 and s32["rel_residual"] <= 1e-10
    assert rel(x32.cpu().numpy(), xo) <= 1e-9
    assert s32["iterations"] <= s64["iterations"] + 2
    for a, c in zip(mg32.levels, mg64.levels):
        assert abs(a["lambda_max"] / c["lambda_max"] - 1) < 1e-3


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_update_follows_moved_mesh(precision):
    shape, p = (3, 3, 3), 4
    op = F().Operator(*shape, FI.perturbed_cube_vertices(*shape, seed=1), p, form="diffusion")
    op.set_essential(op.boundary_dofs())
    mg = F().Multigrid(op, precision=precision)
    verts2 = FI.perturbed_cube_vertices(*shape, seed=2)
    op.set_vertices(verts2)
    mg.update()
    b = op.rhs_sine(1.0)
    x1, s1 = mg.solve(b, rtol=1e-10)
    op2 = F().Operator(*shape, verts2, p, form="diffusion")
    op2.set_essential(op2.boundary_dofs())
    mg2 = F().Multigrid(op2, precision=precision)
    x2, s2 = mg2.solve(op2.rhs_sine(1.0), rtol=1e-10)
    assert abs(s1["iterations"] - s2["iterations"]) <= 1   # atomic summation order may move the stop
    assert rel(x1.cpu().numpy(), x2.cpu().numpy()) <= 1e-9
    tol = 1e-9 if precision == "fp64" else 1e-5   # FP32 atomics reorder the Lanczos process's sums
    for a, c in zip(mg.levels, mg2.levels):
        assert abs(a["lambda_max"] / c["lambda_max"] - 1) < tol


@pytest.mark.parametrize("form,p,shape", [("diffusion", 4, (3, 3, 3)), ("mass", 4, (2, 3, 2)),
                                          ("diffusion", 6, (2, 2, 3))])
def test_vcycle_matches_oracle_and_is_deterministic(form, p, shape):
    """The GPU V-cycle equals the oracle's V-cycle built from the level matrices and
    prolongations with the same eigenvalue bounds, and repeated cycles agree."""
    op, mg, mesh = setup(shape, p, form, seed=3)
    orders = [lv["order"] for lv in mg.levels]
    probs = [O.Problem(mesh, o, None, form) for o in orders]
    As = [pr.Ac for pr in probs]
    Ps = [O.order_prolongation(mesh, orders[l + 1], orders[l]) for l in range(len(orders) - 1)]
    ess = [pr.ess if form == "diffusion" else None for pr in probs]
    b = FI.uniform_vector(op.N, seed=9)
    if form == "diffusion":
        b[probs[0].ess] = 0.0
    ref = O.pmg_vcycle(As, [A.diagonal() for A in As], Ps, [lv["lambda_max"] for lv in mg.levels], 2, 24, b,
                        smooth=(SMOOTH_LO, SMOOTH_HI), coarse=(COARSE_LO, COARSE_HI), ess=ess)
    z1 = mg.vcycle(dev(b)).cpu().numpy()
    z2 = mg.vcycle(dev(b)).cpu().numpy()
    assert rel(z1, ref) <= 1e-11
    assert rel(z1, z2) <= 1e-13
