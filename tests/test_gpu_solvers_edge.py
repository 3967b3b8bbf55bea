"""Degenerate and full-size cases of the solvers: a zero right-hand side (every solver returns
x = 0 at once), and the reliable-update and p-multigrid solves at the size of the BP3
benchmark (diffusion, p=4 on 64^3 perturbed hexes, 257^3 DOFs) with sampled rows of the FP64
residual checked one by one against the oracle."""
import math

import numpy as np
import pytest

import fem_inputs as FI
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def F():
    import paper_2402_15940_b300 as mod
    return mod


def make(shape, p, form, seed=0):
    verts = FI.perturbed_cube_vertices(*shape, seed=seed)
    op = F().Operator(*shape, verts, p, form=form)
    if form == "diffusion":
        op.set_essential(op.boundary_dofs())
    return op, O.HexGridMesh(*shape, verts)


@pytest.mark.parametrize("form", ["mass", "diffusion"])
@pytest.mark.parametrize("solver", ["cg", "refined", "reliable", "mg"])
def test_zero_rhs_returns_zero(solver, form):
    op, _ = make((3, 3, 2), 3, form, seed=2)
    b = torch.zeros(op.N, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    if solver == "cg":
        _, st = op.solve(b, x, rtol=1e-10)
        assert st["iterations"] == 0
    elif solver == "refined":
        _, st = op.solve_refined(b, x, rtol=1e-10)
        assert st["outer_iterations"] == 0
    elif solver == "reliable":
        _, st = op.solve_reliable(b, x, rtol=1e-10)
        assert st["inner_iterations"] == 0
    else:
        _, st = F().Multigrid(op).solve(b, x, rtol=1e-10)
        assert st["iterations"] == 0
    assert st["status"] == 0
    assert float(x.abs().max()) == 0.0


def sampled_residual_check(op, mesh, p, x, b, ess, rows=40, seed=7):
    xh, bh = x.cpu().numpy(), b.cpu().numpy()
    rng = np.random.default_rng(seed)
    r = rng.choice(op.N, rows, replace=False)
    Ax = O.action_rows(mesh, p, p + 2, O.DIFFUSION, xh, r, ess=ess.astype(np.int64))
    return np.max(np.abs(bh[r] - Ax)) / np.linalg.norm(bh)


@pytest.mark.parametrize("solver", ["reliable", "mg32"])
def test_full_size_bp3_p4_solvers(solver):
    shape, p = (64, 64, 64), 4
    op, mesh = make(shape, p, "diffusion", seed=0)
    ess = op.boundary_dofs()
    b = op.rhs_sine(3 * math.pi ** 2)
    if solver == "reliable":
        x, st = op.solve_reliable(b, rtol=1e-10)
        assert st["status"] == 0 and st["rel_residual"] <= 1e-10
        assert st["inner_iterations"] <= 1.3 * 1123
    else:
        x, st = F().Multigrid(op, precision="fp32").solve(b, rtol=1e-10)
        assert st["status"] == 0 and st["rel_residual"] <= 1e-10 and st["iterations"] <= 15
    assert sampled_residual_check(op, mesh, p, x, b, ess) <= 1e-10
    # and the same solution as the plain FP64 solve
    x64, _ = op.solve(b, rtol=1e-12, maxit=20000)
    rel = float((x - x64).norm() / x64.norm())
    assert rel <= 1e-8
