"""Failure paths, made on the host without faulting the GPU.

* A kernel's bounded wait that runs out: the test lowers the poll limit of the FP32 action's
  first wait (for its TMA copy of D) to zero through the library's test knob, so every block
  gives up at once, records the expiry in the op's error word and still drains its copy in
  flight.  The blocking call reports FEPA_ERR_TIMEOUT once; with the limit restored the same op
  solves normally (the context stays usable and the word was cleared).
* Non-finite inputs (NaN or infinity in b or in the initial guess): every solver stops at once
  with FEPA_ERR_NONFINITE instead of iterating to maxit; in a batch only the affected problem
  stops, and the others' results are those of the same batch without the bad value.
"""
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


def fepa():
    from paper_2402_15940_b300 import fepa as mod
    return mod


def make(shape, p, form, seed=0):
    verts = FI.perturbed_cube_vertices(*shape, seed=seed)
    op = F().Operator(*shape, verts, p, form=form)
    if form == "diffusion":
        op.set_essential(op.boundary_dofs())
    return op, O.HexGridMesh(*shape, verts)


@pytest.mark.parametrize("variant", [0, 3])
def test_expired_wait_reports_timeout_once_and_recovers(variant):
    op, mesh = make((5, 4, 3), 4, "diffusion", seed=61)
    op.set_f32_variant(variant)          # the launch shapes that stage D by TMA
    b = op.rhs_sine(3 * math.pi ** 2)
    x = torch.zeros(op.N, dtype=torch.float64, device="cuda")
    try:
        fepa().test_set_first_wait_limit(0)
        with pytest.raises(fepa().FepaError) as ei:
            op.solve_refined(b, x, rtol=1e-10, max_outer=1, inner_maxit=3)
        assert ei.value.code == fepa().ERR_TIMEOUT
    finally:
        fepa().test_set_first_wait_limit(-1)
    x.zero_()
    _, st = op.solve_refined(b, x, rtol=1e-12)           # no stale error, same op and context
    assert st["status"] == 0
    prob = O.Problem(mesh, 4, None, O.DIFFUSION)
    xo, _, _ = prob.solve(prob.sine_rhs(), rtol=1e-14)
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-10 * np.linalg.norm(xo)


@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
@pytest.mark.parametrize("where", ["b", "x0"])
@pytest.mark.parametrize("solver", ["cg", "refined", "reliable", "mg", "noalloc"])
def test_non_finite_input_stops_at_once(solver, where, bad):
    op, _ = make((3, 3, 2), 3, "diffusion", seed=62)
    b = op.rhs_sine(1.0)
    x = torch.zeros(op.N, dtype=torch.float64, device="cuda")
    i = op.N // 2 + 3                     # an interior DOF
    (b if where == "b" else x)[i] = bad
    l0 = F().launch_count()
    with pytest.raises(fepa().FepaError) as ei:
        if solver == "cg":
            op.solve(b, x, rtol=1e-10, maxit=5000)
        elif solver == "refined":
            op.solve_refined(b, x, rtol=1e-10, max_outer=50)
        elif solver == "reliable":
            op.solve_reliable(b, x, rtol=1e-10, maxit=5000)
        elif solver == "noalloc":
            import ctypes
            st = fepa().CgStats()
            lib = fepa().load_library()
            rc = lib.fepa_cg_solve_noalloc(op._h, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                           1e-10, 5000, 1, ctypes.byref(st))
            assert st.status == fepa().ERR_NONFINITE
            fepa()._check(rc)
        else:
            F().Multigrid(op, precision="fp64").solve(b, x, rtol=1e-10, maxit=500)
    assert ei.value.code == fepa().ERR_NONFINITE, str(ei.value)
    assert F().launch_count() - l0 < 400       # stopped at once, not after thousands of iterations


def test_batch_non_finite_problem_stops_alone():
    shapes = [((3, 2, 2), 2, "diffusion"), ((2, 3, 2), 3, "mass"), ((2, 2, 3), 2, "diffusion")]
    probs = [{"n": s, "p": p, "form": f, "vertices": FI.perturbed_cube_vertices(*s, seed=70 + k)}
             for k, (s, p, f) in enumerate(shapes)]
    bt = F().Batch(probs)
    bh = FI.uniform_vector(bt.N, seed=71)
    for k, pr in enumerate(probs):
        if pr["form"] == "diffusion":
            op = F().Operator(*pr["n"], pr["vertices"], pr["p"], form="diffusion")
            bh[bt.offsets[k] + op.boundary_dofs()] = 0.0
    b = torch.from_numpy(bh).cuda()
    x_ok, st_ok = bt.solve(b, rtol=1e-10)
    bad = b.clone()
    bad[int(bt.offsets[1]) + 1] = float("nan")
    x_bad, st = bt.solve(bad, rtol=1e-10, raise_on_noconv=False)
    assert st["status"] == fepa().ERR_NOCONV and st["converged"] == 2
    assert st["iterations"][1] <= 1
    for k in (0, 2):   # (the atomic scatter's summation order varies: iterations within 1)
        lo, hi = int(bt.offsets[k]), int(bt.offsets[k + 1])
        assert abs(int(st["iterations"][k]) - int(st_ok["iterations"][k])) <= 1
        assert torch.linalg.norm(x_bad[lo:hi] - x_ok[lo:hi]) <= 1e-9 * torch.linalg.norm(x_ok[lo:hi])
