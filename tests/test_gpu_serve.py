"""GPU tests of resumable solves and of the continuous-batching server: every result
is the same alone and in the mix (iteration counts within 1, solutions within 1e-9,
the tolerance of the solver parity tests), and matches the oracle."""
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


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def make(n, p, form, seed):
    op = F().Operator(*n, FI.perturbed_cube_vertices(*n, seed=seed), p, form=form)
    if form == "diffusion":
        op.set_essential(op.boundary_dofs())
        b = op.rhs_sine(3 * math.pi ** 2)
    else:
        b = op.rhs_sine(1.0)
    return op, b


@pytest.mark.parametrize("kind", ["cg", "refined"])
@pytest.mark.parametrize("step", [1, 7, 100000])
def test_resumable_solve_equals_one_shot(kind, step):
    op, b = make((4, 3, 4), 3, "diffusion", seed=2)
    x1, s1 = (op.solve(b, rtol=1e-10) if kind == "cg" else op.solve_refined(b, rtol=1e-10))
    x2 = torch.zeros_like(b)
    op.solver_start(b, x2, kind=kind, rtol=1e-10)
    st = None
    for _ in range(100000):
        op.solver_advance(step)
        st = op.solver_poll(blocking=True)
        if st["done"]:
            break
    assert st["done"] and st["status"] == 0 and st["rel_residual"] <= 1e-10
    key = "iterations" if kind == "cg" else "inner_iterations"
    # FP64 CG is reproducible to one iteration; the FP32 inner counts may move by a few
    # (the FP32 scatter's atomic summation order varies from run to run)
    assert abs(st["iterations"] - s1[key]) <= (1 if kind == "cg" else max(4, 0.1 * s1[key]))
    assert rel(x2.cpu().numpy(), x1.cpu().numpy()) <= 1e-9


def test_nonblocking_poll_reports_busy_or_state():
    op, b = make((6, 6, 6), 4, "diffusion", seed=3)
    x = torch.zeros_like(b)
    op.solver_start(b, x, kind="cg", rtol=1e-10)
    seen_busy = False
    for _ in range(1000000):
        op.solver_advance(5)
        st = op.solver_poll(blocking=False)
        while st is None:
            seen_busy = True
            st = op.solver_poll(blocking=False)
        if st["done"]:
            break
    assert st["done"] and st["status"] == 0
    assert seen_busy or st["iterations"] > 0


@pytest.mark.parametrize("async_start", [False, True])
def test_server_results_same_alone_and_in_the_mix(async_start):
    from paper_2402_15940_b300.serve import GpuExecutor, Request, Server, poisson_arrivals
    specs = [("diffusion", 2, (4, 4, 4), "fp64"), ("mass", 3, (3, 3, 3), "mixed"), ("diffusion", 4, (3, 3, 2), "mixed"),
             ("diffusion", 1, (9, 8, 7), "fp64"), ("mass", 5, (2, 2, 2), "fp64"), ("diffusion", 6, (2, 2, 3), "mixed"),
             ("diffusion", 3, (5, 5, 5), "fp64"), ("mass", 2, (6, 5, 4), "mixed")]
    reqs = [Request(rid=i, form=f, p=p, n=n, mesh_seed=50 + i, precision=pr) for i, (f, p, n, pr) in enumerate(specs)]
    poisson_arrivals(reqs, rate=500.0, seed=1)
    vf = lambda n, seed: FI.perturbed_cube_vertices(*n, seed=seed)  # noqa: E731
    make((2, 2, 2), 1, "mass", 0)   # the library's one-time set-up happens before the memory checks
    srv = Server(GpuExecutor(vf, async_start=async_start), hbm_budget=2e9, tick_iters=4, keep_results=True,
                 policy="sjf" if async_start else "fifo")
    out = srv.run(reqs)
    assert len(out) == len(reqs) and all(o.status == 0 for o in out)
    assert srv.max_concurrent >= 2
    for o, r in zip(out, reqs):
        op, b = make(r.n, r.p, r.form, r.mesh_seed)
        if r.precision == "fp64":
            xa, sa = op.solve(b, rtol=1e-10)
            assert abs(sa["iterations"] - o.iterations) <= 1
        else:
            xa, sa = op.solve_refined(b, rtol=1e-10)
            # the FP32 scatter's atomic summation order varies from run to run, so the inner
            # FP32 iteration counts may move by a few; the solutions are compared below
            assert abs(sa["inner_iterations"] - o.iterations) <= max(4, 0.1 * sa["inner_iterations"])
        assert rel(o.result, xa.cpu().numpy()) <= 1e-9, r
        # and the oracle's tight solution of the same problem
        mesh = O.HexGridMesh(*r.n, FI.perturbed_cube_vertices(*r.n, seed=r.mesh_seed))
        prob = O.Problem(mesh, r.p, None, r.form, assemble=r.p <= 5)
        xo, _, _ = prob.solve(prob.sine_rhs(), rtol=1e-13)
        assert rel(o.result, xo) <= 1e-8
    rep = srv.report()
    assert rep["completed"] == len(reqs) and rep["p99_latency_s"] >= rep["p50_latency_s"] > 0
    # the admission estimate bounds the device memory each request actually took
    chk = rep["device_bytes_check"]
    if not async_start:
        assert chk["requests"] == len(reqs) and chk["max_measured_over_estimate"] <= 1.0, chk


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("step", [1, 3, 40])
def test_resumable_multigrid_solve_equals_one_shot(precision, step):
    """fepa_mg_solver_start/advance/poll reach fepa_mg_solve's iterate: the same iteration count
    and solution, also when an advance enqueues iterations past the stopping test (step 40)."""
    op, b = make((4, 4, 3), 4, "diffusion", seed=7)
    mg = F().Multigrid(op, smooth_degree=2, coarse_degree=24, precision=precision)
    x1, s1 = mg.solve(b, rtol=1e-10)
    x2 = torch.zeros_like(b)
    mg.solver_start(b, x2, rtol=1e-10)
    st = None
    for _ in range(1000):
        mg.solver_advance(step)
        st = mg.solver_poll(blocking=True)
        if st["done"]:
            break
    assert st["done"] and st["status"] == 0 and st["rel_residual"] <= 1e-10
    assert abs(st["iterations"] - s1["iterations"]) <= (0 if precision == "fp64" else 1)
    assert rel(x2.cpu().numpy(), x1.cpu().numpy()) <= 1e-9
    # a second solve on the same hierarchy starts from the caller's x again; while it runs the
    # hierarchy cannot be moved nor a second solve started
    x3 = torch.zeros_like(b)
    mg.solver_start(b, x3, rtol=1e-10)
    with pytest.raises(F().FepaError):
        mg.update()
    with pytest.raises(F().FepaError):
        mg.solver_start(b, torch.zeros_like(b), rtol=1e-10)
    while not mg.solver_poll(blocking=True)["done"]:
        mg.solver_advance(2)
    assert rel(x3.cpu().numpy(), x1.cpu().numpy()) <= 1e-9
    mg.close()


def test_server_with_multigrid_policy_same_alone_and_in_the_mix():
    """solver="auto": the diffusion requests above the threshold run multigrid-preconditioned CG
    (FP64 or FP32 V-cycle) beside Jacobi requests; each result equals the same solve run alone
    and the oracle's, and the admission estimate bounds each request's device memory."""
    from paper_2402_15940_b300.serve import GpuExecutor, Request, Server, poisson_arrivals
    specs = [("diffusion", 4, (4, 4, 3), "fp64"), ("mass", 3, (3, 3, 3), "mixed"), ("diffusion", 2, (6, 6, 5), "mixed"),
             ("diffusion", 1, (3, 3, 3), "fp64"), ("diffusion", 6, (2, 2, 3), "fp64"), ("diffusion", 3, (5, 4, 4), "mixed")]
    reqs = [Request(rid=i, form=f, p=p, n=n, mesh_seed=70 + i, precision=pr) for i, (f, p, n, pr) in enumerate(specs)]
    poisson_arrivals(reqs, rate=500.0, seed=2)
    vf = lambda n, seed: FI.perturbed_cube_vertices(*n, seed=seed)  # noqa: E731
    make((2, 2, 2), 1, "mass", 0)   # the library's one-time set-up happens before the memory checks
    srv = Server(GpuExecutor(vf), hbm_budget=4e9, tick_iters=4, keep_results=True, solver="auto", pmg_min_dofs=1000)
    out = srv.run(reqs)
    assert len(out) == len(reqs) and all(o.status == 0 for o in out)
    assert [r.solver for r in reqs] == ["pmg", "jacobi", "pmg", "jacobi", "pmg", "pmg"]
    for o, r in zip(out, reqs):
        op, b = make(r.n, r.p, r.form, r.mesh_seed)
        if r.solver == "pmg":
            mg = F().Multigrid(op, smooth_degree=2, coarse_degree=24,
                               precision="fp32" if r.precision == "mixed" else "fp64")
            xa, sa = mg.solve(b, rtol=1e-10)
            assert abs(sa["iterations"] - o.iterations) <= 1
            mg.close()
        elif r.precision == "fp64":
            xa, sa = op.solve(b, rtol=1e-10)
            assert abs(sa["iterations"] - o.iterations) <= 1
        else:
            xa, sa = op.solve_refined(b, rtol=1e-10)
        assert rel(o.result, xa.cpu().numpy()) <= 1e-9, r
        mesh = O.HexGridMesh(*r.n, FI.perturbed_cube_vertices(*r.n, seed=r.mesh_seed))
        prob = O.Problem(mesh, r.p, None, r.form, assemble=r.p <= 5)
        xo, _, _ = prob.solve(prob.sine_rhs(), rtol=1e-13)
        assert rel(o.result, xo) <= 1e-8
    rep = srv.report()
    assert rep["pmg_requests"] == 4
    chk = rep["device_bytes_check"]
    assert chk["requests"] == len(reqs) and chk["max_measured_over_estimate"] <= 1.0, chk
