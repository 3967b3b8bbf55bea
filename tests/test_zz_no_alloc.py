"""The allocation-free CG entry point, fepa_cg_solve_noalloc.

Some callers cannot allocate device memory once they are running: a program whose
framework has already reserved the whole GPU for its own caching pool (cudaMalloc
would fail), or a latency-bound loop that must not call cudaMalloc/cudaFree because
they can synchronise the device.  For them the library keeps the CG work vectors in
one static device array of bounded size.  These tests call that entry point through
the C ABI and check it against the ordinary fepa_cg_solve, twice in a row (the array
keeps the previous call's contents), and check that it rejects operators larger than
its limit and leaves free device memory unchanged.
"""
import ctypes
import math

import numpy as np
import pytest

import fem_inputs as FI

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SOLVE_TOL = 1e-9   # the solution tolerance of the solver parity tests


def _ops():
    import paper_2402_15940_b300 as F
    from paper_2402_15940_b300 import fepa
    return F, fepa


def noalloc_solve(op, b, x, rtol, maxit, precond):
    F, fepa = _ops()
    lib = fepa.load_library()
    st = fepa.CgStats()
    torch.cuda.synchronize()
    rc = lib.fepa_cg_solve_noalloc(op._h, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                   float(rtol), int(maxit), int(precond), ctypes.byref(st))
    torch.cuda.synchronize()
    return rc, st.as_dict()


def rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def _problem(form, p, shape, seed):
    F, _ = _ops()
    op = F.Operator(*shape, FI.perturbed_cube_vertices(*shape, seed=seed), p, form=form)
    if form == "diffusion":
        op.set_essential(op.boundary_dofs())
        b = op.rhs_sine(3 * math.pi ** 2)
    else:
        b = torch.from_numpy(FI.uniform_vector(op.N, seed=seed)).cuda()
    return op, b


@pytest.mark.parametrize("form,p,shape,precond", [("diffusion", 3, (4, 4, 4), 1), ("mass", 2, (5, 4, 3), 0),
                                                  ("diffusion", 5, (3, 2, 3), 1)])
def test_noalloc_matches_cg_solve_twice(form, p, shape, precond):
    op, b = _problem(form, p, shape, seed=p)
    x_ref, st_ref = op.solve(b, rtol=1e-10, maxit=2000, precond=precond)
    for _ in range(2):   # the second call finds the array holding the first call's data
        x = torch.zeros(op.N, dtype=torch.float64, device="cuda")
        rc, st = noalloc_solve(op, b, x, 1e-10, 2000, precond)
        assert rc == 0, _ops()[1].load_library().fepa_last_error()
        assert st["status"] == 0 and st["rel_residual"] <= 1e-10
        assert abs(st["iterations"] - st_ref["iterations"]) <= 1
        assert rel(x, x_ref) <= SOLVE_TOL


def test_noalloc_rejects_large_operator():
    F, fepa = _ops()
    shape = (64, 64, 32)   # p = 1: 65*65*33 = 139,425 DOFs > FEPA_NOALLOC_MAX_DOFS
    op = F.Operator(*shape, FI.perturbed_cube_vertices(*shape, seed=0), 1, form="mass")
    assert op.N > fepa.NOALLOC_MAX_DOFS
    b = torch.ones(op.N, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    rc, _ = noalloc_solve(op, b, x, 1e-10, 10, 1)
    assert rc == fepa.ERR_ARG
    assert b"at most 131072 DOFs" in fepa.load_library().fepa_last_error()
    assert float(x.abs().max()) == 0.0   # nothing ran


def test_noalloc_leaves_free_memory_unchanged():
    op, b = _problem("diffusion", 2, (6, 5, 4), seed=9)
    x = torch.zeros(op.N, dtype=torch.float64, device="cuda")
    rc, _ = noalloc_solve(op, b, x, 1e-10, 2000, 1)    # first call on this device sets up
    assert rc == 0
    op2, b2 = _problem("diffusion", 4, (3, 3, 3), seed=10)
    x2 = torch.zeros(op2.N, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    rc, st = noalloc_solve(op2, b2, x2, 1e-10, 2000, 1)
    free1, _ = torch.cuda.mem_get_info()
    assert rc == 0 and st["status"] == 0
    assert free1 == free0
