"""Full-size sampled parity of the FP64-accurate (double-float) and FP32 operator actions at the
high orders of the operator sweep (about 1.4e7 DOFs each) and at the second size of the
mixed-precision configuration (p = 6 on 32^3): rows of y = A x computed one by one by the
oracle from the elements that touch them.  At these orders both kernels run their packed
forms (even/odd stage 3 over mirrored point pairs in the double-float action, paired outputs
in the FP32 contractions), so these check the launch shapes the benchmark times, at the sizes
it times them.

Tolerances: the FP64-accurate action 1e-12 of max |y| (the FP64 action's bound); the FP32
action 1e-5 of max |y| against the oracle applied to the same FP32 input (the bound derived in
test_gpu_mixed).
"""
import numpy as np
import pytest

import fem_inputs as FI
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def F():
    import paper_2402_15940_b300 as mod
    return mod


@pytest.mark.parametrize("form,p,n", [("diffusion", 5, 48), ("diffusion", 6, 32), ("diffusion", 7, 34),
                                      ("diffusion", 8, 30), ("mass", 6, 40), ("mass", 8, 30)])
def test_actions_full_size_sampled(form, p, n):
    verts = FI.perturbed_cube_vertices(n, n, n, seed=p)
    op = F().Operator(n, n, n, verts, p, form=form)
    mesh = O.HexGridMesh(n, n, n, verts)
    ess = op.boundary_dofs() if form == "diffusion" else np.zeros(0, dtype=np.int32)
    if len(ess):
        op.set_essential(ess)
    ess64 = ess.astype(np.int64) if len(ess) else None
    x = FI.uniform_vector(op.N, seed=p + 1)
    rng = np.random.default_rng(100 + p)
    rows = np.concatenate([rng.choice(op.N, 40, replace=False), [0, op.N - 1, op.N // 2]])
    if len(ess):
        rows = np.concatenate([rows, ess[rng.choice(len(ess), 6, replace=False)]])
    # FP64-accurate action (the double-float kernel, forced)
    op.set_f64_variant(1)
    y = op.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = O.action_rows(mesh, p, p + 2, form, x, rows, ess=ess64)
    assert np.max(np.abs(y[rows] - ref)) <= 1e-12 * np.max(np.abs(ref))
    # FP32 action (autotuned variant) on the same x rounded to FP32
    x32 = x.astype(np.float32)
    y32 = op.apply_f32(torch.from_numpy(x32).cuda()).cpu().numpy()
    ref32 = O.action_rows(mesh, p, p + 2, form, x32.astype(np.float64), rows, ess=ess64)
    assert np.max(np.abs(y32[rows] - ref32)) <= 1e-5 * np.max(np.abs(ref32))


@pytest.mark.parametrize("form,p,n", [("diffusion", 1, 160), ("diffusion", 2, 100), ("diffusion", 3, 64),
                                      ("mass", 2, 100)])
def test_half_block_double_float_full_size_sampled(form, p, n):
    """The double-float action in half-size blocks (FP64 variant 2, the autotuner's pick at these
    orders on large meshes, 4-8e6 DOFs here), sampled rows against the oracle, and against the
    full-size blocks (the same per-element arithmetic; only the atomic summation order differs)."""
    verts = FI.perturbed_cube_vertices(n, n, n, seed=p + 20)
    op = F().Operator(n, n, n, verts, p, form=form)
    mesh = O.HexGridMesh(n, n, n, verts)
    ess = op.boundary_dofs() if form == "diffusion" else np.zeros(0, dtype=np.int32)
    if len(ess):
        op.set_essential(ess)
    ess64 = ess.astype(np.int64) if len(ess) else None
    x = FI.uniform_vector(op.N, seed=p + 21)
    rng = np.random.default_rng(200 + p)
    rows = np.concatenate([rng.choice(op.N, 40, replace=False), [0, op.N - 1, op.N // 2]])
    xd = torch.from_numpy(x).cuda()
    op.set_f64_variant(2)
    y2 = op.apply(xd).cpu().numpy()
    ref = O.action_rows(mesh, p, p + 2, form, x, rows, ess=ess64)
    assert np.max(np.abs(y2[rows] - ref)) <= 1e-12 * np.max(np.abs(ref))
    op.set_f64_variant(1)
    y1 = op.apply(xd).cpu().numpy()
    assert np.max(np.abs(y2 - y1)) <= 1e-14 * np.max(np.abs(y1))
