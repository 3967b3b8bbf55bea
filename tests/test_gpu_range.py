"""Exponent range of the FP64-accurate double-float arithmetic.

A double-float value (hi + lo, two binary32 words) keeps ~48 bits only while its low word and
the error terms of its products are normal floats.  The double-float action finds the largest
|x| of each block as it gathers, and where that or its products with D would leave the safe
range it re-gathers x times an exact power of two and scales the element results back, so
inputs anywhere in the FP64 range keep the 1e-12 contract.  The sine load vector takes its
amplitude as m 2^k the same way.  The set-up (geometry, D) is checked per element instead: an
element outside the double-float geometry's range (extent below 2^-20, coordinates above 2^20
or above 2^10 times the extent) makes creation return FEPA_ERR_UNSUPPORTED rather than a less
accurate D."""
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


@pytest.mark.parametrize("scale", [1e-33, 1e-25, 1.0, 1e25, 1e33])
@pytest.mark.parametrize("form,p", [("diffusion", 4), ("mass", 4), ("diffusion", 2), ("mass", 7)])
def test_double_float_action_at_any_scale(form, p, scale):
    shape = (4, 3, 3) if p < 6 else (2, 2, 1)
    verts = FI.perturbed_cube_vertices(*shape, seed=80 + p)
    op = F().Operator(*shape, verts, p, form=form)
    mesh = O.HexGridMesh(*shape, verts)
    ess = O.boundary_dofs(mesh, p) if form == "diffusion" else None
    if ess is not None:
        op.set_essential(ess.astype(np.int32))
    x = FI.uniform_vector(op.N, seed=81) * scale
    ya = O.action_elementwise(mesh, p, p + 2, form, x, ess=ess)
    for v in (1, 0):            # double-float, then the DFMA kernel as a second witness
        op.set_f64_variant(v)
        y = op.apply(torch.from_numpy(x).cuda()).cpu().numpy()
        assert rel(y, ya) <= 1e-12, (v, rel(y, ya))


@pytest.mark.parametrize("scale", [1e-30, 1e30])
def test_solve_of_a_scaled_problem(scale):
    shape, p = (4, 4, 3), 3
    verts = FI.perturbed_cube_vertices(*shape, seed=82)
    op = F().Operator(*shape, verts, p, form="diffusion")
    op.set_essential(op.boundary_dofs())
    b1 = op.rhs_sine(3 * math.pi ** 2)
    bs = op.rhs_sine(3 * math.pi ** 2 * scale)
    assert rel(bs.cpu().numpy(), scale * b1.cpu().numpy()) <= 1e-14
    x1, s1 = op.solve(b1, rtol=1e-10)
    xs, ss = op.solve(bs, rtol=1e-10)
    assert abs(s1["iterations"] - ss["iterations"]) <= 1
    assert rel(xs.cpu().numpy(), scale * x1.cpu().numpy()) <= 1e-9
    xr, sr = op.solve_refined(bs, rtol=1e-10)
    assert sr["status"] == 0 and rel(xr.cpu().numpy(), scale * x1.cpu().numpy()) <= 1e-9


def test_mesh_outside_double_float_range_is_refused():
    from paper_2402_15940_b300 import fepa
    shape = (3, 3, 3)
    verts = FI.perturbed_cube_vertices(*shape, seed=83)
    for bad in (verts + np.array([1.0e4, 0.0, 0.0]),     # coordinates ~3e4 times the extent
                verts * 1e-7,                           # extent below 2^-20
                verts * 1e7):                           # coordinates above 2^20
        with pytest.raises(fepa.FepaError) as ei:
            F().Operator(*shape, bad, 2, form="diffusion")
        assert ei.value.code == fepa.ERR_UNSUPPORTED
    # inside the range: a shifted and rescaled mesh keeps D to 1e-12 against the oracle
    ok = verts * 2.0 ** -12 + np.array([3.0e-3, -1.0e-3, 2.0e-3])
    op = F().Operator(*shape, ok, 3, form="diffusion")
    F_o = O.qp_factors(O.HexGridMesh(*shape, ok).element_corners(), O.rule(3, 5), O.DIFFUSION)
    comps = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    Do = np.stack([F_o[..., a, b] for a, b in comps], axis=1)
    assert rel(op.qdata().cpu().numpy(), Do) <= 1e-12
    # and moving a valid op's vertices out of range is refused the same way
    with pytest.raises(fepa.FepaError) as ei:
        op.set_vertices(verts * 1e-7)
    assert ei.value.code == fepa.ERR_UNSUPPORTED
