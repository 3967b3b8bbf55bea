"""GPU parity of batched independent problems (fepa_batch_*): every problem of a batch
must match the oracle and its own solve run alone.

Tolerances are those of the single-problem tests: relative l2 <= 1e-12 for the FP64
action, CG iteration counts within 1 and solutions within 1e-9 at the 1e-10 stop.
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


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def small_mix(seed=0, count=10):
    rng = np.random.default_rng(seed)
    probs = []
    for i in range(count):
        p = int(rng.integers(1, 7))
        n = tuple(int(v) for v in rng.integers(1, 4 if p > 3 else 5, size=3))
        form = "mass" if i % 3 == 0 else "diffusion"
        probs.append({"n": n, "p": p, "form": form, "vertices": FI.perturbed_cube_vertices(*n, seed=100 + i)})
    return probs


def oracle_problem(pr):
    mesh = O.HexGridMesh(*pr["n"], pr["vertices"])
    return O.Problem(mesh, pr["p"], None, pr["form"], assemble=pr["p"] <= 5)


def rhs_for(probs, offsets, seed=7):
    """Random nodal right-hand sides, boundary rows zero for diffusion problems."""
    b = FI.uniform_vector(int(offsets[-1]), seed=seed)
    for i, pr in enumerate(probs):
        if pr["form"] == "diffusion":
            mesh = O.HexGridMesh(*pr["n"], pr["vertices"])
            b[offsets[i] + O.boundary_dofs(mesh, pr["p"])] = 0.0
    return b


def test_batch_layout_and_groups():
    probs = small_mix()
    bt = F().Batch(probs)
    sizes = [O.num_dofs(O.HexGridMesh(*pr["n"], pr["vertices"]), pr["p"]) for pr in probs]
    assert np.array_equal(np.diff(bt.offsets), sizes)
    assert bt.N == sum(sizes)
    assert bt.groups == len({(pr["p"], pr["form"]) for pr in probs})


@pytest.mark.parametrize("variant", [-1, 0, 1])
def test_batch_apply_matches_oracle(variant):
    """Both FP64 action kernels (DFMA, double-float) and the measured choice."""
    probs = small_mix(seed=1)
    bt = F().Batch(probs)
    bt.set_f64_variant(variant)
    x = FI.uniform_vector(bt.N, seed=3)
    y = bt.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    for i, pr in enumerate(probs):
        sl = slice(bt.offsets[i], bt.offsets[i + 1])
        op = oracle_problem(pr)
        assert rel(y[sl], op.apply(x[sl], constrained=True)) <= 1e-12, i


@pytest.mark.parametrize("variant", [0, 1])
def test_batch_solve_matches_oracle_and_alone(variant):
    probs = small_mix(seed=2, count=12)
    bt = F().Batch(probs)
    bt.set_f64_variant(variant)
    b = rhs_for(probs, bt.offsets)
    x, st = bt.solve(torch.from_numpy(b).cuda(), rtol=1e-10)
    x = x.cpu().numpy()
    assert st["converged"] == len(probs) and st["status"] == 0
    assert st["max_rel_residual"] <= 1e-10
    its = st["iterations"]
    assert st["max_iterations"] == its.max()
    for i, pr in enumerate(probs):
        sl = slice(bt.offsets[i], bt.offsets[i + 1])
        prob = oracle_problem(pr)
        xo, it_o, _ = prob.solve(b[sl], rtol=1e-10)
        assert abs(its[i] - it_o) <= 1, (i, its[i], it_o)
        assert rel(x[sl], xo) <= 1e-9, i
        # the same problem solved alone
        op = F().Operator(*pr["n"], pr["vertices"], pr["p"], form=pr["form"])
        if pr["form"] == "diffusion":
            op.set_essential(op.boundary_dofs())
        xa, sa = op.solve(torch.from_numpy(np.ascontiguousarray(b[sl])).cuda(), rtol=1e-10)
        assert abs(sa["iterations"] - its[i]) <= 1
        assert rel(x[sl], xa.cpu().numpy()) <= 1e-9


def test_batch_is_independent_of_its_mix():
    """A problem's result does not depend on which other problems share the batch."""
    probs = small_mix(seed=4, count=9)
    full = F().Batch(probs)
    b = rhs_for(probs, full.offsets)
    xf, sf = full.solve(torch.from_numpy(b).cuda(), rtol=1e-10)
    keep = [0, 3, 5, 8]
    sub = F().Batch([probs[i] for i in keep])
    bs = np.concatenate([b[full.offsets[i]:full.offsets[i + 1]] for i in keep])
    xs, ss = sub.solve(torch.from_numpy(bs).cuda(), rtol=1e-10)
    xf, xs = xf.cpu().numpy(), xs.cpu().numpy()
    for k, i in enumerate(keep):
        assert abs(int(sf["iterations"][i]) - int(ss["iterations"][k])) <= 1
        assert rel(xs[sub.offsets[k]:sub.offsets[k + 1]], xf[full.offsets[i]:full.offsets[i + 1]]) <= 1e-9


def test_batch_512_problem_mix_sampled():
    """512 independent problems (form mass/diffusion with probability 1/2, p uniform in
    1..6, elements per direction uniform in 2..24, seeded perturbed cubes, random nodal
    right-hand sides), FP64 Jacobi-PCG to 1e-10 in one graph-driven batch.  Sampled
    problems are checked against the same problem solved alone and, on sampled rows,
    against the oracle's residual."""
    mix = FI.problem_mix(512, seed=0)
    probs = [{"n": m["n"], "p": m["p"], "form": m["form"],
              "vertices": FI.perturbed_cube_vertices(*m["n"], seed=m["mesh_seed"])} for m in mix]
    bt = F().Batch(probs)
    b = rhs_for(probs, bt.offsets, seed=11)
    x, st = bt.solve(torch.from_numpy(b).cuda(), rtol=1e-10, maxit=20000)
    x = x.cpu().numpy()
    assert st["converged"] == 512 and st["max_rel_residual"] <= 1e-10
    rng = np.random.default_rng(5)
    for i in rng.choice(512, 6, replace=False):
        pr = probs[i]
        sl = slice(bt.offsets[i], bt.offsets[i + 1])
        op = F().Operator(*pr["n"], pr["vertices"], pr["p"], form=pr["form"])
        mesh = O.HexGridMesh(*pr["n"], pr["vertices"])
        ess = None
        if pr["form"] == "diffusion":
            ess = op.boundary_dofs()
            op.set_essential(ess)
        xa, sa = op.solve(torch.from_numpy(np.ascontiguousarray(b[sl])).cuda(), rtol=1e-10)
        assert abs(sa["iterations"] - int(st["iterations"][i])) <= 1
        assert rel(x[sl], xa.cpu().numpy()) <= 1e-9
        rows = rng.choice(op.N, min(op.N, 20), replace=False)
        Ax = O.action_rows(mesh, pr["p"], pr["p"] + 2, pr["form"], x[sl], rows,
                           ess=None if ess is None else ess.astype(np.int64))
        assert np.max(np.abs(b[sl][rows] - Ax)) <= 1e-10 * np.linalg.norm(b[sl])
