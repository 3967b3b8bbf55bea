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


@pytest.mark.parametrize("variant", [-1, 0, 1, 2])
def test_batch_apply_matches_oracle(variant):
    """The FP64 action kernels (DFMA, double-float in full- and half-size tiles) and the
    measured choice."""
    probs = small_mix(seed=1)
    bt = F().Batch(probs)
    bt.set_f64_variant(variant)
    x = FI.uniform_vector(bt.N, seed=3)
    y = bt.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    for i, pr in enumerate(probs):
        sl = slice(bt.offsets[i], bt.offsets[i + 1])
        op = oracle_problem(pr)
        assert rel(y[sl], op.apply(x[sl], constrained=True)) <= 1e-12, i


@pytest.mark.parametrize("variant", [0, 1, 2])
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


# ---------------------------------------------------------------------------
# Mixed-precision batched solve: FP64 refinement around batched FP32 Jacobi-PCG.
# The FP64 residual decides each problem's stop, so every solution is checked to the
# same 1e-10 residual and 1e-9 solution tolerance as the FP64 batch; FP32 iteration
# counts depend on the atomic summation order of the FP32 action and are compared
# loosely (within 10 % or 4 of the problem solved alone).
# ---------------------------------------------------------------------------
def test_batch_refined_matches_oracle_and_alone():
    probs = small_mix(seed=2, count=12)
    bt = F().Batch(probs)
    b = rhs_for(probs, bt.offsets)
    x, st = bt.solve_refined(torch.from_numpy(b).cuda(), rtol=1e-10)
    x = x.cpu().numpy()
    assert st["converged"] == len(probs) and st["status"] == 0
    assert st["max_rel_residual"] <= 1e-10 and st["outer_iterations"] >= 1
    its = st["iterations"]
    assert st["max_inner_iterations"] == its.max()
    sizes = np.diff(bt.offsets)
    assert st["dof_iterations"] == pytest.approx(float(np.dot(sizes, its)))
    for i, pr in enumerate(probs):
        sl = slice(bt.offsets[i], bt.offsets[i + 1])
        xo, _, _ = oracle_problem(pr).solve(b[sl], rtol=1e-12)
        assert rel(x[sl], xo) <= 1e-9, i
        op = F().Operator(*pr["n"], pr["vertices"], pr["p"], form=pr["form"])
        if pr["form"] == "diffusion":
            op.set_essential(op.boundary_dofs())
        xa, sa = op.solve_refined(torch.from_numpy(np.ascontiguousarray(b[sl])).cuda(), rtol=1e-10)
        assert abs(sa["inner_iterations"] - int(its[i])) <= max(4, 0.1 * sa["inner_iterations"]), i
        assert rel(x[sl], xa.cpu().numpy()) <= 1e-9, i


def test_batch_refined_skips_finished_problems():
    """A zero right-hand side and an exact initial guess finish before any FP32 step (no
    iterations); the others still converge, and repeated solves reuse the FP32 data."""
    probs = small_mix(seed=3, count=6)
    bt = F().Batch(probs)
    b = rhs_for(probs, bt.offsets, seed=9)
    b[bt.offsets[1]:bt.offsets[2]] = 0.0
    x_ref, _ = bt.solve(torch.from_numpy(b).cuda(), rtol=1e-12)
    x0 = torch.zeros(bt.N, dtype=torch.float64, device="cuda")
    sl4 = slice(int(bt.offsets[4]), int(bt.offsets[5]))
    x0[sl4] = x_ref[sl4]
    x, st = bt.solve_refined(torch.from_numpy(b).cuda(), x=x0, rtol=1e-10)
    its = st["iterations"]
    assert its[1] == 0 and its[4] == 0
    # the others iterate unless all their DOFs are on the boundary (b_i = 0 there too)
    live = [i for i in (0, 2, 3, 5) if np.any(b[bt.offsets[i]:bt.offsets[i + 1]] != 0.0)]
    assert len(live) >= 3 and all(its[i] > 0 for i in live)
    assert all(its[i] == 0 for i in (0, 2, 3, 5) if i not in live)
    assert st["converged"] == len(probs) and st["max_rel_residual"] <= 1e-10
    assert float(torch.abs(x[bt.offsets[1]:bt.offsets[2]]).max()) == 0.0
    x2, st2 = bt.solve_refined(torch.from_numpy(b).cuda(), rtol=1e-10)
    assert st2["converged"] == len(probs)
    assert rel(x2.cpu().numpy(), x_ref.cpu().numpy()) <= 1e-9


def test_batch_refined_noconv_and_arguments():
    probs = small_mix(seed=5, count=4)
    bt = F().Batch(probs)
    b = torch.from_numpy(rhs_for(probs, bt.offsets)).cuda()
    from paper_2402_15940_b300.fepa import ERR_NOCONV
    x, st = bt.solve_refined(b, rtol=1e-14, max_outer=1, inner_maxit=3, raise_on_noconv=False)
    assert st["status"] == ERR_NOCONV and st["converged"] < len(probs)
    assert st["outer_iterations"] == 1 and st["max_inner_iterations"] <= 3
    with pytest.raises(F().FepaError):
        bt.solve_refined(b, max_outer=1, inner_maxit=3, rtol=1e-14)
    for kw in ({"inner_rtol": 0.0}, {"inner_rtol": 1.0}, {"max_outer": 0}, {"inner_maxit": 0}, {"rtol": -1.0}):
        with pytest.raises(F().FepaError):
            bt.solve_refined(b, **kw)


def test_batch_refined_512_problem_mix_sampled():
    """The 512-problem mix of the FP64 batch test solved by batched mixed-precision
    refinement: every problem reaches 1e-10 on its FP64 residual; sampled problems match
    the FP64 batch solution and, on sampled rows, the oracle's residual."""
    mix = FI.problem_mix(512, seed=0)
    probs = [{"n": m["n"], "p": m["p"], "form": m["form"],
              "vertices": FI.perturbed_cube_vertices(*m["n"], seed=m["mesh_seed"])} for m in mix]
    bt = F().Batch(probs)
    b = rhs_for(probs, bt.offsets, seed=11)
    bd = torch.from_numpy(b).cuda()
    x, st = bt.solve_refined(bd, rtol=1e-10)
    assert st["converged"] == 512 and st["max_rel_residual"] <= 1e-10
    x64, _ = bt.solve(bd, rtol=1e-10, maxit=20000)
    x, x64 = x.cpu().numpy(), x64.cpu().numpy()
    rng = np.random.default_rng(6)
    for i in rng.choice(512, 6, replace=False):
        pr = probs[i]
        sl = slice(bt.offsets[i], bt.offsets[i + 1])
        assert rel(x[sl], x64[sl]) <= 1e-8, i
        mesh = O.HexGridMesh(*pr["n"], pr["vertices"])
        n_i = int(bt.offsets[i + 1] - bt.offsets[i])
        rows = rng.choice(n_i, min(n_i, 20), replace=False)
        ess = O.boundary_dofs(mesh, pr["p"]).astype(np.int64) if pr["form"] == "diffusion" else None
        Ax = O.action_rows(mesh, pr["p"], pr["p"] + 2, pr["form"], x[sl], rows, ess=ess)
        assert np.max(np.abs(b[sl][rows] - Ax)) <= 1e-10 * np.linalg.norm(b[sl])


# ---------------------------------------------------------------------------
# Batched reliable updates: one FP32 recurrence per problem with FP64 residual replacement.
# ---------------------------------------------------------------------------
def test_batch_reliable_matches_oracle_and_alone():
    probs = small_mix(seed=2, count=12)
    bt = F().Batch(probs)
    b = rhs_for(probs, bt.offsets)
    x, st = bt.solve_reliable(torch.from_numpy(b).cuda(), rtol=1e-10)
    x = x.cpu().numpy()
    assert st["converged"] == len(probs) and st["status"] == 0
    assert st["max_rel_residual"] <= 1e-10
    its = st["iterations"]
    assert st["max_inner_iterations"] == its.max()
    for i, pr in enumerate(probs):
        sl = slice(bt.offsets[i], bt.offsets[i + 1])
        xo, _, _ = oracle_problem(pr).solve(b[sl], rtol=1e-12)
        assert rel(x[sl], xo) <= 1e-9, i
        op = F().Operator(*pr["n"], pr["vertices"], pr["p"], form=pr["form"])
        if pr["form"] == "diffusion":
            op.set_essential(op.boundary_dofs())
        xa, sa = op.solve_reliable(torch.from_numpy(np.ascontiguousarray(b[sl])).cuda(), rtol=1e-10)
        # the batch replaces when every running problem has ended its segment, so a problem's
        # replacements (and FP32 count) can differ a little from its solve alone
        assert abs(sa["inner_iterations"] - int(its[i])) <= max(6, 0.15 * sa["inner_iterations"]), i
        assert rel(x[sl], xa.cpu().numpy()) <= 1e-9, i


def test_batch_reliable_finished_problems_and_errors():
    probs = small_mix(seed=3, count=6)
    bt = F().Batch(probs)
    b = rhs_for(probs, bt.offsets, seed=9)
    b[bt.offsets[1]:bt.offsets[2]] = 0.0
    bd = torch.from_numpy(b).cuda()
    x, st = bt.solve_reliable(bd, rtol=1e-10)
    assert st["iterations"][1] == 0 and st["converged"] == len(probs)
    assert float(torch.abs(x[bt.offsets[1]:bt.offsets[2]]).max()) == 0.0
    from paper_2402_15940_b300.fepa import ERR_NOCONV
    x, st = bt.solve_reliable(bd, rtol=1e-14, maxit=5, raise_on_noconv=False)
    assert st["status"] == ERR_NOCONV and st["max_inner_iterations"] <= 5 + 1
    for kw in ({"delta": 0.0}, {"delta": 1.0}, {"maxit": 0}, {"rtol": -1.0}):
        with pytest.raises(F().FepaError):
            bt.solve_reliable(bd, **kw)


def test_batch_reliable_512_problem_mix_sampled():
    mix = FI.problem_mix(512, seed=0)
    probs = [{"n": m["n"], "p": m["p"], "form": m["form"],
              "vertices": FI.perturbed_cube_vertices(*m["n"], seed=m["mesh_seed"])} for m in mix]
    bt = F().Batch(probs)
    b = rhs_for(probs, bt.offsets, seed=11)
    bd = torch.from_numpy(b).cuda()
    x, st = bt.solve_reliable(bd, rtol=1e-10)
    assert st["converged"] == 512 and st["max_rel_residual"] <= 1e-10
    x64, _ = bt.solve(bd, rtol=1e-10, maxit=20000)
    x, x64 = x.cpu().numpy(), x64.cpu().numpy()
    rng = np.random.default_rng(7)
    for i in rng.choice(512, 6, replace=False):
        sl = slice(bt.offsets[i], bt.offsets[i + 1])
        assert rel(x[sl], x64[sl]) <= 1e-8, i


def test_batch_records_the_autotuners_picks_per_group():
    """After an FP64 solve every group has an FP64 variant picked (0-2), after a refined solve an
    FP32 tile shape (variant 1 or 2's elements per block); the groups list every (p, form) once."""
    probs = small_mix(seed=5, count=10)
    bt = F().Batch(probs)
    info = bt.group_info()
    assert len(info) == bt.groups == len({(pr["p"], pr["form"]) for pr in probs})
    assert {(g["p"], g["form"]) for g in info} == {(pr["p"], pr["form"]) for pr in probs}
    assert all(g["f64_variant"] == -1 and g["f32_elements_per_block"] == 0 for g in info)
    b = rhs_for(probs, bt.offsets)
    bt.solve(torch.from_numpy(b).cuda(), rtol=1e-10)
    bt.solve_refined(torch.from_numpy(b).cuda(), rtol=1e-10)
    for g, e in zip(bt.group_info(), info):
        assert g["elements"] == e["elements"] > 0
        assert g["f64_variant"] in (0, 1, 2)
        q = g["p"] + 2
        ne0 = max(1, 256 // (q * q))
        assert g["f32_elements_per_block"] in (ne0, max(1, ne0 // 2)), g
