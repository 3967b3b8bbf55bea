"""Pins for the CPU oracle: closed forms, invariants, brute force and convergence.

Every check here is fixed by the mathematics of the method (the paper prints no
worked example for this path), and each is chosen so that a plausible mistake in
the oracle (a dropped term, a transposed Jacobian, a wrong index) fails one.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

import fem_inputs as FI
import oracle as O

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms_1d.json")))


def _num(s):
    return float(eval(s, {"sqrt": math.sqrt}))


def perturbed(nx, ny, nz, seed=0):
    return O.HexGridMesh(nx, ny, nz, FI.perturbed_cube_vertices(nx, ny, nz, seed=seed))


def unperturbed(nx, ny, nz):
    return O.HexGridMesh(nx, ny, nz, FI.perturbed_cube_vertices(nx, ny, nz, seed=0, amp=0.0))


# ---------------------------------------------------------------- 1D rules

@pytest.mark.parametrize("q", [2, 3])
def test_gauss_closed_form(q):
    pts, wts = O.gauss_legendre(q)
    g = GOLD["gauss_legendre_on_m1_1"][str(q)]
    np.testing.assert_allclose(2 * pts - 1, [_num(s) for s in g["points"]], atol=1e-15)
    np.testing.assert_allclose(2 * wts, [_num(s) for s in g["weights"]], atol=1e-15)


@pytest.mark.parametrize("q", range(1, 12))
def test_gauss_exactness(q):
    pts, wts = O.gauss_legendre(q)
    assert abs(wts.sum() - 1) < 1e-14
    for k in range(2 * q):
        assert abs(wts @ pts ** k - 1.0 / (k + 1)) < 1e-14, k
    # degree 2q is no longer exact: the remainder of the q-point rule on [0,1] for t^(2q) is
    # (q!)^4 / ((2q+1) ((2q)!)^2) (standard Gauss error term with f^(2q) = (2q)!)
    if q <= 7:
        err = 1.0 / (2 * q + 1) - wts @ pts ** (2 * q)
        expect = math.factorial(q) ** 4 / ((2 * q + 1) * math.factorial(2 * q) ** 2)
        assert abs(err / expect - 1) < 1e-3


@pytest.mark.parametrize("p", [2, 3, 4])
def test_gll_closed_form(p):
    t = O.gll_points(p)
    assert t[0] == 0.0 and t[-1] == 1.0
    np.testing.assert_allclose(2 * t[1:-1] - 1, [_num(s) for s in GOLD["gll_interior_on_m1_1"][str(p)]], atol=1e-15)


@pytest.mark.parametrize("p", range(1, 9))
def test_gll_lobatto_rule_exact(p):
    # With weights 2/(p(p+1) P_p(t)^2) the GLL nodes integrate degree 2p-1 exactly on [-1,1];
    # P_p is evaluated by numpy's Legendre series, independent of the oracle's recurrence.
    t = 2 * O.gll_points(p) - 1
    Pp = np.polynomial.legendre.legval(t, [0] * p + [1])
    w = 2.0 / (p * (p + 1) * Pp ** 2)
    assert np.all(np.diff(t) > 0)
    np.testing.assert_allclose(t, -t[::-1], atol=1e-15)
    for k in range(2 * p):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(w @ t ** k - exact) < 1e-13, (p, k)


@pytest.mark.parametrize("p", range(1, 9))
def test_lagrange_identities(p):
    nodes = O.gll_points(p)
    V, dV = O.lagrange(nodes, nodes)
    np.testing.assert_allclose(V, np.eye(p + 1), atol=1e-14)
    t = np.linspace(-0.2, 1.3, 17)
    V, dV = O.lagrange(nodes, t)
    for k in range(p + 1):   # reproduces t^k and its derivative exactly
        np.testing.assert_allclose(V @ nodes ** k, t ** k, atol=1e-11)
        np.testing.assert_allclose(dV @ nodes ** k, k * t ** max(k - 1, 0) if k else 0 * t, atol=1e-10)


# ---------------------------------------------------------------- closed forms in 3D

def _closed_1d(p, n, h):
    g = GOLD["element_matrices_unit_interval"]["p%d" % p]
    Ke = np.array(g["stiffness"], float) * _num(g["stiffness_scale"]) / h
    Me = np.array(g["mass"], float) * _num(g["mass_scale"]) * h
    N = p * n + 1
    K, M = np.zeros((N, N)), np.zeros((N, N))
    for e in range(n):
        s = slice(p * e, p * e + p + 1)
        K[s, s] += Ke
        M[s, s] += Me
    return K, M


@pytest.mark.parametrize("p", [1, 2])
def test_unperturbed_kronecker_closed_form(p):
    nx, ny, nz = 3, 2, 2
    mesh = unperturbed(nx, ny, nz)
    Kx, Mx = _closed_1d(p, nx, 1.0 / nx)
    Ky, My = _closed_1d(p, ny, 1.0 / ny)
    Kz, Mz = _closed_1d(p, nz, 1.0 / nz)
    # global index x fastest -> kron(z, kron(y, x))
    M3 = np.kron(Mz, np.kron(My, Mx))
    K3 = np.kron(Mz, np.kron(My, Kx)) + np.kron(Mz, np.kron(Ky, Mx)) + np.kron(Kz, np.kron(My, Mx))
    np.testing.assert_allclose(O.assemble_csr(mesh, p, p + 2, O.MASS).toarray(), M3, atol=1e-15)
    np.testing.assert_allclose(O.assemble_csr(mesh, p, p + 2, O.DIFFUSION).toarray(), K3, atol=1e-13)


# ---------------------------------------------------------------- invariants on perturbed meshes

@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_volume_and_constant_nullspace(p):
    mesh = perturbed(2, 3, 2, seed=p)
    M = O.assemble_csr(mesh, p, p + 2, O.MASS)
    K = O.assemble_csr(mesh, p, p + 2, O.DIFFUSION)
    one = np.ones(M.shape[0])
    assert abs(one @ (M @ one) - 1.0) < 1e-14           # 1^T M 1 = |Omega| = 1
    assert np.abs(K @ one).max() < 1e-12                 # K 1 = 0
    assert abs((M - M.T)).max() < 1e-16 and abs((K - K.T)).max() < 1e-13


@pytest.mark.parametrize("p", [1, 2, 3])
def test_stiffness_psd_one_dim_nullspace(p):
    mesh = perturbed(2, 2, 2, seed=7)
    K = O.assemble_csr(mesh, p, p + 2, O.DIFFUSION).toarray()
    ev = np.linalg.eigvalsh(K)
    assert ev[0] > -1e-12 and abs(ev[0]) < 1e-12
    assert ev[1] > 1e-3
    M = O.assemble_csr(mesh, p, p + 2, O.MASS).toarray()
    assert np.linalg.eigvalsh(M)[0] > 0


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_mass_quadrature_exact(p):
    # phi_a phi_b detJ has degree <= 2p+2 per variable: q = p+2 is exact, so more points change nothing
    mesh = perturbed(2, 1, 2, seed=3)
    A = O.assemble_csr(mesh, p, p + 2, O.MASS).toarray()
    B = O.assemble_csr(mesh, p, p + 6, O.MASS).toarray()
    np.testing.assert_allclose(A, B, atol=1e-14 * np.abs(A).max())


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_patch_test_linear(p):
    # For a linear field u, adj(J)^T grad-hat(phi) . a has degree <= p+2 per variable, so the
    # quadrature is exact and interior rows of K u_I vanish.
    mesh = perturbed(3, 2, 2, seed=11)
    K = O.assemble_csr(mesh, p, p + 2, O.DIFFUSION)
    xyz = O.node_coords(mesh, p)
    u = 0.3 + 1.1 * xyz[:, 0] - 0.7 * xyz[:, 1] + 2.3 * xyz[:, 2]
    interior = np.setdiff1d(np.arange(len(u)), O.boundary_dofs(mesh, p))
    assert np.abs((K @ u)[interior]).max() < 1e-12


@pytest.mark.parametrize("p", [1, 2, 3])
def test_dirichlet_solve_reproduces_linear(p):
    mesh = perturbed(2, 3, 2, seed=5)
    prob = O.Problem(mesh, p, None, O.DIFFUSION)
    xyz = O.node_coords(mesh, p)
    u = 0.3 + 1.1 * xyz[:, 0] - 0.7 * xyz[:, 1] + 2.3 * xyz[:, 2]
    ess = prob.ess
    b = -(prob.A @ np.where(np.isin(np.arange(len(u)), ess), u, 0.0))   # lift of the boundary data
    b[ess] = u[ess]
    x, it, res = prob.solve(b, rtol=1e-14)
    np.testing.assert_allclose(x, u, atol=1e-11)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_mass_projection_reproduces_polynomials(p):
    # u of total degree <= p in physical coordinates is in Q_p after the trilinear map, and
    # the load-vector quadrature is exact, so M c = b(u) returns the nodal values of u.
    mesh = perturbed(2, 2, 3, seed=13)
    M = O.assemble_csr(mesh, p, p + 2, O.MASS).toarray()
    def u(x):
        X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
        return (0.5 + X - 2 * Y + 0.25 * Z) ** p + (X * Y if p >= 2 else 0.0)
    b = O.rhs_from_qp(mesh, p, p + 2, u(O.qp_coords(mesh, p, p + 2)))
    c = sla.solve(M, b, assume_a="pos")
    np.testing.assert_allclose(c, u(O.node_coords(mesh, p)), atol=1e-10)


# ---------------------------------------------------------------- brute force and internal consistency

@pytest.mark.parametrize("form", [O.MASS, O.DIFFUSION])
@pytest.mark.parametrize("p,shape", [(1, (2, 2, 2)), (2, (2, 1, 2)), (3, (1, 2, 1))])
def test_bruteforce_equals_csr(form, p, shape):
    mesh = perturbed(*shape, seed=17)
    A = O.assemble_csr(mesh, p, p + 2, form).toarray()
    B = O.dense_bruteforce(mesh, p, p + 2, form)
    np.testing.assert_allclose(A, B, atol=1e-13 * np.abs(B).max())


@pytest.mark.parametrize("form", [O.MASS, O.DIFFUSION])
@pytest.mark.parametrize("p", [1, 3, 5])
def test_elementwise_action_rows_diag_match_csr(form, p):
    mesh = perturbed(3, 2, 2, seed=19)
    prob = O.Problem(mesh, p, None, form)
    x = FI.uniform_vector(prob.N, seed=1)
    for constrained in (False, True):
        ess = prob.ess if constrained else None
        y = (prob.Ac if constrained else prob.A) @ x
        y2 = O.action_elementwise(mesh, p, p + 2, form, x, ess=ess)
        np.testing.assert_allclose(y2, y, atol=1e-13 * np.abs(y).max())
        rows = np.random.default_rng(0).choice(prob.N, 25, replace=False)
        np.testing.assert_allclose(O.action_rows(mesh, p, p + 2, form, x, rows, ess=ess), y[rows],
                                   atol=1e-13 * np.abs(y).max())
        d = O.diagonal_elementwise(mesh, p, p + 2, form, ess=ess)
        np.testing.assert_allclose(d, (prob.Ac if constrained else prob.A).diagonal(), rtol=1e-13)


def test_rhs_of_one_is_mass_times_one():
    mesh = perturbed(2, 2, 2, seed=23)
    for p in (1, 2, 4):
        b = O.rhs_from_qp(mesh, p, p + 2, np.ones((mesh.num_elements, (p + 2) ** 3)))
        M = O.assemble_csr(mesh, p, p + 2, O.MASS)
        np.testing.assert_allclose(b, M @ np.ones(M.shape[0]), atol=1e-15)
        assert abs(b.sum() - 1.0) < 1e-14


@pytest.mark.parametrize("form", [O.MASS, O.DIFFUSION])
def test_cg_matches_dense_solve(form):
    mesh = perturbed(3, 3, 2, seed=29)
    prob = O.Problem(mesh, 2, None, form)
    b = prob.sine_rhs()
    x, it, res = prob.solve(b, rtol=1e-13)
    xd = sla.solve(prob.Ac.toarray(), b, assume_a="pos")
    assert res <= 1e-13
    assert np.linalg.norm(x - xd) <= 1e-11 * np.linalg.norm(xd)


def test_planted_transpose_mistake_is_caught(monkeypatch):
    # Using J^{-T} J^{-1} in place of J^{-1} J^{-T} (a transposed Jacobian) must fail the
    # linear patch test on a perturbed mesh: the pins are sensitive to it.
    orig = O.fem_oracle.qp_factors

    def wrong(X, R, form):
        F = orig(X, R, form)
        if form != O.DIFFUSION:
            return F
        _, J = O.trilinear(X, R.xi)
        Jinv = np.linalg.inv(J)
        wdet = R.w[None, :] * np.linalg.det(J)
        return wdet[..., None, None] * np.einsum("emdr,emds->emrs", Jinv, Jinv)

    monkeypatch.setattr(O.fem_oracle, "qp_factors", wrong)
    mesh = perturbed(3, 2, 2, seed=11)
    K = O.fem_oracle.assemble_csr(mesh, 2, 4, O.DIFFUSION)
    xyz = O.node_coords(mesh, 2)
    u = 0.3 + 1.1 * xyz[:, 0] - 0.7 * xyz[:, 1] + 2.3 * xyz[:, 2]
    interior = np.setdiff1d(np.arange(len(u)), O.boundary_dofs(mesh, 2))
    assert np.abs((K @ u)[interior]).max() > 1e-6


# ---------------------------------------------------------------- p-multigrid pieces

@pytest.mark.parametrize("pc,pf", [(1, 2), (2, 4), (1, 3), (3, 6)])
def test_prolongation_reproduces_coarse_polynomials(pc, pf):
    # interpolating a coarse-space function onto the fine nodes is exact: P u_c equals the
    # fine nodal values of the same polynomial (degree <= pc in each reference variable)
    mesh = perturbed(2, 1, 2, seed=9)
    P = O.order_prolongation(mesh, pc, pf)
    xc, xf = O.node_coords(mesh, pc), O.node_coords(mesh, pf)
    f = lambda x: (1 + x[:, 0] - 0.5 * x[:, 1] + 2 * x[:, 2]) ** pc  # noqa: E731
    # on a trilinear mesh this is in Q_pc only for pc = 1 or an affine element; use the
    # element map instead: nodal values of a Q_pc function of the reference coordinates
    np.testing.assert_allclose(P @ np.ones(P.shape[1]), np.ones(P.shape[0]), atol=1e-14)
    if pc == 1:
        np.testing.assert_allclose(P @ f(xc), f(xf), atol=1e-12)
    # the fine mass matrix restricted by P is the coarse mass matrix (the spaces are nested)
    Mf = O.assemble_csr(mesh, pf, pf + 2, O.MASS)
    Mc = O.assemble_csr(mesh, pc, pc + 2, O.MASS)
    np.testing.assert_allclose((P.T @ Mf @ P).toarray(), Mc.toarray(), atol=1e-14)


def test_chebyshev_smoother_polynomial_bound():
    # for [lmin, lmax] containing the spectrum of D^{-1}A the A-norm error after k steps is
    # at most 1/T_k(sigma) times the initial one (Chebyshev minimax property); and with a wide
    # interval it converges to the solution
    mesh = perturbed(2, 2, 2, seed=4)
    prob = O.Problem(mesh, 2, None, O.DIFFUSION)
    A = prob.Ac.toarray()
    dg = np.diag(A).copy()
    ev = np.linalg.eigvals(A / dg[:, None]).real
    lmin, lmax = ev.min(), ev.max()
    b = FI.uniform_vector(prob.N, seed=2)
    x = np.linalg.solve(A, b)
    sigma = (lmax + lmin) / (lmax - lmin)
    for k in (1, 3, 8, 20):
        xk = O.chebyshev_smoother(lambda v: A @ v, dg, b, lmin, lmax, k)
        e = xk - x
        bound = 1.0 / np.cosh(k * np.arccosh(sigma))
        assert np.sqrt(e @ A @ e) <= bound * np.sqrt(x @ A @ x) * (1 + 1e-9)
    xk = O.chebyshev_smoother(lambda v: A @ v, dg, b, lmin, lmax, 200)
    np.testing.assert_allclose(xk, x, rtol=0, atol=1e-10 * np.abs(x).max())


def test_pmg_vcycle_two_levels_reduces_error_and_is_symmetric():
    # a symmetric V-cycle is a symmetric operator and, with a convergent smoother and an
    # accurate coarse solve, a good preconditioner: kappa(M A) far below kappa(D^{-1} A)
    mesh = perturbed(3, 3, 3, seed=8)
    pf, pc = 4, 2
    prf, prc = O.Problem(mesh, pf, None, O.DIFFUSION), O.Problem(mesh, pc, None, O.DIFFUSION)
    As = [prf.Ac, prc.Ac]
    P = O.order_prolongation(mesh, pc, pf)
    lam = [np.linalg.eigvals(A.toarray() / A.diagonal()[:, None]).real.max() for A in As]
    M = np.stack([O.pmg_vcycle(As, [A.diagonal() for A in As], [P], lam, 2, 40, e, ess=[prf.ess, prc.ess])
                  for e in np.eye(prf.N)], axis=1)
    interior = np.setdiff1d(np.arange(prf.N), prf.ess)
    Mi = M[np.ix_(interior, interior)]
    np.testing.assert_allclose(Mi, Mi.T, atol=1e-10 * np.abs(Mi).max())
    Ai = As[0].toarray()[np.ix_(interior, interior)]
    ev = np.sort(np.linalg.eigvals(Mi @ Ai).real)
    evj = np.sort(np.linalg.eigvals(Ai / np.diag(Ai)[:, None]).real)
    assert ev[0] > 0 and ev[-1] / ev[0] < 0.1 * evj[-1] / evj[0]


# ---------------------------------------------------------------- L2 norm of the error

def _l2_pins(p, mesh):
    """The values l2_error must give on a perturbed unit cube, each fixed in closed form:
    with u_h = 0 it is ||u||, so ||1|| = 1 (|Omega| = 1), ||x|| = 1/sqrt(3) and
    ||sin(pi x) sin(pi y) sin(pi z)|| = (1/2)^(3/2) (each factor integrates sin^2 to 1/2);
    the nodal interpolant of a polynomial of total degree <= p in physical coordinates is in
    the space (its pull-back by a trilinear map is in Q_p), so its error is zero; and the
    interpolant of x against u = 0 gives ||x|| again.  Returns the deviations."""
    N = O.num_dofs(mesh, p)
    zero = np.zeros(N)
    xyz = O.node_coords(mesh, p)
    poly = lambda X: (0.3 + X[..., 0] - 2.0 * X[..., 1] + 0.5 * X[..., 2]) ** p  # noqa: E731
    nil = lambda X: np.zeros(X.shape[:-1])  # noqa: E731
    return {
        "one": abs(O.l2_error(mesh, p, zero, lambda X: np.ones(X.shape[:-1])) - 1.0),
        "x": abs(O.l2_error(mesh, p, zero, lambda X: X[..., 0]) - 1.0 / math.sqrt(3.0)),
        "sine": abs(O.l2_error(mesh, p, zero, O.sine_solution) - 0.5 ** 1.5),
        "interpolant": O.l2_error(mesh, p, poly(xyz), poly),
        "interp_x": abs(O.l2_error(mesh, p, xyz[:, 0], nil) - 1.0 / math.sqrt(3.0)),
    }


# the sine is integrated by the p+5 rule, not exactly: 5e-12 holds its error for p = 1..3 on
# this mesh (5.8e-13 at p = 1) while the operator's own p+2 rule misses by 1e-10 .. 1e-6
_L2_TOL = {"one": 1e-13, "x": 1e-13, "sine": 5e-12, "interpolant": 1e-13, "interp_x": 1e-13}


def _l2_mesh():
    return perturbed(2, 3, 2, seed=37)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_l2_error_closed_forms(p):
    dev = _l2_pins(p, _l2_mesh())
    for k, v in dev.items():
        assert v <= _L2_TOL[k], (k, v)


def _some_l2_pin_fails():
    return any(any(v > _L2_TOL[k] for k, v in _l2_pins(p, _l2_mesh()).items()) for p in (1, 2))


def test_l2_error_planted_missing_sqrt_is_caught(monkeypatch):
    monkeypatch.setattr(O.fem_oracle, "math", type("M", (), {"sqrt": staticmethod(lambda v: v)}))
    assert _some_l2_pin_fails()


def test_l2_error_planted_missing_detj_is_caught(monkeypatch):
    orig = O.fem_oracle.qp_factors

    def weights_only(X, R, form):
        F = orig(X, R, form)
        return np.broadcast_to(R.w[None, :], F.shape).copy() if form == O.MASS else F

    monkeypatch.setattr(O.fem_oracle, "qp_factors", weights_only)
    assert _some_l2_pin_fails()


def test_l2_error_planted_operator_rule_is_caught(monkeypatch):
    orig = O.fem_oracle.rule
    monkeypatch.setattr(O.fem_oracle, "rule", lambda p, q: orig(p, p + 2))
    assert _some_l2_pin_fails()


@pytest.mark.parametrize("p", [1, 2, 3])
def test_l2_convergence_rate_two_sided(p):
    # the discrete solution's L2 error falls at rate p+1, neither slower nor faster (a
    # missing square root would double the observed rate)
    errs = []
    ns = (2, 4, 8) if p < 3 else (2, 4, 6)
    for n in ns:
        mesh = perturbed(n, n, n, seed=31)
        prob = O.Problem(mesh, p, None, O.DIFFUSION)
        x, it, res = prob.solve(prob.sine_rhs(), rtol=1e-12)
        errs.append(O.l2_error(mesh, p, x, O.sine_solution))
    rate = math.log(errs[-2] / errs[-1]) / math.log(ns[-1] / ns[-2])
    assert p + 1 - 0.35 < rate < p + 1 + 0.35, (errs, rate)


def _cheb_smoother_matrix(A, lmin, lmax, k):
    """Closed form of k Chebyshev-Jacobi steps from x0 = 0: the error is R_k(D^-1 A) times the
    initial error, R_k(t) = T_k((theta - t) / delta) / T_k(theta / delta), so x_k = S b with
    S = (I - R_k(D^-1 A)) A^-1.  R_k(D^-1 A) is evaluated through the eigendecomposition of the
    symmetric D^-1/2 A D^-1/2, T_k by numpy's Chebyshev-series routine."""
    d = np.diag(A)
    Ds, Dis = np.diag(np.sqrt(d)), np.diag(1.0 / np.sqrt(d))
    lam, Q = np.linalg.eigh(Dis @ A @ Dis)
    theta, delta = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
    Tk = lambda x: np.polynomial.chebyshev.chebval(x, [0.0] * k + [1.0])  # noqa: E731
    R = Dis @ (Q * (Tk((theta - lam) / delta) / Tk(theta / delta))) @ Q.T @ Ds
    return (np.eye(len(d)) - R) @ np.linalg.inv(A)


def test_chebyshev_smoother_and_vcycle_equal_their_closed_forms():
    """The oracle's smoother recurrence equals the closed-form Chebyshev polynomial of D^-1 A,
    and its V-cycle (levels p = 4, 2, 1) equals the symmetric V-cycle built from dense matrices:
    M_l = (I - S A)[(I - C A) S + C] + S with C = P M_{l+1} Z_{l+1} P^T Z_l (Z_l zeroes the
    essential rows of level l) and M_L the coarsest level's smoother, so its error operator is
    (I - S A)(I - C A)(I - S A).  A dropped smoothing pass, a missing mask, P in place of P^T or a
    wrong recurrence coefficient each change the matrix."""
    mesh = perturbed(2, 2, 2, seed=12)
    ps = [4, 2, 1]
    probs = [O.Problem(mesh, p, None, O.DIFFUSION) for p in ps]
    As = [pr.Ac for pr in probs]
    Ad = [A.toarray() for A in As]
    Ps = [O.order_prolongation(mesh, ps[l + 1], ps[l]) for l in range(len(ps) - 1)]
    ess = [pr.ess for pr in probs]
    lam = [np.linalg.eigvals(A / np.diag(A)[:, None]).real.max() for A in Ad]
    smooth, coarse, deg, cdeg = (0.25, 1.1), (0.003, 1.2), 2, 24
    # the smoother alone, on unit vectors
    S0 = _cheb_smoother_matrix(Ad[0], smooth[0] * lam[0], smooth[1] * lam[0], deg)
    Sor = np.stack([O.chebyshev_smoother(lambda v: Ad[0] @ v, np.diag(Ad[0]), e, smooth[0] * lam[0],
                                         smooth[1] * lam[0], deg) for e in np.eye(probs[0].N)], axis=1)
    np.testing.assert_allclose(Sor, S0, rtol=0, atol=1e-11 * np.abs(S0).max())

    def mask(l):
        z = np.ones(probs[l].N)
        z[ess[l]] = 0.0
        return np.diag(z)

    def vcycle_matrix(l):
        A = Ad[l]
        if l == len(ps) - 1:
            return _cheb_smoother_matrix(A, coarse[0] * lam[l], coarse[1] * lam[l], cdeg)
        S = _cheb_smoother_matrix(A, smooth[0] * lam[l], smooth[1] * lam[l], deg)
        P = Ps[l].toarray()
        C = P @ vcycle_matrix(l + 1) @ mask(l + 1) @ P.T @ mask(l)
        I = np.eye(len(A))
        return (I - S @ A) @ ((I - C @ A) @ S + C) + S

    M = vcycle_matrix(0)
    Mor = np.stack([O.pmg_vcycle(As, [A.diagonal() for A in As], Ps, lam, deg, cdeg, e, smooth=smooth,
                                 coarse=coarse, ess=ess) for e in np.eye(probs[0].N)], axis=1)
    np.testing.assert_allclose(Mor, M, rtol=0, atol=1e-9 * np.abs(M).max())
    # and the error operator factorises as stated
    S = _cheb_smoother_matrix(Ad[0], smooth[0] * lam[0], smooth[1] * lam[0], deg)
    P = Ps[0].toarray()
    C = P @ vcycle_matrix(1) @ mask(1) @ P.T @ mask(0)
    I = np.eye(probs[0].N)
    E = (I - S @ Ad[0]) @ (I - C @ Ad[0]) @ (I - S @ Ad[0])
    np.testing.assert_allclose(I - Mor @ Ad[0], E, rtol=0, atol=1e-8)
