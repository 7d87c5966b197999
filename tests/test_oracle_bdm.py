"""Pins of the (BDM_k, dP_{k-1}) interior-penalty oracle (Case 3 of Sec. 3; Eq. DiscontBilinearForm) against
facts fixed by the mathematics:

* the reference basis is dual to its DoFs (exact), the global space has continuous normal components;
* BDM_k interpolation reproduces vector P_k fields; P reproduces coarse fields on the fine level;
* for continuous polynomial fields every jump term vanishes, so u^T K u = 2 nu int eps(u):eps(u) and
  p^T B u = -int (div u) p (closed forms by sympy);
* the matrix is symmetric, its velocity block is positive definite on the free DoFs, the constant
  pressure is in its kernel after the no-flux rows;
* one extended cell patch per cell with the closed-form interior size;
* the manufactured solution converges at O(h^k) (broken H^1 velocity, L^2 pressure) as the paper states;
* the V-cycle equals its dense composition and FGMRES equals the bordered direct solve.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import bdm, exact, fem, solver

sympy = pytest.importorskip("sympy")


@pytest.mark.parametrize("k", [1, 2, 3])
def test_reference_basis_is_dual_to_the_dofs(k):
    B = bdm.reference_basis(k)
    for i, (bx, by) in enumerate(B):
        for e, (a, b_) in enumerate(bdm._EDGES):
            va, vb = bdm._VERTS[a], bdm._VERTS[b_]
            nu = bdm._rot((vb[0] - va[0], vb[1] - va[1]))
            for j in range(k + 1):
                t = Fraction(j + 1, k + 2)
                x, y = va[0] + t * (vb[0] - va[0]), va[1] + t * (vb[1] - va[1])
                v = bdm._eval(bx, x, y) * nu[0] + bdm._eval(by, x, y) * nu[1]
                assert v == (1 if i == e * (k + 1) + j else 0)
        for m, (qx, qy) in enumerate(bdm._ned_space(k)):
            mom = exact.integrate_ref(exact.mul(bx, qx)) if qx and bx else 0
            mom += exact.integrate_ref(exact.mul(by, qy)) if qy and by else 0
            assert mom == (1 if i == 3 * (k + 1) + m else 0)


def _poly_field(k):
    return (lambda X, Y: (X ** k - 2 * X * Y ** (k - 1) + 0.5, Y ** k + X ** (k - 1) * Y - 0.25))


@pytest.mark.parametrize("k", [1, 2, 3])
def test_normal_continuity_and_polynomial_reproduction(k):
    s = bdm.BDMSpace(3, k)
    rng = np.random.default_rng(5)
    x = rng.standard_normal(s.ndof)
    cells_of = {}
    for c, cell in enumerate(s.cells):
        for (a, b) in bdm._EDGES:
            cells_of.setdefault(s.edge_id[tuple(sorted((cell[a], cell[b]), key=s.vid))], []).append(c)
    h = 1.0 / s.N
    for e, cs in cells_of.items():
        if len(cs) < 2:
            continue
        A, B = (np.array(p, float) * h for p in s.edges[e])
        n = np.array([B[1] - A[1], A[0] - B[0]])
        X = A[None, :] + np.array([0.2, 0.55, 0.9])[:, None] * (B - A)[None, :]
        vals = []
        for c in cs:
            x0, J = s.geometry(c, h)
            ref = np.linalg.solve(J, (X - x0).T).T
            u, _ = bdm.evaluate(s, x, c, ref)
            vals.append(u @ n)
        assert np.allclose(vals[0], vals[1], rtol=0, atol=1e-12 * np.abs(x).max())
    fu = _poly_field(k)
    xI = bdm.interpolate(s, fu)
    pts = np.array([[0.2, 0.3], [0.6, 0.1], [0.1, 0.7]])
    for c in range(len(s.cells)):
        x0, J = s.geometry(c, h)
        u, _ = bdm.evaluate(s, xI, c, pts)
        X = x0[None, :] + pts @ J.T
        want = np.stack(fu(X[:, 0], X[:, 1]), axis=1)
        assert np.abs(u - want).max() <= 1e-12


@pytest.mark.parametrize("k", [1, 2, 3])
def test_energy_and_divergence_moments_equal_closed_forms(k):
    xs, ys = sympy.symbols("x y")
    u1 = xs ** k - 2 * xs * ys ** (k - 1) + sympy.Rational(1, 2)
    u2 = ys ** k + xs ** (k - 1) * ys - sympy.Rational(1, 4)
    p = xs ** (k - 1) + 3 * ys ** (k - 1) * xs ** 0 - 1 if k > 1 else sympy.Integer(2)
    e11, e22 = sympy.diff(u1, xs), sympy.diff(u2, ys)
    e12 = (sympy.diff(u1, ys) + sympy.diff(u2, xs)) / 2
    nu = 1.5
    energy = float(2 * sympy.Rational(3, 2) * sympy.integrate(e11 ** 2 + 2 * e12 ** 2 + e22 ** 2, (xs, 0, 1), (ys, 0, 1)))
    divmom = float(-sympy.integrate((e11 + e22) * p, (xs, 0, 1), (ys, 0, 1)))
    s = bdm.BDMSpace(2, k)
    K = bdm.assemble_full(s, nu)
    fu = _poly_field(k)
    fp = sympy.lambdify((xs, ys), p, "numpy")
    uI = bdm.interpolate(s, fu)
    pI = bdm.interpolate(s, lambda X, Y: (0 * X, 0 * X), lambda X, Y: fp(X, Y) + 0 * X)
    pI[:s.n_u] = 0.0
    assert abs(uI @ K @ uI - energy) <= 1e-10 * abs(energy)
    assert abs(pI @ K @ uI - divmom) <= 1e-10 * max(1.0, abs(divmom))


@pytest.mark.parametrize("k", [1, 2])
def test_symmetry_positivity_and_pressure_nullspace(k):
    s = bdm.BDMSpace(3, k)
    K = bdm.assemble_full(s)
    assert abs(K - K.T).max() == 0.0
    mask = s.dirichlet_mask()
    A = fem.apply_dirichlet(K, mask)
    free = np.flatnonzero(~mask[:s.n_u])
    Av = K.toarray()[np.ix_(free, free)]
    assert np.linalg.eigvalsh(Av).min() > 0
    assert np.abs(A @ s.nullspace()).max() <= 1e-12 * abs(A).max()


@pytest.mark.parametrize("k", [1, 2, 3])
def test_prolongation_reproduces_coarse_fields(k):
    c, f = bdm.BDMSpace(2, k), bdm.BDMSpace(4, k)
    P = bdm.prolongation(c, f)
    fu = _poly_field(k)
    fp = lambda X, Y: X ** (k - 1) - 2 * Y + 0.5 if k > 1 else 0.5 + 0 * X
    xc, xf = bdm.interpolate(c, fu, fp), bdm.interpolate(f, fu, fp)
    assert np.abs(P @ xc - xf).max() <= 1e-12 * np.abs(xf).max()


@pytest.mark.parametrize("k", [1, 2, 3])
def test_extended_cell_patches(k):
    N = 4
    s = bdm.BDMSpace(N, k)
    plist = bdm.build_patches(s)
    assert len(plist) == len(s.cells)
    mask = s.dirichlet_mask()
    cnt = np.zeros(s.ndof, int)
    for _, c, d in plist:
        cnt[d] += 1
        assert not mask[d].any()
    assert np.all(cnt[s.n_u:] == 1) and np.all((cnt[:s.n_u] > 0) == ~mask[:s.n_u])
    # a cell whose three neighbours have no boundary edge has the closed-form size
    lower_mid = (N // 2) * N + N // 2
    assert len(plist[lower_mid][2]) == bdm.interior_patch_size(k)


@pytest.mark.parametrize("k,Ns", [(1, (16, 32)), (2, (8, 16))])
def test_manufactured_convergence_rates(k, Ns):
    errs = []
    for N in Ns:
        s = bdm.BDMSpace(N, k)
        K = bdm.assemble_full(s)
        mask = s.dirichlet_mask()
        A = fem.apply_dirichlet(K, mask)
        b = bdm.load_vector(s)
        b[mask] = 0.0                     # u . n = 0 on the boundary (the exact solution satisfies it)
        x = solver.direct_solve(A, s.nullspace(), solver.project(s, b))
        errs.append(bdm.errors(s, x))
    h1, l2, pl2 = [np.log2(errs[0][i] / errs[1][i]) for i in range(3)]
    assert h1 > k - 0.15 and l2 > k + 0.5 and pl2 > k - 0.2, (h1, l2, pl2)


@pytest.mark.parametrize("k", [1, 2])
def test_bdm_vcycle_dense_composition_and_fgmres(k):
    from test_oracle_solver import _vcycle_matrix
    H = solver.Hierarchy(2, 2, k, cell="bdm")
    fin = H.finest
    b = np.random.default_rng(7).standard_normal(fin.space.ndof)
    want = _vcycle_matrix(H) @ b
    assert np.linalg.norm(H.vcycle(b) - want) <= 1e-12 * np.linalg.norm(want)
    res = solver.solve(H, b, 1e-12, 100)
    bp = solver.project(fin.space, b)
    xd = solver.project(fin.space, solver.direct_solve(fin.A, fin.space.nullspace(), bp))
    assert res.converged and np.linalg.norm(res.x - xd) <= 1e-9 * np.linalg.norm(xd)


@pytest.mark.parametrize("k", [2, 3, 4])
def test_interior_moment_functions_are_orthogonal_and_span_nedelec(k):
    # the interior DoFs' test functions: pairwise L^2-orthogonal on the reference triangle, norms in
    # [1, 2), and the same span as the monomial-generated Nedelec space (exact ranks of the coefficient
    # matrices over the monomials)
    Q = bdm._ned_space(k)
    M = bdm._ned_monomial(k)
    assert len(Q) == len(M) == (k + 1) * (k - 1)
    for i, a in enumerate(Q):
        for j, b in enumerate(Q):
            ip = bdm._ned_inner(a, b)
            if i != j:
                assert ip == 0
            else:
                assert 1 <= ip < 4
    keys = sorted({(c, pq) for f in Q + M for c in (0, 1) for pq in f[c]})
    mat = lambda fs: sympy.Matrix([[f[c].get(pq, 0) for (c, pq) in keys] for f in fs])
    assert mat(Q).rank() == mat(M).rank() == mat(Q + M).rank() == len(M)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_penalty_makes_the_form_coercive_with_margin(k):
    # alpha = (k+1)(k+2) is "sufficiently large" (Sec. 2.1): the velocity block is positive definite on
    # the free DoFs, while a quarter of it loses coercivity (the bound is not vacuous)
    s = bdm.BDMSpace(4, k)
    free = ~s.dirichlet_mask()[:s.n_u]
    mins = []
    for scale in (1.0, 0.25):
        old = bdm.penalty
        bdm.penalty = lambda kk, scale=scale: scale * old(kk)
        try:
            K = bdm.assemble_full(s)
        finally:
            bdm.penalty = old
        Au = K[:s.n_u, :s.n_u].toarray()[np.ix_(free, free)]
        mins.append(np.linalg.eigvalsh(Au).min())
    assert mins[0] > 0 > mins[1], mins


@pytest.mark.parametrize("case", [(2, 2, 1), (2, 3, 1), (2, 2, 2), (2, 3, 2), (2, 2, 3)])
def test_iteration_counts_are_h_and_p_robust(case):
    # Sec. 4.3: with the extended cell patches the counts hardly depend on k or the level count (rtol 1e-10)
    H = solver.Hierarchy(*case, cell="bdm")
    b = np.random.default_rng(0).standard_normal(H.finest.space.ndof)
    res = solver.solve(H, b, 1e-10, 100)
    assert res.converged and 20 <= res.iters <= 40, res.iters
