"""Pins of the quadrilateral Taylor-Hood oracle (Q_k, Q_{k-1}; Case 2 of Sec. 3) against facts fixed by the
mathematics, not by the oracle itself:

* the 1-D Lagrange bases are Kronecker on their nodes and reproduce polynomials;
* element energies 2 nu int eps(u):eps(u) and divergence moments -int (div u) p of polynomial fields equal
  their closed forms (integrated independently with sympy), rigid motions are in the kernel of A;
* the assembled matrix is symmetric and annihilates the constant pressure after the Dirichlet rows;
* P reproduces coarse Q_k / Q_{k-1} functions and P^T K_f P = K_c (rediscretisation equals Galerkin
  coarsening for nested conforming spaces, Sec. 3);
* patch counts and interior sizes equal the closed forms of Sec. 3.1's vertex / edge / cell patches;
* the manufactured solution converges at O(h^k) (velocity H^1, pressure L^2) and O(h^{k+1}) (velocity L^2);
* the V-cycle equals its dense composition and FGMRES equals the bordered direct solve.
"""
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fem, quad, solver

sympy = pytest.importorskip("sympy")


@pytest.mark.parametrize("deg", [1, 2, 3, 4])
def test_lagrange_1d_is_kronecker_and_reproduces_polynomials(deg):
    L = quad.lagrange_1d(deg)
    for i, p in enumerate(L):
        for j in range(deg + 1):
            assert quad._peval(p, Fraction(j, deg)) == (1 if i == j else 0)
    x = Fraction(2, 7)
    for m in range(deg + 1):
        assert sum(quad._peval(p, x) * Fraction(j, deg) ** m for j, p in enumerate(L)) == x ** m


def _interp(space, fu, fp):
    X, Y = space.vnode_xy()
    v = np.zeros(space.ndof)
    v[0:space.n_u:2], v[1:space.n_u:2] = fu(X, Y)
    Xp, Yp = space.pnode_xy()
    v[space.n_u:] = fp(Xp, Yp)
    return v


@pytest.mark.parametrize("k", [2, 3, 4])
@pytest.mark.parametrize("N", [1, 2])
def test_energy_and_divergence_moments_equal_closed_forms(k, N):
    xs, ys = sympy.symbols("x y")
    u1 = xs ** k * ys ** (k - 1) + 3 * xs * ys ** k
    u2 = 2 * xs ** (k - 1) * ys ** k - ys ** 2 * xs
    p = xs ** (k - 1) * ys + 5 * ys ** (k - 1)
    e11, e22 = sympy.diff(u1, xs), sympy.diff(u2, ys)
    e12 = (sympy.diff(u1, ys) + sympy.diff(u2, xs)) / 2
    nu = Fraction(3, 2)
    energy = 2 * sympy.Rational(3, 2) * sympy.integrate(e11 ** 2 + 2 * e12 ** 2 + e22 ** 2, (xs, 0, 1), (ys, 0, 1))
    divmom = -sympy.integrate((e11 + e22) * p, (xs, 0, 1), (ys, 0, 1))
    s = quad.QSpace(N, k)
    K = quad.assemble_full(s, float(nu))
    fu1, fu2, fp = (sympy.lambdify((xs, ys), f, "numpy") for f in (u1, u2, p))
    uI = _interp(s, lambda X, Y: (fu1(X, Y), fu2(X, Y)), lambda X, Y: 0 * X)
    pI = _interp(s, lambda X, Y: (0 * X, 0 * X), lambda X, Y: fp(X, Y) + 0 * X)
    assert abs(uI @ K @ uI - float(energy)) <= 1e-12 * abs(float(energy))
    assert abs(pI @ K @ uI - float(divmom)) <= 1e-12 * max(1.0, abs(float(divmom)))


@pytest.mark.parametrize("k", [2, 3])
def test_rigid_motions_in_kernel_and_symmetry(k):
    s = quad.QSpace(3, k)
    K = quad.assemble_full(s)
    assert abs(K - K.T).max() == 0.0
    for fu in (lambda X, Y: (1 + 0 * X, 0 * X), lambda X, Y: (0 * X, 1 + 0 * X), lambda X, Y: (-Y, X)):
        v = _interp(s, fu, lambda X, Y: 0 * X)
        assert np.abs((K @ v)[:s.n_u]).max() <= 1e-13
    A = fem.apply_dirichlet(K, s.dirichlet_mask())
    assert np.abs(A @ s.nullspace()).max() <= 1e-13 * abs(A).max()


@pytest.mark.parametrize("k", [2, 3, 4])
def test_transfers_reproduce_coarse_functions_and_galerkin_identity(k):
    c, f = quad.QSpace(2, k), quad.QSpace(4, k)
    P = quad.prolongation(c, f)
    g = lambda X, Y: (X ** k * Y + Y ** k, X * Y ** (k - 1))
    h = lambda X, Y: X ** (k - 1) * Y ** (k - 1) - 2 * X
    assert np.abs(P @ _interp(c, g, h) - _interp(f, g, h)).max() <= 1e-13
    Kc, Kf = quad.assemble_full(c), quad.assemble_full(f)
    G = (P.T @ Kf @ P).toarray()
    free_c = ~c.dirichlet_mask()
    # free coarse functions prolong to free fine functions (zero on the boundary): compare on them
    assert np.abs(G[np.ix_(free_c, free_c)] - Kc.toarray()[np.ix_(free_c, free_c)]).max() <= 1e-12 * abs(Kc).max()


@pytest.mark.parametrize("k", [2, 3, 4])
def test_patch_counts_and_interior_sizes(k):
    N = 4
    s = quad.QSpace(N, k)
    plist = quad.build_patches(s)
    nv, ne, ncl = (N + 1) ** 2, (2 * N * (N + 1) if k >= 3 else 0), (N * N if k >= 3 else 0)
    kinds = [p[0] for p in plist]
    assert kinds.count("vertex") == nv and kinds.count("edge") == ne and kinds.count("cell") == ncl
    # every pressure DoF in exactly one patch, every free velocity DoF in some patch
    cnt = np.zeros(s.ndof, int)
    for _, _, d in plist:
        cnt[d] += 1
    assert np.all(cnt[s.n_u:] >= 1)
    pres = np.zeros(s.n_p, int)
    for _, _, d in plist:
        pres[d[d >= s.n_u] - s.n_u] += 1
    assert np.all(pres == 1)
    mask = s.dirichlet_mask()
    assert np.all((cnt[:s.n_u] > 0) == ~mask[:s.n_u])
    # interior patches (cells of the star closure away from the boundary) have the closed-form sizes
    checked = 0
    for kind, (ek, e), d in plist:
        cells = quad._cells_of(ek, e, N)
        full = len(cells) == {"vertex": 4, "hedge": 2, "vedge": 2, "cell": 1}[ek]
        if full and all(1 <= a <= N - 2 and 1 <= b <= N - 2 for a, b in cells):
            assert len(d) == quad.interior_patch_size(k, kind), (kind, e)
            checked += 1
    assert checked > 0
    # pressure DoFs of a patch lie on its entity: vertex / edge interior / cell interior
    Xp, Yp = s.pnode_xy()
    for kind, (ek, (i, j)), d in plist:
        for q in d[d >= s.n_u] - s.n_u:
            X, Y = Xp[q] * N, Yp[q] * N
            if ek == "vertex":
                assert (X, Y) == (i, j)
            elif ek == "hedge":
                assert Y == j and i < X < i + 1
            elif ek == "vedge":
                assert X == i and j < Y < j + 1
            else:
                assert i < X < i + 1 and j < Y < j + 1


def _errors(N, k):
    s = quad.QSpace(N, k)
    K = quad.assemble_full(s)
    A = fem.apply_dirichlet(K, s.dirichlet_mask())
    b = solver.project(s, quad.manufactured_rhs(s, K))
    x = solver.direct_solve(A, s.nullspace(), b)
    return quad.errors(s, x)


@pytest.mark.parametrize("k,Ns", [(2, (8, 16)), (3, (4, 8)), (4, (2, 4))])
def test_manufactured_convergence_rates(k, Ns):
    e = [_errors(N, k) for N in Ns]
    h1, l2, pl2 = [np.log2(e[0][i] / e[1][i]) for i in range(3)]
    assert h1 > k - 0.15 and l2 > k + 1 - 0.25 and pl2 > k - 0.25, (h1, l2, pl2)


@pytest.mark.parametrize("k", [2, 3])
def test_quad_vcycle_equals_dense_composition_and_fgmres_equals_direct_solve(k):
    from test_oracle_solver import _vcycle_matrix
    H = solver.Hierarchy(2, 2, k, cell="quad")
    fin = H.finest
    b = np.random.default_rng(91).standard_normal(fin.space.ndof)
    want = _vcycle_matrix(H) @ b
    assert np.linalg.norm(H.vcycle(b) - want) <= 1e-13 * np.linalg.norm(want)
    res = solver.solve(H, b, 1e-12, 100)
    bp = solver.project(fin.space, b)
    xd = solver.project(fin.space, solver.direct_solve(fin.A, fin.space.nullspace(), bp))
    assert res.converged and np.linalg.norm(res.x - xd) <= 1e-10 * np.linalg.norm(xd)
