"""Pins for the oracle's patches, additive Vanka, Chebyshev, eigenvalue estimate, V-cycle and FGMRES."""
from fractions import Fraction
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fem, patches, solver, splitmix

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ patches (Sec. 3.1)

HAND_DERIVED_SIZES = {
    # distinct patch sizes (Dirichlet DoFs excluded) on an 8x8 mesh, by kind; derived by hand from
    # the closure-of-star rule: interior, edge-adjacent, corner patches ...
    2: {"vertex": {3, 9, 11, 15, 27, 29, 33, 39}},
    3: {"vertex": {7, 19, 25, 31, 59, 61, 67, 75}, "edge": {7, 13, 19, 23, 25, 31, 33}},
    4: {"vertex": {13, 33, 45, 53, 103, 105, 113, 123}, "edge": {14, 22, 34, 40, 42, 50, 52},
        "cell": {13, 21, 27, 29, 31}},
}


@pytest.mark.parametrize("k", [2, 3, 4])
def test_patch_counts_sizes_and_pressure_partition(k):
    N = 8
    s = fem.Space(N, k)
    P = patches.build_patches(s)
    kinds = {}
    for kind, ent, dofs in P:
        kinds.setdefault(kind, []).append(len(dofs))
    assert len(kinds["vertex"]) == (N + 1) ** 2
    if k >= 3:
        assert len(kinds["edge"]) == 3 * N * N + 2 * N
    if k >= 4:
        assert len(kinds["cell"]) == 2 * N * N
    for kind, sizes in HAND_DERIVED_SIZES[k].items():
        assert set(kinds[kind]) == sizes
        assert max(kinds[kind]) == patches.interior_patch_size(k, kind)
    # every pressure DoF is in exactly one patch; no Dirichlet DoF is in any patch
    allp = np.concatenate([d[d >= s.n_u] for _, _, d in P])
    assert np.array_equal(np.sort(allp), np.arange(s.n_u, s.ndof))
    mask = s.dirichlet_mask()
    assert not any(mask[d].any() for _, _, d in P)
    for _, _, d in P:
        assert np.all(np.diff(d) > 0)


def _point_in_closed_triangle(p, tri):
    (x, y) = p
    (x0, y0), (x1, y1), (x2, y2) = tri
    d = (x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0)
    l1 = ((x - x0) * (y2 - y0) - (x2 - x0) * (y - y0)) / d
    l2 = ((x1 - x0) * (y - y0) - (x - x0) * (y1 - y0)) / d
    return l1 >= 0 and l2 >= 0 and l1 + l2 <= 1


def _point_strictly_inside(p, tri):
    (x, y) = p
    (x0, y0), (x1, y1), (x2, y2) = tri
    d = (x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0)
    l1 = ((x - x0) * (y2 - y0) - (x2 - x0) * (y - y0)) / d
    l2 = ((x1 - x0) * (y - y0) - (x - x0) * (y1 - y0)) / d
    return l1 > 0 and l2 > 0 and l1 + l2 < 1


@pytest.mark.parametrize("k", [2, 3, 4])
def test_patches_equal_brute_force_geometry(k):
    # brute force: a velocity node is in the patch of entity E iff it lies in a closed cell that
    # contains all of E's vertices; a pressure node belongs to E iff it lies on E and not on a
    # lower-dimensional sub-entity (vertex inside an edge, edge inside a cell).
    N = 3
    s = fem.Space(N, k)
    P = patches.build_patches(s)
    mask = s.dirichlet_mask()
    X, Y = s.vnode_xy()
    XP, YP = s.pnode_xy()
    cells = [[(Fraction(a, N), Fraction(b, N)) for a, b in c] for c in s.mesh.cells]
    vx = [(Fraction(int(round(x * k * N)), k * N), Fraction(int(round(y * k * N)), k * N)) for x, y in zip(X, Y)]
    px = [(Fraction(int(round(x * (k - 1) * N)), (k - 1) * N), Fraction(int(round(y * (k - 1) * N)), (k - 1) * N))
          for x, y in zip(XP, YP)]
    for kind, ent, dofs in P:
        E = [(Fraction(a, N), Fraction(b, N)) for a, b in ent]
        star = [c for c in cells if all(v in c for v in E)]
        vel = []
        for n, p in enumerate(vx):
            if any(_point_in_closed_triangle(p, c) for c in star):
                vel += [2 * n, 2 * n + 1]
        vel = [d for d in vel if not mask[d]]
        # pressure nodes on the entity's relative interior
        prs = []
        for n, p in enumerate(px):
            if len(E) == 1:
                on = p == E[0]
            elif len(E) == 2:
                (ax, ay), (bx, by) = E
                cross = (bx - ax) * (p[1] - ay) - (by - ay) * (p[0] - ax)
                t = ((p[0] - ax) * (bx - ax) + (p[1] - ay) * (by - ay)) / ((bx - ax) ** 2 + (by - ay) ** 2)
                on = cross == 0 and 0 < t < 1
            else:
                on = _point_strictly_inside(p, E)
            if on:
                prs.append(s.n_u + n)
        assert list(dofs) == sorted(vel) + sorted(prs), (kind, ent)


# ------------------------------------------------------------------ additive Vanka (Algorithm 1)

def _toy_level(A, patch_dofs, mask):
    class S:
        pass
    space = S()
    space.ndof = A.shape[0]
    space.n_u = A.shape[0]
    return solver.Level(space, sp.csr_matrix(A), mask, [("toy", None, np.array(d)) for d in patch_dofs])


def test_vanka_on_block_diagonal_operator_is_exact_inverse():
    # non-overlapping patches that match the blocks of a block-diagonal matrix: M^{-1} A = I
    rng = np.random.default_rng(3)
    n = 12
    perm = rng.permutation(n)
    groups = [np.sort(perm[:5]), np.sort(perm[5:9]), np.sort(perm[9:])]
    A = np.zeros((n, n))
    for g in groups:
        B = rng.standard_normal((len(g), len(g)))
        A[np.ix_(g, g)] = B @ B.T + len(g) * np.eye(len(g))
    lev = _toy_level(A, groups, np.zeros(n, dtype=bool))
    for _ in range(3):
        x = rng.standard_normal(n)
        assert np.allclose(solver.vanka_apply(lev, A @ x), x, rtol=1e-12, atol=1e-12)


def test_vanka_is_symmetric_and_sums_overlaps():
    s = fem.Space(3, 2)
    A = fem.apply_dirichlet(fem.assemble_full(s), s.dirichlet_mask())
    lev = solver.Level(s, A, s.dirichlet_mask(), patches.build_patches(s))
    n = s.ndof
    M = np.stack([solver.vanka_apply(lev, e) for e in np.eye(n)], axis=1)
    assert np.abs(M - M.T).max() < 1e-10 * np.abs(M).max()
    # a DoF in no patch is only a Dirichlet DoF, where M acts as the identity
    mask = s.dirichlet_mask()
    assert np.array_equal(M[np.ix_(mask, mask)], np.eye(mask.sum()))


@pytest.mark.parametrize("N,k", [(3, 2), (2, 3), (2, 4)])
def test_vanka_weights_on_the_identity_operator(N, k):
    # With A = I every local problem is A_i = I, so Algorithm 1 reduces to sum_i R_i^T W_i R_i r:
    # multiplicity weights (1 / number of patches of the DoF) are a partition of unity, so M^{-1} r = r
    # at every DoF; plain weights give count * r.  The counts come from a brute-force scan of the patch
    # lists; Dirichlet DoFs (in no patch) keep the identity.
    s = fem.Space(N, k)
    mask = s.dirichlet_mask()
    plist = patches.build_patches(s)
    count = np.zeros(s.ndof)
    for _, _, dofs in plist:
        for d in dofs:
            count[d] += 1
    assert np.all((count == 0) == mask)
    I = sp.identity(s.ndof, format="csr")
    r = np.random.default_rng(41).standard_normal(s.ndof)
    zm = solver.vanka_apply(solver.Level(s, I, mask, plist, "multiplicity"), r)
    assert np.allclose(zm, r, rtol=4e-16 * count.max(), atol=0)
    zp = solver.vanka_apply(solver.Level(s, I, mask, plist, "plain"), r)
    want = np.where(mask, r, count * r)
    assert np.allclose(zp, want, rtol=4e-16 * count.max(), atol=0)
    assert count.max() > 1     # overlaps exist, so the two weightings differ


def test_single_patch_vanka_makes_fgmres_converge_in_one_iteration():
    # one patch = all free DoFs but one pressure DoF (pins the pressure): M^{-1} inverts A on its range
    s = fem.Space(3, 2)
    mask = s.dirichlet_mask()
    A = fem.apply_dirichlet(fem.assemble_full(s), mask)
    free = np.flatnonzero(~mask)
    free = free[free != s.ndof - 1]
    lev = solver.Level(s, A, mask, [("all", None, free)])
    b = np.random.default_rng(5).standard_normal(s.ndof)
    res = solver.fgmres(lambda v: A @ v, lambda r: solver.vanka_apply(lev, r), b, 1e-10, 10,
                        lambda v: solver.project(s, v))
    assert res.iters == 1
    assert res.true_res <= 1e-10 * np.linalg.norm(solver.project(s, b))


# ------------------------------------------------------------------ Chebyshev (Sec. 3, Relaxation)

@pytest.mark.parametrize("nu", [1, 2, 3, 5])
def test_chebyshev_error_is_the_scaled_chebyshev_polynomial(nu):
    # A = diag(lams), M = I, b = 0: x_nu = T_nu((theta - lam)/delta) / T_nu(theta/delta) * x_0
    lam_max = 2.0
    lams = np.linspace(0.05, 2.2, 40)
    x0 = np.random.default_rng(2).standard_normal(len(lams))
    x = solver.chebyshev(lambda v: lams * v, lambda r: r, np.zeros_like(x0), x0, lam_max, nu)
    lo, hi = 0.25 * lam_max, 1.1 * lam_max
    theta, delta = (hi + lo) / 2, (hi - lo) / 2
    T = np.polynomial.chebyshev.Chebyshev.basis(nu)
    expect = T((theta - lams) / delta) / T(theta / delta) * x0
    assert np.allclose(x, expect, rtol=1e-12, atol=1e-12)


def test_chebyshev_zero_initial_guess_matches_explicit_zero():
    lams = np.linspace(0.1, 1.0, 9)
    b = np.arange(1.0, 10.0)
    a = solver.chebyshev(lambda v: lams * v, lambda r: r / 2, b, None, 1.0, 3)
    c = solver.chebyshev(lambda v: lams * v, lambda r: r / 2, b, np.zeros(9), 1.0, 3)
    assert np.allclose(a, c, rtol=0, atol=1e-15)


# ------------------------------------------------------------------ eigenvalue estimate

def test_arnoldi_ritz_exact_on_small_invariant_space():
    lams = np.array([0.3, 1.0, 1.7, 2.5, 4.0, 0.9])
    v0 = np.ones(6)
    ritz = solver.arnoldi_ritz(lambda v: lams * v, v0, 10)
    assert abs(np.max(ritz.real) - 4.0) < 1e-12
    assert len(ritz) == 6


def test_arnoldi_ritz_symmetric_lower_bound():
    rng = np.random.default_rng(4)
    B = rng.standard_normal((60, 60))
    S = B @ B.T
    ev = np.linalg.eigvalsh(S)
    ritz = solver.arnoldi_ritz(lambda v: S @ v, rng.standard_normal(60), 10)
    assert np.max(ritz.real) <= ev[-1] * (1 + 1e-12)
    assert np.max(ritz.real) >= 0.8 * ev[-1]


def test_splitmix_published_outputs():
    with open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt")) as f:
        want = [int(l) for l in f if l.strip() and not l.startswith("#")]
    assert [int(v) for v in splitmix.splitmix64(1234567, 5)] == want
    u = splitmix.uniform_pm1(7, 10000)
    assert u.min() >= -1 and u.max() < 1 and abs(u.mean()) < 0.05


# ------------------------------------------------------------------ FGMRES

def test_fgmres_with_exact_preconditioner_takes_one_iteration():
    rng = np.random.default_rng(6)
    A = rng.standard_normal((30, 30)) + 10 * np.eye(30)
    b = rng.standard_normal(30)
    res = solver.fgmres(lambda v: A @ v, lambda r: np.linalg.solve(A, r), b, 1e-12, 5)
    assert res.iters == 1
    assert np.allclose(res.x, np.linalg.solve(A, b), rtol=1e-10)


def test_fgmres_unpreconditioned_converges_within_n_steps():
    rng = np.random.default_rng(7)
    A = rng.standard_normal((25, 25)) + 3 * np.eye(25)
    b = rng.standard_normal(25)
    res = solver.fgmres(lambda v: A @ v, lambda r: r, b, 1e-12, 25)
    assert res.iters <= 25 and res.converged
    assert np.allclose(res.x, np.linalg.solve(A, b), rtol=1e-8, atol=1e-10)
    # the Givens estimate is the true residual of the iterate (exact arithmetic); check at the end
    assert abs(res.hist[-1] - res.true_res) <= 1e-10 * np.linalg.norm(b)
    assert all(res.hist[i + 1] <= res.hist[i] * (1 + 1e-14) for i in range(len(res.hist) - 1))


@pytest.mark.parametrize("orth", ["mgs", "cgs2"])
def test_fgmres_orthogonalisations_pinned_to_direct_solves(orth):
    # both readings of the unspecified orthogonalisation: exact preconditioner -> one iteration; no
    # preconditioner -> at most n steps, iterate = the dense solve, Givens estimate = true residual
    rng = np.random.default_rng(8)
    A = rng.standard_normal((30, 30)) + 10 * np.eye(30)
    b = rng.standard_normal(30)
    res = solver.fgmres(lambda v: A @ v, lambda r: np.linalg.solve(A, r), b, 1e-12, 5, orth=orth)
    assert res.iters == 1 and np.allclose(res.x, np.linalg.solve(A, b), rtol=1e-10)
    A = rng.standard_normal((40, 40)) + 4 * np.eye(40)
    b = rng.standard_normal(40)
    res = solver.fgmres(lambda v: A @ v, lambda r: r, b, 1e-13, 40, orth=orth)
    xd = np.linalg.solve(A, b)
    assert res.converged and res.iters <= 40
    assert np.linalg.norm(res.x - xd) <= 1e-11 * np.linalg.norm(xd)
    assert abs(res.hist[-1] - res.true_res) <= 1e-11 * np.linalg.norm(b)


def test_fgmres_cgs2_matches_mgs_on_a_well_conditioned_system():
    rng = np.random.default_rng(9)
    A = rng.standard_normal((40, 40)) + 4 * np.eye(40)
    b = rng.standard_normal(40)
    r1 = solver.fgmres(lambda v: A @ v, lambda r: r, b, 1e-13, 40, orth="mgs")
    r2 = solver.fgmres(lambda v: A @ v, lambda r: r, b, 1e-13, 40, orth="cgs2")
    xd = np.linalg.solve(A, b)
    for r in (r1, r2):
        assert r.converged and np.linalg.norm(r.x - xd) <= 1e-11 * np.linalg.norm(xd)
        assert abs(r.hist[-1] - r.true_res) <= 1e-11 * np.linalg.norm(b)
    assert r1.iters == r2.iters
    assert np.max(np.abs(np.array(r1.hist) - np.array(r2.hist))) <= 1e-12 * np.linalg.norm(b)
    with pytest.raises(ValueError):
        solver.fgmres(lambda v: A @ v, lambda r: r, b, 1e-13, 40, orth="householder")


def test_multigrid_fgmres_equals_bordered_direct_solve_on_4x4_p2():
    H = solver.Hierarchy(2, 2, 2)   # 2x2 -> 4x4, P2/P1: 187 DoFs on the fine level
    fin = H.finest
    assert fin.space.ndof == 187
    b = np.random.default_rng(0).standard_normal(187)
    res = solver.solve(H, b, 1e-12, 100)
    bp = solver.project(fin.space, b)
    xd = solver.project(fin.space, solver.direct_solve(fin.A, fin.space.nullspace(), bp))
    assert res.converged
    assert np.linalg.norm(res.x - xd) <= 1e-10 * np.linalg.norm(xd)


def test_vcycle_coarse_level_is_exact_bordered_solve():
    H = solver.Hierarchy(2, 1, 2)
    c = H.levels[0]
    b = solver.project(c.space, np.random.default_rng(1).standard_normal(c.space.ndof))
    x = H.vcycle(b)
    assert np.linalg.norm(c.A @ x - b) <= 1e-12 * np.linalg.norm(b)
    assert abs(x[c.space.n_u:].sum()) <= 1e-10 * np.linalg.norm(x)


def _dense_vanka(lev):
    """M^{-1} of Algorithm 1 as a dense matrix: sum_i R_i^T inv(A_i) R_i (+ W_i), identity on Dirichlet
    rows, built from explicit inverses of the dense blocks (no LU solves, no scatter code)."""
    A = lev.A.toarray()
    n = A.shape[0]
    M = np.zeros((n, n))
    for _, _, d in lev.patches:
        M[np.ix_(d, d)] += np.linalg.inv(A[np.ix_(d, d)])
    M = lev.weight[:, None] * M
    M[lev.mask, :] = 0.0
    M[lev.mask, lev.mask] = 1.0
    return M


def _smoother_matrix(lev, Minv, nu):
    """nu Chebyshev steps on [lam/4, 1.1 lam] from a zero guess as a matrix G (x = G b).  The error
    after the steps is q(M^{-1} A) e_0 with q(t) = T_nu((theta - t)/delta) / T_nu(theta/delta) (the
    closed form of the Chebyshev polynomial), so x = s(M^{-1} A) M^{-1} b with s(t) = (1 - q(t)) / t."""
    from numpy.polynomial import Chebyshev, Polynomial
    lam = lev.lam
    lo, hi = 0.25 * lam, 1.1 * lam
    theta, delta = (hi + lo) / 2, (hi - lo) / 2
    T = Chebyshev.basis(nu).convert(kind=Polynomial)
    q = T(Polynomial([theta / delta, -1.0 / delta])) / T(theta / delta)
    one_minus_q = Polynomial([1.0]) - q
    assert abs(one_minus_q.coef[0]) < 1e-14
    s_coef = one_minus_q.coef[1:]
    X = Minv @ lev.A.toarray()
    S = np.zeros_like(X)
    for c in s_coef[::-1]:                      # Horner in the matrix X
        S = S @ X + c * np.eye(len(X))
    return S @ Minv


def _vcycle_matrix(H, l=None):
    """The V(nu, nu) cycle of Sec. 3 as a matrix B (x = B b), composed from dense pieces: pre-smoothing
    G, coarse correction K = P B_c D_c R (D_c zeroes the coarse Dirichlet entries), post-smoothing G;
    the coarsest level is the top-left block of the inverse of the bordered matrix."""
    if l is None:
        l = len(H.levels) - 1
    lev = H.levels[l]
    if l == 0:
        n = lev.A.shape[0]
        z = lev.space.nullspace()
        Bd = np.zeros((n + 1, n + 1))
        Bd[:n, :n] = lev.A.toarray()
        Bd[:n, n] = z
        Bd[n, :n] = z
        return np.linalg.inv(Bd)[:n, :n]
    A = lev.A.toarray()
    I = np.eye(A.shape[0])
    G = _smoother_matrix(lev, _dense_vanka(lev), H.sweeps)
    Dc = np.diag((~H.levels[l - 1].mask).astype(float))
    K = lev.P.toarray() @ _vcycle_matrix(H, l - 1) @ Dc @ lev.R.toarray()
    X1 = G                                      # x1 = G b
    X2 = X1 + K @ (I - A @ X1)                  # x2 = x1 + K (b - A x1)
    return X2 + G @ (I - A @ X2)                # x3 = x2 + G (b - A x2)


@pytest.mark.parametrize("Nc,L,k,nu", [(2, 2, 2, 1), (2, 2, 2, 2), (2, 2, 3, 1), (2, 2, 3, 2), (2, 3, 2, 1)])
def test_vcycle_equals_its_dense_composition(Nc, L, k, nu):
    H = solver.Hierarchy(Nc, L, k, sweeps=nu)
    fin = H.finest
    B = _vcycle_matrix(H)
    rng = np.random.default_rng(43)
    for _ in range(2):
        b = rng.standard_normal(fin.space.ndof)
        want = B @ b
        dev = np.linalg.norm(H.vcycle(b) - want) / np.linalg.norm(want)
        assert dev <= 1e-13, dev
    if L == 2:
        # two levels: x = (I - E) A^+ b_hat with E = S_post C S_pre the error propagation operator
        A = fin.A.toarray()
        E = np.eye(len(A)) - B @ A
        bh = solver.project(fin.space, rng.standard_normal(fin.space.ndof))
        xs = np.linalg.lstsq(A, bh, rcond=None)[0]
        assert np.linalg.norm(H.vcycle(bh) - (xs - E @ xs)) <= 1e-10 * np.linalg.norm(xs)


def test_vcycle_pin_detects_planted_mistakes(monkeypatch):
    # the dense-composition pin must fail for a cycle that skips post-smoothing or the zeroing of the
    # coarse Dirichlet entries after restriction (mistakes planted in the oracle, on the CPU)
    H = solver.Hierarchy(2, 2, 2, sweeps=1)
    B = _vcycle_matrix(H)
    b = np.random.default_rng(44).standard_normal(H.finest.space.ndof)
    want = B @ b
    assert np.linalg.norm(H.vcycle(b) - want) <= 1e-13 * np.linalg.norm(want)
    orig_smooth = H.smooth
    monkeypatch.setattr(H, "smooth", lambda l, bb, x: x if x is not None else orig_smooth(l, bb, x))
    assert np.linalg.norm(H.vcycle(b) - want) > 1e-1 * np.linalg.norm(want)
    monkeypatch.setattr(H, "smooth", orig_smooth)
    coarse = H.levels[0]
    monkeypatch.setattr(coarse, "mask", np.zeros_like(coarse.mask))
    assert np.linalg.norm(H.vcycle(b) - want) > 1e-2 * np.linalg.norm(want)


def test_vcycle_is_a_contraction_config1():
    # two-level V(1,1) as a stationary iteration must reduce the error of A x = b
    H = solver.Hierarchy(4, 2, 2)
    fin = H.finest
    b = solver.project(fin.space, np.random.default_rng(2).standard_normal(fin.space.ndof))
    x = np.zeros_like(b)
    r0 = np.linalg.norm(b)
    for _ in range(30):
        x = x + solver.project(fin.space, H.vcycle(b - fin.A @ x))
    assert np.linalg.norm(b - fin.A @ x) < 1e-3 * r0


# ------------------------------------------------------------------ discretization (Theorem 2.1)

def _manufactured_errors(N, k):
    s = fem.Space(N, k)
    K = fem.assemble_full(s)
    mask = s.dirichlet_mask()
    A = fem.apply_dirichlet(K, mask)
    b = fem.manufactured_rhs(s, K)
    b = solver.project(s, b)
    x = solver.direct_solve(A, s.nullspace(), b)
    return fem.errors(s, x)


@pytest.mark.parametrize("k,Ns", [(2, (8, 16, 32)), (3, (4, 8, 16)), (4, (2, 4, 8))])
def test_manufactured_convergence_rates(k, Ns):
    errs = [_manufactured_errors(N, k) for N in Ns]
    rates = [[np.log2(errs[i][j] / errs[i + 1][j]) for j in range(3)] for i in range(len(Ns) - 1)]
    h1, l2, pl2 = rates[-1]
    assert h1 > k - 0.15, rates          # velocity H^1: O(h^k)   (Theorem 2.1 with TH interpolation)
    assert l2 > k + 1 - 0.25, rates      # velocity L^2: O(h^{k+1}) (duality)
    assert pl2 > k - 0.25, rates         # pressure L^2: O(h^k)   (Theorem 2.1)


def test_manufactured_rhs_solved_by_multigrid_fgmres_config1():
    H = solver.Hierarchy(4, 2, 2)
    fin = H.finest
    b = fem.manufactured_rhs(fin.space, fin.K)
    res = solver.solve(H, b, 1e-10, 100)
    assert res.converged and res.iters < 100
    xd = solver.direct_solve(fin.A, fin.space.nullspace(), solver.project(fin.space, b))
    xd = solver.project(fin.space, xd)
    assert np.linalg.norm(res.x - xd) <= 1e-8 * np.linalg.norm(xd)
    h1, l2, p = fem.errors(fin.space, res.x)
    h1d, l2d, pd = fem.errors(fin.space, xd)
    assert abs(h1 - h1d) <= 1e-6 * h1d and abs(l2 - l2d) <= 1e-6 * l2d
    assert h1 < 0.02 and l2 < 2e-3


@pytest.mark.slow
def test_paper_soft_pin_p3_nu4_four_refinements():
    # Sec. 4.1: TH P3/P2, nu = 4, l = 4 (5x5 -> 80x80) needs 26 FGMRES iterations to 1e-10.
    with open(os.path.join(GOLDEN, "paper_iteration_counts.txt")) as f:
        rows = [list(map(int, l.split())) for l in f if l.strip() and not l.startswith("#")]
    k, nu, lref, Nc, iters = rows[0]
    H = solver.Hierarchy(Nc, lref + 1, k, sweeps=nu)
    fin = H.finest
    b = fem.manufactured_rhs(fin.space, fin.K)
    res = solver.solve(H, b, 1e-10, 100)
    assert res.converged
    assert 0.5 * iters <= res.iters <= 1.6 * iters, res.iters
