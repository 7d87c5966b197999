"""Pins for the oracle's assembly (oracle/fem.py): exact energies of polynomial fields, divergence
moments, symmetry, the constant-pressure nullspace, Dirichlet rows, and the canonical transfers."""
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fem


def square_integral(poly):
    """Exact integral over the unit square of a polynomial dict {(a, b): coeff}."""
    return sum(Fraction(c) / ((a + 1) * (b + 1)) for (a, b), c in poly.items())


def pmul(p, q):
    out = {}
    for (a1, b1), c1 in p.items():
        for (a2, b2), c2 in q.items():
            out[(a1 + a2, b1 + b2)] = out.get((a1 + a2, b1 + b2), 0) + Fraction(c1) * c2
    return out


def padd(*ps):
    out = {}
    for p in ps:
        for key, c in p.items():
            out[key] = out.get(key, 0) + Fraction(c)
    return out


def pscale(p, s):
    return {key: Fraction(c) * s for key, c in p.items()}


def pd(p, var):
    out = {}
    for (a, b), c in p.items():
        if var == 0 and a:
            out[(a - 1, b)] = out.get((a - 1, b), 0) + c * a
        if var == 1 and b:
            out[(a, b - 1)] = out.get((a, b - 1), 0) + c * b
    return out


def peval(p, x, y):
    return sum(c * x ** a * y ** b for (a, b), c in p.items())


def interp_velocity(space, u1, u2):
    X, Y = space.vnode_xy()
    v = np.zeros(space.ndof)
    v[0:space.n_u:2] = [float(peval(u1, x, y)) for x, y in zip(X, Y)]
    v[1:space.n_u:2] = [float(peval(u2, x, y)) for x, y in zip(X, Y)]
    return v


def interp_pressure(space, q):
    X, Y = space.pnode_xy()
    v = np.zeros(space.ndof)
    v[space.n_u:] = [float(peval(q, x, y)) for x, y in zip(X, Y)]
    return v


CASES = [
    # (k, u1, u2, q): velocity of degree <= k, pressure of degree <= k-1
    (2, {(2, 0): 1, (0, 1): 3}, {(1, 1): -2, (0, 2): 1}, {(1, 0): 2, (0, 0): 1}),
    (3, {(2, 1): 1, (0, 3): -1}, {(3, 0): 2, (1, 1): 1}, {(1, 1): 3, (0, 2): -1}),
    (4, {(2, 2): 1, (4, 0): 1}, {(1, 3): -1, (0, 1): 5}, {(3, 0): 1, (1, 2): 2}),
]


@pytest.mark.parametrize("k,u1,u2,q", CASES)
def test_energy_and_divergence_of_polynomial_fields(k, u1, u2, q):
    # u_I^T A u_I = 2 nu int eps(u):eps(u) and q_I^T B u_I = -int (div u) q, exactly on the unit square
    nu = 1.7
    space = fem.Space(3, k)
    K = fem.assemble_full(space, nu)
    u = interp_velocity(space, u1, u2)
    p = interp_pressure(space, q)
    e11, e22 = pd(u1, 0), pd(u2, 1)
    e12 = pscale(padd(pd(u1, 1), pd(u2, 0)), Fraction(1, 2))
    energy = 2 * nu * float(square_integral(padd(pmul(e11, e11), pmul(e22, e22), pscale(pmul(e12, e12), 2))))
    assert abs(u @ (K @ u) - energy) <= 1e-12 * abs(energy)
    div = padd(e11, e22)
    bq = -float(square_integral(pmul(div, q)))
    assert abs(p @ (K @ u) - bq) <= 1e-12 * max(1.0, abs(bq))
    # the same moment from the transposed block
    assert abs(u @ (K @ p) - bq) <= 1e-12 * max(1.0, abs(bq))


@pytest.mark.parametrize("k", [2, 3, 4])
def test_rigid_motions_are_in_the_kernel_of_A(k):
    space = fem.Space(2, k)
    K = fem.assemble_full(space)
    X, Y = space.vnode_xy()
    for u1, u2 in ((1 + 0 * X, 0 * X), (0 * X, 1 + 0 * X), (-Y, X)):
        v = np.zeros(space.ndof)
        v[0:space.n_u:2] = u1
        v[1:space.n_u:2] = u2
        assert np.abs((K @ v)[:space.n_u]).max() < 1e-13


@pytest.mark.parametrize("N,k", [(4, 2), (3, 3), (2, 4)])
def test_symmetry_nullspace_and_dirichlet_rows(N, k):
    space = fem.Space(N, k)
    K = fem.assemble_full(space)
    mask = space.dirichlet_mask()
    A = fem.apply_dirichlet(K, mask)
    assert abs(K - K.T).max() == 0.0
    assert abs(A - A.T).max() == 0.0
    z = space.nullspace()
    assert np.abs(A @ z).max() < 1e-13 * abs(A).max()
    D = A[mask].toarray()
    assert np.array_equal(D, np.eye(space.ndof)[mask])
    assert np.count_nonzero(A[:, mask].toarray()[~mask]) == 0
    # the pressure-pressure block is empty
    assert abs(A[space.n_u:, space.n_u:]).max() == 0
    # number of boundary velocity nodes
    assert mask.sum() == 2 * 4 * k * N


@pytest.mark.parametrize("Nc,k", [(2, 2), (2, 3), (1, 4)])
def test_prolongation_reproduces_coarse_polynomials(Nc, k):
    c, f = fem.Space(Nc, k), fem.Space(2 * Nc, k)
    P = fem.prolongation(c, f)
    rng = np.random.default_rng(1)
    for deg, interp, block in ((k, interp_velocity, slice(0, c.n_u)), (k - 1, None, None)):
        mons = [(a, b) for b in range(deg + 1) for a in range(deg + 1 - b)]
        coef = {m: Fraction(int(rng.integers(-3, 4))) for m in mons}
        if interp is not None:
            coef2 = {m: Fraction(int(rng.integers(-3, 4))) for m in mons}
            vc, vf = interp_velocity(c, coef, coef2), interp_velocity(f, coef, coef2)
            err = np.abs(P @ vc - vf)[:f.n_u].max()
        else:
            vc, vf = interp_pressure(c, coef), interp_pressure(f, coef)
            err = np.abs(P @ vc - vf)[f.n_u:].max()
        assert err < 1e-12


@pytest.mark.parametrize("Nc,k", [(2, 2), (4, 2), (2, 3), (2, 4)])
def test_galerkin_equals_rediscretization(Nc, k):
    # conforming nested spaces: P^T K_fine P == K_coarse (Sec. 3, coarse-grid operators)
    c, f = fem.Space(Nc, k), fem.Space(2 * Nc, k)
    Kc, Kf = fem.assemble_full(c), fem.assemble_full(f)
    P = fem.prolongation(c, f)
    G = (P.T @ Kf @ P).tocsr()
    assert abs(G - Kc).max() <= 1e-12 * abs(Kc).max()
    # and on the free block with Dirichlet rows
    mc, mf = c.dirichlet_mask(), f.dirichlet_mask()
    Ac, Af = fem.apply_dirichlet(Kc, mc), fem.apply_dirichlet(Kf, mf)
    Pff = P[~mf][:, ~mc]
    assert abs(Pff.T @ Af[~mf][:, ~mf] @ Pff - Ac[~mc][:, ~mc]).max() <= 1e-12 * abs(Ac).max()
    # fine boundary rows take values from coarse boundary columns only
    assert abs(P[mf][:, ~mc]).max() == 0


def test_element_count_and_sizes():
    for N, k in [(8, 2), (16, 2), (4, 3), (4, 4)]:
        s = fem.Space(N, k)
        assert s.ndof == 2 * (k * N + 1) ** 2 + ((k - 1) * N + 1) ** 2
        assert len(s.mesh.cells) == 2 * N * N
    # 128^2 P2/P1: 132,098 velocity + 16,641 pressure DoFs
    s = fem.Space(128, 2)
    assert (s.n_u, s.n_p) == (132098, 16641)
