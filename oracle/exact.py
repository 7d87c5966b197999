"""Exact rational P_k Lagrange basis on the reference triangle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The Taylor-Hood pair of Case 1 (Sec. 3) uses continuous P_k velocity and P_{k-1} pressure on
triangles (Sec. 2, the paragraph defining P_k and the Taylor-Hood pairs).  The paper never states the
node placement; the reading used here is equispaced Lagrange nodes, which on the structured mesh make
the global nodes exactly a lattice.

The reference triangle is T^ = {(x, y): x >= 0, y >= 0, x + y <= 1}.  The basis is obtained by
inverting the monomial Vandermonde matrix in exact rationals, and integrals use the closed form
    int_T^ x^p y^q = p! q! / (p + q + 2)!
so every reference matrix is an exact rational.
"""
from fractions import Fraction
from functools import lru_cache
from math import factorial


def lattice_nodes(k):
    """Reference nodes (s/k, t/k), s + t <= k, ordered t-major then s (lexicographic, s fastest).

    Returned as integer pairs (s, t); the point is (s/k, t/k).  For k = 0 the single node is the
    centroid-free constant case and is returned as [(0, 0)]."""
    return [(s, t) for t in range(k + 1) for s in range(k + 1 - t)]


def monomials(k):
    return [(p, q) for q in range(k + 1) for p in range(k + 1 - q)]


def _solve_exact(M, B):
    """Gauss-Jordan elimination over the rationals: returns X with M X = B (lists of lists)."""
    n = len(M)
    m = len(B[0])
    A = [list(M[i]) + list(B[i]) for i in range(n)]
    for c in range(n):
        piv = next(r for r in range(c, n) if A[r][c] != 0)
        A[c], A[piv] = A[piv], A[c]
        pv = A[c][c]
        A[c] = [v / pv for v in A[c]]
        for r in range(n):
            if r != c and A[r][c] != 0:
                f = A[r][c]
                A[r] = [a - f * b for a, b in zip(A[r], A[c])]
    return [row[n:n + m] for row in A]


@lru_cache(maxsize=None)
def basis(k):
    """P_k Lagrange basis as a tuple of polynomials; each polynomial is a dict {(p, q): Fraction}.

    basis(k)[i] is 1 at lattice_nodes(k)[i] and 0 at the other nodes."""
    nodes = lattice_nodes(k)
    mons = monomials(k)
    if k == 0:
        return ({(0, 0): Fraction(1)},)
    V = [[Fraction(s, k) ** p * Fraction(t, k) ** q for (p, q) in mons] for (s, t) in nodes]
    n = len(nodes)
    eye = [[Fraction(int(i == j)) for j in range(n)] for i in range(n)]
    C = _solve_exact(V, eye)  # V C = I  => column i of C holds the coefficients of basis i
    out = []
    for i in range(n):
        poly = {mons[m]: C[m][i] for m in range(len(mons)) if C[m][i] != 0}
        out.append(poly)
    return tuple(out)


def deriv(poly, var):
    """d/dx (var = 0) or d/dy (var = 1) of a polynomial dict."""
    out = {}
    for (p, q), c in poly.items():
        if var == 0 and p > 0:
            out[(p - 1, q)] = out.get((p - 1, q), 0) + c * p
        elif var == 1 and q > 0:
            out[(p, q - 1)] = out.get((p, q - 1), 0) + c * q
    return out


def mul(a, b):
    out = {}
    for (p1, q1), c1 in a.items():
        for (p2, q2), c2 in b.items():
            key = (p1 + p2, q1 + q2)
            out[key] = out.get(key, 0) + c1 * c2
    return out


def integrate_ref(poly):
    """Exact integral over the reference triangle: int x^p y^q = p! q! / (p+q+2)!."""
    tot = Fraction(0)
    for (p, q), c in poly.items():
        tot += c * Fraction(factorial(p) * factorial(q), factorial(p + q + 2))
    return tot


def evaluate(poly, x, y):
    return sum(c * x ** p * y ** q for (p, q), c in poly.items())


@lru_cache(maxsize=None)
def grad_grad(k):
    """G[m][n][a][b] = int_T^ d_m phi_a d_n phi_b  (exact)."""
    B = basis(k)
    dB = [[deriv(f, v) for f in B] for v in (0, 1)]
    nb = len(B)
    return tuple(tuple(tuple(tuple(integrate_ref(mul(dB[m][a], dB[n][b])) for b in range(nb))
                             for a in range(nb)) for n in (0, 1)) for m in (0, 1))


@lru_cache(maxsize=None)
def pressure_div(k):
    """K[m][q][a] = int_T^ psi_q d_m phi_a, psi in P_{k-1}, phi in P_k (exact)."""
    B = basis(k)
    Q = basis(k - 1)
    dB = [[deriv(f, v) for f in B] for v in (0, 1)]
    return tuple(tuple(tuple(integrate_ref(mul(Q[q], dB[m][a])) for a in range(len(B)))
                       for q in range(len(Q))) for m in (0, 1))


def monomial_coeff_matrix(k):
    """Float coefficient matrix C (n_mon x n_basis) with phi_i(x, y) = sum_m C[m, i] x^p_m y^q_m."""
    import numpy as np
    mons = monomials(k)
    B = basis(k)
    C = np.zeros((len(mons), len(B)))
    for i, f in enumerate(B):
        for m, pq in enumerate(mons):
            C[m, i] = float(f.get(pq, 0))
    return mons, C
