"""Pins of the oracle's discretisation-error integrals (Sec. 4.4; errors against Eq. model_problem) for
the three discretisations: for a polynomial velocity u_p of degree <= k and pressure p_p of degree <= k-1,
which every space reproduces exactly through its interpolant, the relative H^1 and L^2 velocity errors
and the L^2 pressure error after removing the mean equal their closed forms on the unit square,
integrated symbolically against u = (sin pi x cos pi y, -cos pi x sin pi y), p = 0."""
import numpy as np
import pytest

from oracle import bdm, fem, quad

sympy = pytest.importorskip("sympy")
X, Y = sympy.symbols("x y")


def closed_forms(up, pp):
    u = (sympy.sin(sympy.pi * X) * sympy.cos(sympy.pi * Y), -sympy.cos(sympy.pi * X) * sympy.sin(sympy.pi * Y))
    I = lambda f: sympy.integrate(sympy.integrate(sympy.expand(f), (X, 0, 1)), (Y, 0, 1))
    e_l2 = sum(I((up[c] - u[c]) ** 2) for c in (0, 1))
    n_l2 = sum(I(u[c] ** 2) for c in (0, 1))
    e_h1 = sum(I(sympy.diff(up[c] - u[c], v) ** 2) for c in (0, 1) for v in (X, Y))
    n_h1 = sum(I(sympy.diff(u[c], v) ** 2) for c in (0, 1) for v in (X, Y))
    mean = I(pp)
    p_err = I((pp - mean) ** 2)
    return (float(sympy.sqrt((e_l2 + e_h1) / (n_l2 + n_h1))), float(sympy.sqrt(e_l2 / n_l2)), float(sympy.sqrt(p_err)))


def fields(k):
    up = (X ** k - 2 * X * Y ** (k - 1) + sympy.Rational(1, 2), Y ** k + X ** (k - 1) * Y - sympy.Rational(1, 4))
    pp = X ** (k - 1) + 3 * X * Y ** max(k - 2, 0) - 1 if k > 1 else sympy.Integer(2)
    return up, pp


def as_np(expr):
    f = sympy.lambdify((X, Y), expr, "numpy")
    return lambda a, b: f(a, b) + 0 * a


@pytest.mark.parametrize("cell,N,k", [("tri", 3, 2), ("tri", 2, 3), ("quad", 3, 2), ("quad", 2, 3),
                                      ("bdm", 3, 2), ("bdm", 2, 3)])
def test_error_integrals_equal_closed_forms(cell, N, k):
    up, pp = fields(k)
    want = closed_forms(up, pp)
    fu = [as_np(e) for e in up]
    fp = as_np(pp)
    if cell == "bdm":
        s = bdm.BDMSpace(N, k)
        x = bdm.interpolate(s, lambda a, b: (fu[0](a, b), fu[1](a, b)), fp)
        got = bdm.errors(s, x)
    else:
        s = (quad.QSpace if cell == "quad" else fem.Space)(N, k)
        x = np.zeros(s.ndof)
        vx, vy = s.vnode_xy()
        x[0:s.n_u:2] = fu[0](vx, vy)
        x[1:s.n_u:2] = fu[1](vx, vy)
        px, py = s.pnode_xy()
        x[s.n_u:] = fp(px, py)
        got = (quad.errors if cell == "quad" else fem.errors)(s, x)
    for g, w in zip(got, want):
        assert abs(g - w) <= 1e-10 * max(w, 1e-12), (cell, got, want)
