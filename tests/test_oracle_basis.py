"""Pins for the exact P_k basis and reference integrals (oracle/exact.py)."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import exact, fem


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_kronecker_at_nodes(k):
    nodes = exact.lattice_nodes(k)
    B = exact.basis(k)
    for i, f in enumerate(B):
        for j, (s, t) in enumerate(nodes):
            assert exact.evaluate(f, Fraction(s, k), Fraction(t, k)) == (1 if i == j else 0)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_reproduces_every_monomial(k):
    # sum_i p(node_i) phi_i == p for every monomial p of degree <= k (at random rational points)
    nodes = exact.lattice_nodes(k)
    B = exact.basis(k)
    pts = [(Fraction(1, 7), Fraction(2, 9)), (Fraction(3, 11), Fraction(5, 13)), (Fraction(0), Fraction(1, 3))]
    for p, q in exact.monomials(k):
        for x, y in pts:
            val = sum(Fraction(s, k) ** p * Fraction(t, k) ** q * exact.evaluate(f, x, y)
                      for (s, t), f in zip(nodes, B))
            assert val == x ** p * y ** q


def test_reference_integrals_textbook_values():
    # area 1/2, first moments 1/6, second moments 1/12 and 1/24 of the unit right triangle
    assert exact.integrate_ref({(0, 0): Fraction(1)}) == Fraction(1, 2)
    assert exact.integrate_ref({(1, 0): Fraction(1)}) == Fraction(1, 6)
    assert exact.integrate_ref({(0, 1): Fraction(1)}) == Fraction(1, 6)
    assert exact.integrate_ref({(2, 0): Fraction(1)}) == Fraction(1, 12)
    assert exact.integrate_ref({(1, 1): Fraction(1)}) == Fraction(1, 24)


@pytest.mark.parametrize("p,q", [(0, 0), (3, 1), (2, 4), (5, 0), (1, 6)])
def test_reference_integrals_vs_gauss(p, q):
    x, y, w = fem.ref_quadrature(8)
    assert abs(float(exact.integrate_ref({(p, q): Fraction(1)})) - np.sum(w * x ** p * y ** q)) < 1e-15


def test_collapsed_gauss_rule_on_triangle_area_and_centroid():
    x, y, w = fem.ref_quadrature(3)
    assert abs(w.sum() - 0.5) < 1e-15
    assert abs((w * x).sum() / w.sum() - 1 / 3) < 1e-15
    assert abs((w * y).sum() / w.sum() - 1 / 3) < 1e-15
