"""Pins of the oracle's 1D rules against closed forms and library routines."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import rules

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _eval(expr):
    return float(eval(expr, {"sqrt": math.sqrt}))


def test_closed_forms_from_golden_file():
    with open(os.path.join(GOLDEN, "rules_closed_forms.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            kind, nk, idx, node, weight = line.split()
            nk, idx = int(nk), int(idx)
            if kind == "gauss":
                x, w = rules.gauss_legendre(nk)
                assert abs(x[idx] - _eval(node)) < 1e-15
                assert abs(w[idx] - _eval(weight)) < 1e-15
            else:
                x = rules.gauss_lobatto(nk)
                assert abs(x[idx] - _eval(node)) < 1e-15


@pytest.mark.parametrize("n", range(1, 13))
def test_gauss_matches_numpy_leggauss(n):
    x, w = rules.gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.allclose(x, 0.5 * (xr + 1), atol=2e-16, rtol=0)
    assert np.allclose(w, 0.5 * wr, atol=1e-15, rtol=0)
    assert abs(w.sum() - 1.0) < 1e-15


@pytest.mark.parametrize("n", range(1, 11))
def test_gauss_exactness_degree(n):
    x, w = rules.gauss_legendre(n)
    for m in range(2 * n):
        assert abs(np.dot(w, x ** m) - 1.0 / (m + 1)) < 1e-14
    # one degree higher is no longer exact
    assert abs(np.dot(w, x ** (2 * n)) - 1.0 / (2 * n + 1)) > 1e-13


@pytest.mark.parametrize("k", range(2, 10))
def test_lobatto_are_roots_of_legendre_derivative(k):
    x = rules.gauss_lobatto(k)
    roots = np.sort(np.polynomial.legendre.Legendre.basis(k).deriv().roots().real)
    assert np.allclose(x[1:-1], 0.5 * (roots + 1), atol=1e-14)
    assert x[0] == 0.0 and x[-1] == 1.0
    if k % 2 == 0:
        assert x[k // 2] == 0.5


@pytest.mark.parametrize("k", range(1, 9))
def test_lagrange_delta_partition_and_derivative(k):
    nodes = rules.gauss_lobatto(k)
    n = k + 1
    for i in range(n):
        for j in range(n):
            assert rules.lagrange(nodes, j, nodes[i]) == (1.0 if i == j else 0.0)
    t = np.linspace(0, 1, 17)
    s = sum(rules.lagrange(nodes, j, t) for j in range(n))
    ds = sum(rules.lagrange_deriv(nodes, j, t) for j in range(n))
    assert np.allclose(s, 1.0, atol=1e-13)
    assert np.allclose(ds, 0.0, atol=1e-11)
    # derivative against numpy's polynomial class built from the roots
    for j in range(n):
        others = [nodes[m] for m in range(n) if m != j]
        p = np.polynomial.Polynomial.fromroots(others)
        p = p / p(nodes[j])
        # the power-basis reference loses digits as k grows
        tol = 1e-12 * 10.0 ** max(0, k - 4)
        assert np.allclose(rules.lagrange(nodes, j, t), p(t), atol=tol)
        assert np.allclose(rules.lagrange_deriv(nodes, j, t), p.deriv()(t), atol=100 * tol)


def test_lagrange_rational_k2():
    # k = 2: nodes {0, 1/2, 1}; l_0(x) = 2 (x - 1/2)(x - 1), l_1 = -4 x (x - 1), l_2 = 2 x (x - 1/2)
    nodes = rules.gauss_lobatto(2)
    for x in (0.1, 0.25, 0.8):
        X = Fraction(x)
        ref = [2 * (X - Fraction(1, 2)) * (X - 1), -4 * X * (X - 1), 2 * X * (X - Fraction(1, 2))]
        dref = [4 * X - 3, -8 * X + 4, 4 * X - 1]
        for j in range(3):
            assert abs(rules.lagrange(nodes, j, x) - float(ref[j])) < 1e-15
            assert abs(rules.lagrange_deriv(nodes, j, x) - float(dref[j])) < 1e-14


@pytest.mark.parametrize("k", range(1, 9))
def test_nodes_and_points_are_the_correctly_rounded_roots(k):
    """Each GLL node and Gauss point is the FP64 number nearest to the root that defines it (interior
    GLL nodes: roots of P_k'; Gauss points: roots of P_{k+1}; both mapped to [0, 1]), checked against
    roots computed independently to 50 digits.  Equal nodes on both sides of the parity tests rest on this."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    nodes = rules.gauss_lobatto(k)
    assert nodes[0] == 0.0 and nodes[-1] == 1.0
    for i in range(1, k):
        r = mp.findroot(lambda t: mp.diff(lambda s: mp.legendre(k, s), t), 2 * mp.mpf(nodes[i]) - 1)
        assert float((r + 1) / 2) == nodes[i], (k, i)
    n = k + 1
    x, _ = rules.gauss_legendre(n)
    for i in range(n):
        r = mp.findroot(lambda t: mp.legendre(n, t), 2 * mp.mpf(x[i]) - 1)
        assert float((r + 1) / 2) == x[i], (n, i)
