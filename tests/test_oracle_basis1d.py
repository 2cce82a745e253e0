"""Pins for the oracle's 1D building blocks (Sec. 2.2, Eq. element_matrices).

Each check compares against a closed form or an identity of the calculus,
not against the oracle's own formulas.
"""
import math
import os

import numpy as np
import pytest

from oracle.basis1d import Matrices1D, gll_nodes, lagrange

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "gll_closed_forms.txt")


def _parse(tok):
    tok = tok.strip()
    sgn = -1.0 if tok.startswith("-") else 1.0
    tok = tok.lstrip("-")
    if tok.startswith("sqrt("):
        return sgn * math.sqrt(_parse(tok[5:-1]))
    if "/" in tok:
        a, b = tok.split("/")
        return sgn * float(a) / float(b)
    return sgn * float(tok)


def _golden_rows():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        n, pts, wts = line.split("|")
        rows.append((int(n), [_parse(t) for t in pts.split(",")], [_parse(t) for t in wts.split(",")]))
    return rows


@pytest.mark.parametrize("n,pts,wts", _golden_rows())
def test_gll_closed_forms(n, pts, wts):
    x, w = gll_nodes(n)
    np.testing.assert_allclose(x, pts, atol=1e-15)
    np.testing.assert_allclose(w, wts, atol=1e-15)


@pytest.mark.parametrize("n", [6, 9, 13, 17])
def test_gll_rule_exactness(n):
    # the GLL rule integrates polynomials of degree <= 2n - 3 exactly
    x, w = gll_nodes(n)
    for deg in range(2 * n - 2):
        exact = 0.0 if deg % 2 else 2.0 / (deg + 1)
        assert abs(w @ x ** deg - exact) < 2e-14


@pytest.mark.parametrize("p", [1, 2, 5, 8, 16])
def test_lagrange_cardinal_and_derivative(p):
    x, _ = gll_nodes(p + 1)
    V, _ = lagrange(x, x)
    np.testing.assert_allclose(V, np.eye(p + 1), atol=1e-13)
    t = np.linspace(-0.97, 0.93, 11)
    V, dV = lagrange(x, t)
    np.testing.assert_allclose(V.sum(1), 1.0, atol=1e-12)
    np.testing.assert_allclose(dV.sum(1), 0.0, atol=1e-10)
    for a in range(1, p + 1):
        np.testing.assert_allclose(dV @ x ** a, a * t ** (a - 1), atol=1e-9)


def _int_monomial(k):
    return 0.0 if k % 2 else 2.0 / (k + 1)


@pytest.mark.parametrize("p", [1, 2, 3, 6, 10])
def test_mass_and_derivative_moments(p):
    m = Matrices1D(p, tau_hat=1.0)
    x = m.nodes
    for a in range(p + 1):
        for b in range(p + 1):
            ua, ub = x ** a, x ** b
            # M_ij = int phi_i phi_j  =>  ub^T M ua = int x^(a+b)
            assert abs(ub @ m.M @ ua - _int_monomial(a + b)) < 1e-13
            # D_ij = int phi_i phi_j'  =>  ub^T D ua = int x^b (x^a)'
            want = a * _int_monomial(a + b - 1) if a > 0 else 0.0
            assert abs(ub @ m.D @ ua - want) < 1e-12


@pytest.mark.parametrize("p", [1, 3, 7])
def test_integration_by_parts(p):
    m = Matrices1D(p, tau_hat=1.0)
    n = p + 1
    bnd = np.zeros((n, n))
    bnd[0, 0], bnd[-1, -1] = -1.0, 1.0
    np.testing.assert_allclose(m.D + m.D.T, bnd, atol=1e-13)


@pytest.mark.parametrize("p", [2, 4])
def test_gll_lumped_mass(p):
    m = Matrices1D(p, tau_hat=1.0, mass="gll")
    _, w = gll_nodes(p + 1)
    np.testing.assert_allclose(m.M, np.diag(w))
    x = m.nodes
    # exact for products up to degree 2p - 1, not for degree 2p
    for a in range(p + 1):
        for b in range(p + 1):
            err = abs((x ** b) @ m.M @ (x ** a) - _int_monomial(a + b))
            if a + b <= 2 * p - 1:
                assert err < 1e-13
    assert abs((x ** p) @ m.M @ (x ** p) - _int_monomial(2 * p)) > 1e-3


@pytest.mark.parametrize("p,tau", [(1, 2.0), (4, 25.0)])
def test_boundary_matrices_closed_form(p, tau):
    m = Matrices1D(p, tau_hat=tau)
    n = p + 1
    e0, en = np.eye(n)[0], np.eye(n)[-1]
    np.testing.assert_allclose(m.E, tau * (np.outer(e0, e0) + np.outer(en, en)), atol=1e-13)
    np.testing.assert_allclose(m.G, tau * np.eye(2), atol=1e-15)
    np.testing.assert_allclose(m.B, -tau * np.stack([e0, en], 1), atol=1e-13)
    np.testing.assert_allclose(m.C, np.stack([-e0, en], 1), atol=1e-13)
    # L = E + D M^-1 D^T is symmetric positive definite
    np.testing.assert_allclose(m.L, m.L.T, atol=1e-12)
    assert np.linalg.eigvalsh(m.L).min() > 0
