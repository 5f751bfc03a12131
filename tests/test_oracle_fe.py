"""Pins of the oracle's finite-element tables (oracle/fe.py) against closed forms."""
import numpy as np
import pytest

from oracle.fe import CellTables, gauss01, lagrange1d


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_gauss_exact_degree(n):
    x, w = gauss01(n)
    for deg in range(2 * n):
        assert abs(np.dot(w, x ** deg) - 1.0 / (deg + 1)) < 1e-14


@pytest.mark.parametrize("k", [1, 2])
def test_lagrange_kronecker_and_derivative(k):
    t = np.arange(k + 1) / k
    L, dL = lagrange1d(k, t)
    assert np.allclose(L, np.eye(k + 1), atol=1e-15)
    # derivative against central differences of the values
    x = np.linspace(0.1, 0.9, 7)
    e = 1e-6
    Lp, _ = lagrange1d(k, x + e)
    Lm, _ = lagrange1d(k, x - e)
    _, d = lagrange1d(k, x)
    assert np.allclose((Lp - Lm) / (2 * e), d, atol=1e-8)


@pytest.mark.parametrize("k", [1, 2])
def test_polynomial_reproduction(k):
    """Q_k interpolation reproduces every polynomial of degree <= k in each variable."""
    hx, hy = 0.7, 0.3
    T = CellTables(k, hx, hy)
    a = np.arange(k + 1) / k
    X = np.array([a[i % (k + 1)] * hx for i in range((k + 1) ** 2)])
    Y = np.array([a[i // (k + 1)] * hy for i in range((k + 1) ** 2)])
    xq = T.xi[:, 0] * hx
    yq = T.xi[:, 1] * hy
    for px in range(k + 1):
        for py in range(k + 1):
            f = X ** px * Y ** py
            val = T.N @ f
            assert np.allclose(val, xq ** px * yq ** py, atol=1e-14)
            gx = T.dN[:, :, 0] @ f
            gy = T.dN[:, :, 1] @ f
            ex = px * xq ** max(px - 1, 0) * yq ** py if px > 0 else 0 * xq
            ey = py * yq ** max(py - 1, 0) * xq ** px if py > 0 else 0 * yq
            assert np.allclose(gx, ex, atol=1e-13)
            assert np.allclose(gy, ey, atol=1e-13)


def test_q1_square_closed_forms():
    """Q1 on a square of side h: Laplace (1/6)[4,-1,-2,-1] and mass h^2/36 [4,2,1,2]."""
    h = 0.37
    T = CellTables(1, h, h)
    K = np.einsum('q,qad,qbd->ab', T.JxW, T.dN, T.dN)
    M = np.einsum('q,qa,qb->ab', T.JxW, T.N, T.N)
    # local order (0,0),(1,0),(0,1),(1,1): edge neighbours differ in one index
    Kref = np.zeros((4, 4))
    Mref = np.zeros((4, 4))
    for A in range(4):
        for B in range(4):
            dist = (A % 2 != B % 2) + (A // 2 != B // 2)
            Kref[A, B] = {0: 4.0, 1: -1.0, 2: -2.0}[dist] / 6.0
            Mref[A, B] = {0: 4.0, 1: 2.0, 2: 1.0}[dist] * h * h / 36.0
    assert np.allclose(K, Kref, atol=1e-15)
    assert np.allclose(M, Mref, atol=1e-17)
