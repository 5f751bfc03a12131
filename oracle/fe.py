"""Finite-element tables for the oracle: Gauss rule and Q_k Lagrange basis.

Test infrastructure only (see ``oracle/__init__``).

Sec. 3 discretises u and phi with H^1-conforming tensor-product elements on
quadrilaterals (bilinear, k=1, in the paper; k=2 is supported the same way).
The paper does not name the quadrature; the oracle uses the (k+1)-point
Gauss-Legendre rule per direction, which integrates every term of the Q_k
mass and stiffness matrices exactly on Cartesian cells.

Local node numbering on the reference cell [0,1]^2: node (a, b) with
a, b in 0..k sits at (a/k, b/k) and has local index a + (k+1) * b
(x fastest).

Pinned by tests/test_oracle_fe.py: polynomial reproduction up to degree k
(values and gradients), closed-form Q1 Laplace and mass element matrices,
1^T M 1 = |Omega|.
"""
import numpy as np


def gauss01(n):
    """n-point Gauss-Legendre points and weights mapped to [0, 1]."""
    t, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (t + 1.0), 0.5 * w


def lagrange1d(k, x):
    """Values and derivatives of the k+1 equispaced 1D Lagrange polynomials.

    Nodes t_a = a / k.  Returns (L, dL) with shape (k+1, len(x)).
    Written directly from the product formula L_a(x) = prod_{b != a} (x - t_b)/(t_a - t_b).
    """
    x = np.asarray(x, dtype=np.float64)
    t = np.arange(k + 1) / k
    L = np.ones((k + 1, x.size))
    dL = np.zeros((k + 1, x.size))
    for a in range(k + 1):
        for b in range(k + 1):
            if b == a:
                continue
            L[a] *= (x - t[b]) / (t[a] - t[b])
        # derivative by the product rule
        for c in range(k + 1):
            if c == a:
                continue
            term = np.ones(x.size) / (t[a] - t[c])
            for b in range(k + 1):
                if b == a or b == c:
                    continue
                term *= (x - t[b]) / (t[a] - t[b])
            dL[a] += term
    return L, dL


class CellTables:
    """Full (not sum-factorised) Q_k tables at the (k+1)^2 Gauss points of a
    Cartesian hx-by-hy cell.

    N[q, A]      basis value
    dN[q, A, d]  physical gradient component d (d=0: x, d=1: y)
    JxW[q]       quadrature weight times |cell|
    Quadrature point q = q1 + (k+1) * q2 (x fastest).
    """

    def __init__(self, k, hx, hy, nq=None):
        self.k = k
        nq1 = (k + 1) if nq is None else nq
        xq, wq = gauss01(nq1)
        L, dL = lagrange1d(k, xq)
        nb = (k + 1) ** 2
        nqp = nq1 * nq1
        self.N = np.zeros((nqp, nb))
        self.dN = np.zeros((nqp, nb, 2))
        self.JxW = np.zeros(nqp)
        self.xi = np.zeros((nqp, 2))
        for q2 in range(nq1):
            for q1 in range(nq1):
                q = q1 + nq1 * q2
                self.JxW[q] = wq[q1] * wq[q2] * hx * hy
                self.xi[q] = (xq[q1], xq[q2])
                for b in range(k + 1):
                    for a in range(k + 1):
                        A = a + (k + 1) * b
                        self.N[q, A] = L[a, q1] * L[b, q2]
                        self.dN[q, A, 0] = dL[a, q1] * L[b, q2] / hx
                        self.dN[q, A, 1] = L[a, q1] * dL[b, q2] / hy
