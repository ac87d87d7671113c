"""1-D operators of flux reconstruction, in plain FP64 (test infrastructure).

Follows Sec. 2.1 of the paper (FR divergence equation): solution points are
the Gauss-Legendre points of the reference element [-1, 1] (Fig.
tensor_product), l_k is the k-th Lagrange polynomial through them, and the
left/right correction functions h_l, h_r satisfy h_l(-1) = h_r(1) = 1 and
h_l(1) = h_r(-1) = 0.

The paper fixes only those endpoint conditions.  Two standard choices are
provided (Huynh 2007): the DG correction h_l = right Radau polynomial of degree
p+1, and Huynh's g2.  In both h_r(x) = h_l(-x).

Pins (tests/test_oracle_ops1d.py): closed-form nodes/weights for m = 2, 3;
agreement with numpy.polynomial.legendre.leggauss; quadrature exact to degree
2m-1; interpolation and differentiation exact on degree <= p; endpoint
conditions of the correction functions; DG roots at the right-Radau points;
g2 has a double root at +1.
"""
import math

import numpy as np


def legendre(n, x):
    """P_n(x) and P_n'(x) by Bonnet's three-term recurrence."""
    x = np.asarray(x, dtype=np.float64)
    p_prev = np.ones_like(x)
    if n == 0:
        return p_prev, np.zeros_like(x)
    p = x.copy()
    for k in range(1, n):
        # (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}
        p_prev, p = p, ((2 * k + 1) * x * p - k * p_prev) / (k + 1)
    # P_n' from P_n and P_{n-1}: (x^2 - 1) P_n' = n (x P_n - P_{n-1})
    with np.errstate(divide="ignore", invalid="ignore"):
        dp = n * (x * p - p_prev) / (x * x - 1.0)
    # endpoint values P_n'(+-1) = (+-1)^(n-1) n(n+1)/2
    end = np.isclose(np.abs(x), 1.0, rtol=0.0, atol=0.0)
    if np.any(end):
        dp = np.where(end, np.sign(x) ** (n - 1) * n * (n + 1) / 2.0, dp)
    return p, dp


def gauss_legendre(m):
    """Nodes (ascending) and weights of the m-point Gauss-Legendre rule.

    Newton iteration on P_m from the Chebyshev-like guess
    cos(pi (i + 3/4) / (m + 1/2)); weights 2 / ((1 - x^2) P_m'(x)^2).
    """
    nodes = np.empty(m)
    for i in range(m):
        x = math.cos(math.pi * (i + 0.75) / (m + 0.5))
        for _ in range(100):
            p, dp = legendre(m, x)
            dx = float(p) / float(dp)
            x -= dx
            if abs(dx) < 1e-16:
                break
        nodes[i] = x
    nodes = np.sort(nodes)
    _, dp = legendre(m, nodes)
    weights = 2.0 / ((1.0 - nodes ** 2) * dp ** 2)
    return nodes, weights


def lagrange(nodes, x):
    """Matrix L[j, k] = l_k(x_j): Lagrange basis through `nodes` at points x.

    Plain product formula l_k(x) = prod_{q != k} (x - x_q) / (x_k - x_q).
    """
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    m = len(nodes)
    out = np.ones((len(x), m))
    for k in range(m):
        for q in range(m):
            if q != k:
                out[:, k] *= (x - nodes[q]) / (nodes[k] - nodes[q])
    return out


def lagrange_deriv(nodes, x):
    """Matrix D[j, k] = l_k'(x_j), by the product rule on the product formula."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    m = len(nodes)
    out = np.zeros((len(x), m))
    for k in range(m):
        denom = 1.0
        for q in range(m):
            if q != k:
                denom *= nodes[k] - nodes[q]
        for r in range(m):  # the factor that is differentiated
            if r == k:
                continue
            term = np.ones(len(x))
            for q in range(m):
                if q != k and q != r:
                    term *= x - nodes[q]
            out[:, k] += term
        out[:, k] /= denom
    return out


def radau_right(k, x):
    """Right Radau polynomial of degree k and its derivative:
    R_{R,k} = ((-1)^k / 2) (P_k - P_{k-1}); it is 1 at x = -1 and 0 at x = 1.
    """
    pk, dpk = legendre(k, x)
    pk1, dpk1 = legendre(k - 1, x)
    s = (-1.0) ** k / 2.0
    return s * (pk - pk1), s * (dpk - dpk1)


def correction_left(kind, m, x):
    """Left correction function h_l and its derivative at points x.

    m = p + 1 is the number of solution points per direction, so h_l has
    degree m = p + 1.
      'dg': h_l = R_{R,m}                                  (Huynh's g_DG)
      'g2': h_l = ((m-1) R_{R,m} + m R_{R,m-1}) / (2m-1)    (Huynh's g_2)
    """
    if kind == "dg":
        return radau_right(m, x)
    if kind == "g2":
        a, da = radau_right(m, x)
        b, db = radau_right(m - 1, x)
        ca, cb = (m - 1) / (2.0 * m - 1.0), m / (2.0 * m - 1.0)
        return ca * a + cb * b, ca * da + cb * db
    raise ValueError(f"unknown correction function {kind!r}")


def correction_right(kind, m, x):
    """Right correction function h_r(x) = h_l(-x); derivative -h_l'(-x)."""
    x = np.asarray(x, dtype=np.float64)
    h, dh = correction_left(kind, m, -x)
    return h, -dh


class Ops1D:
    """The 1-D operators for order p (m = p + 1 Gauss-Legendre points).

    Attributes
    ----------
    xi, w      nodes and weights
    D          D[j, k] = l_k'(xi_j)
    lm, lp     l_k(-1), l_k(+1): interpolation of a line to its two ends
    dhl, dhr   h_l'(xi_j), h_r'(xi_j)
    """

    def __init__(self, order, correction="dg"):
        m = order + 1
        self.order, self.m, self.correction = order, m, correction
        self.xi, self.w = gauss_legendre(m)
        self.D = lagrange_deriv(self.xi, self.xi)
        self.lm = lagrange(self.xi, [-1.0])[0]
        self.lp = lagrange(self.xi, [1.0])[0]
        self.dhl = correction_left(correction, m, self.xi)[1]
        self.dhr = correction_right(correction, m, self.xi)[1]
