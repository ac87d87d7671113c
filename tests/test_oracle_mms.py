"""Manufactured-solution pin of the oracle: the steady discrete solution
converges to the exact one at order p + 1.

Sec. 2.1 (FR divergence equation) gives a scheme whose solution error on
smooth data is O(h^(p+1)).  A mistake that keeps the truncation error of the
RHS at O(h^p) - which the pin of tests/test_oracle_fr.py accepts - but spoils
the solution (e.g. a correction function of the wrong degree that still
conserves) shows up here.

Recipe.  U_ex: smooth periodic P and V on [0, 2 pi]^2 (sympy expressions)
with the gradient variables equal to the exact gradients.  Forcing: f =
-R_c(U_ex) at the solution points, R_c the textbook continuous operator of
the steady system (Chorin's -zeta div V; incompressible Navier-Stokes
momentum -div(V V) - grad P + nu Lap V; and zero for the relaxation of the
gradient variables, which U_ex satisfies), derived with sympy independently
of the oracle.  The discrete steady problem R_h(U) + f = 0 is solved by
Newton's method with a Jacobian assembled from central differences of the
oracle's RHS (elements coloured so that perturbations do not overlap; the
flux is quadratic, so the differences are exact up to rounding except at
the Rusanov kinks).  R_h conserves P and V (the quadrature-weighted sums of
their rows vanish for every state), so the Jacobian has a (1 + d)-
dimensional left null space and the steady solution is fixed only up to the
means of P and V: the Newton system is bordered with those d + 1 weighted
means, held at U_ex's values, and their multipliers absorb the quadrature
error of the forcing's means.

Measured orders (DG, 2-D; mesh pairs n -> 2n):

  variable          p=1 (8->16)  p=2 (4->8, 8->16)  p=3 (4->8, 8->16)
  velocity          2.2          3.5, 3.6           4.0-4.1, 3.9
  pressure          2.0          2.8, 2.9           3.6, 3.3
  gradient vars     1.0-1.1      2.6, 2.4-2.7       2.7-3.0, 2.8-2.9

The velocity converges at p + 1.  The pressure converges between p and
p + 1, as equal-order discontinuous schemes whose pressure jumps are
penalised at O(1) strength (here the Rusanov dissipation on the P
equation) are known to; the gradient variables, whose common flux is the
plain mean, converge at order p.  Bounds asserted (the coarse pairs, which
keep the test to about a minute): velocity >= p + 1 - 0.3, pressure >= p,
gradient variables >= p - 0.3.  The g2 correction meets the same bounds.
A correction function of degree p instead of p + 1 (endpoint values kept,
so it still conserves) fails (test_low_degree_correction_is_caught).
"""
import numpy as np
import pytest
import scipy.sparse as sps
import scipy.sparse.linalg as spla
import sympy as sp

from oracle import fr
from oracle.ops1d import Ops1D

ZETA, NU, T_R, AMP = 1.5, 0.1, 0.05, 0.5


def _mms_case():
    """2-D fields and the continuous steady RHS R_c(U_ex) (sympy)."""
    x, y = sp.symbols("x y")
    xs = (x, y)
    V = [AMP * sp.sin(x) * sp.cos(y) + sp.Rational(1, 5),
         AMP * (sp.cos(x + y) - sp.sin(y)) / 2 - sp.Rational(1, 10)]
    P = AMP * sp.cos(x) * sp.sin(y) + sp.Rational(1, 10)
    grads = [sp.diff(V[i], xs[b]) for i in range(2) for b in range(2)]
    fields = [P] + V + grads
    RP = -ZETA * sum(sp.diff(V[a], xs[a]) for a in range(2))
    RV = [-sum(sp.diff(V[i] * V[a], xs[a]) for a in range(2)) - sp.diff(P, xs[i])
          + NU * sum(sp.diff(V[i], xs[a], 2) for a in range(2)) for i in range(2)]
    exact = [RP] + RV + [sp.Integer(0)] * 4
    return ([sp.lambdify(xs, f, "numpy") for f in fields],
            [sp.lambdify(xs, f, "numpy") for f in exact])


def _sample(fs, X):
    return np.stack([np.broadcast_to(np.asarray(f(*X), dtype=float), X[0].shape) for f in fs])


def _weights(mesh, p):
    w = Ops1D(p).w
    W = w
    for _ in range(mesh.d - 1):
        W = np.kron(w, W)
    return W * np.prod(mesh.h) / 2.0 ** mesh.d


def fd_jacobian(rhs_fn, U, mesh, h=1e-5):
    """Sparse dR/dU by central differences.  Elements are coloured by their
    coordinates modulo k (k >= 3 dividing every n[a]), so that no element's
    R depends on two perturbed elements (R of an element depends on itself
    and its 2d face neighbours)."""
    nv, npt, ne = U.shape
    d = mesh.d
    k = next(k for k in range(3, 64) if all(n % k == 0 for n in mesh.n))
    coords = np.array([mesh.elem_coords(e) for e in range(ne)])
    color = sum((coords[:, a] % k) * k ** a for a in range(d))
    nbh = [[e] + [mesh.neighbour(e, a, s) for a in range(d) for s in (-1, 1)] for e in range(ne)]
    idx = np.arange(nv * npt * ne).reshape(nv, npt, ne)
    rows, cols, vals = [], [], []
    for c in range(k ** d):
        elems = np.where(color == c)[0]
        owner = -np.ones(ne, dtype=int)
        for e in elems:
            for f in nbh[e]:
                assert owner[f] in (-1, e)
                owner[f] = e
        fs = np.where(owner >= 0)[0]
        for v in range(nv):
            for q in range(npt):
                Up, Um = U.copy(), U.copy()
                Up[v, q, elems] += h
                Um[v, q, elems] -= h
                blk = ((rhs_fn(Up) - rhs_fn(Um)) / (2 * h))[:, :, fs]
                nz = np.nonzero(blk)
                rows.append(idx[nz[0], nz[1], fs[nz[2]]])
                cols.append(idx[v, q, owner[fs[nz[2]]]])
                vals.append(blk[nz])
    N = nv * npt * ne
    return sps.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(N, N))


def steady_error(p, n, corr="dg", max_iter=16):
    """Per-variable quadrature L2 error of the steady discrete solution, and
    the final residual.  Newton iterations on the bordered system; the
    Jacobian is assembled at U_ex and re-assembled at the current iterate
    whenever an iteration reduces the residual by less than a factor 20."""
    fields, exact = _mms_case()
    mesh = fr.Mesh((n, n), (0.0, 0.0), (2 * np.pi, 2 * np.pi))
    prm = fr.Params(ZETA, NU, T_R)
    X = fr.point_coords(mesh, p)
    U_ex = _sample(fields, X)
    force = -_sample(exact, X)

    def R(U):
        return fr.rhs(U, mesh, p, prm, corr)

    nv, npt, ne = U_ex.shape
    N = nv * npt * ne
    w = _weights(mesh, p)
    rows = []
    for v in range(3):                      # P, u, v: the conserved rows
        r = np.zeros((nv, npt, ne))
        r[v] = w[:, None]
        rows.append(r.ravel())
    Wm = sps.csc_matrix(np.array(rows))

    def factor(U):
        J = fd_jacobian(R, U, mesh)
        return spla.splu(sps.bmat([[J, Wm.T], [Wm, None]], format="csc"),
                         permc_spec="MMD_AT_PLUS_A")

    U = U_ex.copy()
    lu = factor(U)
    lam = np.zeros(3)
    res_prev = np.inf
    for _ in range(max_iter):
        r = (R(U) + force).ravel()
        res = np.abs(r + Wm.T @ lam).max()
        if res < 1e-12:
            break
        if res > res_prev / 20:
            lu = factor(U)
        res_prev = res
        sol = lu.solve(np.concatenate([-r, -(Wm @ (U - U_ex).ravel())]))
        U = U + sol[:N].reshape(U.shape)
        lam = sol[N:]
    res = np.abs((R(U) + force).ravel() + Wm.T @ lam).max()
    e = U - U_ex
    err = np.sqrt(np.einsum("p,vpe->v", w, e * e) / (np.sum(w) * ne))
    return err, res


def mms_orders(p, n_coarse, corr="dg"):
    e0, r0 = steady_error(p, n_coarse, corr)
    e1, r1 = steady_error(p, 2 * n_coarse, corr)
    assert r0 < 1e-10 and r1 < 1e-10, (r0, r1)    # Newton converged
    return np.log2(e0 / e1)


def orders_meet_bounds(p, rates):
    return bool(rates[0] >= p and np.all(rates[1:3] >= p + 1 - 0.3)
                and np.all(rates[3:] >= p - 0.3))


@pytest.mark.parametrize("corr", ["dg", "g2"])
@pytest.mark.parametrize("p,n", [(1, 8), (2, 4), (3, 4)])
def test_steady_solution_converges_at_order_p_plus_1(p, n, corr):
    rates = mms_orders(p, n, corr)
    assert orders_meet_bounds(p, rates), (p, corr, rates)


def test_low_degree_correction_is_caught(monkeypatch):
    """Planted mistake: the right Radau polynomial of degree p (not p + 1)
    as the correction function.  It keeps h_l(-1) = 1, h_l(1) = 0, so the
    scheme still conserves; the manufactured solution is not reached at
    order p + 1 (or the Newton solve fails)."""
    from oracle import ops1d
    orig = ops1d.Ops1D.__init__

    def init(self, order, correction="dg"):
        orig(self, order, correction)
        m = order + 1
        self.dhl = ops1d.radau_right(m - 1, self.xi)[1]
        self.dhr = -ops1d.radau_right(m - 1, -self.xi)[1]

    monkeypatch.setattr(ops1d.Ops1D, "__init__", init)
    try:
        caught = not orders_meet_bounds(2, mms_orders(2, 4))
    except (AssertionError, RuntimeError, np.linalg.LinAlgError):
        caught = True
    assert caught
