"""Pins for the oracle's ACM-HD flux-reconstruction RHS.

Nothing here retypes the oracle's formulas.  The checks are:
  * convergence (at order >= p) to continuous operators derived with sympy
    from textbook forms: Chorin's -zeta div V, the incompressible
    Navier-Stokes momentum -div(V V) - grad P + nu Lap V, and relaxation of
    the gradient variables, (grad V - q) / T (Sec. 1, Eq. hd, read with the
    sign of Eq. acmhd_nd);
  * discrete invariants: free stream, conservation of the P and V equations
    on a periodic mesh, energy dissipation of the acoustic part with the
    DG correction, invariance under a constant shift of P, symmetry under
    an axis permutation and under a periodic shift of the mesh;
  * the paper's printed sparsity of the ACM-HD flux (Sec. 3);
  * agreement of the sum-factorised path with the dense element-by-element
    path that applies the FR divergence equation without the grouping;
  * the semi-discrete spectrum of the acoustic part (V = 0, nu = 0) with the
    DG correction equals upwind DG's closed form, the roots of
    R(-lambda h / c) = exp(+-i theta) with R the (p, p+1) Pade approximant
    of exp, to 1e-9 of the largest eigenvalue (p = 1..5);
  * the exact energy balance of the operator linearised at V = 0 with the
    DG correction and the gradient variables on: the weighted energy
    1/2 sum W (P^2/zeta + |V|^2 + nu T |q|^2) changes at -nu sum W |q|^2
    minus the Rusanov jump penalty, to 1e-10.
"""
import json
import os

import numpy as np
import pytest
import sympy as sp

from oracle import acmhd, fr
from oracle.ops1d import Ops1D

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_state(d, p, n, seed, amp=1.0):
    rng = np.random.default_rng(seed)
    m = p + 1
    return rng.uniform(-amp, amp, size=(acmhd.nvars(d), m ** d, int(np.prod(n))))


# ---------------------------------------------------------------------------
# convergence to the continuous operators
# ---------------------------------------------------------------------------

def _continuous_case(d, with_offset):
    """Smooth periodic fields and their textbook continuous RHS (sympy)."""
    xs = sp.symbols("x y z")[:d]
    if d == 2:
        x, y = xs
        V = [sp.sin(x) * sp.cos(2 * y) + sp.Rational(3, 10), sp.cos(x + y) - sp.Rational(1, 5)]
        P = sp.sin(2 * x) * sp.cos(y) + sp.Rational(1, 10)
    else:
        x, y, z = xs
        V = [sp.sin(x) * sp.cos(y) * sp.cos(z) + sp.Rational(1, 5),
             sp.cos(x + z) * sp.sin(y) - sp.Rational(1, 10),
             sp.sin(y + z) * sp.cos(x)]
        P = sp.cos(x) * sp.sin(2 * y) * sp.cos(z)
    grads = [[sp.diff(V[i], xs[b]) for b in range(d)] for i in range(d)]
    # optional smooth offset of the gradient variables
    delta = [[(sp.cos(xs[(b + 1) % d]) * (i + 1) / 10 if with_offset else 0)
              for b in range(d)] for i in range(d)]
    aux_fields = [grads[i][b] + delta[i][b] for i in range(d) for b in range(d)]
    fields = [P] + V + aux_fields
    zeta, nu, T = 1.3, 0.05, 0.02
    RP = -zeta * sum(sp.diff(V[a], xs[a]) for a in range(d))
    RV = []
    for i in range(d):
        conv = sum(sp.diff(V[i] * V[a], xs[a]) for a in range(d))
        lap = sum(sp.diff(V[i], xs[a], 2) for a in range(d))
        RV.append(-conv - sp.diff(P, xs[i]) + nu * lap)
    Raux = [-delta[i][b] / T for i in range(d) for b in range(d)]
    exact = [RP] + RV + Raux
    f_fields = [sp.lambdify(xs, f, "numpy") for f in fields]
    f_exact = [sp.lambdify(xs, f, "numpy") for f in exact]
    return f_fields, f_exact, (zeta, nu, T)


def _sample(fs, X):
    return np.stack([np.broadcast_to(np.asarray(f(*X), dtype=float), X[0].shape) for f in fs])


@pytest.mark.parametrize("d,p,ns", [
    (2, 1, (16, 32)), (2, 2, (8, 16)), (2, 3, (16, 32)), (2, 4, (8, 16)),
    (3, 1, (6, 12)), (3, 2, (8, 16)),
])
@pytest.mark.parametrize("with_offset", [False, True])
def test_converges_to_continuous_operators(d, p, ns, with_offset):
    f_fields, f_exact, (zeta, nu, T) = _continuous_case(d, with_offset)
    errs = []
    for n in ns:
        mesh = fr.Mesh((n,) * d, (0.0,) * d, (2 * np.pi,) * d)
        X = fr.point_coords(mesh, p)
        U = _sample(f_fields, X)
        R = fr.rhs(U, mesh, p, fr.Params(zeta, nu, T))
        Re = _sample(f_exact, X)
        errs.append(np.sqrt(np.mean((R - Re) ** 2, axis=(1, 2))))
    rate = np.log2(errs[0] / errs[1])
    # the FR truncation error at the solution points is O(h^p)
    assert np.all(rate > p - 0.35), (rate, errs)


# ---------------------------------------------------------------------------
# discrete invariants
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("d,p", [(2, 1), (2, 3), (3, 2), (3, 3)])
@pytest.mark.parametrize("corr", ["dg", "g2"])
def test_free_stream(d, p, corr):
    n = (3,) * d
    mesh = fr.Mesh(n, (0.0,) * d, (1.0,) * d)
    prm = fr.Params(2.5, 1e-2, 5e-3)
    U = np.zeros((acmhd.nvars(d), (p + 1) ** d, mesh.ne))
    U[0], U[1], U[2] = 0.7, -0.4, 0.25
    if d == 3:
        U[3] = 0.1
    R = fr.rhs(U, mesh, p, prm, corr)
    assert np.abs(R).max() < 1e-12
    # constant state with non-zero gradient variables: R equals the source
    U[1 + d:] = np.arange(d * d)[:, None, None] * 0.1 + 0.05
    R = fr.rhs(U, mesh, p, prm, corr)
    np.testing.assert_allclose(R[: 1 + d], 0.0, atol=1e-11)
    np.testing.assert_allclose(R[1 + d:], -U[1 + d:] / prm.T, rtol=1e-12)


def _weights(d, p, mesh):
    """Tensor-product quadrature weight x physical Jacobian per point."""
    w = Ops1D(p).w
    W = w
    for _ in range(d - 1):
        W = np.kron(w, W)
    return W * np.prod(mesh.h) / 2.0 ** d


@pytest.mark.parametrize("d,p", [(2, 1), (2, 2), (3, 1), (3, 3)])
@pytest.mark.parametrize("corr", ["dg", "g2"])
def test_conservation(d, p, corr):
    """Sum over the mesh of the quadrature-weighted divergence vanishes: the
    P and V equations (no source) are conserved on a periodic mesh, for any
    discontinuous data."""
    n = (3, 4, 2)[:d]
    mesh = fr.Mesh(n, (0.0,) * d, (1.0, 2.0, 1.5)[:d])
    prm = fr.Params(2.5, 0.3, 0.5)
    U = _rand_state(d, p, n, seed=3)
    R = fr.rhs(U, mesh, p, prm, corr)
    W = _weights(d, p, mesh)
    div_part = R - acmhd.source(U, prm.T)           # -div F only
    tot = np.einsum("p,vpe->v", W, div_part)
    scale = np.einsum("p,vpe->v", W, np.abs(div_part))
    assert np.all(np.abs(tot) < 1e-12 * scale), tot / scale


@pytest.mark.parametrize("d,p", [(2, 1), (2, 3), (3, 2)])
def test_energy_dissipation_acoustic(d, p):
    """Linear acoustics (nu = 0, tiny amplitude so V (x) V is negligible) with
    the DG correction is energy stable under an upwind flux:
    sum w (P R_P / zeta + V . R_V) < 0 for discontinuous data."""
    n = (4, 3, 2)[:d]
    mesh = fr.Mesh(n, (0.0,) * d, (1.0,) * d)
    prm = fr.Params(2.0, 0.0, 1.0)
    eps = 1e-5
    U = _rand_state(d, p, n, seed=11, amp=eps)
    U[1 + d:] = 0.0
    R = fr.rhs(U, mesh, p, prm, "dg")
    W = _weights(d, p, mesh)
    dE = np.einsum("p,pe->", W, U[0] * R[0] / prm.zeta)
    for i in range(1, 1 + d):
        dE += np.einsum("p,pe->", W, U[i] * R[i])
    mag = np.einsum("p,pe->", W, U[0] ** 2 + (U[1:1 + d] ** 2).sum(0)) * np.sqrt(prm.zeta)
    assert dE < -1e-3 * mag, (dE, mag)


def test_pressure_shift_invariance():
    d, p = 3, 2
    mesh = fr.Mesh((3, 2, 2), (0.0,) * 3, (1.0,) * 3)
    prm = fr.Params(2.5, 0.01, 0.05)
    U = _rand_state(d, p, mesh.n, seed=5)
    R0 = fr.rhs(U, mesh, p, prm)
    U[0] += 112.0
    R1 = fr.rhs(U, mesh, p, prm)
    np.testing.assert_allclose(R1, R0, rtol=0, atol=1e-10)


@pytest.mark.parametrize("d", [2, 3])
def test_axis_permutation_symmetry(d):
    """Exchanging x and y (with u <-> v and the matching gradient variables)
    maps R to the exchanged R."""
    p = 2
    m = p + 1
    n = (3, 4, 2)[:d]
    h = (1.0, 1.3, 0.7)[:d]
    mesh = fr.Mesh(n, (0.0,) * d, h)
    prm = fr.Params(1.7, 0.2, 0.3)
    U = _rand_state(d, p, n, seed=7)
    R = fr.rhs(U, mesh, p, prm)

    axperm = [1, 0, 2][:d]                       # new axis a <- old axis axperm[a]
    n2 = tuple(n[axperm[a]] for a in range(d))
    h2 = tuple(h[axperm[a]] for a in range(d))
    mesh2 = fr.Mesh(n2, (0.0,) * d, h2)
    vperm = [0] + [1 + axperm[i] for i in range(d)]
    vperm += [acmhd.aux(d, axperm[i], axperm[b]) for i in range(d) for b in range(d)]

    def permute(X):
        G = fr.to_grid(X, mesh, m)
        ax = [0] + [1 + axperm[a] for a in range(d)] + [1 + d + axperm[a] for a in range(d)]
        G2 = G.transpose(ax)[vperm]
        return fr.from_grid(np.ascontiguousarray(G2), mesh2, m)

    R2 = fr.rhs(permute(U), mesh2, p, prm)
    np.testing.assert_allclose(R2, permute(R), rtol=1e-12, atol=1e-12)


def test_periodic_shift_equivariance():
    d, p = 2, 3
    m = p + 1
    mesh = fr.Mesh((5, 3), (0.0, 0.0), (1.0, 1.0))
    prm = fr.Params(1.0, 0.1, 0.2)
    U = _rand_state(d, p, mesh.n, seed=9)
    R = fr.rhs(U, mesh, p, prm)

    def shift(X):
        G = fr.to_grid(X, mesh, m)
        return fr.from_grid(np.ascontiguousarray(np.roll(G, 2, axis=1)), mesh, m)

    np.testing.assert_allclose(fr.rhs(shift(U), mesh, p, prm), shift(R), rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------------------
# the paper's printed sparsity of the flux (Sec. 3)
# ---------------------------------------------------------------------------

def test_flux_sparsity_matches_paper():
    with open(os.path.join(GOLDEN, "sparsity.json")) as f:
        gold = json.load(f)
    rng = np.random.default_rng(0)
    for d in (2, 3):
        nv = acmhd.nvars(d)
        nnz = 0
        for a in range(d):
            U = rng.normal(size=(nv, 8))
            F = acmhd.flux(U, a, 1.3, 0.7, 0.9)
            nnz += int(np.sum(np.any(F != 0.0, axis=1)))
        s = 1.0 - nnz / (d * nv)
        assert nnz == d * (1 + 2 * d)
        assert abs(s - gold[f"d{d}"]["sparsity"]) < gold[f"d{d}"]["abs_tol"]


# ---------------------------------------------------------------------------
# Rusanov common flux
# ---------------------------------------------------------------------------

def test_common_flux_consistency_and_symmetry():
    rng = np.random.default_rng(1)
    for d in (2, 3):
        nv = acmhd.nvars(d)
        U = rng.normal(size=(nv, 5))
        W = rng.normal(size=(nv, 5))
        for a in range(d):
            np.testing.assert_allclose(acmhd.common_flux(U, U, a, 2.0, 0.1, 0.3),
                                       acmhd.flux(U, a, 2.0, 0.1, 0.3), rtol=1e-14)
            # the average of the two one-sided orders is the central flux
            c = 0.5 * (acmhd.flux(U, a, 2.0, 0.1, 0.3) + acmhd.flux(W, a, 2.0, 0.1, 0.3))
            FI = acmhd.common_flux(U, W, a, 2.0, 0.1, 0.3)
            np.testing.assert_allclose(FI[1 + d:], c[1 + d:], rtol=1e-14)


# ---------------------------------------------------------------------------
# dense vs sum-factorised
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("d,p", [(2, 1), (2, 4), (2, 6), (3, 1), (3, 3), (3, 5)])
@pytest.mark.parametrize("corr", ["dg", "g2"])
def test_dense_matches_sum_factorised(d, p, corr):
    n = (3, 2, 2)[:d]
    mesh = fr.Mesh(n, (0.0,) * d, (1.0, 0.8, 1.2)[:d])
    prm = fr.Params(2.5, 0.05, 0.1)
    U = _rand_state(d, p, n, seed=p)
    R = fr.rhs(U, mesh, p, prm, corr)
    Rd = fr.rhs_dense(U, mesh, p, prm, corr)
    np.testing.assert_allclose(Rd, R, rtol=0, atol=1e-12 * np.abs(R).max())
    # the per-element sampler returns the same columns
    Rs = fr.rhs_dense(U, mesh, p, prm, corr, elems=[mesh.ne - 1, 0])
    np.testing.assert_allclose(Rs, R[:, :, [mesh.ne - 1, 0]], rtol=0, atol=1e-12 * np.abs(R).max())


# ---------------------------------------------------------------------------
# Rusanov wave speed = spectral radius of the ACM flux Jacobian
# ---------------------------------------------------------------------------

def _acm_spectral_radius(U, a, zeta):
    """Largest |eigenvalue| of dF_a/dU restricted to the hyperbolic (P, V)
    block, from numpy's eigenvalue routine applied to the Jacobian of the
    oracle's flux (central differences; the flux is quadratic, so they are
    exact up to rounding).  nu = 0: the viscous part is not hyperbolic."""
    d = {7: 2, 13: 3}[U.shape[0]]
    k = 1 + d
    A = np.zeros((k, k))
    h = 1e-3
    for j in range(k):
        Up, Um = U.copy(), U.copy()
        Up[j] += h
        Um[j] -= h
        A[:, j] = (acmhd.flux(Up, a, zeta, 0.0, 1.0)[:k] - acmhd.flux(Um, a, zeta, 0.0, 1.0)[:k]) / (2 * h)
    return np.abs(np.linalg.eigvals(A)).max()


def _rusanov_speed_is_spectral_radius(seed=2):
    """The dissipation coefficient of the common flux on the P equation,
    s = -2 dF^I_P / dP_R, equals max(rho(U_L), rho(U_R)), rho the spectral
    radius of the ACM flux Jacobian (Sec. 5: a Rusanov solver for the
    hyperbolic part)."""
    rng = np.random.default_rng(seed)
    ok = True
    for d in (2, 3):
        nv = acmhd.nvars(d)
        for trial in range(6):
            UL = rng.normal(size=(nv, 1)) * 1.5
            UR = rng.normal(size=(nv, 1)) * 1.5
            zeta = float(rng.uniform(0.5, 3.0))
            for a in range(d):
                h = 1e-3
                Rp, Rm = UR.copy(), UR.copy()
                Rp[0] += h
                Rm[0] -= h
                dF = (acmhd.common_flux(UL, Rp, a, zeta, 0.1, 0.3)[0]
                      - acmhd.common_flux(UL, Rm, a, zeta, 0.1, 0.3)[0]) / (2 * h)
                s = -2.0 * float(dF[0])
                rho = max(_acm_spectral_radius(UL[:, 0], a, zeta),
                          _acm_spectral_radius(UR[:, 0], a, zeta))
                ok &= abs(s - rho) <= 1e-9 * rho
    return bool(ok)


def test_rusanov_speed_is_the_acm_spectral_radius():
    assert _rusanov_speed_is_spectral_radius()


def test_acm_eigenvalues_closed_form():
    """The eigenvalues of the ACM flux Jacobian in direction a are V_a and
    V_a +- sqrt(V_a^2 + zeta) (Chorin's artificial compressibility): checked
    against numpy's eigenvalues of the oracle's flux Jacobian."""
    rng = np.random.default_rng(5)
    for d in (2, 3):
        U = rng.normal(size=acmhd.nvars(d))
        zeta = 1.7
        for a in range(d):
            k = 1 + d
            A = np.zeros((k, k))
            for j in range(k):
                Up, Um = U.copy(), U.copy()
                Up[j] += 1e-3
                Um[j] -= 1e-3
                A[:, j] = (acmhd.flux(Up, a, zeta, 0.0, 1.0)[:k]
                           - acmhd.flux(Um, a, zeta, 0.0, 1.0)[:k]) / 2e-3
            lam = np.sort(np.linalg.eigvals(A).real)
            va = U[1 + a]
            c = np.sqrt(va * va + zeta)
            expect = np.sort([va - c] + [va] * (d - 1) + [va + c])
            np.testing.assert_allclose(lam, expect, rtol=0, atol=1e-9)


# ---------------------------------------------------------------------------
# semi-discrete acoustic spectrum against upwind DG's closed form
# ---------------------------------------------------------------------------

def _pade_sub_diagonal(p):
    """Ascending coefficients of the numerator (degree p) and denominator
    (degree p + 1) of the (p, p + 1) Pade approximant of exp(w)."""
    from math import factorial as f
    q = p + 1
    num = [f(p + q - j) * f(p) / (f(p + q) * f(j) * f(p - j)) for j in range(p + 1)]
    den = [(-1) ** j * f(p + q - j) * f(q) / (f(p + q) * f(j) * f(q - j)) for j in range(q + 1)]
    return np.array(num + [0.0]), np.array(den)


def _acoustic_spectrum_is_upwind_dg(p=2, N=5, zeta=2.5, L=3.0):
    """With nu = 0 and the Jacobian taken at U = 0, the (P, u) rows of the RHS
    for fields constant along y (a 2-D mesh of N x 1 elements) are 1-D linear
    acoustics P_t + zeta u_x = 0, u_t + P_x = 0 (the gradient variables do not
    feed back without viscosity, and the y faces see no jump).  There Rusanov
    with s = sqrt(zeta) is the characteristic upwind flux (|A| = sqrt(zeta) I),
    and FR with the DG correction is nodal DG (Huynh 2007), so the scheme is
    upwind DG for the two characteristic families at speeds +-c, c = sqrt(zeta).
    Upwind DG of degree p carries an element's inflow value g to its outflow
    value R(-z) g, z = lambda h / c, R the (p, p+1) Pade approximant of exp
    (Lesaint and Raviart 1974: DG in the marching variable).  On N periodic
    elements a Bloch mode of phase theta therefore has R(-z) = exp(+-i theta).
    The oracle's Jacobian comes from central differences at amplitude 1e-12,
    at which the quadratic terms and the |V_n| part of the speed vanish
    below rounding."""
    from scipy.optimize import linear_sum_assignment
    m = p + 1
    mesh = fr.Mesh((N, 1), (0.0, 0.0), (L, 1.0))
    prm = fr.Params(zeta, 0.0, 1.0)
    n = 2 * m * N
    Jm = np.zeros((n, n))
    eps = 1e-12
    col = 0
    ok = True
    for var in (0, 1):
        for e in range(N):
            for i in range(m):
                X = np.zeros((acmhd.nvars(2), m * m, N))
                X[var, i + m * np.arange(m), e] = 1.0
                dR = (fr.rhs(eps * X, mesh, p, prm) - fr.rhs(-eps * X, mesh, p, prm)) / (2 * eps)
                G = dR[:2].reshape(2, m, m, N)            # [var, j, i, e]
                scale = np.abs(G).max()
                ok &= bool(np.abs(G - G[:, :1]).max() <= 1e-9 * scale)   # constant along y
                ok &= bool(np.abs(dR[2]).max() <= 1e-9 * scale)          # v stays zero
                Jm[:, col] = G[:, 0].transpose(0, 2, 1).reshape(-1)      # (var, e, i)
                col += 1
    lam = np.linalg.eigvals(Jm)
    num, den = _pade_sub_diagonal(p)
    c, h = np.sqrt(zeta), L / N
    expect = []
    for k in range(N):
        for sgn in (1.0, -1.0):
            w = np.roots((num - np.exp(sgn * 2j * np.pi * k / N) * den)[::-1])
            expect.extend(-w * c / h)
    expect = np.array(expect)
    if len(expect) != len(lam):
        return False
    cost = np.abs(lam[:, None] - expect[None, :])
    r, cidx = linear_sum_assignment(cost)
    return ok and bool(cost[r, cidx].max() <= 1e-9 * np.abs(expect).max())


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_acoustic_spectrum_is_upwind_dg(p):
    assert _acoustic_spectrum_is_upwind_dg(p=p)


# ---------------------------------------------------------------------------
# exact energy balance of the linearised operator
# ---------------------------------------------------------------------------

def _energy_balance(d, p, n, lengths, zeta=2.5, nu=0.3, T=0.2, seed=4, correction="dg"):
    """(E', closed form) for the RHS linearised at U = 0 on random
    discontinuous data with the gradient variables switched on.

    At V = 0 the flux is linear, F_a = A_a U, and H = diag(1/zeta, I, nu T I)
    makes every H A_a symmetric (the P-V_a pair couples by zeta and 1, the
    V_i-q_ia pair by -nu and -1/T).  FR with the DG correction is DG with
    exact Gauss-Legendre integration of these fluxes, so the energy
    E = 1/2 sum W U.HU changes at exactly
        E' = -nu sum W |q|^2 - (sqrt(zeta)/2) sum_faces sum w_f ([P]^2/zeta + |[V]|^2):
    the volume terms integrate to face terms, the central parts of the
    common flux cancel them, the Rusanov part (speed sqrt(zeta) at V = 0, on
    P and V only) leaves the jump penalty, and the source -q/T gives the
    first term.  Quadrature nodes, weights and end values come from numpy's
    Gauss-Legendre rule here, not from the oracle."""
    m = p + 1
    mesh = fr.Mesh(n, (0.0,) * d, lengths)
    prm = fr.Params(zeta, nu, T)
    U = _rand_state(d, p, n, seed)
    eps = 1e-12
    R = (fr.rhs(eps * U, mesh, p, prm, correction)
         - fr.rhs(-eps * U, mesh, p, prm, correction)) / (2 * eps)
    xi, w = np.polynomial.legendre.leggauss(m)
    ends = {}
    for side in (-1.0, 1.0):
        ends[side] = np.array([np.prod([(side - xi[j]) / (xi[k] - xi[j]) for j in range(m) if j != k])
                               for k in range(m)])
    nv = acmhd.nvars(d)
    # A[v, point axes (slowest direction first), element axes (slowest first)]
    A = U.reshape((nv,) + (m,) * d + tuple(reversed(n)))

    def pax(a):
        return 1 + (d - 1 - a)

    def eax(a):
        return 1 + d + (d - 1 - a)

    Wpt = np.ones((m,) * d)
    for a in range(d):
        shape = [1] * d
        shape[d - 1 - a] = m
        Wpt = Wpt * (w * mesh.h[a] / 2).reshape(shape)
    Wpt = Wpt.reshape(-1)                       # matches pt = i + m j + m^2 k
    H = np.array([1.0 / zeta] + [1.0] * d + [nu * T] * (d * d))
    lhs = float(np.einsum("v,p,vpe,vpe->", H, Wpt, U, R))
    rhs = -nu * float(np.einsum("p,vpe->", Wpt, U[1 + d:] ** 2))
    for a in range(d):
        hi = np.tensordot(A, ends[1.0], axes=([pax(a)], [0]))
        lo = np.tensordot(A, ends[-1.0], axes=([pax(a)], [0]))
        # after contracting the point axis, element axis of a sits one lower
        jump = np.roll(lo, -1, axis=eax(a) - 1) - hi       # right neighbour's low face - own high
        wf = np.ones((m,) * (d - 1))
        others = [b for b in range(d) if b != a]
        for b in others:
            shape = [1] * (d - 1)
            shape[(d - 2) - others.index(b)] = m
            wf = wf * (w * mesh.h[b] / 2).reshape(shape)
        wf = wf.reshape(wf.shape + (1,) * d)
        pen = jump[0] ** 2 / zeta + (jump[1:1 + d] ** 2).sum(0)
        rhs -= 0.5 * np.sqrt(zeta) * float((wf * pen).sum())
    return lhs, rhs


@pytest.mark.parametrize("d,p,n", [(2, 1, (4, 3)), (2, 3, (3, 4)), (3, 2, (3, 2, 4)), (3, 4, (2, 3, 2))])
def test_energy_balance_of_the_linearised_operator(d, p, n):
    lhs, rhs = _energy_balance(d, p, n, (1.0, 1.7, 0.8)[:d])
    assert rhs < 0
    assert abs(lhs - rhs) <= 1e-10 * abs(rhs), (lhs, rhs)
