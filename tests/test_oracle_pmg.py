"""Pins of the oracle's P-multigrid (oracle/pmg.py).

Nothing here retypes the transfer formulas: the operators are checked on
polynomials evaluated by numpy.polynomial, the smoother against the RK4
stability polynomial, and the cycle against plain RK4 pseudo-stepping
(timestep.pseudo_solve), which must reach the same discrete state.
"""
import numpy as np
import numpy.polynomial.polynomial as P
import pytest

from oracle import fr, pmg, timestep
from paper_2107_14027_gb300 import workloads as W


def _nodes(order):
    return np.polynomial.legendre.leggauss(order + 1)


@pytest.mark.parametrize("pf", [2, 3, 4, 5, 6])
def test_transfer_operators_on_polynomials(pf):
    pc = pf - 1
    Ir, Ip = pmg.transfer_1d(pf, pc)
    xf, wf = _nodes(pf)
    xc, _ = _nodes(pc)
    rng = np.random.default_rng(pf)
    for deg in range(pc + 1):
        c = rng.normal(size=deg + 1)
        # prolongation interpolates exactly, restriction reproduces exactly
        np.testing.assert_allclose(Ip @ P.polyval(xc, c), P.polyval(xf, c), atol=1e-13)
        np.testing.assert_allclose(Ir @ P.polyval(xf, c), P.polyval(xc, c), atol=1e-13)
    np.testing.assert_allclose(Ir @ Ip, np.eye(pc + 1), atol=1e-13)
    # the projection error of any fine function is orthogonal to the coarse
    # polynomials (fine quadrature is exact for the products)
    f = rng.normal(size=pf + 1)
    e = f - Ip @ (Ir @ f)
    for deg in range(pc + 1):
        assert abs(np.sum(wf * e * P.polyval(xf, np.eye(deg + 1)[deg]))) < 1e-13


@pytest.mark.parametrize("d", [2, 3])
def test_tensor_restriction_reproduces_coarse_polynomials(d):
    pf, pc = 3, 2
    Ir, Ip = pmg.transfer_1d(pf, pc)
    mesh = fr.Mesh((2,) * d, (0.0,) * d, (1.0,) * d)
    Xf = fr.point_coords(mesh, pf)
    Xc = fr.point_coords(mesh, pc)

    def field(X):      # degree <= pc in each direction, different per element
        out = 1.0 + 0.3 * X[0] ** 2 - 0.7 * X[0] * X[1]
        if d == 3:
            out = out + 0.2 * X[2] ** 2 * X[1] - X[2]
        return out

    Uf = np.stack([field(Xf), 2 * field(Xf)])
    Uc = np.stack([field(Xc), 2 * field(Xc)])
    np.testing.assert_allclose(pmg.apply_tensor(Ir, Uf, d), Uc, atol=1e-13)
    np.testing.assert_allclose(pmg.apply_tensor(Ip, Uc, d), Uf, atol=1e-13)


def test_scaled_rk4_on_pure_relaxation_is_the_stability_polynomial():
    """V = 0, P = 0, uniform gradient variables q: the flux vanishes and the
    pseudo RHS is -q/T, so one scaled RK4 step multiplies q by
    1 + z + z^2/2 + z^3/6 + z^4/24 with z = -dtau D / T, D = 1/(1 + dtau/T)."""
    mesh = fr.Mesh((3, 2), (0.0, 0.0), (1.0, 1.0))
    prm = fr.Params(2.0, 0.01, 0.05)
    lev = pmg.Level(mesh, 2, prm)
    U = np.zeros((7, 9, 6))
    U[3:] = np.arange(1, 5)[:, None, None] * 0.1
    for dtau in (1e-3, 0.04, 0.5):
        out = pmg.smooth(lev, U, np.zeros_like(U), 150.0, dtau, 1, implicit=True)
        z = -dtau / (1.0 + dtau / prm.T) / prm.T
        np.testing.assert_allclose(out[3:], U[3:] * (1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24),
                                   rtol=1e-13)
        np.testing.assert_allclose(out[:3], 0.0, atol=1e-15)
    # without the scaling the step is exactly the plain RK4 of timestep
    plain = pmg.smooth(lev, U, np.zeros_like(U), 150.0, 1e-3, 1, implicit=False)
    ref = timestep.rk4_step(lambda X: lev.N(X, 150.0), U, 1e-3)
    np.testing.assert_array_equal(plain, ref)


def test_paper_schedule():
    assert pmg.paper_schedule(4) == [(4, 1), (3, 1), (2, 1), (1, 4), (2, 1), (3, 1), (4, 7)]
    assert pmg.paper_schedule(2) == [(2, 1), (1, 4), (2, 7)]


def _case(d, order, n):
    lo, hi = (-np.pi,) * d, (np.pi,) * d
    U0 = W.add_noise(W.taylor_green(n, lo, hi, order))
    mesh = fr.Mesh(n, lo, hi)
    prm = fr.Params(2.5, 1.0 / 400.0, 5e-3)
    levels = {q: pmg.Level(mesh, q, prm) for q in range(1, order + 1)}
    return U0, mesh, prm, levels


def _tuned_schedule(p, bottom=32, post=1):
    """The paper's cycle shape with `bottom` iterations on order 1 and `post`
    on the finest order going up (the dual-time bench's cycle)."""
    return ([(q, 1) for q in range(p, 1, -1)] + [(1, bottom)] +
            [(q, 1) for q in range(2, p)] + [(p, post)])


@pytest.mark.parametrize("shape", ["paper", "tuned"])
@pytest.mark.parametrize("d,order,n", [(2, 2, (4, 4)), (3, 3, (2, 2, 3))])
def test_cycles_reach_the_rk4_fixed_point(d, order, n, shape):
    """From the same guess, P-multigrid cycles and plain RK4 pseudo-steps
    converge to the same discrete state (BDF1 step of the noisy
    Taylor-Green field); a converged state is a fixed point of a cycle.
    Both the paper's cycle and the tuned one (32 on order 1, one iteration on
    the finest order going up) solve the same problem; the tuned cycle, like
    the dual-time solver that uses it, with Anderson mixing (memory 8) of its
    cycles, without which its single smoothing pass on the way up leaves the
    3-D case stalling near 1e-8.
    dt = 1: with dt = 1e-2 the pressure's pseudo-time dynamics become a
    diffusion of rate zeta k^2 dt / a0 per unit pseudo time, and plain RK4
    needs far more than the test's iterations to converge its k = 1 mode."""
    U0, mesh, prm, levels = _case(d, order, n)
    Un = U0.copy()
    dt, dtau = 1.0, 1e-2

    def rhs(X):
        return fr.rhs(X, mesh, order, prm)

    ref, it, res, ok = timestep.pseudo_solve(rhs, U0, Un, Un, dt, dtau, 1e-11, 4000, 1, d,
                                             check_every=10)
    assert ok, res
    sched = pmg.paper_schedule(order) if shape == "paper" else _tuned_schedule(order)
    U, cyc, res_m, ok_m = pmg.pseudo_solve(levels, U0, Un, Un, dt, 1, dtau, 1e-11, 500, sched,
                                           anderson=0 if shape == "paper" else 8)
    assert ok_m, res_m
    # both are converged to 1e-11 in the velocity residual; the states agree
    np.testing.assert_allclose(U, ref, rtol=0, atol=1e-8)
    # fewer fine-level iterations than plain RK4 (8 per cycle at the finest)
    top = sum(k for q, k in sched if q == order)
    assert cyc * top < it, (cyc, it)
    # fixed point
    g, a0dt = pmg.bdf_forcing(Un, Un, dt, 1, d)
    again = pmg.cycle(levels, U, g, a0dt, dtau, sched, 1.75)
    assert np.abs(again - U).max() < 1e-9


def test_schedule_must_move_by_one_order():
    U0, mesh, prm, levels = _case(2, 3, (2, 2))
    g = np.zeros_like(U0)
    with pytest.raises(ValueError):
        pmg.cycle(levels, U0, g, 100.0, 1e-3, [(3, 1), (1, 2), (3, 1)], 1.75)


def test_anderson_terminates_on_a_linear_map():
    """On x <- M x + b in dimension n, Anderson mixing with memory >= n
    reaches the fixed point within n + 1 steps (it is GMRES on (I - M) x = b
    for linear maps), while the plain iteration is still far from it."""
    rng = np.random.default_rng(3)
    n = 6
    Q = np.linalg.qr(rng.normal(size=(n, n)))[0]
    M = Q @ np.diag(np.linspace(0.5, 0.99, n)) @ Q.T
    b = rng.normal(size=n)
    xs = np.linalg.solve(np.eye(n) - M, b)
    mix = pmg.Anderson(n)
    x = np.zeros(n)
    for _ in range(n + 1):
        x = mix.step(x, M @ x + b)
    assert np.linalg.norm(x - xs) < 1e-9 * np.linalg.norm(xs)
    y = np.zeros(n)
    plain = pmg.Anderson(0)
    for _ in range(n + 1):
        y = plain.step(y, M @ y + b)
    # m = 0 is the plain iteration: from 0, x_{n+1} = sum_{k<=n} M^k b
    np.testing.assert_allclose(y, sum(np.linalg.matrix_power(M, k) @ b for k in range(n + 1)),
                               rtol=1e-13)
    assert np.linalg.norm(y - xs) > 1e-2 * np.linalg.norm(xs)
