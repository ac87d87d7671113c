"""Pins for the oracle's pseudo-time (RK4) and physical-time (BDF) stepping."""
import numpy as np
import pytest

from oracle import timestep


@pytest.mark.parametrize("lam", [-1.0, -7.5, 2.0, -3.0 + 4.0j])
def test_rk4_taylor_factor(lam):
    """One classical RK4 step on u' = lambda u multiplies u by the degree-4
    Taylor polynomial of exp(lambda dtau)."""
    u0 = np.array([1.0 + 0.5j, -2.0])
    dtau = 0.13
    z = lam * dtau
    u1 = timestep.rk4_step(lambda u: lam * u, u0, dtau)
    np.testing.assert_allclose(u1, u0 * (1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24), rtol=1e-15)


def _state(d, npts=5, ne=3):
    rng = np.random.default_rng(0)
    return rng.normal(size=(1 + d + d * d, npts, ne))


@pytest.mark.parametrize("order,deg", [(1, 1), (2, 2)])
def test_bdf_exact_on_polynomials(order, deg):
    """BDF1 (BDF2) is exact for solutions linear (quadratic) in time: the
    pseudo RHS vanishes at the exact next state when R(U) = dV/dt there."""
    d, dt, t1 = 3, 0.01, 0.37
    a, b, c = _state(d), _state(d) * 0.3, _state(d) * (0.7 if deg == 2 else 0.0)

    def V(t):
        return a + b * t + c * t * t

    def rhs_fn(U):  # the exact time derivative at t1 on the velocity block
        out = np.zeros_like(U)
        out[1:1 + d] = (b + 2 * c * t1)[1:1 + d]
        return out

    Rt = timestep.pseudo_rhs(rhs_fn, V(t1), V(t1 - dt), V(t1 - 2 * dt), dt, order, d)
    np.testing.assert_allclose(Rt[1:1 + d], 0.0, atol=1e-11)
    if order == 1 and deg == 1:
        return
    # one degree higher is not exact
    c2 = _state(d) * 0.5
    Rt = timestep.pseudo_rhs(lambda U: np.zeros_like(U) + 0 * U, c2 * t1 ** 3, c2 * (t1 - dt) ** 3,
                             c2 * (t1 - 2 * dt) ** 3, dt, order, d)
    assert np.abs(Rt[1:1 + d]).max() > 1e-8


def test_pseudo_solve_reaches_dual_time_fixed_point():
    """With R(U) = -k (U - U*), the converged BDF2 step solves
    (1.5 V - 2 V^n + 0.5 V^{n-1}) / dt = -k (V - V*) exactly."""
    d = 2
    k, dt = 3.0, 0.05
    Ustar, Un, Unm1 = _state(d), _state(d) * 0.4, _state(d) * 0.2

    def rhs_fn(U):
        return -k * (U - Ustar)

    U, it, res, ok = timestep.pseudo_solve(rhs_fn, Un, Un, Unm1, dt, dtau=0.01, tol=1e-12,
                                           max_iter=20000, order=2, d=d)
    assert ok and res < 1e-12
    vel = slice(1, 1 + d)
    expect = (k * Ustar[vel] + (2 * Un[vel] - 0.5 * Unm1[vel]) / dt) / (k + 1.5 / dt)
    np.testing.assert_allclose(U[vel], expect, rtol=0, atol=1e-11)
    # iteration count is reported and capped
    U2, it2, res2, ok2 = timestep.pseudo_solve(rhs_fn, Un, Un, Unm1, dt, 0.01, 1e-12, 5, 2, d)
    assert it2 == 5 and not ok2 and res2 > 1e-12


def test_extrapolation_exact_for_quadratics():
    a, b, c = _state(2), _state(2), _state(2)
    f = [a + b * t + c * t * t for t in (0.0, 1.0, 2.0, 3.0)]
    np.testing.assert_allclose(timestep.extrapolate_guess(f[2], f[1], f[0]), f[3], rtol=1e-13, atol=1e-13)
