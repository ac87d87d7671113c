"""Pseudo-time and physical-time stepping in plain FP64 (test infrastructure).

Sec. 5: physical time is integrated by BDF2 in dual time stepping; each
physical step is a steady problem in pseudo time tau, iterated until the
l2 residual in the velocity field drops below a tolerance.  The paper
pseudo-steps with an embedded RK34 pair and locally adaptive steps; the
reading taken here is classical four-stage RK4 with a fixed step dtau.

Readings where the paper is silent:
  * the first physical step uses BDF1 (backward Euler), later steps BDF2;
  * the residual is the RMS of the pseudo RHS over all velocity degrees of
    freedom (absolute, FP64);
  * the physical-time derivative acts on V only (Eq. acmhd_nd: d/dt applies
    to [0; V; 0; 0; 0]).

Pins (tests/test_oracle_timestep.py): RK4 reproduces the degree-4 Taylor
factor on u' = lambda u; BDF2 and BDF1 reproduce the exact step on
polynomial-in-time solutions of degree 2 and 1; the pseudo-solve converges
to the fixed point of a linear contraction.
"""
import numpy as np


def rk4_step(rhs_fn, U, dtau):
    """Classical RK4: U + dtau/6 (k1 + 2 k2 + 2 k3 + k4)."""
    k1 = rhs_fn(U)
    k2 = rhs_fn(U + 0.5 * dtau * k1)
    k3 = rhs_fn(U + 0.5 * dtau * k2)
    k4 = rhs_fn(U + dtau * k3)
    return U + (dtau / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)


def bdf_coeffs(order):
    """(a0, a1, a2) with dV/dt ~ (a0 V^{n+1} + a1 V^n + a2 V^{n-1}) / dt."""
    if order == 1:
        return 1.0, -1.0, 0.0
    if order == 2:
        return 1.5, -2.0, 0.5
    raise ValueError("BDF order must be 1 or 2")


def pseudo_rhs(rhs_fn, U, Un, Unm1, dt, order, d):
    """R_tau(U) = R(U) - I_V dV/dt with the BDF approximation of dV/dt."""
    a0, a1, a2 = bdf_coeffs(order)
    R = rhs_fn(U).copy()
    vel = slice(1, 1 + d)
    dvdt = a0 * U[vel] + a1 * Un[vel]
    if a2 != 0.0:
        dvdt = dvdt + a2 * Unm1[vel]
    R[vel] -= dvdt / dt
    return R


def velocity_residual(Rtau, d):
    """RMS of the pseudo RHS over the velocity degrees of freedom."""
    Rv = Rtau[1:1 + d]
    return float(np.sqrt(np.mean(Rv * Rv)))


def pseudo_solve(rhs_fn, U0, Un, Unm1, dt, dtau, tol, max_iter, order, d,
                 check_every=1):
    """Iterate RK4 in pseudo time on R_tau until the velocity residual < tol.

    Returns (U, iterations, residual, converged).  The residual is that of
    the returned iterate, checked every `check_every` iterations.
    """
    U = np.array(U0, dtype=np.float64, copy=True)

    def f(X):
        return pseudo_rhs(rhs_fn, X, Un, Unm1, dt, order, d)

    res = velocity_residual(f(U), d)
    it = 0
    while res >= tol and it < max_iter:
        for _ in range(check_every):
            U = rk4_step(f, U, dtau)
            it += 1
            if it >= max_iter:
                break
        res = velocity_residual(f(U), d)
    return U, it, res, res < tol


def extrapolate_guess(Un, Unm1, Unm2):
    """Plain initial guess for the next physical step: quadratic
    extrapolation 3 U^n - 3 U^{n-1} + U^{n-2}."""
    return 3.0 * Un - 3.0 * Unm1 + Unm2
