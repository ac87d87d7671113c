"""ACM-HD physics in plain FP64 (test infrastructure).

The artificial-compressibility Navier-Stokes system with hyperbolised
diffusion, Sec. 2.2, Eq. acmhd_2d (2-D, 7 variables) and Eq. acmhd_nd (d-D,
1 + d + d^2 variables):

    d/dtau [P; V; q; r; s] + div [ zeta V^T ; V (x) V + P I - nu S^T ;
                                   -(1/T) V (x) I ]  =  -(1/T) [0; 0; q; r; s]

with S = [q, r, s] (q ~ grad u, r ~ grad v, s ~ grad w).  Variable order:
0 = P, 1..d = velocity V, then the auxiliary block, index 1 + d + i*d + b
holding d(V_i)/dx_b (3-D: P,u,v,w,qx,qy,qz,rx,ry,rz,sx,sy,sz; 2-D:
P,u,v,qx,qy,rx,ry).

Common interface flux (Sec. 5): a Rusanov solver for the hyperbolic part and
the mean of the left and right flux for the additional (auxiliary)
equations.  Reading taken where the paper is silent: the Rusanov dissipation
acts on the P and V equations with speed s = max over both sides of
|V_n| + sqrt(V_n^2 + zeta) (the largest ACM eigenvalue in the face-normal
direction); the auxiliary equations get the plain mean.

Pins (tests/test_oracle_fr.py): the discrete RHS converges to the textbook
continuous operators (Chorin's -zeta div V, incompressible Navier-Stokes
momentum, relaxation (grad u - q)/T) computed independently with sympy; the
count of structurally non-zero flux entries equals the paper's sparsity
formula; the eigenvalues of the flux Jacobian's (P, V) block are Chorin's
V_a, V_a +- sqrt(V_a^2 + zeta); the Rusanov dissipation coefficient
-2 dF^I_P/dP_R equals the larger of the two sides' spectral radii of that
Jacobian (numpy eigenvalues); Rusanov consistency F^I(U, U) = F(U) and
energy dissipation.  tests/test_oracle_mms.py: the steady manufactured
solution is reached at order p + 1 in the velocity.
"""
import numpy as np


def nvars(d):
    return 1 + d + d * d


def aux(d, i, b):
    """Index of the auxiliary variable d(V_i)/dx_b."""
    return 1 + d + i * d + b


def flux(U, a, zeta, nu, T):
    """Flux component F_a(U) (direction a) at every point; U has shape (nv, ...)."""
    d = {7: 2, 13: 3}[U.shape[0]]
    F = np.zeros_like(U)
    V = [U[1 + i] for i in range(d)]
    P = U[0]
    F[0] = zeta * V[a]
    for i in range(d):
        # momentum row i, column a of  V (x) V + P I - nu S^T,  with
        # (S^T)[i, a] = S[a, i] = d(V_i)/dx_a
        F[1 + i] = V[i] * V[a] + (P if i == a else 0.0) - nu * U[aux(d, i, a)]
    for i in range(d):
        # row (i, b) of -(1/T) V (x) I, column a: -(1/T) V_i delta_{ab}
        F[aux(d, i, a)] = -V[i] / T
    return F


def source(U, T):
    """Source -(1/T) [0; 0; q; r; s]."""
    d = {7: 2, 13: 3}[U.shape[0]]
    S = np.zeros_like(U)
    S[1 + d:] = -U[1 + d:] / T
    return S


def wave_speed(U, a, zeta):
    """Largest |eigenvalue| of the ACM part in direction a: |V_a| + sqrt(V_a^2 + zeta)."""
    Va = U[1 + a]
    return np.abs(Va) + np.sqrt(Va * Va + zeta)


def common_flux(UL, UR, a, zeta, nu, T):
    """Common interface flux on a face with normal +e_a, UL on the low side.

    F^I = (F_a(UL) + F_a(UR)) / 2 - (s / 2) (UR - UL) on the P and V
    equations (Rusanov); the auxiliary equations take the mean flux only.
    """
    d = {7: 2, 13: 3}[UL.shape[0]]
    FL = flux(UL, a, zeta, nu, T)
    FR = flux(UR, a, zeta, nu, T)
    s = np.maximum(wave_speed(UL, a, zeta), wave_speed(UR, a, zeta))
    FI = 0.5 * (FL + FR)
    FI[: 1 + d] -= 0.5 * s * (UR[: 1 + d] - UL[: 1 + d])
    return FI
