"""Seeded synthetic input states (no arithmetic of the method lives here).

Both the CUDA path and the oracle are fed from this module.  It only places
points and samples analytic fields: the solution-point positions come from
numpy's own Gauss-Legendre routine (numpy.polynomial.legendre.leggauss), the
fields are the Taylor-Green vortex of Sec. 5 (3-D) and its 2-D analogue,
and the noise is numpy's PCG64 stream.

State layout: U[v, pt, e] with pt = i + m j + m^2 k (i along x) and
e = ex + nx (ey + ny ez); variables ordered P, V, then d(V_i)/dx_b at index
1 + d + i d + b.

Readings of the paper that this module fixes:
  * 3-D TGV pressure is (cos 2x + cos 2y)(cos 2z + 2) / 16 (the printed
    "cos(2z + 2)" is read as the standard Taylor-Green pressure), and the
    constant 1/(gamma M^2) offset is dropped (P0 = 0): the RHS is invariant
    under a constant shift of P.
  * 2-D Taylor-Green: u = sin x cos y, v = -cos x sin y,
    P = (cos 2x + cos 2y) / 4.
  * Gradient variables are initialised with the exact derivatives.
  * "Seeded 1e-3 uniform noise": U(-1e-3, 1e-3) added to every variable at
    every point, PCG64 seeded with 20210729 unless another seed is given.
"""
import numpy as np

NOISE_SEED = 20210729


def nvars(d):
    return 1 + d + d * d


def point_coords(n, lo, hi, order):
    """x[a][pt, e]: physical coordinates of the solution points."""
    d = len(n)
    m = order + 1
    xi, _ = np.polynomial.legendre.leggauss(m)
    h = [(hi[a] - lo[a]) / n[a] for a in range(d)]
    ne = int(np.prod(n))
    e = np.arange(ne)
    ecoord, rest = [], e.copy()
    for a in range(d):
        ecoord.append(rest % n[a])
        rest = rest // n[a]
    pt = np.arange(m ** d)
    out = []
    for a in range(d):
        ia = (pt // m ** a) % m
        out.append(lo[a] + (ecoord[a][None, :] + 0.5 * (xi[ia][:, None] + 1.0)) * h[a])
    return out


def taylor_green(n, lo, hi, order, dtype=np.float64):
    """Taylor-Green initial field with exact gradients, shape [nv, m^d, ne]."""
    d = len(n)
    X = point_coords(n, lo, hi, order)
    nv = nvars(d)
    U = np.zeros((nv, X[0].shape[0], X[0].shape[1]), dtype=dtype)
    if d == 2:
        x, y = X
        sx, cx, sy, cy = np.sin(x), np.cos(x), np.sin(y), np.cos(y)
        U[0] = (np.cos(2 * x) + np.cos(2 * y)) / 4.0
        U[1] = sx * cy
        U[2] = -cx * sy
        U[3] = cx * cy          # du/dx
        U[4] = -sx * sy         # du/dy
        U[5] = sx * sy          # dv/dx
        U[6] = -cx * cy         # dv/dy
        return U
    x, y, z = X
    sx, cx, sy, cy, sz, cz = np.sin(x), np.cos(x), np.sin(y), np.cos(y), np.sin(z), np.cos(z)
    U[0] = (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0) / 16.0
    U[1] = sx * cy * cz
    U[2] = -cx * sy * cz
    # U[3] = w = 0
    U[4] = cx * cy * cz         # du/dx
    U[5] = -sx * sy * cz        # du/dy
    U[6] = -sx * cy * sz        # du/dz
    U[7] = sx * sy * cz         # dv/dx
    U[8] = -cx * cy * cz        # dv/dy
    U[9] = cx * sy * sz         # dv/dz
    # dw/dx_b = 0
    return U


def add_noise(U, amplitude=1e-3, seed=NOISE_SEED):
    rng = np.random.Generator(np.random.PCG64(seed))
    noise = rng.uniform(-amplitude, amplitude, size=U.shape)
    return (U.astype(np.float64) + noise).astype(U.dtype)


def random_state(d, order, ne, seed, scale=1.0, dtype=np.float64):
    """Unstructured random state (uniform in [-scale, scale]) for edge cases."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m = order + 1
    return rng.uniform(-scale, scale, size=(nvars(d), m ** d, ne)).astype(dtype)


# The workloads the kernels are measured and checked on.
TWO_PI = 2.0 * np.pi
WORKLOADS = {
    # 2-D quads p=2, 16x16 periodic mesh on [-pi, pi]^2, 7 variables,
    # zeta = 1, nu = 1/400, T_r = nu / zeta, TGV + seeded noise, FP64, 10 RK4 steps
    "quad_p2_16x16": dict(n=(16, 16), lo=(-np.pi,) * 2, hi=(np.pi,) * 2, order=2,
                          zeta=1.0, nu=1.0 / 400.0, t_r=(1.0 / 400.0) / 1.0,
                          noise=True, rk_steps=10, dtau=1e-3),
    # 3-D hexes p=3, 64^3 periodic mesh on [-pi, pi]^3, 13 variables, TGV Re=1600
    # (zeta = 2.5, nu = 1/1600, T_r = 5e-3), one RHS evaluation
    "hex_p3_64cube": dict(n=(64, 64, 64), lo=(-np.pi,) * 3, hi=(np.pi,) * 3, order=3,
                          zeta=2.5, nu=1.0 / 1600.0, t_r=5e-3, noise=False),
}

# Order sweep at ~37.9M solution points per variable (67^3 at p=4 has no exact
# cube match).
ORDER_SWEEP_MESH = {1: 168, 2: 112, 3: 84, 4: 67, 5: 56, 6: 48}
