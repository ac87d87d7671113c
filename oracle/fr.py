"""Flux-reconstruction right-hand side of ACM-HD in plain FP64 (test infrastructure).

Computes R = -div F + S on a periodic, uniform, axis-aligned mesh of affine
quadrilaterals (d = 2) or hexahedra (d = 3) with m = p + 1 Gauss-Legendre
solution points per direction, following the six stages of Table fr_adv:

  1 (M) project the solution to the flux points of every face,
  2 (P) flux at the solution points,
  3 (M) partially corrected flux divergence
        J_a [ D F_a - h_l' (l(-1) . F_a) - h_r' (l(+1) . F_a) ],
  4 (I) common interface flux (acmhd.common_flux),
  5 (M) accumulate the correction J_a [ h_l' F^I_l + h_r' F^I_r ],
  6 (P) negate and add the source.

Stages 3 + 5 are the per-axis FR divergence of Sec. 2.1 (FR divergence
equation) with the flux interpolated to the interface taken as f^delta; the
grouping of stage 3 is the paper's "partially corrected" divergence.  J_a =
2 / h_a is the inverse of the constant 1-D mapping derivative.

Layouts.  A state is an array U[v, pt, e] with pt = i + m j + m^2 k (i along
x) and e = ex + nx (ey + ny ez).  Internally the sum-factorised path works on
the grid form G[v, ex, ey, (ez,) i, j, (k)].

Reading taken where the paper is silent: the common flux at a face is
computed once with the lower-index element (periodic wrap: the last
element) on the left, and used by both elements.

Pins (tests/test_oracle_fr.py): free stream gives R = 0 (and R = S for a
constant state with non-zero gradients), discrete conservation on a
periodic mesh, energy dissipation of the acoustic part, convergence to the
continuous operators evaluated symbolically, axis-permutation symmetry, and
agreement of the sum-factorised path with the dense Kronecker-product path
(which applies the FR divergence equation directly, without the stage-3
grouping), the Bloch spectrum of the acoustic part with the DG
correction against upwind DG's Pade closed form, and the exact energy
balance of the operator linearised at V = 0.  tests/test_oracle_mms.py: the steady solution of a manufactured
problem converges at order p + 1 in the velocity (at least p in the
pressure, p in the gradient variables).
"""
import numpy as np

from . import acmhd
from .ops1d import Ops1D


class Mesh:
    """Periodic uniform mesh: n[a] elements on [lo[a], hi[a]] per direction."""

    def __init__(self, n, lo, hi):
        self.d = len(n)
        self.n = tuple(int(x) for x in n)
        self.lo = tuple(float(x) for x in lo)
        self.hi = tuple(float(x) for x in hi)
        self.h = tuple((self.hi[a] - self.lo[a]) / self.n[a] for a in range(self.d))
        self.ne = int(np.prod(self.n))

    def elem_coords(self, e):
        c, rest = [], int(e)
        for a in range(self.d):
            c.append(rest % self.n[a])
            rest //= self.n[a]
        return tuple(c)

    def elem_index(self, c):
        e, stride = 0, 1
        for a in range(self.d):
            e += (c[a] % self.n[a]) * stride
            stride *= self.n[a]
        return e

    def neighbour(self, e, a, step):
        c = list(self.elem_coords(e))
        c[a] += step
        return self.elem_index(c)


class Params:
    def __init__(self, zeta, nu, T):
        self.zeta, self.nu, self.T = float(zeta), float(nu), float(T)


# ----------------------------------------------------------------------------
# layout helpers
# ----------------------------------------------------------------------------

def to_grid(U, mesh, m):
    nv = U.shape[0]
    if mesh.d == 2:
        nx, ny = mesh.n
        return U.reshape(nv, m, m, ny, nx).transpose(0, 4, 3, 2, 1)
    nx, ny, nz = mesh.n
    return U.reshape(nv, m, m, m, nz, ny, nx).transpose(0, 6, 5, 4, 3, 2, 1)


def from_grid(G, mesh, m):
    nv = G.shape[0]
    if mesh.d == 2:
        return G.transpose(0, 4, 3, 2, 1).reshape(nv, m * m, mesh.ne)
    return G.transpose(0, 6, 5, 4, 3, 2, 1).reshape(nv, m ** 3, mesh.ne)


def _apply_along(A, X, axis):
    """Y[..., j, ...] = sum_k A[j, k] X[..., k, ...] along `axis`."""
    return np.moveaxis(np.tensordot(A, X, axes=([1], [axis])), 0, axis)


def _dot_along(vec, X, axis):
    """sum_k vec[k] X[..., k, ...]: contracts (removes) `axis`."""
    return np.tensordot(X, vec, axes=([axis], [0]))


def _lift_along(vec, X, axis):
    """Outer product: Y[..., j, ...] = vec[j] X[...] with j inserted at `axis`."""
    shape = [1] * (X.ndim + 1)
    shape[axis] = len(vec)
    return np.expand_dims(X, axis) * vec.reshape(shape)


# ----------------------------------------------------------------------------
# sum-factorised six-stage RHS (Table fr_adv)
# ----------------------------------------------------------------------------

def rhs(U, mesh, order, params, correction="dg", ops=None):
    """R = -div F + S for the whole mesh.  U, R: [nv, m^d, ne] FP64."""
    ops = ops or Ops1D(order, correction)
    d, m = mesh.d, ops.m
    G = to_grid(np.asarray(U, dtype=np.float64), mesh, m)
    zeta, nu, T = params.zeta, params.nu, params.T

    def pax(a):  # grid axis of the point index along direction a
        return 1 + d + a

    def eax(a):  # grid axis of the element index along direction a
        return 1 + a

    # stage 1: project the solution to both faces of every direction
    Uf_lo = [_dot_along(ops.lm, G, pax(a)) for a in range(d)]
    Uf_hi = [_dot_along(ops.lp, G, pax(a)) for a in range(d)]

    # stage 2: flux at the solution points
    F = [acmhd.flux(G, a, zeta, nu, T) for a in range(d)]

    # stage 3: partially corrected flux divergence
    div = np.zeros_like(G)
    for a in range(d):
        J = 2.0 / mesh.h[a]
        Fd_lo = _dot_along(ops.lm, F[a], pax(a))
        Fd_hi = _dot_along(ops.lp, F[a], pax(a))
        div += J * (_apply_along(ops.D, F[a], pax(a))
                    - _lift_along(ops.dhl, Fd_lo, pax(a))
                    - _lift_along(ops.dhr, Fd_hi, pax(a)))

    # stage 4: common interface flux, one value per face; the face between
    # element e and e+1 along a has e on its low side
    FI_hi, FI_lo = [], []
    for a in range(d):
        # after contracting pax(a) the element axes keep their positions
        UR = np.roll(Uf_lo[a], -1, axis=eax(a))      # Uf_lo of element e+1
        FI_face = acmhd.common_flux(Uf_hi[a], UR, a, zeta, nu, T)
        FI_hi.append(FI_face)                            # right face of e
        FI_lo.append(np.roll(FI_face, 1, axis=eax(a)))   # left face of e

    # stage 5: accumulate the correction
    for a in range(d):
        J = 2.0 / mesh.h[a]
        div += J * (_lift_along(ops.dhl, FI_lo[a], pax(a))
                    + _lift_along(ops.dhr, FI_hi[a], pax(a)))

    # stage 6: negate and add the source
    R = -div + acmhd.source(G, T)
    return from_grid(R, mesh, m)


# ----------------------------------------------------------------------------
# dense Kronecker-product variant, element by element (tiny meshes, sampling)
# ----------------------------------------------------------------------------

def _kron_axis(A, a, d, m):
    """Operator acting on point direction a of a flattened pt = i + m j + m^2 k.

    A is (r x m); the result maps m^d values to r * m^(d-1) values.  The
    flattened index has direction 0 fastest, so direction a sits at Kronecker
    position d-1-a counted from the left.
    """
    I = np.eye(m)
    mats = [I] * d
    mats[d - 1 - a] = A
    out = mats[0]
    for M in mats[1:]:
        out = np.kron(out, M)
    return out


class DenseOps:
    def __init__(self, d, ops):
        m = ops.m
        self.d, self.m = d, m
        self.D = [_kron_axis(ops.D, a, d, m) for a in range(d)]
        self.Elo = [_kron_axis(ops.lm[None, :], a, d, m) for a in range(d)]
        self.Ehi = [_kron_axis(ops.lp[None, :], a, d, m) for a in range(d)]
        self.Hlo = [_kron_axis(ops.dhl[:, None], a, d, m) for a in range(d)]
        self.Hhi = [_kron_axis(ops.dhr[:, None], a, d, m) for a in range(d)]


def rhs_element_dense(U, mesh, e, params, ops, dops):
    """R for one element e from the FR divergence equation applied directly:
    div_a F = J_a [ D F + h_l' (F^I_l - F^delta_l) + h_r' (F^I_r - F^delta_r) ].
    U is the whole state [nv, m^d, ne]; returns R[:, :, e].
    """
    zeta, nu, T = params.zeta, params.nu, params.T
    d = mesh.d
    Ue = U[:, :, e]
    div = np.zeros_like(Ue)
    for a in range(d):
        J = 2.0 / mesh.h[a]
        Fa = acmhd.flux(Ue, a, zeta, nu, T)
        e_lo = mesh.neighbour(e, a, -1)
        e_hi = mesh.neighbour(e, a, +1)
        # traces (stage 1) of this element and of its two neighbours
        own_lo = Ue @ dops.Elo[a].T
        own_hi = Ue @ dops.Ehi[a].T
        nb_lo = U[:, :, e_lo] @ dops.Ehi[a].T   # left neighbour's right face
        nb_hi = U[:, :, e_hi] @ dops.Elo[a].T   # right neighbour's left face
        FI_l = acmhd.common_flux(nb_lo, own_lo, a, zeta, nu, T)
        FI_r = acmhd.common_flux(own_hi, nb_hi, a, zeta, nu, T)
        Fdl = Fa @ dops.Elo[a].T
        Fdr = Fa @ dops.Ehi[a].T
        div += J * (Fa @ dops.D[a].T
                    + (FI_l - Fdl) @ dops.Hlo[a].T
                    + (FI_r - Fdr) @ dops.Hhi[a].T)
    return -div + acmhd.source(Ue, T)


def rhs_dense(U, mesh, order, params, correction="dg", elems=None):
    """R from the dense per-element path; only for `elems` if given.

    Returns [nv, m^d, len(elems)] when elems is given, else [nv, m^d, ne].
    """
    ops = Ops1D(order, correction)
    dops = DenseOps(mesh.d, ops)
    U = np.asarray(U, dtype=np.float64)
    idx = range(mesh.ne) if elems is None else elems
    out = [rhs_element_dense(U, mesh, int(e), params, ops, dops) for e in idx]
    return np.stack(out, axis=-1)


def point_coords(mesh, order):
    """Physical coordinates x[a][pt, e] of the solution points (oracle nodes)."""
    ops = Ops1D(order)
    m, d = ops.m, mesh.d
    out = []
    for a in range(d):
        X = np.empty((m ** d, mesh.ne))
        for e in range(mesh.ne):
            c = mesh.elem_coords(e)
            for pt in range(m ** d):
                ia = (pt // m ** a) % m
                X[pt, e] = mesh.lo[a] + (c[a] + 0.5 * (ops.xi[ia] + 1.0)) * mesh.h[a]
        out.append(X)
    return out
