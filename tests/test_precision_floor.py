"""Why the dual time step hands its last iterations to FP64 right-hand sides,
and which form would keep them in FP32 (CPU, oracle arithmetic).

Sec. 5 iterates each BDF physical step in pseudo time until the l2 velocity
residual is below a tolerance (1e-6 for the 48^3 p = 4 Taylor-Green dual-time
workload).  With the RHS evaluated in FP32 that residual stalls at the RHS's
rounding floor (about 3.4e-6 measured on the GPU at h = 2 pi / 48, p = 4),
even with an FP64 master state, BDF term and residual: an FP32 RHS sees only
the FP32-rounded state, so nothing controls the master's low bits.  The
library therefore switches to an FP64 twin below 5e-6.

This test replays the question with the oracle's stage arithmetic run in
float32 (acmhd.flux, common_flux and source keep the dtype of their input
with Python-float parameters) on a periodic box of 2^3 elements with the
workload's element size, order, zeta, nu, T_r, dt and dtau, the field a
Taylor-Green vortex scaled to the box, first step BDF1:

  * FP64 RHS: below 1e-9 after 400 RK4 pseudo steps;
  * FP32 RHS: stalls above 1e-6;
  * FP32 RHS plus a frozen defect d = R64(U_k) - R32(U_k) refreshed every 5
    pseudo steps: stalls above 1e-6 too (the defect corrects the RHS's bias
    at U_k, not the part of the state the FP32 RHS cannot see);
  * correction form (mixed-precision iterative refinement): per outer step
    the FP64 pseudo residual r_k = R_tau(U_k), then RK4 pseudo steps on the
    correction delta with g(delta) = r_k + L_tau(U_k) delta, L the RHS
    linearised at U_k (Rusanov speed frozen there) in FP32, whose rounding
    error scales with |delta|; U_{k+1} = U_k + delta.  It follows the FP64
    history below 1e-9 with one FP64 RHS per 50 pseudo steps;
  * the same with L_tau(U_k) delta taken as a scaled FP32 difference of the
    plain RHS: below 1e-9 as well, with no operator beyond the FP32 RHS.
"""
import numpy as np
import pytest

from oracle import acmhd, fr, timestep
from oracle.ops1d import Ops1D
from paper_2107_14027_gb300 import workloads as wl

ORDER, NEL = 4, 2
ZETA, NU, T_R = 2.5, 1.0 / 1600.0, 5e-3
DT, DTAU, STEPS = 1e-2, 1e-3, 400
D = 3


def _flux_lin(U0, dU, a):
    """dF_a/dU at U0 applied to dU; the flux is linear but for V (x) V."""
    F = np.zeros_like(dU)
    F[0] = ZETA * dU[1 + a]
    for i in range(D):
        F[1 + i] = (U0[1 + i] * dU[1 + a] + dU[1 + i] * U0[1 + a]
                    + (dU[0] if i == a else 0.0) - NU * dU[acmhd.aux(D, i, a)])
    for i in range(D):
        F[acmhd.aux(D, i, a)] = -dU[1 + i] / T_R
    return F


def _rhs_grid(G, mesh, ops, G0=None):
    """The six stages in the dtype of G (grid form); with G0 the RHS
    linearised at G0 and applied to G (the source is linear)."""
    cast = G.dtype.type
    lm, lp, Dm, dhl, dhr = (x.astype(G.dtype) for x in (ops.lm, ops.lp, ops.D, ops.dhl, ops.dhr))
    div = np.zeros_like(G)
    for a in range(D):
        pa, ea = 1 + D + a, 1 + a
        J = cast(2.0 / mesh.h[a])
        Fa = acmhd.flux(G, a, ZETA, NU, T_R) if G0 is None else _flux_lin(G0, G, a)
        div += J * (fr._apply_along(Dm, Fa, pa)
                    - fr._lift_along(dhl, fr._dot_along(lm, Fa, pa), pa)
                    - fr._lift_along(dhr, fr._dot_along(lp, Fa, pa), pa))
        UL = fr._dot_along(lp, G, pa)
        UR = np.roll(fr._dot_along(lm, G, pa), -1, axis=ea)
        if G0 is None:
            FI = acmhd.common_flux(UL, UR, a, ZETA, NU, T_R)
        else:
            UL0 = fr._dot_along(lp, G0, pa)
            UR0 = np.roll(fr._dot_along(lm, G0, pa), -1, axis=ea)
            s = np.maximum(acmhd.wave_speed(UL0, a, ZETA), acmhd.wave_speed(UR0, a, ZETA))
            FI = 0.5 * (_flux_lin(UL0, UL, a) + _flux_lin(UR0, UR, a))
            FI[:1 + D] -= 0.5 * s * (UR[:1 + D] - UL[:1 + D])
        div += J * (fr._lift_along(dhl, np.roll(FI, 1, axis=ea), pa)
                    + fr._lift_along(dhr, FI, pa))
    return -div + acmhd.source(G, T_R)


class _Box:
    """2^3 periodic elements of the 48^3 workload's size, Taylor-Green field
    of the box's period (gradient variables scaled with it)."""

    def __init__(self):
        L = NEL * 2.0 * np.pi / 48.0
        lo, hi = (-L / 2,) * 3, (L / 2,) * 3
        self.mesh = fr.Mesh((NEL,) * 3, lo, hi)
        self.ops = Ops1D(ORDER)
        self.m = ORDER + 1
        k = 2.0 * np.pi / L
        U = wl.taylor_green((NEL,) * 3, tuple(k * x for x in lo), tuple(k * x for x in hi), ORDER)
        U[1 + D:] *= k
        self.Un = U
        self.n64 = 0

    def R(self, U, dtype=np.float64, U0=None):
        G = fr.to_grid(U.astype(dtype), self.mesh, self.m)
        G0 = None if U0 is None else fr.to_grid(U0.astype(dtype), self.mesh, self.m)
        out = _rhs_grid(G, self.mesh, self.ops, G0)
        assert out.dtype == dtype
        if dtype == np.float64 and U0 is None:
            self.n64 += 1
        return fr.from_grid(out, self.mesh, self.m).astype(np.float64)

    def tau(self, rhs_fn, U):
        """Pseudo RHS of the first physical step (BDF1), BDF term in FP64."""
        return timestep.pseudo_rhs(rhs_fn, U, self.Un, None, DT, 1, D)

    def residual(self, U):
        return timestep.velocity_residual(self.tau(self.R, U), D)


@pytest.fixture(scope="module")
def box():
    return _Box()


def test_stage_copy_matches_the_oracle_in_fp64(box):
    R = box.R(box.Un)
    ref = fr.rhs(box.Un, box.mesh, ORDER, fr.Params(ZETA, NU, T_R))
    np.testing.assert_allclose(R, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_linearised_rhs_is_the_derivative(box):
    rng = np.random.Generator(np.random.PCG64(7))
    dU = rng.uniform(-1.0, 1.0, size=box.Un.shape)
    L = box.R(dU, U0=box.Un)
    errs = []
    for eps in (1e-3, 1e-4):
        fd = (box.R(box.Un + eps * dU) - box.R(box.Un - eps * dU)) / (2 * eps)
        errs.append(np.abs(fd - L).max() / np.abs(L).max())
    # only the frozen Rusanov speed separates them (its variation times the
    # small jump of the smooth field)
    assert max(errs) < 1e-4, errs


def _plain(box, rhs_fn, every=None):
    U = box.Un.copy()
    hist = []
    for it in range(STEPS):
        if it % 100 == 0:
            hist.append(box.residual(U))
        U = timestep.rk4_step(lambda X: box.tau(rhs_fn(it), X), U, DTAU)
    hist.append(box.residual(U))
    return hist


def test_fp64_rhs_converges(box):
    hist = _plain(box, lambda it: box.R)
    assert hist[-1] < 1e-9, hist


def test_fp32_rhs_stalls_above_the_tolerance(box):
    hist = _plain(box, lambda it: (lambda X: box.R(X, np.float32)))
    assert min(hist[-2:]) > 1e-6, hist
    assert hist[-1] > 0.3 * hist[-2], hist


def test_frozen_fp64_defect_stalls_too(box):
    state = {"d": None}

    def rhs_at(it):
        def f(X):
            return box.R(X, np.float32) + state["d"]
        return f

    U = box.Un.copy()
    hist = []
    for it in range(STEPS):
        if it % 5 == 0:
            state["d"] = box.R(U) - box.R(U, np.float32)
        if it % 100 == 0:
            hist.append(box.residual(U))
        U = timestep.rk4_step(lambda X: box.tau(rhs_at(it), X), U, DTAU)
    hist.append(box.residual(U))
    assert min(hist[-2:]) > 1e-6, hist


def test_correction_form_reaches_fp64_residuals_with_fp32_operators(box):
    inner = 50
    U = box.Un.copy()
    box.n64 = 0
    for _ in range(STEPS // inner):
        r = box.tau(box.R, U)                      # FP64, once per outer step
        U32 = U.astype(np.float32)

        def g(dl):
            out = r + box.R(dl, np.float32, U0=U32)
            out[1:1 + D] -= dl[1:1 + D] / DT       # BDF1 term of the correction
            return out
        dl = np.zeros_like(U)
        for _ in range(inner):
            dl = timestep.rk4_step(g, dl, DTAU)
        U = U + dl
    n64 = box.n64
    res = box.residual(U)
    assert n64 == STEPS // inner
    assert res < 1e-9, res


def test_correction_form_with_the_existing_fp32_rhs(box):
    """The same outer FP64 iteration with L_tau(U_k) delta replaced by a scaled
    FP32 difference of the plain RHS, [R32(U_k + s delta) - R32(U_k)] / s, s
    fixed per outer step so that s delta is ~1e-3 of the state: the rounding
    of the difference is then ~1e-2 of L delta, and the outer iteration still
    follows the FP64 history.  With W = U_k + s delta this is the plain FP32
    pseudo iteration on W with the constant source s r_k - R32(U_k), i.e. the
    frozen defect amplified by s: it needs no kernel beyond the FP32 RHS."""
    inner = 50
    U = box.Un.copy()
    box.n64 = 0
    for _ in range(STEPS // inner):
        r = box.tau(box.R, U)
        U32 = U.astype(np.float32)
        R0 = box.R(U32, np.float32)
        s = 1e-3 * float(np.sqrt(np.mean(U * U))) / max(
            float(np.sqrt(np.mean(r * r))) * DTAU * inner, 1e-300)

        def g(dl):
            W = U32 + (s * dl).astype(np.float32)
            out = r + (box.R(W, np.float32) - R0) / s
            out[1:1 + D] -= dl[1:1 + D] / DT
            return out
        dl = np.zeros_like(U)
        for _ in range(inner):
            dl = timestep.rk4_step(g, dl, DTAU)
        U = U + dl
    n64 = box.n64
    res = box.residual(U)
    assert n64 == STEPS // inner
    assert res < 1e-9, res
