"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in the oracle (on the CPU, by monkeypatching)
and checks that at least one of the independent pins of
tests/test_oracle_fr.py fails: convergence to the sympy continuous
operators, discrete conservation, acoustic energy dissipation, agreement
of the sum-factorised and dense paths, the Rusanov speed against the
spectral radius of the flux Jacobian, the acoustic Bloch spectrum against
upwind DG's Pade closed form, or the exact energy balance of the operator
linearised at V = 0.  (The manufactured-solution pin has its own planted
mistake in tests/test_oracle_mms.py.)  The last two are also checked alone
on the mistakes they can see: the spectrum those in the inviscid (P, V)
part at V = 0, the energy balance all but the two that change the Rusanov
speed only where V is not zero.
"""
import numpy as np
import pytest

from oracle import acmhd, fr, ops1d
from tests.test_oracle_fr import (_acoustic_spectrum_is_upwind_dg, _continuous_case, _energy_balance,
                                  _rand_state, _rusanov_speed_is_spectral_radius, _sample, _weights)


def _converges(d=2, p=2, ns=(8, 16), with_offset=True):
    f_fields, f_exact, (zeta, nu, T) = _continuous_case(d, with_offset)
    errs = []
    for n in ns:
        mesh = fr.Mesh((n,) * d, (0.0,) * d, (2 * np.pi,) * d)
        X = fr.point_coords(mesh, p)
        R = fr.rhs(_sample(f_fields, X), mesh, p, fr.Params(zeta, nu, T))
        errs.append(np.sqrt(np.mean((R - _sample(f_exact, X)) ** 2, axis=(1, 2))))
    return bool(np.all(np.log2(errs[0] / errs[1]) > p - 0.35))


def _conserves(d=2, p=2):
    mesh = fr.Mesh((3, 4), (0.0, 0.0), (1.0, 2.0))
    prm = fr.Params(2.5, 0.3, 0.5)
    U = _rand_state(d, p, mesh.n, seed=3)
    R = fr.rhs(U, mesh, p, prm) - acmhd.source(U, prm.T)
    W = _weights(d, p, mesh)
    tot = np.einsum("p,vpe->v", W, R)
    scale = np.einsum("p,vpe->v", W, np.abs(R))
    return bool(np.all(np.abs(tot[: 1 + d]) < 1e-12 * scale[: 1 + d]))


def _dissipates(d=2, p=1):
    mesh = fr.Mesh((4, 3), (0.0, 0.0), (1.0, 1.0))
    prm = fr.Params(2.0, 0.0, 1.0)
    U = _rand_state(d, p, mesh.n, seed=11, amp=1e-5)
    U[1 + d:] = 0.0
    R = fr.rhs(U, mesh, p, prm)
    W = _weights(d, p, mesh)
    dE = np.einsum("p,pe->", W, U[0] * R[0] / prm.zeta)
    for i in range(1, 1 + d):
        dE += np.einsum("p,pe->", W, U[i] * R[i])
    mag = np.einsum("p,pe->", W, U[0] ** 2 + (U[1:1 + d] ** 2).sum(0)) * np.sqrt(prm.zeta)
    return bool(dE < -1e-3 * mag)


def _dense_agrees(d=2, p=2):
    mesh = fr.Mesh((3, 2), (0.0, 0.0), (1.0, 0.8))
    prm = fr.Params(2.5, 0.05, 0.1)
    U = _rand_state(d, p, mesh.n, seed=p)
    R = fr.rhs(U, mesh, p, prm)
    return bool(np.allclose(fr.rhs_dense(U, mesh, p, prm), R, rtol=0, atol=1e-12 * np.abs(R).max()))


def _energy_balance_holds():
    lhs, rhs = _energy_balance(2, 2, (3, 4), (1.0, 1.7))
    return bool(abs(lhs - rhs) <= 1e-10 * abs(rhs))


def _all_pins_pass():
    return (_converges() and _conserves() and _dissipates() and _dense_agrees()
            and _rusanov_speed_is_spectral_radius() and _acoustic_spectrum_is_upwind_dg()
            and _energy_balance_holds())


def test_unmutated_oracle_passes_all_pins():
    assert _all_pins_pass()


_orig_flux = acmhd.flux
_orig_common = acmhd.common_flux
_orig_init = ops1d.Ops1D.__init__
_orig_speed = acmhd.wave_speed


def _flux_nu_sign(U, a, zeta, nu, T):
    return _orig_flux(U, a, zeta, -nu, T)


def _flux_untransposed(U, a, zeta, nu, T):
    d = {7: 2, 13: 3}[U.shape[0]]
    F = _orig_flux(U, a, zeta, 0.0, T)
    for i in range(d):
        F[1 + i] -= nu * U[acmhd.aux(d, a, i)]   # S instead of S^T
    return F


def _flux_aux_sign(U, a, zeta, nu, T):
    d = {7: 2, 13: 3}[U.shape[0]]
    F = _orig_flux(U, a, zeta, nu, T)
    F[1 + d:] *= -1.0
    return F


def _flux_zeta_dropped(U, a, zeta, nu, T):
    F = _orig_flux(U, a, zeta, nu, T)
    F[0] /= zeta
    return F


def _common_anti_dissipative(UL, UR, a, zeta, nu, T):
    central = 0.5 * (_orig_flux(UL, a, zeta, nu, T) + _orig_flux(UR, a, zeta, nu, T))
    return 2.0 * central - _orig_common(UL, UR, a, zeta, nu, T)


def _common_one_sided(UL, UR, a, zeta, nu, T):
    return _orig_flux(UL, a, zeta, nu, T)


def _speed_sqrt_zeta(U, a, zeta):
    return np.sqrt(zeta) * np.ones_like(U[0])


def _speed_plus_zeta(U, a, zeta):
    return np.abs(U[1 + a]) + zeta


def _common_min_speed(UL, UR, a, zeta, nu, T):
    """Rusanov with the smaller of the two sides' speeds."""
    d = {7: 2, 13: 3}[UL.shape[0]]
    FI = 0.5 * (_orig_flux(UL, a, zeta, nu, T) + _orig_flux(UR, a, zeta, nu, T))
    s = np.minimum(_orig_speed(UL, a, zeta), _orig_speed(UR, a, zeta))
    FI[: 1 + d] -= 0.5 * s * (UR[: 1 + d] - UL[: 1 + d])
    return FI


def _ops_mutator(kind):
    def init(self, order, correction="dg"):
        _orig_init(self, order, correction)
        if kind == "D_transposed":
            self.D = self.D.T.copy()
        elif kind == "corrections_swapped":
            self.dhl, self.dhr = self.dhr.copy(), self.dhl.copy()
        elif kind == "ends_swapped":
            self.lm, self.lp = self.lp.copy(), self.lm.copy()
        elif kind == "correction_sign":
            self.dhl, self.dhr = -self.dhl, -self.dhr
    return init


class _RollReversed:
    def __getattr__(self, name):
        return getattr(np, name)

    @staticmethod
    def roll(a, shift, axis=None):
        return np.roll(a, -shift, axis=axis)


MUTATIONS = {
    "nu_sign": lambda mp: mp.setattr(acmhd, "flux", _flux_nu_sign),
    "S_not_transposed": lambda mp: mp.setattr(acmhd, "flux", _flux_untransposed),
    "aux_flux_sign": lambda mp: mp.setattr(acmhd, "flux", _flux_aux_sign),
    "zeta_dropped": lambda mp: mp.setattr(acmhd, "flux", _flux_zeta_dropped),
    "source_dropped": lambda mp: mp.setattr(acmhd, "source", lambda U, T: np.zeros_like(U)),
    "source_sign": lambda mp: mp.setattr(acmhd, "source", _source_sign),
    "anti_dissipative": lambda mp: mp.setattr(acmhd, "common_flux", _common_anti_dissipative),
    "one_sided_flux": lambda mp: mp.setattr(acmhd, "common_flux", _common_one_sided),
    "speed_sqrt_zeta": lambda mp: mp.setattr(acmhd, "wave_speed", _speed_sqrt_zeta),
    "speed_plus_zeta": lambda mp: mp.setattr(acmhd, "wave_speed", _speed_plus_zeta),
    "speed_min_of_sides": lambda mp: mp.setattr(acmhd, "common_flux", _common_min_speed),
    "D_transposed": lambda mp: mp.setattr(ops1d.Ops1D, "__init__", _ops_mutator("D_transposed")),
    "corrections_swapped": lambda mp: mp.setattr(ops1d.Ops1D, "__init__", _ops_mutator("corrections_swapped")),
    "ends_swapped": lambda mp: mp.setattr(ops1d.Ops1D, "__init__", _ops_mutator("ends_swapped")),
    "correction_sign": lambda mp: mp.setattr(ops1d.Ops1D, "__init__", _ops_mutator("correction_sign")),
    "neighbour_reversed": lambda mp: mp.setattr(fr, "np", _RollReversed()),
}


def _source_sign(U, T):
    d = {7: 2, 13: 3}[U.shape[0]]
    S = np.zeros_like(U)
    S[1 + d:] = U[1 + d:] / T
    return S


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, monkeypatch):
    MUTATIONS[name](monkeypatch)
    assert not _all_pins_pass(), f"mutation {name} went undetected"


# mistakes in the inviscid (P, V) part at V = 0, which the acoustic spectrum
# sees without help (the reversed neighbour maps the Bloch spectrum onto itself)
SPECTRUM_CATCHES = ["D_transposed", "anti_dissipative", "correction_sign", "corrections_swapped",
                    "ends_swapped", "one_sided_flux", "speed_plus_zeta", "zeta_dropped"]


@pytest.mark.parametrize("name", SPECTRUM_CATCHES)
def test_acoustic_spectrum_pin_alone_catches(name, monkeypatch):
    MUTATIONS[name](monkeypatch)
    assert not _acoustic_spectrum_is_upwind_dg(), f"mutation {name} went undetected"


# every mistake but the two whose Rusanov speed differs only where V != 0
ENERGY_CATCHES = sorted(set(MUTATIONS) - {"speed_sqrt_zeta", "speed_min_of_sides"})


@pytest.mark.parametrize("name", ENERGY_CATCHES)
def test_energy_balance_pin_alone_catches(name, monkeypatch):
    MUTATIONS[name](monkeypatch)
    assert not _energy_balance_holds(), f"mutation {name} went undetected"
