"""GPU parity of dual time stepping (BDF1/BDF2 + RK4 pseudo iterations)
against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

from oracle import fr, timestep
from tests import parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def abi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_14027_gb300 import build
    build.build()
    from paper_2107_14027_gb300 import abi as _abi
    return _abi


def _case(d=2, n=(6, 5), order=2):
    U, mesh, _, lo, hi = parity.make_case(n, order)
    prm = fr.Params(2.5, 1.0 / 400.0, 5e-3)
    return U, mesh, prm, lo, hi


def _vel_dev(abi, ctx, Vnp, d, order):
    """[d, npts, ne] FP64 numpy -> padded FP64 device rows."""
    V = abi.new_velocity(ctx, d, order)
    stride, ne, _ = abi.fr_layout(ctx)
    V[:, :ne] = torch.from_numpy(Vnp.reshape(-1, ne)).to("cuda")
    return V


def _vel_np(abi, ctx, V, d):
    stride, ne, _ = abi.fr_layout(ctx)
    return V[:, :ne].cpu().numpy().reshape(d, -1, ne)


@pytest.mark.parametrize("precision", [64, 65])
@pytest.mark.parametrize("bdf_order", [1, 2])
@pytest.mark.parametrize("n,order", [((6, 5), 2), ((3, 4, 3), 2)])
def test_pseudo_solve_matches_oracle_fixed_iterations(abi, n, order, bdf_order, precision):
    """FP64, and the double-float mode (FP64 storage, ~48-bit arithmetic in
    the RHS kernels), against the oracle's pseudo-solve."""
    d = len(n)
    nv = 1 + d + d * d
    U0, mesh, prm, lo, hi = _case(n=n, order=order)
    rng = np.random.default_rng(3)
    Un = U0 + 1e-3 * rng.standard_normal(U0.shape)
    Unm1 = U0 + 2e-3 * rng.standard_normal(U0.shape)
    dt, dtau, iters = 1e-2, 1e-3, 12
    ctx = abi.fr_create(n, lo, hi, order, nv, prm.zeta, prm.nu, prm.T, precision)
    try:
        Ud = abi.pack_state(ctx, U0, 64)
        V = _vel_dev(abi, ctx, U0[1:1 + d], d, order)
        Vn = _vel_dev(abi, ctx, Un[1:1 + d], d, order)
        Vm = _vel_dev(abi, ctx, Unm1[1:1 + d], d, order)
        st, it, res = abi.fr_pseudo_solve(ctx, Ud, V, Vn, Vm if bdf_order == 2 else None, dt,
                                          bdf_order, dtau, 0.0, iters, check_every=5,
                                          allow_noconv=True)
        torch.cuda.synchronize()
        assert st == abi.FR_ENOCONV and it == iters
        Ug = abi.unpack_state(ctx, Ud, nv)
        Vg = _vel_np(abi, ctx, V, d)
    finally:
        abi.fr_destroy(ctx)
    rhs = lambda X: fr.rhs(X, mesh, order, prm)
    Uo, ito, reso, ok = timestep.pseudo_solve(rhs, U0, Un, Unm1, dt, dtau, 0.0, iters, bdf_order,
                                              d, check_every=5)
    assert ito == iters and not ok
    scale = np.sqrt(np.mean(Uo ** 2, axis=(1, 2)))
    err = np.sqrt(np.mean((Ug - Uo) ** 2, axis=(1, 2))) / scale
    assert np.all(err < 1e-12), err
    # the FP64 master velocity is the returned velocity
    np.testing.assert_array_equal(Vg, Ug[1:1 + d])
    assert abs(res - reso) <= 1e-10 * abs(reso), (res, reso)


def test_pseudo_solve_converges_and_reports(abi):
    n, order, d = (6, 5), 2, 2
    U0, mesh, prm, lo, hi = _case(n=n, order=order)
    ctx = abi.fr_create(n, lo, hi, order, 7, prm.zeta, prm.nu, prm.T, 64)
    try:
        Ud = abi.pack_state(ctx, U0, 64)
        V = _vel_dev(abi, ctx, U0[1:3], d, order)
        Vn = _vel_dev(abi, ctx, U0[1:3], d, order)
        st, it, res = abi.fr_pseudo_solve(ctx, Ud, V, Vn, None, 1e-2, 1, 1e-2, 1e-4, 5000,
                                          check_every=4)
        assert st == abi.FR_OK and res < 1e-4 and it % 4 == 0 and it > 0
        Ug = abi.unpack_state(ctx, Ud, 7)
        # same iteration count and residual as the oracle
        rhs = lambda X: fr.rhs(X, mesh, order, prm)
        Uo, ito, reso, ok = timestep.pseudo_solve(rhs, U0, U0, U0, 1e-2, 1e-2, 1e-4, 5000, 1, d,
                                                  check_every=4)
        assert ok and ito == it
        assert abs(res - reso) < 1e-9 * reso + 1e-15
        assert np.sqrt(np.mean((Ug - Uo) ** 2)) < 1e-10
        # max_iter reached -> FR_ENOCONV with the iterate kept
        st2, it2, res2 = abi.fr_pseudo_solve(ctx, Ud, V, Vn, Vn, 1e-2, 2, 1e-3, 1e-30, 3,
                                             allow_noconv=True)
        assert st2 == abi.FR_ENOCONV and it2 == 3 and res2 > 0
        # bad arguments
        with pytest.raises(abi.FrError) as ei:
            abi.fr_pseudo_solve(ctx, Ud, V, Vn, None, 1e-2, 3, 1e-3, 1e-6, 3)
        assert ei.value.status == abi.FR_EINVAL
        # a non-finite state is reported, not iterated
        Ud[0, 0] = float("nan")
        with pytest.raises(abi.FrError) as ei:
            abi.fr_pseudo_solve(ctx, Ud, V, Vn, None, 1e-2, 1, 1e-3, 1e-6, 3)
        assert ei.value.status == abi.FR_ENONFINITE
    finally:
        abi.fr_destroy(ctx)


@pytest.mark.parametrize("precision", [64, 32])
def test_dual_steps_match_oracle(abi, precision):
    """Three physical steps (BDF1, then BDF2) with extrapolated guesses and a
    fixed number of pseudo iterations, against the oracle."""
    n, order, d = (6, 5), 2, 2
    nv = 7
    U0, mesh, prm, lo, hi = _case(n=n, order=order)
    dt, dtau, iters = 1e-2, 1e-3, 8
    ctx = abi.fr_create(n, lo, hi, order, nv, prm.zeta, prm.nu, prm.T, precision)
    try:
        Ud = abi.pack_state(ctx, U0, precision)
        U_used = abi.unpack_state(ctx, Ud, nv)
        abi.fr_dual_init(ctx, Ud)
        steps = []
        for _ in range(3):
            st, stats = abi.fr_dual_step(ctx, Ud, dt, dtau, 0.0, iters, check_every=4,
                                         allow_noconv=True)
            it, res = stats.iters, stats.res
            assert st == abi.FR_ENOCONV and it == iters and stats.iters_refine == 0
            V = abi.new_velocity(ctx, d, order)
            abi.fr_dual_velocity(ctx, V)
            torch.cuda.synchronize()
            steps.append((abi.unpack_state(ctx, Ud, nv), _vel_np(abi, ctx, V, d), res))
    finally:
        abi.fr_destroy(ctx)
    rhs = lambda X: fr.rhs(X, mesh, order, prm)
    hist = [U_used]
    for k in range(3):
        if len(hist) == 1:
            guess, bdf, Un, Unm1 = hist[-1], 1, hist[-1], hist[-1]
        elif len(hist) == 2:
            guess, bdf, Un, Unm1 = 2 * hist[-1] - hist[-2], 2, hist[-1], hist[-2]
        else:
            guess = timestep.extrapolate_guess(hist[-1], hist[-2], hist[-3])
            bdf, Un, Unm1 = 2, hist[-1], hist[-2]
        Uo, ito, reso, _ = timestep.pseudo_solve(rhs, guess, Un, Unm1, dt, dtau, 0.0, iters, bdf,
                                                 d, check_every=4)
        hist.append(Uo)
        Ug, Vg, res = steps[k]
        scale = np.sqrt(np.mean(Uo ** 2, axis=(1, 2)))
        err = np.sqrt(np.mean((Ug - Uo) ** 2, axis=(1, 2))) / scale
        verr = np.sqrt(np.mean((Vg - Uo[1:1 + d]) ** 2)) / np.sqrt(np.mean(Uo[1:1 + d] ** 2))
        if precision == 64:
            assert np.all(err < 1e-12), (k, err)
            assert verr < 1e-12
            assert abs(res - reso) < 1e-9 * reso
        else:
            # FP32 RHS, FP64 velocity master and BDF source
            assert np.all(err < 2e-5), (k, err)
            assert verr < 2e-6, (k, verr)
            assert abs(res - reso) < 1e-3 * reso + 1e-5, (res, reso)


@pytest.mark.parametrize("twin", [64, 65])
def test_mixed_precision_step_hands_over_to_fp64(abi, twin):
    """The FP32 context iterates until tol_switch, then its FP64 twin (FP64 or
    double-float arithmetic) takes the residual (evaluated in FP64) to tol;
    the step agrees with an all-FP64 step at the same tolerance, and the
    FP64 velocity master carries over."""
    n, order, d, nv = (6, 5), 2, 2, 7
    U0, mesh, prm, lo, hi = _case(n=n, order=order)
    dt, dtau, tol = 1e-2, 1e-2, 1e-5
    c32 = abi.fr_create(n, lo, hi, order, nv, prm.zeta, prm.nu, prm.T, 32)
    c64 = abi.fr_create(n, lo, hi, order, nv, prm.zeta, prm.nu, prm.T, twin)
    cref = abi.fr_create(n, lo, hi, order, nv, prm.zeta, prm.nu, prm.T, 64)
    try:
        U32 = abi.pack_state(c32, U0, 32)
        U64w = abi.new_state(c64, 64)
        Uref = abi.pack_state(cref, U0.astype(np.float32).astype(np.float64), 64)
        abi.fr_dual_init(c32, U32)
        abi.fr_dual_init(cref, Uref)
        st, s = abi.fr_dual_step(c32, U32, dt, dtau, tol, 4000, check_every=5, refine=c64,
                                 U_refine=U64w, tol_switch=1e-4)
        st2, s2 = abi.fr_dual_step(cref, Uref, dt, dtau, tol, 4000, check_every=5)
        assert st == abi.FR_OK and st2 == abi.FR_OK
        assert s.res < tol and 1e-5 <= s.res_switch < 1e-4
        assert s.iters > 0 and s.iters_refine > 0 and s.iters % 5 == 0
        assert s2.res < tol and s2.iters_refine == 0
        V32 = abi.new_velocity(c32, d, order)
        Vref = abi.new_velocity(cref, d, order)
        abi.fr_dual_velocity(c32, V32)
        abi.fr_dual_velocity(cref, Vref)
        torch.cuda.synchronize()
        # both new levels satisfy the same FP64 residual tolerance
        assert (V32 - Vref).abs().max().item() < 1e-4
        with pytest.raises(abi.FrError) as ei:   # refine must be an FP64 twin
            abi.fr_dual_step(c32, U32, dt, dtau, tol, 10, refine=c32, U_refine=U64w)
        assert ei.value.status == abi.FR_EINVAL
    finally:
        for c in (c32, c64, cref):
            abi.fr_destroy(c)
