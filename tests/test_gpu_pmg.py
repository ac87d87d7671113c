"""GPU P-multigrid (fr_pmg_*) against the oracle's P-multigrid (oracle/pmg.py).

FP64: the same cycles from the same state give the same state and residual
as the oracle to 1e-12 (BDF1 and BDF2, 2-D and 3-D, the default cycle and a
custom one, with and without the point-implicit scaling).  FP32: the solve
converges where the FP64 one does.  Calls go through the C ABI.
"""
import numpy as np
import pytest

from oracle import fr, pmg
from paper_2107_14027_gb300 import workloads as W

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


PRM = fr.Params(2.5, 1.0 / 400.0, 5e-3)


def _states(d, order, n, seed=0):
    lo, hi = (-np.pi,) * d, (np.pi,) * d
    U = W.add_noise(W.taylor_green(n, lo, hi, order), seed=W.NOISE_SEED + seed)
    Un = W.add_noise(W.taylor_green(n, lo, hi, order), seed=W.NOISE_SEED + seed + 1)
    Unm1 = W.add_noise(W.taylor_green(n, lo, hi, order), seed=W.NOISE_SEED + seed + 2)
    return U, Un, Unm1, lo, hi


CASES = [
    # (d, order, mesh, dt, bdf, cycle or None, factors or None, implicit)
    (2, 2, (4, 5), 1.0, 1, None, None, True),
    (2, 3, (3, 4), 1e-2, 2, [(3, 1), (2, 2), (1, 3), (2, 1), (3, 2)], {3: 1.0, 2: 2.0, 1: 3.0},
     True),
    (3, 3, (2, 2, 3), 1e-2, 2, None, None, False),
    (3, 4, (2, 3, 2), 1e-2, 1, None, {4: 1.0, 3: 2.0, 2: 4.0, 1: 8.0}, True),
]


@pytest.mark.parametrize("d,order,n,dt,bdf,sched,factors,implicit", CASES)
def test_cycles_match_oracle_fp64(abi, d, order, n, dt, bdf, sched, factors, implicit):
    nv = 1 + d + d * d
    U, Un, Unm1, lo, hi = _states(d, order, n)
    dtau, ncyc = 1e-3, 3
    ctx = abi.fr_create(n, lo, hi, order, nv, PRM.zeta, PRM.nu, PRM.T, 64)
    m = abi.fr_pmg_create(ctx, 1)
    try:
        if sched is not None:
            abi.fr_pmg_set_cycle(m, sched)
        abi.fr_pmg_set_dtau(m, factors, implicit)
        stride, ne, _ = abi.fr_layout(ctx)
        Ud = abi.pack_state(ctx, U, 64)
        V = abi.new_velocity(ctx, d, order)
        Vn = abi.new_velocity(ctx, d, order)
        Vnm1 = abi.new_velocity(ctx, d, order)
        for dst, X in ((V, U), (Vn, Un), (Vnm1, Unm1)):
            dst[:, :ne] = torch.from_numpy(np.ascontiguousarray(X[1:1 + d]).reshape(-1, ne)).cuda()
        st, cyc, res = abi.fr_pmg_solve(m, Ud, V, Vn, Vnm1, dt, bdf, dtau, 0.0, ncyc,
                                        allow_noconv=True)
        assert st == abi.FR_ENOCONV and cyc == ncyc
        Ug = abi.unpack_state(ctx, Ud, nv)
        Vg = V[:, :ne].cpu().numpy().reshape(d, -1, ne)
    finally:
        abi.fr_pmg_destroy(m)
        abi.fr_destroy(ctx)
    mesh = fr.Mesh(n, lo, hi)
    levels = {q: pmg.Level(mesh, q, PRM) for q in range(1, order + 1)}
    schedule = sched if sched is not None else pmg.paper_schedule(order)
    factor = factors if factors is not None else 1.75
    g, a0dt = pmg.bdf_forcing(Un, Unm1, dt, bdf, d)
    Uo = U.copy()
    for _ in range(ncyc):
        Uo = pmg.cycle(levels, Uo, g, a0dt, dtau, schedule, factor, implicit)
    res_o = pmg.fine_residual(levels[order], Uo, g, a0dt)
    scale = np.sqrt(np.mean(Uo ** 2, axis=(1, 2))) + 1e-300
    err = np.sqrt(np.mean((Ug - Uo) ** 2, axis=(1, 2))) / scale
    assert np.all(err < 1e-12), err
    np.testing.assert_allclose(Vg, Uo[1:1 + d], rtol=0, atol=1e-12 * np.abs(Uo[1:1 + d]).max())
    assert abs(res - res_o) <= 1e-10 * res_o, (res, res_o)


@pytest.mark.parametrize("precision", [64, 32])
def test_solve_converges_and_dual_step_uses_it(abi, precision):
    """A BDF1 step (dt = 1) converges to 1e-9 (FP64) / 1e-5 (FP32) with
    cycles; fr_dual_step with the solver attached takes the same cycles."""
    d, order, n = 2, 3, (4, 4)
    nv = 7
    U, _, _, lo, hi = _states(d, order, n)
    tol = 1e-9 if precision == 64 else 1e-5
    ctx = abi.fr_create(n, lo, hi, order, nv, PRM.zeta, PRM.nu, PRM.T, precision)
    m = abi.fr_pmg_create(ctx, 1)
    try:
        stride, ne, _ = abi.fr_layout(ctx)
        Ud = abi.pack_state(ctx, U, precision)
        npts = (order + 1) ** d
        V = abi.new_velocity(ctx, d, order)
        V[:, :ne] = Ud[npts:(1 + d) * npts, :ne].double()     # as fr_dual_init widens it
        Vn = V.clone()
        st, cyc, res = abi.fr_pmg_solve(m, Ud, V, Vn, None, 1.0, 1, 1e-2, tol, 200)
        assert st == abi.FR_OK and res < tol and cyc >= 1
        Ud2 = abi.pack_state(ctx, U, precision)
        abi.fr_dual_init(ctx, Ud2)
        st2, s = abi.fr_dual_step(ctx, Ud2, 1.0, 1e-2, tol, 200, guess=abi.FR_GUESS_PREVIOUS,
                                  pmg=m)
        assert st2 == abi.FR_OK and s.iters == cyc and s.res == res
        torch.cuda.synchronize()
        assert torch.equal(Ud[:, :ne], Ud2[:, :ne])
    finally:
        abi.fr_pmg_destroy(m)
        abi.fr_destroy(ctx)


def test_invalid_cycles_are_refused(abi):
    ctx = abi.fr_create((3, 3), (0, 0), (1, 1), 3, 7, 2.5, 1e-3, 5e-3, 64)
    m = abi.fr_pmg_create(ctx, 1)
    try:
        for bad in ([(2, 1), (3, 1)], [(3, 1), (1, 1), (3, 1)], [(3, 0), (3, 1)],
                    [(3, 1), (2, 1)], [(3, 1), (0, 1), (1, 1), (2, 1), (3, 1)]):
            with pytest.raises(abi.FrError) as ei:
                abi.fr_pmg_set_cycle(m, bad)
            assert ei.value.status == abi.FR_EINVAL
        with pytest.raises(abi.FrError):
            abi.fr_pmg_set_dtau(m, {3: 1.0, 2: -1.0, 1: 2.0})
        with pytest.raises(abi.FrError):
            abi.fr_pmg_create(ctx, 4)
    finally:
        abi.fr_pmg_destroy(m)
        abi.fr_destroy(ctx)


@pytest.mark.parametrize("memory", [1, 3])
def test_anderson_mixing_matches_oracle_fp64(abi, memory):
    """Five cycles with Anderson mixing of memory 1 and 3 (BDF2, dt = 1e-2,
    3-D p = 3): the same states as the oracle's mixing (least squares by
    QR there, regularised normal equations here), to 1e-9."""
    d, order, n = 3, 3, (2, 3, 2)
    nv = 13
    U, Un, Unm1, lo, hi = _states(d, order, n, seed=5)
    dt, dtau, ncyc = 1e-2, 1e-3, 5
    ctx = abi.fr_create(n, lo, hi, order, nv, PRM.zeta, PRM.nu, PRM.T, 64)
    m = abi.fr_pmg_create(ctx, 1)
    try:
        abi.fr_pmg_set_anderson(m, memory)
        stride, ne, _ = abi.fr_layout(ctx)
        Ud = abi.pack_state(ctx, U, 64)
        V, Vn, Vnm1 = (abi.new_velocity(ctx, d, order) for _ in range(3))
        for dst, X in ((V, U), (Vn, Un), (Vnm1, Unm1)):
            dst[:, :ne] = torch.from_numpy(np.ascontiguousarray(X[1:1 + d]).reshape(-1, ne)).cuda()
        st, cyc, res = abi.fr_pmg_solve(m, Ud, V, Vn, Vnm1, dt, 2, dtau, 0.0, ncyc,
                                        allow_noconv=True)
        assert cyc == ncyc
        Ug = abi.unpack_state(ctx, Ud, nv)
    finally:
        abi.fr_pmg_destroy(m)
        abi.fr_destroy(ctx)
    mesh = fr.Mesh(n, lo, hi)
    levels = {q: pmg.Level(mesh, q, PRM) for q in range(1, order + 1)}
    g, a0dt = pmg.bdf_forcing(Un, Unm1, dt, 2, d)
    mix = pmg.Anderson(memory)
    Uo = U.copy()
    for _ in range(ncyc):
        Uo = mix.step(Uo, pmg.cycle(levels, Uo, g, a0dt, dtau, pmg.paper_schedule(order), 1.75))
    scale = np.sqrt(np.mean(Uo ** 2, axis=(1, 2))) + 1e-300
    err = np.sqrt(np.mean((Ug - Uo) ** 2, axis=(1, 2))) / scale
    assert np.all(err < 1e-9), err
    res_o = pmg.fine_residual(levels[order], Uo, g, a0dt)
    assert abs(res - res_o) <= 1e-7 * res_o, (res, res_o)
