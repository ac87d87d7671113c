"""The fused RK4 stage schedule (RK4 combination, FP64 velocity rows, residual
partials and next-stage face traces in the epilogue of the volume kernel)
against the separate trace + volume + update kernels, through the C ABI.

Both schedules perform the same floating-point operations in the same order,
so the states they produce are compared bit for bit; the residual, a sum in a
different order, to 1e-12 relative.  Parity of the default (fused) schedule
with the FP64 oracle is covered by the RK4 and dual-time tests."""
import numpy as np
import pytest

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


# 2-D and 3-D, p = 1..6, both precisions; ragged element counts, a direction
# with a single element (the element is its own neighbour), and x-rows longer
# than a lane group (group ends inside a row)
CASES = [((6, 5), 1, 64), ((6, 5), 2, 32), ((7, 3), 4, 32), ((5, 4), 6, 64), ((37, 3), 3, 32),
         ((3, 4, 3), 2, 64), ((5, 4, 3), 3, 32), ((4, 3, 2), 4, 32), ((3, 2, 2), 5, 64),
         ((2, 2, 3), 6, 32), ((1, 3, 2), 3, 32), ((40, 3, 2), 1, 32), ((3, 3, 2), 4, 64)]


def _ctx(abi, n, order, precision):
    d = len(n)
    nv = 1 + d + d * d
    U, mesh, prm, lo, hi = parity.make_case(n, order)
    ctx = abi.fr_create(n, lo, hi, order, nv, prm.zeta, prm.nu, prm.T, precision, 0)
    return ctx, U, nv


@pytest.mark.parametrize("n,order,precision", CASES)
def test_fused_rk_step_is_bitwise_the_separate_update(abi, n, order, precision):
    ctx, U, nv = _ctx(abi, n, order, precision)
    try:
        out = {}
        for sched in (abi.FR_SCHEDULE_FUSED_STAGE, abi.FR_SCHEDULE_TWO_KERNELS):
            abi.fr_set_schedule(ctx, sched)
            Ud = abi.pack_state(ctx, U, precision)
            for _ in range(3):
                abi.fr_rk_step(ctx, Ud, 1e-3)
            out[sched] = Ud
        torch.cuda.synchronize()
        stride, ne, _ = abi.fr_layout(ctx)
        a, b = out[abi.FR_SCHEDULE_FUSED_STAGE][:, :ne], out[abi.FR_SCHEDULE_TWO_KERNELS][:, :ne]
        assert torch.isfinite(a).all()
        assert torch.equal(a, b), (a - b).abs().max().item()
        assert not torch.equal(a, abi.pack_state(ctx, U, precision)[:, :ne])
    finally:
        abi.fr_destroy(ctx)


DUAL_CASES = [((6, 5), 2, 64), ((7, 3), 4, 32), ((3, 4, 3), 2, 64), ((5, 4, 3), 3, 32),
              ((4, 3, 2), 4, 32), ((1, 3, 2), 5, 64)]


@pytest.mark.parametrize("n,order,precision", DUAL_CASES)
def test_fused_pseudo_solve_is_bitwise_the_separate_update(abi, n, order, precision):
    d = len(n)
    ctx, U, nv = _ctx(abi, n, order, precision)
    rng = np.random.default_rng(11)
    Un = U + 1e-3 * rng.standard_normal(U.shape)
    Unm1 = U + 2e-3 * rng.standard_normal(U.shape)
    try:
        stride, ne, _ = abi.fr_layout(ctx)
        out = {}
        for sched in (abi.FR_SCHEDULE_FUSED_STAGE, abi.FR_SCHEDULE_TWO_KERNELS):
            abi.fr_set_schedule(ctx, sched)
            Ud = abi.pack_state(ctx, U, precision)
            V = abi.new_velocity(ctx, d, order)
            Vn = abi.new_velocity(ctx, d, order)
            Vm = abi.new_velocity(ctx, d, order)
            for dst, X in ((V, U), (Vn, Un), (Vm, Unm1)):
                dst[:, :ne] = torch.from_numpy(np.ascontiguousarray(X[1:1 + d]).reshape(-1, ne)).to(
                    "cuda")
            st, it, res = abi.fr_pseudo_solve(ctx, Ud, V, Vn, Vm, 1e-2, 2, 1e-3, 0.0, 9,
                                              check_every=4, allow_noconv=True)
            assert st == abi.FR_ENOCONV and it == 9
            out[sched] = (Ud, V, res)
        torch.cuda.synchronize()
        (Ua, Va, ra), (Ub, Vb, rb) = out[abi.FR_SCHEDULE_FUSED_STAGE], out[abi.FR_SCHEDULE_TWO_KERNELS]
        assert torch.equal(Ua[:, :ne], Ub[:, :ne])
        assert torch.equal(Va[:, :ne], Vb[:, :ne])
        assert np.isfinite(ra) and abs(ra - rb) <= 1e-12 * abs(rb), (ra, rb)
    finally:
        abi.fr_destroy(ctx)


def test_fused_pseudo_solve_converges_like_the_separate_update(abi):
    """Same stopping iteration and residual (to rounding) on a converging
    solve: the residual check reads the fused stage's per-CTA partials."""
    n, order, precision = (6, 5), 2, 64
    d = 2
    ctx, U, nv = _ctx(abi, n, order, precision)
    try:
        stride, ne, _ = abi.fr_layout(ctx)
        out = {}
        for sched in (abi.FR_SCHEDULE_FUSED_STAGE, abi.FR_SCHEDULE_TWO_KERNELS):
            abi.fr_set_schedule(ctx, sched)
            Ud = abi.pack_state(ctx, U, precision)
            V = abi.new_velocity(ctx, d, order)
            Vn = abi.new_velocity(ctx, d, order)
            for dst in (V, Vn):
                dst[:, :ne] = torch.from_numpy(np.ascontiguousarray(U[1:1 + d]).reshape(-1, ne)).to(
                    "cuda")
            st, it, res = abi.fr_pseudo_solve(ctx, Ud, V, Vn, None, 1e-2, 1, 1e-2, 1e-4, 5000,
                                              check_every=1)
            assert st == abi.FR_OK and res < 1e-4
            out[sched] = (it, res)
        (ia, ra), (ib, rb) = out[abi.FR_SCHEDULE_FUSED_STAGE], out[abi.FR_SCHEDULE_TWO_KERNELS]
        assert ia == ib and abs(ra - rb) <= 1e-12 * rb
    finally:
        abi.fr_destroy(ctx)


def test_fused_stage_full_size_step_matches_separate_update(abi):
    """One RK4 step at the full 64^3 p = 3 FP32 size in the launch shape of
    the benchmark: the two schedules agree bit for bit on every entry."""
    from paper_2107_14027_gb300 import workloads as W
    n, order = (64, 64, 64), 3
    U = W.taylor_green(n, (-np.pi,) * 3, (np.pi,) * 3, order, dtype=np.float32)
    ctx = abi.fr_create(n, (-np.pi,) * 3, (np.pi,) * 3, order, 13, 2.5, 1 / 1600, 5e-3, 32, 0)
    try:
        stride, ne, _ = abi.fr_layout(ctx)
        outs = []
        for sched in (abi.FR_SCHEDULE_FUSED_STAGE, abi.FR_SCHEDULE_TWO_KERNELS):
            abi.fr_set_schedule(ctx, sched)
            Ud = abi.pack_state(ctx, U, 32)
            abi.fr_rk_step(ctx, Ud, 1e-3)
            outs.append(Ud)
            torch.cuda.synchronize()
        a, b = outs
        assert torch.equal(a[:, :ne], b[:, :ne])
    finally:
        abi.fr_destroy(ctx)


@pytest.mark.parametrize("n,order,precision", [((32, 2, 8), 3, 32), ((32, 5), 2, 64)])
def test_pseudo_solve_on_every_schedule_gives_the_same_state(abi, n, order, precision):
    """Two kernels + separate update, the fused stage and the automatic
    choice: one state, bit for bit, after fixed iterations."""
    d = len(n)
    ctx, U, nv = _ctx(abi, n, order, precision)
    rng = np.random.default_rng(5)
    Un = U + 1e-3 * rng.standard_normal(U.shape)
    try:
        stride, ne, _ = abi.fr_layout(ctx)
        out = []
        for sched in (abi.FR_SCHEDULE_TWO_KERNELS, abi.FR_SCHEDULE_FUSED_STAGE,
                      abi.FR_SCHEDULE_AUTO):
            abi.fr_set_schedule(ctx, sched)
            Ud = abi.pack_state(ctx, U, precision)
            V = abi.new_velocity(ctx, d, order)
            Vn = abi.new_velocity(ctx, d, order)
            for dst, X in ((V, U), (Vn, Un)):
                dst[:, :ne] = torch.from_numpy(np.ascontiguousarray(X[1:1 + d]).reshape(-1, ne)).to(
                    "cuda")
            st, it, res = abi.fr_pseudo_solve(ctx, Ud, V, Vn, Vn, 1e-2, 2, 1e-3, 0.0, 6,
                                              check_every=3, allow_noconv=True)
            assert st == abi.FR_ENOCONV and it == 6
            out.append((Ud, V))
        torch.cuda.synchronize()
        abi.fr_check(ctx)                         # no asynchronous error
        for Ux, Vx in out[1:]:
            assert torch.equal(out[0][0][:, :ne], Ux[:, :ne])
            assert torch.equal(out[0][1][:, :ne], Vx[:, :ne])
    finally:
        abi.fr_destroy(ctx)
