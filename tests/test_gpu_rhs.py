"""GPU parity of the fused and unfused RHS against the FP64 oracle.

All calls go through the C ABI (paper_2107_14027_gb300.abi).  Inputs are
the seeded Taylor-Green states of paper_2107_14027_gb300.workloads; the FP32
path is compared with the oracle evaluated on the same FP32-rounded values.
Tolerances are stated in tests/parity.py.
"""
import numpy as np
import pytest

from oracle import fr
from tests import parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="session")
def abi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_14027_gb300 import build
    build.build()
    from paper_2107_14027_gb300 import abi as _abi
    return _abi


def _run(abi, U, n, lo, hi, order, prm, precision, corr=0, which="fused"):
    d = len(n)
    ctx = abi.fr_create(n, lo, hi, order, 1 + d + d * d, prm.zeta, prm.nu, prm.T, precision, corr)
    try:
        Ud = abi.pack_state(ctx, U, precision)
        Rd = abi.new_state(ctx, precision, fill=float("nan"))
        (abi.fr_rhs if which == "fused" else abi.fr_rhs_unfused)(ctx, Ud, Rd)
        torch.cuda.synchronize()
        R = abi.unpack_state(ctx, Rd, 1 + d + d * d)
        U_used = abi.unpack_state(ctx, Ud, 1 + d + d * d)
    finally:
        abi.fr_destroy(ctx)
    return R, U_used


CASES = [
    # (n, order) -- element counts with ragged tails and several tiles
    ((5, 7), 1), ((5, 7), 2), ((5, 7), 3), ((6, 5), 4), ((5, 7), 5), ((3, 11), 6),
    ((3, 4, 5), 1), ((3, 4, 5), 2), ((3, 4, 5), 3), ((4, 3, 5), 4), ((3, 4, 3), 5), ((3, 2, 5), 6),
    ((9, 8, 7), 3), ((1, 2, 3), 2), ((1, 1, 1), 3), ((2, 1, 1), 4), ((40, 3), 2),
    # rows along x of whole lane groups: the x-face traces at group ends are
    # stored by group (every precision's tile size divides these n_x)
    ((32, 3, 2), 3), ((64, 3), 2), ((16, 3, 2), 4), ((8, 2, 2), 6),
]


@pytest.mark.parametrize("precision,which", [(64, "fused"), (64, "unfused"), (32, "fused"),
                                             (32, "unfused"), (65, "fused")])
@pytest.mark.parametrize("n,order", CASES)
def test_rhs_matches_oracle(abi, n, order, which, precision):
    U, mesh, prm, lo, hi = parity.make_case(n, order)
    R, U_used = _run(abi, U, n, lo, hi, order, prm, precision, which=which)
    R_ref = fr.rhs(U_used, mesh, order, prm)
    scale = parity.term_scale(U_used, mesh, order, prm)
    parity.assert_parity(R, R_ref, scale, precision, plain=True, label=f"{which} {n} p={order}")


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("n,order", [((5, 7), 3), ((3, 4, 5), 2), ((3, 4, 5), 4)])
def test_g2_correction(abi, n, order, precision):
    U, mesh, prm, lo, hi = parity.make_case(n, order)
    R, U_used = _run(abi, U, n, lo, hi, order, prm, precision, corr=1)
    R_ref = fr.rhs(U_used, mesh, order, prm, "g2")
    scale = parity.term_scale(U_used, mesh, order, prm, "g2")
    parity.assert_parity(R, R_ref, scale, precision, plain=True, label="g2")


@pytest.mark.parametrize("precision", [64, 32, 65])
def test_anisotropic_mesh_and_parameters(abi, precision):
    n, order = (6, 3, 4), 3
    lo, hi = (0.0, -1.0, 2.0), (1.0, 2.0, 2.5)
    rng = np.random.default_rng(4)
    U = rng.uniform(-1, 1, size=(13, 64, 72))
    prm = fr.Params(1.7, 0.03, 0.2)
    mesh = fr.Mesh(n, lo, hi)
    R, U_used = _run(abi, U, n, lo, hi, order, prm, precision)
    R_ref = fr.rhs(U_used, mesh, order, prm)
    scale = parity.term_scale(U_used, mesh, order, prm)
    parity.assert_parity(R, R_ref, scale, precision, plain=True, label="random state")
    # a random state does not cancel: the plain bound is checked on every row
    _, _, cancel = parity.errors(R, R_ref, scale)
    assert np.all(cancel >= parity.CANCEL_MIN[precision]), cancel


@pytest.mark.parametrize("precision", [64, 32, 65])
def test_conservation_on_gpu(abi, precision):
    """The two elements of a face use bit-identical common fluxes, so the
    quadrature-weighted sum of the P and V residuals vanishes to rounding."""
    from oracle.ops1d import Ops1D
    n, order = (6, 5, 4), 3
    U, mesh, prm, lo, hi = parity.make_case(n, order)
    R, U_used = _run(abi, U, n, lo, hi, order, prm, precision)
    w = Ops1D(order).w
    Wt = np.kron(w, np.kron(w, w))
    tot = np.einsum("p,vpe->v", Wt, R[:4])
    mag = np.einsum("p,vpe->v", Wt, np.abs(R[:4]))
    eps = {64: 1e-14, 65: 1e-13, 32: 2e-6}[precision]
    assert np.all(np.abs(tot) < eps * mag), tot / mag


@pytest.mark.parametrize("precision,noise", [(32, False), (64, False), (32, True), (64, True)])
def test_full_size_hex_p3_64cube_sampled(abi, precision, noise):
    """The 64^3, p = 3, 13-variable Taylor-Green workload in the launch
    configuration the benchmark times; 256 sampled elements (including the
    mesh corners and the last CTA) against the oracle's per-element path.
    With the seeded U(-1e-3, 1e-3) noise the result no longer cancels in the
    P and V rows, and the plain relative bound applies there too."""
    from paper_2107_14027_gb300 import workloads as W
    cfg = W.WORKLOADS["hex_p3_64cube"]
    n, order = cfg["n"], cfg["order"]
    U = W.taylor_green(n, cfg["lo"], cfg["hi"], order)
    if noise:
        U = W.add_noise(U)
    U = U.astype(np.float32 if precision == 32 else np.float64)
    prm = fr.Params(cfg["zeta"], cfg["nu"], cfg["t_r"])
    mesh = fr.Mesh(n, cfg["lo"], cfg["hi"])
    ctx = abi.fr_create(n, cfg["lo"], cfg["hi"], order, 13, prm.zeta, prm.nu, prm.T, precision, 0)
    try:
        Ud = abi.pack_state(ctx, U, precision)
        Rd = abi.new_state(ctx, precision, fill=float("nan"))
        abi.fr_rhs(ctx, Ud, Rd)
        torch.cuda.synchronize()
        stride, ne, _ = abi.fr_layout(ctx)
        R = Rd[:, :ne].cpu().numpy().astype(np.float64).reshape(13, 64, ne)
    finally:
        abi.fr_destroy(ctx)
    assert np.all(np.isfinite(R))
    rng = np.random.default_rng(0)
    ne = mesh.ne
    elems = np.unique(np.concatenate([[0, 63, 64 * 63, ne - 64, ne - 1, ne - 32],
                                      rng.choice(ne, 250, replace=False)]))
    U64 = U.astype(np.float64)
    R_ref = fr.rhs_dense(U64, mesh, order, prm, elems=elems)
    # term scale on the sampled elements: evaluate on a small mesh-independent
    # proxy by restricting the grid computation to the samples
    scale = _sampled_term_scale(U64, mesh, order, prm, elems)
    parity.assert_parity(R[:, :, elems], R_ref, scale, precision, plain=noise,
                         label=f"64^3 noise={noise}")


FULL_SIZE = [(1, 168, 32), (2, 112, 32), (3, 84, 32), (4, 67, 32), (5, 56, 32), (6, 48, 32),
             (4, 48, 32), (4, 48, 64), (4, 48, 65)]


@pytest.mark.parametrize("order,nside,precision", FULL_SIZE)
def test_full_size_order_sweep_and_dual_mesh_sampled(abi, order, nside, precision):
    """The order-sweep meshes (about 38M points per variable, p = 1..6) and
    the dual-time workload's p = 4, 48^3 mesh at full size, in the launch
    configuration of their benchmarks (fr_rhs, two kernels); 256 sampled
    elements, including the mesh corners and the last CTA, against the
    oracle's per-element path."""
    from paper_2107_14027_gb300 import workloads as W
    n = (nside,) * 3
    lo, hi = (-np.pi,) * 3, (np.pi,) * 3
    m = order + 1
    U = W.taylor_green(n, lo, hi, order, dtype=np.float32 if precision == 32 else np.float64)
    prm = fr.Params(2.5, 1.0 / 1600.0, 5e-3)
    mesh = fr.Mesh(n, lo, hi)
    # (precision 65: FP64 storage, double-float arithmetic)
    ctx = abi.fr_create(n, lo, hi, order, 13, prm.zeta, prm.nu, prm.T, precision, 0)
    try:
        Ud = abi.pack_state(ctx, U, precision)
        Rd = abi.new_state(ctx, precision, fill=float("nan"))
        abi.fr_rhs(ctx, Ud, Rd)
        torch.cuda.synchronize()
        stride, ne, _ = abi.fr_layout(ctx)
        rng = np.random.default_rng(order)
        elems = np.unique(np.concatenate([[0, nside - 1, nside * (nside - 1), ne - nside, ne - 1,
                                           (ne - 1) // 32 * 32],
                                          rng.choice(ne, 250, replace=False)]))
        idx = torch.as_tensor(elems, device="cuda")
        R = Rd[:, :ne].index_select(1, idx).cpu().numpy().astype(np.float64)
        R = R.reshape(13, m ** 3, len(elems))
        del Ud, Rd
    finally:
        abi.fr_destroy(ctx)
    assert np.all(np.isfinite(R))
    U64 = U.astype(np.float64)
    del U
    R_ref = fr.rhs_dense(U64, mesh, order, prm, elems=elems)
    scale = _sampled_term_scale(U64, mesh, order, prm, elems)
    parity.assert_parity(R, R_ref, scale, precision, plain=False,
                         label=f"{nside}^3 p={order} f{precision}")


def _sampled_term_scale(U, mesh, order, prm, elems):
    from oracle import acmhd
    from oracle.ops1d import Ops1D
    ops = Ops1D(order)
    Dt = ops.D - np.outer(ops.dhl, ops.lm) - np.outer(ops.dhr, ops.lp)
    m, d = ops.m, mesh.d
    Ue = U[:, :, elems].reshape(U.shape[0], m, m, m, len(elems))  # (v, k, j, i, e)
    B = np.abs(acmhd.source(Ue, prm.T))
    for a in range(d):
        F = np.abs(acmhd.flux(Ue, a, prm.zeta, prm.nu, prm.T))
        ax = 3 - a  # axis of direction a in (v, k, j, i, e)
        B = B + (2.0 / mesh.h[a]) * np.moveaxis(np.tensordot(np.abs(Dt), F, axes=([1], [ax])), 0, ax)
    B = B.reshape(U.shape[0], m ** 3, len(elems))
    return np.sqrt(np.mean(B * B, axis=(1, 2)))


def test_rk4_steps_match_oracle(abi):
    """Ten classical RK4 pseudo-steps on the 2-D p = 2, 16 x 16 Taylor-Green
    workload (zeta = 1, nu = 1/400, T_r = nu/zeta, noise), FP64."""
    from oracle import timestep
    from paper_2107_14027_gb300 import workloads as W
    cfg = W.WORKLOADS["quad_p2_16x16"]
    n, order = cfg["n"], cfg["order"]
    U, mesh, prm, lo, hi = parity.make_case(n, order, zeta=cfg["zeta"], nu=cfg["nu"], t_r=cfg["t_r"])
    ctx = abi.fr_create(n, lo, hi, order, 7, prm.zeta, prm.nu, prm.T, 64, 0)
    try:
        Ud = abi.pack_state(ctx, U, 64)
        for _ in range(cfg["rk_steps"]):
            abi.fr_rk_step(ctx, Ud, cfg["dtau"])
        torch.cuda.synchronize()
        Ug = abi.unpack_state(ctx, Ud, 7)
    finally:
        abi.fr_destroy(ctx)
    Uo = U.copy()
    for _ in range(cfg["rk_steps"]):
        Uo = timestep.rk4_step(lambda X: fr.rhs(X, mesh, order, prm), Uo, cfg["dtau"])
    rel = np.sqrt(np.mean((Ug - Uo) ** 2, axis=(1, 2))) / np.sqrt(np.mean(Uo ** 2, axis=(1, 2)))
    assert np.all(rel < 1e-12), rel


def test_invalid_arguments_are_rejected(abi):
    ctx = abi.fr_create((4, 4), (0, 0), (1, 1), 2, 7, 1.0, 0.01, 0.1, 32, 0)
    try:
        A = abi.new_state(ctx, 32)
        with pytest.raises(abi.FrError) as ei:
            abi.fr_rhs(ctx, A, A)                     # aliasing
        assert ei.value.status == abi.FR_EINVAL
        B = torch.zeros(A.numel() + 4, dtype=A.dtype, device="cuda")
        with pytest.raises(abi.FrError):
            abi.fr_rhs(ctx, B[1:], A)                  # misaligned
        abi.fr_check(ctx)
    finally:
        abi.fr_destroy(ctx)
