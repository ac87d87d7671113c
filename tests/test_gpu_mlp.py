"""GPU parity of the learned initial guess (MLP) against the FP64 oracle,
and what the trained network gains over the plain extrapolation.

The GPU computes with BF16 operands (features, weights, hidden activations,
back-propagated gradients) and FP32 accumulation.  As for the RHS, every
quantity is a sum of terms that may cancel (a weight gradient sums
dZ_j x_j^T over samples), so the bound is on the error against the size
of the summed terms: || G_gpu - G_oracle || <= tol * || sum_j |dZ_j| |x_j|^T ||,
with tol a few BF16 unit round-offs (2^-8).
"""
import numpy as np
import pytest

from oracle import fr, mlp as omlp
from tests import parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

BF16_TOL = 3e-2


@pytest.fixture(scope="module")
def abi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_14027_gb300 import build
    build.build()
    from paper_2107_14027_gb300 import abi as _abi
    return _abi


def _bf16(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(torch.bfloat16)


@pytest.mark.parametrize("amode,bmode", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_tensor_core_gemm_all_orientations(abi, amode, bmode):
    rng = np.random.default_rng(amode * 2 + bmode)
    N, M, K = 70, 130, 100          # ragged against the 64 x 64 x 32 tiles
    A = rng.normal(size=(N, K))
    B = rng.normal(size=(K, M))
    Ab, Bb = _bf16(A), _bf16(B)
    A_ref = Ab.float().numpy().astype(np.float64)
    B_ref = Bb.float().numpy().astype(np.float64)
    Ad = (Ab if amode == 0 else Ab.t().contiguous()).cuda()
    Bd = (Bb if bmode == 0 else Bb.t().contiguous()).cuda()
    lda = K if amode == 0 else N
    ldb = M if bmode == 0 else K
    C = torch.zeros((N, M), dtype=torch.float32, device="cuda")
    abi.fr_gemm_bf16(amode, bmode, N, M, K, Ad, lda, Bd, ldb, C, M)
    torch.cuda.synchronize()
    ref = A_ref @ B_ref
    err = np.abs(C.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err < 1e-5, err


@pytest.mark.parametrize("K,lda", [(4875, 4875), (264, 264), (100, 104), (37, 40)])
def test_tensor_core_gemm_pipelined_path(abi, K, lda):
    """The forward orientation with 16-byte aligned B rows takes the pipelined
    kernel (128 x 128 tiles, cp.async, ldmatrix); A rows aligned (lda % 8 == 0)
    or not (the first layer's K = 3 n_v (p+1)^d); ragged N, M, K."""
    rng = np.random.default_rng(K)
    N, M, ldb = 300, 1000, 1024
    A = rng.normal(size=(N, K))
    B = rng.normal(size=(K, M))
    Ab, Bb = _bf16(A), _bf16(B)
    A_ref = Ab.float().numpy().astype(np.float64)
    B_ref = Bb.float().numpy().astype(np.float64)
    Ad = torch.zeros((N, lda), dtype=torch.bfloat16)
    Ad[:, :K] = Ab
    Bd = torch.zeros((K, ldb), dtype=torch.bfloat16)
    Bd[:, :M] = Bb
    Ad, Bd = Ad.cuda(), Bd.cuda()
    C = torch.full((N, M), float("nan"), dtype=torch.float32, device="cuda")
    abi.fr_gemm_bf16(0, 0, N, M, K, Ad, lda, Bd, ldb, C, M)
    torch.cuda.synchronize()
    ref = A_ref @ B_ref
    err = np.abs(C.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err < 3e-5 * max(1.0, np.sqrt(K / 100.0)), err


def _history_case(abi, precision=64, n=(5, 4), order=1, steps=4, dtau=1e-2):
    """A small run with four history levels; returns host copies."""
    d = len(n)
    nv = 1 + d + d * d
    U0, mesh, prm, lo, hi = parity.make_case(n, order)
    prm = fr.Params(2.5, 1.0 / 400.0, 5e-3)
    ctx = abi.fr_create(n, lo, hi, order, nv, prm.zeta, prm.nu, prm.T, precision)
    Ud = abi.pack_state(ctx, U0, precision)
    abi.fr_dual_init(ctx, Ud)
    levels = [abi.unpack_state(ctx, Ud, nv)]
    for _ in range(steps):
        abi.fr_dual_step(ctx, Ud, 1e-2, dtau, 1e-8, 400, check_every=10, allow_noconv=True)
        levels.append(abi.unpack_state(ctx, Ud, nv))
    return ctx, Ud, levels, nv


def _unflatten(flat, sizes):
    out, off = [], 0
    for (o, i) in sizes:
        W = flat[off:off + o * i].reshape(o, i)
        off += o * i
        b = flat[off:off + o]
        off += o
        out.append((W.astype(np.float64), b.astype(np.float64)))
    return out


MLP_CASES = [
    # (mesh, order, hidden, samples): a small 2-D net, and the production
    # shape of the dual-time workload's network (3-D p = 4: 4875 -> 256 ->
    # 256 -> 1625) on 512 samples
    ((5, 4), 1, 32, 40),
    ((8, 8, 8), 4, 256, 512),
]


@pytest.mark.parametrize("kind", ["tcgen05", "mma_sync"])
@pytest.mark.parametrize("n,order,H,S", MLP_CASES)
def test_loss_gradients_adam_and_prediction_match_oracle(abi, n, order, H, S, kind):
    """Both GEMM kernels of the forward products (the tensor-memory kernel,
    the default, and the warp-level mma.sync kernel) against the oracle."""
    d = len(n)
    abi.fr_gemm_set_kernel(abi.FR_GEMM_AUTO if kind == "tcgen05" else abi.FR_GEMM_MMA_SYNC)
    ctx, Ud, levels, nv = _history_case(abi, n=n, order=order, dtau=1e-2 if d == 2 else 2e-3)
    net = abi.fr_mlp_create(ctx, H, S, seed=7)
    try:
        K, Hh, NO, _, npar = abi.fr_mlp_info(net)
        assert (K, Hh, NO) == (3 * NO, H, nv * (order + 1) ** d)
        el = abi.fr_mlp_collect(net, S, seed=3)
        scales = abi.fr_mlp_params(net, 2, count=4 * nv)
        s0, s1, s2 = scales[:nv], scales[nv:2 * nv], scales[2 * nv:3 * nv]
        # the feature scales are the RMS of the blocks over the mesh
        Un, Unm1, Unm2, Unp1 = levels[-2], levels[-3], levels[-4], levels[-1]
        np.testing.assert_allclose(s0, np.sqrt(np.mean(Un ** 2, axis=(1, 2))), rtol=1e-5)
        np.testing.assert_allclose(s1, np.sqrt(np.mean((Un - Unm1) ** 2, axis=(1, 2))), rtol=1e-5)
        np.testing.assert_allclose(
            s2, np.sqrt(np.mean((Un - 2 * Unm1 + Unm2) ** 2, axis=(1, 2))), rtol=1e-5)
        # the collected samples are the oracle's features (to BF16) and raw targets
        Xg = abi.fr_mlp_params(net, 3, count=K * S).reshape(K, S)
        Xo = omlp.features(Un, Unm1, Unm2, (s0, s1, s2), el)
        np.testing.assert_allclose(Xg, Xo, rtol=2 ** -8, atol=1e-30)
        Tr = abi.fr_mlp_params(net, 4, count=NO * S).reshape(NO, S)
        raw_o = (Unp1 - omlp.extrapolate(Un, Unm1, Unm2))[:, :, el].reshape(NO, S)
        np.testing.assert_allclose(Tr, raw_o, rtol=1e-6, atol=1e-12 * np.abs(raw_o).max())
        loss = abi.fr_mlp_loss_grad(net)
        scales = abi.fr_mlp_params(net, 2, count=4 * nv)
        t = scales[3 * nv:].astype(np.float64)
        sizes = [(H, K), (H, H), (NO, H)]
        params = _unflatten(abi.fr_mlp_params(net, 0, count=npar), sizes)
        grads = _unflatten(abi.fr_mlp_params(net, 1, count=npar), sizes)
        # the network's inputs are the collected (BF16-rounded) features,
        # checked against the oracle's features above
        X = Xg.astype(np.float64)
        Tg = omlp.targets(Unp1, Un, Unm1, Unm2, t, el)
        # output scales: RMS of the raw corrections of the samples
        raw = (Unp1 - omlp.extrapolate(Un, Unm1, Unm2))[:, :, el]
        np.testing.assert_allclose(t, np.sqrt(np.mean(raw ** 2, axis=(1, 2))), rtol=1e-4)
        Y, cache = omlp.forward(params, X)
        lo = omlp.loss(Y, Tg)
        go = omlp.backward(params, cache, Y, Tg)
        assert abs(loss - lo) <= BF16_TOL * lo, (loss, lo)
        # magnitudes of the summed terms of each gradient (oracle quantities)
        Xo_, Z1o, H1o, Z2o, H2o = cache
        dYo = 2.0 * (Y - Tg) / Y.size
        dZ2o = (params[2][0].T @ dYo) * (Z2o > 0)
        dZ1o = (params[1][0].T @ dZ2o) * (Z1o > 0)
        mags = [(np.abs(dZ1o) @ np.abs(Xo_).T, np.abs(dZ1o).sum(1)),
                (np.abs(dZ2o) @ np.abs(H1o).T, np.abs(dZ2o).sum(1)),
                (np.abs(dYo) @ np.abs(H2o).T, np.abs(dYo).sum(1))]
        Xe = omlp.features(Un, Unm1, Unm2, (s0, s1, s2), el)
        Ye, ce = omlp.forward(params, Xe)
        ge = omlp.backward(params, ce, Ye, Tg)
        # (diagnostic: the FP64 gradient itself is sensitive to the BF16
        # rounding of the features - a few samples sit next to ReLU kinks)
        print("exact-feature oracle vs rounded-feature oracle, W1:",
              np.linalg.norm(ge[0][0] - go[0][0]) / np.linalg.norm(mags[0][0]))
        for li, ((gW, gb), (oW, ob), (mW, mb)) in enumerate(zip(grads, go, mags)):
            for nm, a, b, mg in (("W", gW, oW, mW), ("b", gb, ob, mb)):
                err = np.linalg.norm(a - b) / np.linalg.norm(mg)
                assert err < BF16_TOL, (f"{nm}{li + 1}", err)
        # one Adam step from the same gradients as the oracle's Adam
        abi.fr_mlp_train(net, 1, 1e-3)
        new = _unflatten(abi.fr_mlp_params(net, 0, count=npar), sizes)
        expect = omlp.Adam(params, lr=1e-3).step(params, grads)
        for (W0, b0), (W1, b1), (E1, e1) in zip(params, new, expect):
            for p0, p1, pe in ((W0, W1, E1), (b0, b1, e1)):
                np.testing.assert_allclose(p0 - p1, p0 - pe, rtol=1e-4, atol=1e-7)
        # prediction from the three newest levels against the oracle network
        Ug = abi.new_state(ctx, 64)
        Vg = abi.new_velocity(ctx, d, order)
        abi.fr_mlp_predict(net, Ug, Vg)
        torch.cuda.synchronize()
        G = abi.unpack_state(ctx, Ug, nv)
        a, b_, c = levels[-1], levels[-2], levels[-3]
        ne = a.shape[2]
        Xall = omlp.features(a, b_, c, (s0, s1, s2), np.arange(ne))
        Yall, _ = omlp.forward(new, Xall)
        Go = omlp.apply_guess(Yall, a, b_, c, t)
        corr_gpu = G - omlp.extrapolate(a, b_, c)
        corr_ref = Go - omlp.extrapolate(a, b_, c)
        _, (Xa, Z1a, H1a, Z2a, H2a) = omlp.forward(new, Xall)
        mag = (np.abs(new[2][0]) @ np.abs(H2a) + np.abs(new[2][1])[:, None])
        mag = mag.reshape(corr_ref.shape) * t[:, None, None]
        assert np.linalg.norm(corr_gpu - corr_ref) < BF16_TOL * np.linalg.norm(mag)
        stride, _, _ = abi.fr_layout(ctx)
        V = Vg[:, :ne].cpu().numpy().reshape(d, -1, ne)
        np.testing.assert_allclose(V, G[1:1 + d], rtol=0, atol=1e-12)
        abi.fr_gemm_check()
    finally:
        abi.fr_gemm_set_kernel(abi.FR_GEMM_AUTO)
        abi.fr_mlp_destroy(net)
        abi.fr_destroy(ctx)


def test_mlp_guess_error_paths(abi):
    ctx, Ud, levels, nv = _history_case(abi, steps=2)
    net = abi.fr_mlp_create(ctx, 16, 8, seed=1)
    try:
        with pytest.raises(abi.FrError):        # three levels only: no target yet
            abi.fr_mlp_collect(net, 4, seed=1)
        with pytest.raises(abi.FrError):        # nothing collected
            abi.fr_mlp_train(net, 1, 1e-3)
        with pytest.raises(abi.FrError):        # untrained network
            abi.fr_mlp_predict(net, abi.new_state(ctx, 64), abi.new_velocity(ctx, 2, 1))
    finally:
        abi.fr_mlp_destroy(net)
        abi.fr_destroy(ctx)


def _chosen_is_best(abi, s):
    """The state iterated is the candidate (extrapolation, network, blend)
    with the smallest initial residual, and its weight is consistent."""
    cand = {0.0: s.res_guess[0], 1.0: s.res_guess[1]}
    if np.isfinite(s.res_blend):
        cand[s.mlp_weight if 0.0 < s.mlp_weight < 1.0 else -1.0] = s.res_blend
    best = min(v for v in cand.values())
    ok = 0.0 <= s.mlp_weight <= 1.0
    ok &= (s.guess_used == abi.FR_GUESS_MLP) == (s.mlp_weight > 0.0)
    return bool(ok and cand.get(s.mlp_weight, np.nan) == best)


def test_learned_guess_gain_over_extrapolation(abi):
    """Train on samples from the first physical steps of a 2-D run, then
    compare the initial residual and the pseudo iterations to tolerance of
    the learned guess with the plain extrapolation on the following steps.
    The fallback guarantees the learned run never starts worse."""
    n, order, nv = (8, 8), 2, 7
    U0, mesh, _, lo, hi = parity.make_case(n, order, noise=False)
    prm = fr.Params(2.5, 1.0 / 400.0, 5e-3)
    dt, dtau, tol = 1e-2, 1e-2, 1e-6
    runs, s_m_of = {}, {}
    for mode in ("plain", "mlp"):
        ctx = abi.fr_create(n, lo, hi, order, nv, prm.zeta, prm.nu, prm.T, 64)
        net = abi.fr_mlp_create(ctx, 64, 4096, seed=11)
        try:
            Ud = abi.pack_state(ctx, U0, 64)
            abi.fr_dual_init(ctx, Ud)
            res = []
            for k in range(14):
                guess = abi.FR_GUESS_EXTRAPOLATE
                if mode == "mlp" and k >= 10:
                    guess = abi.FR_GUESS_MLP
                st, s = abi.fr_dual_step(ctx, Ud, dt, dtau, tol, 6000, check_every=5, guess=guess,
                                         mlp=net, allow_noconv=True)
                res.append((s.iters, s.res, s.guess_used, tuple(s.res_guess)))
                s_m_of[id(res[-1][3])] = s
                if mode == "mlp" and 3 <= k < 10:
                    abi.fr_mlp_collect(net, 64, seed=100 + k)
                if mode == "mlp" and k == 9:
                    abi.fr_mlp_train(net, 300, 2e-3)
            runs[mode] = res
        finally:
            abi.fr_mlp_destroy(net)
            abi.fr_destroy(ctx)
    print("plain", runs["plain"][10:])
    print("mlp", runs["mlp"][10:])
    chosen = 0
    for (it_p, r_p, _, _), (it_m, r_m, used, rg) in zip(runs["plain"][10:], runs["mlp"][10:]):
        assert r_m < tol and r_p < tol
        # the learned step starts from the best of the candidates
        assert _chosen_is_best(abi, s_m_of[id(rg)])
        chosen += used == abi.FR_GUESS_MLP
    # the trained network beats the extrapolation on some held-out step, and
    # the learned run needs fewer pseudo iterations in total
    assert chosen >= 1
    assert sum(r[0] for r in runs["mlp"][10:]) < sum(r[0] for r in runs["plain"][10:])


def test_learned_guess_reads_the_stepping_context_history(abi):
    """A network trained on context A and used by forks B and C of A (same
    history): each fork's guess comes from its own history, so B and C get
    the same guess even after A has moved on, and a context of another
    discretization is refused."""
    n, order, nv = (4, 3, 3), 2, 13
    U0, mesh, prm, lo, hi = parity.make_case(n, order)
    dt, dtau, tol = 1e-2, 1e-2, 1e-8
    ctxs = [abi.fr_create(n, lo, hi, order, nv, prm.zeta, prm.nu, prm.T, 64) for _ in range(3)]
    other = abi.fr_create(n, lo, hi, order + 1, nv, prm.zeta, prm.nu, prm.T, 64)
    A, B, C = ctxs
    net = abi.fr_mlp_create(A, 32, 256, seed=7)
    try:
        Ua = abi.pack_state(A, U0, 64)
        abi.fr_dual_init(A, Ua)
        for k in range(5):
            abi.fr_dual_step(A, Ua, dt, dtau, tol, 40, check_every=10, allow_noconv=True)
            if k >= 2:
                abi.fr_mlp_collect(net, 24, seed=k)
        abi.fr_mlp_train(net, 20, 1e-3)
        abi.fr_dual_copy(B, A)
        abi.fr_dual_copy(C, A)
        Ub, Uc = Ua.clone(), Ua.clone()
        # C steps with the learned guess before A moves on; B after
        _, sc = abi.fr_dual_step(C, Uc, dt, dtau, tol, 3, check_every=3, guess=abi.FR_GUESS_MLP,
                                 mlp=net, allow_noconv=True)
        abi.fr_dual_step(A, Ua, dt, dtau, tol, 40, check_every=10, allow_noconv=True)
        _, sb = abi.fr_dual_step(B, Ub, dt, dtau, tol, 3, check_every=3, guess=abi.FR_GUESS_MLP,
                                 mlp=net, allow_noconv=True)
        torch.cuda.synchronize()
        assert np.isfinite(sb.res_guess[1])
        assert sb.res_guess[1] == sc.res_guess[1] and sb.res_guess[0] == sc.res_guess[0]
        assert torch.equal(Ub, Uc)
        Uo = abi.new_state(other, 64)
        Vo = abi.new_velocity(other, 3, order + 1)
        with pytest.raises(abi.FrError) as ei:
            abi.fr_mlp_predict_for(net, other, Uo, Vo)
        assert ei.value.status == abi.FR_EINVAL
    finally:
        abi.fr_mlp_destroy(net)
        for c in ctxs + [other]:
            abi.fr_destroy(c)


def test_learned_guess_gain_in_3d_through_a_fork(abi):
    """3-D p = 2, 8^3 Taylor-Green (zeta 2.5, nu 1/1600, T_r 5e-3), BDF2
    dt = 1e-2, RK4 dtau = 1e-2 to 1e-6, FP64.  Solver A takes 3 steps, then 7
    more while element samples are collected, trains the network, and a fork
    B of A (same history) takes the held-out steps with the learned guess
    while A takes them with the extrapolation."""
    from paper_2107_14027_gb300 import workloads as W
    n, order, nv = (8, 8, 8), 2, 13
    lo, hi = (-np.pi,) * 3, (np.pi,) * 3
    U0 = W.taylor_green(n, lo, hi, order)
    A = abi.fr_create(n, lo, hi, order, nv, 2.5, 1 / 1600, 5e-3, 64)
    B = abi.fr_create(n, lo, hi, order, nv, 2.5, 1 / 1600, 5e-3, 64)
    net = abi.fr_mlp_create(A, 256, 4096, seed=2021)
    dt, dtau, tol = 1e-2, 1e-2, 1e-6
    try:
        Ua = abi.pack_state(A, U0, 64)
        Ub = Ua.clone()
        abi.fr_dual_init(A, Ua)
        for k in range(1, 11):
            st, _ = abi.fr_dual_step(A, Ua, dt, dtau, tol, 6000, check_every=5)
            if k > 3:
                abi.fr_mlp_collect(net, 4096 // 7, seed=1000 + k)
        abi.fr_mlp_train(net, 300, 2e-3)
        abi.fr_dual_copy(B, A)
        plain, learned, chosen = [], [], 0
        for k in range(4):
            _, sa = abi.fr_dual_step(A, Ua, dt, dtau, tol, 6000, check_every=5)
            _, sb = abi.fr_dual_step(B, Ub, dt, dtau, tol, 6000, check_every=5,
                                     guess=abi.FR_GUESS_MLP, mlp=net)
            assert sa.res < tol and sb.res < tol
            assert _chosen_is_best(abi, sb)
            chosen += sb.guess_used == abi.FR_GUESS_MLP
            plain.append(sa.iters)
            learned.append(sb.iters)
        print("plain", plain, "learned", learned)
        assert chosen >= 1
        assert sum(learned) < 0.8 * sum(plain)
    finally:
        abi.fr_mlp_destroy(net)
        abi.fr_destroy(A)
        abi.fr_destroy(B)


def test_save_load_round_trip(abi, tmp_path):
    """A saved and reloaded network predicts bit for bit what the original
    predicts, and training resumes from the saved Adam state: one more step
    on the same samples gives identical weights.  Foreign and corrupt files
    are refused."""
    ctx, Ud, levels, nv = _history_case(abi)
    net = abi.fr_mlp_create(ctx, 32, 64, seed=7)
    net2 = None
    other = abi.fr_create((5, 4), (0, 0), (1, 1), 2, nv, 2.5, 1e-3, 5e-3, 64)
    path = str(tmp_path / "net.bin")
    try:
        abi.fr_mlp_collect(net, 40, seed=3)
        abi.fr_mlp_train(net, 5, 1e-3)
        U1, V1 = abi.new_state(ctx, 64), abi.new_velocity(ctx, 2, 1)
        abi.fr_mlp_predict(net, U1, V1)
        abi.fr_mlp_save(net, path)
        net2 = abi.fr_mlp_load(ctx, path, capacity=64)
        U2, V2 = abi.new_state(ctx, 64), abi.new_velocity(ctx, 2, 1)
        abi.fr_mlp_predict(net2, U2, V2)
        torch.cuda.synchronize()
        assert torch.equal(U1, U2) and torch.equal(V1, V2)
        _, _, _, _, npar = abi.fr_mlp_info(net)
        assert np.array_equal(abi.fr_mlp_params(net, 0, count=npar),
                              abi.fr_mlp_params(net2, 0, count=npar))
        abi.fr_mlp_collect(net2, 40, seed=3)       # the same samples, same scales
        l1 = abi.fr_mlp_train_step(net, 1e-3)
        l2 = abi.fr_mlp_train_step(net2, 1e-3)
        assert l1 == l2
        assert np.array_equal(abi.fr_mlp_params(net, 0, count=npar),
                              abi.fr_mlp_params(net2, 0, count=npar))
        with pytest.raises(abi.FrError) as ei:       # another order
            abi.fr_mlp_load(other, path)
        assert ei.value.status == abi.FR_EINVAL
        raw = bytearray(open(path, "rb").read())
        raw[100] ^= 0x5A
        bad = str(tmp_path / "bad.bin")
        open(bad, "wb").write(bytes(raw))
        with pytest.raises(abi.FrError) as ei:       # checksum
            abi.fr_mlp_load(ctx, bad)
        assert "checksum" in abi.fr_last_error()
        with pytest.raises(abi.FrError):
            abi.fr_mlp_load(ctx, str(tmp_path / "missing.bin"))
    finally:
        abi.fr_mlp_destroy(net)
        if net2:
            abi.fr_mlp_destroy(net2)
        abi.fr_destroy(other)
        abi.fr_destroy(ctx)


def test_validation_split_and_weight_decay_match_oracle(abi):
    """With the newest 10 of 40 samples held out and weight decay 0.3: the
    training loss is the oracle's on the other 30, one Adam step is the
    oracle's AdamW step from the GPU gradients, and the validation loss is
    the oracle's on the held-out 10 with the new weights."""
    ctx, Ud, levels, nv = _history_case(abi)
    H, S, NVAL, WD = 32, 40, 10, 0.3
    net = abi.fr_mlp_create(ctx, H, S, seed=9)
    try:
        K, _, NO, _, npar = abi.fr_mlp_info(net)
        el = abi.fr_mlp_collect(net, S, seed=5)
        abi.fr_mlp_set_training(net, NVAL, WD)
        loss = abi.fr_mlp_loss_grad(net)
        scales = abi.fr_mlp_params(net, 2, count=4 * nv)
        t = scales[3 * nv:].astype(np.float64)
        sizes = [(H, K), (H, H), (NO, H)]
        params = _unflatten(abi.fr_mlp_params(net, 0, count=npar), sizes)
        grads = _unflatten(abi.fr_mlp_params(net, 1, count=npar), sizes)
        X = abi.fr_mlp_params(net, 3, count=K * S).reshape(K, S).astype(np.float64)
        Un, Unm1, Unm2, Unp1 = levels[-2], levels[-3], levels[-4], levels[-1]
        Tg = omlp.targets(Unp1, Un, Unm1, Unm2, t, el)
        ntr = S - NVAL
        Y, _ = omlp.forward(params, X[:, :ntr])
        lo = omlp.loss(Y, Tg[:, :ntr])
        assert abs(loss - lo) <= BF16_TOL * lo, (loss, lo)
        abi.fr_mlp_train(net, 1, 1e-3)
        new = _unflatten(abi.fr_mlp_params(net, 0, count=npar), sizes)
        expect = omlp.Adam(params, lr=1e-3, weight_decay=WD).step(params, grads)
        for (W0, b0), (W1, b1), (E1, e1) in zip(params, new, expect):
            for p0, p1, pe in ((W0, W1, E1), (b0, b1, e1)):
                np.testing.assert_allclose(p0 - p1, p0 - pe, rtol=1e-4, atol=1e-7)
        vl = abi.fr_mlp_validation_loss(net)
        Yv, _ = omlp.forward(new, X[:, ntr:])
        lv = omlp.loss(Yv, Tg[:, ntr:])
        assert abs(vl - lv) <= BF16_TOL * lv, (vl, lv)
        with pytest.raises(abi.FrError):
            abi.fr_mlp_set_training(net, -1, 0.0)
    finally:
        abi.fr_mlp_destroy(net)
        abi.fr_destroy(ctx)


def test_learned_guess_gain_on_the_dual_time_workload_24cube(abi):
    """The dual-time workload at a budget size: 3-D p = 4, 24^3 Taylor-Green,
    BDF2 dt = 1e-2, tolerance 1e-6; FP32 RHS with an FP64 twin below the FP32
    floor, P-multigrid cycles (16 iterations on order 1), Anderson mixing (8)
    in the FP64 phase.  Solver A takes 3 + 8 steps while 5000 element samples
    are collected; the network (4875 -> 256 -> 256 -> 1625) trains with the
    newest 500 samples held out and weight decay; a fork B of A then takes 5
    held-out steps with the learned guess while A takes them with the plain
    extrapolation.  Every step converges, and B needs fewer wall-seconds per
    step (host clock around each synchronised step)."""
    import time
    from paper_2107_14027_gb300 import workloads as W
    n, order, nv = (24, 24, 24), 4, 13
    lo, hi = (-np.pi,) * 3, (np.pi,) * 3
    zeta, nu, tr = 2.5, 1.0 / 1600.0, 5e-3
    U0 = W.taylor_green(n, lo, hi, order, dtype=np.float32)
    sched = [(4, 1), (3, 1), (2, 1), (1, 16), (2, 1), (3, 1), (4, 7)]
    solvers, objs = [], []
    try:
        for _ in range(2):
            c = abi.fr_create(n, lo, hi, order, nv, zeta, nu, tr, 32)
            c64 = abi.fr_create(n, lo, hi, order, nv, zeta, nu, tr, 64)
            pm, pm64 = abi.fr_pmg_create(c, 1), abi.fr_pmg_create(c64, 1)
            for x in (pm, pm64):
                abi.fr_pmg_set_cycle(x, sched)
            abi.fr_pmg_set_anderson(pm64, 8)
            objs += [pm, pm64]
            solvers.append((c, c64, pm, pm64, abi.pack_state(c, U0, 32), abi.new_state(c64, 64)))
        net = abi.fr_mlp_create(solvers[0][0], 256, 5000, seed=2021)
        objs.append(("mlp", net))

        def step(i, guess):
            c, c64, pm, pm64, U, U64 = solvers[i]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, s = abi.fr_dual_step(c, U, 1e-2, 1e-3, 1e-6, 120, guess=guess, refine=c64,
                                     U_refine=U64, tol_switch=5e-6, mlp=net, pmg=pm,
                                     refine_pmg=pm64, allow_noconv=True)
            torch.cuda.synchronize()
            return st, s, time.perf_counter() - t0

        A = solvers[0]
        abi.fr_dual_init(A[0], A[4])
        for k in range(11):
            st, _, _ = step(0, abi.FR_GUESS_EXTRAPOLATE)
            assert st == abi.FR_OK
            if k >= 3:
                abi.fr_mlp_collect(net, 625, seed=1000 + k)
        abi.fr_mlp_set_training(net, 500, 1e-2)
        abi.fr_mlp_train(net, 100, 1e-3)
        assert abi.fr_mlp_validation_loss(net) < 1.0    # better than predicting zero
        abi.fr_dual_copy(solvers[1][0], A[0])
        wall = {0: 0.0, 1: 0.0}
        for k in range(5):
            for i, g in ((0, abi.FR_GUESS_EXTRAPOLATE), (1, abi.FR_GUESS_MLP)):
                st, s, w = step(i, g)
                assert st == abi.FR_OK and s.res < 1e-6, (i, k, s.res)
                if i == 1:
                    assert _chosen_is_best(abi, s)
                wall[i] += w
        print("held-out wall-s per step: plain %.3f, learned %.3f" % (wall[0] / 5, wall[1] / 5))
        assert wall[1] < wall[0]
    finally:
        for o in objs:
            if isinstance(o, tuple):
                abi.fr_mlp_destroy(o[1])
            else:
                abi.fr_pmg_destroy(o)
        for c, c64, *_ in solvers:
            abi.fr_destroy(c)
            abi.fr_destroy(c64)


@pytest.mark.parametrize("n,order,q", [((6, 5), 2, 1), ((4, 4, 3), 3, 1), ((4, 3, 3), 4, 2)])
def test_output_degree_projection_matches_oracle(abi, n, order, q):
    """fr_mlp_set_output_degree(q): the collected targets and the predicted
    corrections are the oracle's, projected per element onto degree <= q
    (oracle.mlp.project_degree, pinned on the CPU)."""
    d = len(n)
    ctx, Ud, levels, nv = _history_case(abi, n=n, order=order, dtau=1e-2 if d == 2 else 2e-3)
    S, H = 48, 32
    net = abi.fr_mlp_create(ctx, H, S, seed=5)
    try:
        with pytest.raises(abi.FrError):
            abi.fr_mlp_set_output_degree(net, order + 1)
        abi.fr_mlp_set_output_degree(net, q)
        K, Hh, NO, _, npar = abi.fr_mlp_info(net)
        el = abi.fr_mlp_collect(net, S, seed=9)
        Un, Unm1, Unm2, Unp1 = levels[-2], levels[-3], levels[-4], levels[-1]
        Tr = abi.fr_mlp_params(net, 4, count=NO * S).reshape(NO, S).astype(np.float64)
        raw = (Unp1 - omlp.extrapolate(Un, Unm1, Unm2))[:, :, el].reshape(NO, S)
        ref = omlp.project_degree(raw, order, d, q)
        scale = np.abs(raw).max()
        assert np.abs(Tr - ref).max() <= 1e-5 * scale, np.abs(Tr - ref).max() / scale
        abi.fr_mlp_train(net, 2, 1e-3)
        scales = abi.fr_mlp_params(net, 2, count=4 * nv)
        s0, s1, s2 = scales[:nv], scales[nv:2 * nv], scales[2 * nv:3 * nv]
        t = scales[3 * nv:].astype(np.float64)
        sizes = [(H, K), (H, H), (NO, H)]
        params = _unflatten(abi.fr_mlp_params(net, 0, count=npar), sizes)
        Ug = abi.new_state(ctx, 64)
        Vg = abi.new_velocity(ctx, d, order)
        abi.fr_mlp_predict(net, Ug, Vg)
        torch.cuda.synchronize()
        G = abi.unpack_state(ctx, Ug, nv)
        a, b_, c = levels[-1], levels[-2], levels[-3]
        ne = a.shape[2]
        Xall = omlp.features(a, b_, c, (s0, s1, s2), np.arange(ne))
        Yall, (_, _, _, _, H2a) = omlp.forward(params, Xall)
        Yp = omlp.project_degree(Yall, order, d, q)
        corr_gpu = (G - omlp.extrapolate(a, b_, c)).reshape(NO, ne)
        corr_ref = t.repeat(NO // nv)[:, None] * Yp
        mag = (np.abs(params[2][0]) @ np.abs(H2a) + np.abs(params[2][1])[:, None])
        mag = t.repeat(NO // nv)[:, None] * mag
        assert np.linalg.norm(corr_gpu - corr_ref) < BF16_TOL * np.linalg.norm(mag)
        # the predicted correction has no content above degree q
        np.testing.assert_allclose(omlp.project_degree(corr_gpu, order, d, q), corr_gpu,
                                   rtol=0, atol=1e-5 * np.abs(corr_gpu).max())
    finally:
        abi.fr_mlp_destroy(net)
        abi.fr_destroy(ctx)
