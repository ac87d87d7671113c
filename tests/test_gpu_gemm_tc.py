"""The fifth-generation tensor-core GEMM (tcgen05.mma, TMEM accumulators, TMA
operand tiles) of the network, C[N x M] = A[N x K] . B[K x M] with either
operand stored either way, against numpy on the BF16-rounded operands and
against the warp-level mma.sync kernels, through the C ABI.

Both kernels multiply BF16 values exactly and accumulate in FP32, so the
error bound is a few FP32 unit round-offs of the summed magnitudes:
|C - ref| <= 1e-5 * (|A| |B|) element by element, which covers any
summation order for K up to ~10^4.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def abi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_14027_gb300 import build
    build.build()
    from paper_2107_14027_gb300 import abi as _abi
    yield _abi
    _abi.fr_gemm_set_kernel(_abi.FR_GEMM_AUTO)


def _case(N, M, K, lda, ldb, seed):
    rng = np.random.default_rng(seed)
    A = torch.from_numpy(rng.normal(size=(N, K)).astype(np.float32)).to(torch.bfloat16)
    B = torch.from_numpy(rng.normal(size=(K, M)).astype(np.float32)).to(torch.bfloat16)
    Ad = torch.zeros((N, lda), dtype=torch.bfloat16)
    Ad[:, :K] = A
    Bd = torch.zeros((K, ldb), dtype=torch.bfloat16)
    Bd[:, :M] = B
    A64 = A.float().numpy().astype(np.float64)
    B64 = B.float().numpy().astype(np.float64)
    return Ad.cuda(), Bd.cuda(), A64 @ B64, np.abs(A64) @ np.abs(B64)


def _run(abi, kind, N, M, K, Ad, lda, Bd, ldb):
    abi.fr_gemm_set_kernel(kind)
    C = torch.full((N, M), float("nan"), dtype=torch.float32, device="cuda")
    abi.fr_gemm_bf16(0, 0, N, M, K, Ad, lda, Bd, ldb, C, M)
    abi.fr_gemm_check()
    return C.cpu().numpy().astype(np.float64)


SHAPES = [
    # (N, M, K, lda, ldb): one tile and one K step; ragged in every
    # dimension; several K steps (ring wrap-around) and sample tiles; the
    # network's three layers at a reduced sample count (layer 1 with the
    # padded W1 pitch); fewer tiles than SMs and more tiles than SMs
    (256, 128, 64, 64, 128),
    (70, 130, 100, 104, 136),
    (16, 8, 8, 8, 8),
    (300, 1000, 264, 264, 1024),
    (256, 4096, 4875, 4880, 4096),
    (256, 2000, 256, 256, 2000),
    (1625, 700, 256, 256, 704),
    (257, 40000, 72, 72, 40000),
]


@pytest.mark.parametrize("N,M,K,lda,ldb", SHAPES)
def test_tcgen05_gemm_vs_numpy(abi, N, M, K, lda, ldb):
    Ad, Bd, ref, mag = _case(N, M, K, lda, ldb, seed=N * 7 + M + K)
    C = _run(abi, abi.FR_GEMM_AUTO, N, M, K, Ad, lda, Bd, ldb)
    assert np.all(np.isfinite(C))
    bad = np.abs(C - ref) > 1e-5 * mag + 1e-30
    assert not bad.any(), (int(bad.sum()), float(np.max(np.abs(C - ref) / (mag + 1e-30))))


@pytest.mark.parametrize("N,M,K,lda,ldb", [SHAPES[1], SHAPES[3], SHAPES[6]])
def test_tcgen05_gemm_matches_mma_sync(abi, N, M, K, lda, ldb):
    """Same operands through both kernels: equal within the FP32 accumulation
    bound (the summation orders differ)."""
    Ad, Bd, ref, mag = _case(N, M, K, lda, ldb, seed=3)
    C_tc = _run(abi, abi.FR_GEMM_AUTO, N, M, K, Ad, lda, Bd, ldb)
    C_ms = _run(abi, abi.FR_GEMM_MMA_SYNC, N, M, K, Ad, lda, Bd, ldb)
    assert np.all(np.abs(C_tc - C_ms) <= 2e-5 * mag + 1e-30)


def test_tcgen05_gemm_repeated_calls_identical(abi):
    """The kernel's schedule is fixed (no atomics, no split K): repeated
    calls give the same bits, also on a non-default stream."""
    N, M, K, lda, ldb = SHAPES[4]
    Ad, Bd, _, _ = _case(N, M, K, lda, ldb, seed=11)
    abi.fr_gemm_set_kernel(abi.FR_GEMM_AUTO)
    s = torch.cuda.Stream()
    outs = []
    for stream in (None, s, s):
        C = torch.empty((N, M), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        abi.fr_gemm_bf16(0, 0, N, M, K, Ad, lda, Bd, ldb, C, M, stream)
        abi.fr_gemm_check(stream)
        outs.append(C)
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[1], outs[2])


def test_unaligned_operands_take_mma_sync(abi):
    """lda not a multiple of 8 (TMA needs 16-byte row pitches): the call is
    served by the mma.sync kernel and is still correct."""
    N, M, K = 70, 130, 37
    Ad, Bd, ref, mag = _case(N, M, K, K, 136, seed=5)
    C = _run(abi, abi.FR_GEMM_AUTO, N, M, K, Ad, K, Bd, 136)
    assert np.all(np.abs(C - ref) <= 1e-5 * mag + 1e-30)


def test_set_kernel_rejects_unknown(abi):
    with pytest.raises(abi.FrError):
        abi.fr_gemm_set_kernel(7)


ORIENT_SHAPES = [
    # (N, M, K): one tile; ragged; the weight gradients of the network
    # (dW3: 1625 x 256 over 4500 samples, dW1: 256 x 4875) and W^T dY
    # (256 x 4500 over 1625 features)
    (256, 128, 64),
    (70, 130, 100),
    (1625, 256, 4500),
    (256, 4875, 4500),
    (256, 4500, 1625),
]


def _pad8(n):
    return (n + 7) // 8 * 8


@pytest.mark.parametrize("amode,bmode", [(0, 0), (0, 1), (1, 0), (1, 1)])
@pytest.mark.parametrize("N,M,K", ORIENT_SHAPES)
def test_tcgen05_gemm_every_orientation(abi, amode, bmode, N, M, K):
    """amode 0: A[n][k], 1: A[k][n]; bmode 0: B[k][m], 1: B[m][k] (the
    backward products read the operands the other way), with 16-byte row
    pitches so that the tensor-memory kernel serves all four."""
    rng = np.random.default_rng(N + 3 * M + 7 * K + amode * 2 + bmode)
    A = torch.from_numpy(rng.normal(size=(N, K)).astype(np.float32)).to(torch.bfloat16)
    B = torch.from_numpy(rng.normal(size=(K, M)).astype(np.float32)).to(torch.bfloat16)
    A64 = A.float().numpy().astype(np.float64)
    B64 = B.float().numpy().astype(np.float64)
    As = A if amode == 0 else A.t()
    Bs = B if bmode == 0 else B.t()
    lda, ldb = _pad8(As.shape[1]) + 8, _pad8(Bs.shape[1]) + 8
    Ad = torch.zeros((As.shape[0], lda), dtype=torch.bfloat16)
    Ad[:, :As.shape[1]] = As
    Bd = torch.zeros((Bs.shape[0], ldb), dtype=torch.bfloat16)
    Bd[:, :Bs.shape[1]] = Bs
    Ad, Bd = Ad.cuda(), Bd.cuda()
    abi.fr_gemm_set_kernel(abi.FR_GEMM_AUTO)
    C = torch.full((N, M), float("nan"), dtype=torch.float32, device="cuda")
    abi.fr_gemm_bf16(amode, bmode, N, M, K, Ad, lda, Bd, ldb, C, M)
    abi.fr_gemm_check()
    C = C.cpu().numpy().astype(np.float64)
    ref, mag = A64 @ B64, np.abs(A64) @ np.abs(B64)
    assert np.all(np.isfinite(C))
    bad = np.abs(C - ref) > 1e-5 * mag + 1e-30
    assert not bad.any(), (int(bad.sum()), float(np.max(np.abs(C - ref) / (mag + 1e-30))))
