// Fifth-generation tensor-core GEMM of the per-element MLP (no counterpart in
// the paper; see fr_mlp.cu):
//
//     C[N x M] = W[N x K] . X[K x M]
//
// N output features, K inputs, M samples (elements), the sample index
// contiguous as in the solver state.  The tensor cores compute the
// transposed product D[m][n] = sum_k X[k][m] W[n][k] with D in tensor memory
// (TMEM), so one accumulator lane holds one sample and the epilogue writes
// each output row as 128-byte coalesced stores.  The forward products read
// W as [n][k] and X as [k][m]; the backward products read X as [m][k] (the
// weight gradients dW = dZ . H^T, X = H) or W as [k][n] (W^T dY): the MMA
// takes either operand K-major or MN-major, so all four are the same kernel
// with other TMA boxes and shared-memory descriptors (template XK, WMN).
//
// Design (GB300, sm_103a):
//   * persistent CTAs, one per SM (196 KB of shared memory each), tiles of
//     128 samples x 256 features taken in order with the feature tiles of a
//     sample block adjacent (the X block is then read from HBM once);
//   * warp 0: one thread issues the TMA loads (cp.async.bulk.tensor, 128-byte
//     swizzle) of each K step, 64 deep, into a 4-stage ring of 48 KB: the
//     128 x 64 tile of X (the MMA's A operand: two 64-sample boxes when the
//     samples are contiguous, one box of k rows otherwise) and the 256 x 64
//     tile of W (the B operand: one box of k rows, or four 64-feature boxes);
//   * warp 1: allocates 512 TMEM columns (two 128 x 256 FP32 accumulators)
//     and one thread issues tcgen05.mma (kind::f16, BF16 in, FP32 out,
//     M = 128, N = 256, K = 16), committing each stage back to the loader
//     and each finished accumulator to the epilogue;
//   * warps 2-9: the epilogue, tcgen05.ld of 32 columns at a time from the
//     TMEM lane quarter the warp may access, then bias, mask, per-row scale,
//     FP32 and/or BF16 (ReLU) stores; it drains one accumulator while the
//     MMAs fill the other.
// Every wait on an mbarrier gives up after about two seconds: the kernel then
// records an error (read by gemm_tc_status), stops issuing work, waits (again
// bounded) for its copies and MMAs in flight and frees its TMEM.
#include <cuda.h>
#include <cuda_bf16.h>

#include <cstdint>
#include <atomic>

#include "async_copy.cuh"
#include "fr_mlp.h"
#include "per_device_once.h"

namespace acmhd {

namespace {

constexpr int TBM = 128;                    // samples per tile (MMA M)
constexpr int TBN = 256;                    // features per tile (MMA N)
constexpr int TBK = 64;                     // K per stage: one 128-byte swizzle row of BF16
constexpr int TSTAGES = 4;
constexpr int X_BOX = 64 * TBK * 2;         // one 64-sample x 64-k box: 8 KB
constexpr int X_BYTES = 2 * X_BOX;          // 16 KB
constexpr int W_BYTES = TBN * TBK * 2;      // 32 KB
constexpr int STAGE_BYTES = X_BYTES + W_BYTES;
constexpr int N_EPI_WARPS = 8;
constexpr int TC_THREADS = 32 * (2 + N_EPI_WARPS);
constexpr int TMEM_COLS = 2 * TBN;
constexpr int SMEM_BYTES = 1024 + TSTAGES * STAGE_BYTES + 256;
constexpr unsigned long long WAIT_LIMIT_NS = 2000000000ull;

// instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator (bits
// 4-5 = 1), A and B BF16 (bits 7-9 and 10-12 = 1), A MN-major (bit 15) unless
// X is given k-contiguous, B MN-major (bit 16) when W is given n-contiguous,
// N >> 3 in bits 17-22, M >> 4 in bits 24-28
template <bool XK, bool WMN>
constexpr uint32_t idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | (XK ? 0u : (1u << 15)) | (WMN ? (1u << 16) : 0u) |
         (uint32_t(TBN >> 3) << 17) | (uint32_t(TBM >> 4) << 24);
}

__device__ int g_tc_error = 0;

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
      : "memory");
}

// shared-memory matrix descriptor: start address, leading and stride byte
// offsets (16-byte units), descriptor version 1, 128-byte swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

// the mbarrier completes when every MMA this thread issued before has finished
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
        "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
        "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ void give_up(volatile int* abort, int code) {
  *abort = 1;
  atomicMax(&g_tc_error, code);
}

// Epilogue flags: which parts of GemmArgs a launch uses, so that the code of
// the 32-row chunk carries no run-time tests per value.  EP_ANY tests them
// at run time (combinations the network does not use).
enum : int {
  EP_BIAS = 1, EP_MASK = 2, EP_RSCALE = 4, EP_C = 8, EP_ACC = 16, EP_CB = 32, EP_RELU = 64,
  EP_ANY = 128
};

template <int FL>
__device__ __forceinline__ bool ep_has(int bit, bool runtime) {
  return (FL & EP_ANY) ? runtime : (FL & bit) != 0;
}

// 32 output rows n0 .. n0+31 of sample m (this thread's TMEM lane), values
// v[j] = D[m][n0 + j]: z = v + bias[n]; z = 0 where mask[n][m] <= 0;
// z *= row_scale[n / rows_per_scale]; C[n][m] = z (or += z); Cb[n][m] =
// bf16(relu ? max(z, 0) : z).  Per-row operands are loaded once per chunk
// (lane j holds row n0 + j) and broadcast by shuffles; for each row the warp
// writes 32 consecutive samples.
template <int FL>
__device__ __forceinline__ void epilogue_chunk(const GemmArgs& g, const uint32_t (&v)[32], int n0,
                                               long long m, bool m_ok, int lane) {
  const bool has_bias = ep_has<FL>(EP_BIAS, g.bias != nullptr);
  const bool has_mask = ep_has<FL>(EP_MASK, g.mask != nullptr);
  const bool has_rs = ep_has<FL>(EP_RSCALE, g.row_scale != nullptr);
  const bool has_c = ep_has<FL>(EP_C, g.C != nullptr);
  const bool acc = ep_has<FL>(EP_ACC, g.accumulate != 0);
  const bool has_cb = ep_has<FL>(EP_CB, g.Cb != nullptr);
  const bool relu = ep_has<FL>(EP_RELU, g.relu != 0);
  const int jmax = g.N - n0 < 32 ? g.N - n0 : 32;
  const int nl = n0 + (lane < jmax ? lane : 0);
  const float bias_l = has_bias ? g.bias[nl] : 0.0f;
  const float rs_l = has_rs ? g.row_scale[nl / g.rows_per_scale] : 1.0f;
  float* cp = has_c ? g.C + (long long)n0 * g.ldc + m : nullptr;
  __nv_bfloat16* cbp = has_cb ? g.Cb + (long long)n0 * g.ldcb + m : nullptr;
  const float* mp = has_mask ? g.mask + (long long)n0 * g.ldm + m : nullptr;
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    float z = __uint_as_float(v[j]);
    if (has_bias) z += __shfl_sync(0xffffffffu, bias_l, j);
    const float rs = has_rs ? __shfl_sync(0xffffffffu, rs_l, j) : 1.0f;
    if (j < jmax && m_ok) {
      if (has_mask && !(mp[0] > 0.0f)) z = 0.0f;
      if (has_rs) z *= rs;
      if (has_c) *cp = acc ? *cp + z : z;
      if (has_cb) *cbp = __float2bfloat16(relu ? fmaxf(z, 0.0f) : z);
    }
    if (has_c) cp += g.ldc;
    if (has_cb) cbp += g.ldcb;
    if (has_mask) mp += g.ldm;
  }
}

// XK: X given as [m][k] (k contiguous; the weight-gradient products) instead
// of [k][m].  WMN: W given as [k][n] (n contiguous; W^T dY) instead of [n][k].
template <int FL, bool XK, bool WMN>
__global__ void __launch_bounds__(TC_THREADS, 1)
gemm_tc_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmW,
               const GemmArgs g) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ int abort_flag;
  __shared__ uint32_t tmem_slot;
  volatile int* abort = &abort_flag;

  const uint32_t raw = smem_u32addr(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;  // swizzle atoms need 1024-byte alignment
  const uint32_t bars = base + TSTAGES * STAGE_BYTES;
  auto full = [&](int s) { return bars + 8u * s; };
  auto empty = [&](int s) { return bars + 8u * (TSTAGES + s); };
  auto tfull = [&](int b) { return bars + 8u * (2 * TSTAGES + b); };
  auto tempty = [&](int b) { return bars + 8u * (2 * TSTAGES + 2 + b); };
  const uint32_t drain = bars + 8u * (2 * TSTAGES + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_tiles = (g.N + TBN - 1) / TBN;
  const int m_tiles = (g.M + TBM - 1) / TBM;
  const long long tiles = (long long)n_tiles * m_tiles;
  const int nk = (g.K + TBK - 1) / TBK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < TSTAGES; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull(b), 1);
      mbar_init(tempty(b), N_EPI_WARPS);
    }
    mbar_init(drain, 1);
    abort_flag = 0;
    mbar_init_fence();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32addr(&tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // loader
      int s = 0;
      uint32_t ph = 0;
      int armed[TSTAGES];
      for (int i = 0; i < TSTAGES; ++i) armed[i] = -1;
      bool ok = true;
      for (long long t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
        const int nt = (int)(t % n_tiles), mt = (int)(t / n_tiles);
        for (int kb = 0; kb < nk; ++kb) {
          if (!mbar_wait(empty(s), ph ^ 1u, WAIT_LIMIT_NS, abort)) {
            give_up(abort, 1);
            ok = false;
            break;
          }
          const uint32_t xs = base + s * STAGE_BYTES, ws = xs + X_BYTES;
          mbar_arrive_expect_tx(full(s), STAGE_BYTES);
          if (XK) {
            // one 128-sample x 64-k box, rows of k
            tma_load_2d(xs, &tmX, full(s), kb * TBK, mt * TBM);
          } else {
            // two 64-sample x 64-k boxes, rows of samples
            tma_load_2d(xs, &tmX, full(s), mt * TBM, kb * TBK);
            tma_load_2d(xs + X_BOX, &tmX, full(s), mt * TBM + 64, kb * TBK);
          }
          if (WMN) {
            // four 64-feature x 64-k boxes, rows of features
#pragma unroll
            for (int q4 = 0; q4 < 4; ++q4)
              tma_load_2d(ws + q4 * X_BOX, &tmW, full(s), nt * TBN + 64 * q4, kb * TBK);
          } else {
            tma_load_2d(ws, &tmW, full(s), kb * TBK, nt * TBN);
          }
          armed[s] = (int)ph;
          if (++s == TSTAGES) {
            s = 0;
            ph ^= 1u;
          }
        }
      }
      // copies in flight land before the CTA may exit (bounded)
      for (int i = 0; i < TSTAGES; ++i)
        if (armed[i] >= 0 && !mbar_wait(full(i), (uint32_t)armed[i], WAIT_LIMIT_NS)) give_up(abort, 2);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer
      int s = 0, i = 0;
      uint32_t ph = 0;
      bool ok = true;
      for (long long t = blockIdx.x; t < tiles && ok; t += gridDim.x, ++i) {
        const int b = i & 1;
        const uint32_t bph = (uint32_t)(i >> 1) & 1u;
        if (!mbar_wait(tempty(b), bph ^ 1u, WAIT_LIMIT_NS, abort)) {
          give_up(abort, 3);
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem_base + (uint32_t)(b * TBN);
        for (int kb = 0; kb < nk; ++kb) {
          if (!mbar_wait(full(s), ph, WAIT_LIMIT_NS, abort)) {
            give_up(abort, 4);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t xs = base + s * STAGE_BYTES, ws = xs + X_BYTES;
#pragma unroll
          for (int k = 0; k < TBK / 16; ++k) {
            // X: 64-sample blocks 8 KB apart (LBO), 8-row k groups 1 KB apart (SBO);
            // 16 k rows = 2 KB per MMA.  W: 8-row groups 1 KB apart; 16 k = 32 bytes.
            // K-major operands (rows of 64 k): 8-row groups 1 KB apart, 16 k = 32 bytes.
            const uint64_t adesc = XK ? smem_desc(xs + k * 32, 16, 1024)
                                      : smem_desc(xs + k * 2048, X_BOX, 1024);
            const uint64_t bdesc = WMN ? smem_desc(ws + k * 2048, X_BOX, 1024)
                                       : smem_desc(ws + k * 32, 16, 1024);
            tc_mma(d, adesc, bdesc, idesc<XK, WMN>(), (kb | k) != 0 ? 1u : 0u);
          }
          tc_commit(empty(s));
          if (++s == TSTAGES) {
            s = 0;
            ph ^= 1u;
          }
        }
        if (ok) tc_commit(tfull(b));
      }
      // every MMA issued has finished before TMEM is freed (bounded)
      tc_commit(drain);
      if (!mbar_wait(drain, 0, WAIT_LIMIT_NS)) give_up(abort, 5);
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (its samples) and
    // half (w - 2) / 4 of the 256 columns (features)
    const int q = warp & 3, half = (warp - 2) >> 2;
    int i = 0;
    for (long long t = blockIdx.x; t < tiles; t += gridDim.x, ++i) {
      const int b = i & 1;
      const uint32_t bph = (uint32_t)(i >> 1) & 1u;
      // one lane waits; the warp then proceeds (or gives up) as a whole, since
      // tcgen05.ld is a warp-wide instruction
      int ok = 0;
      if (lane == 0) {
        ok = mbar_wait(tfull(b), bph, WAIT_LIMIT_NS, abort) ? 1 : 0;
        if (!ok) give_up(abort, 6);
      }
      if (!__shfl_sync(0xffffffffu, ok, 0)) break;
      tc_fence_after();
      const int nt = (int)(t % n_tiles), mt = (int)(t / n_tiles);
      const long long m = (long long)mt * TBM + q * 32 + lane;
      const bool m_ok = m < g.M;
#pragma unroll 1
      for (int c = 0; c < TBN / 2 / 32; ++c) {
        const int col = half * (TBN / 2) + c * 32;
        const int n0 = nt * TBN + col;
        if (n0 >= g.N) break;
        uint32_t v[32];
        tmem_ld32(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * TBN + col), v);
        epilogue_chunk<FL>(g, v, n0, m, m_ok, lane);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty(b));
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                 const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                 const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
  static const EncodeTiled fn = []() -> EncodeTiled {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<EncodeTiled>(p);
  }();
  return fn;
}

// 2-D BF16 tensor map over rows of `inner` values, `outer` rows `ld` apart,
// boxes of 64 x box_outer with the 128-byte swizzle; zero fill out of range
bool make_map(CUtensorMap* map, const void* ptr, long long inner, long long outer, long long ld,
              int box_outer) {
  const EncodeTiled enc = encode_fn();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {64, (cuuint32_t)box_outer};
  const cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

std::atomic<int> g_tc_mode{GEMM_KERNEL_AUTO};

}  // namespace

void set_gemm_kernel(int mode) { g_tc_mode.store(mode); }
int get_gemm_kernel() { return g_tc_mode.load(); }

bool gemm_tc_eligible(int amode, int bmode, const GemmArgs& g) {
  const auto al = [](const void* p, long long ld, long long inner) {
    return p && (reinterpret_cast<uintptr_t>(p) & 15u) == 0 && ld % 8 == 0 && ld >= inner &&
           ld < (1ll << 36);
  };
  const bool xk = bmode == GEMM_B_MK, wmn = amode == GEMM_A_KN;
  return g_tc_mode.load() != GEMM_KERNEL_MMA_SYNC && (amode == GEMM_A_NK || wmn) &&
         (bmode == GEMM_B_KM || xk) && g.N > 0 && g.M > 0 && g.K > 0 &&
         al(g.A, g.lda, wmn ? g.N : g.K) && al(g.B, g.ldb, xk ? g.K : g.M) &&
         encode_fn() != nullptr;
}

namespace {

template <int FL, bool XK, bool WMN>
cudaError_t launch_tc(const CUtensorMap& mx, const CUtensorMap& mw, const GemmArgs& g, int grid,
                      cudaStream_t s) {
  static PerDeviceOnce attr;  // per instance: the attribute is per device and kernel
  const int st = attr.run([](int* d) { return cudaGetDevice(d); },
                          [] {
                            return cudaFuncSetAttribute(
                                gemm_tc_kernel<FL, XK, WMN>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
                          });
  if (st != 0) return static_cast<cudaError_t>(st);
  gemm_tc_kernel<FL, XK, WMN><<<grid, TC_THREADS, SMEM_BYTES, s>>>(mx, mw, g);
  return cudaGetLastError();
}

// the epilogue operand sets each orientation is used with (forward layers,
// weight gradients, W^T dY masked by the pre-activation, fr_gemm_bf16); any
// other set takes the run-time-tested epilogue
template <bool XK, bool WMN>
cudaError_t dispatch_tc(int fl, const CUtensorMap& mx, const CUtensorMap& mw, const GemmArgs& g,
                        int grid, cudaStream_t s) {
  if (fl == EP_C) return launch_tc<EP_C, XK, WMN>(mx, mw, g, grid, s);
  if (!XK && !WMN) {
    switch (fl) {
      case EP_BIAS | EP_C | EP_CB | EP_RELU:
        return launch_tc<EP_BIAS | EP_C | EP_CB | EP_RELU, XK, WMN>(mx, mw, g, grid, s);
      case EP_BIAS | EP_CB | EP_RELU:
        return launch_tc<EP_BIAS | EP_CB | EP_RELU, XK, WMN>(mx, mw, g, grid, s);
      case EP_BIAS | EP_C: return launch_tc<EP_BIAS | EP_C, XK, WMN>(mx, mw, g, grid, s);
      case EP_BIAS | EP_C | EP_RSCALE:
        return launch_tc<EP_BIAS | EP_C | EP_RSCALE, XK, WMN>(mx, mw, g, grid, s);
      default: break;
    }
  }
  if (!XK && WMN && fl == (EP_MASK | EP_C | EP_CB))
    return launch_tc<EP_MASK | EP_C | EP_CB, XK, WMN>(mx, mw, g, grid, s);
  return launch_tc<EP_ANY, XK, WMN>(mx, mw, g, grid, s);
}

}  // namespace

cudaError_t launch_gemm_tc(int amode, int bmode, const GemmArgs& g, cudaStream_t s) {
  const bool xk = bmode == GEMM_B_MK, wmn = amode == GEMM_A_KN;
  CUtensorMap mx, mw;
  const bool okx = xk ? make_map(&mx, g.B, g.K, g.M, g.ldb, TBM) : make_map(&mx, g.B, g.M, g.K, g.ldb, TBK);
  const bool okw = wmn ? make_map(&mw, g.A, g.N, g.K, g.lda, TBK) : make_map(&mw, g.A, g.K, g.N, g.lda, TBN);
  if (!okx || !okw) return cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const long long tiles =
      (long long)((g.N + TBN - 1) / TBN) * (long long)((g.M + TBM - 1) / TBM);
  const int grid = (int)(tiles < sms ? tiles : sms);
  const int fl = (g.bias ? EP_BIAS : 0) | (g.mask ? EP_MASK : 0) | (g.row_scale ? EP_RSCALE : 0) |
                 (g.C ? EP_C : 0) | (g.C && g.accumulate ? EP_ACC : 0) | (g.Cb ? EP_CB : 0) |
                 (g.Cb && g.relu ? EP_RELU : 0);
  if (!xk && !wmn) return dispatch_tc<false, false>(fl, mx, mw, g, grid, s);
  if (xk && !wmn) return dispatch_tc<true, false>(fl, mx, mw, g, grid, s);
  if (!xk && wmn) return dispatch_tc<false, true>(fl, mx, mw, g, grid, s);
  return dispatch_tc<true, true>(fl, mx, mw, g, grid, s);
}

int gemm_tc_status() {
  int h = 0;
  if (cudaMemcpyFromSymbol(&h, g_tc_error, sizeof(int)) != cudaSuccess) return -1;
  if (h != 0) {
    const int zero = 0;
    cudaMemcpyToSymbol(g_tc_error, &zero, sizeof(int));
  }
  return h;
}

}  // namespace acmhd
