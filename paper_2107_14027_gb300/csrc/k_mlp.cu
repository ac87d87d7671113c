// Kernels of the per-element MLP that predicts the initial guess of a
// physical time step (no counterpart in the paper; see fr_mlp.cu).
//
// All matrices are "features x samples" with the sample (element) index
// contiguous, the layout of the solver state, so a layer is
//     C[N x M] = A[N x K] . B[K x M]      (N outputs, K inputs, M samples)
// and the backward products are the same GEMM with the operands read in
// the other orientation.  The GEMM runs on the tensor cores (mma.sync,
// BF16 operands, FP32 accumulation); weights keep FP32 master copies.
#include <cuda_bf16.h>

#include <cstdint>

#include "fr_device.cuh"
#include "fr_mlp.h"

namespace acmhd {

namespace {

constexpr int TN = 64, TM = 64, TK = 32, PAD = 8, GEMM_THREADS = 128;

__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4],
                                         const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// 64 x 64 output tile per CTA, 4 warps of 32 x 32, K in steps of 32.
// Operand tiles are staged in shared memory as sA[n][k] and sB[m][k] (k
// contiguous), transposing on the way in when the global operand is stored
// the other way; fragments are then plain 32-bit shared loads.
template <int AMODE, int BMODE>
__global__ void __launch_bounds__(GEMM_THREADS) gemm_bf16_kernel(const GemmArgs g) {
  __shared__ __align__(16) __nv_bfloat16 sA[TN][TK + PAD];
  __shared__ __align__(16) __nv_bfloat16 sB[TM][TK + PAD];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wn = warp >> 1, wm = warp & 1;
  const int gid = lane >> 2, tig = lane & 3;
  const int n0 = blockIdx.y * TN, m0 = blockIdx.x * TM;
  const __nv_bfloat16 zero = __float2bfloat16(0.0f);
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.0f;

  for (int k0 = 0; k0 < g.K; k0 += TK) {
    for (int idx = tid; idx < TN * TK; idx += GEMM_THREADS) {
      int n, k;
      if (AMODE == GEMM_A_NK) {
        n = idx / TK;
        k = idx % TK;
      } else {
        k = idx / TN;
        n = idx % TN;
      }
      const long long gn = n0 + n, gk = k0 + k;
      __nv_bfloat16 v = zero;
      if (gn < g.N && gk < g.K) v = (AMODE == GEMM_A_NK) ? g.A[gn * g.lda + gk] : g.A[gk * g.lda + gn];
      sA[n][k] = v;
    }
    for (int idx = tid; idx < TM * TK; idx += GEMM_THREADS) {
      int m, k;
      if (BMODE == GEMM_B_KM) {
        k = idx / TM;
        m = idx % TM;
      } else {
        m = idx / TK;
        k = idx % TK;
      }
      const long long gm = m0 + m, gk = k0 + k;
      __nv_bfloat16 v = zero;
      if (gm < g.M && gk < g.K) v = (BMODE == GEMM_B_KM) ? g.B[gk * g.ldb + gm] : g.B[gm * g.ldb + gk];
      sB[m][k] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; kk += 16) {
      uint32_t af[2][4], bf[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int nb = wn * 32 + i * 16;
        af[i][0] = ld_pair(&sA[nb + gid][kk + tig * 2]);
        af[i][1] = ld_pair(&sA[nb + gid + 8][kk + tig * 2]);
        af[i][2] = ld_pair(&sA[nb + gid][kk + tig * 2 + 8]);
        af[i][3] = ld_pair(&sA[nb + gid + 8][kk + tig * 2 + 8]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int mb = wm * 32 + j * 8;
        bf[j][0] = ld_pair(&sB[mb + gid][kk + tig * 2]);
        bf[j][1] = ld_pair(&sB[mb + gid][kk + tig * 2 + 8]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bf[j]);
    }
    __syncthreads();
  }
  // epilogue: z = acc (+ bias[n]); masked by mask > 0; scaled per row group;
  // stored as FP32 (optionally accumulated) and/or BF16 (optionally relu'd)
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const long long n = n0 + wn * 32 + i * 16 + gid + ((r >= 2) ? 8 : 0);
        const long long m = m0 + wm * 32 + j * 8 + tig * 2 + (r & 1);
        if (n >= g.N || m >= g.M) continue;
        float z = acc[i][j][r];
        if (g.bias) z += g.bias[n];
        if (g.mask && !(g.mask[n * g.ldm + m] > 0.0f)) z = 0.0f;
        if (g.row_scale) z *= g.row_scale[n / g.rows_per_scale];
        if (g.C) g.C[n * g.ldc + m] = g.accumulate ? g.C[n * g.ldc + m] + z : z;
        if (g.Cb) g.Cb[n * g.ldcb + m] = __float2bfloat16(g.relu ? fmaxf(z, 0.0f) : z);
      }
}

// Pipelined kernel for the forward orientation (A[n][k] rows of k, B[k][m]
// rows of m), used when B's rows start on 16-byte boundaries: 128 x 128
// output tile per CTA, 8 warps of 64 x 32, K in steps of 32 through two
// shared-memory stages.  B tiles (the large operand: features or hidden
// activations of every element) arrive by 16-byte cp.async while the
// previous stage is multiplied; A tiles (weights, read by every CTA from
// L2) by cp.async as well when A's rows are 16-byte aligned, else through
// registers loaded one stage ahead.  Fragments come from ldmatrix (A
// row-major, B transposed on the fly).  Out-of-range rows and columns are
// zero-filled (partial copies), so any N, M, K work.
constexpr int FN = 128, FM = 128, FK = 32, FPAD = 8, FAST_THREADS = 256;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// 16-byte copy global -> shared of which the first `bytes` (0..16) are read
// and the rest zero-filled
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
               "r"(bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}

template <bool A_ALIGNED>
__global__ void __launch_bounds__(FAST_THREADS) gemm_bf16_fast_kernel(const GemmArgs g) {
  __shared__ __align__(16) __nv_bfloat16 sA[2][FN][FK + FPAD];
  __shared__ __align__(16) __nv_bfloat16 sB[2][FK][FM + FPAD];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wn = warp >> 2, wm = warp & 3;  // warp tile: rows wn*64.., cols wm*32..
  const int gid = lane >> 2, tig = lane & 3;
  const int n0 = blockIdx.x * FN, m0 = blockIdx.y * FM;
  const int nk = (g.K + FK - 1) / FK;
  const __nv_bfloat16 zero = __float2bfloat16(0.0f);

  // B tile: FK rows of FM values = 512 chunks of 8; thread: 2 chunks
  auto load_b = [&](int st, int k0) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int q = tid + c * FAST_THREADS;
      const int k = q / (FM / 8), mc = (q % (FM / 8)) * 8;
      const long long gk = k0 + k, gm = m0 + mc;
      int bytes = 0;
      const __nv_bfloat16* src = g.B;
      if (gk < g.K && gm < g.M) {
        const long long left = g.M - gm;
        bytes = (left >= 8 ? 8 : (int)left) * 2;
        src = g.B + gk * g.ldb + gm;
      }
      cp_async16(&sB[st][k][mc], src, bytes);
    }
  };
  // A tile: FN rows of FK values = 512 chunks of 8; thread: 2 chunks
  auto load_a_async = [&](int st, int k0) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int q = tid + c * FAST_THREADS;
      const int n = q / (FK / 8), kc = (q % (FK / 8)) * 8;
      const long long gn = n0 + n, gk = k0 + kc;
      int bytes = 0;
      const __nv_bfloat16* src = g.A;
      if (gn < g.N && gk < g.K) {
        const long long left = g.K - gk;
        bytes = (left >= 8 ? 8 : (int)left) * 2;
        src = g.A + gn * g.lda + gk;
      }
      cp_async16(&sA[st][n][kc], src, bytes);
    }
  };
  __nv_bfloat16 areg[16];  // unaligned A: 16 values per thread and stage
  auto load_a_regs = [&](int k0) {
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const int q = tid + c * FAST_THREADS;  // 4096 values = FN x FK
      const int n = q / FK, k = q % FK;
      const long long gn = n0 + n, gk = k0 + k;
      areg[c] = (gn < g.N && gk < g.K) ? g.A[gn * g.lda + gk] : zero;
    }
  };
  auto store_a_regs = [&](int st) {
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const int q = tid + c * FAST_THREADS;
      sA[st][q / FK][q % FK] = areg[c];
    }
  };

  float acc[4][4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.0f;

  // prologue: stage 0
  if (A_ALIGNED) {
    load_a_async(0, 0);
  } else {
    load_a_regs(0);
    store_a_regs(0);
  }
  load_b(0, 0);
  cp_async_commit();

  for (int kt = 0; kt < nk; ++kt) {
    const int st = kt & 1;
    if (kt + 1 < nk) {
      if (A_ALIGNED) load_a_async(st ^ 1, (kt + 1) * FK);
      else load_a_regs((kt + 1) * FK);
      load_b(st ^ 1, (kt + 1) * FK);
    }
    cp_async_commit();
    cp_async_wait1();  // stage kt has arrived
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < FK; kk += 16) {
      uint32_t af[4][4], bfr[2][4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = wn * 64 + i * 16 + (lane & 7) + ((lane >> 3) & 1) * 8;
        ldsm_x4(af[i], &sA[st][r][kk + (lane >> 4) * 8]);
      }
#pragma unroll
      for (int jj = 0; jj < 2; ++jj) {
        // two adjacent 8-column tiles: lanes 0-15 the first, 16-31 the second
        const int kr = kk + (lane & 7) + ((lane >> 3) & 1) * 8;
        const int mc = wm * 32 + jj * 16 + (lane >> 4) * 8;
        ldsm_x4_t(bfr[jj], &sB[st][kr][mc]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint32_t b[2] = {bfr[j >> 1][(j & 1) * 2], bfr[j >> 1][(j & 1) * 2 + 1]};
          mma_bf16(acc[i][j], af[i], b);
        }
    }
    if (!A_ALIGNED && kt + 1 < nk) store_a_regs(st ^ 1);
    __syncthreads();  // stage st is refilled in the next iteration
  }

#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const long long n = n0 + wn * 64 + i * 16 + gid + ((r >= 2) ? 8 : 0);
        const long long m = m0 + wm * 32 + j * 8 + tig * 2 + (r & 1);
        if (n >= g.N || m >= g.M) continue;
        float z = acc[i][j][r];
        if (g.bias) z += g.bias[n];
        if (g.mask && !(g.mask[n * g.ldm + m] > 0.0f)) z = 0.0f;
        if (g.row_scale) z *= g.row_scale[n / g.rows_per_scale];
        if (g.C) g.C[n * g.ldc + m] = g.accumulate ? g.C[n * g.ldc + m] + z : z;
        if (g.Cb) g.Cb[n * g.ldcb + m] = __float2bfloat16(g.relu ? fmaxf(z, 0.0f) : z);
      }
}

// ---------------------------------------------------------------------------
// features, targets and statistics
// ---------------------------------------------------------------------------

// Value of row r (= v * npts + pt), element e of history level `lev`: the
// velocity rows come from the FP64 velocity history, the others from the
// state history (precision T).
template <typename T>
__device__ __forceinline__ double level_value(const MlpHist<T>& h, int lev, int r, int e) {
  const int npts = h.npts;
  if (r >= npts && r < (1 + h.dim) * npts)
    return h.v[lev][(size_t)(r - npts) * h.stride + e];
  return static_cast<double>(h.u[lev][(size_t)r * h.stride + e]);
}

// X[b * NO + r][j] = block b (level, first or second difference) of row r at
// element e_j, divided by its per-variable scale; rows beyond 3 NO are zero.
template <typename T>
__global__ void __launch_bounds__(256)
gather_features_kernel(const MlpHist<T> h, const int* __restrict__ elems, int ncols,
                       const float* __restrict__ inv_scale, int Kpad, __nv_bfloat16* __restrict__ X,
                       long long ldx) {
  const int NO = h.nv * h.npts;
  const long long total = (long long)Kpad * ncols;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(idx % ncols);
    const int row = (int)(idx / ncols);
    float out = 0.0f;
    if (row < 3 * NO) {
      const int b = row / NO, r = row % NO;
      const int e = elems ? elems[j] : j;
      if (e < h.ne) {
        const double u0 = level_value(h, 0, r, e);
        double x = u0;
        if (b >= 1) {
          const double u1 = level_value(h, 1, r, e);
          x = (b == 1) ? u0 - u1 : (u0 - 2.0 * u1 + level_value(h, 2, r, e));
        }
        out = static_cast<float>(x * inv_scale[b * h.nv + r / h.npts]);
      }
    }
    X[(long long)row * ldx + j] = __float2bfloat16(out);
  }
}

// Tg[r][j] = U^{n+1} - (3 U^n - 3 U^{n-1} + U^{n-2}) at row r, element e_j
// (raw, FP32); level 3 of h is U^{n+1}.
template <typename T>
__global__ void __launch_bounds__(256)
gather_targets_kernel(const MlpHist<T> h, const int* __restrict__ elems, int ncols,
                      float* __restrict__ Tg, long long ldt) {
  const int NO = h.nv * h.npts;
  const long long total = (long long)NO * ncols;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(idx % ncols);
    const int r = (int)(idx / ncols);
    const int e = elems[j];
    const double ex = 3.0 * level_value(h, 0, r, e) - 3.0 * level_value(h, 1, r, e) +
                      level_value(h, 2, r, e);
    Tg[(long long)r * ldt + j] = static_cast<float>(level_value(h, 3, r, e) - ex);
  }
}

// Per-variable RMS of block b of the features (b = 0, 1, 2) over real
// elements: one CTA per (block, variable), fixed-order reduction.
template <typename T>
__global__ void __launch_bounds__(256)
feature_rms_kernel(const MlpHist<T> h, float* __restrict__ rms_out) {
  __shared__ double red[256];
  const int b = blockIdx.x / h.nv, v = blockIdx.x % h.nv;
  double s = 0.0;
  const long long total = (long long)h.npts * h.ne;
  for (long long idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int r = v * h.npts + (int)(idx / h.ne);
    const int e = (int)(idx % h.ne);
    const double u0 = level_value(h, 0, r, e);
    double x = u0;
    if (b >= 1) {
      const double u1 = level_value(h, 1, r, e);
      x = (b == 1) ? u0 - u1 : (u0 - 2.0 * u1 + level_value(h, 2, r, e));
    }
    s = fma(x, x, s);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) rms_out[blockIdx.x] = static_cast<float>(sqrt(red[0] / (double)total));
}

// Per-variable RMS of raw targets Tg[NO x ncols]: one CTA per variable.
__global__ void __launch_bounds__(256)
target_rms_kernel(const float* __restrict__ Tg, long long ldt, int ncols, int npts,
                  float* __restrict__ rms_out) {
  __shared__ double red[256];
  const int v = blockIdx.x;
  double s = 0.0;
  const long long total = (long long)npts * ncols;
  for (long long idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const long long r = (long long)v * npts + idx / ncols;
    const double x = Tg[r * ldt + idx % ncols];
    s = fma(x, x, s);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) rms_out[v] = static_cast<float>(sqrt(red[0] / (double)total));
}

// dY = 2 (Y - Tg / t_v) / (NO * ncols) as BF16 and FP32; per-CTA partial of
// the squared error (fixed order) for the loss.
__global__ void __launch_bounds__(256)
loss_grad_kernel(const float* __restrict__ Y, const float* __restrict__ Tg, long long ld, int NO,
                 int ncols, int npts, const float* __restrict__ inv_tscale,
                 float* __restrict__ dY, __nv_bfloat16* __restrict__ dYb,
                 double* __restrict__ partial) {
  __shared__ double red[256];
  const long long total = (long long)NO * ncols;
  const double norm = 2.0 / (double)total;
  double s = 0.0;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long r = idx / ncols, j = idx % ncols;
    const long long o = r * ld + j;
    const double d = (double)Y[o] - (double)Tg[o] * inv_tscale[r / npts];
    s = fma(d, d, s);
    const float gval = static_cast<float>(norm * d);
    dY[o] = gval;
    dYb[o] = __float2bfloat16(gval);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// loss = sum(partial) / count (one CTA, fixed order)
__global__ void __launch_bounds__(256)
sum_partials_kernel(const double* __restrict__ partial, int n, double count,
                    double* __restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0] / count;
}

// db[n] = sum_m dZ[n][m] (one CTA per row, fixed order)
__global__ void __launch_bounds__(256)
row_sum_kernel(const float* __restrict__ dZ, long long ld, int ncols, float* __restrict__ db) {
  __shared__ double red[256];
  const long long n = blockIdx.x;
  double s = 0.0;
  for (int j = threadIdx.x; j < ncols; j += blockDim.x) s += dZ[n * ld + j];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) db[n] = static_cast<float>(red[0]);
}

// Adam on an FP32 master array p with gradient g; also writes the BF16 copy.
__global__ void __launch_bounds__(256)
adam_kernel(size_t n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
            float* __restrict__ v, __nv_bfloat16* __restrict__ pb, float lr, float b1, float b2,
            float eps, float c1, float c2, float wd) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    // decoupled weight decay (AdamW; wd = 0: plain Adam)
    const float pi = p[i] - lr * ((mi / c1) / (sqrtf(vi / c2) + eps) + wd * p[i]);
    p[i] = pi;
    if (pb) pb[i] = __float2bfloat16(pi);
  }
}

__global__ void __launch_bounds__(256)
to_bf16_kernel(size_t n, const float* __restrict__ x, __nv_bfloat16* __restrict__ y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16(x[i]);
}

// Guess of the new level: U = 3U^n - 3U^{n-1} + U^{n-2} + Yc (row r, element
// e; Yc already scaled by the output scale), the velocity rows in FP64 into V.
template <typename T>
__global__ void __launch_bounds__(256)
apply_guess_kernel(const MlpHist<T> h, const float* __restrict__ Yc, long long ldy,
                   T* __restrict__ U, double* __restrict__ V) {
  const int NO = h.nv * h.npts;
  const long long total = (long long)NO * h.stride;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(idx / h.stride), e = (int)(idx % h.stride);
    if (e >= h.ne) continue;
    const double g = 3.0 * level_value(h, 0, r, e) - 3.0 * level_value(h, 1, r, e) +
                     level_value(h, 2, r, e) + (double)Yc[(long long)r * ldy + e];
    U[(size_t)r * h.stride + e] = static_cast<T>(g);
    if (r >= h.npts && r < (1 + h.dim) * h.npts) V[(size_t)(r - h.npts) * h.stride + e] = g;
  }
}

__global__ void __launch_bounds__(256)
pad_rows_kernel(const __nv_bfloat16* __restrict__ src, int rows, int cols,
                __nv_bfloat16* __restrict__ dst, int ldd) {
  const long long total = (long long)rows * ldd;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / ldd, c = i % ldd;
    dst[i] = c < cols ? src[r * cols + c] : __float2bfloat16(0.0f);
  }
}

// One line of M points along `axis` of one variable of one column per thread
// (columns fastest: every access is a contiguous row segment), in place.
template <int M>
__global__ void __launch_bounds__(256)
project_lines_kernel(float* __restrict__ Y, long long ld, int ncols, int nv, int dim, int axis,
                     const LineProj p) {
  const int npts = dim == 3 ? M * M * M : M * M;
  const int nl = npts / M;
  const int ma = axis == 0 ? 1 : (axis == 1 ? M : M * M);
  const long long total = (long long)ncols * nv * nl;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long j = idx % ncols;
    const long long rest = idx / ncols;
    const int l = (int)(rest % nl), v = (int)(rest / nl);
    const int base = v * npts + (l % ma) + ma * M * (l / ma);
    float x[M];
#pragma unroll
    for (int t = 0; t < M; ++t) x[t] = Y[(long long)(base + ma * t) * ld + j];
#pragma unroll
    for (int i = 0; i < M; ++i) {
      float y = 0.0f;
#pragma unroll
      for (int k = 0; k < M; ++k) y = fmaf(p.P[i][k], x[k], y);
      Y[(long long)(base + ma * i) * ld + j] = y;
    }
  }
}

int blocks_for(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}

}  // namespace

cudaError_t launch_gemm(int amode, int bmode, const GemmArgs& g, cudaStream_t s) {
  if (gemm_tc_eligible(amode, bmode, g)) return launch_gemm_tc(amode, bmode, g, s);
  const auto a16 = [](const void* p, long long ld) {
    return (reinterpret_cast<uintptr_t>(p) & 15u) == 0 && ld % 8 == 0;
  };
  if (amode == GEMM_A_NK && bmode == GEMM_B_KM && a16(g.B, g.ldb) &&
      (g.M + FM - 1) / FM <= 65535) {
    // N tiles fastest, so the CTAs that share a B tile run together (L2)
    const dim3 grid((g.N + FN - 1) / FN, (g.M + FM - 1) / FM);
    if (a16(g.A, g.lda))
      gemm_bf16_fast_kernel<true><<<grid, FAST_THREADS, 0, s>>>(g);
    else
      gemm_bf16_fast_kernel<false><<<grid, FAST_THREADS, 0, s>>>(g);
    return cudaGetLastError();
  }
  const dim3 grid((g.M + TM - 1) / TM, (g.N + TN - 1) / TN);
  if (amode == GEMM_A_NK && bmode == GEMM_B_KM)
    gemm_bf16_kernel<GEMM_A_NK, GEMM_B_KM><<<grid, GEMM_THREADS, 0, s>>>(g);
  else if (amode == GEMM_A_NK && bmode == GEMM_B_MK)
    gemm_bf16_kernel<GEMM_A_NK, GEMM_B_MK><<<grid, GEMM_THREADS, 0, s>>>(g);
  else if (amode == GEMM_A_KN && bmode == GEMM_B_KM)
    gemm_bf16_kernel<GEMM_A_KN, GEMM_B_KM><<<grid, GEMM_THREADS, 0, s>>>(g);
  else if (amode == GEMM_A_KN && bmode == GEMM_B_MK)
    gemm_bf16_kernel<GEMM_A_KN, GEMM_B_MK><<<grid, GEMM_THREADS, 0, s>>>(g);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_pad_rows(const __nv_bfloat16* src, int rows, int cols, __nv_bfloat16* dst,
                            int ldd, cudaStream_t s) {
  pad_rows_kernel<<<blocks_for((long long)rows * ldd), 256, 0, s>>>(src, rows, cols, dst, ldd);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gather_features(const MlpHist<T>& h, const int* elems, int ncols,
                                   const float* inv_scale, int Kpad, __nv_bfloat16* X,
                                   long long ldx, cudaStream_t s) {
  gather_features_kernel<T><<<blocks_for((long long)Kpad * ncols), 256, 0, s>>>(
      h, elems, ncols, inv_scale, Kpad, X, ldx);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gather_targets(const MlpHist<T>& h, const int* elems, int ncols, float* Tg,
                                  long long ldt, cudaStream_t s) {
  gather_targets_kernel<T><<<blocks_for((long long)h.nv * h.npts * ncols), 256, 0, s>>>(
      h, elems, ncols, Tg, ldt);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_feature_rms(const MlpHist<T>& h, float* rms_out, cudaStream_t s) {
  feature_rms_kernel<T><<<3 * h.nv, 256, 0, s>>>(h, rms_out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_apply_guess(const MlpHist<T>& h, const float* Yc, long long ldy, T* U,
                               double* V, cudaStream_t s) {
  apply_guess_kernel<T><<<blocks_for((long long)h.nv * h.npts * h.stride), 256, 0, s>>>(
      h, Yc, ldy, U, V);
  return cudaGetLastError();
}

#define ACMHD_MLP_INST(T)                                                                       \
  template cudaError_t launch_gather_features<T>(const MlpHist<T>&, const int*, int,           \
                                                 const float*, int, __nv_bfloat16*, long long, \
                                                 cudaStream_t);                                \
  template cudaError_t launch_gather_targets<T>(const MlpHist<T>&, const int*, int, float*,    \
                                                long long, cudaStream_t);                      \
  template cudaError_t launch_feature_rms<T>(const MlpHist<T>&, float*, cudaStream_t);         \
  template cudaError_t launch_apply_guess<T>(const MlpHist<T>&, const float*, long long, T*,   \
                                             double*, cudaStream_t);
ACMHD_MLP_INST(float)
ACMHD_MLP_INST(double)
#undef ACMHD_MLP_INST

cudaError_t launch_target_rms(const float* Tg, long long ldt, int ncols, int nv, int npts,
                              float* rms_out, cudaStream_t s) {
  target_rms_kernel<<<nv, 256, 0, s>>>(Tg, ldt, ncols, npts, rms_out);
  return cudaGetLastError();
}

cudaError_t launch_loss_grad(const float* Y, const float* Tg, long long ld, int NO, int ncols,
                             int npts, const float* inv_tscale, float* dY, __nv_bfloat16* dYb,
                             double* partial, int nparts, cudaStream_t s) {
  loss_grad_kernel<<<nparts, 256, 0, s>>>(Y, Tg, ld, NO, ncols, npts, inv_tscale, dY, dYb,
                                          partial);
  return cudaGetLastError();
}

cudaError_t launch_sum_partials(const double* partial, int n, double count, double* out,
                                cudaStream_t s) {
  sum_partials_kernel<<<1, 256, 0, s>>>(partial, n, count, out);
  return cudaGetLastError();
}

cudaError_t launch_row_sum(const float* dZ, long long ld, int nrows, int ncols, float* db,
                           cudaStream_t s) {
  row_sum_kernel<<<nrows, 256, 0, s>>>(dZ, ld, ncols, db);
  return cudaGetLastError();
}

cudaError_t launch_adam(size_t n, float* p, const float* g, float* m, float* v, __nv_bfloat16* pb,
                        float lr, float b1, float b2, float eps, float c1, float c2, float wd,
                        cudaStream_t s) {
  adam_kernel<<<blocks_for((long long)n), 256, 0, s>>>(n, p, g, m, v, pb, lr, b1, b2, eps, c1, c2,
                                                       wd);
  return cudaGetLastError();
}

cudaError_t launch_project_lines(float* Y, long long ld, int ncols, int nv, int m, int dim,
                                 const LineProj& p, cudaStream_t s) {
  if (ncols < 1) return cudaSuccess;
  const long long total = (long long)ncols * nv * (dim == 3 ? m * m : m);
  for (int axis = 0; axis < dim; ++axis) {
    switch (m) {
#define ACMHD_PROJ(MM)                                                                     \
  case MM:                                                                                 \
    project_lines_kernel<MM><<<blocks_for(total), 256, 0, s>>>(Y, ld, ncols, nv, dim, axis, \
                                                               p);                         \
    break;
      ACMHD_PROJ(2) ACMHD_PROJ(3) ACMHD_PROJ(4) ACMHD_PROJ(5) ACMHD_PROJ(6) ACMHD_PROJ(7)
#undef ACMHD_PROJ
      default: return cudaErrorInvalidValue;
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_to_bf16(size_t n, const float* x, __nv_bfloat16* y, cudaStream_t s) {
  to_bf16_kernel<<<blocks_for((long long)n), 256, 0, s>>>(n, x, y);
  return cudaGetLastError();
}

}  // namespace acmhd
