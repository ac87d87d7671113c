// Internal declarations of the per-element MLP (learned initial guess).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "fr_internal.h"

namespace acmhd {

enum { GEMM_A_NK = 0, GEMM_A_KN = 1 };  // A[n][k] (k contiguous) / A[k][n] (n contiguous)
enum { GEMM_B_KM = 0, GEMM_B_MK = 1 };  // B[k][m] (m contiguous) / B[m][k] (k contiguous)

// C[N x M] = A[N x K] . B[K x M] with the epilogue
//   z = acc + bias[n];  z = 0 where mask[n][m] <= 0;  z *= row_scale[n / rows_per_scale]
//   C[n][m] = z (or += z);  Cb[n][m] = bf16(relu ? max(z, 0) : z)
// Every pointer of the epilogue is optional (null).
struct GemmArgs {
  int N, M, K;
  const __nv_bfloat16* A;
  long long lda;
  const __nv_bfloat16* B;
  long long ldb;
  float* C;
  long long ldc;
  __nv_bfloat16* Cb;
  long long ldcb;
  const float* bias;
  const float* mask;
  long long ldm;
  const float* row_scale;
  int rows_per_scale;
  int relu;
  int accumulate;
};

// Four history levels as seen by the MLP kernels: levels 0, 1, 2 are the
// inputs (U^n, U^{n-1}, U^{n-2}); level 3 is the target level U^{n+1}.
template <typename T>
struct MlpHist {
  const T* u[4];        // state levels (precision T), rows (v, pt), stride columns
  const double* v[4];   // FP64 velocity levels, rows (i, pt)
  int dim, nv, npts, ne, stride;
};

// Which kernel serves a GEMM: AUTO takes the tcgen05 kernel (k_gemm_tc.cu,
// every orientation) whenever its TMA alignment rules hold (both operands
// 16-byte aligned with row pitches a multiple of 8 values), the mma.sync
// kernels otherwise; MMA_SYNC always takes the mma.sync kernels.
enum { GEMM_KERNEL_AUTO = 0, GEMM_KERNEL_MMA_SYNC = 1 };
void set_gemm_kernel(int mode);
int get_gemm_kernel();
bool gemm_tc_eligible(int amode, int bmode, const GemmArgs& g);
cudaError_t launch_gemm_tc(int amode, int bmode, const GemmArgs& g, cudaStream_t s);
// Error code left by a tcgen05 GEMM whose bounded wait gave up (0: none;
// reading clears it; synchronises the device).
int gemm_tc_status();

cudaError_t launch_gemm(int amode, int bmode, const GemmArgs& g, cudaStream_t s);
// dst[r][0..cols) = src[r][0..cols), dst rows padded with zeros to ldd
cudaError_t launch_pad_rows(const __nv_bfloat16* src, int rows, int cols, __nv_bfloat16* dst,
                            int ldd, cudaStream_t s);
template <typename T>
cudaError_t launch_gather_features(const MlpHist<T>& h, const int* elems, int ncols,
                                   const float* inv_scale, int Kpad, __nv_bfloat16* X,
                                   long long ldx, cudaStream_t s);
template <typename T>
cudaError_t launch_gather_targets(const MlpHist<T>& h, const int* elems, int ncols, float* Tg,
                                  long long ldt, cudaStream_t s);
template <typename T>
cudaError_t launch_feature_rms(const MlpHist<T>& h, float* rms_out, cudaStream_t s);
template <typename T>
cudaError_t launch_apply_guess(const MlpHist<T>& h, const float* Yc, long long ldy, T* U,
                               double* V, cudaStream_t s);
cudaError_t launch_target_rms(const float* Tg, long long ldt, int ncols, int nv, int npts,
                              float* rms_out, cudaStream_t s);
cudaError_t launch_loss_grad(const float* Y, const float* Tg, long long ld, int NO, int ncols,
                             int npts, const float* inv_tscale, float* dY, __nv_bfloat16* dYb,
                             double* partial, int nparts, cudaStream_t s);
cudaError_t launch_sum_partials(const double* partial, int n, double count, double* out,
                                cudaStream_t s);
cudaError_t launch_row_sum(const float* dZ, long long ld, int nrows, int ncols, float* db,
                           cudaStream_t s);
cudaError_t launch_adam(size_t n, float* p, const float* g, float* m, float* v, __nv_bfloat16* pb,
                        float lr, float b1, float b2, float eps, float c1, float c2, float wd,
                        cudaStream_t s);
cudaError_t launch_to_bf16(size_t n, const float* x, __nv_bfloat16* y, cudaStream_t s);

// Per column and variable of Y[(v npts + pt) * ld + j] (npts = m^dim points,
// pt = i + m j + m^2 k), the tensor-product projection with the 1-D matrix P
// along every axis, in place (columns [0, ncols)).
struct LineProj {
  float P[kMaxM][kMaxM];
};
cudaError_t launch_project_lines(float* Y, long long ld, int ncols, int nv, int m, int dim,
                                 const LineProj& p, cudaStream_t s);

}  // namespace acmhd
