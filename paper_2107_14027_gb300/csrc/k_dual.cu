// Dual time stepping kernels (Sec. 5): BDF in physical time, classical RK4
// in pseudo time, convergence on the RMS of the pseudo RHS over the
// velocity degrees of freedom.
//
// Precision: the right-hand side R(U) runs in the context's precision T.
// The velocity is carried as an FP64 master V (rows 1..d of the state), so
// the physical-time source
//     S_BDF = -(a0 V + a1 V^n + a2 V^{n-1}) / dt = -(a0/dt) V + C,
//     C = -(a1 V^n + a2 V^{n-1}) / dt          (FP64, once per physical step)
// the velocity part of the RK4 update, and the residual norm are FP64; the
// work state U keeps T copies of V for the RHS kernels.
//
// Residual reduction: every thread accumulates a fixed, grid-stride set of
// entries in FP64, each block reduces in a fixed tree order into a partial,
// and one block sums the partials in order: the result does not depend on
// timing.
#include "fr_device.cuh"

namespace acmhd {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  return red[0];
}

// U_V = (T) V, velocity rows of the state
template <typename T>
__global__ void __launch_bounds__(kThreads)
sync_velocity_kernel(size_t nvel, size_t vel0, const double* __restrict__ V, T* __restrict__ U) {
  for (size_t i = blockIdx.x * (size_t)kThreads + threadIdx.x; i < nvel;
       i += (size_t)gridDim.x * kThreads)
    U[vel0 + i] = static_cast<T>(V[i]);
}

// V = (double) U_V, velocity rows of the state
template <typename T>
__global__ void __launch_bounds__(kThreads)
widen_velocity_kernel(size_t nvel, size_t vel0, const T* __restrict__ U, double* __restrict__ V) {
  for (size_t i = blockIdx.x * (size_t)kThreads + threadIdx.x; i < nvel;
       i += (size_t)gridDim.x * kThreads)
    V[i] = static_cast<double>(U[vel0 + i]);
}

// C = c1 Vn + c2 Vnm1
__global__ void __launch_bounds__(kThreads)
bdf_const_kernel(size_t n, double c1, double c2, const double* __restrict__ Vn,
                 const double* __restrict__ Vnm1, double* __restrict__ C) {
  for (size_t i = blockIdx.x * (size_t)kThreads + threadIdx.x; i < n;
       i += (size_t)gridDim.x * kThreads)
    C[i] = (c2 != 0.0) ? fma(c1, Vn[i], c2 * Vnm1[i]) : c1 * Vn[i];
}

// One RK4 stage combination of the dual-time pseudo step.
//   non-velocity rows (T):  as fr_rk_step
//   velocity rows (FP64):   kv = k + C - (a0/dt) Vin, Vin = V (stage 0) or Vs
// At stage 0 the sum of kv^2 over real elements goes to partial[blockIdx.x].
// With point-implicit scaling (P-multigrid smoother), the velocity
// derivative is multiplied by dV and the gradient rows' by dA before the
// combination; the residual partial stays that of the unscaled pseudo RHS.
// dV = dA = 1 leaves every result bit-identical to no scaling.
template <typename T, int STAGE>
__global__ void __launch_bounds__(kThreads)
dual_stage_kernel(size_t n, size_t vel0, size_t nvel, int stride, int ne, double dtau,
                  double a0dt, double dV, T dA, T* __restrict__ U, T* __restrict__ Us,
                  T* __restrict__ acc, const T* __restrict__ k, double* __restrict__ V,
                  double* __restrict__ Vs, double* __restrict__ Vacc,
                  const double* __restrict__ C, double* __restrict__ partial) {
  __shared__ double red[kThreads];
  const double c = (STAGE == 2) ? dtau : (STAGE == 3 ? dtau / 6.0 : 0.5 * dtau);
  const T ct = static_cast<T>(c);
  double sq = 0.0;
  for (size_t i = blockIdx.x * (size_t)kThreads + threadIdx.x; i < n;
       i += (size_t)gridDim.x * kThreads) {
    const bool vel = i >= vel0 && i < vel0 + nvel;
    if (!vel) {
      const T kk = (i >= vel0 + nvel) ? dA * k[i] : k[i];
      if (STAGE == 3) {
        U[i] = fma(ct, acc[i] + kk, U[i]);
      } else {
        acc[i] = (STAGE == 0) ? kk : fma(T(2), kk, acc[i]);
        Us[i] = fma(ct, kk, U[i]);
      }
      continue;
    }
    const size_t j = i - vel0;
    const double vin = (STAGE == 0) ? V[j] : Vs[j];
    const double kv0 = static_cast<double>(k[i]) + fma(-a0dt, vin, C[j]);
    if (STAGE == 0 && (int)(j % (size_t)stride) < ne) sq = fma(kv0, kv0, sq);
    const double kv = dV * kv0;
    if (STAGE == 3) {
      const double vn = fma(c, Vacc[j] + kv, V[j]);
      V[j] = vn;
      U[i] = static_cast<T>(vn);
    } else {
      Vacc[j] = (STAGE == 0) ? kv : fma(2.0, kv, Vacc[j]);
      const double vs = fma(c, kv, V[j]);
      Vs[j] = vs;
      Us[i] = static_cast<T>(vs);
    }
  }
  if (STAGE == 0) {
    const double b = block_sum(sq, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = b;
  }
}

// rms = sqrt(sum(partial) / count), one block, fixed order
__global__ void __launch_bounds__(kThreads)
norm_final_kernel(int nparts, const double* __restrict__ partial, double count,
                  double* __restrict__ out) {
  __shared__ double red[kThreads];
  double s = 0.0;
  for (int i = threadIdx.x; i < nparts; i += kThreads) s += partial[i];
  const double b = block_sum(s, red);
  if (threadIdx.x == 0) *out = sqrt(b / count);
}

// out = c0 x0 + c1 x1 + c2 x2 (x1, x2 may be null when their weight is 0)
template <typename T>
__global__ void __launch_bounds__(kThreads)
combine3_kernel(size_t n, double c0, double c1, double c2, const T* __restrict__ x0,
                const T* __restrict__ x1, const T* __restrict__ x2, T* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)kThreads + threadIdx.x; i < n;
       i += (size_t)gridDim.x * kThreads) {
    double v = c0 * static_cast<double>(x0[i]);
    if (c1 != 0.0) v = fma(c1, static_cast<double>(x1[i]), v);
    if (c2 != 0.0) v = fma(c2, static_cast<double>(x2[i]), v);
    out[i] = static_cast<T>(v);
  }
}

template <typename Tin, typename Tout>
__global__ void __launch_bounds__(kThreads)
convert_kernel(size_t n, const Tin* __restrict__ x, Tout* __restrict__ y) {
  for (size_t i = blockIdx.x * (size_t)kThreads + threadIdx.x; i < n;
       i += (size_t)gridDim.x * kThreads)
    y[i] = static_cast<Tout>(x[i]);
}

// partial sums over the real entries of two FP64 velocity vectors a, b:
// partial[2 blk] = sum a (b - a), partial[2 blk + 1] = sum (b - a)^2
__global__ void __launch_bounds__(kThreads)
pair_dots_kernel(size_t n, int stride, int ne, const double* __restrict__ a,
                 const double* __restrict__ b, double* __restrict__ partial) {
  __shared__ double red[kThreads];
  double s0 = 0.0, s1 = 0.0;
  for (size_t i = blockIdx.x * (size_t)kThreads + threadIdx.x; i < n;
       i += (size_t)gridDim.x * kThreads) {
    if ((int)(i % (size_t)stride) >= ne) continue;
    const double d = b[i] - a[i];
    s0 = fma(a[i], d, s0);
    s1 = fma(d, d, s1);
  }
  const double t0 = block_sum(s0, red);
  if (threadIdx.x == 0) partial[2 * blockIdx.x] = t0;
  __syncthreads();
  const double t1 = block_sum(s1, red);
  if (threadIdx.x == 0) partial[2 * blockIdx.x + 1] = t1;
}

// out[k] = sum over blocks of partial[2 blk + k], fixed order (one block)
__global__ void __launch_bounds__(kThreads)
pair_dots_final_kernel(int nparts, const double* __restrict__ partial, double* __restrict__ out) {
  __shared__ double red[kThreads];
  for (int k = 0; k < 2; ++k) {
    double s = 0.0;
    for (int i = threadIdx.x; i < nparts; i += kThreads) s += partial[2 * i + k];
    const double t = block_sum(s, red);
    if (threadIdx.x == 0) out[k] = t;
    __syncthreads();
  }
}

int grid_blocks(const fr_ctx* c) {
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
  return nsm * 8;
}

}  // namespace

int dual_norm_blocks(const fr_ctx* c) { return grid_blocks(c); }

cudaError_t launch_sync_velocity(const fr_ctx* c, const double* V, void* U, cudaStream_t s) {
  const size_t nvel = (size_t)c->dim * c->npts * c->stride;
  const size_t vel0 = (size_t)c->npts * c->stride;
  const int nb = grid_blocks(c);
  if (c->precision == FR_F32)
    sync_velocity_kernel<float><<<nb, kThreads, 0, s>>>(nvel, vel0, V, static_cast<float*>(U));
  else
    sync_velocity_kernel<double><<<nb, kThreads, 0, s>>>(nvel, vel0, V, static_cast<double*>(U));
  return cudaGetLastError();
}

cudaError_t launch_widen_velocity(const fr_ctx* c, const void* U, double* V, cudaStream_t s) {
  const size_t nvel = (size_t)c->dim * c->npts * c->stride;
  const size_t vel0 = (size_t)c->npts * c->stride;
  const int nb = grid_blocks(c);
  if (c->precision == FR_F32)
    widen_velocity_kernel<float><<<nb, kThreads, 0, s>>>(nvel, vel0, static_cast<const float*>(U), V);
  else
    widen_velocity_kernel<double><<<nb, kThreads, 0, s>>>(nvel, vel0, static_cast<const double*>(U),
                                                          V);
  return cudaGetLastError();
}

cudaError_t launch_bdf_const(const fr_ctx* c, double c1, double c2, const double* Vn,
                             const double* Vnm1, double* C, cudaStream_t s) {
  const size_t n = (size_t)c->dim * c->npts * c->stride;
  bdf_const_kernel<<<grid_blocks(c), kThreads, 0, s>>>(n, c1, c2, Vn, Vnm1, C);
  return cudaGetLastError();
}

template <typename T>
cudaError_t dual_stage_t(const fr_ctx* c, int stage, double dtau, double a0dt, void* U,
                         double* V, const double* C, double* partial, double dV, double dA,
                         cudaStream_t s) {
  const size_t n = (size_t)c->nv * c->npts * c->stride;
  const size_t vel0 = (size_t)c->npts * c->stride;
  const size_t nvel = (size_t)c->dim * c->npts * c->stride;
  const int nb = grid_blocks(c);
  T* u = static_cast<T*>(U);
  T* us = static_cast<T*>(c->rk_stage);
  T* a = static_cast<T*>(c->rk_acc);
  const T* k = static_cast<const T*>(c->rk_k);
  double* vs = c->dual_vs;
  double* va = c->dual_vacc;
  const int st = static_cast<int>(c->stride);
#define ACMHD_STAGE(S)                                                                      \
  dual_stage_kernel<T, S><<<nb, kThreads, 0, s>>>(n, vel0, nvel, st, c->ne, dtau, a0dt, dV, \
                                                  (T)dA, u, us, a, k, V, vs, va, C, partial)
  switch (stage) {
    case 0: ACMHD_STAGE(0); break;
    case 1: ACMHD_STAGE(1); break;
    case 2: ACMHD_STAGE(2); break;
    case 3: ACMHD_STAGE(3); break;
    default: return cudaErrorInvalidValue;
  }
#undef ACMHD_STAGE
  return cudaGetLastError();
}

cudaError_t launch_dual_stage(const fr_ctx* c, int stage, double dtau, double a0dt, void* U,
                              double* V, const double* C, double* partial, cudaStream_t s,
                              double dV, double dA) {
  return c->precision == FR_F32
             ? dual_stage_t<float>(c, stage, dtau, a0dt, U, V, C, partial, dV, dA, s)
             : dual_stage_t<double>(c, stage, dtau, a0dt, U, V, C, partial, dV, dA, s);
}

cudaError_t launch_pair_dots(const fr_ctx* c, const double* a, const double* b, double* partial,
                             double* out, cudaStream_t s) {
  const size_t n = (size_t)c->dim * c->npts * c->stride;
  const int nb = grid_blocks(c);
  pair_dots_kernel<<<nb, kThreads, 0, s>>>(n, (int)c->stride, c->ne, a, b, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  pair_dots_final_kernel<<<1, kThreads, 0, s>>>(nb, partial, out);
  return cudaGetLastError();
}

cudaError_t launch_norm_final(const fr_ctx* c, const double* partial, int nparts, double count,
                              double* out, cudaStream_t s) {
  (void)c;
  norm_final_kernel<<<1, kThreads, 0, s>>>(nparts, partial, count, out);
  return cudaGetLastError();
}

cudaError_t launch_convert(const fr_ctx* c, size_t n, int prec_in, const void* x, int prec_out,
                           void* y, cudaStream_t s) {
  const int nb = grid_blocks(c);
  if (prec_in == FR_F32 && prec_out == FR_F64)
    convert_kernel<float, double><<<nb, kThreads, 0, s>>>(n, static_cast<const float*>(x),
                                                          static_cast<double*>(y));
  else if (prec_in == FR_F64 && prec_out == FR_F32)
    convert_kernel<double, float><<<nb, kThreads, 0, s>>>(n, static_cast<const double*>(x),
                                                          static_cast<float*>(y));
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_combine3(const fr_ctx* c, int precision, size_t n, double c0, double c1,
                            double c2, const void* x0, const void* x1, const void* x2, void* out,
                            cudaStream_t s) {
  const int nb = grid_blocks(c);
  if (precision == FR_F32)
    combine3_kernel<float><<<nb, kThreads, 0, s>>>(
        n, c0, c1, c2, static_cast<const float*>(x0), static_cast<const float*>(x1),
        static_cast<const float*>(x2), static_cast<float*>(out));
  else
    combine3_kernel<double><<<nb, kThreads, 0, s>>>(
        n, c0, c1, c2, static_cast<const double*>(x0), static_cast<const double*>(x1),
        static_cast<const double*>(x2), static_cast<double*>(out));
  return cudaGetLastError();
}

}  // namespace acmhd
