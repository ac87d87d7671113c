// P-multigrid kernels (Sec. 5: P-multigrid pseudo-time acceleration of the
// dual time step), all element-local and streaming:
//
//   transfer   between adjacent orders on the same mesh, per element and
//              variable, by a 1-D matrix applied along every direction
//              (sum factorisation): restriction U_c = I_r U_f (L2
//              projection), prolongation of a coarse correction
//              U_f += I_p (U_c - U0_c), with the FP64 velocity master of the
//              finest level updated in FP64;
//   residual   r = N(U) + g of a level for the restriction, N = R - I_V a0/dt V:
//              finest level r = k + [velocity: C - a0/dt V64] (FP64, also
//              summed in squares for the convergence test), coarse levels
//              r = k + g - [velocity: a0/dt U];
//   forcing    g_c = I_r r_f - N_c(U0_c) = restricted residual - k_c
//              + [velocity: a0/dt U0_c];
//   smoother   one RK4 stage of a coarse level on dU/dtau = D (N(U) + g),
//              D = 1 / (1 + dtau a0/dt) on the velocity rows and
//              1 / (1 + dtau / T) on the gradient rows (point-implicit
//              scaling of the linear stiff terms; D = 1 disables it).
//
// Thread mapping: one thread per (variable, element column) for the
// transfers (every load and store is a contiguous row segment across the
// threads of a warp); grid-stride over entries for the streaming kernels.
#include "fr_device.cuh"
#include "fr_pmg.h"

namespace acmhd {

namespace {

constexpr int kThreads = 256;

// out[o0,o1,o2] = sum A[o_a][i_a] in[...] along axis A of a row-major
// (axis 0 fastest) array; sizes of the three axes before (S0, S1, S2).
template <int AX, int R, int S0, int S1, int S2, typename T>
__device__ __forceinline__ void contract(const T* __restrict__ in, T* __restrict__ out,
                                         const T (&A)[kMaxM][kMaxM]) {
  constexpr int O0 = AX == 0 ? R : S0, O1 = AX == 1 ? R : S1, O2 = AX == 2 ? R : S2;
#pragma unroll
  for (int c = 0; c < O2; ++c)
#pragma unroll
    for (int b = 0; b < O1; ++b)
#pragma unroll
      for (int a = 0; a < O0; ++a) {
        T acc = T(0);
        constexpr int M = AX == 0 ? S0 : (AX == 1 ? S1 : S2);
#pragma unroll
        for (int t = 0; t < M; ++t) {
          const int i0 = AX == 0 ? t : a, i1 = AX == 1 ? t : b, i2 = AX == 2 ? t : c;
          const int o = AX == 0 ? a : (AX == 1 ? b : c);
          acc = fma(A[o][t], in[(i2 * S1 + i1) * S0 + i0], acc);
        }
        out[(c * O1 + b) * O0 + a] = acc;
      }
}

// y (MO^D values) = A applied along every direction of x (MI^D values).
template <int D, int MI, int MO, typename T>
__device__ __forceinline__ void tensor_apply(const T* x, T* y, const T (&A)[kMaxM][kMaxM]) {
  if constexpr (D == 2) {
    T t1[MI * MO];
    contract<0, MO, MI, MI, 1>(x, t1, A);
    contract<1, MO, MO, MI, 1>(t1, y, A);
  } else {
    T t1[MI * MI * MO], t2[MI * MO * MO];
    contract<0, MO, MI, MI, MI>(x, t1, A);
    contract<1, MO, MO, MI, MI>(t1, t2, A);
    contract<2, MO, MO, MO, MI>(t2, y, A);
  }
}

// Restriction: Yc[v][pt_c][e] = (I_r along every direction) Xf[v][.][e].
template <int D, int MF, typename T>
__global__ void __launch_bounds__(kThreads)
restrict_kernel(int nv, int stride, const T* __restrict__ Xf, T* __restrict__ Yc,
                const PmgTransfer<T> tr) {
  constexpr int MC = MF - 1, NF = ipow<MF>(D), NC = ipow<MC>(D);
  const long long tid = blockIdx.x * (long long)kThreads + threadIdx.x;
  if (tid >= (long long)nv * stride) return;
  const int v = (int)(tid / stride), e = (int)(tid - (long long)v * stride);
  T x[NF], y[NC];
#pragma unroll
  for (int q = 0; q < NF; ++q) x[q] = __ldg(Xf + ((size_t)v * NF + q) * stride + e);
  tensor_apply<D, MF, MC>(x, y, tr.Ir);
#pragma unroll
  for (int q = 0; q < NC; ++q) Yc[((size_t)v * NC + q) * stride + e] = y[q];
}

// Prolongation of a correction: Xf += I_p (Yc - Y0c); the velocity rows of
// the finest level go to the FP64 master V (and its rounded copy in Xf).
template <int D, int MF, typename T>
__global__ void __launch_bounds__(kThreads)
prolong_kernel(int nv, int stride, const T* __restrict__ Yc, const T* __restrict__ Y0c,
               T* __restrict__ Xf, double* __restrict__ V, const PmgTransfer<T> tr) {
  constexpr int MC = MF - 1, NF = ipow<MF>(D), NC = ipow<MC>(D);
  const long long tid = blockIdx.x * (long long)kThreads + threadIdx.x;
  if (tid >= (long long)nv * stride) return;
  const int v = (int)(tid / stride), e = (int)(tid - (long long)v * stride);
  T x[NC], y[NF];
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    const size_t i = ((size_t)v * NC + q) * stride + e;
    x[q] = __ldg(Yc + i) - __ldg(Y0c + i);
  }
  tensor_apply<D, MC, MF>(x, y, tr.Ip);
  const bool vel = V != nullptr && v >= 1 && v <= D;
#pragma unroll
  for (int q = 0; q < NF; ++q) {
    const size_t i = ((size_t)v * NF + q) * stride + e;
    if (vel) {
      const size_t j = ((size_t)(v - 1) * NF + q) * stride + e;
      const double vn = V[j] + static_cast<double>(y[q]);
      V[j] = vn;
      Xf[i] = static_cast<T>(vn);
    } else {
      Xf[i] = Xf[i] + y[q];
    }
  }
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  return red[0];
}

// r = N(U) + g.  Finest level (V != null): velocity rows in FP64 from the
// master V and the BDF constant C, squares of real elements summed into
// partial[block]; coarse levels: r = k + g - a0dt U on the velocity rows.
template <typename T>
__global__ void __launch_bounds__(kThreads)
residual_kernel(size_t n, size_t vel0, size_t nvel, int stride, int ne, double a0dt,
                const T* __restrict__ k, const T* __restrict__ U, const T* __restrict__ g,
                const double* __restrict__ V, const double* __restrict__ C, T* __restrict__ r,
                double* __restrict__ partial) {
  __shared__ double red[kThreads];
  double sq = 0.0;
  for (size_t i = blockIdx.x * (size_t)kThreads + threadIdx.x; i < n;
       i += (size_t)gridDim.x * kThreads) {
    const bool vel = i >= vel0 && i < vel0 + nvel;
    if (V != nullptr) {
      if (vel) {
        const size_t j = i - vel0;
        const double kv = static_cast<double>(k[i]) + fma(-a0dt, V[j], C[j]);
        if ((int)(j % (size_t)stride) < ne) sq = fma(kv, kv, sq);
        r[i] = static_cast<T>(kv);
      } else {
        r[i] = k[i];
      }
    } else {
      T x = k[i] + g[i];
      if (vel) x = fma(static_cast<T>(-a0dt), U[i], x);
      r[i] = x;
    }
  }
  if (partial != nullptr) {
    const double b = block_sum(sq, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = b;
  }
}

// g = Rr - k + [velocity rows] a0dt U0  (Rr: restricted residual, k = R(U0))
template <typename T>
__global__ void __launch_bounds__(kThreads)
forcing_kernel(size_t n, size_t vel0, size_t nvel, double a0dt, const T* __restrict__ Rr,
               const T* __restrict__ k, const T* __restrict__ U0, T* __restrict__ g) {
  for (size_t i = blockIdx.x * (size_t)kThreads + threadIdx.x; i < n;
       i += (size_t)gridDim.x * kThreads) {
    T x = Rr[i] - k[i];
    if (i >= vel0 && i < vel0 + nvel) x = fma(static_cast<T>(a0dt), U0[i], x);
    g[i] = x;
  }
}

// One RK4 stage of a coarse level: kt = D (k + g - [velocity] a0dt Uin),
// Uin = U (stage 0) or Us; then the classical combination of k_update.cu.
template <typename T, int STAGE>
__global__ void __launch_bounds__(kThreads)
coarse_stage_kernel(size_t n, size_t vel0, size_t nvel, T dtau, T a0dt, T dV, T dA,
                    T* __restrict__ U, T* __restrict__ Us, T* __restrict__ acc,
                    const T* __restrict__ k, const T* __restrict__ g) {
  const T c = (STAGE == 2) ? dtau : (STAGE == 3 ? dtau / T(6) : dtau * T(0.5));
  for (size_t i = blockIdx.x * (size_t)kThreads + threadIdx.x; i < n;
       i += (size_t)gridDim.x * kThreads) {
    const bool vel = i >= vel0 && i < vel0 + nvel;
    const T uin = (STAGE == 0) ? U[i] : Us[i];
    T kt = k[i] + g[i];
    if (vel) kt = dV * fma(-a0dt, uin, kt);
    else if (i >= vel0 + nvel) kt = dA * kt;
    if (STAGE == 3) {
      U[i] = fma(c, acc[i] + kt, U[i]);
    } else {
      acc[i] = (STAGE == 0) ? kt : fma(T(2), kt, acc[i]);
      Us[i] = fma(c, kt, U[i]);
    }
  }
}

int stream_blocks(const fr_ctx* c) {
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
  return nsm * 8;
}

template <typename T>
cudaError_t transfer_t(const fr_ctx* fine, bool prolong, const void* a, const void* b, void* out,
                       double* V, const PmgTransfer<T>& tr, cudaStream_t s) {
  const long long work = (long long)fine->nv * (long long)fine->stride;
  const int nb = (int)((work + kThreads - 1) / kThreads);
  const int st = (int)fine->stride;
  switch (fine->dim * 10 + fine->m) {
#define ACMHD_PMG_CASE(DD, MM)                                                                  \
  case DD * 10 + MM:                                                                            \
    if (prolong)                                                                                \
      prolong_kernel<DD, MM, T><<<nb, kThreads, 0, s>>>(fine->nv, st, static_cast<const T*>(a), \
                                                        static_cast<const T*>(b),               \
                                                        static_cast<T*>(out), V, tr);           \
    else                                                                                        \
      restrict_kernel<DD, MM, T><<<nb, kThreads, 0, s>>>(fine->nv, st,                          \
                                                         static_cast<const T*>(a),              \
                                                         static_cast<T*>(out), tr);             \
    break;
    ACMHD_PMG_CASE(2, 3) ACMHD_PMG_CASE(2, 4) ACMHD_PMG_CASE(2, 5) ACMHD_PMG_CASE(2, 6)
    ACMHD_PMG_CASE(2, 7) ACMHD_PMG_CASE(3, 3) ACMHD_PMG_CASE(3, 4) ACMHD_PMG_CASE(3, 5)
    ACMHD_PMG_CASE(3, 6) ACMHD_PMG_CASE(3, 7)
#undef ACMHD_PMG_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pmg_restrict(const fr_ctx* fine, const void* Xf, void* Yc,
                                const PmgTransferPair& tr, cudaStream_t s) {
  return fine->precision == FR_F32
             ? transfer_t<float>(fine, false, Xf, nullptr, Yc, nullptr, tr.f, s)
             : transfer_t<double>(fine, false, Xf, nullptr, Yc, nullptr, tr.d, s);
}

cudaError_t launch_pmg_prolong(const fr_ctx* fine, const void* Yc, const void* Y0c, void* Xf,
                               double* V, const PmgTransferPair& tr, cudaStream_t s) {
  return fine->precision == FR_F32 ? transfer_t<float>(fine, true, Yc, Y0c, Xf, V, tr.f, s)
                                   : transfer_t<double>(fine, true, Yc, Y0c, Xf, V, tr.d, s);
}

cudaError_t launch_pmg_residual(const fr_ctx* c, const void* k, const void* U, const void* g,
                                const double* V, const double* C, double a0dt, void* r,
                                double* partial, cudaStream_t s) {
  const size_t n = (size_t)c->nv * c->npts * c->stride;
  const size_t vel0 = (size_t)c->npts * c->stride, nvel = (size_t)c->dim * vel0;
  const int nb = stream_blocks(c);
  const int st = (int)c->stride;
  if (c->precision == FR_F32)
    residual_kernel<float><<<nb, kThreads, 0, s>>>(
        n, vel0, nvel, st, c->ne, a0dt, static_cast<const float*>(k), static_cast<const float*>(U),
        static_cast<const float*>(g), V, C, static_cast<float*>(r), partial);
  else
    residual_kernel<double><<<nb, kThreads, 0, s>>>(
        n, vel0, nvel, st, c->ne, a0dt, static_cast<const double*>(k),
        static_cast<const double*>(U), static_cast<const double*>(g), V, C,
        static_cast<double*>(r), partial);
  return cudaGetLastError();
}

int pmg_norm_blocks(const fr_ctx* c) { return stream_blocks(c); }

cudaError_t launch_pmg_forcing(const fr_ctx* c, const void* Rr, const void* k, const void* U0,
                               double a0dt, void* g, cudaStream_t s) {
  const size_t n = (size_t)c->nv * c->npts * c->stride;
  const size_t vel0 = (size_t)c->npts * c->stride, nvel = (size_t)c->dim * vel0;
  const int nb = stream_blocks(c);
  if (c->precision == FR_F32)
    forcing_kernel<float><<<nb, kThreads, 0, s>>>(n, vel0, nvel, a0dt, static_cast<const float*>(Rr),
                                                  static_cast<const float*>(k),
                                                  static_cast<const float*>(U0),
                                                  static_cast<float*>(g));
  else
    forcing_kernel<double><<<nb, kThreads, 0, s>>>(
        n, vel0, nvel, a0dt, static_cast<const double*>(Rr), static_cast<const double*>(k),
        static_cast<const double*>(U0), static_cast<double*>(g));
  return cudaGetLastError();
}

template <typename T>
static cudaError_t coarse_stage_t(const fr_ctx* c, int stage, double dtau, double a0dt, double dV,
                                  double dA, void* U, const void* g, cudaStream_t s) {
  const size_t n = (size_t)c->nv * c->npts * c->stride;
  const size_t vel0 = (size_t)c->npts * c->stride, nvel = (size_t)c->dim * vel0;
  const int nb = stream_blocks(c);
  T* u = static_cast<T*>(U);
  T* us = static_cast<T*>(c->rk_stage);
  T* a = static_cast<T*>(c->rk_acc);
  const T* k = static_cast<const T*>(c->rk_k);
  const T* gg = static_cast<const T*>(g);
  const T dt = (T)dtau, ad = (T)a0dt, v = (T)dV, x = (T)dA;
  switch (stage) {
    case 0: coarse_stage_kernel<T, 0><<<nb, kThreads, 0, s>>>(n, vel0, nvel, dt, ad, v, x, u, us, a, k, gg); break;
    case 1: coarse_stage_kernel<T, 1><<<nb, kThreads, 0, s>>>(n, vel0, nvel, dt, ad, v, x, u, us, a, k, gg); break;
    case 2: coarse_stage_kernel<T, 2><<<nb, kThreads, 0, s>>>(n, vel0, nvel, dt, ad, v, x, u, us, a, k, gg); break;
    case 3: coarse_stage_kernel<T, 3><<<nb, kThreads, 0, s>>>(n, vel0, nvel, dt, ad, v, x, u, us, a, k, gg); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_pmg_coarse_stage(const fr_ctx* c, int stage, double dtau, double a0dt,
                                    double dV, double dA, void* U, const void* g,
                                    cudaStream_t s) {
  return c->precision == FR_F32 ? coarse_stage_t<float>(c, stage, dtau, a0dt, dV, dA, U, g, s)
                                : coarse_stage_t<double>(c, stage, dtau, a0dt, dV, dA, U, g, s);
}

}  // namespace acmhd

// ---------------------------------------------------------------------------
// Anderson mixing (finest level): record, inner products, combination.
// Element e of row r is a real entry when e < ne; the velocity rows of the
// state are represented by the FP64 master V, so the state's own velocity
// rows are skipped in the inner products and rewritten from V.
// ---------------------------------------------------------------------------

namespace acmhd {
namespace {

template <typename T>
__global__ void __launch_bounds__(kThreads)
aa_record_kernel(size_t n, size_t nvel, const T* __restrict__ U, const double* __restrict__ V,
                 const T* __restrict__ Xu, const double* __restrict__ Xv, T* __restrict__ Gu,
                 double* __restrict__ Gv, T* __restrict__ Fu, double* __restrict__ Fv) {
  for (size_t i = blockIdx.x * (size_t)kThreads + threadIdx.x; i < n;
       i += (size_t)gridDim.x * kThreads) {
    const T u = U[i];
    Gu[i] = u;
    Fu[i] = u - Xu[i];
    if (i < nvel) {
      const double v = V[i];
      Gv[i] = v;
      Fv[i] = v - Xv[i];
    }
  }
}

// partial[j * gridDim.x + block] = block's share of <F, W_j>
template <typename T>
__global__ void __launch_bounds__(kThreads)
aa_dots_kernel(size_t n, size_t vel0, size_t nvel, int stride, int ne, const T* __restrict__ Fu,
               const double* __restrict__ Fv, const AaVectors W, double* __restrict__ partial) {
  __shared__ double red[kThreads];
  double acc[kAaMax];
#pragma unroll
  for (int j = 0; j < kAaMax; ++j) acc[j] = 0.0;
  for (size_t i = blockIdx.x * (size_t)kThreads + threadIdx.x; i < n;
       i += (size_t)gridDim.x * kThreads) {
    if ((int)(i % (size_t)stride) >= ne) continue;
    const bool vel = i >= vel0 && i < vel0 + nvel;
    if (!vel) {
      const double f = static_cast<double>(Fu[i]);
#pragma unroll
      for (int j = 0; j < kAaMax; ++j)
        if (j < W.n) acc[j] = fma(f, static_cast<double>(static_cast<const T*>(W.u[j])[i]), acc[j]);
    }
    if (i < nvel) {
      const double f = Fv[i];
#pragma unroll
      for (int j = 0; j < kAaMax; ++j)
        if (j < W.n) acc[j] = fma(f, W.v[j][i], acc[j]);
    }
  }
  for (int j = 0; j < W.n; ++j) {
    const double b = block_sum(acc[j], red);
    if (threadIdx.x == 0) partial[(size_t)j * gridDim.x + blockIdx.x] = b;
    __syncthreads();
  }
}

// dots[j] = sum over blocks of partial[j][.], in order (one block per j)
__global__ void __launch_bounds__(kThreads)
aa_dots_final_kernel(int nparts, const double* __restrict__ partial, double* __restrict__ dots) {
  __shared__ double red[kThreads];
  double s = 0.0;
  for (int i = threadIdx.x; i < nparts; i += kThreads) s += partial[(size_t)blockIdx.x * nparts + i];
  const double b = block_sum(s, red);
  if (threadIdx.x == 0) dots[blockIdx.x] = b;
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
aa_combine_kernel(size_t n, size_t vel0, size_t nvel, const AaVectors W, T* __restrict__ U,
                  double* __restrict__ V) {
  for (size_t i = blockIdx.x * (size_t)kThreads + threadIdx.x; i < n;
       i += (size_t)gridDim.x * kThreads) {
    const bool vel = i >= vel0 && i < vel0 + nvel;
    if (!vel) {
      double x = 0.0;
      for (int j = 0; j < W.n; ++j)
        x = fma(W.c[j], static_cast<double>(static_cast<const T*>(W.u[j])[i]), x);
      U[i] = static_cast<T>(x);
    }
    if (i < nvel) {
      double x = 0.0;
      for (int j = 0; j < W.n; ++j) x = fma(W.c[j], W.v[j][i], x);
      V[i] = x;
      U[vel0 + i] = static_cast<T>(x);
    }
  }
}

}  // namespace

int aa_dot_blocks(const fr_ctx* c) { return stream_blocks(c); }

cudaError_t launch_aa_record(const fr_ctx* c, const void* U, const double* V, const void* Xu,
                             const double* Xv, void* Gu, double* Gv, void* Fu, double* Fv,
                             cudaStream_t s) {
  const size_t n = (size_t)c->nv * c->npts * c->stride;
  const size_t nvel = (size_t)c->dim * c->npts * c->stride;
  const int nb = stream_blocks(c);
  if (c->precision == FR_F32)
    aa_record_kernel<float><<<nb, kThreads, 0, s>>>(n, nvel, static_cast<const float*>(U), V,
                                                    static_cast<const float*>(Xu), Xv,
                                                    static_cast<float*>(Gu), Gv,
                                                    static_cast<float*>(Fu), Fv);
  else
    aa_record_kernel<double><<<nb, kThreads, 0, s>>>(n, nvel, static_cast<const double*>(U), V,
                                                     static_cast<const double*>(Xu), Xv,
                                                     static_cast<double*>(Gu), Gv,
                                                     static_cast<double*>(Fu), Fv);
  return cudaGetLastError();
}

cudaError_t launch_aa_dots(const fr_ctx* c, const void* Fu, const double* Fv, const AaVectors& W,
                           double* partial, int nparts, double* dots, cudaStream_t s) {
  if (W.n < 1 || W.n > kAaMax) return cudaErrorInvalidValue;
  const size_t n = (size_t)c->nv * c->npts * c->stride;
  const size_t vel0 = (size_t)c->npts * c->stride, nvel = (size_t)c->dim * vel0;
  const int st = (int)c->stride;
  if (c->precision == FR_F32)
    aa_dots_kernel<float><<<nparts, kThreads, 0, s>>>(n, vel0, nvel, st, c->ne,
                                                      static_cast<const float*>(Fu), Fv, W, partial);
  else
    aa_dots_kernel<double><<<nparts, kThreads, 0, s>>>(n, vel0, nvel, st, c->ne,
                                                       static_cast<const double*>(Fu), Fv, W,
                                                       partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  aa_dots_final_kernel<<<W.n, kThreads, 0, s>>>(nparts, partial, dots);
  return cudaGetLastError();
}

cudaError_t launch_aa_combine(const fr_ctx* c, const AaVectors& W, void* U, double* V,
                              cudaStream_t s) {
  if (W.n < 1 || W.n > kAaMax) return cudaErrorInvalidValue;
  const size_t n = (size_t)c->nv * c->npts * c->stride;
  const size_t vel0 = (size_t)c->npts * c->stride, nvel = (size_t)c->dim * vel0;
  const int nb = stream_blocks(c);
  if (c->precision == FR_F32)
    aa_combine_kernel<float><<<nb, kThreads, 0, s>>>(n, vel0, nvel, W, static_cast<float*>(U), V);
  else
    aa_combine_kernel<double><<<nb, kThreads, 0, s>>>(n, vel0, nvel, W, static_cast<double*>(U),
                                                      V);
  return cudaGetLastError();
}

}  // namespace acmhd
