// Unfused baseline: the six stages of Table fr_adv as six kernels with
// global-memory intermediates, laid out as in the table:
//   1 (M) U_s[n_e n_v n_s]          -> U_f[n_e n_v n_f]      (all variables)
//   2 (P) U_s                       -> F_s[d n_e n_v n_s]    (dense flux)
//   3 (M) F_s                       -> div^a F_s             (partially corrected)
//   4 (I) U_f                       -> F^I_f[n_e n_v n_f]
//   5 (M) F^I_f, div^a F_s          -> div^c F_s             (in place)
//   6 (P) div^c F_s, U_s            -> -div F_s + s_s
// Mapping: block (32, 8); lane -> element (contiguous rows), threadIdx.y and
// blockIdx.y enumerate the per-element tasks of the stage.
#include "fr_device.cuh"

namespace acmhd {

namespace {

constexpr int kWarps = 8;

template <int D, typename T>
__device__ __forceinline__ void full_flux(const T (&u)[1 + D + D * D], int a, T zeta, T nu,
                                          T inv_t, T (&f)[1 + D + D * D]) {
#pragma unroll
  for (int v = 0; v < 1 + D + D * D; ++v) f[v] = T(0);
  const T va = u[1 + a];
  f[0] = rn_mul(zeta, va);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    T t = rn_mul(nu, u[aux_var<D>(i, a)]);
    t = (i == a) ? rn_sub(u[0], t) : -t;
    f[1 + i] = rn_fma(u[1 + i], va, t);
    f[aux_var<D>(i, a)] = -rn_mul(u[1 + i], inv_t);
  }
}

template <int D, typename T>
__device__ __forceinline__ void full_common_flux(const T (&uL)[1 + D + D * D],
                                                 const T (&uR)[1 + D + D * D], int a, T zeta,
                                                 T nu, T inv_t, T (&fi)[1 + D + D * D]) {
  constexpr int NV = 1 + D + D * D;
  T fL[NV], fR[NV];
  full_flux<D>(uL, a, zeta, nu, inv_t, fL);
  full_flux<D>(uR, a, zeta, nu, inv_t, fR);
  const T vl = uL[1 + a], vr = uR[1 + a];
  const T sl = rn_add(vabs(vl), rn_sqrt(rn_fma(vl, vl, zeta)));
  const T sr = rn_add(vabs(vr), rn_sqrt(rn_fma(vr, vr, zeta)));
  const T hs = rn_mul(T(0.5), vmax(sl, sr));
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const T mean = rn_mul(T(0.5), rn_add(fL[v], fR[v]));
    fi[v] = (v <= D) ? rn_fma(-hs, rn_sub(uR[v], uL[v]), mean) : mean;
  }
}

// coordinate of point pt along axis a, and its line index for axis a
template <int M>
__device__ __forceinline__ void pt_line(int pt, int a, int& t, int& l) {
  const int ma = (a == 0) ? 1 : (a == 1 ? M : M * M);
  t = (pt / ma) % M;
  l = (pt % ma) + ma * (pt / (ma * M));
}

template <int D, int M, typename T>
__global__ void __launch_bounds__(256)
s1_project(const T* __restrict__ U, T* __restrict__ Uf, const FrConst<T> c) {
  constexpr int NP = ipow<M>(D), NL = ipow<M>(D - 1), NV = 1 + D + D * D;
  const int e = blockIdx.x * 32 + threadIdx.x;
  const int task = blockIdx.y * kWarps + threadIdx.y;
  if (e >= c.ne || task >= D * NL * NV) return;
  const size_t S = c.stride;
  const int a = task / (NL * NV), rem = task % (NL * NV), l = rem / NV, v = rem % NV;
  T x[M];
#pragma unroll
  for (int t = 0; t < M; ++t) x[t] = U[((size_t)v * NP + line_pt<D, M>(a, l, t)) * S + e];
  Uf[(((size_t)(2 * a) * NV + v) * NL + l) * S + e] = trace_dot<M>(x, c.lm);
  Uf[(((size_t)(2 * a + 1) * NV + v) * NL + l) * S + e] = trace_dot<M>(x, c.lp);
}

template <int D, int M, typename T>
__global__ void __launch_bounds__(256)
s2_flux(const T* __restrict__ U, T* __restrict__ F, const FrConst<T> c) {
  constexpr int NP = ipow<M>(D), NV = 1 + D + D * D;
  const int e = blockIdx.x * 32 + threadIdx.x;
  const int pt = blockIdx.y * kWarps + threadIdx.y;
  if (e >= c.ne || pt >= NP) return;
  const size_t S = c.stride;
  T u[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) u[v] = U[((size_t)v * NP + pt) * S + e];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    T f[NV];
    full_flux<D>(u, a, c.zeta, c.nu, c.inv_t, f);
#pragma unroll
    for (int v = 0; v < NV; ++v) F[(((size_t)a * NV + v) * NP + pt) * S + e] = f[v];
  }
}

template <int D, int M, typename T>
__global__ void __launch_bounds__(256)
s3_divergence(const T* __restrict__ F, T* __restrict__ div, const FrConst<T> c) {
  constexpr int NP = ipow<M>(D), NV = 1 + D + D * D;
  const int e = blockIdx.x * 32 + threadIdx.x;
  const int task = blockIdx.y * kWarps + threadIdx.y;
  if (e >= c.ne || task >= NV * NP) return;
  const size_t S = c.stride;
  const int v = task / NP, pt = task % NP;
  T acc = T(0);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    int t, l;
    pt_line<M>(pt, a, t, l);
    T da = T(0);
#pragma unroll
    for (int k = 0; k < M; ++k)
      da = fma(c.Dt[t][k], F[(((size_t)a * NV + v) * NP + line_pt<D, M>(a, l, k)) * S + e], da);
    acc = fma(c.J[a], da, acc);
  }
  div[((size_t)v * NP + pt) * S + e] = acc;
}

template <int D, int M, typename T>
__global__ void __launch_bounds__(256)
s4_common_flux(const T* __restrict__ Uf, T* __restrict__ FI, const FrConst<T> c) {
  constexpr int NL = ipow<M>(D - 1), NV = 1 + D + D * D;
  const int e = blockIdx.x * 32 + threadIdx.x;
  const int task = blockIdx.y * kWarps + threadIdx.y;
  if (e >= c.ne || task >= 2 * D * NL) return;
  const size_t S = c.stride;
  const int f = task / NL, l = task % NL, a = f / 2, side = f % 2;
  int nb[3][2];
  neighbours<D>(e, c.n, nb);
  const int eL = side ? e : nb[a][0];
  const int eR = side ? nb[a][1] : e;
  T uL[NV], uR[NV], fi[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    uL[v] = Uf[(((size_t)(2 * a + 1) * NV + v) * NL + l) * S + eL];
    uR[v] = Uf[(((size_t)(2 * a) * NV + v) * NL + l) * S + eR];
  }
  full_common_flux<D>(uL, uR, a, c.zeta, c.nu, c.inv_t, fi);
#pragma unroll
  for (int v = 0; v < NV; ++v) FI[(((size_t)f * NV + v) * NL + l) * S + e] = fi[v];
}

template <int D, int M, typename T>
__global__ void __launch_bounds__(256)
s5_correction(const T* __restrict__ FI, T* __restrict__ div, const FrConst<T> c) {
  constexpr int NP = ipow<M>(D), NL = ipow<M>(D - 1), NV = 1 + D + D * D;
  const int e = blockIdx.x * 32 + threadIdx.x;
  const int task = blockIdx.y * kWarps + threadIdx.y;
  if (e >= c.ne || task >= NV * NP) return;
  const size_t S = c.stride;
  const int v = task / NP, pt = task % NP;
  T acc = div[((size_t)v * NP + pt) * S + e];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    int t, l;
    pt_line<M>(pt, a, t, l);
    const T fl = FI[(((size_t)(2 * a) * NV + v) * NL + l) * S + e];
    const T fr = FI[(((size_t)(2 * a + 1) * NV + v) * NL + l) * S + e];
    acc = fma(c.J[a], fma(c.dhl[t], fl, c.dhr[t] * fr), acc);
  }
  div[((size_t)v * NP + pt) * S + e] = acc;
}

template <int D, int M, typename T>
__global__ void __launch_bounds__(256)
s6_negate_source(const T* __restrict__ div, const T* __restrict__ U, T* __restrict__ R,
                 const FrConst<T> c) {
  constexpr int NP = ipow<M>(D), NV = 1 + D + D * D;
  const int e = blockIdx.x * 32 + threadIdx.x;
  const int task = blockIdx.y * kWarps + threadIdx.y;
  if (e >= c.ne || task >= NV * NP) return;
  const size_t S = c.stride;
  const int v = task / NP;
  const size_t o = (size_t)task * S + e;
  R[o] = (v > D) ? fma(-U[o], c.inv_t, -div[o]) : -div[o];
}

inline dim3 grid_for(int ne, int ntask) { return dim3((ne + 31) / 32, (ntask + kWarps - 1) / kWarps); }

template <int D, int M, typename T>
cudaError_t unfused_launch(const fr_ctx* ctx, const FrConst<T>& c, const void* U_, void* R_,
                           cudaStream_t s) {
  constexpr int NP = ipow<M>(D), NL = ipow<M>(D - 1), NV = 1 + D + D * D;
  const T* U = static_cast<const T*>(U_);
  T* R = static_cast<T*>(R_);
  T* Uf = static_cast<T*>(ctx->unf_uf);
  T* F = static_cast<T*>(ctx->unf_f);
  T* dv = static_cast<T*>(ctx->unf_div);
  T* FI = static_cast<T*>(ctx->unf_fi);
  const dim3 blk(32, kWarps);
  const int ne = ctx->ne;
  s1_project<D, M, T><<<grid_for(ne, D * NL * NV), blk, 0, s>>>(U, Uf, c);
  s2_flux<D, M, T><<<grid_for(ne, NP), blk, 0, s>>>(U, F, c);
  s3_divergence<D, M, T><<<grid_for(ne, NV * NP), blk, 0, s>>>(F, dv, c);
  s4_common_flux<D, M, T><<<grid_for(ne, 2 * D * NL), blk, 0, s>>>(Uf, FI, c);
  s5_correction<D, M, T><<<grid_for(ne, NV * NP), blk, 0, s>>>(FI, dv, c);
  s6_negate_source<D, M, T><<<grid_for(ne, NV * NP), blk, 0, s>>>(dv, U, R, c);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_unfused(const fr_ctx* c, const void* U, void* R, cudaStream_t s) {
  if (c->precision == FR_F32) {
    ACMHD_DISPATCH_DM(c->dim, c->m, return (unfused_launch<D_, M_, float>(c, c->cf, U, R, s)));
  } else {
    ACMHD_DISPATCH_DM(c->dim, c->m, return (unfused_launch<D_, M_, double>(c, c->cd, U, R, s)));
  }
  return cudaErrorInvalidValue;
}

}  // namespace acmhd
