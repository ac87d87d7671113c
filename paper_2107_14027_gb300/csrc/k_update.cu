// Pseudo-time update kernels: the classical RK4 stage combinations
// (Sec. 5, pseudo-time stepping read as fixed-step RK4).
//
//   stage 0: acc  = k1;          Us = U + dtau/2 k1
//   stage 1: acc += 2 k2;        Us = U + dtau/2 k2
//   stage 2: acc += 2 k3;        Us = U + dtau   k3
//   stage 3: U    = U + dtau/6 (acc + k4)
//
// Element-wise over whole state buffers (padding included), 16-byte vector
// accesses, grid-stride loop sized to the SM count.
#include "fr_device.cuh"

namespace acmhd {

namespace {

template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
  static constexpr int n = 4;
};
template <>
struct Vec16<double> {
  using type = double2;
  static constexpr int n = 2;
};

template <typename T, int STAGE>
__global__ void __launch_bounds__(256)
rk_stage_kernel(size_t nvec, T dtau, T* __restrict__ U, T* __restrict__ Us, T* __restrict__ acc,
                const T* __restrict__ k) {
  using V = typename Vec16<T>::type;
  constexpr int NE = Vec16<T>::n;
  V* Uv = reinterpret_cast<V*>(U);
  V* Usv = reinterpret_cast<V*>(Us);
  V* Av = reinterpret_cast<V*>(acc);
  const V* Kv = reinterpret_cast<const V*>(k);
  const T c = (STAGE == 2) ? dtau : (STAGE == 3 ? dtau / T(6) : dtau * T(0.5));
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nvec;
       i += (size_t)gridDim.x * blockDim.x) {
    const V kv = Kv[i];
    const V uv = Uv[i];
    const T* kk = reinterpret_cast<const T*>(&kv);
    const T* uu = reinterpret_cast<const T*>(&uv);
    if (STAGE == 3) {
      const V av = Av[i];
      const T* aa = reinterpret_cast<const T*>(&av);
      V out;
      T* oo = reinterpret_cast<T*>(&out);
#pragma unroll
      for (int j = 0; j < NE; ++j) oo[j] = fma(c, aa[j] + kk[j], uu[j]);
      Uv[i] = out;
    } else {
      V an, sn;
      T* a2 = reinterpret_cast<T*>(&an);
      T* s2 = reinterpret_cast<T*>(&sn);
      if (STAGE == 0) {
        an = kv;
      } else {
        const V av = Av[i];
        const T* aa = reinterpret_cast<const T*>(&av);
#pragma unroll
        for (int j = 0; j < NE; ++j) a2[j] = fma(T(2), kk[j], aa[j]);
      }
#pragma unroll
      for (int j = 0; j < NE; ++j) s2[j] = fma(c, kk[j], uu[j]);
      Av[i] = an;
      Usv[i] = sn;
    }
  }
}

template <typename T>
cudaError_t rk_launch(const fr_ctx* ctx, int stage, double dtau, void* U, cudaStream_t s) {
  const size_t nvec = ctx->bytes_state / 16;
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device);
  const int nblk = nsm * 8;
  T* u = static_cast<T*>(U);
  T* us = static_cast<T*>(ctx->rk_stage);
  T* a = static_cast<T*>(ctx->rk_acc);
  const T* k = static_cast<const T*>(ctx->rk_k);
  const T dt = static_cast<T>(dtau);
  switch (stage) {
    case 0: rk_stage_kernel<T, 0><<<nblk, 256, 0, s>>>(nvec, dt, u, us, a, k); break;
    case 1: rk_stage_kernel<T, 1><<<nblk, 256, 0, s>>>(nvec, dt, u, us, a, k); break;
    case 2: rk_stage_kernel<T, 2><<<nblk, 256, 0, s>>>(nvec, dt, u, us, a, k); break;
    case 3: rk_stage_kernel<T, 3><<<nblk, 256, 0, s>>>(nvec, dt, u, us, a, k); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rk_stage(const fr_ctx* c, int stage, double dtau, void* U, cudaStream_t s) {
  return c->precision == FR_F32 ? rk_launch<float>(c, stage, dtau, U, s)
                                : rk_launch<double>(c, stage, dtau, U, s);
}

}  // namespace acmhd
