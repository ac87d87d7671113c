// Fused RK4 stage kernels: the volume work of the right-hand side with one
// classical RK4 stage combination in its epilogue (StageOut), so that a
// pseudo-time step needs neither a stored R nor a trace kernel per stage.
#include "fused_tile.cuh"

namespace acmhd {

// One RK4 stage: volume work on the stage input U with the traces Tr, the
// stage combination in the epilogue (StageOut), the traces of the result to
// o.tr, and at stage 0 of a dual step the residual partial of this CTA.
template <int D, int M, typename T, int E, int NW, int MINB>
__global__ void __launch_bounds__(NW * 32, MINB)
stage_kernel(const T* __restrict__ U, const T* __restrict__ Tr, StageOut<T> o,
             double* __restrict__ partial, const FrConst<T> c) {
  constexpr int NP = ipow<M>(D);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sU = reinterpret_cast<T*>(smem_raw);
  T* sA = sU + (1 + D) * NP * E;
  __shared__ double s_red[NW];
  o.sq = 0.0;
  fused_tile<D, M, T, E, NW>(U, Tr, o, c, blockIdx.x * E, sU, sA);
  if (o.dual && o.stage == 0) {
    // fixed-order block sum: warp tree, then the warps in order
    double v = o.sq;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < NW; ++w) t += s_red[w];
      partial[blockIdx.x] = t;
    }
  }
}

template <int D, int M, typename T>
cudaError_t stage_launch(const fr_ctx* ctx, const FrConst<T>& c, const void* U, const void* Tr,
                         const StageArgs& a, double* partial, cudaStream_t s) {
  using C = FusedCfg<D, M, T>;
  auto kern = stage_kernel<D, M, T, C::E, C::NW, C::MINB>;
  static PerDeviceOnce smem_once;  // per template instance
  cudaError_t err = set_smem_limit(smem_once, kern, C::SMEM);
  if (err != cudaSuccess) return err;
  StageOut<T> o;
  o.U = static_cast<T*>(a.U);
  o.next = static_cast<T*>(a.next);
  o.acc = static_cast<T*>(a.acc);
  o.tr = static_cast<T*>(a.tr);
  o.ct = static_cast<T>(a.ct);
  o.c = a.c;
  o.a0dt = a.a0dt;
  o.stage = a.stage;
  o.dual = a.dual;
  o.vel0 = (size_t)ctx->npts * ctx->stride;
  o.vel1 = (size_t)(1 + ctx->dim) * ctx->npts * ctx->stride;
  o.V = a.V;
  o.Vs = a.Vs;
  o.Vacc = a.Vacc;
  o.C = a.C;
  o.sq = 0.0;
  const int nblk = (ctx->ne + C::E - 1) / C::E;
  kern<<<nblk, C::NW * 32, C::SMEM, s>>>(static_cast<const T*>(U), static_cast<const T*>(Tr), o,
                                          partial, c);
  return cudaGetLastError();
}

cudaError_t launch_stage(const fr_ctx* c, const void* U, const void* Tr, const StageArgs& a,
                         double* partial, cudaStream_t s) {
  if (c->precision == FR_F32) {
    ACMHD_DISPATCH_DM(c->dim, c->m,
                      return (stage_launch<D_, M_, float>(c, c->cf, U, Tr, a, partial, s)));
  } else {
    ACMHD_DISPATCH_DM(c->dim, c->m,
                      return (stage_launch<D_, M_, double>(c, c->cd, U, Tr, a, partial, s)));
  }
  return cudaErrorInvalidValue;
}

int stage_blocks(const fr_ctx* c) {
  const int e = fused_tile_elements(c->dim, c->m, c->precision);
  return e > 0 ? (c->ne + e - 1) / e : 0;
}

}  // namespace acmhd
