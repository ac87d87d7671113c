// Fused right-hand-side kernels: stages 2-6 of Table fr_adv in one pass, and
// the layer sweep that also runs stage 1 in the same persistent kernel.  The
// tile work (fused_tile) and the RHS kernel template are in fused_tile.cuh;
// this file holds the whole-mesh launcher and the sweep.
//
// For every element and every axis a the volume work evaluates the normal
// flux F_a at the solution points (stage 2), the partially corrected
// divergence along the axis lines (stage 3), the common interface flux at
// both faces of each line (stage 4, from this element's own face trace and
// the neighbour's stored trace), the correction (stage 5), and the negation
// plus source (stage 6):
//
//   R = sum_a  -J_a [ Dt F_a + h_l' F^I_l + h_r' F^I_r ]  -  (1/T) [0; 0; q; r; s]
//
// with Dt = D - h_l' l(-1)^T - h_r' l(+1)^T and J_a = 2 / h_a (Sec. 2.1, FR
// divergence equation).
//
// Work decomposition (GB300): a tile is E consecutive elements, lane ->
// element, so every global row access is contiguous.  P and V of the tile
// are staged once in shared memory, because every axis needs them; each
// auxiliary variable is needed by exactly one axis and is read straight
// from global memory by the thread that owns the line.  The axes run as
// phases; in each phase a thread owns whole lines along the axis, so the
// 1-D contractions are register FMAs against operator constants that come
// from the kernel-parameter (constant) bank.  Only the P and V equations
// receive contributions from more than one axis; their partial sums live in
// shared memory between phases.  The auxiliary equations are finished and
// written in the phase of their axis.
//
// Layer sweep.  Two kernels (trace, then volume) read U twice from HBM and
// write and re-read the face traces.  The sweep kernel is persistent: its
// CTAs claim work units in a fixed queue that interleaves the trace unit of
// tile t + K with the volume unit of tile t (K tiles = one element layer),
// so that the tile's U and its neighbours' traces are still in L2 when the
// volume unit needs them.  A volume unit waits (bounded) on per-tile flags
// of the trace units it depends on; those units precede it in the queue and
// never wait, so the schedule cannot deadlock.
#include "fused_tile.cuh"

namespace acmhd {

namespace {

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// traces are read through L2 only when other CTAs of the same kernel write them
}  // namespace

// Stage 1 for one tile of E elements, with the lane layout of the volume
// work (lane -> element, 32/E lines per warp, NW warps).
template <int D, int M, typename T, int E, int NW>
__device__ __forceinline__ void trace_tile(const T* __restrict__ U, T* __restrict__ Tr,
                                           const FrConst<T>& c, int e0) {
  constexpr int NP = ipow<M>(D), NL = ipow<M>(D - 1), NS = 1 + 2 * D, SUB = 32 / E;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int e = e0 + lane % E, sub = lane / E;
  if (e >= c.ne) return;
  const size_t S = c.stride;
  int nb[3][2];
  neighbours<D>(e, c.n, nb);
  const bool need_x_lo = !x_pair_on_chip(nb[0][0], e, E);
  const bool need_x_hi = !x_pair_on_chip(e, nb[0][1], E);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const bool need_lo = (a == 0) ? need_x_lo : true;
    const bool need_hi = (a == 0) ? need_x_hi : true;
    if (!need_lo && !need_hi) continue;
    for (int l = warp * SUB + sub; l < NL; l += NW * SUB) {
      T x[NS][M];
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        const int v = slot_var<D>(s, a);
#pragma unroll
        for (int t = 0; t < M; ++t)
          x[s][t] = __ldg(U + ((size_t)v * NP + line_pt<D, M>(a, l, t)) * S + e);
      }
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        if (need_lo) Tr[(((size_t)(2 * a) * NS + s) * NL + l) * S + e] = trace_dot<M>(x[s], c.lm);
        if (need_hi)
          Tr[(((size_t)(2 * a + 1) * NS + s) * NL + l) * S + e] = trace_dot<M>(x[s], c.lp);
      }
    }
  }
}

template <int D, int M, typename T, int E, int NW, int MINB>
__global__ void __launch_bounds__(NW * 32, MINB)
sweep_kernel(const T* __restrict__ U, T* __restrict__ Tr, T* __restrict__ R, const FrConst<T> c,
             const int* __restrict__ units, int nunits, unsigned* __restrict__ flags,
             unsigned epoch, int ntiles, int K, unsigned* __restrict__ queue, int* __restrict__ err) {
  constexpr int NP = ipow<M>(D);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sU = reinterpret_cast<T*>(smem_raw);
  T* sA = sU + (1 + D) * NP * E;
  __shared__ int s_unit;
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) s_unit = (int)atomicAdd(queue, 1u);
    __syncthreads();
    const int q = s_unit;
    __syncthreads();
    if (q >= nunits) break;
    const int u = units[q];
    const int tile = u & (kSweepVolume - 1);
    if (!(u & kSweepVolume)) {
      trace_tile<D, M, T, E, NW>(U, Tr, c, tile * E);
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        st_release(flags + tile, epoch);
      }
    } else {
      // wait for the traces of tiles tile-K .. tile+K (periodic), bounded
      const unsigned long long t0 = global_ns();
      for (int j = tid; j <= 2 * K; j += NW * 32) {
        int t = tile - K + j;
        t = (t % ntiles + ntiles) % ntiles;
        while (ld_acquire(flags + t) != epoch) {
          if (global_ns() - t0 > 1000000000ull) {
            atomicExch(err, 1);
            break;
          }
          __nanosleep(64);
        }
      }
      __syncthreads();
      __threadfence();
      RhsOut<T> out{R};
      fused_tile<D, M, T, E, NW, true>(U, Tr, out, c, tile * E, sU, sA);
    }
  }
}

template <int D, int M, typename T>
cudaError_t sweep_launch(const fr_ctx* ctx, const FrConst<T>& c, const void* U, void* Tr,
                         void* R, const SweepPlan& p, unsigned epoch, cudaStream_t s) {
  using C = FusedCfg<D, M, T>;
  auto kern = sweep_kernel<D, M, T, C::E, C::NW, C::MINB>;
  static int blocks_per_sm = 0;  // per template instance
  if (!blocks_per_sm) {
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)C::SMEM);
    if (err != cudaSuccess) return err;
    int b = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, C::NW * 32, C::SMEM);
    if (err != cudaSuccess) return err;
    blocks_per_sm = b < 1 ? 1 : b;
  }
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device);
  cudaError_t err = cudaMemsetAsync(p.queue, 0, sizeof(unsigned), s);
  if (err != cudaSuccess) return err;
  kern<<<nsm * blocks_per_sm, C::NW * 32, C::SMEM, s>>>(
      static_cast<const T*>(U), static_cast<T*>(Tr), static_cast<T*>(R), c, p.units, p.nunits,
      p.flags, epoch, p.ntiles, p.K, p.queue, ctx->err);
  return cudaGetLastError();
}

cudaError_t launch_fused(const fr_ctx* c, const void* U, const void* Tr, void* R, cudaStream_t s) {
  if (c->precision == FR_F32) {
    ACMHD_DISPATCH_DM(c->dim, c->m,
                      return (fused_launch<D_, M_, float, false>(c->cf, U, Tr, R, 0, c->ne, s)));
  } else {
    ACMHD_DISPATCH_DM(c->dim, c->m,
                      return (fused_launch<D_, M_, double, false>(c->cd, U, Tr, R, 0, c->ne, s)));
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_sweep(const fr_ctx* c, const void* U, void* Tr, void* R, const SweepPlan& p,
                         unsigned epoch, cudaStream_t s) {
  if (c->precision == FR_F32) {
    ACMHD_DISPATCH_DM(c->dim, c->m,
                      return (sweep_launch<D_, M_, float>(c, c->cf, U, Tr, R, p, epoch, s)));
  } else {
    ACMHD_DISPATCH_DM(c->dim, c->m,
                      return (sweep_launch<D_, M_, double>(c, c->cd, U, Tr, R, p, epoch, s)));
  }
  return cudaErrorInvalidValue;
}

template <typename T>
static cudaError_t tile_elements_t(int dim, int m, int* e) {
  ACMHD_DISPATCH_DM(dim, m, (*e = FusedCfg<D_, M_, T>::E));
  return cudaSuccess;
}

int fused_tile_elements(int dim, int m, int precision) {
  int e = 0;
  if (precision == FR_F32)
    tile_elements_t<float>(dim, m, &e);
  else
    tile_elements_t<double>(dim, m, &e);
  return e;
}

}  // namespace acmhd
