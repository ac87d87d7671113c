// Fused right-hand-side kernel: stages 2-6 of Table fr_adv in one pass.
//
// For every element and every axis a it evaluates the normal flux F_a at
// the solution points (stage 2), the partially corrected divergence along
// the axis lines (stage 3), the common interface flux at both faces of each
// line (stage 4, from this element's own face trace and the neighbour's
// stored trace), the correction (stage 5), and the negation plus source
// (stage 6):
//
//   R = sum_a  -J_a [ Dt F_a + h_l' F^I_l + h_r' F^I_r ]  -  (1/T) [0; 0; q; r; s]
//
// with Dt = D - h_l' l(-1)^T - h_r' l(+1)^T and J_a = 2 / h_a (Sec. 2.1, FR
// divergence equation).
//
// Work decomposition (GB300): one CTA owns E consecutive elements; lane ->
// element, so every global row access is contiguous.  P and V of the CTA's
// elements are staged once in shared memory, because every axis needs
// them; each auxiliary variable is needed by exactly one axis and is read
// straight from global memory by the thread that owns the line.  The
// three axes run as phases; in each phase a thread owns whole lines along
// the axis, so the 1-D contractions are register FMAs against operator
// constants that come from the kernel-parameter (constant) bank.  Only the
// P and V equations receive contributions from more than one axis; their
// partial sums live in shared memory between phases.  The auxiliary
// equations are finished and written in the phase of their axis.
#include "fr_device.cuh"

namespace acmhd {

template <int D, int M, typename T, int E, int NW, int MINB>
__global__ void __launch_bounds__(NW * 32, MINB)
fused_kernel(const T* __restrict__ U, const T* __restrict__ Tr, T* __restrict__ R,
             const FrConst<T> c) {
  constexpr int NP = ipow<M>(D), NL = ipow<M>(D - 1), NS = 1 + 2 * D, SUB = 32 / E;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sU = reinterpret_cast<T*>(smem_raw);  // [1+D][NP][E]
  T* sA = sU + (1 + D) * NP * E;           // [1+D][NP][E]

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int el = lane % E, sub = lane / E;
  const int e0 = blockIdx.x * E;
  const int e = e0 + el;
  const bool valid = e < c.ne;
  const size_t S = c.stride;

  // stage P and V of the CTA's elements (rows of E contiguous values)
  for (int idx = tid; idx < (1 + D) * NP * E; idx += NW * 32) {
    const int row = idx / E, x = idx - row * E;
    sU[idx] = __ldg(U + (size_t)row * S + e0 + x);
  }
  int nb[3][2];
  neighbours<D>(valid ? e : 0, c.n, nb);
  __syncthreads();

#pragma unroll
  for (int a = 0; a < D; ++a) {
    // the trip count is uniform across the warp (shuffles need every lane)
    for (int l0 = warp * SUB; l0 < NL; l0 += NW * SUB) {
      const bool lvalid = l0 + sub < NL;
      const int l = lvalid ? l0 + sub : NL - 1;
      const bool act = valid && lvalid;
      // slot values along the line
      T u[NS][M];
#pragma unroll
      for (int t = 0; t < M; ++t) {
        const int pt = line_pt<D, M>(a, l, t);
#pragma unroll
        for (int s = 0; s <= D; ++s) u[s][t] = sU[(s * NP + pt) * E + el];
#pragma unroll
        for (int i = 0; i < D; ++i)
          u[1 + D + i][t] = __ldg(U + ((size_t)aux_var<D>(i, a) * NP + pt) * S + e);
      }
      // neighbour traces: issued right after the line's own loads.  In the
      // x phase a neighbour inside the lane group is served by a shuffle
      // below, so only the others are read from memory.
      const bool lo_mem = (a != 0) || (act && !x_pair_on_chip(nb[0][0], e, E));
      const bool hi_mem = (a != 0) || (act && !x_pair_on_chip(e, nb[0][1], E));
      T nb_lo[NS], nb_hi[NS];
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        nb_lo[s] = lo_mem ? __ldg(Tr + (((size_t)(2 * a + 1) * NS + s) * NL + l) * S + nb[a][0])
                          : T(0);
        nb_hi[s] = hi_mem ? __ldg(Tr + (((size_t)(2 * a) * NS + s) * NL + l) * S + nb[a][1])
                          : T(0);
      }
      // own traces, and the common fluxes at the two faces (stage 4)
      T own_lo[NS], own_hi[NS];
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        own_lo[s] = trace_dot<M>(u[s], c.lm);
        own_hi[s] = trace_dot<M>(u[s], c.lp);
      }
      if (a == 0) {
#pragma unroll
        for (int s = 0; s < NS; ++s) {
          const T from_left = __shfl_up_sync(0xffffffffu, own_hi[s], 1, E);
          const T from_right = __shfl_down_sync(0xffffffffu, own_lo[s], 1, E);
          if (!lo_mem) nb_lo[s] = from_left;
          if (!hi_mem) nb_hi[s] = from_right;
        }
      }
      T fl[NS], fr[NS];
      common_flux<D>(nb_lo, own_lo, a, c.zeta, c.nu, c.inv_t, fl);
      common_flux<D>(own_hi, nb_hi, a, c.zeta, c.nu, c.inv_t, fr);
      if (!act) continue;
      // per slot: pointwise flux (stage 2), then divergence + correction +
      // negation (stages 3, 5, 6) along the line
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        T f[M];
#pragma unroll
        for (int t = 0; t < M; ++t) f[t] = point_flux<D>(u, t, s, a, c.zeta, c.nu, c.inv_t);
#pragma unroll
        for (int i = 0; i < M; ++i) {
          T r = fma(c.br[a][i], fr[s], c.bl[a][i] * fl[s]);
#pragma unroll
          for (int k = 0; k < M; ++k) r = fma(c.A[a][i][k], f[k], r);
          const int pt = line_pt<D, M>(a, l, i);
          if (s <= D) {
            const int idx = (s * NP + pt) * E + el;
            if (a == 0) {
              sA[idx] = r;
            } else if (a < D - 1) {
              sA[idx] += r;
            } else {
              R[((size_t)s * NP + pt) * S + e] = sA[idx] + r;
            }
          } else {
            // auxiliary equation of slot s: finished here, with its source
            const int v = aux_var<D>(s - D - 1, a);
            R[((size_t)v * NP + pt) * S + e] = fma(-u[s][i], c.inv_t, r);
          }
        }
      }
    }
    if (a < D - 1) __syncthreads();  // partial sums complete before the next axis
  }
}

template <int D, int M, typename T>
cudaError_t fused_launch(const fr_ctx* ctx, const FrConst<T>& c, const void* U, const void* Tr,
                         void* R, cudaStream_t s) {
  using C = FusedCfg<D, M, T>;
  auto kern = fused_kernel<D, M, T, C::E, C::NW, C::MINB>;
  static bool attr_done = false;  // per template instance
  if (!attr_done) {
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)C::SMEM);
    if (err != cudaSuccess) return err;
    attr_done = true;
  }
  const int nblk = (ctx->ne + C::E - 1) / C::E;
  kern<<<nblk, C::NW * 32, C::SMEM, s>>>(static_cast<const T*>(U), static_cast<const T*>(Tr),
                                          static_cast<T*>(R), c);
  return cudaGetLastError();
}

cudaError_t launch_fused(const fr_ctx* c, const void* U, const void* Tr, void* R, cudaStream_t s) {
  if (c->precision == FR_F32) {
    ACMHD_DISPATCH_DM(c->dim, c->m, return (fused_launch<D_, M_, float>(c, c->cf, U, Tr, R, s)));
  } else {
    ACMHD_DISPATCH_DM(c->dim, c->m, return (fused_launch<D_, M_, double>(c, c->cd, U, Tr, R, s)));
  }
  return cudaErrorInvalidValue;
}

}  // namespace acmhd
