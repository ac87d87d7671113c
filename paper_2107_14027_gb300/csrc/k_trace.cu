// Face-trace kernel: stage 1 of Table fr_adv ("project solution to x_f"),
// restricted to the 1 + 2d slots that the normal flux of each face needs.
//
// Output layout: Tr[f][s][l][e], f = 2a + side (side 0: the face at -1 of
// axis a, side 1: the face at +1), s the slot (fr_device.cuh), l the line
// index along axis a, e the element (stride c.stride); the x faces (a = 0)
// at the column x_col gives (by lane group where the rows allow it).
//
// Mapping: a warp covers E consecutive elements (lane -> element, so every
// global access is one contiguous row) and 32/E lines at once; each thread
// interpolates one line of each slot variable to both ends.  x-face traces
// are stored only for the elements whose x-neighbour will read them from
// memory (x_pair_on_chip): the fused kernel exchanges the others between
// lanes.  P and V are slots of every face, so where they fit in 32 KB the
// tile's P and V are read from HBM once into shared memory and the axes take
// them from there (otherwise each axis reads them again through the caches).
#include "fr_device.cuh"

namespace acmhd {

template <int D, int M, typename T>
constexpr bool trace_stages_pv() {
  return size_t(1 + D) * ipow<M>(D) * 32 * sizeof(T) <= 32 * 1024;
}

// U, Tr hold the storage type S; the interpolation runs in T (S = T, or
// S = double with T = df64), and the stored trace is its value in S.
template <int D, int M, typename S, typename T, int E, int EF>
__global__ void __launch_bounds__(256)
trace_kernel(const S* __restrict__ U, S* __restrict__ Tr, const FrConst<T> c, int tile0) {
  constexpr int NP = ipow<M>(D), NL = ipow<M>(D - 1), NS = 1 + 2 * D, SUB = 32 / E;
  constexpr bool PV = trace_stages_pv<D, M, T>();
  __shared__ T sPV[PV ? (1 + D) * NP * E : 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int el = lane % E;
  const int tile = tile0 + blockIdx.x;
  const int e = tile * E + el;
  const int sub = lane / E;
  if constexpr (PV) {
    // rows of E contiguous elements; the tile lies inside the padded stride
#pragma unroll 8
    for (int idx = threadIdx.x; idx < (1 + D) * NP * E; idx += blockDim.x) {
      const int row = idx / E, x = idx - row * E;
      sPV[idx] = cvt<T>(__ldg(U + (size_t)row * c.stride + tile * E + x));
    }
    __syncthreads();
  }
  if (e >= c.ne) return;
  const size_t Sd = c.stride;
  int nb[3][2];
  neighbours<D>(e, c.n, nb);
  // x faces: stored only where the fused kernel (EF elements per lane
  // group) cannot take them from the neighbouring lane
  const bool need_x_lo = !x_pair_on_chip(nb[0][0], e, EF);
  const bool need_x_hi = !x_pair_on_chip(e, nb[0][1], EF);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const bool need_lo = (a == 0) ? need_x_lo : true;
    const bool need_hi = (a == 0) ? need_x_hi : true;
    if (!need_lo && !need_hi) continue;
    for (int l = warp * SUB + sub; l < NL; l += nw * SUB) {
      // all loads of the line first, then the interpolations
      T x[NS][M];
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        const int v = slot_var<D>(s, a);
#pragma unroll
        for (int t = 0; t < M; ++t) {
          const int pt = line_pt<D, M>(a, l, t);
          x[s][t] = (PV && s <= D) ? sPV[(s * NP + pt) * E + el]
                                   : cvt<T>(__ldg(U + ((size_t)v * NP + pt) * Sd + e));
        }
      }
      // x faces stored by group (x_col)
      const size_t clo = (a == 0) ? x_col(e, EF, c.xcompact, false) : (size_t)e;
      const size_t chi = (a == 0) ? x_col(e, EF, c.xcompact, true) : (size_t)e;
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        if (need_lo)
          Tr[(((size_t)(2 * a) * NS + s) * NL + l) * Sd + clo] = cvt<S>(trace_dot<M>(x[s], c.lm));
        if (need_hi)
          Tr[(((size_t)(2 * a + 1) * NS + s) * NL + l) * Sd + chi] =
              cvt<S>(trace_dot<M>(x[s], c.lp));
      }
    }
  }
}

// elements [e_begin, e_end); e_begin a multiple of 32
template <int D, int M, typename S, typename T>
cudaError_t trace_launch(const FrConst<T>& c, const void* U, void* Tr, int e_begin, int e_end,
                         cudaStream_t s) {
  constexpr int E = 32;
  const int nblk = (e_end - e_begin + E - 1) / E;
  if (nblk <= 0) return cudaSuccess;
  trace_kernel<D, M, S, T, E, FusedCfg<D, M, T>::E>
      <<<nblk, 256, 0, s>>>(static_cast<const S*>(U), static_cast<S*>(Tr), c, e_begin / E);
  return cudaGetLastError();
}

cudaError_t launch_trace_range(const fr_ctx* c, const void* U, void* Tr, int e_begin, int e_end,
                               cudaStream_t s) {
  if (e_begin % 32 != 0) return cudaErrorInvalidValue;
  if (c->precision == FR_F32) {
    ACMHD_DISPATCH_DM(c->dim, c->m,
                      return (trace_launch<D_, M_, float, float>(c->cf, U, Tr, e_begin, e_end, s)));
  } else if (c->df64) {
    ACMHD_DISPATCH_DM(c->dim, c->m,
                      return (trace_launch<D_, M_, double, df64>(c->cdf, U, Tr, e_begin, e_end, s)));
  } else {
    ACMHD_DISPATCH_DM(c->dim, c->m,
                      return (trace_launch<D_, M_, double, double>(c->cd, U, Tr, e_begin, e_end,
                                                                  s)));
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_trace(const fr_ctx* c, const void* U, void* Tr, cudaStream_t s) {
  return launch_trace_range(c, U, Tr, 0, c->ne, s);
}

}  // namespace acmhd
