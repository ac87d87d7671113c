// Fused right-hand-side kernel: stages 2-6 of Table fr_adv in one pass.  The
// tile work (fused_tile) and the RHS kernel template are in fused_tile.cuh;
// this file holds the whole-mesh launcher.
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
#include "fused_tile.cuh"

namespace acmhd {

cudaError_t launch_fused(const fr_ctx* c, const void* U, const void* Tr, void* R, cudaStream_t s) {
  if (c->precision == FR_F32) {
    ACMHD_DISPATCH_DM(c->dim, c->m,
                      return (fused_launch<D_, M_, float, float, false>(c->cf, U, Tr, R, 0, c->ne,
                                                                       s)));
  } else if (c->df64) {
    ACMHD_DISPATCH_DM(c->dim, c->m,
                      return (fused_launch<D_, M_, double, df64, false>(c->cdf, U, Tr, R, 0, c->ne,
                                                                       s)));
  } else {
    ACMHD_DISPATCH_DM(c->dim, c->m,
                      return (fused_launch<D_, M_, double, double, false>(c->cd, U, Tr, R, 0,
                                                                         c->ne, s)));
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
