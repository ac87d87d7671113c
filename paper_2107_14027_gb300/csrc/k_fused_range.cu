// The fused RHS kernel on a range of elements (RANGED instantiations), for
// the slab pipeline of the host-buffer RHS; kept apart from k_fused.cu so the
// two compile in parallel.
#include "fused_tile.cuh"

namespace acmhd {

cudaError_t launch_fused_range(const fr_ctx* c, const void* U, const void* Tr, void* R,
                               int e_begin, int e_end, cudaStream_t s) {
  if (e_begin % 32 != 0) return cudaErrorInvalidValue;
  if (c->precision == FR_F32) {
    ACMHD_DISPATCH_DM(
        c->dim, c->m,
        return (fused_launch<D_, M_, float, float, true>(c->cf, U, Tr, R, e_begin, e_end, s)));
  } else if (c->df64) {
    ACMHD_DISPATCH_DM(
        c->dim, c->m,
        return (fused_launch<D_, M_, double, df64, true>(c->cdf, U, Tr, R, e_begin, e_end, s)));
  } else {
    ACMHD_DISPATCH_DM(
        c->dim, c->m,
        return (fused_launch<D_, M_, double, double, true>(c->cd, U, Tr, R, e_begin, e_end, s)));
  }
  return cudaErrorInvalidValue;
}

}  // namespace acmhd
