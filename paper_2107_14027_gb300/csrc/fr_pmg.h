// Internal declarations of the P-multigrid pseudo solver (fr_pmg.cu,
// k_pmg.cu).
#pragma once

#include <cuda_runtime.h>

#include "fr_internal.h"

namespace acmhd {

// 1-D transfer matrices between order q (m = q + 1 points) and q - 1:
// Ir[i][k] (coarse i, fine k): L2 projection; Ip[k][i]: interpolation.
template <typename T>
struct PmgTransfer {
  T Ir[kMaxM][kMaxM];
  T Ip[kMaxM][kMaxM];
};

struct PmgTransferPair {
  PmgTransfer<float> f;
  PmgTransfer<double> d;
};

// The fine side's context gives the layout (order, variables, stride); the
// coarse side has order - 1 on the same mesh.
cudaError_t launch_pmg_restrict(const fr_ctx* fine, const void* Xf, void* Yc,
                                const PmgTransferPair& tr, cudaStream_t s);
cudaError_t launch_pmg_prolong(const fr_ctx* fine, const void* Yc, const void* Y0c, void* Xf,
                               double* V, const PmgTransferPair& tr, cudaStream_t s);
cudaError_t launch_pmg_residual(const fr_ctx* c, const void* k, const void* U, const void* g,
                                const double* V, const double* C, double a0dt, void* r,
                                double* partial, cudaStream_t s);
int pmg_norm_blocks(const fr_ctx* c);
cudaError_t launch_pmg_forcing(const fr_ctx* c, const void* Rr, const void* k, const void* U0,
                               double a0dt, void* g, cudaStream_t s);
cudaError_t launch_pmg_coarse_stage(const fr_ctx* c, int stage, double dtau, double a0dt,
                                    double dV, double dA, void* U, const void* g, cudaStream_t s);

// Anderson mixing over the finest level's state: the vectors are the state
// rows other than the velocity (precision T) plus the FP64 velocity master.
constexpr int kAaMax = 16;   // most vectors in a mixing window (memory + 1)
struct AaVectors {
  void* u[kAaMax];
  double* v[kAaMax];
  double c[kAaMax];
  int n;
};

// G <- (U, V); F <- (U, V) - (Xu, Xv)
cudaError_t launch_aa_record(const fr_ctx* c, const void* U, const double* V, const void* Xu,
                             const double* Xv, void* Gu, double* Gv, void* Fu, double* Fv,
                             cudaStream_t s);
// dots[j] = <F, W.u[j] ++ W.v[j]> over real elements (velocity rows from v)
cudaError_t launch_aa_dots(const fr_ctx* c, const void* Fu, const double* Fv, const AaVectors& W,
                           double* partial, int nparts, double* dots, cudaStream_t s);
int aa_dot_blocks(const fr_ctx* c);
// (U, V) <- sum_j W.c[j] (W.u[j], W.v[j]); U's velocity rows <- (T) V
cudaError_t launch_aa_combine(const fr_ctx* c, const AaVectors& W, void* U, double* V,
                              cudaStream_t s);

}  // namespace acmhd
