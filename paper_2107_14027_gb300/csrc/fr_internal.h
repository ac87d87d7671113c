// Internal declarations of the ACM-HD flux-reconstruction library (host side).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "acmhd_fr.h"
#include "df64.cuh"

namespace acmhd {

constexpr int kMaxM = 7;  // p <= 6

// 1-D operators of FR for m = p + 1 Gauss-Legendre solution points, FP64.
// Sec. 2.1 (FR divergence equation): l_k Lagrange basis, h_l / h_r the left
// and right correction functions with h_l(-1) = h_r(1) = 1, h_l(1) = h_r(-1) = 0.
struct Ops1D {
  int m;
  double xi[kMaxM], w[kMaxM];
  double D[kMaxM][kMaxM];   // D[i][k] = l_k'(xi_i)
  double lm[kMaxM];         // l_k(-1)
  double lp[kMaxM];         // l_k(+1)
  double dhl[kMaxM];        // h_l'(xi_i)
  double dhr[kMaxM];        // h_r'(xi_i)
  double Dt[kMaxM][kMaxM];  // partially corrected divergence operator
                            // D - h_l' l(-1)^T - h_r' l(+1)^T (Table fr_adv, stage 3)
};

// Builds the operators; correction is FR_CORR_DG or FR_CORR_G2.
bool build_ops1d(int order, int correction, Ops1D* out);

// 1-D L2 projection onto polynomials of degree <= q on the GL points of o:
// P[i][k] = sum_{n <= q} phi_n(x_i) phi_n(x_k) w_k, phi_n the orthonormal
// Legendre polynomials (smoothing of the learned initial guess's correction).
void degree_projector(const Ops1D& o, int q, double (*P)[kMaxM]);

// Everything a kernel needs, passed by value (lands in the constant bank).
template <typename T>
struct FrConst {
  // fused kernel: per-axis operators pre-scaled by -J_a (J_a = 2 / h_a), so
  // that R gets  sum_k A[a][i][k] F_k + bl[a][i] F^I_l + br[a][i] F^I_r
  T A[3][kMaxM][kMaxM];
  T bl[3][kMaxM];
  T br[3][kMaxM];
  // unscaled operators (unfused stage kernels)
  T Dt[kMaxM][kMaxM];
  T dhl[kMaxM], dhr[kMaxM];
  T J[3];
  T lm[kMaxM], lp[kMaxM];
  T zeta, nu, inv_t;
  int n[3];        // elements per direction (n[2] = 1 in 2-D)
  int ne;          // number of elements
  int stride;      // elem_stride
  int xcompact;    // x-face trace columns at lane-group ends (x_col): 0, 1 or 2
};

// most slabs of the host-buffer RHS pipeline (fr_rhs_host).  Measured on
// GB300 (64^3 p=3 FP32, 872 MB each way): 1 slab 9.43 ms per call, 2 9.07,
// 3 8.99, 4 8.61, 8 9.71.  A slab's copy is one 2-D copy of nv m^d row
// segments; narrower segments copy more slowly (8 slabs: 6.9 ms in, 6.0 ms
// out, against 4.1 ms for one contiguous copy), which cancels the overlap.
constexpr int kHostSlabsMax = 4;

// ring slot of the level `back` steps before the newest one
inline int hist_slot(int head, int back) { return (head + 4 - back) % 4; }

// Arguments of one fused RK4 stage (k_fused.cu, StageOut): the stage input
// is read by the volume work, its result goes to `next` (stages 0..2) or to
// U (stage 3), and the traces of that result to `tr`.
struct StageArgs {
  void* U;
  void* next;
  void* acc;
  void* tr;
  double ct;          // stage coefficient, already rounded to the precision
  double c, a0dt;     // FP64 velocity rows (dual)
  int stage;
  int dual;
  double* V;
  double* Vs;
  double* Vacc;
  const double* C;
};

}  // namespace acmhd

struct fr_ctx {
  int device;
  int dim, order, m, nv, precision, correction;
  fr_mesh mesh;
  double zeta, nu, t_r;
  int ne;
  size_t stride;       // elem_stride (multiple of 32)
  int npts;            // m^dim
  size_t bytes_state;  // nv * npts * stride * sizeof(T)
  size_t elem_bytes;   // sizeof(T)
  acmhd::Ops1D ops;
  acmhd::FrConst<float> cf;
  acmhd::FrConst<double> cd;
  acmhd::FrConst<acmhd::df64> cdf;
  int df64;            // FR_DF64: FP64 storage, double-float arithmetic in the RHS kernels
  // device scratch owned by the context
  void* trace;         // [2d faces][1+2d slots][m^(d-1)][stride]
  size_t trace_bytes;
  void* rk_stage;      // RK4 stage input
  void* rk_acc;        // RK4 accumulator
  void* rk_k;          // RK4 stage derivative
  void* rk_stage2;     // second stage input of the fused-stage schedule
  void* trace2;        // second trace buffer of the fused-stage schedule
  double* stage_partial;  // residual partial sums of the fused stage (one per CTA)
  void* unf_uf;        // unfused: traces of all variables [2d][nv][m^(d-1)][stride]
  void* unf_f;         // unfused: flux [d][nv][m^d][stride]
  void* unf_div;       // unfused: divergence [nv][m^d][stride]
  void* unf_fi;        // unfused: common flux [2d][nv][m^(d-1)][stride]
  void* host_u;        // fr_rhs_host device staging
  void* host_r;
  cudaStream_t hs[3];  // fr_rhs_host pipeline: copies in, kernels, copies out
  cudaEvent_t hev[2 * acmhd::kHostSlabsMax + 2];  // per slab: in, computed; start; done
  int hs_ready;
  // dual time stepping (FP64 velocity rows: dim * npts * stride doubles)
  double* dual_vs;     // RK4 stage velocity
  double* dual_vacc;   // RK4 velocity accumulator
  double* dual_c;      // BDF constant part -(a1 V^n + a2 V^{n-1}) / dt
  double* dual_partial;  // residual partial sums (one per block)
  double* dual_res;    // residual (one double)
  double* dual_v;      // velocity master of fr_dual_step
  void* hist_u[4];     // physical-time levels of the state (precision T)
  double* hist_v[4];   // physical-time levels of the velocity (FP64)
  int hist_head;       // ring slot of the newest level
  int hist_levels;     // number of valid levels (0..4)
  void* guess_u;       // alternative initial guess (state, precision T)
  double* guess_v;     // alternative initial guess (FP64 velocity)
  double* guess_r0;    // pseudo residual (velocity rows, FP64) of the extrapolation
  double* guess_dots;  // [2 dual_norm_blocks] partial sums, then the two dots
  int schedule;        // FR_SCHEDULE_* requested for the pseudo steps
};

namespace acmhd {

// The kernel constants of a context: the 1-D operators pre-scaled by the
// mesh's -J_a, the parameters and the mesh shape (defined in fr_api.cu; used
// by fr_create and fr_rhs_static alike).
void fill_const(const fr_ctx* c, FrConst<float>* k);
void fill_const(const fr_ctx* c, FrConst<double>* k);
void fill_const(const fr_ctx* c, FrConst<df64>* k);

// Allocate (on first use) a context's RK4 registers / FP64 dual-time
// registers; map a CUDA status to an FR_* code (recording its text).
int ensure_rk_registers(fr_ctx* c);
int ensure_dual_registers(fr_ctx* c);
int status_of(cudaError_t e, const char* where);

// kernel launchers (defined in the k_*.cu files)
cudaError_t launch_trace(const fr_ctx* c, const void* U, void* trace, cudaStream_t s);
cudaError_t launch_fused(const fr_ctx* c, const void* U, const void* trace, void* R,
                         cudaStream_t s);
// The same on the elements [e_begin, e_end) only (e_begin a multiple of 32).
cudaError_t launch_trace_range(const fr_ctx* c, const void* U, void* trace, int e_begin,
                               int e_end, cudaStream_t s);
cudaError_t launch_fused_range(const fr_ctx* c, const void* U, const void* trace, void* R,
                               int e_begin, int e_end, cudaStream_t s);
cudaError_t launch_unfused(const fr_ctx* c, const void* U, void* R, cudaStream_t s);
int fused_tile_elements(int dim, int m, int precision);
int dual_norm_blocks(const fr_ctx* c);
cudaError_t launch_sync_velocity(const fr_ctx* c, const double* V, void* U, cudaStream_t s);
cudaError_t launch_widen_velocity(const fr_ctx* c, const void* U, double* V, cudaStream_t s);
cudaError_t launch_bdf_const(const fr_ctx* c, double c1, double c2, const double* Vn,
                             const double* Vnm1, double* C, cudaStream_t s);
cudaError_t launch_dual_stage(const fr_ctx* c, int stage, double dtau, double a0dt, void* U,
                              double* V, const double* C, double* partial, cudaStream_t s,
                              double dV = 1.0, double dA = 1.0);
// out[0] = <a, b - a>, out[1] = |b - a|^2 over the real entries of two FP64
// velocity vectors; partial holds 2 * dual_norm_blocks doubles
cudaError_t launch_pair_dots(const fr_ctx* c, const double* a, const double* b, double* partial,
                             double* out, cudaStream_t s);
cudaError_t launch_norm_final(const fr_ctx* c, const double* partial, int nparts, double count,
                              double* out, cudaStream_t s);
cudaError_t launch_stage(const fr_ctx* c, const void* U, const void* Tr, const StageArgs& a,
                         double* partial, cudaStream_t s);
int stage_blocks(const fr_ctx* c);
cudaError_t launch_convert(const fr_ctx* c, size_t n, int prec_in, const void* x, int prec_out,
                           void* y, cudaStream_t s);
cudaError_t launch_combine3(const fr_ctx* c, int precision, size_t n, double c0, double c1,
                            double c2, const void* x0, const void* x1, const void* x2, void* out,
                            cudaStream_t s);
// Sets the text that fr_last_error() returns in the calling thread.
void set_last_error(const char* msg);

cudaError_t launch_rk_stage(const fr_ctx* c, int stage, double dtau, void* U,
                            cudaStream_t s);

}  // namespace acmhd
