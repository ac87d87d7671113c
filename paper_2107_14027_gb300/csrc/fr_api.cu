// C ABI of the ACM-HD flux-reconstruction library (declared in acmhd_fr.h):
// argument checking, context and scratch ownership, and the sequencing of
// kernel launches.  All arithmetic of the method runs in the k_*.cu kernels.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "fr_internal.h"
#include "xface_layout.h"

namespace {

thread_local char g_last_error[256] = "";

void set_cuda_error(cudaError_t e, const char* where) {
  std::snprintf(g_last_error, sizeof(g_last_error), "%s: %s", where, cudaGetErrorString(e));
}

int cuda_status(cudaError_t e, const char* where) {
  if (e == cudaSuccess) return FR_OK;
  set_cuda_error(e, where);
  return (e == cudaErrorMemoryAllocation) ? FR_ENOMEM : FR_ECUDA;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

template <typename T>
void fill_const_t(const fr_ctx* c, acmhd::FrConst<T>* k) {
  std::memset(k, 0, sizeof(*k));
  const acmhd::Ops1D& o = c->ops;
  for (int a = 0; a < c->dim; ++a) {
    const double h = (c->mesh.hi[a] - c->mesh.lo[a]) / c->mesh.n[a];
    const double J = 2.0 / h;
    k->J[a] = static_cast<T>(J);
    for (int i = 0; i < o.m; ++i) {
      for (int q = 0; q < o.m; ++q) k->A[a][i][q] = static_cast<T>(-J * o.Dt[i][q]);
      k->bl[a][i] = static_cast<T>(-J * o.dhl[i]);
      k->br[a][i] = static_cast<T>(-J * o.dhr[i]);
    }
  }
  for (int i = 0; i < o.m; ++i) {
    for (int q = 0; q < o.m; ++q) k->Dt[i][q] = static_cast<T>(o.Dt[i][q]);
    k->dhl[i] = static_cast<T>(o.dhl[i]);
    k->dhr[i] = static_cast<T>(o.dhr[i]);
    k->lm[i] = static_cast<T>(o.lm[i]);
    k->lp[i] = static_cast<T>(o.lp[i]);
  }
  k->zeta = static_cast<T>(c->zeta);
  k->nu = static_cast<T>(c->nu);
  k->inv_t = static_cast<T>(1.0 / c->t_r);
  k->n[0] = c->mesh.n[0];
  k->n[1] = c->mesh.n[1];
  k->n[2] = c->dim == 3 ? c->mesh.n[2] : 1;
  k->ne = c->ne;
  k->stride = static_cast<int>(c->stride);
  const int E = acmhd::fused_tile_elements(c->dim, c->m, sizeof(T) == 4 ? FR_F32 : FR_F64);
  // x-face trace columns (x_col): by group where the rows allow it
  k->xcompact = acmhd::x_compact_mode(c->mesh.n[0], E);
}

int alloc_zeroed(void** p, size_t bytes, const char* what) {
  if (*p) return FR_OK;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_status(e, what);
  }
  e = cudaMemset(*p, 0, bytes);
  return cuda_status(e, what);
}

int ensure_rk(fr_ctx* c) {
  int st;
  if ((st = alloc_zeroed(&c->rk_stage, c->bytes_state, "rk registers")) != FR_OK) return st;
  if ((st = alloc_zeroed(&c->rk_acc, c->bytes_state, "rk registers")) != FR_OK) return st;
  return alloc_zeroed(&c->rk_k, c->bytes_state, "rk registers");
}

// Scratch of the fused-stage schedule: a second stage input and a second
// trace buffer (stage inputs U -> S1 -> S2 -> S1 -> U, traces alternating
// between the two buffers), and one residual partial per CTA.
int ensure_stage(fr_ctx* c) {
  int st = ensure_rk(c);
  if (st == FR_OK) st = alloc_zeroed(&c->rk_stage2, c->bytes_state, "rk registers");
  if (st == FR_OK) st = alloc_zeroed(&c->trace2, c->trace_bytes, "trace scratch");
  if (st == FR_OK)
    st = alloc_zeroed((void**)&c->stage_partial,
                      (size_t)acmhd::stage_blocks(c) * sizeof(double), "dual registers");
  return st;
}

// Stage `stage` (0..3) of the fused-stage schedule.  Stage 0 reads the traces
// of U from c->trace; every stage writes the traces of its result to the
// other buffer, so after stage 3 the traces of the new U are in c->trace.
int fused_stage(fr_ctx* c, int stage, void* U, acmhd::StageArgs a, cudaStream_t s) {
  static const int kIn[4] = {0, 1, 2, 1};    // 0 = U, 1 = S1, 2 = S2
  static const int kNext[4] = {1, 2, 1, 0};
  void* buf[3] = {U, c->rk_stage, c->rk_stage2};
  a.U = U;
  a.next = buf[kNext[stage]];  // stage 3 stores to U (and never through `next`)
  a.acc = c->rk_acc;
  a.tr = (stage % 2 == 0) ? c->trace2 : c->trace;
  a.stage = stage;
  const void* tr_in = (stage % 2 == 0) ? c->trace : c->trace2;
  return cuda_status(acmhd::launch_stage(c, buf[kIn[stage]], tr_in, a, c->stage_partial, s),
                     "fused stage");
}

// Host-buffer RHS pipeline.  The elements are cut into S slabs of whole
// 32-element tiles, each at least one element layer (z-plane in 3-D, x-row
// in 2-D) plus a tile, so the face neighbours of a slab lie in the two
// adjacent slabs (periodically).  Each slab is copied in, its traces are
// computed as soon as it has arrived, its volume work runs once its
// neighbours' traces exist (slabs 1 .. S-1, then 0, which needs the last
// slab's traces), and its R is copied out while later slabs are still
// arriving or being computed: copies in both directions and the kernels
// overlap on three streams.
using acmhd::kHostSlabsMax;

int host_slabs(const fr_ctx* c, int* bounds) {
  const long long layer = c->dim == 3 ? (long long)c->mesh.n[0] * c->mesh.n[1] : c->mesh.n[0];
  const long long ntile = (c->ne + 31) / 32;
  const long long min_tiles = (layer + 31) / 32 + 1;
  int S = kHostSlabsMax;
  while (S > 1 && ntile / S < min_tiles) --S;
  for (int i = 0; i <= S; ++i) {
    const long long b = ntile * i / S * 32;
    bounds[i] = (int)(b < c->ne ? b : c->ne);
  }
  return S;
}

int ensure_host_pipeline(fr_ctx* c) {
  if (c->hs_ready) return FR_OK;
  for (int i = 0; i < 3; ++i) {
    int st = cuda_status(cudaStreamCreateWithFlags(&c->hs[i], cudaStreamNonBlocking),
                         "pipeline streams");
    if (st != FR_OK) return st;
  }
  for (int i = 0; i < 2 * kHostSlabsMax + 2; ++i) {
    int st = cuda_status(cudaEventCreateWithFlags(&c->hev[i], cudaEventDisableTiming),
                         "pipeline events");
    if (st != FR_OK) return st;
  }
  c->hs_ready = 1;
  return FR_OK;
}

// One slab's rows between the padded host and device layouts: nv m^d rows of
// (e_end - e_begin) values at pitch elem_stride.
cudaError_t copy_slab(const fr_ctx* c, void* dst, const void* src, int e_begin, int e_end,
                      cudaMemcpyKind kind, cudaStream_t s) {
  const size_t pitch = c->stride * c->elem_bytes, off = (size_t)e_begin * c->elem_bytes;
  return cudaMemcpy2DAsync(static_cast<char*>(dst) + off, pitch,
                           static_cast<const char*>(src) + off, pitch,
                           (size_t)(e_end - e_begin) * c->elem_bytes, (size_t)c->nv * c->npts,
                           kind, s);
}

int rhs_host_pipelined(fr_ctx* c, const void* U_host, void* R_host, const int* b, int S,
                       cudaStream_t s) {
  cudaStream_t in = c->hs[0], k = c->hs[1], out = c->hs[2];
  cudaEvent_t* ev_in = c->hev;
  cudaEvent_t* ev_done = c->hev + kHostSlabsMax;
  cudaEvent_t ev_start = c->hev[2 * kHostSlabsMax], ev_end = c->hev[2 * kHostSlabsMax + 1];
  cudaError_t e = cudaEventRecord(ev_start, s);  // after the caller's earlier work
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(c->hs[i], ev_start, 0);
  for (int i = 0; i < S && e == cudaSuccess; ++i) {
    e = copy_slab(c, c->host_u, U_host, b[i], b[i + 1], cudaMemcpyHostToDevice, in);
    if (e == cudaSuccess) e = cudaEventRecord(ev_in[i], in);
  }
  auto volume = [&](int i) {
    cudaError_t r = acmhd::launch_fused_range(c, c->host_u, c->trace, c->host_r, b[i], b[i + 1], k);
    if (r == cudaSuccess) r = cudaEventRecord(ev_done[i], k);
    if (r == cudaSuccess) r = cudaStreamWaitEvent(out, ev_done[i], 0);
    if (r == cudaSuccess) r = copy_slab(c, R_host, c->host_r, b[i], b[i + 1],
                                        cudaMemcpyDeviceToHost, out);
    return r;
  };
  for (int i = 0; i < S && e == cudaSuccess; ++i) {
    e = cudaStreamWaitEvent(k, ev_in[i], 0);
    if (e == cudaSuccess) e = acmhd::launch_trace_range(c, c->host_u, c->trace, b[i], b[i + 1], k);
    if (e == cudaSuccess && i >= 2) e = volume(i - 1);  // traces i-2 .. i exist
  }
  if (e == cudaSuccess && S >= 2) e = volume(S - 1);    // needs traces S-2, S-1, 0
  if (e == cudaSuccess) e = volume(0);                    // needs traces S-1, 0, 1
  if (e == cudaSuccess) e = cudaEventRecord(ev_end, out);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev_end, 0);
  return cuda_status(e, "host-buffer pipeline");
}

// Pseudo steps with the update fused into the volume kernel: on request, and
// by default at p <= 2.  Measured on GB300 (FP32 RK4 steps on the 3-D order
// sweep meshes of about 38M points per variable, fused / separate):
// p = 1 11.5 / 14.0 ms, p = 2 11.3 / 13.7, p = 3 11.7-12.8 / 11.6, p = 4
// 17.0 / 13.2 (at p = 3 the fused stage led, 11.4 / 12.6, until the trace
// and volume kernels stored the x-face traces by group).  At p >= 4 the stage
// kernel's larger line work leaves too few resident warps to stream the
// update traffic as fast as the separate update kernel does.  FP64 (ALU bound
// on this part): equal times at p = 1..3.
bool use_fused_stage(const fr_ctx* c) {
  if (c->df64) return false;   // the fused stage has no double-float instance
  return c->schedule == FR_SCHEDULE_FUSED_STAGE ||
         (c->schedule == FR_SCHEDULE_AUTO && c->order <= 2);
}

// RK4 stage coefficient (dtau/2, dtau/2, dtau, dtau/6) rounded to the
// context precision as the separate update kernels round it: computed in T
// for the plain step, in FP64 and then rounded for the dual step.
double stage_coef(const fr_ctx* c, int stage, double dtau, bool dual) {
  if (dual) {
    const double v = stage == 2 ? dtau : (stage == 3 ? dtau / 6.0 : 0.5 * dtau);
    return c->precision == FR_F32 ? (double)(float)v : v;
  }
  if (c->precision == FR_F32) {
    const float d = (float)dtau;
    return (double)(stage == 2 ? d : (stage == 3 ? d / 6.0f : d * 0.5f));
  }
  return stage == 2 ? dtau : (stage == 3 ? dtau / 6.0 : dtau * 0.5);
}

int ensure_unfused(fr_ctx* c) {
  const size_t nl = c->npts / c->m;
  const size_t row = c->stride * c->elem_bytes;
  int st;
  if ((st = alloc_zeroed(&c->unf_uf, 2 * c->dim * c->nv * nl * row, "unfused traces")) != FR_OK)
    return st;
  if ((st = alloc_zeroed(&c->unf_f, (size_t)c->dim * c->bytes_state, "unfused flux")) != FR_OK)
    return st;
  if ((st = alloc_zeroed(&c->unf_div, c->bytes_state, "unfused divergence")) != FR_OK) return st;
  return alloc_zeroed(&c->unf_fi, 2 * c->dim * c->nv * nl * row, "unfused common flux");
}

bool bad_state_ptr(const void* p) { return p == nullptr || !aligned16(p); }

size_t vel_doubles(const fr_ctx* c) { return (size_t)c->dim * c->npts * c->stride; }

int ensure_dual(fr_ctx* c) {
  const size_t vb = vel_doubles(c) * sizeof(double);
  int st;
  if ((st = alloc_zeroed((void**)&c->dual_vs, vb, "dual registers")) != FR_OK) return st;
  if ((st = alloc_zeroed((void**)&c->dual_vacc, vb, "dual registers")) != FR_OK) return st;
  if ((st = alloc_zeroed((void**)&c->dual_c, vb, "dual registers")) != FR_OK) return st;
  if ((st = alloc_zeroed((void**)&c->dual_partial,
                         acmhd::dual_norm_blocks(c) * sizeof(double), "dual registers")) != FR_OK)
    return st;
  return alloc_zeroed((void**)&c->dual_res, sizeof(double), "dual registers");
}

int ensure_history(fr_ctx* c) {
  int st;
  if ((st = alloc_zeroed((void**)&c->dual_v, vel_doubles(c) * sizeof(double), "history")) != FR_OK)
    return st;
  for (int i = 0; i < 4; ++i) {
    if ((st = alloc_zeroed(&c->hist_u[i], c->bytes_state, "history")) != FR_OK) return st;
    if ((st = alloc_zeroed((void**)&c->hist_v[i], vel_doubles(c) * sizeof(double), "history")) !=
        FR_OK)
      return st;
  }
  return FR_OK;
}

}  // namespace

int acmhd::ensure_rk_registers(fr_ctx* c) { return ensure_rk(c); }
int acmhd::ensure_dual_registers(fr_ctx* c) { return ensure_dual(c); }
int acmhd::status_of(cudaError_t e, const char* where) { return cuda_status(e, where); }

void acmhd::fill_const(const fr_ctx* c, FrConst<float>* k) { fill_const_t(c, k); }
void acmhd::fill_const(const fr_ctx* c, FrConst<double>* k) { fill_const_t(c, k); }
void acmhd::fill_const(const fr_ctx* c, FrConst<df64>* k) { fill_const_t(c, k); }

void acmhd::set_last_error(const char* msg) {
  std::snprintf(g_last_error, sizeof(g_last_error), "%s", msg);
}

extern "C" {

int fr_create(const fr_mesh* mesh, int order, int nvars, double zeta, double nu, double t_r,
              int precision, int correction, fr_ctx** out) {
  g_last_error[0] = '\0';
  if (!mesh || !out) return FR_EINVAL;
  const int d = mesh->dim;
  if (d != 2 && d != 3) return FR_EINVAL;
  if (order < 1 || order > acmhd::kMaxM - 1) return FR_EINVAL;
  if (nvars != 1 + d + d * d) return FR_EINVAL;
  if (precision != FR_F32 && precision != FR_F64 && precision != FR_DF64) return FR_EINVAL;
  if (correction != FR_CORR_DG && correction != FR_CORR_G2) return FR_EINVAL;
  if (!(zeta > 0.0) || !(nu >= 0.0) || !(t_r > 0.0) || !std::isfinite(zeta) ||
      !std::isfinite(nu) || !std::isfinite(t_r))
    return FR_EINVAL;
  long long ne = 1;
  for (int a = 0; a < d; ++a) {
    if (mesh->n[a] < 1) return FR_EINVAL;
    if (!(mesh->hi[a] > mesh->lo[a]) || !std::isfinite(mesh->hi[a] - mesh->lo[a]))
      return FR_EINVAL;
    ne *= mesh->n[a];
  }
  if (ne > (1LL << 30)) return FR_EINVAL;

  fr_ctx* c = new (std::nothrow) fr_ctx;
  if (!c) return FR_ENOMEM;
  std::memset(c, 0, sizeof(*c));
  c->dim = d;
  c->order = order;
  c->m = order + 1;
  c->nv = nvars;
  // FR_DF64 stores FP64 like FR_F64 (every buffer and the FP64 kernels treat
  // it so); only the trace and volume kernels compute in double-float
  c->precision = precision == FR_DF64 ? FR_F64 : precision;
  c->df64 = precision == FR_DF64 ? 1 : 0;
  c->correction = correction;
  c->mesh = *mesh;
  c->zeta = zeta;
  c->nu = nu;
  c->t_r = t_r;
  c->ne = static_cast<int>(ne);
  c->stride = (static_cast<size_t>(ne) + 31) / 32 * 32;
  c->npts = 1;
  for (int a = 0; a < d; ++a) c->npts *= c->m;
  c->elem_bytes = c->precision == FR_F32 ? 4 : 8;
  c->bytes_state = (size_t)c->nv * c->npts * c->stride * c->elem_bytes;
  if (c->stride > 0x7fffffff) {
    delete c;
    return FR_EINVAL;
  }
  if (!acmhd::build_ops1d(order, correction, &c->ops)) {
    delete c;
    return FR_EINVAL;
  }
  acmhd::fill_const(c, &c->cf);
  acmhd::fill_const(c, &c->cd);
  acmhd::fill_const(c, &c->cdf);

  int st = cuda_status(cudaGetDevice(&c->device), "cudaGetDevice");
  if (st == FR_OK) {
    const size_t nl = c->npts / c->m;
    c->trace_bytes = (size_t)(2 * d) * (1 + 2 * d) * nl * c->stride * c->elem_bytes;
    st = alloc_zeroed(&c->trace, c->trace_bytes, "trace scratch");
  }
  if (st != FR_OK) {
    fr_destroy(c);
    return st;
  }
  *out = c;
  return FR_OK;
}

void fr_destroy(fr_ctx* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  if (c->hs_ready) {
    for (int i = 0; i < 3; ++i) cudaStreamDestroy(c->hs[i]);
    for (int i = 0; i < 2 * kHostSlabsMax + 2; ++i) cudaEventDestroy(c->hev[i]);
  }
  void* bufs[] = {c->trace, c->rk_stage, c->rk_acc, c->rk_k, c->rk_stage2, c->trace2,
                  c->stage_partial, c->unf_uf, c->unf_f,
                  c->unf_div, c->unf_fi, c->host_u, c->host_r,
                  c->dual_vs, c->dual_vacc, c->dual_c, c->dual_partial, c->dual_res, c->dual_v,
                  c->hist_u[0], c->hist_u[1], c->hist_u[2], c->hist_u[3],
                  c->hist_v[0], c->hist_v[1], c->hist_v[2], c->hist_v[3],
                  c->guess_u, c->guess_v, c->guess_r0, c->guess_dots};
  for (void* p : bufs)
    if (p) cudaFree(p);
  delete c;
}

int fr_layout(const fr_ctx* c, size_t* elem_stride, size_t* n_elem, size_t* bytes_per_state) {
  if (!c) return FR_EINVAL;
  if (elem_stride) *elem_stride = c->stride;
  if (n_elem) *n_elem = static_cast<size_t>(c->ne);
  if (bytes_per_state) *bytes_per_state = c->bytes_state;
  return FR_OK;
}

int fr_rhs(fr_ctx* c, const void* U, void* R, void* stream) {
  if (!c || bad_state_ptr(U) || bad_state_ptr(R) || U == R) return FR_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int st = cuda_status(acmhd::launch_trace(c, U, c->trace, s), "trace kernel");
  if (st != FR_OK) return st;
  return cuda_status(acmhd::launch_fused(c, U, c->trace, R, s), "fused kernel");
}

int fr_set_schedule(fr_ctx* c, int schedule) {
  if (!c) return FR_EINVAL;
  if (schedule != FR_SCHEDULE_AUTO && schedule != FR_SCHEDULE_TWO_KERNELS &&
      schedule != FR_SCHEDULE_FUSED_STAGE)
    return FR_EINVAL;
  c->schedule = schedule;
  return FR_OK;
}

int fr_trace(fr_ctx* c, const void* U, void* stream) {
  if (!c || bad_state_ptr(U)) return FR_EINVAL;
  return cuda_status(acmhd::launch_trace(c, U, c->trace, static_cast<cudaStream_t>(stream)),
                     "trace kernel");
}

int fr_rhs_volume(fr_ctx* c, const void* U, void* R, void* stream) {
  if (!c || bad_state_ptr(U) || bad_state_ptr(R) || U == R) return FR_EINVAL;
  return cuda_status(acmhd::launch_fused(c, U, c->trace, R, static_cast<cudaStream_t>(stream)),
                     "fused kernel");
}

int fr_rhs_unfused(fr_ctx* c, const void* U, void* R, void* stream) {
  if (!c || bad_state_ptr(U) || bad_state_ptr(R) || U == R) return FR_EINVAL;
  int st = ensure_unfused(c);
  if (st != FR_OK) return st;
  return cuda_status(acmhd::launch_unfused(c, U, R, static_cast<cudaStream_t>(stream)),
                     "unfused kernels");
}

int fr_rhs_host(fr_ctx* c, const void* U_host, void* R_host, void* stream) {
  if (!c || !U_host || !R_host) return FR_EINVAL;
  int st;
  if ((st = alloc_zeroed(&c->host_u, c->bytes_state, "host staging")) != FR_OK) return st;
  if ((st = alloc_zeroed(&c->host_r, c->bytes_state, "host staging")) != FR_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int bounds[kHostSlabsMax + 1];
  const int S = host_slabs(c, bounds);
  if (S > 1) {
    if ((st = ensure_host_pipeline(c)) != FR_OK) return st;
    st = rhs_host_pipelined(c, U_host, R_host, bounds, S, s);
    if (st == FR_OK) st = cuda_status(cudaStreamSynchronize(s), "stream synchronize");
    return st;
  }
  st = cuda_status(cudaMemcpyAsync(c->host_u, U_host, c->bytes_state, cudaMemcpyHostToDevice, s),
                   "copy to device");
  if (st == FR_OK) st = fr_rhs(c, c->host_u, c->host_r, stream);
  if (st == FR_OK)
    st = cuda_status(
        cudaMemcpyAsync(R_host, c->host_r, c->bytes_state, cudaMemcpyDeviceToHost, s),
        "copy to host");
  if (st == FR_OK) st = cuda_status(cudaStreamSynchronize(s), "stream synchronize");
  return st;
}

int fr_rk_step(fr_ctx* c, void* U, double dtau, void* stream) {
  if (!c || bad_state_ptr(U) || !std::isfinite(dtau)) return FR_EINVAL;
  int st = ensure_rk(c);
  if (st != FR_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (use_fused_stage(c)) {
    // fused stages: one trace kernel, then the update inside each RHS
    if ((st = ensure_stage(c)) != FR_OK) return st;
    st = cuda_status(acmhd::launch_trace(c, U, c->trace, s), "trace kernel");
    for (int stage = 0; stage < 4 && st == FR_OK; ++stage) {
      acmhd::StageArgs a = {};
      a.ct = stage_coef(c, stage, dtau, false);
      st = fused_stage(c, stage, U, a, s);
    }
    return st;
  }
  for (int stage = 0; stage < 4; ++stage) {
    const void* in = stage == 0 ? U : c->rk_stage;
    if ((st = fr_rhs(c, in, c->rk_k, stream)) != FR_OK) return st;
    st = cuda_status(acmhd::launch_rk_stage(c, stage, dtau, U, s), "rk update");
    if (st != FR_OK) return st;
  }
  return FR_OK;
}

int fr_pseudo_solve(fr_ctx* c, void* U, double* V, const double* Vn, const double* Vnm1,
                    double dt, int bdf_order, double dtau, double tol, int max_iter,
                    int check_every, double stall, int* iters, double* res, void* stream) {
  if (!c || bad_state_ptr(U) || bad_state_ptr(V) || bad_state_ptr(Vn)) return FR_EINVAL;
  if (bdf_order != 1 && bdf_order != 2) return FR_EINVAL;
  if (bdf_order == 2 && bad_state_ptr(Vnm1)) return FR_EINVAL;
  if (!(dt > 0.0) || !std::isfinite(dt) || !(dtau > 0.0) || !std::isfinite(dtau) ||
      !(tol >= 0.0) || max_iter < 0 || check_every < 1 || !(stall >= 0.0))
    return FR_EINVAL;
  int st = ensure_rk(c);
  if (st == FR_OK) st = ensure_dual(c);
  if (st != FR_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // BDF coefficients: dV/dt ~ (a0 V + a1 V^n + a2 V^{n-1}) / dt
  const double a0 = bdf_order == 1 ? 1.0 : 1.5;
  const double a1 = bdf_order == 1 ? -1.0 : -2.0;
  const double a2 = bdf_order == 1 ? 0.0 : 0.5;
  st = cuda_status(acmhd::launch_bdf_const(c, -a1 / dt, -a2 / dt, Vn, bdf_order == 2 ? Vnm1 : Vn,
                                           c->dual_c, s),
                   "bdf source");
  if (st == FR_OK) st = cuda_status(acmhd::launch_sync_velocity(c, V, U, s), "velocity sync");
  if (st != FR_OK) return st;
  const double count = (double)c->dim * c->npts * c->ne;
  // fused stages: the RK4 combination, the FP64 velocity rows and the
  // residual partials run inside the volume kernel
  const bool fused = use_fused_stage(c);
  acmhd::StageArgs sa = {};
  sa.dual = 1;
  sa.a0dt = a0 / dt;
  sa.V = V;
  sa.Vs = c->dual_vs;
  sa.Vacc = c->dual_vacc;
  sa.C = c->dual_c;
  if (fused) {
    if ((st = ensure_stage(c)) != FR_OK) return st;
    st = cuda_status(acmhd::launch_trace(c, U, c->trace, s), "trace kernel");
    if (st != FR_OK) return st;
  }
  auto stage_step = [&](int stage) -> int {
    if (fused) {
      acmhd::StageArgs a = sa;
      a.c = stage == 2 ? dtau : (stage == 3 ? dtau / 6.0 : 0.5 * dtau);
      a.ct = stage_coef(c, stage, dtau, true);
      return fused_stage(c, stage, U, a, s);
    }
    int r = fr_rhs(c, stage == 0 ? U : c->rk_stage, c->rk_k, stream);
    if (r != FR_OK) return r;
    return cuda_status(acmhd::launch_dual_stage(c, stage, dtau, a0 / dt, U, V, c->dual_c,
                                                c->dual_partial, s),
                       "dual stage");
  };
  double last = NAN, prev = INFINITY;
  bool converged = false;
  int it = 0;
  for (;;) {
    if ((st = stage_step(0)) != FR_OK) return st;
    if (it % check_every == 0 || it == max_iter) {
      st = cuda_status(
          fused ? acmhd::launch_norm_final(c, c->stage_partial, acmhd::stage_blocks(c), count,
                                           c->dual_res, s)
                : acmhd::launch_norm_final(c, c->dual_partial, acmhd::dual_norm_blocks(c), count,
                                           c->dual_res, s),
          "residual norm");
      if (st == FR_OK)
        st = cuda_status(cudaMemcpyAsync(&last, c->dual_res, sizeof(double),
                                         cudaMemcpyDeviceToHost, s),
                         "read residual");
      if (st == FR_OK) st = cuda_status(cudaStreamSynchronize(s), "stream synchronize");
      if (st != FR_OK) return st;
      if (!std::isfinite(last)) {
        if (iters) *iters = it;
        if (res) *res = last;
        return FR_ENONFINITE;
      }
      if (last < tol) {
        converged = true;
        break;
      }
      // stalled: the residual no longer drops by the factor `stall` per check
      if (stall > 0.0 && it > 0 && last > stall * prev) break;
      prev = last;
    }
    if (it == max_iter) break;
    for (int stage = 1; stage < 4; ++stage)
      if ((st = stage_step(stage)) != FR_OK) return st;
    ++it;
  }
  if (iters) *iters = it;
  if (res) *res = last;
  return converged ? FR_OK : FR_ENOCONV;
}

int fr_dual_init(fr_ctx* c, const void* U, void* stream) {
  if (!c || bad_state_ptr(U)) return FR_EINVAL;
  int st = ensure_history(c);
  if (st != FR_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t n = (size_t)c->nv * c->npts * c->stride;
  const size_t vel0 = (size_t)c->npts * c->stride;
  c->hist_head = 0;
  st = cuda_status(acmhd::launch_combine3(c, c->precision, n, 1.0, 0.0, 0.0, U, nullptr, nullptr,
                                          c->hist_u[0], s),
                   "history");
  // FP64 velocity level from the state's velocity rows
  if (st == FR_OK)
    st = cuda_status(acmhd::launch_widen_velocity(c, U, c->hist_v[0], s), "history");
  if (st != FR_OK) return st;
  c->hist_levels = 1;
  return FR_OK;
}

// Residual of a candidate initial guess (U, V) of the pseudo iteration:
// one RHS and the velocity RMS of R_tau, as the first RK stage computes it.
int guess_residual(fr_ctx* c, void* U, double* V, const double* Vn, const double* Vnm1, double dt,
                   int order, double* res, cudaStream_t s) {
  int st = ensure_rk(c);
  if (st == FR_OK) st = ensure_dual(c);
  if (st != FR_OK) return st;
  const double a0 = order == 1 ? 1.0 : 1.5, a1 = order == 1 ? -1.0 : -2.0;
  const double a2 = order == 1 ? 0.0 : 0.5;
  st = cuda_status(acmhd::launch_bdf_const(c, -a1 / dt, -a2 / dt, Vn, order == 2 ? Vnm1 : Vn,
                                           c->dual_c, s), "bdf source");
  if (st == FR_OK) st = cuda_status(acmhd::launch_sync_velocity(c, V, U, s), "velocity sync");
  if (st == FR_OK) st = fr_rhs(c, U, c->rk_k, s);
  if (st == FR_OK)
    st = cuda_status(acmhd::launch_dual_stage(c, 0, 1.0, a0 / dt, U, V, c->dual_c,
                                              c->dual_partial, s), "guess residual");
  if (st == FR_OK)
    st = cuda_status(acmhd::launch_norm_final(c, c->dual_partial, acmhd::dual_norm_blocks(c),
                                              (double)c->dim * c->npts * c->ne, c->dual_res, s),
                     "guess residual");
  if (st == FR_OK)
    st = cuda_status(cudaMemcpyAsync(res, c->dual_res, sizeof(double), cudaMemcpyDeviceToHost, s),
                     "guess residual");
  if (st == FR_OK) st = cuda_status(cudaStreamSynchronize(s), "stream synchronize");
  return st;
}

int fr_dual_step(fr_ctx* c, void* U, const fr_dual_opts* o, fr_dual_stats* out, void* stream) {
  if (!c || bad_state_ptr(U) || !o || c->hist_levels < 1) return FR_EINVAL;
  if (o->guess != FR_GUESS_PREVIOUS && o->guess != FR_GUESS_EXTRAPOLATE &&
      o->guess != FR_GUESS_MLP)
    return FR_EINVAL;
  if (o->guess == FR_GUESS_MLP && !o->mlp) return FR_EINVAL;
  fr_ctx* rf = o->refine;
  if (rf) {
    // the refinement context must be the FP64 twin of this one
    if (rf->precision != FR_F64 || rf->dim != c->dim || rf->order != c->order ||
        rf->ne != c->ne || rf->stride != c->stride || rf->correction != c->correction ||
        rf->zeta != c->zeta || rf->nu != c->nu || rf->t_r != c->t_r ||
        std::memcmp(rf->mesh.n, c->mesh.n, sizeof(c->mesh.n)) != 0 ||
        bad_state_ptr(o->U_refine) || !(o->tol_switch >= 0.0))
      return FR_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int L = c->hist_levels < 3 ? c->hist_levels : 3;  // levels used by the guess
  const int h0 = c->hist_head;
  const int h1 = acmhd::hist_slot(h0, 1), h2 = acmhd::hist_slot(h0, 2);  // n, n-1, n-2
  const size_t n = (size_t)c->nv * c->npts * c->stride;
  const size_t nv = vel_doubles(c);
  // initial guess of the new level: the previous level, or the polynomial
  // extrapolation through the stored levels (linear with two, quadratic with
  // three: 3 U^n - 3 U^{n-1} + U^{n-2})
  const bool extrap = o->guess != FR_GUESS_PREVIOUS;
  double w0 = 1.0, w1 = 0.0, w2 = 0.0;
  if (extrap && L == 2) w0 = 2.0, w1 = -1.0;
  if (extrap && L == 3) w0 = 3.0, w1 = -3.0, w2 = 1.0;
  int st = cuda_status(acmhd::launch_combine3(c, c->precision, n, w0, w1, w2, c->hist_u[h0],
                                              c->hist_u[h1], c->hist_u[h2], U, s),
                       "initial guess");
  if (st == FR_OK)
    st = cuda_status(acmhd::launch_combine3(c, FR_F64, nv, w0, w1, w2, c->hist_v[h0],
                                            c->hist_v[h1], c->hist_v[h2], c->dual_v, s),
                     "initial guess");
  if (st != FR_OK) return st;
  const int order = L >= 2 ? 2 : 1;
  fr_dual_stats stats = {0, 0, NAN, NAN, extrap ? FR_GUESS_EXTRAPOLATE : FR_GUESS_PREVIOUS,
                         {NAN, NAN}, 0.0, NAN};
  if (o->guess == FR_GUESS_MLP && L == 3) {
    // the network's guess competes with the extrapolation on the residual,
    // and so does the point of the segment between them where the
    // linearised residual is least
    const int nb = acmhd::dual_norm_blocks(c);
    if ((st = alloc_zeroed(&c->guess_u, c->bytes_state, "guess")) != FR_OK) return st;
    if ((st = alloc_zeroed((void**)&c->guess_v, nv * sizeof(double), "guess")) != FR_OK) return st;
    if ((st = alloc_zeroed((void**)&c->guess_r0, nv * sizeof(double), "guess")) != FR_OK) return st;
    if ((st = alloc_zeroed((void**)&c->guess_dots, (2 * (size_t)nb + 2) * sizeof(double),
                           "guess")) != FR_OK)
      return st;
    // the guess of this context's next level, from this context's history
    if ((st = fr_mlp_predict_for(o->mlp, c, c->guess_u, c->guess_v, stream)) != FR_OK) return st;
    st = guess_residual(c, U, c->dual_v, c->hist_v[h0], c->hist_v[h1], o->dt, order,
                        &stats.res_guess[0], s);
    // stage 0 of the residual evaluation leaves the velocity residual in dual_vacc
    if (st == FR_OK)
      st = cuda_status(cudaMemcpyAsync(c->guess_r0, c->dual_vacc, nv * sizeof(double),
                                       cudaMemcpyDeviceToDevice, s), "guess");
    if (st == FR_OK)
      st = guess_residual(c, c->guess_u, c->guess_v, c->hist_v[h0], c->hist_v[h1], o->dt, order,
                          &stats.res_guess[1], s);
    double dots[2] = {0.0, 0.0};
    if (st == FR_OK)
      st = cuda_status(acmhd::launch_pair_dots(c, c->guess_r0, c->dual_vacc, c->guess_dots,
                                               c->guess_dots + 2 * nb, s), "guess");
    if (st == FR_OK)
      st = cuda_status(cudaMemcpyAsync(dots, c->guess_dots + 2 * nb, sizeof(dots),
                                       cudaMemcpyDeviceToHost, s), "guess");
    if (st == FR_OK) st = cuda_status(cudaStreamSynchronize(s), "guess");
    if (st != FR_OK) return st;
    // r(alpha) ~ r0 + alpha (r1 - r0): least at alpha = -<r0, r1 - r0> / |r1 - r0|^2
    double alpha = dots[1] > 0.0 ? -dots[0] / dots[1] : 0.0;
    alpha = std::isfinite(alpha) ? (alpha < 0.0 ? 0.0 : (alpha > 1.0 ? 1.0 : alpha)) : 0.0;
    double best = stats.res_guess[0] <= stats.res_guess[1] ? stats.res_guess[0]
                                                           : stats.res_guess[1];
    double weight = stats.res_guess[1] < stats.res_guess[0] ? 1.0 : 0.0;
    if (alpha > 0.0 && alpha < 1.0) {
      // the blend (1 - alpha) extrapolation + alpha network, in guess_u / guess_v
      st = cuda_status(acmhd::launch_combine3(c, c->precision, n, 1.0 - alpha, alpha, 0.0, U,
                                              c->guess_u, nullptr, c->guess_u, s), "guess");
      if (st == FR_OK)
        st = cuda_status(acmhd::launch_combine3(c, FR_F64, nv, 1.0 - alpha, alpha, 0.0,
                                                c->dual_v, c->guess_v, nullptr, c->guess_v, s),
                         "guess");
      double res_a = NAN;
      if (st == FR_OK)
        st = guess_residual(c, c->guess_u, c->guess_v, c->hist_v[h0], c->hist_v[h1], o->dt,
                            order, &res_a, s);
      if (st != FR_OK) return st;
      stats.res_blend = res_a;
      if (res_a < best) {
        best = res_a;
        weight = alpha;
      } else if (weight == 1.0) {
        // the blend lost to the network's own guess, which guess_u no longer holds
        if ((st = fr_mlp_predict_for(o->mlp, c, c->guess_u, c->guess_v, stream)) != FR_OK)
          return st;
      }
    }
    stats.mlp_weight = weight;
    if (weight > 0.0) {
      stats.guess_used = FR_GUESS_MLP;
      st = cuda_status(cudaMemcpyAsync(U, c->guess_u, c->bytes_state, cudaMemcpyDeviceToDevice, s),
                       "guess");
      if (st == FR_OK)
        st = cuda_status(cudaMemcpyAsync(c->dual_v, c->guess_v, nv * sizeof(double),
                                         cudaMemcpyDeviceToDevice, s), "guess");
      if (st != FR_OK) return st;
    }
  }
  // iterations in this context's precision; with a refinement context they
  // stop at tol_switch or when the residual stalls
  const double tol1 = rf ? (o->tol > o->tol_switch ? o->tol : o->tol_switch) : o->tol;
  int solve =
      o->pmg ? fr_pmg_solve(o->pmg, U, c->dual_v, c->hist_v[h0], c->hist_v[h1], o->dt, order,
                            o->dtau, tol1, o->max_iter, rf ? 0.99 : 0.0, &stats.iters, &stats.res,
                            stream)
             : fr_pseudo_solve(c, U, c->dual_v, c->hist_v[h0], c->hist_v[h1], o->dt, order,
                               o->dtau, tol1, o->max_iter, o->check_every, rf ? 0.99 : 0.0,
                               &stats.iters, &stats.res, stream);
  if (solve != FR_OK && solve != FR_ENOCONV) return solve;
  stats.res_switch = stats.res;
  if (rf && !(stats.res < o->tol) && stats.iters < o->max_iter) {
    st = cuda_status(acmhd::launch_convert(c, n, c->precision, U, FR_F64, o->U_refine, s),
                     "widen state");
    if (st != FR_OK) return st;
    solve = o->refine_pmg
                ? fr_pmg_solve(o->refine_pmg, o->U_refine, c->dual_v, c->hist_v[h0],
                               c->hist_v[h1], o->dt, order, o->dtau, o->tol,
                               o->max_iter - stats.iters, 0.0, &stats.iters_refine, &stats.res,
                               stream)
                : fr_pseudo_solve(rf, o->U_refine, c->dual_v, c->hist_v[h0], c->hist_v[h1],
                                  o->dt, order, o->dtau, o->tol, o->max_iter - stats.iters,
                                  o->check_every, 0.0, &stats.iters_refine, &stats.res, stream);
    if (solve != FR_OK && solve != FR_ENOCONV) return solve;
    st = cuda_status(acmhd::launch_convert(c, n, FR_F64, o->U_refine, c->precision, U, s),
                     "narrow state");
    if (st != FR_OK) return st;
  }
  if (out) *out = stats;
  // the new level replaces level n-3 in the ring
  const int hn = (h0 + 1) % 4;
  st = cuda_status(acmhd::launch_combine3(c, c->precision, n, 1.0, 0.0, 0.0, U, nullptr, nullptr,
                                          c->hist_u[hn], s),
                   "history");
  if (st == FR_OK)
    st = cuda_status(cudaMemcpyAsync(c->hist_v[hn], c->dual_v, nv * sizeof(double),
                                     cudaMemcpyDeviceToDevice, s),
                     "history");
  if (st != FR_OK) return st;
  c->hist_head = hn;
  c->hist_levels = c->hist_levels < 4 ? c->hist_levels + 1 : 4;
  return solve;
}

int fr_dual_copy(fr_ctx* dst, const fr_ctx* src, void* stream) {
  if (!dst || !src || dst == src || src->hist_levels < 1 || dst->precision != src->precision ||
      dst->dim != src->dim || dst->order != src->order || dst->ne != src->ne ||
      dst->stride != src->stride)
    return FR_EINVAL;
  int st = ensure_history(dst);
  if (st != FR_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < 4 && st == FR_OK; ++i) {
    st = cuda_status(cudaMemcpyAsync(dst->hist_u[i], src->hist_u[i], src->bytes_state,
                                     cudaMemcpyDeviceToDevice, s), "copy history");
    if (st == FR_OK)
      st = cuda_status(cudaMemcpyAsync(dst->hist_v[i], src->hist_v[i],
                                       vel_doubles(src) * sizeof(double),
                                       cudaMemcpyDeviceToDevice, s), "copy history");
  }
  if (st != FR_OK) return st;
  dst->hist_head = src->hist_head;
  dst->hist_levels = src->hist_levels;
  return FR_OK;
}

int fr_dual_velocity(const fr_ctx* c, double* V, void* stream) {
  if (!c || bad_state_ptr(V) || c->hist_levels < 1) return FR_EINVAL;
  return cuda_status(cudaMemcpyAsync(V, c->hist_v[c->hist_head], vel_doubles(c) * sizeof(double),
                                     cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream)),
                     "copy velocity");
}

int fr_check(fr_ctx* c, void* stream) {
  if (!c) return FR_EINVAL;
  int st = cuda_status(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)),
                       "stream synchronize");
  if (st == FR_OK) st = cuda_status(cudaGetLastError(), "asynchronous error");
  return st;
}

const char* fr_strerror(int status) {
  switch (status) {
    case FR_OK: return "success";
    case FR_EINVAL: return "invalid argument";
    case FR_ECUDA: return "CUDA error";
    case FR_ENOCONV: return "pseudo-time iteration did not converge";
    case FR_ENONFINITE: return "non-finite residual";
    case FR_ENOMEM: return "out of memory";
    default: return "unknown status";
  }
}

const char* fr_last_error(void) { return g_last_error; }

}  // extern "C"
