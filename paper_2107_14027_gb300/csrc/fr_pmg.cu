// P-multigrid pseudo solver of one dual time step (Sec. 5: the dual time
// stepping of the Taylor-Green runs accelerates its pseudo-iterations by
// P-multigrid, cycling through the orders p .. 1 of the same mesh with the
// pseudo step enlarged on the lower orders).  Full approximation scheme;
// the kernels are in k_pmg.cu, the finest level's smoother is the dual-time
// RK4 stage of k_dual.cu (FP64 velocity master, BDF constant, residual).
//
// Level q < p is an internal context of order q on the finest level's mesh,
// parameters, precision and correction, with four state buffers: U (its
// iterate), U0 (the restricted state it started from), g (its FAS forcing)
// and r (restricted residual / scratch).  All levels share the element
// stride, so the transfer kernels index one layout.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "fr_pmg.h"

struct fr_pmg {
  fr_ctx* fine;
  int pmin;
  fr_ctx* lev[acmhd::kMaxM];
  void* U[acmhd::kMaxM];
  void* U0[acmhd::kMaxM];
  void* g[acmhd::kMaxM];
  void* r[acmhd::kMaxM];   // index p: the finest level's residual
  acmhd::PmgTransferPair tr[acmhd::kMaxM];  // tr[q]: order q <-> q - 1
  int nsched;
  int sorder[64];
  int siters[64];
  double factor[acmhd::kMaxM];
  int implicit;
  // Anderson mixing over the cycles: memory aa_m (0: off); ring of aa_m + 1
  // (G, F) pairs of the finest state (rows other than the velocity in the
  // context precision, velocity FP64); inner products of the F's on the host
  int aa_m;
  void* aa_xu;
  double* aa_xv;
  void* aa_gu[acmhd::kAaMax];
  double* aa_gv[acmhd::kAaMax];
  void* aa_fu[acmhd::kAaMax];
  double* aa_fv[acmhd::kAaMax];
  double* aa_partial;
  double* aa_dots;
  double gram[acmhd::kAaMax][acmhd::kAaMax];
};

namespace {

using acmhd::status_of;

// l_i(x) through the nodes (product formula)
double lagrange(const double* nodes, int m, int i, double x) {
  double v = 1.0;
  for (int q = 0; q < m; ++q)
    if (q != i) v *= (x - nodes[q]) / (nodes[i] - nodes[q]);
  return v;
}

bool build_transfer(int order, acmhd::PmgTransferPair* out) {
  acmhd::Ops1D f, c;
  if (!acmhd::build_ops1d(order, FR_CORR_DG, &f) || !acmhd::build_ops1d(order - 1, FR_CORR_DG, &c))
    return false;
  std::memset(out, 0, sizeof(*out));
  for (int k = 0; k < f.m; ++k)
    for (int i = 0; i < c.m; ++i) {
      const double l = lagrange(c.xi, c.m, i, f.xi[k]);
      const double ir = f.w[k] * l / c.w[i];
      out->d.Ip[k][i] = l;
      out->d.Ir[i][k] = ir;
      out->f.Ip[k][i] = static_cast<float>(l);
      out->f.Ir[i][k] = static_cast<float>(ir);
    }
  return true;
}

int alloc(void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return status_of(e, "pmg allocation");
  }
  return status_of(cudaMemset(*p, 0, bytes), "pmg allocation");
}

// the paper's cycle shape for order p: one iteration per order on the way
// down, `bottom` on the coarsest, one per order on the way up, `top` on p
void default_schedule(fr_pmg* m, int p) {
  int n = 0;
  for (int q = p; q > m->pmin; --q) m->sorder[n] = q, m->siters[n++] = 1;
  m->sorder[n] = m->pmin, m->siters[n++] = 4;
  for (int q = m->pmin + 1; q < p; ++q) m->sorder[n] = q, m->siters[n++] = 1;
  m->sorder[n] = p, m->siters[n++] = 7;
  m->nsched = n;
}

}  // namespace

extern "C" {

int fr_pmg_create(fr_ctx* c, int coarsest_order, fr_pmg** out) {
  if (!c || !out || coarsest_order < 1 || coarsest_order > c->order) return FR_EINVAL;
  fr_pmg* m = new (std::nothrow) fr_pmg;
  if (!m) return FR_ENOMEM;
  std::memset(m, 0, sizeof(*m));
  m->fine = c;
  m->pmin = coarsest_order;
  m->implicit = 1;
  const int p = c->order;
  for (int q = 0; q <= p; ++q) m->factor[q] = std::pow(1.75, p - q);
  int st = FR_OK;
  for (int q = m->pmin; q < p && st == FR_OK; ++q) {
    st = fr_create(&c->mesh, q, c->nv, c->zeta, c->nu, c->t_r, c->df64 ? FR_DF64 : c->precision,
                   c->correction, &m->lev[q]);
    if (st == FR_OK) st = acmhd::ensure_rk_registers(m->lev[q]);
    const size_t b = st == FR_OK ? m->lev[q]->bytes_state : 0;
    if (st == FR_OK) st = alloc(&m->U[q], b);
    if (st == FR_OK) st = alloc(&m->U0[q], b);
    if (st == FR_OK) st = alloc(&m->g[q], b);
    if (st == FR_OK) st = alloc(&m->r[q], b);
  }
  if (st == FR_OK && p > m->pmin) st = alloc(&m->r[p], c->bytes_state);
  for (int q = m->pmin + 1; q <= p && st == FR_OK; ++q)
    if (!build_transfer(q, &m->tr[q])) st = FR_EINVAL;
  if (st != FR_OK) {
    fr_pmg_destroy(m);
    return st;
  }
  default_schedule(m, p);
  *out = m;
  return FR_OK;
}

static void free_anderson(fr_pmg* m) {
  void* bufs[] = {m->aa_xu, m->aa_xv, m->aa_partial, m->aa_dots};
  for (void* b : bufs)
    if (b) cudaFree(b);
  for (int j = 0; j < acmhd::kAaMax; ++j)
    for (void* b : {m->aa_gu[j], (void*)m->aa_gv[j], m->aa_fu[j], (void*)m->aa_fv[j]})
      if (b) cudaFree(b);
  m->aa_xu = nullptr;
  m->aa_xv = m->aa_partial = m->aa_dots = nullptr;
  for (int j = 0; j < acmhd::kAaMax; ++j)
    m->aa_gu[j] = m->aa_fu[j] = nullptr, m->aa_gv[j] = m->aa_fv[j] = nullptr;
  m->aa_m = 0;
}

void fr_pmg_destroy(fr_pmg* m) {
  if (!m) return;
  cudaDeviceSynchronize();
  free_anderson(m);
  for (int q = 0; q < acmhd::kMaxM; ++q) {
    for (void* b : {m->U[q], m->U0[q], m->g[q], m->r[q]})
      if (b) cudaFree(b);
    if (m->lev[q]) fr_destroy(m->lev[q]);
  }
  delete m;
}

int fr_pmg_set_cycle(fr_pmg* m, int n, const int* orders, const int* iters) {
  if (!m || n < 1 || n > 64 || !orders || !iters) return FR_EINVAL;
  const int p = m->fine->order;
  if (orders[0] != p || orders[n - 1] != p || iters[0] < 1) return FR_EINVAL;
  for (int i = 0; i < n; ++i) {
    if (orders[i] < m->pmin || orders[i] > p || iters[i] < 0) return FR_EINVAL;
    if (i > 0 && std::abs(orders[i] - orders[i - 1]) > 1) return FR_EINVAL;
  }
  for (int i = 0; i < n; ++i) m->sorder[i] = orders[i], m->siters[i] = iters[i];
  m->nsched = n;
  return FR_OK;
}

int fr_pmg_set_anderson(fr_pmg* m, int memory) {
  if (!m || memory < 0 || memory >= acmhd::kAaMax) return FR_EINVAL;
  cudaDeviceSynchronize();
  free_anderson(m);
  if (memory == 0) return FR_OK;
  const fr_ctx* c = m->fine;
  const size_t vb = (size_t)c->dim * c->npts * c->stride * sizeof(double);
  int st = alloc(&m->aa_xu, c->bytes_state);
  if (st == FR_OK) st = alloc((void**)&m->aa_xv, vb);
  for (int j = 0; j <= memory && st == FR_OK; ++j) {
    st = alloc(&m->aa_gu[j], c->bytes_state);
    if (st == FR_OK) st = alloc((void**)&m->aa_gv[j], vb);
    if (st == FR_OK) st = alloc(&m->aa_fu[j], c->bytes_state);
    if (st == FR_OK) st = alloc((void**)&m->aa_fv[j], vb);
  }
  if (st == FR_OK)
    st = alloc((void**)&m->aa_partial,
               (size_t)acmhd::kAaMax * acmhd::aa_dot_blocks(c) * sizeof(double));
  if (st == FR_OK) st = alloc((void**)&m->aa_dots, acmhd::kAaMax * sizeof(double));
  if (st != FR_OK) {
    free_anderson(m);
    return st;
  }
  m->aa_m = memory;
  return FR_OK;
}

int fr_pmg_set_dtau(fr_pmg* m, const double* factor, int implicit) {
  if (!m) return FR_EINVAL;
  const int p = m->fine->order;
  if (factor) {
    for (int q = m->pmin; q <= p; ++q)
      if (!(factor[q] > 0.0) || !std::isfinite(factor[q])) return FR_EINVAL;
    for (int q = m->pmin; q <= p; ++q) m->factor[q] = factor[q];
  }
  m->implicit = implicit ? 1 : 0;
  return FR_OK;
}

}  // extern "C"

namespace {

struct Solve {
  fr_pmg* m;
  fr_ctx* c;
  void* U;
  double* V;
  double a0dt;
  double dtau;
  cudaStream_t s;
};

void scaling(const Solve& S, double dtq, double* dV, double* dA) {
  *dV = S.m->implicit ? 1.0 / (1.0 + dtq * S.a0dt) : 1.0;
  *dA = S.m->implicit ? 1.0 / (1.0 + dtq / S.c->t_r) : 1.0;
}

// one RK4 stage of the finest level (dual-time stage kernel, FP64 velocity)
int fine_stage(Solve& S, int stage, double dtq) {
  fr_ctx* c = S.c;
  int st = fr_rhs(c, stage == 0 ? S.U : c->rk_stage, c->rk_k, S.s);
  if (st != FR_OK) return st;
  double dV, dA;
  scaling(S, dtq, &dV, &dA);
  return status_of(acmhd::launch_dual_stage(c, stage, dtq, S.a0dt, S.U, S.V, c->dual_c,
                                            c->dual_partial, S.s, dV, dA),
                   "pmg fine stage");
}

int coarse_iteration(Solve& S, int q, double dtq) {
  fr_ctx* l = S.m->lev[q];
  double dV, dA;
  scaling(S, dtq, &dV, &dA);
  for (int stage = 0; stage < 4; ++stage) {
    int st = fr_rhs(l, stage == 0 ? S.m->U[q] : l->rk_stage, l->rk_k, S.s);
    if (st == FR_OK)
      st = status_of(acmhd::launch_pmg_coarse_stage(l, stage, dtq, S.a0dt, dV, dA, S.m->U[q],
                                                    S.m->g[q], S.s),
                     "pmg coarse stage");
    if (st != FR_OK) return st;
  }
  return FR_OK;
}

// from order f to the coarser q = f - 1: restrict the state and the
// residual, and form the FAS forcing of q
int down(Solve& S, int f, int q) {
  fr_pmg* m = S.m;
  const int p = S.c->order;
  fr_ctx* cf = f == p ? S.c : m->lev[f];
  void* Xf = f == p ? S.U : m->U[f];
  fr_ctx* cq = m->lev[q];
  int st = fr_rhs(cf, Xf, cf->rk_k, S.s);
  if (st != FR_OK) return st;
  cudaError_t e =
      f == p ? acmhd::launch_pmg_residual(cf, cf->rk_k, Xf, nullptr, S.V, cf->dual_c, S.a0dt,
                                          m->r[f], nullptr, S.s)
             : acmhd::launch_pmg_residual(cf, cf->rk_k, Xf, m->g[f], nullptr, nullptr, S.a0dt,
                                          m->r[f], nullptr, S.s);
  if (e == cudaSuccess) e = acmhd::launch_pmg_restrict(cf, Xf, m->U0[q], m->tr[f], S.s);
  if (e == cudaSuccess) e = acmhd::launch_pmg_restrict(cf, m->r[f], m->r[q], m->tr[f], S.s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(m->U[q], m->U0[q], cq->bytes_state, cudaMemcpyDeviceToDevice, S.s);
  if ((st = status_of(e, "pmg restriction")) != FR_OK) return st;
  if ((st = fr_rhs(cq, m->U0[q], cq->rk_k, S.s)) != FR_OK) return st;
  return status_of(acmhd::launch_pmg_forcing(cq, m->r[q], cq->rk_k, m->U0[q], S.a0dt, m->g[q],
                                             S.s),
                   "pmg forcing");
}

// from order q to the finer f = q + 1: add the prolonged correction
int up(Solve& S, int q, int f) {
  fr_pmg* m = S.m;
  const int p = S.c->order;
  fr_ctx* cf = f == p ? S.c : m->lev[f];
  return status_of(acmhd::launch_pmg_prolong(cf, m->U[q], m->U0[q], f == p ? S.U : m->U[f],
                                             f == p ? S.V : nullptr, m->tr[f], S.s),
                   "pmg prolongation");
}

// Solves (A + lambda I) x = b by Cholesky (A symmetric, n <= kAaMax);
// false if A is not positive definite to working precision.
bool cholesky_solve(int n, double A[][acmhd::kAaMax], const double* b, double* x) {
  double L[acmhd::kAaMax][acmhd::kAaMax] = {};
  double dmax = 0.0;
  for (int i = 0; i < n; ++i) dmax = std::fmax(dmax, A[i][i]);
  if (!(dmax > 0.0)) return false;
  const double lambda = 1e-13 * dmax;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j <= i; ++j) {
      double v = A[i][j] + (i == j ? lambda : 0.0);
      for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k];
      if (i == j) {
        if (!(v > 1e-15 * dmax)) return false;
        L[i][i] = std::sqrt(v);
      } else {
        L[i][j] = v / L[j][j];
      }
    }
  double y[acmhd::kAaMax];
  for (int i = 0; i < n; ++i) {
    double v = b[i];
    for (int k = 0; k < i; ++k) v -= L[i][k] * y[k];
    y[i] = v / L[i][i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double v = y[i];
    for (int k = i + 1; k < n; ++k) v -= L[k][i] * x[k];
    x[i] = v / L[i][i];
  }
  return true;
}

// Anderson step after cycle k of a solve: (U, V) holds G(x_k), aa_x* holds
// x_k.  Records (G, F), updates the inner products of the window's F's, and
// replaces (U, V) by G(x_k) - dG gamma, gamma the least-squares solution of
// dF gamma = f_k (normal equations; oldest columns dropped if singular).
int anderson_step(fr_pmg* m, void* U, double* V, int k, cudaStream_t s) {
  const fr_ctx* c = m->fine;
  const int M = m->aa_m, ring = M + 1;
  const int slot = k % ring;
  int st = status_of(acmhd::launch_aa_record(c, U, V, m->aa_xu, m->aa_xv, m->aa_gu[slot],
                                             m->aa_gv[slot], m->aa_fu[slot], m->aa_fv[slot], s),
                     "anderson record");
  if (st != FR_OK) return st;
  const int w = k + 1 < ring ? k + 1 : ring;
  int slots[acmhd::kAaMax];
  for (int t = 0; t < w; ++t) slots[t] = (k - (w - 1) + t) % ring;
  acmhd::AaVectors W = {};
  W.n = w;
  for (int t = 0; t < w; ++t) W.u[t] = m->aa_fu[slots[t]], W.v[t] = m->aa_fv[slots[t]];
  double dots[acmhd::kAaMax];
  st = status_of(acmhd::launch_aa_dots(c, m->aa_fu[slot], m->aa_fv[slot], W, m->aa_partial,
                                       acmhd::aa_dot_blocks(c), m->aa_dots, s),
                 "anderson dots");
  if (st == FR_OK)
    st = status_of(cudaMemcpyAsync(dots, m->aa_dots, w * sizeof(double), cudaMemcpyDeviceToHost, s),
                   "anderson dots");
  if (st == FR_OK) st = status_of(cudaStreamSynchronize(s), "stream synchronize");
  if (st != FR_OK) return st;
  for (int t = 0; t < w; ++t) m->gram[slot][slots[t]] = m->gram[slots[t]][slot] = dots[t];
  for (int first = 0; first < w - 1; ++first) {
    const int mk = w - 1 - first;   // columns: differences of window entries first .. w-1
    auto G = [&](int a, int b) { return m->gram[slots[first + a]][slots[first + b]]; };
    double A[acmhd::kAaMax][acmhd::kAaMax], rhs[acmhd::kAaMax], gamma[acmhd::kAaMax];
    for (int a = 0; a < mk; ++a) {
      for (int b = 0; b < mk; ++b) A[a][b] = G(a + 1, b + 1) - G(a + 1, b) - G(a, b + 1) + G(a, b);
      rhs[a] = G(a + 1, mk) - G(a, mk);
    }
    if (!cholesky_solve(mk, A, rhs, gamma)) continue;
    acmhd::AaVectors Wg = {};
    Wg.n = mk + 1;
    for (int t = 0; t <= mk; ++t) {
      Wg.u[t] = m->aa_gu[slots[first + t]];
      Wg.v[t] = m->aa_gv[slots[first + t]];
      Wg.c[t] = 0.0;
    }
    Wg.c[mk] = 1.0;
    for (int a = 0; a < mk; ++a) {
      Wg.c[a + 1] -= gamma[a];
      Wg.c[a] += gamma[a];
    }
    return status_of(acmhd::launch_aa_combine(c, Wg, U, V, s), "anderson combine");
  }
  return FR_OK;   // no usable columns: keep G(x_k)
}

}  // namespace

extern "C" int fr_pmg_solve(fr_pmg* m, void* U, double* V, const double* Vn, const double* Vnm1,
                            double dt, int bdf_order, double dtau, double tol, int max_cycles,
                            double stall, int* cycles, double* res, void* stream) {
  if (!m || !U || !V || !Vn || (bdf_order != 1 && bdf_order != 2) ||
      (bdf_order == 2 && !Vnm1) || !(dt > 0.0) || !std::isfinite(dt) || !(dtau > 0.0) ||
      !std::isfinite(dtau) || !(tol >= 0.0) || max_cycles < 0 || !(stall >= 0.0))
    return FR_EINVAL;
  fr_ctx* c = m->fine;
  int st = acmhd::ensure_rk_registers(c);
  if (st == FR_OK) st = acmhd::ensure_dual_registers(c);
  if (st != FR_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const double a0 = bdf_order == 1 ? 1.0 : 1.5, a1 = bdf_order == 1 ? -1.0 : -2.0;
  const double a2 = bdf_order == 1 ? 0.0 : 0.5;
  st = status_of(acmhd::launch_bdf_const(c, -a1 / dt, -a2 / dt, Vn, bdf_order == 2 ? Vnm1 : Vn,
                                         c->dual_c, s),
                 "bdf source");
  if (st == FR_OK) st = status_of(acmhd::launch_sync_velocity(c, V, U, s), "velocity sync");
  if (st != FR_OK) return st;
  Solve S{m, c, U, V, a0 / dt, dtau, s};
  const int p = c->order;
  const double count = (double)c->dim * c->npts * c->ne;
  double last = NAN, prev = INFINITY;
  bool converged = false;
  int n = 0;
  for (;;) {
    // convergence check: stage 0 of the cycle's first finest-level
    // iteration sums the squared residual of the current state
    const double dtp = dtau * m->factor[p];
    if ((st = fine_stage(S, 0, dtp)) != FR_OK) return st;
    st = status_of(acmhd::launch_norm_final(c, c->dual_partial, acmhd::dual_norm_blocks(c), count,
                                            c->dual_res, s),
                   "residual norm");
    if (st == FR_OK)
      st = status_of(cudaMemcpyAsync(&last, c->dual_res, sizeof(double), cudaMemcpyDeviceToHost, s),
                     "read residual");
    if (st == FR_OK) st = status_of(cudaStreamSynchronize(s), "stream synchronize");
    if (st != FR_OK) return st;
    if (!std::isfinite(last)) {
      if (cycles) *cycles = n;
      if (res) *res = last;
      return FR_ENONFINITE;
    }
    if (last < tol) {
      converged = true;
      break;
    }
    if (n == max_cycles || (stall > 0.0 && n > 0 && last > stall * prev)) break;
    prev = last;
    if (m->aa_m > 0) {   // keep x_k for the mixing
      st = status_of(cudaMemcpyAsync(m->aa_xu, U, c->bytes_state, cudaMemcpyDeviceToDevice, s),
                     "anderson state");
      if (st == FR_OK)
        st = status_of(cudaMemcpyAsync(m->aa_xv, V,
                                       (size_t)c->dim * c->npts * c->stride * sizeof(double),
                                       cudaMemcpyDeviceToDevice, s),
                       "anderson state");
      if (st != FR_OK) return st;
    }
    int cur = p;
    for (int i = 0; i < m->nsched && st == FR_OK; ++i) {
      const int q = m->sorder[i];
      if (q == cur - 1) st = down(S, cur, q);
      else if (q == cur + 1) st = up(S, cur, q);
      cur = q;
      const double dtq = dtau * m->factor[q];
      for (int k = 0; k < m->siters[i] && st == FR_OK; ++k) {
        if (q == p) {
          for (int stage = (i == 0 && k == 0) ? 1 : 0; stage < 4 && st == FR_OK; ++stage)
            st = fine_stage(S, stage, dtq);
        } else {
          st = coarse_iteration(S, q, dtq);
        }
      }
    }
    if (st != FR_OK) return st;
    if (m->aa_m > 0 && (st = anderson_step(m, U, V, n, s)) != FR_OK) return st;
    ++n;
  }
  if (cycles) *cycles = n;
  if (res) *res = last;
  return converged ? FR_OK : FR_ENOCONV;
}
