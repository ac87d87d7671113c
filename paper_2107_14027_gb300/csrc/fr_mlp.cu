// Per-element MLP that predicts the initial guess of a physical time step.
// The paper has no learned component; this is the build's own extension of
// the dual time stepping of Sec. 5.
//
//   features  x_e = [U^n / s0, (U^n - U^{n-1}) / s1, (U^n - 2U^{n-1} + U^{n-2}) / s2]
//             per element e (each block flattened as (variable, point); s0,
//             s1, s2 per-variable RMS of the blocks, fixed at the first
//             collection), K = 3 n_v (p+1)^d;
//   network   h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = W3 h2 + b3;
//   guess     U^{n+1} ~ 3U^n - 3U^{n-1} + U^{n-2} + t (.) y, t the
//             per-variable RMS of the collected corrections.
// Training: full-batch Adam on the MSE of the normalised correction over
// element samples collected from the solver's own physical steps.  BF16
// operands on the tensor cores, FP32 accumulation and FP32 master weights.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "fr_mlp.h"

struct fr_mlp {
  fr_ctx* ctx;
  int K, H, NO, cap, n;
  float* p[6];
  __nv_bfloat16* pb[6];
  float* g[6];
  float* m[6];
  float* v[6];
  size_t cnt[6];
  int adam_t;
  int n_val;             // the newest n_val collected samples: validation only
  float wd;              // decoupled weight decay of Adam (weights, not biases)
  double* val_loss;      // [1]
  float* in_scale;       // [3 nv] RMS of the feature blocks
  float* in_scale_inv;   // [3 nv]
  float* out_scale;      // [nv]
  float* out_scale_inv;  // [nv]
  int scales_set;
  __nv_bfloat16* Xs;     // [K x cap]
  float* Ts;             // [NO x cap] raw corrections
  int* elems;            // [cap]
  float *Z1, *Z2, *Y, *dY, *dZ2, *dZ1;
  __nv_bfloat16 *H1b, *H2b, *dYb, *dZ2b, *dZ1b;
  double* partial;
  double* loss;
  int nparts;
  __nv_bfloat16* Xi;     // inference features [K x stride]
  __nv_bfloat16 *Hi1, *Hi2;
  float* Yc;             // [NO x stride] scaled corrections
  __nv_bfloat16* w1p;    // [H x Kp] BF16 W1 with rows padded to a multiple of 8
  int Kp;                //   values (16 bytes), the tensor-memory GEMM's TMA pitch
  int out_degree;        // corrections projected onto degree <= out_degree (-1: off)
  acmhd::LineProj proj;  //   the 1-D projector of that degree
};

namespace {

using acmhd::GemmArgs;

int st_of(cudaError_t e, const char* where) {
  if (e == cudaSuccess) return FR_OK;
  char msg[200];
  std::snprintf(msg, sizeof(msg), "%s: %s", where, cudaGetErrorString(e));
  acmhd::set_last_error(msg);
  return e == cudaErrorMemoryAllocation ? FR_ENOMEM : FR_ECUDA;
}

template <typename P>
int dalloc(P** p, size_t count) {
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(P));
  if (e != cudaSuccess) {
    *p = nullptr;
    return st_of(e, "mlp allocation");
  }
  return st_of(cudaMemset(*p, 0, count * sizeof(P)), "mlp allocation");
}

// splitmix64: a counter-based generator for the weight initialisation
uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
double uniform01(uint64_t& s) { return (splitmix64(s) >> 11) * (1.0 / 9007199254740992.0); }

template <typename T>
acmhd::MlpHist<T> hist_view(const fr_ctx* c, const int lev[4]) {
  acmhd::MlpHist<T> h;
  for (int i = 0; i < 4; ++i) {
    const int slot = acmhd::hist_slot(c->hist_head, lev[i] < 0 ? 0 : lev[i]);
    h.u[i] = static_cast<const T*>(c->hist_u[slot]);
    h.v[i] = c->hist_v[slot];
  }
  h.dim = c->dim;
  h.nv = c->nv;
  h.npts = c->npts;
  h.ne = c->ne;
  h.stride = static_cast<int>(c->stride);
  return h;
}

GemmArgs gemm(int N, int M, int K, const __nv_bfloat16* A, long long lda, const __nv_bfloat16* B,
              long long ldb) {
  GemmArgs g;
  std::memset(&g, 0, sizeof(g));
  g.N = N;
  g.M = M;
  g.K = K;
  g.A = A;
  g.lda = lda;
  g.B = B;
  g.ldb = ldb;
  g.rows_per_scale = 1;
  return g;
}

// Forward pass over `cols` samples stored with leading dimension ld:
// X [K x ld] -> Z1/H1 -> Z2/H2 -> Y (FP32, optionally scaled per variable).
int forward(fr_mlp* q, const __nv_bfloat16* X, long long ld, int cols, float* Z1,
            __nv_bfloat16* H1, float* Z2, __nv_bfloat16* H2, float* Y, const float* row_scale,
            cudaStream_t s) {
  const __nv_bfloat16* W1 = q->pb[0];
  long long ldw1 = q->K;
  if (q->w1p) {
    int st = st_of(acmhd::launch_pad_rows(q->pb[0], q->H, q->K, q->w1p, q->Kp, s), "mlp pad W1");
    if (st != FR_OK) return st;
    W1 = q->w1p;
    ldw1 = q->Kp;
  }
  GemmArgs g = gemm(q->H, cols, q->K, W1, ldw1, X, ld);
  g.bias = q->p[1];
  g.C = Z1;
  g.ldc = ld;
  g.Cb = H1;
  g.ldcb = ld;
  g.relu = 1;
  int st = st_of(acmhd::launch_gemm(acmhd::GEMM_A_NK, acmhd::GEMM_B_KM, g, s), "mlp layer 1");
  if (st != FR_OK) return st;
  g = gemm(q->H, cols, q->H, q->pb[2], q->H, H1, ld);
  g.bias = q->p[3];
  g.C = Z2;
  g.ldc = ld;
  g.Cb = H2;
  g.ldcb = ld;
  g.relu = 1;
  st = st_of(acmhd::launch_gemm(acmhd::GEMM_A_NK, acmhd::GEMM_B_KM, g, s), "mlp layer 2");
  if (st != FR_OK) return st;
  g = gemm(q->NO, cols, q->H, q->pb[4], q->H, H2, ld);
  g.bias = q->p[5];
  g.C = Y;
  g.ldc = ld;
  if (row_scale) {
    g.row_scale = row_scale;
    g.rows_per_scale = q->ctx->npts;
  }
  return st_of(acmhd::launch_gemm(acmhd::GEMM_A_NK, acmhd::GEMM_B_KM, g, s), "mlp layer 3");
}

// Loss and gradients over the training samples, the collected ones except
// the newest n_val (gradients into q->g).
int loss_grad(fr_mlp* q, cudaStream_t s) {
  const int n = q->n - q->n_val;
  const long long ld = q->cap;
  int st = forward(q, q->Xs, ld, n, q->Z1, q->H1b, q->Z2, q->H2b, q->Y, nullptr, s);
  if (st != FR_OK) return st;
  // the partial sums hold sum (y - t)^2; the loss is their mean
  st = st_of(acmhd::launch_loss_grad(q->Y, q->Ts, ld, q->NO, n, q->ctx->npts, q->out_scale_inv,
                                     q->dY, q->dYb, q->partial, q->nparts, s),
             "mlp loss");
  if (st == FR_OK)
    st = st_of(acmhd::launch_sum_partials(q->partial, q->nparts, (double)q->NO * n, q->loss, s),
               "mlp loss");
  if (st != FR_OK) return st;
  // layer 3: dW3 = dY H2^T, db3 = rowsum dY, dH2 = W3^T dY (masked by Z2 > 0)
  GemmArgs g = gemm(q->NO, q->H, n, q->dYb, ld, q->H2b, ld);
  g.C = q->g[4];
  g.ldc = q->H;
  if ((st = st_of(acmhd::launch_gemm(acmhd::GEMM_A_NK, acmhd::GEMM_B_MK, g, s), "mlp dW3")))
    return st;
  if ((st = st_of(acmhd::launch_row_sum(q->dY, ld, q->NO, n, q->g[5], s), "mlp db3"))) return st;
  g = gemm(q->H, n, q->NO, q->pb[4], q->H, q->dYb, ld);
  g.mask = q->Z2;
  g.ldm = ld;
  g.C = q->dZ2;
  g.ldc = ld;
  g.Cb = q->dZ2b;
  g.ldcb = ld;
  if ((st = st_of(acmhd::launch_gemm(acmhd::GEMM_A_KN, acmhd::GEMM_B_KM, g, s), "mlp dH2")))
    return st;
  // layer 2
  g = gemm(q->H, q->H, n, q->dZ2b, ld, q->H1b, ld);
  g.C = q->g[2];
  g.ldc = q->H;
  if ((st = st_of(acmhd::launch_gemm(acmhd::GEMM_A_NK, acmhd::GEMM_B_MK, g, s), "mlp dW2")))
    return st;
  if ((st = st_of(acmhd::launch_row_sum(q->dZ2, ld, q->H, n, q->g[3], s), "mlp db2"))) return st;
  g = gemm(q->H, n, q->H, q->pb[2], q->H, q->dZ2b, ld);
  g.mask = q->Z1;
  g.ldm = ld;
  g.C = q->dZ1;
  g.ldc = ld;
  g.Cb = q->dZ1b;
  g.ldcb = ld;
  if ((st = st_of(acmhd::launch_gemm(acmhd::GEMM_A_KN, acmhd::GEMM_B_KM, g, s), "mlp dH1")))
    return st;
  // layer 1
  g = gemm(q->H, q->K, n, q->dZ1b, ld, q->Xs, ld);
  g.C = q->g[0];
  g.ldc = q->K;
  if ((st = st_of(acmhd::launch_gemm(acmhd::GEMM_A_NK, acmhd::GEMM_B_MK, g, s), "mlp dW1")))
    return st;
  return st_of(acmhd::launch_row_sum(q->dZ1, ld, q->H, n, q->g[1], s), "mlp db1");
}

// Loss of the current network on the validation samples (columns
// n - n_val .. n - 1 of the sample store) into q->val_loss.
int validation_loss(fr_mlp* q, cudaStream_t s) {
  const int n0 = q->n - q->n_val, nv = q->n_val;
  const long long ld = q->cap;
  int st = forward(q, q->Xs + n0, ld, nv, q->Z1 + n0, q->H1b + n0, q->Z2 + n0, q->H2b + n0,
                   q->Y + n0, nullptr, s);
  if (st == FR_OK)
    st = st_of(acmhd::launch_loss_grad(q->Y + n0, q->Ts + n0, ld, q->NO, nv, q->ctx->npts,
                                       q->out_scale_inv, q->dY + n0, q->dYb + n0, q->partial,
                                       q->nparts, s),
               "mlp validation loss");
  if (st == FR_OK)
    st = st_of(acmhd::launch_sum_partials(q->partial, q->nparts, (double)q->NO * nv, q->val_loss,
                                          s),
               "mlp validation loss");
  return st;
}

bool ptr16(const void* p) { return p && (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" {

int fr_mlp_create(fr_ctx* c, int hidden, int capacity, unsigned long long seed, fr_mlp** out) {
  if (!c || !out || hidden < 8 || hidden > 4096 || capacity < 1 || capacity > (1 << 22))
    return FR_EINVAL;
  fr_mlp* q = new (std::nothrow) fr_mlp;
  if (!q) return FR_ENOMEM;
  std::memset(q, 0, sizeof(*q));
  q->out_degree = -1;
  q->ctx = c;
  q->NO = c->nv * c->npts;
  q->K = 3 * q->NO;
  q->H = hidden;
  q->cap = capacity;
  q->nparts = 152 * 4;
  const size_t cnt[6] = {(size_t)q->H * q->K, (size_t)q->H, (size_t)q->H * q->H, (size_t)q->H,
                         (size_t)q->NO * q->H, (size_t)q->NO};
  const int fan_in[6] = {q->K, q->K, q->H, q->H, q->H, q->H};
  int st = FR_OK;
  std::vector<float> host;
  uint64_t rng = seed;
  for (int i = 0; i < 6 && st == FR_OK; ++i) {
    q->cnt[i] = cnt[i];
    if ((st = dalloc(&q->p[i], cnt[i])) || (st = dalloc(&q->pb[i], cnt[i])) ||
        (st = dalloc(&q->g[i], cnt[i])) || (st = dalloc(&q->m[i], cnt[i])) ||
        (st = dalloc(&q->v[i], cnt[i])))
      break;
    // weights: uniform in +-sqrt(6 / fan_in) (ReLU layers), the output layer
    // ten times smaller; biases zero
    host.assign(cnt[i], 0.0f);
    if (i % 2 == 0) {
      const double a = std::sqrt(6.0 / fan_in[i]) * (i == 4 ? 0.1 : 1.0);
      for (size_t j = 0; j < cnt[i]; ++j) host[j] = (float)((2.0 * uniform01(rng) - 1.0) * a);
    }
    st = st_of(cudaMemcpy(q->p[i], host.data(), cnt[i] * sizeof(float), cudaMemcpyHostToDevice),
               "mlp init");
    if (st == FR_OK) st = st_of(acmhd::launch_to_bf16(cnt[i], q->p[i], q->pb[i], 0), "mlp init");
  }
  const long long ld = capacity;
  if (st == FR_OK &&
      ((st = dalloc(&q->in_scale, 3 * c->nv)) || (st = dalloc(&q->in_scale_inv, 3 * c->nv)) ||
       (st = dalloc(&q->out_scale, c->nv)) || (st = dalloc(&q->out_scale_inv, c->nv)) ||
       (st = dalloc(&q->Xs, (size_t)q->K * ld)) || (st = dalloc(&q->Ts, (size_t)q->NO * ld)) ||
       (st = dalloc(&q->elems, (size_t)capacity)) || (st = dalloc(&q->Z1, (size_t)q->H * ld)) ||
       (st = dalloc(&q->Z2, (size_t)q->H * ld)) || (st = dalloc(&q->Y, (size_t)q->NO * ld)) ||
       (st = dalloc(&q->dY, (size_t)q->NO * ld)) || (st = dalloc(&q->dZ2, (size_t)q->H * ld)) ||
       (st = dalloc(&q->dZ1, (size_t)q->H * ld)) || (st = dalloc(&q->H1b, (size_t)q->H * ld)) ||
       (st = dalloc(&q->H2b, (size_t)q->H * ld)) || (st = dalloc(&q->dYb, (size_t)q->NO * ld)) ||
       (st = dalloc(&q->dZ2b, (size_t)q->H * ld)) || (st = dalloc(&q->dZ1b, (size_t)q->H * ld)) ||
       (st = dalloc(&q->partial, (size_t)q->nparts)) || (st = dalloc(&q->loss, 1)) ||
       (st = dalloc(&q->val_loss, 1))))
    ;
  q->Kp = (q->K + 7) / 8 * 8;
  if (st == FR_OK && q->Kp != q->K) st = dalloc(&q->w1p, (size_t)q->H * q->Kp);
  if (st == FR_OK) st = st_of(cudaDeviceSynchronize(), "mlp init");
  if (st != FR_OK) {
    fr_mlp_destroy(q);
    return st;
  }
  *out = q;
  return FR_OK;
}

void fr_mlp_destroy(fr_mlp* q) {
  if (!q) return;
  cudaDeviceSynchronize();
  for (int i = 0; i < 6; ++i) {
    cudaFree(q->p[i]);
    cudaFree(q->pb[i]);
    cudaFree(q->g[i]);
    cudaFree(q->m[i]);
    cudaFree(q->v[i]);
  }
  void* bufs[] = {q->in_scale, q->in_scale_inv, q->out_scale, q->out_scale_inv, q->Xs, q->Ts,
                  q->elems, q->Z1, q->Z2, q->Y, q->dY, q->dZ2, q->dZ1, q->H1b, q->H2b, q->dYb,
                  q->dZ2b, q->dZ1b, q->partial, q->loss, q->val_loss, q->Xi, q->Hi1, q->Hi2,
                  q->Yc, q->w1p};
  for (void* p : bufs)
    if (p) cudaFree(p);
  delete q;
}

int fr_mlp_info(const fr_mlp* q, int* n_in, int* hidden, int* n_out, int* n_samples,
                size_t* n_params) {
  if (!q) return FR_EINVAL;
  if (n_in) *n_in = q->K;
  if (hidden) *hidden = q->H;
  if (n_out) *n_out = q->NO;
  if (n_samples) *n_samples = q->n;
  if (n_params) {
    size_t t = 0;
    for (int i = 0; i < 6; ++i) t += q->cnt[i];
    *n_params = t;
  }
  return FR_OK;
}

int fr_mlp_params(fr_mlp* q, int which, float* host, size_t count, int set) {
  if (!q || !host || which < 0 || which > 4) return FR_EINVAL;
  if (which == 3 || which == 4) {
    // collected samples (read only): features (K x n, from BF16) or raw
    // targets (NO x n)
    const size_t rows = which == 3 ? q->K : q->NO;
    if (set || count != rows * (size_t)q->n) return FR_EINVAL;
    if (q->n == 0) return FR_OK;
    if (which == 4)
      return st_of(cudaMemcpy2D(host, q->n * sizeof(float), q->Ts, q->cap * sizeof(float),
                                q->n * sizeof(float), rows, cudaMemcpyDeviceToHost), "samples");
    std::vector<uint16_t> raw(rows * q->n);
    int st = st_of(cudaMemcpy2D(raw.data(), q->n * 2, q->Xs, q->cap * 2, q->n * 2, rows,
                                cudaMemcpyDeviceToHost), "samples");
    for (size_t i = 0; i < raw.size() && st == FR_OK; ++i) {
      const uint32_t bits = (uint32_t)raw[i] << 16;
      std::memcpy(&host[i], &bits, 4);
    }
    return st;
  }
  if (which == 2) {
    const size_t nv = q->ctx->nv;
    if (count != 4 * nv) return FR_EINVAL;
    if (set) {
      std::vector<float> inv(4 * nv);
      for (size_t i = 0; i < 4 * nv; ++i) inv[i] = host[i] > 0.0f ? 1.0f / host[i] : 1.0f;
      int st = st_of(cudaMemcpy(q->in_scale, host, 3 * nv * 4, cudaMemcpyHostToDevice), "scales");
      if (!st) st = st_of(cudaMemcpy(q->in_scale_inv, inv.data(), 3 * nv * 4, cudaMemcpyHostToDevice), "scales");
      if (!st) st = st_of(cudaMemcpy(q->out_scale, host + 3 * nv, nv * 4, cudaMemcpyHostToDevice), "scales");
      if (!st) st = st_of(cudaMemcpy(q->out_scale_inv, inv.data() + 3 * nv, nv * 4, cudaMemcpyHostToDevice), "scales");
      if (!st) q->scales_set = 1;
      return st;
    }
    int st = st_of(cudaMemcpy(host, q->in_scale, 3 * nv * 4, cudaMemcpyDeviceToHost), "scales");
    if (!st) st = st_of(cudaMemcpy(host + 3 * nv, q->out_scale, nv * 4, cudaMemcpyDeviceToHost), "scales");
    return st;
  }
  size_t total = 0;
  for (int i = 0; i < 6; ++i) total += q->cnt[i];
  if (count != total) return FR_EINVAL;
  float** src = which == 0 ? q->p : q->g;
  size_t off = 0;
  for (int i = 0; i < 6; ++i) {
    int st;
    if (set) {
      st = st_of(cudaMemcpy(src[i], host + off, q->cnt[i] * 4, cudaMemcpyHostToDevice), "params");
      if (!st && which == 0) st = st_of(acmhd::launch_to_bf16(q->cnt[i], q->p[i], q->pb[i], 0), "params");
    } else {
      st = st_of(cudaMemcpy(host + off, src[i], q->cnt[i] * 4, cudaMemcpyDeviceToHost), "params");
    }
    if (st) return st;
    off += q->cnt[i];
  }
  return st_of(cudaDeviceSynchronize(), "params");
}

int fr_mlp_collect(fr_mlp* q, int count, unsigned long long seed, int* elems_out, void* stream) {
  if (!q || count < 1) return FR_EINVAL;
  fr_ctx* c = q->ctx;
  if (c->hist_levels < 4 || q->n + count > q->cap) return FR_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // newest level is the target; the three before it are the inputs
  const int lev[4] = {1, 2, 3, 0};
  std::vector<int> el(count);
  uint64_t rng = seed;
  for (int j = 0; j < count; ++j) el[j] = (int)(splitmix64(rng) % (uint64_t)c->ne);
  if (elems_out) std::memcpy(elems_out, el.data(), count * sizeof(int));
  int st = st_of(cudaMemcpyAsync(q->elems + q->n, el.data(), count * sizeof(int),
                                 cudaMemcpyHostToDevice, s),
                 "mlp collect");
  if (st == FR_OK && !q->scales_set) {
    // feature scales from the whole mesh at the first collection
    std::vector<float> rms(3 * c->nv), inv(3 * c->nv);
    if (c->precision == FR_F32)
      st = st_of(acmhd::launch_feature_rms(hist_view<float>(c, lev), q->in_scale, s), "scales");
    else
      st = st_of(acmhd::launch_feature_rms(hist_view<double>(c, lev), q->in_scale, s), "scales");
    if (st == FR_OK)
      st = st_of(cudaMemcpyAsync(rms.data(), q->in_scale, rms.size() * 4, cudaMemcpyDeviceToHost, s),
                 "scales");
    if (st == FR_OK) st = st_of(cudaStreamSynchronize(s), "scales");
    for (size_t i = 0; i < rms.size(); ++i) inv[i] = rms[i] > 0.0f ? 1.0f / rms[i] : 1.0f;
    if (st == FR_OK)
      st = st_of(cudaMemcpyAsync(q->in_scale_inv, inv.data(), inv.size() * 4,
                                 cudaMemcpyHostToDevice, s),
                 "scales");
    if (st == FR_OK) st = st_of(cudaStreamSynchronize(s), "scales");
    q->scales_set = (st == FR_OK);
  }
  if (st != FR_OK) return st;
  const long long ld = q->cap;
  if (c->precision == FR_F32) {
    const auto h = hist_view<float>(c, lev);
    st = st_of(acmhd::launch_gather_features(h, q->elems + q->n, count, q->in_scale_inv, q->K,
                                             q->Xs + q->n, ld, s), "mlp features");
    if (!st) st = st_of(acmhd::launch_gather_targets(h, q->elems + q->n, count, q->Ts + q->n, ld, s),
                        "mlp targets");
  } else {
    const auto h = hist_view<double>(c, lev);
    st = st_of(acmhd::launch_gather_features(h, q->elems + q->n, count, q->in_scale_inv, q->K,
                                             q->Xs + q->n, ld, s), "mlp features");
    if (!st) st = st_of(acmhd::launch_gather_targets(h, q->elems + q->n, count, q->Ts + q->n, ld, s),
                        "mlp targets");
  }
  // smoothed targets: the corrections projected onto degree <= out_degree
  if (st == FR_OK && q->out_degree >= 0)
    st = st_of(acmhd::launch_project_lines(q->Ts + q->n, ld, count, c->nv, c->m, c->dim, q->proj,
                                           s),
               "mlp targets");
  if (st == FR_OK) st = st_of(cudaStreamSynchronize(s), "mlp collect");
  if (st == FR_OK) q->n += count;
  return st;
}

// Output scales from the collected corrections (first training call).
static int set_output_scales(fr_mlp* q, cudaStream_t s) {
  const int nv = q->ctx->nv;
  std::vector<float> t(nv), inv(nv);
  int st = st_of(acmhd::launch_target_rms(q->Ts, q->cap, q->n, nv, q->ctx->npts, q->out_scale, s),
                 "mlp scales");
  if (st == FR_OK)
    st = st_of(cudaMemcpyAsync(t.data(), q->out_scale, nv * 4, cudaMemcpyDeviceToHost, s), "scales");
  if (st == FR_OK) st = st_of(cudaStreamSynchronize(s), "scales");
  for (int i = 0; i < nv; ++i) inv[i] = t[i] > 0.0f ? 1.0f / t[i] : 1.0f;
  if (st == FR_OK)
    st = st_of(cudaMemcpyAsync(q->out_scale_inv, inv.data(), nv * 4, cudaMemcpyHostToDevice, s),
               "scales");
  if (st == FR_OK) st = st_of(cudaStreamSynchronize(s), "scales");
  return st;
}

int fr_mlp_set_training(fr_mlp* q, int n_val, double weight_decay) {
  if (!q || n_val < 0 || n_val > q->cap || !(weight_decay >= 0.0) || !std::isfinite(weight_decay))
    return FR_EINVAL;
  q->n_val = n_val;
  q->wd = static_cast<float>(weight_decay);
  return FR_OK;
}

int fr_mlp_validation_loss(fr_mlp* q, double* loss, void* stream) {
  if (!q || !loss || q->n_val < 1 || q->n_val >= q->n || q->adam_t == 0) return FR_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int st = validation_loss(q, s);
  double l = NAN;
  if (st == FR_OK)
    st = st_of(cudaMemcpyAsync(&l, q->val_loss, sizeof(double), cudaMemcpyDeviceToHost, s),
               "mlp validation loss");
  if (st == FR_OK) st = st_of(cudaStreamSynchronize(s), "mlp validation loss");
  *loss = l;
  return st;
}

int fr_mlp_loss_grad(fr_mlp* q, double* loss, void* stream) {
  if (!q || q->n - q->n_val < 1) return FR_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int st = FR_OK;
  if (q->adam_t == 0 && (st = set_output_scales(q, s)) != FR_OK) return st;
  if ((st = loss_grad(q, s)) != FR_OK) return st;
  double l = NAN;
  st = st_of(cudaMemcpyAsync(&l, q->loss, sizeof(double), cudaMemcpyDeviceToHost, s), "mlp loss");
  if (st == FR_OK) st = st_of(cudaStreamSynchronize(s), "mlp loss");
  if (loss) *loss = l;
  return st;
}

int fr_mlp_train(fr_mlp* q, int epochs, double lr, double* loss, void* stream) {
  if (!q || q->n - q->n_val < 1 || epochs < 0 || !(lr > 0.0) || !std::isfinite(lr))
    return FR_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int st = FR_OK;
  if (q->adam_t == 0 && (st = set_output_scales(q, s)) != FR_OK) return st;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int ep = 0; ep < epochs; ++ep) {
    if ((st = loss_grad(q, s)) != FR_OK) return st;
    ++q->adam_t;
    const float c1 = 1.0f - std::pow(b1, (float)q->adam_t);
    const float c2 = 1.0f - std::pow(b2, (float)q->adam_t);
    for (int i = 0; i < 6; ++i)
      if ((st = st_of(acmhd::launch_adam(q->cnt[i], q->p[i], q->g[i], q->m[i], q->v[i], q->pb[i],
                                         (float)lr, b1, b2, eps, c1, c2, i % 2 == 0 ? q->wd : 0.0f,
                                         s),
                      "mlp adam")))
        return st;
  }
  double l = NAN;
  if (epochs > 0) {
    st = st_of(cudaMemcpyAsync(&l, q->loss, sizeof(double), cudaMemcpyDeviceToHost, s), "loss");
    if (st == FR_OK) st = st_of(cudaStreamSynchronize(s), "loss");
  }
  if (loss) *loss = l;
  return st;
}

int fr_mlp_predict(fr_mlp* q, void* U, double* V, void* stream) {
  if (!q) return FR_EINVAL;
  return fr_mlp_predict_for(q, q->ctx, U, V, stream);
}

int fr_mlp_predict_for(fr_mlp* q, fr_ctx* c, void* U, double* V, void* stream) {
  if (!q || !c || !ptr16(U) || !ptr16(V)) return FR_EINVAL;
  // any context of the network's discretization (its history is read)
  const fr_ctx* o = q->ctx;
  if (c->dim != o->dim || c->order != o->order || c->nv != o->nv || c->ne != o->ne ||
      c->stride != o->stride || c->precision != o->precision)
    return FR_EINVAL;
  if (c->hist_levels < 3 || !q->scales_set || q->adam_t == 0) return FR_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long ld = (long long)c->stride;
  int st = FR_OK;
  if (!q->Xi && ((st = dalloc(&q->Xi, (size_t)q->K * ld)) || (st = dalloc(&q->Hi1, (size_t)q->H * ld)) ||
                 (st = dalloc(&q->Hi2, (size_t)q->H * ld)) || (st = dalloc(&q->Yc, (size_t)q->NO * ld))))
    return st;
  const int lev[4] = {0, 1, 2, 0};
  if (c->precision == FR_F32)
    st = st_of(acmhd::launch_gather_features(hist_view<float>(c, lev), nullptr, (int)ld,
                                             q->in_scale_inv, q->K, q->Xi, ld, s), "mlp features");
  else
    st = st_of(acmhd::launch_gather_features(hist_view<double>(c, lev), nullptr, (int)ld,
                                             q->in_scale_inv, q->K, q->Xi, ld, s), "mlp features");
  if (st != FR_OK) return st;
  // hidden layers keep only their BF16 activations; the output is scaled
  if ((st = forward(q, q->Xi, ld, (int)ld, nullptr, q->Hi1, nullptr, q->Hi2, q->Yc, q->out_scale, s)))
    return st;
  if (q->out_degree >= 0 &&
      (st = st_of(acmhd::launch_project_lines(q->Yc, ld, c->ne, c->nv, c->m, c->dim, q->proj, s),
                  "mlp smoothing")))
    return st;
  if (c->precision == FR_F32)
    st = st_of(acmhd::launch_apply_guess(hist_view<float>(c, lev), q->Yc, ld, static_cast<float*>(U), V, s),
               "mlp guess");
  else
    st = st_of(acmhd::launch_apply_guess(hist_view<double>(c, lev), q->Yc, ld, static_cast<double*>(U), V, s),
               "mlp guess");
  return st;
}

int fr_mlp_set_output_degree(fr_mlp* q, int degree) {
  if (!q || degree < -1 || degree > q->ctx->order) return FR_EINVAL;
  q->out_degree = degree;
  if (degree >= 0) {
    double P[acmhd::kMaxM][acmhd::kMaxM];
    acmhd::degree_projector(q->ctx->ops, degree, P);
    for (int i = 0; i < acmhd::kMaxM; ++i)
      for (int k = 0; k < acmhd::kMaxM; ++k)
        q->proj.P[i][k] = (i < q->ctx->m && k < q->ctx->m) ? (float)P[i][k] : 0.0f;
  }
  return FR_OK;
}

int fr_mlp_train_step(fr_mlp* q, double lr, double* loss, void* stream) {
  return fr_mlp_train(q, 1, lr, loss, stream);
}

// Network file (little-endian):
//   char[8] "ACMHDMLP", uint32 version (1), int32 dim, order, nv, npts, K, H,
//   NO, adam_t, scales_set; float in_scale[3 nv], out_scale[nv]; then for
//   each of W1 b1 W2 b2 W3 b3 the FP32 master values, then the same blocks of
//   Adam's first and second moments; uint64 FNV-1a hash of everything before.
namespace {
constexpr char kMlpMagic[8] = {'A', 'C', 'M', 'H', 'D', 'M', 'L', 'P'};
constexpr uint32_t kMlpVersion = 1;

struct MlpFile {
  std::vector<unsigned char> bytes;
  void put(const void* p, size_t n) {
    const auto* c = static_cast<const unsigned char*>(p);
    bytes.insert(bytes.end(), c, c + n);
  }
};

uint64_t fnv1a(const unsigned char* p, size_t n) {
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < n; ++i) h = (h ^ p[i]) * 1099511628211ull;
  return h;
}

int mlp_fail(int st, const char* msg) {
  acmhd::set_last_error(msg);
  return st;
}
}  // namespace

int fr_mlp_save(const fr_mlp* q, const char* path) {
  if (!q || !path) return FR_EINVAL;
  const fr_ctx* c = q->ctx;
  MlpFile f;
  f.put(kMlpMagic, 8);
  f.put(&kMlpVersion, 4);
  const int32_t hdr[9] = {c->dim, c->order, c->nv, c->npts, q->K, q->H, q->NO, q->adam_t,
                          q->scales_set};
  f.put(hdr, sizeof(hdr));
  std::vector<float> sc(4 * (size_t)c->nv);
  int st = st_of(cudaMemcpy(sc.data(), q->in_scale, 3 * c->nv * 4, cudaMemcpyDeviceToHost), "save");
  if (!st) st = st_of(cudaMemcpy(sc.data() + 3 * c->nv, q->out_scale, c->nv * 4, cudaMemcpyDeviceToHost),
                      "save");
  if (st) return st;
  f.put(sc.data(), sc.size() * 4);
  for (float* const* arr : {q->p, q->m, q->v}) {
    for (int i = 0; i < 6; ++i) {
      std::vector<float> h(q->cnt[i]);
      if ((st = st_of(cudaMemcpy(h.data(), arr[i], q->cnt[i] * 4, cudaMemcpyDeviceToHost), "save")))
        return st;
      f.put(h.data(), h.size() * 4);
    }
  }
  const uint64_t hash = fnv1a(f.bytes.data(), f.bytes.size());
  f.put(&hash, 8);
  FILE* fp = std::fopen(path, "wb");
  if (!fp) return mlp_fail(FR_EINVAL, "fr_mlp_save: cannot open the file for writing");
  const size_t w = std::fwrite(f.bytes.data(), 1, f.bytes.size(), fp);
  const int closed = std::fclose(fp);
  if (w != f.bytes.size() || closed != 0) return mlp_fail(FR_EINVAL, "fr_mlp_save: write failed");
  return FR_OK;
}

int fr_mlp_load(fr_ctx* c, const char* path, int capacity, fr_mlp** out) {
  if (!c || !path || !out) return FR_EINVAL;
  FILE* fp = std::fopen(path, "rb");
  if (!fp) return mlp_fail(FR_EINVAL, "fr_mlp_load: cannot open the file");
  std::vector<unsigned char> b;
  unsigned char buf[1 << 16];
  size_t r;
  while ((r = std::fread(buf, 1, sizeof(buf), fp)) > 0) b.insert(b.end(), buf, buf + r);
  std::fclose(fp);
  const size_t head = 8 + 4 + 9 * 4;
  if (b.size() < head + 8 || std::memcmp(b.data(), kMlpMagic, 8) != 0)
    return mlp_fail(FR_EINVAL, "fr_mlp_load: not a network file");
  uint32_t ver;
  std::memcpy(&ver, b.data() + 8, 4);
  if (ver != kMlpVersion) return mlp_fail(FR_EINVAL, "fr_mlp_load: unsupported file version");
  uint64_t hash;
  std::memcpy(&hash, b.data() + b.size() - 8, 8);
  if (fnv1a(b.data(), b.size() - 8) != hash)
    return mlp_fail(FR_EINVAL, "fr_mlp_load: checksum mismatch (corrupt file)");
  int32_t hdr[9];
  std::memcpy(hdr, b.data() + 12, sizeof(hdr));
  const int dim = hdr[0], order = hdr[1], nv = hdr[2], npts = hdr[3], K = hdr[4], H = hdr[5],
            NO = hdr[6];
  if (dim != c->dim || order != c->order || nv != c->nv || npts != c->npts || NO != nv * npts ||
      K != 3 * NO)
    return mlp_fail(FR_EINVAL, "fr_mlp_load: the network belongs to another discretization");
  const size_t cnt[6] = {(size_t)H * K, (size_t)H, (size_t)H * H, (size_t)H, (size_t)NO * H,
                         (size_t)NO};
  size_t total = 0;
  for (size_t x : cnt) total += x;
  if (H < 8 || H > 4096 || b.size() != head + 4 * (4 * (size_t)nv + 3 * total) + 8)
    return mlp_fail(FR_EINVAL, "fr_mlp_load: file size does not match its header");
  fr_mlp* q = nullptr;
  int st = fr_mlp_create(c, H, capacity, 0, &q);
  if (st != FR_OK) return st;
  const unsigned char* p = b.data() + head;
  std::vector<float> sc(4 * (size_t)nv), inv(4 * (size_t)nv);
  std::memcpy(sc.data(), p, sc.size() * 4);
  p += sc.size() * 4;
  for (size_t i = 0; i < sc.size(); ++i) inv[i] = sc[i] > 0.0f ? 1.0f / sc[i] : 1.0f;
  st = st_of(cudaMemcpy(q->in_scale, sc.data(), 3 * nv * 4, cudaMemcpyHostToDevice), "load");
  if (!st) st = st_of(cudaMemcpy(q->in_scale_inv, inv.data(), 3 * nv * 4, cudaMemcpyHostToDevice), "load");
  if (!st) st = st_of(cudaMemcpy(q->out_scale, sc.data() + 3 * nv, nv * 4, cudaMemcpyHostToDevice), "load");
  if (!st)
    st = st_of(cudaMemcpy(q->out_scale_inv, inv.data() + 3 * nv, nv * 4, cudaMemcpyHostToDevice), "load");
  float** dst[3] = {q->p, q->m, q->v};
  for (int a = 0; a < 3 && !st; ++a) {
    for (int i = 0; i < 6 && !st; ++i) {
      st = st_of(cudaMemcpy(dst[a][i], p, cnt[i] * 4, cudaMemcpyHostToDevice), "load");
      p += cnt[i] * 4;
      if (!st && a == 0) st = st_of(acmhd::launch_to_bf16(cnt[i], q->p[i], q->pb[i], 0), "load");
    }
  }
  if (!st) st = st_of(cudaDeviceSynchronize(), "load");
  if (st) {
    fr_mlp_destroy(q);
    return st;
  }
  q->adam_t = hdr[7];
  q->scales_set = hdr[8];
  *out = q;
  return FR_OK;
}

int fr_gemm_bf16(int amode, int bmode, int N, int M, int K, const void* A, long long lda,
                 const void* B, long long ldb, float* C, long long ldc, void* stream) {
  if (N < 1 || M < 1 || K < 1 || !A || !B || !C || (amode != 0 && amode != 1) ||
      (bmode != 0 && bmode != 1))
    return FR_EINVAL;
  GemmArgs g = gemm(N, M, K, static_cast<const __nv_bfloat16*>(A), lda,
                    static_cast<const __nv_bfloat16*>(B), ldb);
  g.C = C;
  g.ldc = ldc;
  return st_of(acmhd::launch_gemm(amode, bmode, g, static_cast<cudaStream_t>(stream)), "gemm");
}

int fr_gemm_set_kernel(int kind) {
  if (kind != FR_GEMM_AUTO && kind != FR_GEMM_MMA_SYNC) return FR_EINVAL;
  acmhd::set_gemm_kernel(kind == FR_GEMM_AUTO ? acmhd::GEMM_KERNEL_AUTO
                                              : acmhd::GEMM_KERNEL_MMA_SYNC);
  return FR_OK;
}

int fr_gemm_check(void* stream) {
  int st = st_of(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)), "gemm");
  if (st != FR_OK) return st;
  const int code = acmhd::gemm_tc_status();
  if (code != 0) {
    char msg[160];
    std::snprintf(msg, sizeof(msg),
                  "tensor-memory GEMM: a bounded wait gave up (code %d); its output is invalid",
                  code);
    acmhd::set_last_error(msg);
    return FR_ECUDA;
  }
  return FR_OK;
}

}  // extern "C"
