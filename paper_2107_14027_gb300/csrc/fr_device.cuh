// Device-side building blocks shared by the trace, fused and unfused kernels.
//
// Face vectors use "slots": for a face with normal along axis a the normal
// flux F_a of ACM-HD (Sec. 2.2, Eq. acmhd_nd) is non-zero in exactly 1 + 2d
// equations (Sec. 3, sparsity equation): slot 0 = P, slots 1..d = V_i, slots
// d+1..2d = the auxiliary equation d(V_i)/dx_a.  Only these slots of the
// face traces are ever needed.
//
// Functions whose results must agree bit for bit between the two elements
// that share a face (face traces, the common flux) use explicit
// round-to-nearest intrinsics, so the compiler cannot contract or reorder
// them differently at different call sites.
#pragma once

#include <cuda_runtime.h>

#include "df64.cuh"
#include "fr_internal.h"
#include "per_device_once.h"
#include "xface_layout.h"

namespace acmhd {

__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rn_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double rn_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rn_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double rn_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float rn_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rn_fma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float rn_sqrt(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ double rn_sqrt(double a) { return __dsqrt_rn(a); }
__device__ __forceinline__ float vabs(float a) { return fabsf(a); }
__device__ __forceinline__ double vabs(double a) { return fabs(a); }
__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double vmax(double a, double b) { return fmax(a, b); }
// double-float versions (df64.cuh; every operation is already exactly rounded
// in a fixed order)
__device__ __forceinline__ df64 rn_mul(df64 a, df64 b) { return df_mul(a, b); }
__device__ __forceinline__ df64 rn_add(df64 a, df64 b) { return df_add(a, b); }
__device__ __forceinline__ df64 rn_sub(df64 a, df64 b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ df64 rn_fma(df64 a, df64 b, df64 c) { return df_add(df_mul(a, b), c); }
__device__ __forceinline__ df64 rn_sqrt(df64 a) { return df_sqrt(a); }
__device__ __forceinline__ df64 vabs(df64 a) { return a.hi < 0.0f ? df_neg(a) : a; }
__device__ __forceinline__ df64 vmax(df64 a, df64 b) {
  return (a.hi > b.hi || (a.hi == b.hi && a.lo >= b.lo)) ? a : b;
}

// variable index of d(V_i)/dx_b
template <int D>
__host__ __device__ constexpr int aux_var(int i, int b) {
  return 1 + D + i * D + b;
}

// variable held in slot s of a face with normal axis a
template <int D>
__host__ __device__ constexpr int slot_var(int s, int a) {
  return s <= D ? s : aux_var<D>(s - D - 1, a);
}

template <int M>
__host__ __device__ constexpr int ipow(int e) {
  return e == 0 ? 1 : M * ipow<M>(e - 1);
}

// point index of the t-th point of line l along axis a (pt = i + m j + m^2 k;
// the line index enumerates the other coordinates, lower axis fastest)
template <int D, int M>
__host__ __device__ __forceinline__ int line_pt(int a, int l, int t) {
  const int ma = (a == 0) ? 1 : (a == 1 ? M : M * M);
  return (l % ma) + ma * t + ma * M * (l / ma);
}

// Interpolation of a line to one end: sum_k ell_k x_k, fixed order, explicit FMA.
template <int M, typename T>
__device__ __forceinline__ T trace_dot(const T (&x)[M], const T* ell) {
  T acc = rn_mul(x[0], ell[0]);
#pragma unroll
  for (int k = 1; k < M; ++k) acc = rn_fma(x[k], ell[k], acc);
  return acc;
}

// Slot s of the normal flux F_a at point t of a line held as u[slot][point]:
// slot 0 zeta V_a; slot 1+i V_i V_a + P delta_ia - nu d(V_i)/dx_a; slot
// 1+D+i -V_i / T.
template <int D, int M, typename T>
__device__ __forceinline__ T point_flux(const T (&u)[1 + 2 * D][M], int t, int s, int a, T zeta,
                                        T nu, T inv_t) {
  const T va = u[1 + a][t];
  if (s == 0) return rn_mul(zeta, va);
  if (s <= D) {
    const int i = s - 1;
    T q = rn_mul(nu, u[1 + D + i][t]);
    q = (i == a) ? rn_sub(u[0][t], q) : -q;
    return rn_fma(u[1 + i][t], va, q);
  }
  return -rn_mul(u[s - D][t], inv_t);
}

// Common interface flux on a face with normal +e_a, uL on the low side:
// mean flux plus Rusanov dissipation (s/2)(uR - uL) on P and V, where
// s = max(|V_a| + sqrt(V_a^2 + zeta)) over both sides (Sec. 5).
//  * |V| + sqrt(V^2 + zeta), each operation rounded to nearest, does not
//    decrease as |V| grows, so the larger of the two sides' speeds is the
//    speed of the larger |V_a|, bit for bit: one square root per face point.
//  * The P and auxiliary slots are linear in the state (zeta V_a, -V_i / T),
//    so their mean flux is formed from the sum of the two states.
// Both elements of a face call this with the same (uL, uR) and obtain the
// same bits.
template <int D, typename T>
__device__ __forceinline__ void common_flux(const T (&uL)[1 + 2 * D], const T (&uR)[1 + 2 * D],
                                            int a, T zeta, T nu, T inv_t,
                                            T (&fi)[1 + 2 * D]) {
  const T vl = uL[1 + a], vr = uR[1 + a];
  const T vm = vmax(vabs(vl), vabs(vr));
  const T hs = rn_mul(T(0.5), rn_add(vm, rn_sqrt(rn_fma(vm, vm, zeta))));
  const T hz = rn_mul(T(0.5), zeta);
  const T hit = rn_mul(T(-0.5), inv_t);
  fi[0] = rn_fma(-hs, rn_sub(uR[0], uL[0]), rn_mul(hz, rn_add(vl, vr)));
#pragma unroll
  for (int i = 0; i < D; ++i) {
    // V_i V_a + P delta_ia - nu d(V_i)/dx_a on each side, then the mean
    T tl = rn_mul(nu, uL[1 + D + i]);
    T tr = rn_mul(nu, uR[1 + D + i]);
    tl = (i == a) ? rn_sub(uL[0], tl) : -tl;
    tr = (i == a) ? rn_sub(uR[0], tr) : -tr;
    const T mean = rn_mul(T(0.5), rn_add(rn_fma(uL[1 + i], vl, tl), rn_fma(uR[1 + i], vr, tr)));
    fi[1 + i] = rn_fma(-hs, rn_sub(uR[1 + i], uL[1 + i]), mean);
    fi[1 + D + i] = rn_mul(hit, rn_add(uL[1 + i], uR[1 + i]));
  }
}

// Element coordinates and neighbours on the periodic mesh.
template <int D>
__device__ __forceinline__ void neighbours(int e, const int* n, int (&nb)[3][2]) {
  const int ex = e % n[0];
  const int r = e / n[0];
  const int ey = (D == 3) ? r % n[1] : r;
  const int ez = (D == 3) ? r / n[1] : 0;
  const int sy = n[0], sz = n[0] * n[1];
  nb[0][0] = e + ((ex == 0) ? n[0] - 1 : -1);
  nb[0][1] = e + ((ex == n[0] - 1) ? 1 - n[0] : 1);
  nb[1][0] = e + ((ey == 0) ? (n[1] - 1) * sy : -sy);
  nb[1][1] = e + ((ey == n[1] - 1) ? (1 - n[1]) * sy : sy);
  if (D == 3) {
    nb[2][0] = e + ((ez == 0) ? (n[2] - 1) * sz : -sz);
    nb[2][1] = e + ((ez == n[2] - 1) ? (1 - n[2]) * sz : sz);
  } else {
    nb[2][0] = nb[2][1] = e;
  }
}

// Work decomposition of the fused kernel: E consecutive elements per CTA
// (lane -> element, 32/E lines per warp), NW warps, MINB CTAs per SM.
//  * E: the largest of {32, 16, 8, 4} whose shared memory (P, V and their
//    partial sums) lets two CTAs share an SM;
//  * NW: the m^(d-1) lines of a phase come in WT = ceil(lines / (32/E))
//    warp tasks, spread over at most 12 warps in equal rounds;
//  * MINB: as many CTAs per SM as shared memory allows, as long as each
//    thread keeps at least REG_FLOOR registers (the FP32 kernel is latency
//    bound: resident warps keep loads in flight).
template <int D, int M, typename T>
struct FusedCfg {
  static constexpr int NP = ipow<M>(D);
  static constexpr int NL = ipow<M>(D - 1);
  static constexpr size_t bytes(int e) { return size_t(2) * (1 + D) * NP * e * sizeof(T); }
  static constexpr int E = bytes(32) <= 112 * 1024 ? 32
                           : bytes(16) <= 112 * 1024 ? 16
                           : bytes(8) <= 112 * 1024 ? 8 : 4;
  static constexpr size_t SMEM = bytes(E);
  static constexpr int WT = (NL + 32 / E - 1) / (32 / E);
  static constexpr int ROUNDS = (WT + 11) / 12;
  static constexpr int NW = (WT + ROUNDS - 1) / ROUNDS;
  // FP64 at m = 5: three CTAs per SM would cap the kernel at 80 registers
  // and spill about 2.4 KB per thread; FP64 is bound by the FP64 pipe on
  // GB300, so two CTAs without spills serve it better
  static constexpr int REG_FLOOR =
      ((M >= 6) ? 80 : (sizeof(T) == 8 && M == 5 ? 64 : 48)) * int(sizeof(T) / 4);
  static constexpr int SMEM_BLOCKS = int((228 * 1024) / (SMEM + 1024));
  static constexpr int REG_BLOCKS = 65536 / (NW * 32 * REG_FLOOR);
  static constexpr int MINB_RAW = SMEM_BLOCKS < REG_BLOCKS ? SMEM_BLOCKS : REG_BLOCKS;
  static constexpr int MINB = MINB_RAW < 1 ? 1 : (MINB_RAW > 8 ? 8 : MINB_RAW);
};

// Raises a kernel's dynamic shared memory limit to `bytes` on the current
// device, once per device (the attribute is per device context).
template <class Kernel>
cudaError_t set_smem_limit(PerDeviceOnce& once, Kernel kern, size_t bytes) {
  const int st = once.run([](int* d) { return static_cast<int>(cudaGetDevice(d)); },
                          [&] {
                            return static_cast<int>(cudaFuncSetAttribute(
                                kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
                          });
  return static_cast<cudaError_t>(st);
}



}  // namespace acmhd

// Dispatch a runtime (dim, m) pair to a template call FN<D, M>(args...).
#define ACMHD_DISPATCH_DM(dim, m, CALL)                        \
  do {                                                         \
    switch ((dim) * 10 + (m)) {                                \
      case 22: { constexpr int D_ = 2, M_ = 2; CALL; } break;  \
      case 23: { constexpr int D_ = 2, M_ = 3; CALL; } break;  \
      case 24: { constexpr int D_ = 2, M_ = 4; CALL; } break;  \
      case 25: { constexpr int D_ = 2, M_ = 5; CALL; } break;  \
      case 26: { constexpr int D_ = 2, M_ = 6; CALL; } break;  \
      case 27: { constexpr int D_ = 2, M_ = 7; CALL; } break;  \
      case 32: { constexpr int D_ = 3, M_ = 2; CALL; } break;  \
      case 33: { constexpr int D_ = 3, M_ = 3; CALL; } break;  \
      case 34: { constexpr int D_ = 3, M_ = 4; CALL; } break;  \
      case 35: { constexpr int D_ = 3, M_ = 5; CALL; } break;  \
      case 36: { constexpr int D_ = 3, M_ = 6; CALL; } break;  \
      case 37: { constexpr int D_ = 3, M_ = 7; CALL; } break;  \
      default: return cudaErrorInvalidValue;                   \
    }                                                          \
  } while (0)
