// The volume work of the fused right-hand side for one tile of elements
// (stages 2-6 of Table fr_adv; the method and the work decomposition are
// described at the top of k_fused.cu), and the fused RHS kernel built on it.
// Shared by the whole-mesh RHS (k_fused.cu), the RHS on element ranges for
// the host-buffer pipeline (k_fused_range.cu) and the fused RK4 stage
// kernels (k_stage.cu).
#pragma once

#include "fr_device.cuh"

namespace acmhd {

// Output policies of the volume work.  Every entry i of R is produced
// exactly once and handed over as out.store(i, value, pre), which returns the
// value of the state that the entry leaves behind; pre holds the operands the
// policy reads for that entry, loaded ahead of the store (out.load /
// out.load_in), so that the stores, which the compiler must assume may alias
// later loads, do not serialise the loads behind them.
//
// RhsOut stores R (storage type S, computed in T), from the thread that
// finishes the entry.
template <typename T, typename S = T>
struct RhsOut {
  static constexpr bool kStage = false;
  struct Pre {};
  S* __restrict__ R;
  __device__ __forceinline__ Pre load_in(size_t, T) const { return Pre{}; }
  __device__ __forceinline__ T store(size_t i, T r, const Pre&) {
    R[i] = cvt<S>(r);
    return r;
  }
};

// StageOut folds one classical RK4 stage into the volume work (Sec. 5,
// pseudo-time stepping), with the combinations of the separate update
// kernels, so R itself is never stored:
//   stage 0: acc  = k;       next = U + dtau/2 k
//   stage 1: acc += 2 k;     next = U + dtau/2 k
//   stage 2: acc += 2 k;     next = U + dtau   k
//   stage 3: U    = U + dtau/6 (acc + k)            (next = U)
// With `dual`, the velocity rows use the FP64 master of the dual time step,
// k_V = R_V + C - (a0/dt) V_in, V_in = V (stage 0) or Vs, and stage 0 sums
// k_V^2 (the residual) into `sq`.  The traces of `next` go to `tr`, the
// other trace buffer, so the next stage needs no trace kernel.
// Every entry of U, acc, V, Vs and Vacc is read once, by the thread that
// then writes it, and by no one after that.
template <typename T>
struct StageOut {
  static constexpr bool kStage = true;
  T* U;              // RK4 base state: read; written at stage 3
  T* next;           // next stage input (stages 0..2)
  T* acc;            // RK4 accumulator
  T* tr;             // traces of the state this stage leaves behind
  T ct;              // stage coefficient in T (plain rows)
  double c, a0dt;    // stage coefficient and a0/dt (velocity rows of `dual`)
  int stage;
  int dual;
  size_t vel0, vel1;  // velocity rows: [vel0, vel1)
  double* V;         // FP64 velocity: base, stage, accumulator, BDF constant
  double* Vs;
  double* Vacc;
  const double* C;
  double sq;

  // plain rows (P, auxiliary; velocity without `dual`)
  struct Pre {
    T a, u0;
  };
  __device__ __forceinline__ Pre load(size_t i) const {
    Pre p;
    p.a = (stage == 0) ? T(0) : __ldg(acc + i);
    p.u0 = __ldg(U + i);
    return p;
  }
  // uin: entry i of the stage input, which is U itself at stage 0
  __device__ __forceinline__ Pre load_in(size_t i, T uin) const {
    Pre p;
    p.a = (stage == 0) ? T(0) : __ldg(acc + i);
    p.u0 = (stage == 0) ? uin : __ldg(U + i);
    return p;
  }
  // One code path for all four stages (selects and a predicated store, the
  // same operations as the separate update kernels): this is inlined at
  // every point of every line, and branches per stage would multiply the
  // kernel's code beyond what the instruction cache holds.
  __device__ __forceinline__ T store(size_t i, T k, const Pre& p) {
    const bool last = (stage == 3);
    const T un = fma(ct, last ? p.a + k : k, p.u0);
    if (!last) acc[i] = (stage == 0) ? k : fma(T(2), k, p.a);
    (last ? U : next)[i] = un;
    return un;
  }

  // velocity rows of `dual` (j = i - vel0)
  struct PreV {
    double vin, cc, v, vacc;
  };
  __device__ __forceinline__ PreV load_v(size_t j) const {
    PreV p;
    p.vin = __ldg((stage == 0) ? V + j : Vs + j);
    p.cc = __ldg(C + j);
    p.v = (stage == 0) ? p.vin : __ldg(V + j);
    p.vacc = (stage == 0) ? 0.0 : __ldg(Vacc + j);
    return p;
  }
  __device__ __forceinline__ T store_v(size_t i, size_t j, T k, const PreV& p) {
    const bool last = (stage == 3);
    const double kv = static_cast<double>(k) + fma(-a0dt, p.vin, p.cc);
    sq = (stage == 0) ? fma(kv, kv, sq) : sq;
    const double vn = fma(c, last ? p.vacc + kv : kv, p.v);
    if (!last) Vacc[j] = (stage == 0) ? kv : fma(2.0, kv, p.vacc);
    (last ? V : Vs)[j] = vn;
    const T un = static_cast<T>(vn);
    (last ? U : next)[i] = un;
    return un;
  }
};

// Stages 2-6 for one tile of E elements starting at e0 (a multiple of E).
// U, Tr hold values of the storage type S; the arithmetic runs in T (S = T,
// or S = double with T = df64, the double-float mode).
// sU, sA: shared memory of (1+D) NP E values each.  Every thread of the CTA
// must call it (it synchronises the CTA).
// RhsOut: each entry is stored by the thread that finishes it.
// StageOut (Out::kStage): an auxiliary entry is handed over by the thread
// that finishes it, with its operands loaded at the start of its slot, and
// that thread also writes the traces of the new auxiliary values on the
// faces of its axis.  The P and V entries stay in sA after the last phase; a
// pointwise pass over the tile hands them over in batches of coalesced
// entries, and their traces on all faces are taken from sA.  Traces go to
// out.tr (layout of the trace kernel, x faces only where the lane exchange
// cannot serve them).
template <int D, int M, typename T, int E, int NW, class Out, typename S>
__device__ __forceinline__ void fused_tile(const S* __restrict__ U, const S* __restrict__ Tr,
                                           Out& out, const FrConst<T>& c, int e0, T* sU,
                                           T* sA) {
  constexpr int NP = ipow<M>(D), NL = ipow<M>(D - 1), NS = 1 + 2 * D, SUB = 32 / E;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int el = lane % E, sub = lane / E;
  const int e = e0 + el;
  const bool valid = e < c.ne;
  const size_t Sd = c.stride;

  int nb[3][2];
  neighbours<D>(valid ? e : 0, c.n, nb);

  // The operands of one line that come from global memory: the auxiliary
  // slots along the line and the neighbours' traces at its two faces.  In
  // the x phase a neighbour inside the lane group is served by a shuffle
  // below, so only the others are read from memory.
  struct LineOps {
    T aux[D][M];
    T lo[NS], hi[NS];
  };
  auto line_of = [&](int l0) { return l0 + sub < NL ? l0 + sub : NL - 1; };
  auto load_ops = [&](int a, int l0, LineOps& o) {
    const int l = line_of(l0);
    const bool act = valid && (l0 + sub < NL);
#pragma unroll
    for (int t = 0; t < M; ++t) {
      const int pt = line_pt<D, M>(a, l, t);
#pragma unroll
      for (int i = 0; i < D; ++i)
        o.aux[i][t] = cvt<T>(__ldg(U + ((size_t)aux_var<D>(i, a) * NP + pt) * Sd + e));
    }
    const bool lo_mem = (a != 0) || (act && !x_pair_on_chip(nb[0][0], e, E));
    const bool hi_mem = (a != 0) || (act && !x_pair_on_chip(e, nb[0][1], E));
#pragma unroll
    // x faces of the neighbours outside the lane group: by group (x_col)
    // (the low neighbour's high face, the high neighbour's low face)
    const size_t clo = (a == 0) ? x_col(nb[0][0], E, c.xcompact, true) : (size_t)nb[a][0];
    const size_t chi = (a == 0) ? x_col(nb[0][1], E, c.xcompact, false) : (size_t)nb[a][1];
    for (int s = 0; s < NS; ++s) {
      o.lo[s] = lo_mem ? cvt<T>(__ldg(Tr + (((size_t)(2 * a + 1) * NS + s) * NL + l) * Sd + clo))
                       : T(0);
      o.hi[s] = hi_mem ? cvt<T>(__ldg(Tr + (((size_t)(2 * a) * NS + s) * NL + l) * Sd + chi))
                       : T(0);
    }
  };

  // The first line of each axis phase has its global operands requested
  // before the CTA barrier that opens the phase (they do not depend on it),
  // so their latency overlaps the staging of P and V and the barrier waits;
  // every other line issues its loads at its start.
  LineOps pre;
  load_ops(0, warp * SUB, pre);

  // stage P and V of the tile (rows of E contiguous values); unrolled so
  // that each thread has several independent loads in flight
#pragma unroll 8
  for (int idx = tid; idx < (1 + D) * NP * E; idx += NW * 32) {
    const int row = idx / E, x = idx - row * E;
    sU[idx] = cvt<T>(__ldg(U + (size_t)row * Sd + e0 + x));
  }
  __syncthreads();

#pragma unroll
  for (int a = 0; a < D; ++a) {
    // the trip count is uniform across the warp (shuffles need every lane)
    for (int l0 = warp * SUB; l0 < NL; l0 += NW * SUB) {
      const bool lvalid = l0 + sub < NL;
      const int l = lvalid ? l0 + sub : NL - 1;
      const bool act = valid && lvalid;
      LineOps ops;
      if (l0 == warp * SUB)
        ops = pre;
      else
        load_ops(a, l0, ops);
      const bool lo_mem = (a != 0) || (act && !x_pair_on_chip(nb[0][0], e, E));
      const bool hi_mem = (a != 0) || (act && !x_pair_on_chip(e, nb[0][1], E));
      // slot values along the line
      T u[NS][M];
#pragma unroll
      for (int t = 0; t < M; ++t) {
        const int pt = line_pt<D, M>(a, l, t);
#pragma unroll
        for (int s = 0; s <= D; ++s) u[s][t] = sU[(s * NP + pt) * E + el];
#pragma unroll
        for (int i = 0; i < D; ++i) u[1 + D + i][t] = ops.aux[i][t];
      }
      T nb_lo[NS], nb_hi[NS];
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        nb_lo[s] = ops.lo[s];
        nb_hi[s] = ops.hi[s];
      }
      // own traces, and the common fluxes at the two faces (stage 4).  On
      // the y and z faces the trace kernel (or the previous fused stage)
      // stored exactly these values (same inputs, same trace_dot); in FP64,
      // where this kernel is bound by arithmetic on GB300, they are read
      // back instead of recomputed (e < elem_stride: in bounds for every
      // lane; padding lanes' values are not used)
      constexpr bool kOwnFromMemory = sizeof(T) == 8;
      T own_lo[NS], own_hi[NS];
      if (kOwnFromMemory && a != 0) {
#pragma unroll
        for (int s = 0; s < NS; ++s) {
          own_lo[s] = cvt<T>(__ldg(Tr + (((size_t)(2 * a) * NS + s) * NL + l) * Sd + e));
          own_hi[s] = cvt<T>(__ldg(Tr + (((size_t)(2 * a + 1) * NS + s) * NL + l) * Sd + e));
        }
      } else {
#pragma unroll
        for (int s = 0; s < NS; ++s) {
          // through the storage type, as the trace kernel stores them, so
          // both elements of a face use identical values
          own_lo[s] = cvt<T>(cvt<S>(trace_dot<M>(u[s], c.lm)));
          own_hi[s] = cvt<T>(cvt<S>(trace_dot<M>(u[s], c.lp)));
        }
      }
      if (a == 0) {
#pragma unroll
        for (int s = 0; s < NS; ++s) {
          const T from_left = shfl_up(own_hi[s], 1, E);
          const T from_right = shfl_down(own_lo[s], 1, E);
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
        // operands of the auxiliary entries of this slot
        typename Out::Pre pq[M];
        if (s > D) {
#pragma unroll
          for (int t = 0; t < M; ++t)
            pq[t] = out.load_in(((size_t)aux_var<D>(s - D - 1, a) * NP + line_pt<D, M>(a, l, t)) *
                                    Sd + e,
                                u[s][t]);
        }
        T f[M];
#pragma unroll
        for (int t = 0; t < M; ++t) f[t] = point_flux<D>(u, t, s, a, c.zeta, c.nu, c.inv_t);
        // the new values of an auxiliary slot feed the traces of the face
        // pair of axis a, accumulated point by point in the order and
        // rounding of trace_dot
        T t_lo = T(0), t_hi = T(0);
#pragma unroll
        for (int i = 0; i < M; ++i) {
          T r = fma(c.br[a][i], fr[s], c.bl[a][i] * fl[s]);
#pragma unroll
          for (int k = 0; k < M; ++k) r = fma(c.A[a][i][k], f[k], r);
          const int pt = line_pt<D, M>(a, l, i);
          T nx = T(0);
          if (s <= D) {
            const int idx = (s * NP + pt) * E + el;
            if (a == 0) {
              sA[idx] = r;
            } else if (a < D - 1 || Out::kStage) {
              sA[idx] += r;
            } else {
              out.store(((size_t)s * NP + pt) * Sd + e, sA[idx] + r, typename Out::Pre{});
            }
          } else {
            // auxiliary equation of slot s: finished here, with its source
            const int v = aux_var<D>(s - D - 1, a);
            nx = out.store(((size_t)v * NP + pt) * Sd + e, fma(-u[s][i], c.inv_t, r),
                           pq[i]);
          }
          if constexpr (Out::kStage) {
            t_lo = (i == 0) ? rn_mul(nx, c.lm[0]) : rn_fma(nx, c.lm[i], t_lo);
            t_hi = (i == 0) ? rn_mul(nx, c.lp[0]) : rn_fma(nx, c.lp[i], t_hi);
          }
        }
        if constexpr (Out::kStage) {
          const bool w_lo = (a != 0) || !x_pair_on_chip(nb[0][0], e, E);
          const bool w_hi = (a != 0) || !x_pair_on_chip(e, nb[0][1], E);
          const size_t clo = (a == 0) ? x_col(e, E, c.xcompact, false) : (size_t)e;
          const size_t chi = (a == 0) ? x_col(e, E, c.xcompact, true) : (size_t)e;
          if (s > D && w_lo) out.tr[(((size_t)(2 * a) * NS + s) * NL + l) * Sd + clo] = t_lo;
          if (s > D && w_hi) out.tr[(((size_t)(2 * a + 1) * NS + s) * NL + l) * Sd + chi] = t_hi;
        }
      }
    }
    if (a + 1 < D) load_ops(a + 1, warp * SUB, pre);
    __syncthreads();  // partial sums complete before the next axis; smem free after the last
  }
  if constexpr (Out::kStage) {
    // P and V rows: R of the whole tile is in sA; hand it over entry by
    // entry (E consecutive entries of a row are E consecutive elements) and
    // keep the new state in sA for the traces
    constexpr int NPE = NP * E, TOT = (1 + D) * NPE, NT = NW * 32;
    auto gidx = [&](int idx) {
      const int row = idx / E;
      return (size_t)row * Sd + e0 + (idx - row * E);
    };
    auto real = [&](int idx, int end) { return idx < end && e0 + idx % E < c.ne; };
    // plain rows: P, and V unless `dual`; KB entries per thread in flight
    constexpr int KB = 8;
    const int pend = out.dual ? NPE : TOT;
    for (int base = tid; base < pend; base += NT * KB) {
      typename Out::Pre p[KB];
#pragma unroll
      for (int k = 0; k < KB; ++k)
        if (real(base + k * NT, pend)) p[k] = out.load(gidx(base + k * NT));
#pragma unroll
      for (int k = 0; k < KB; ++k) {
        const int idx = base + k * NT;
        if (real(idx, pend)) sA[idx] = out.store(gidx(idx), sA[idx], p[k]);
      }
    }
    if (out.dual) {
      constexpr int KV = 4;
      for (int base = NPE + tid; base < TOT; base += NT * KV) {
        typename Out::PreV q[KV];
#pragma unroll
        for (int k = 0; k < KV; ++k)
          if (real(base + k * NT, TOT)) q[k] = out.load_v(gidx(base + k * NT) - out.vel0);
#pragma unroll
        for (int k = 0; k < KV; ++k) {
          const int idx = base + k * NT;
          if (real(idx, TOT)) {
            const size_t i = gidx(idx);
            sA[idx] = out.store_v(i, i - out.vel0, sA[idx], q[k]);
          }
        }
      }
    }
    __syncthreads();
    // P and V slots of the new state on the faces of every axis, from sA
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const bool w_lo = (a != 0) || !x_pair_on_chip(nb[0][0], e, E);
      const bool w_hi = (a != 0) || !x_pair_on_chip(e, nb[0][1], E);
      if (!valid || (!w_lo && !w_hi)) continue;
      for (int l = warp * SUB + sub; l < NL; l += NW * SUB) {
#pragma unroll
        for (int s = 0; s <= D; ++s) {
          T x[M];
#pragma unroll
          for (int t = 0; t < M; ++t) x[t] = sA[(s * NP + line_pt<D, M>(a, l, t)) * E + el];
          const size_t clo = (a == 0) ? x_col(e, E, c.xcompact, false) : (size_t)e;
          const size_t chi = (a == 0) ? x_col(e, E, c.xcompact, true) : (size_t)e;
          if (w_lo) out.tr[(((size_t)(2 * a) * NS + s) * NL + l) * Sd + clo] = trace_dot<M>(x, c.lm);
          if (w_hi)
            out.tr[(((size_t)(2 * a + 1) * NS + s) * NL + l) * Sd + chi] = trace_dot<M>(x, c.lp);
        }
      }
    }
  }
}

// The fused RHS kernel: one tile of E elements per CTA.  RANGED kernels
// start at tile tile0 (the host-buffer pipeline runs the mesh in slabs);
// the whole-mesh kernel keeps the tile index free of the offset (measured:
// the offset alone cost 2 % of the 64^3 p=3 volume kernel's time).
template <int D, int M, typename S, typename T, int E, int NW, int MINB, bool RANGED>
__global__ void __launch_bounds__(NW * 32, MINB)
fused_kernel(const S* __restrict__ U, const S* __restrict__ Tr, S* __restrict__ R,
             const FrConst<T> c, int tile0) {
  constexpr int NP = ipow<M>(D);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sU = reinterpret_cast<T*>(smem_raw);  // [1+D][NP][E]
  T* sA = sU + (1 + D) * NP * E;           // [1+D][NP][E]
  RhsOut<T, S> out{R};
  const int tile = RANGED ? tile0 + (int)blockIdx.x : (int)blockIdx.x;
  fused_tile<D, M, T, E, NW>(U, Tr, out, c, tile * E, sU, sA);
}

// elements [e_begin, e_end); e_begin a multiple of 32 (and so of E), and 0
// unless RANGED
template <int D, int M, typename S, typename T, bool RANGED>
cudaError_t fused_launch(const FrConst<T>& c, const void* U, const void* Tr, void* R, int e_begin,
                         int e_end, cudaStream_t s) {
  using C = FusedCfg<D, M, T>;
  auto kern = fused_kernel<D, M, S, T, C::E, C::NW, C::MINB, RANGED>;
  static PerDeviceOnce smem_once;  // per template instance
  cudaError_t err = set_smem_limit(smem_once, kern, C::SMEM);
  if (err != cudaSuccess) return err;
  const int nblk = (e_end - e_begin + C::E - 1) / C::E;
  if (nblk <= 0) return cudaSuccess;
  kern<<<nblk, C::NW * 32, C::SMEM, s>>>(static_cast<const S*>(U), static_cast<const S*>(Tr),
                                          static_cast<S*>(R), c, e_begin / C::E);
  return cudaGetLastError();
}

}  // namespace acmhd
