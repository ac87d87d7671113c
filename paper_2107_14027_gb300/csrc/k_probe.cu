// Arithmetic peak probe: the FMA throughput of this GPU in FP32 or FP64,
// measured by a kernel that does nothing else.  It gives the denominator of
// the roofline fraction of a kernel that is bound by arithmetic rather than
// by memory (the FP64 right-hand side on GB300).
//
// Each thread runs kChains independent FMA chains (enough independent work
// to cover the FMA pipe's latency) for `iters` iterations; the grid fills
// every SM with kBlocksPerSm blocks of 256 threads.  The result of all chains
// is written only if it is exactly zero, which the inputs rule out, so the
// compiler cannot drop the work and memory traffic stays negligible.
#include <cuda_runtime.h>

#include "acmhd_fr.h"
#include "fr_internal.h"

namespace acmhd {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;
constexpr int kUnroll = 16;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_probe_kernel(int iters, T a, T b, T* out) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == T(0)) out[blockIdx.x] = s;
}

}  // namespace
}  // namespace acmhd

extern "C" int fr_fma_probe(int precision, int iters, void* out, double* flops, void* stream) {
  if ((precision != FR_F32 && precision != FR_F64) || iters < 1 || !out) return FR_EINVAL;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    acmhd::set_last_error(cudaGetErrorString(e));
    return FR_ECUDA;
  }
  const int blocks = nsm * acmhd::kBlocksPerSm;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // x <- x a + b with |a| < 1 stays bounded and never becomes exactly zero
  if (precision == FR_F32)
    acmhd::fma_probe_kernel<float><<<blocks, acmhd::kThreads, 0, s>>>(
        iters, 0.999f, 1e-4f, static_cast<float*>(out));
  else
    acmhd::fma_probe_kernel<double><<<blocks, acmhd::kThreads, 0, s>>>(
        iters, 0.999, 1e-4, static_cast<double*>(out));
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    acmhd::set_last_error(cudaGetErrorString(e));
    return FR_ECUDA;
  }
  if (flops)
    *flops = 2.0 * acmhd::kChains * acmhd::kUnroll * (double)iters * acmhd::kThreads * blocks;
  return FR_OK;
}
