// fr_rhs_static: the fused right-hand side for callers that cannot allocate
// device memory.  The paper has no counterpart; it is a deployment variant of
// fr_rhs (face-trace kernel + fused kernel, the same kernels and results).
//
// Why: some callers must not allocate device memory once they are running,
// e.g. a host application whose own pool allocator reserved the device's
// memory at start-up, or a time-critical loop in which a device allocation
// (which can synchronise the whole device) is not allowed.  fr_create
// allocates the face-trace scratch with cudaMalloc; this entry point takes
// the scratch from a fixed array that is part of the library's device image
// instead, and calls no cudaMalloc, cudaFree or other allocating routine.
//
// The array is kStaticTraceBytes (16 MiB) and every GPU that loads the
// library holds it until the process exits.  All calls share it and it keeps
// the previous call's contents: nothing needs clearing, because the trace
// kernel writes every entry that the fused kernel then reads, but calls whose
// kernels overlap on the GPU (other streams, other host threads) race on it.
//
// The library is linked without relocatable device code, so this file is a
// module of its own.  Under CUDA's default lazy module loading the module -
// the array included - is loaded onto a device at the first
// cudaGetSymbolAddress or launch that needs it, and loading allocates device
// memory.  So the first call on each device may allocate (and fail with
// FR_ECUDA when the device's memory is already taken); later calls do not.
// Callers make that first call before their pool reserves memory, or set
// CUDA_MODULE_LOADING=EAGER.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "fr_internal.h"

static constexpr size_t kStaticTraceBytes = size_t(16) << 20;

// The face-trace scratch of fr_rhs_static.  In host code this name is only a
// host-side stand-in: the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_static_trace[kStaticTraceBytes];

namespace {

constexpr int kMaxDevices = 64;

std::mutex g_static_mu;
void* g_static_addr[kMaxDevices] = {};

// Device address of g_static_trace on the current device, looked up once per
// device (with that device current) and cached.  The cache is not
// invalidated by a device reset.
cudaError_t static_trace_address(int device, void** out) {
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_trace);
    if (e != cudaSuccess) return e;
    g_static_addr[device] = p;
  }
  *out = g_static_addr[device];
  return cudaSuccess;
}

int static_fail(int status, const char* msg) {
  char text[224];
  std::snprintf(text, sizeof(text), "fr_rhs_static: %s", msg);
  acmhd::set_last_error(text);
  return status;
}

}  // namespace

extern "C" int fr_rhs_static(const fr_mesh* mesh, int order, int nvars, double zeta, double nu,
                             double t_r, int precision, int correction, const void* U, void* R,
                             void* stream) {
  if (!mesh || !U || !R || U == R) return static_fail(FR_EINVAL, "null or aliasing pointers");
  if ((reinterpret_cast<uintptr_t>(U) | reinterpret_cast<uintptr_t>(R)) & 15u)
    return static_fail(FR_EINVAL, "state pointers must be 16-byte aligned");
  const int d = mesh->dim;
  if ((d != 2 && d != 3) || order < 1 || order > acmhd::kMaxM - 1 || nvars != 1 + d + d * d ||
      (precision != FR_F32 && precision != FR_F64) ||
      (correction != FR_CORR_DG && correction != FR_CORR_G2) || !(zeta > 0.0) ||
      !(nu >= 0.0) || !(t_r > 0.0) || !std::isfinite(zeta) || !std::isfinite(nu) ||
      !std::isfinite(t_r))
    return static_fail(FR_EINVAL, "invalid order, nvars, precision, correction or parameters");
  long long ne = 1;
  for (int a = 0; a < d; ++a) {
    if (mesh->n[a] < 1 || !(mesh->hi[a] > mesh->lo[a]) ||
        !std::isfinite(mesh->hi[a] - mesh->lo[a]))
      return static_fail(FR_EINVAL, "invalid mesh");
    ne *= mesh->n[a];
  }
  const int m = order + 1;
  long long nl = 1;
  for (int a = 1; a < d; ++a) nl *= m;
  const long long stride = (ne + 31) / 32 * 32;
  const long long esz = precision == FR_F32 ? 4 : 8;
  const long long need = 2LL * d * (1 + 2 * d) * nl * stride * esz;
  if (ne > (1LL << 30) || need > (long long)kStaticTraceBytes) {
    char msg[160];
    std::snprintf(msg, sizeof(msg), "face traces need %lld bytes, more than the %zu-byte static "
                  "scratch", need, kStaticTraceBytes);
    return static_fail(FR_EINVAL, msg);
  }

  fr_ctx c;
  std::memset(&c, 0, sizeof(c));
  c.dim = d;
  c.order = order;
  c.m = m;
  c.nv = nvars;
  c.precision = precision;
  c.correction = correction;
  c.mesh = *mesh;
  c.zeta = zeta;
  c.nu = nu;
  c.t_r = t_r;
  c.ne = static_cast<int>(ne);
  c.stride = static_cast<size_t>(stride);
  c.npts = static_cast<int>(nl * m);
  c.elem_bytes = static_cast<size_t>(esz);
  c.bytes_state = (size_t)nvars * c.npts * c.stride * c.elem_bytes;
  if (!acmhd::build_ops1d(order, correction, &c.ops))
    return static_fail(FR_EINVAL, "operator construction failed");
  if (precision == FR_F32)
    acmhd::fill_const(&c, &c.cf);
  else
    acmhd::fill_const(&c, &c.cd);

  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e == cudaSuccess && (device < 0 || device >= kMaxDevices))
    return static_fail(FR_EINVAL, "device ordinal beyond the supported range");
  void* trace = nullptr;
  if (e == cudaSuccess) e = static_trace_address(device, &trace);
  c.device = device;
  c.trace = trace;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (e == cudaSuccess) e = acmhd::launch_trace(&c, U, trace, s);
  if (e == cudaSuccess) e = acmhd::launch_fused(&c, U, trace, R, s);
  if (e != cudaSuccess) return static_fail(FR_ECUDA, cudaGetErrorString(e));
  return FR_OK;
}
