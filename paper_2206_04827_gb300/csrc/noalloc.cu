// Allocation-free values -> coefficients transform.
//
// cyl_vals2coeffs needs a plan, and building a plan allocates device memory
// (operator tables, factors, two N-element scratch arrays).  Some callers
// cannot allocate at all: hosts that hand every byte of device memory to
// their own pool and forbid other allocations, and latency-critical loops
// that must never enter the allocator.  For them this file provides
// cyl_vals2coeffs_noalloc: the same three axis transforms, with the scratch
// (two intermediate arrays and the three transform matrices) taken from a
// fixed array in the library's own device image.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>
#include <utility>
#include <vector>

#include "../../include/cyl.h"
#include "kernels.cuh"

namespace {

// Fixed scratch of CYL_NOALLOC_SCRATCH_DOUBLES doubles (64 MiB) in every
// device context that loads this library, held until the process exits.
__device__ __align__(256) double g_noalloc_scratch[CYL_NOALLOC_SCRATCH_DOUBLES];

// In host code the symbol name is only a host-side stand-in, so the array's
// device address is looked up (cudaGetSymbolAddress, with the device
// current) and cached.  The cache is keyed by the CUDA context's unique ID,
// not by the device number: after cudaDeviceReset the device gets a new
// primary context, in which the array may sit at another address, and the
// lookup is then made again.
using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);
std::mutex g_scratch_mu;
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;
std::vector<std::pair<unsigned long long, double *>> g_scratch_by_ctx;

// Unique ID of the calling thread's current context (0 when none is current).
cudaError_t current_context_id(unsigned long long *id) {
  *id = 0;
  if (!g_ctx_get_current || !g_ctx_get_id) {
    cudaDriverEntryPointQueryResult q1, q2;
    void *f1 = nullptr, *f2 = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
    if (e == cudaSuccess) e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
    if (e != cudaSuccess) return e;
    if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
      return cudaErrorNotSupported;
    g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
    g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f2);
  }
  CUcontext ctx = nullptr;
  if (g_ctx_get_current(&ctx) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
  if (!ctx) return cudaSuccess;
  if (g_ctx_get_id(ctx, id) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
  return cudaSuccess;
}

// Device address of the scratch array in the current context.
cudaError_t scratch_for_current_context(double **out) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  unsigned long long id = 0;
  cudaError_t e = current_context_id(&id);
  if (e != cudaSuccess) return e;
  if (id != 0)
    for (const auto &kv : g_scratch_by_ctx)
      if (kv.first == id) {
        *out = kv.second;
        return cudaSuccess;
      }
  // first call in this context (or no context yet: the lookup creates the
  // device's primary context and makes it current)
  void *p = nullptr;
  if ((e = cudaGetSymbolAddress(&p, g_noalloc_scratch)) != cudaSuccess) return e;
  if (id == 0 && ((e = current_context_id(&id)) != cudaSuccess || id == 0))
    return e != cudaSuccess ? e : cudaErrorDeviceUninitialized;
  g_scratch_by_ctx.emplace_back(id, static_cast<double *>(p));
  *out = static_cast<double *>(p);
  return cudaSuccess;
}

// cos(pi * num / den) with the argument reduced exactly in integers.
__device__ double cospi_frac(long long num, long long den) {
  long long r = num % (2 * den);
  if (r < 0) r += 2 * den;
  return cospi((double)r / (double)den);
}

__device__ double sinpi_frac(long long num, long long den) {
  long long r = num % (2 * den);
  if (r < 0) r += 2 * den;
  return sinpi((double)r / (double)den);
}

// Forward DCT-I matrix of the Chebyshev grid (Section 2):
// W[j][a] = (2/(L-1)) w_j w_a T_j(x_a), T_j(x_a) = cos(j (L-1-a) pi / (L-1)).
__global__ void fill_cheb_forward(double *W, int L) {
  const int total = L * L;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int j = e / L, a = e - j * L;
    const double wj = (j == 0 || j == L - 1) ? 0.5 : 1.0;
    const double wa = (a == 0 || a == L - 1) ? 0.5 : 1.0;
    W[e] = 2.0 / (L - 1) * wj * wa * cospi_frac((long long)j * (L - 1 - a), L - 1);
  }
}

// Forward theta matrix into half-complex slices: c_w = (1/p) sum_l f_l e^{-i w theta_l},
// theta_l = (2l - p) pi / p; rows 0, (2w-1, 2w) = (Re, Im) of c_w, p-1 = Nyquist.
__global__ void fill_theta_forward(double *W, int p) {
  const int total = p * p, h = p / 2;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int s = e / p, l = e - s * p;
    double v;
    if (s == 0) {
      v = 1.0;
    } else if (s == p - 1) {
      v = cospi_frac((long long)h * (2 * l - p), p);
    } else {
      const int w = (s + 1) / 2;
      v = (s & 1) ? cospi_frac((long long)w * (2 * l - p), p) : -sinpi_frac((long long)w * (2 * l - p), p);
    }
    W[e] = v / p;
  }
}

}  // namespace

extern "C" cyl_status cyl_vals2coeffs_noalloc(int n_r, int n_z, int n_theta, const double *vals, double *coeffs,
                                              void *stream) {
  if (!vals || !coeffs) return CYL_EINVAL;
  if (n_r < 2 || n_z < 2 || n_theta < 2 || (n_theta & 1)) return CYL_EINVAL;
  const long long m = n_r, n = n_z, p = n_theta, N = m * n * p;
  const long long need = 2 * N + m * m + n * n + p * p;
  if (need > (long long)CYL_NOALLOC_SCRATCH_DOUBLES) return CYL_EINVAL;
  // a launch error left pending by the caller's earlier work would otherwise
  // be read back below as a failure of this call: report it before launching
  if (cudaPeekAtLastError() != cudaSuccess) return CYL_ECUDA;
  double *base = nullptr;
  cudaError_t e = scratch_for_current_context(&base);
  if (e != cudaSuccess) return CYL_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double *buf0 = base, *buf1 = base + N;
  double *Wz = buf1 + N, *Wr = Wz + n * n, *Wt = Wr + m * m;
  // Every scratch element that is read below is written earlier in this call,
  // so nothing left by a previous call needs clearing.
  fill_cheb_forward<<<(int)((n * n + 255) / 256), 256, 0, st>>>(Wz, (int)n);
  fill_cheb_forward<<<(int)((m * m + 255) / 256), 256, 0, st>>>(Wr, (int)m);
  fill_theta_forward<<<(int)((p * p + 255) / 256), 256, 0, st>>>(Wt, (int)p);
  if ((e = cudaGetLastError()) != cudaSuccess) return CYL_ECUDA;
  if ((e = cyl::launch_axis_matvec(vals, buf0, Wz, p * m, (int)n, 1, st)) != cudaSuccess) return CYL_ECUDA;
  if ((e = cyl::launch_axis_matvec(buf0, buf1, Wr, p, (int)m, n, st)) != cudaSuccess) return CYL_ECUDA;
  if ((e = cyl::launch_axis_matvec(buf1, coeffs, Wt, 1, (int)p, m * n, st)) != cudaSuccess) return CYL_ECUDA;
  return CYL_OK;
}
