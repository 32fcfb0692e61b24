// FP64 issue-rate probe: the machine figure that the FP64 roofline of the
// ADI kernels divides by.  It is not part of the method; the solver never
// calls it.
//
// Every thread runs CH independent fused multiply-add chains x <- x*a + b
// (a just below 1, b small, so the values stay bounded), fully unrolled, for
// `iters` iterations.  With enough warps per SM sub-partition and CH
// independent chains per thread the FP64 pipe never waits for a result, so
// flops / elapsed time is the SM array's FP64 FMA throughput at the clock
// the GPU runs during the launch.
#include <cuda_runtime.h>

#include "../../include/cyl.h"

namespace {

template <int CH>
__global__ void __launch_bounds__(1024) fp64_fma_probe_kernel(double *sink, long long iters, double a, double b) {
  double x[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) x[c] = 1e-3 * threadIdx.x + c;
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += x[c];
  // never true for the probe's arguments; keeps the chains alive
  if (s == -1.0) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" cyl_status cyl_fp64_fma_probe(int blocks, int threads, long long iters, double *sink, double *flops,
                                         void *stream) {
  if (blocks < 1 || threads < 32 || threads > 1024 || (threads & 31) || iters < 1 || !sink || !flops)
    return CYL_EINVAL;
  constexpr int CH = 8;
  fp64_fma_probe_kernel<CH><<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(sink, iters,
                                                                                         1.0 - 1e-9, 1e-12);
  if (cudaGetLastError() != cudaSuccess) return CYL_ECUDA;
  *flops = 2.0 * CH * (double)iters * (double)threads * (double)blocks;
  return CYL_OK;
}
