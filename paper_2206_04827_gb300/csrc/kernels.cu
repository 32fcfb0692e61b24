// Device kernels of libcyl (sm_103a, FP64 throughout).
//
// adi_kernel        one CTA per work item (one or two half-complex slices x one
//                   radial parity class x one vertical parity class) runs the
//                   whole time loop of its item: right-hand-side assembly of
//                   eq. HelmholtzMatEqn, J iterations of Algorithm 1 and the
//                   Dirichlet expansion X = S_r Y S_z^T, with the work arrays
//                   resident in shared memory.
// axis_matvec       dense value <-> coefficient transform along one axis
//                   (Section 2: DCT-I in r and z, DFT in theta).
//
// GB300 facts that shape the ADI kernel: FP64 runs at 2 FMA/clk/SM (one warp
// instruction occupies an SM sub-partition's FP64 pipe for 64 cycles), so a
// single warp per sub-partition saturates the pipe even on a dependent chain,
// and memory traffic is an order of magnitude below the arithmetic time.  The
// kernel therefore minimises FP64 instructions per element (12 in the radial
// sweep, 8 in the vertical sweep, see plan.hpp for the pre-scaled factors)
// and keeps every sweep sequential per thread: a thread owns one column in
// the radial phase and one row in the vertical phase.
#include <cstdio>

#include "kernels.cuh"

namespace cyl {

size_t adi_smem_bytes(int ld, int smem_rows, int maxM, int maxNz, bool arrays_in_smem) {
  size_t d = (size_t)maxM * RSTRIDE + (size_t)maxNz * ZSTRIDE;
  if (arrays_in_smem) d += (size_t)smem_rows * ld + (size_t)maxM * ld;
  return d * sizeof(double);
}

// One ADI iteration of Algorithm 1 in the form
//   radial  : Z = (A - pC)^-1 [(q-p) E + (A - qC) U]        (U = X_j (D + pB)^T)
//   vertical: X_{j+1} = Z (D + qB)^-T,  U' = X_{j+1} (D + p'B)^T
// which is the paper's two half-steps (with the signs corrected so that the
// fixed point solves A X B^T + C X D^T = E) after eliminating the C solve.
__device__ __forceinline__ void radial_sweep(double *__restrict__ col, const double *__restrict__ Fc, int ld,
                                             const double *__restrict__ RB, int M, bool first) {
  double w0 = 0.0, w1 = 0.0, w2 = 0.0, w3 = 0.0, w4 = 0.0, w5;
  if (!first) {
    if (M > 0) w2 = col[0];
    if (M > 1) w3 = col[ld];
    if (M > 2) w4 = col[2 * ld];
  }
  double y1 = 0.0, y2 = 0.0;
  for (int i = 0; i < M; ++i) {
    const double *rb = RB + i * RSTRIDE;
    double acc = Fc[(size_t)i * ld];
    if (!first) {
      w5 = (i + 3 < M) ? col[(size_t)(i + 3) * ld] : 0.0;
      acc = fma(rb[0], w0, acc);
      acc = fma(rb[1], w1, acc);
      acc = fma(rb[2], w2, acc);
      acc = fma(rb[3], w3, acc);
      acc = fma(rb[4], w4, acc);
      acc = fma(rb[5], w5, acc);
      w0 = w1; w1 = w2; w2 = w3; w3 = w4; w4 = w5;
    }
    acc = fma(rb[6], y1, acc);
    acc = fma(rb[7], y2, acc);
    col[(size_t)i * ld] = acc;
    y2 = y1;
    y1 = acc;
  }
  double z1 = 0.0, z2 = 0.0, z3 = 0.0;
  for (int i = M - 1; i >= 0; --i) {
    const double *rb = RB + i * RSTRIDE;
    double acc = col[(size_t)i * ld];
    acc = fma(rb[8], z1, acc);
    acc = fma(rb[9], z2, acc);
    acc = fma(rb[10], z3, acc);
    const double zi = acc * rb[11];
    col[(size_t)i * ld] = zi;
    z3 = z2; z2 = z1; z1 = zi;
  }
}

__device__ __forceinline__ void vertical_sweep(double *__restrict__ row, const double *__restrict__ ZB, int Nz,
                                               bool last) {
  double w = 0.0;
  for (int b = 0; b < Nz; ++b) {
    w = fma(ZB[b * ZSTRIDE + 0], w, row[b]);
    row[b] = w;
  }
  double x1 = 0.0, x2 = 0.0, x3 = 0.0;
  for (int b = Nz - 1; b >= 0; --b) {
    const double *zb = ZB + b * ZSTRIDE;
    double v = row[b];
    v = fma(zb[1], x1, v);
    v = fma(zb[2], x2, v);
    const double xb = v * zb[3];
    if (last) {
      row[b] = xb;
    } else if (b + 1 < Nz) {
      const double *zn = zb + ZSTRIDE;
      double u = zn[4] * xb;
      u = fma(zn[5], x1, u);
      u = fma(zn[6], x2, u);
      u = fma(zn[7], x3, u);
      row[b + 1] = u;
    }
    x3 = x2; x2 = x1; x1 = xb;
  }
  if (!last && Nz > 0) {
    double u = ZB[5] * x1;
    u = fma(ZB[6], x2, u);
    u = fma(ZB[7], x3, u);
    row[0] = u;
  }
}

__global__ void __launch_bounds__(1024) adi_kernel(const AdiArgs a) {
  extern __shared__ __align__(16) double sm[];
  const Item it = a.items[blockIdx.x];
  const int tid = threadIdx.x, nth = blockDim.x;
  const int M = it.M, Nz = it.Nz, nsl = it.nsl, W = nsl * Nz;
  const int ld = a.ld;
  const int m = a.m, n = a.n;
  const long long slice = (long long)m * n;
  double *RB = sm;
  double *ZB = RB + (size_t)a.maxM * RSTRIDE;
  double *S, *Fa;
  if (a.use_smem) {
    S = ZB + (size_t)a.maxNz * ZSTRIDE;
  } else {
    S = a.gwork + (size_t)blockIdx.x * a.gwork_per_item;
  }
  Fa = S + (size_t)a.smem_rows * ld;
  const double *r2 = a.fac + it.r2off;
  const double *c02 = a.fac + it.c02off;

  const double *Xsrc = a.Xin;
  for (int step = 0; step < a.nsteps; ++step) {
    const double *Gs = a.G ? a.G + (size_t)step * a.gstride : nullptr;
    // Right side of eq. HelmholtzMatEqn, E = trunc(R_2 (X + kappa g) C02^T), in two
    // banded passes: T1 = (X + kappa g) C02^T on the class rows, then E = R_2 T1.
    for (int e = tid; e < it.Mfull * W; e += nth) {
      const int ap = e / W, c = e - ap * W;
      const int sl = c / Nz, b = c - sl * Nz;
      const int i = it.pr + 2 * ap, j = it.pz + 2 * b;
      const size_t base = (size_t)(it.s0 + sl) * slice + (size_t)i * n;
      double acc = 0.0;
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        const int jj = j + 2 * t;
        if (jj < n) {
          double z = Xsrc[base + jj];
          if (Gs) z = fma(a.kappa, Gs[base + jj], z);
          acc = fma(c02[b * C02STRIDE + t], z, acc);
        }
      }
      S[(size_t)ap * ld + c] = acc;
    }
    __syncthreads();
    for (int e = tid; e < M * W; e += nth) {
      const int aa = e / W, c = e - aa * W;
      double acc = 0.0;
#pragma unroll
      for (int s = -1; s <= 3; ++s) {
        const int q = aa + s;
        if (q >= 0 && q < it.Mfull) acc = fma(r2[aa * R2STRIDE + s + 1], S[(size_t)q * ld + c], acc);
      }
      Fa[(size_t)aa * ld + c] = acc;
    }
    __syncthreads();

    // Algorithm 1, J iterations, from X_0 = 0.
    for (int jt = 0; jt < it.J; ++jt) {
      const double *rsrc = a.fac + it.roff + (size_t)jt * M * RSTRIDE;
      const double *zsrc = a.fac + it.zoff + (size_t)jt * Nz * ZSTRIDE;
      for (int e = tid; e < M * RSTRIDE; e += nth) RB[e] = rsrc[e];
      for (int e = tid; e < Nz * ZSTRIDE; e += nth) ZB[e] = zsrc[e];
      __syncthreads();
      if (tid < W) radial_sweep(S + tid, Fa + tid, ld, RB, M, jt == 0);
      __syncthreads();
      if (tid < nsl * M) {
        const int sl = tid / M, aa = tid - sl * M;
        vertical_sweep(S + (size_t)aa * ld + sl * Nz, ZB, Nz, jt + 1 == it.J);
      }
      __syncthreads();
    }

    // X = S_r Y S_z^T on this item's class rows / columns (phi_j = T_{j+2} - T_j).
    const int Wf = nsl * it.Nzfull;
    const bool do_ck = a.ckpt && ((step + 1) % a.ckpt_every == 0);
    double *ck = do_ck ? a.ckpt + (size_t)((step + 1) / a.ckpt_every) * (size_t)a.p * slice : nullptr;
    for (int e = tid; e < it.Mfull * Wf; e += nth) {
      const int ap = e / Wf, cc = e - ap * Wf;
      const int sl = cc / it.Nzfull, b = cc - sl * it.Nzfull;
      const double *Ys = S + sl * Nz;
      const bool r0 = ap - 1 >= 0, r1 = ap < M, c0 = b - 1 >= 0, c1 = b < Nz;
      double x = 0.0;
      if (r0 && c0) x += Ys[(size_t)(ap - 1) * ld + b - 1];
      if (r0 && c1) x -= Ys[(size_t)(ap - 1) * ld + b];
      if (r1 && c0) x -= Ys[(size_t)ap * ld + b - 1];
      if (r1 && c1) x += Ys[(size_t)ap * ld + b];
      const size_t o = (size_t)(it.s0 + sl) * slice + (size_t)(it.pr + 2 * ap) * n + it.pz + 2 * b;
      a.Xout[o] = x;
      if (ck) ck[o] = x;
    }
    if (a.zero_other) {
      const int po = 1 - it.pr, Mo = (m - po + 1) / 2;
      for (int e = tid; e < Mo * Wf; e += nth) {
        const int ap = e / Wf, cc = e - ap * Wf;
        const int sl = cc / it.Nzfull, b = cc - sl * it.Nzfull;
        const size_t o = (size_t)(it.s0 + sl) * slice + (size_t)(po + 2 * ap) * n + it.pz + 2 * b;
        a.Xout[o] = 0.0;
        if (ck) ck[o] = 0.0;
      }
    }
    __syncthreads();
    Xsrc = a.Xout;
  }
}

cudaError_t launch_adi(const AdiArgs &a, int threads, size_t smem, cudaStream_t st) {
  if (a.nitems <= 0 || a.nsteps <= 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(adi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  adi_kernel<<<a.nitems, threads, smem, st>>>(a);
  return cudaGetLastError();
}

__global__ void axis_matvec_kernel(const double *__restrict__ in, double *__restrict__ out,
                                   const double *__restrict__ W, long long outer, int L, long long inner) {
  const long long total = outer * L * inner;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e % inner;
    const long long r = e / inner;
    const int j = (int)(r % L);
    const long long o = r / L;
    const double *src = in + o * L * inner + i;
    const double *w = W + (size_t)j * L;
    double acc = 0.0;
    for (int t = 0; t < L; ++t) acc = fma(w[t], src[(size_t)t * inner], acc);
    out[e] = acc;
  }
}

cudaError_t launch_axis_matvec(const double *in, double *out, const double *W, long long outer, int L,
                               long long inner, cudaStream_t st) {
  const long long total = outer * L * inner;
  if (total <= 0) return cudaSuccess;
  const int threads = 256;
  long long blocks = (total + threads - 1) / threads;
  if (blocks > 152LL * 16) blocks = 152LL * 16;
  axis_matvec_kernel<<<(int)blocks, threads, 0, st>>>(in, out, W, outer, L, inner);
  return cudaGetLastError();
}

}  // namespace cyl
