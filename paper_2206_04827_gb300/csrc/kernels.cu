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
  size_t d = 2 * ((size_t)maxM * RSTRIDE + (size_t)maxNz * ZSTRIDE);   // double-buffered factor tables
  if (arrays_in_smem) d += (size_t)smem_rows * ld + (size_t)maxM * ld;
  return d * sizeof(double);
}

// ------------------------------------------------------------------ TMA / mbarrier
__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// One elected thread: announce `bytes` of transaction and start bulk copies.
__device__ __forceinline__ void mbar_expect(unsigned long long *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// Bounded wait on an mbarrier phase; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity) {
  for (unsigned it = 0; it < (1u << 24); ++it) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// One ADI iteration of Algorithm 1 in the form
//   radial  : Z = (A - pC)^-1 [(q-p) E + (A - qC) U]        (U = X_j (D + pB)^T)
//   vertical: X_{j+1} = Z (D + qB)^-T,  U' = X_{j+1} (D + p'B)^T
// which is the paper's two half-steps (with the signs corrected so that the
// fixed point solves A X B^T + C X D^T = E) after eliminating the C solve.
//
// Every sweep loads the operands of the next row (column) one step ahead
// into registers: with one warp per SM sub-partition an exposed shared-memory
// latency idles the FP64 pipe, which is the only resource that matters here.
template <bool FIRST>
__device__ __forceinline__ void radial_sweep(double *__restrict__ col, const double *__restrict__ Fc, int ld,
                                             const double *__restrict__ RB, int M) {
  double w0 = 0.0, w1 = 0.0, w2 = 0.0, w3 = 0.0, w4 = 0.0;
  if (!FIRST) {
    if (M > 0) w2 = col[0];
    if (M > 1) w3 = col[ld];
    if (M > 2) w4 = col[2 * ld];
  }
  double fn = M > 0 ? Fc[0] : 0.0;
  double un = (!FIRST && M > 3) ? col[3 * ld] : 0.0;
  const double2 *rb2 = reinterpret_cast<const double2 *>(RB);
  double2 n01 = rb2[0], n23 = rb2[1], n45 = rb2[2], n67 = rb2[3];
  double y1 = 0.0, y2 = 0.0;
  for (int i = 0; i < M; ++i) {
    const double f = fn, w5 = un;
    const double2 a01 = n01, a23 = n23, a45 = n45, a67 = n67;
    if (i + 1 < M) {
      fn = Fc[(i + 1) * ld];
      if (!FIRST) un = (i + 4 < M) ? col[(i + 4) * ld] : 0.0;
      const double2 *nx = rb2 + (i + 1) * (RSTRIDE / 2);
      if (!FIRST) { n01 = nx[0]; n23 = nx[1]; n45 = nx[2]; }
      n67 = nx[3];
    }
    double acc = f;
    if (!FIRST) {
      acc = fma(a01.x, w0, acc);
      acc = fma(a01.y, w1, acc);
      acc = fma(a23.x, w2, acc);
      acc = fma(a23.y, w3, acc);
      acc = fma(a45.x, w4, acc);
      acc = fma(a45.y, w5, acc);
      w0 = w1; w1 = w2; w2 = w3; w3 = w4; w4 = w5;
    }
    acc = fma(a67.x, y1, acc);
    acc = fma(a67.y, y2, acc);
    col[i * ld] = acc;
    y2 = y1;
    y1 = acc;
  }
  double z1 = 0.0, z2 = 0.0, z3 = 0.0;
  if (M <= 0) return;
  double yn = col[(M - 1) * ld];
  double2 b89 = rb2[(M - 1) * (RSTRIDE / 2) + 4], bab = rb2[(M - 1) * (RSTRIDE / 2) + 5];
  for (int i = M - 1; i >= 0; --i) {
    const double y = yn;
    const double2 c89 = b89, cab = bab;
    if (i > 0) {
      yn = col[(i - 1) * ld];
      b89 = rb2[(i - 1) * (RSTRIDE / 2) + 4];
      bab = rb2[(i - 1) * (RSTRIDE / 2) + 5];
    }
    double acc = fma(c89.x, z1, y);
    acc = fma(c89.y, z2, acc);
    acc = fma(cab.x, z3, acc);
    const double zi = acc * cab.y;
    col[i * ld] = zi;
    z3 = z2; z2 = z1; z1 = zi;
  }
}

template <bool LAST>
__device__ __forceinline__ void vertical_sweep(double *__restrict__ row, const double *__restrict__ ZB, int Nz) {
  if (Nz <= 0) return;
  double w = 0.0;
  double rn = row[0], cn = ZB[0];
  for (int b = 0; b < Nz; ++b) {
    const double r = rn, c = cn;
    if (b + 1 < Nz) {
      rn = row[b + 1];
      cn = ZB[(b + 1) * ZSTRIDE];
    }
    w = fma(c, w, r);
    row[b] = w;
  }
  const double2 *z2p = reinterpret_cast<const double2 *>(ZB);
  double x1 = 0.0, x2 = 0.0, x3 = 0.0;
  double2 p01 = z2p[(Nz - 1) * 4], p23 = z2p[(Nz - 1) * 4 + 1], p45, p67;
  if (!LAST) { p45 = z2p[(Nz - 1) * 4 + 2]; p67 = z2p[(Nz - 1) * 4 + 3]; }
  double wn = row[Nz - 1];
  double ap0 = 0.0, ap1 = 0.0, ap2 = 0.0, ap3 = 0.0;   // apply band of column b + 1
  for (int b = Nz - 1; b >= 0; --b) {
    const double wb = wn;
    const double2 c01 = p01, c23 = p23;
    double2 c45, c67;
    if (!LAST) { c45 = p45; c67 = p67; }
    if (b > 0) {
      wn = row[b - 1];
      p01 = z2p[(b - 1) * 4];
      p23 = z2p[(b - 1) * 4 + 1];
      if (!LAST) { p45 = z2p[(b - 1) * 4 + 2]; p67 = z2p[(b - 1) * 4 + 3]; }
    }
    double v = fma(c01.y, x1, wb);
    v = fma(c23.x, x2, v);
    const double xb = v * c23.y;
    if (LAST) {
      row[b] = xb;
    } else {
      if (b + 1 < Nz) {
        double u = ap0 * xb;
        u = fma(ap1, x1, u);
        u = fma(ap2, x2, u);
        u = fma(ap3, x3, u);
        row[b + 1] = u;
      }
      ap0 = c45.x; ap1 = c45.y; ap2 = c67.x; ap3 = c67.y;
    }
    x3 = x2; x2 = x1; x1 = xb;
  }
  if (!LAST) {
    double u = ap1 * x1;
    u = fma(ap2, x2, u);
    u = fma(ap3, x3, u);
    row[0] = u;
  }
}

template <bool SMEM>
__global__ void __launch_bounds__(1024) adi_kernel(const AdiArgs a) {
  extern __shared__ __align__(16) double sm[];
  __shared__ __align__(8) unsigned long long bar[2];
  const Item it = a.items[blockIdx.x];
  const int tid = threadIdx.x, nth = blockDim.x;
  const int M = it.M, Nz = it.Nz, nsl = it.nsl, W = nsl * Nz;
  const int ld = a.ld;
  const int m = a.m, n = a.n;
  const long long slice = (long long)m * n;
  const int rlen = a.maxM * RSTRIDE, zlen = a.maxNz * ZSTRIDE;
  double *RB0 = sm;                       // [2][maxM * RSTRIDE]
  double *ZB0 = sm + 2 * rlen;            // [2][maxNz * ZSTRIDE]
  double *S, *Fa;
  if (SMEM) {
    S = ZB0 + 2 * zlen;
  } else {
    S = a.gwork + (size_t)blockIdx.x * a.gwork_per_item;
  }
  Fa = S + (size_t)a.smem_rows * ld;
  const double *r2 = a.fac + it.r2off;
  const double *c02 = a.fac + it.c02off;
  const unsigned rbytes = (unsigned)(M * RSTRIDE * sizeof(double));
  const unsigned zbytes = (unsigned)(Nz * ZSTRIDE * sizeof(double));
  const int J = it.J;
  const long long total_it = (long long)a.nsteps * J;

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // Factor tables of ADI iteration c (c counts iterations over all steps) go to
  // buffer c & 1 by one bulk copy per table; iteration c + 1 is fetched while
  // iteration c computes.
  auto issue = [&](long long c) {
    const int jt = (int)(c % J), buf = (int)(c & 1);
    mbar_expect(&bar[buf], rbytes + zbytes);
    bulk_g2s(RB0 + buf * rlen, a.fac + it.roff + (size_t)jt * M * RSTRIDE, rbytes, &bar[buf]);
    bulk_g2s(ZB0 + buf * zlen, a.fac + it.zoff + (size_t)jt * Nz * ZSTRIDE, zbytes, &bar[buf]);
  };
  if (tid == 0) issue(0);
  bool timed_out = false;

  const double *Xsrc = a.Xin;
  long long c = 0;
  for (int step = 0; step < a.nsteps; ++step) {
    const double *Gs = a.G ? a.G + (size_t)step * a.gstride : nullptr;
    // Right side of eq. HelmholtzMatEqn, E = trunc(R_2 (X + kappa g) C02^T), in two
    // banded passes: T1 = (X + kappa g) C02^T on the class rows, then E = R_2 T1.
    for (int e = tid; e < it.Mfull * W; e += nth) {
      const int ap = e / W, cc = e - ap * W;
      const int sl = cc / Nz, b = cc - sl * Nz;
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
      S[ap * ld + cc] = acc;
    }
    __syncthreads();
    for (int e = tid; e < M * W; e += nth) {
      const int aa = e / W, cc = e - aa * W;
      double acc = 0.0;
#pragma unroll
      for (int s = -1; s <= 3; ++s) {
        const int q = aa + s;
        if (q >= 0 && q < it.Mfull) acc = fma(r2[aa * R2STRIDE + s + 1], S[q * ld + cc], acc);
      }
      Fa[aa * ld + cc] = acc;
    }
    __syncthreads();

    // Algorithm 1, J iterations, from X_0 = 0.
    for (int jt = 0; jt < J; ++jt, ++c) {
      const int buf = (int)(c & 1);
      if (tid == 0 && c + 1 < total_it) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(c + 1);
      }
      if (!mbar_wait(&bar[buf], (unsigned)((c >> 1) & 1))) timed_out = true;
      const double *RB = RB0 + buf * rlen;
      const double *ZB = ZB0 + buf * zlen;
      if (tid < W) {
        if (jt == 0) radial_sweep<true>(S + tid, Fa + tid, ld, RB, M);
        else radial_sweep<false>(S + tid, Fa + tid, ld, RB, M);
      }
      __syncthreads();
      if (tid < nsl * M) {
        const int sl = tid / M, aa = tid - sl * M;
        if (jt + 1 == J) vertical_sweep<true>(S + aa * ld + sl * Nz, ZB, Nz);
        else vertical_sweep<false>(S + aa * ld + sl * Nz, ZB, Nz);
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
      if (r0 && c0) x += Ys[(ap - 1) * ld + b - 1];
      if (r0 && c1) x -= Ys[(ap - 1) * ld + b];
      if (r1 && c0) x -= Ys[ap * ld + b - 1];
      if (r1 && c1) x += Ys[ap * ld + b];
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
  if (timed_out && a.err) atomicExch(a.err, (int)CYL_ERR_TIMEOUT);
}

cudaError_t launch_adi(const AdiArgs &a, int threads, size_t smem, cudaStream_t st) {
  if (a.nitems <= 0 || a.nsteps <= 0) return cudaSuccess;
  cudaError_t e;
  if (a.use_smem) {
    e = cudaFuncSetAttribute(adi_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    adi_kernel<true><<<a.nitems, threads, smem, st>>>(a);
  } else {
    e = cudaFuncSetAttribute(adi_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    adi_kernel<false><<<a.nitems, threads, smem, st>>>(a);
  }
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
