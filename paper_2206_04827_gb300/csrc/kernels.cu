// Device kernels of libcyl (sm_103a, FP64 throughout).
//
// adi_kernel        one CTA per work item (one or two half-complex slices x one
//                   radial parity class x one vertical parity class) runs the
//                   whole time loop of its item: right-hand-side assembly of
//                   eq. HelmholtzMatEqn (BDF1, or delta^(b) over a history ring
//                   for BDF b, plus the lifting correction of Dirichlet data),
//                   J iterations of Algorithm 1 and the Dirichlet expansion
//                   X = S_r Y S_z^T, with the work arrays resident in shared
//                   memory where they fit.
// adi_batch_kernel  the same per item, for many problems: persistent CTAs of G
//                   thread groups pull items (largest first) from a queue.
// adi_adjoint_kernel  the transposed step map run backward over the steps
//                   (BDF1, or the multistep ring of BDF b), through the
//                   forward sweeps on index-reversed arrays.
// axis_matvec       dense value <-> coefficient transform along one axis
//                   (Section 2: DCT-I in r and z, DFT in theta).
// disk_poisson      the horizontal (disk) Poisson solve of Section 4.
// lift_*, permute_slots, sum_partials   boundary-data lifting, history / ring
//                   reordering, reduction of the per-item alpha-gradient parts.
//
// GB300 facts that shape the ADI kernel: FP64 runs at 2 FMA/clk/SM (one warp
// instruction occupies an SM sub-partition's FP64 pipe for 64 cycles) and the
// ADI work is an order of magnitude above the memory traffic, so the kernel
// minimises FP64 instructions per element (12 in the radial sweep, 8 in the
// vertical sweep, see plan.hpp for the pre-scaled factors) and keeps each
// banded solve sequential per thread.  A lone dependent FMA chain reaches the
// 64-cycle interval, but with the shared-memory loads around it one warp per
// sub-partition keeps the pipe busy only about 80 % of the time; a second warp
// lifts that to about 95 %.  Where a sweep has too few chains for two warps
// per sub-partition (grids up to about 130), each solve is split in two
// (twisted sweeps below), two threads per chain.
#include <cstdio>

#include <algorithm>

#include "kernels.cuh"

namespace cyl {

size_t adi_smem_bytes(int ld, int smem_rows, int maxM, int maxNz, int level, int twist_half) {
  // double-buffered factor tables (with the interface maps of twisted solves)
  size_t d = 2 * ((size_t)maxM * RSTRIDE + RTWIST + (size_t)maxNz * ZSTRIDE + ZTWIST);
  if (level >= 1) d += (size_t)smem_rows * ld;                         // iterate S
  if (level >= 2) d += (size_t)maxM * ld;                              // right side Fa
  d += (size_t)TW_SLOTS * twist_half;                                  // twisted-sweep exchange
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

// Bounded wait on an mbarrier phase: false once `limit` SM clock cycles have
// passed without the phase completing.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, long long limit) {
  const long long t0 = clock64();
  for (;;) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > limit) return false;
  }
}

// One ADI iteration of Algorithm 1 in the form
//   radial  : Z = (A - pC)^-1 [(q-p) E + (A - qC) U]        (U = X_j (D + pB)^T)
//   vertical: X_{j+1} = Z (D + qB)^-T,  U' = X_{j+1} (D + p'B)^T
// which is the paper's two half-steps (with the signs corrected so that the
// fixed point solves A X B^T + C X D^T = E) after eliminating the C solve.
// The adjoint's transposed system runs through the same sweeps (its records
// are those of the flipped transposes, on index-reversed arrays).
//
// Every sweep loads the operands of the next row (column) one step ahead
// into registers: with one warp per SM sub-partition an exposed shared-memory
// latency idles the FP64 pipe, which is the only resource that matters here.
template <int K>
__device__ __forceinline__ double comp(const double2 *a) {
  return (K & 1) ? a[K >> 1].y : a[K >> 1].x;
}

template <bool FIRST, int UNR>
__device__ __forceinline__ void radial_sweep(double *__restrict__ col, const double *__restrict__ Fc, int ld,
                                             const double *__restrict__ RB, int M) {
  constexpr int LO = 2, HI = 3;                             // apply band offsets [-LO, HI]
  constexpr int LBW = 2, UBW = 3;                           // L and U bandwidths
  constexpr int NF = 4;                                     // double2 words read going down ([0..7])
  constexpr int B0 = 4;                                     // first double2 word read going up ([8..11])
  constexpr int NB = RSTRIDE / 2 - B0;
  const double2 *rb2 = reinterpret_cast<const double2 *>(RB);
  double w[LO + HI + 1];
#pragma unroll
  for (int k = 0; k <= LO + HI; ++k) w[k] = 0.0;
  if (!FIRST) {
#pragma unroll
    for (int o = 0; o < HI; ++o) w[LO + o] = (o < M) ? col[o * ld] : 0.0;
  }
  double fn = Fc[0];
  double un = (!FIRST && HI < M) ? col[HI * ld] : 0.0;
  double2 nrec[NF];
#pragma unroll
  for (int k = 0; k < NF; ++k) nrec[k] = rb2[k];
  double y[LBW];
#pragma unroll
  for (int k = 0; k < LBW; ++k) y[k] = 0.0;
#pragma unroll UNR
  for (int i = 0; i < M; ++i) {
    const double f = fn;
    double2 rec[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) rec[k] = nrec[k];
    if (!FIRST) w[LO + HI] = un;
    if (i + 1 < M) {
      fn = Fc[(i + 1) * ld];
      if (!FIRST) un = (i + 1 + HI < M) ? col[(i + 1 + HI) * ld] : 0.0;
      const double2 *nx = rb2 + (i + 1) * (RSTRIDE / 2);
#pragma unroll
      for (int k = 0; k < NF; ++k)
        if (!FIRST || 2 * k + 1 >= 6) nrec[k] = nx[k];
    }
    double acc = f;
    if (!FIRST) {
      acc = fma(comp<0>(rec), w[0], acc);
      acc = fma(comp<1>(rec), w[1], acc);
      acc = fma(comp<2>(rec), w[2], acc);
      acc = fma(comp<3>(rec), w[3], acc);
      acc = fma(comp<4>(rec), w[4], acc);
      acc = fma(comp<5>(rec), w[5], acc);
#pragma unroll
      for (int k = 0; k < LO + HI; ++k) w[k] = w[k + 1];
    }
    // L terms, oldest first: only the last one waits for the previous row
    acc = fma(comp<7>(rec), y[1], acc);
    acc = fma(comp<6>(rec), y[0], acc);
    col[i * ld] = acc;
    y[1] = y[0];
    y[0] = acc;
  }
  double z[UBW];
#pragma unroll
  for (int u = 0; u < UBW; ++u) z[u] = 0.0;
  double yn = col[(M - 1) * ld];
  double2 nb[NB];
#pragma unroll
  for (int k = 0; k < NB; ++k) nb[k] = rb2[(M - 1) * (RSTRIDE / 2) + B0 + k];
#pragma unroll UNR
  for (int i = M - 1; i >= 0; --i) {
    const double yv = yn;
    double2 cb[NB];
#pragma unroll
    for (int k = 0; k < NB; ++k) cb[k] = nb[k];
    if (i > 0) {
      yn = col[(i - 1) * ld];
#pragma unroll
      for (int k = 0; k < NB; ++k) nb[k] = rb2[(i - 1) * (RSTRIDE / 2) + B0 + k];
    }
    // U terms carry the pivot; the newest value z_{i+1} enters last  ([8..10] -U/U_ii, [11] (q-p)/U_ii)
    double acc = comp<3>(cb) * yv;
    acc = fma(comp<2>(cb), z[2], acc);
    acc = fma(comp<1>(cb), z[1], acc);
    const double zi = fma(comp<0>(cb), z[0], acc);
    col[i * ld] = zi;
    z[2] = z[1];
    z[1] = z[0];
    z[0] = zi;
  }
}

template <bool LAST, int UNR>
__device__ __forceinline__ void vertical_sweep(double *__restrict__ row, const double *__restrict__ ZB, int Nz) {
  constexpr int ALO = 1;                                    // apply offsets [-1, 2]
  const double2 *z2p = reinterpret_cast<const double2 *>(ZB);
  double wq = 0.0;
  double rn = row[0];
  double2 cn = z2p[0];
#pragma unroll UNR
  for (int b = 0; b < Nz; ++b) {
    const double r = rn;
    const double2 c = cn;
    if (b + 1 < Nz) {
      rn = row[b + 1];
      cn = z2p[(b + 1) * 4];
    }
    const double w = fma(c.x, wq, r);                       // [0] -L[c][c-1]
    row[b] = w;
    wq = w;
  }
  double x1 = 0.0, x2 = 0.0, x3 = 0.0;                      // x_{b+1}, x_{b+2}, x_{b+3}
  double2 p01 = z2p[(Nz - 1) * 4], p23 = z2p[(Nz - 1) * 4 + 1], p45, p67;
  if (!LAST) { p45 = z2p[(Nz - 1) * 4 + 2]; p67 = z2p[(Nz - 1) * 4 + 3]; }
  double wn = row[Nz - 1];
  double2 q45 = make_double2(0.0, 0.0), q67 = make_double2(0.0, 0.0);   // apply record of column b+1
#pragma unroll UNR
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
    // U terms carry the pivot; the newest value x_{b+1} enters last ([1..2] -U/U_cc, [3] 1/U_cc)
    const double v = fma(c23.x, x2, c23.y * wb);
    const double xb = fma(c01.y, x1, v);
    if (LAST) {
      row[b] = xb;
    } else {
      if (b + ALO < Nz) {
        double u = q67.y * x3;
        u = fma(q67.x, x2, u);
        u = fma(q45.y, x1, u);
        u = fma(q45.x, xb, u);
        row[b + ALO] = u;
      }
      q45 = c45;
      q67 = c67;
    }
    x3 = x2; x2 = x1; x1 = xb;
  }
  if (!LAST) {              // column 0 (x_{-1} = 0); q holds column 0's apply record
    double u = q45.y * x1;
    u = fma(q67.x, x2, u);
    u = fma(q67.y, x3, u);
    row[0] = u;
  }
}

// ------------------------------------------------------------------ twisted sweeps
// A banded solve split in two chains that run on two threads (in different
// warps): LU elimination top-down over rows < k and UL elimination bottom-up
// over rows > k + w - 1, then a small interface system (rows k .. k+w-1,
// precomputed map in the table tail), then the two back substitutions
// outward.  Same FP64 work as one LU sweep, half the chain length, twice the
// warps: on GB300 a second warp per SM sub-partition lifts the sweep from
// about 0.80 to about 0.95 of the FP64 pipe.  Records: plan.hpp.  Scratch
// slots (stride xs_stride): radial 0..1 w_{k-2}, w_{k-1}; 2..4 top partial
// interface right sides; 5..7 v_{k+3..k+5}; 8..10 bottom partials.
// Vertical 0 w_{k-1}; 1..2 z_k, z_{k+1}; 3..4 v_{k+2}, v_{k+3}.

// Radial phase 1: top: interface partials (f + apply terms on U rows <= k+2)
// then forward LU rows 0 .. k-1; bottom: interface partials (apply terms on
// U rows >= k+3) then forward UL rows M-1 .. k+3.  In place on col.
template <bool FIRST, int UNR>
__device__ __forceinline__ void radial_tw1(double *__restrict__ col, const double *__restrict__ Fc, int ld,
                                           const double *__restrict__ RB, int M, int k, bool bottom,
                                           double *__restrict__ xs, int xst) {
  const double2 *rb2 = reinterpret_cast<const double2 *>(RB);
  if (!bottom) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      double acc = Fc[(k + r) * ld];
      if (!FIRST) {
        const double *rec = RB + (k + r) * RSTRIDE;
#pragma unroll
        for (int o = -2; o <= 2 - r; ++o) acc = fma(rec[o + 2], col[(k + r + o) * ld], acc);
      }
      xs[(2 + r) * xst] = acc;
    }
    // forward LU rows 0 .. k-1 (as radial_sweep's first loop, stopped at k)
    double w[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) w[q] = 0.0;
    if (!FIRST) {
#pragma unroll
      for (int o = 0; o < 3; ++o) w[2 + o] = col[o * ld];
    }
    double fn = Fc[0];
    double un = FIRST ? 0.0 : col[3 * ld];
    double2 nrec[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) nrec[q] = rb2[q];
    double y0 = 0.0, y1 = 0.0;
#pragma unroll UNR
    for (int i = 0; i < k; ++i) {
      const double f = fn;
      double2 rec[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) rec[q] = nrec[q];
      if (!FIRST) w[5] = un;
      if (i + 1 < k) {
        fn = Fc[(i + 1) * ld];
        if (!FIRST) un = col[(i + 4) * ld];
        const double2 *nx = rb2 + (i + 1) * (RSTRIDE / 2);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (!FIRST || q == 3) nrec[q] = nx[q];
      }
      double acc = f;
      if (!FIRST) {
        acc = fma(comp<0>(rec), w[0], acc);
        acc = fma(comp<1>(rec), w[1], acc);
        acc = fma(comp<2>(rec), w[2], acc);
        acc = fma(comp<3>(rec), w[3], acc);
        acc = fma(comp<4>(rec), w[4], acc);
        acc = fma(comp<5>(rec), w[5], acc);
#pragma unroll
        for (int q = 0; q < 5; ++q) w[q] = w[q + 1];
      }
      acc = fma(comp<7>(rec), y1, acc);
      acc = fma(comp<6>(rec), y0, acc);
      col[i * ld] = acc;
      y1 = y0;
      y0 = acc;
    }
    xs[0] = y1;          // w_{k-2}
    xs[xst] = y0;        // w_{k-1}
  } else {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      double acc = 0.0;
      if (!FIRST) {
        const double *rec = RB + (k + r) * RSTRIDE;
#pragma unroll
        for (int o = 3 - r; o <= 3; ++o) acc = fma(rec[o + 2], col[(k + r + o) * ld], acc);
      }
      xs[(8 + r) * xst] = acc;
    }
    // forward UL rows M-1 .. k+3; wv holds the original U_{i-2} .. U_{i+3}
    double wv[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) wv[q] = 0.0;
    if (!FIRST) {
      wv[0] = col[(M - 3) * ld];
      wv[1] = col[(M - 2) * ld];
      wv[2] = col[(M - 1) * ld];
    }
    double fn = Fc[(M - 1) * ld];
    double un = FIRST ? 0.0 : col[(M - 4) * ld];
    double2 nrec[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) nrec[q] = rb2[(M - 1) * (RSTRIDE / 2) + q];
    double v1 = 0.0, v2 = 0.0, v3 = 0.0;      // v_{i+1}, v_{i+2}, v_{i+3}
#pragma unroll UNR
    for (int i = M - 1; i >= k + 3; --i) {
      const double f = fn;
      double2 rec[5];
#pragma unroll
      for (int q = 0; q < 5; ++q) rec[q] = nrec[q];
      const double unext = un;
      if (i - 1 >= k + 3) {
        fn = Fc[(i - 1) * ld];
        if (!FIRST) un = col[(i - 4) * ld];
        const double2 *nx = rb2 + (i - 1) * (RSTRIDE / 2);
#pragma unroll
        for (int q = 0; q < 5; ++q)
          if (!FIRST || q >= 3) nrec[q] = nx[q];
      }
      double acc = f;
      if (!FIRST) {
        acc = fma(comp<5>(rec), wv[5], acc);
        acc = fma(comp<4>(rec), wv[4], acc);
        acc = fma(comp<3>(rec), wv[3], acc);
        acc = fma(comp<2>(rec), wv[2], acc);
        acc = fma(comp<1>(rec), wv[1], acc);
        acc = fma(comp<0>(rec), wv[0], acc);
#pragma unroll
        for (int q = 5; q > 0; --q) wv[q] = wv[q - 1];
        wv[0] = unext;
      }
      acc = fma(comp<8>(rec), v3, acc);
      acc = fma(comp<7>(rec), v2, acc);
      acc = fma(comp<6>(rec), v1, acc);
      col[i * ld] = acc;
      v3 = v2;
      v2 = v1;
      v1 = acc;
    }
    xs[5 * xst] = v1;    // v_{k+3}
    xs[6 * xst] = v2;    // v_{k+4}
    xs[7 * xst] = v3;    // v_{k+5}
  }
}

// Radial phase 2: interface unknowns z_k .. z_{k+2} from the 3 x 8 map (both
// threads, from scratch), then the back substitutions outward.
template <int UNR>
__device__ __forceinline__ void radial_tw2(double *__restrict__ col, int ld, const double *__restrict__ RB, int M,
                                           int k, bool bottom, const double *__restrict__ xs, int xst) {
  const double *R = RB + M * RSTRIDE;
  double rhs[8];
  rhs[0] = xs[0];
  rhs[1] = xs[xst];
#pragma unroll
  for (int r = 0; r < 3; ++r) rhs[2 + r] = xs[(2 + r) * xst] + xs[(8 + r) * xst];
#pragma unroll
  for (int r = 0; r < 3; ++r) rhs[5 + r] = xs[(5 + r) * xst];
  double zI[3];
#pragma unroll
  for (int o = 0; o < 3; ++o) {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) s = fma(R[o * 8 + q], rhs[q], s);
    zI[o] = s;
  }
  const double2 *rb2 = reinterpret_cast<const double2 *>(RB);
  if (!bottom) {
#pragma unroll
    for (int o = 0; o < 3; ++o) col[(k + o) * ld] = zI[o];
    // back substitution rows k-1 .. 0 (LU records [8..11])
    double z0 = zI[0], z1 = zI[1], z2 = zI[2];
    double yn = col[(k - 1) * ld];
    double2 nb[2];
    nb[0] = rb2[(k - 1) * (RSTRIDE / 2) + 4];
    nb[1] = rb2[(k - 1) * (RSTRIDE / 2) + 5];
#pragma unroll UNR
    for (int i = k - 1; i >= 0; --i) {
      const double yv = yn;
      const double2 c0 = nb[0], c1 = nb[1];
      if (i > 0) {
        yn = col[(i - 1) * ld];
        nb[0] = rb2[(i - 1) * (RSTRIDE / 2) + 4];
        nb[1] = rb2[(i - 1) * (RSTRIDE / 2) + 5];
      }
      double acc = c1.y * yv;                 // (q-p)/U_ii
      acc = fma(c1.x, z2, acc);               // -U[i][i+3]/U_ii
      acc = fma(c0.y, z1, acc);               // -U[i][i+2]/U_ii
      const double zi = fma(c0.x, z0, acc);   // -U[i][i+1]/U_ii
      col[i * ld] = zi;
      z2 = z1;
      z1 = z0;
      z0 = zi;
    }
  } else {
    // forward substitution rows k+3 .. M-1 (UL records [9..11])
    double zm1 = zI[2], zm2 = zI[1];
    double vn = col[(k + 3) * ld];
    double2 nb[2];
    nb[0] = rb2[(k + 3) * (RSTRIDE / 2) + 4];
    nb[1] = rb2[(k + 3) * (RSTRIDE / 2) + 5];
#pragma unroll UNR
    for (int i = k + 3; i < M; ++i) {
      const double vv = vn;
      const double2 c0 = nb[0], c1 = nb[1];
      if (i + 1 < M) {
        vn = col[(i + 1) * ld];
        nb[0] = rb2[(i + 1) * (RSTRIDE / 2) + 4];
        nb[1] = rb2[(i + 1) * (RSTRIDE / 2) + 5];
      }
      double acc = c1.y * vv;                 // (q-p)/Lt_ii
      acc = fma(c1.x, zm2, acc);              // -Lt[i][i-2]/Lt_ii
      const double zi = fma(c0.y, zm1, acc);  // -Lt[i][i-1]/Lt_ii
      col[i * ld] = zi;
      zm2 = zm1;
      zm1 = zi;
    }
  }
}

// Vertical phase 1: top: save z_k, z_{k+1}, forward LU columns 0 .. k-1;
// bottom: forward UL columns Nz-1 .. k+2.  In place on row.  The vertical
// sweeps walk one row per thread, so each step's load is a separate 32-byte
// sector per thread; the row values are read six columns ahead into a queue
// of named registers (q0 .. q5), which keeps the next sectors' loads in
// flight across the steps that use the previous one.  Measured on GB300 at
// 512^3 with the work arrays in global memory (all-twisted kernel): 0.81 /
// 0.80 of the FP64 peak (Poisson / heat) against 0.67 with one column of
// look-ahead and 0.79 / 0.76 with four; an indexed-array queue let the
// compiler sink the loads and lost the gain.
template <int UNR>
__device__ __forceinline__ void vertical_tw1(double *__restrict__ row, const double *__restrict__ ZB, int Nz, int k,
                                             bool bottom, double *__restrict__ xs, int xst) {
  const double2 *z2p = reinterpret_cast<const double2 *>(ZB);
  if (!bottom) {
    xs[xst] = row[k];
    xs[2 * xst] = row[k + 1];
    double wq = 0.0;
    double q0 = 0 < k ? row[0] : 0.0, q1 = 1 < k ? row[1] : 0.0, q2 = 2 < k ? row[2] : 0.0, q3 = 3 < k ? row[3] : 0.0,
           q4 = 4 < k ? row[4] : 0.0, q5 = 5 < k ? row[5] : 0.0;
    double2 cn = z2p[0];
#pragma unroll UNR
    for (int b = 0; b < k; ++b) {
      const double r = q0;
      q0 = q1; q1 = q2; q2 = q3; q3 = q4; q4 = q5;
      q5 = (b + 6 < k) ? row[b + 6] : 0.0;
      const double2 cc = cn;
      if (b + 1 < k) cn = z2p[(b + 1) * 4];
      const double w = fma(cc.x, wq, r);
      row[b] = w;
      wq = w;
    }
    xs[0] = wq;          // w_{k-1}
  } else {
    double v1 = 0.0, v2 = 0.0;
    double q0 = Nz - 1 >= k + 2 ? row[Nz - 1] : 0.0, q1 = Nz - 2 >= k + 2 ? row[Nz - 2] : 0.0,
           q2 = Nz - 3 >= k + 2 ? row[Nz - 3] : 0.0, q3 = Nz - 4 >= k + 2 ? row[Nz - 4] : 0.0,
           q4 = Nz - 5 >= k + 2 ? row[Nz - 5] : 0.0, q5 = Nz - 6 >= k + 2 ? row[Nz - 6] : 0.0;
    double2 cn = z2p[(Nz - 1) * 4];
#pragma unroll UNR
    for (int b = Nz - 1; b >= k + 2; --b) {
      const double r = q0;
      q0 = q1; q1 = q2; q2 = q3; q3 = q4; q4 = q5;
      q5 = (b - 6 >= k + 2) ? row[b - 6] : 0.0;
      const double2 cc = cn;
      if (b - 1 >= k + 2) cn = z2p[(b - 1) * 4];
      const double v = fma(cc.x, v1, fma(cc.y, v2, r));   // -Ut[b][b+1], -Ut[b][b+2]
      row[b] = v;
      v2 = v1;
      v1 = v;
    }
    xs[3 * xst] = v1;    // v_{k+2}
    xs[4 * xst] = v2;    // v_{k+3}
  }
}

// Vertical phase 2: interface x_k .. x_{k+2} from the 3 x 5 map, back
// substitutions outward and (unless LAST) the next iteration's apply band
// u = (D + p'B) x: the top thread writes u_0 .. u_k, the bottom u_{k+1} ..
template <bool LAST, int UNR>
__device__ __forceinline__ void vertical_tw2(double *__restrict__ row, const double *__restrict__ ZB, int Nz, int k,
                                             bool bottom, const double *__restrict__ xs, int xst) {
  const double *R = ZB + Nz * ZSTRIDE;
  double rhs[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) rhs[q] = xs[q * xst];
  double xI[3];
#pragma unroll
  for (int o = 0; o < 3; ++o) {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 5; ++q) s = fma(R[o * 5 + q], rhs[q], s);
    xI[o] = s;
  }
  const double2 *z2p = reinterpret_cast<const double2 *>(ZB);
  if (!bottom) {
    double x1 = xI[0], x2 = xI[1], x3 = xI[2];            // x_{b+1}, x_{b+2}, x_{b+3}
    if (LAST) {
      row[k] = xI[0];
      row[k + 1] = xI[1];
    }
    double2 q45 = z2p[k * 4 + 2], q67 = z2p[k * 4 + 3];    // apply record of column b+1
    double q0 = k - 1 >= 0 ? row[k - 1] : 0.0, q1 = k - 2 >= 0 ? row[k - 2] : 0.0, q2 = k - 3 >= 0 ? row[k - 3] : 0.0,
           q3 = k - 4 >= 0 ? row[k - 4] : 0.0, q4 = k - 5 >= 0 ? row[k - 5] : 0.0, q5 = k - 6 >= 0 ? row[k - 6] : 0.0;
    double2 p01 = z2p[(k - 1) * 4], p23 = z2p[(k - 1) * 4 + 1], p45, p67;
    if (!LAST) { p45 = z2p[(k - 1) * 4 + 2]; p67 = z2p[(k - 1) * 4 + 3]; }
#pragma unroll UNR
    for (int b = k - 1; b >= 0; --b) {
      const double wb = q0;
      q0 = q1; q1 = q2; q2 = q3; q3 = q4; q4 = q5;
      q5 = (b - 6 >= 0) ? row[b - 6] : 0.0;
      const double2 c01 = p01, c23 = p23;
      double2 c45, c67;
      if (!LAST) { c45 = p45; c67 = p67; }
      if (b > 0) {
        p01 = z2p[(b - 1) * 4];
        p23 = z2p[(b - 1) * 4 + 1];
        if (!LAST) { p45 = z2p[(b - 1) * 4 + 2]; p67 = z2p[(b - 1) * 4 + 3]; }
      }
      const double v = fma(c23.x, x2, c23.y * wb);
      const double xb = fma(c01.y, x1, v);
      if (LAST) {
        row[b] = xb;
      } else {
        double u = q67.y * x3;
        u = fma(q67.x, x2, u);
        u = fma(q45.y, x1, u);
        u = fma(q45.x, xb, u);
        row[b + 1] = u;
        q45 = c45;
        q67 = c67;
      }
      x3 = x2;
      x2 = x1;
      x1 = xb;
    }
    if (!LAST) {
      double u = q45.y * x1;                 // column 0: x_{-1} = 0
      u = fma(q67.x, x2, u);
      u = fma(q67.y, x3, u);
      row[0] = u;
    }
  } else {
    double xm3 = 0.0, xm2 = xI[0], xm1 = xI[1];            // x_{b-3}, x_{b-2}, x_{b-1}
    double q0 = k + 2 < Nz ? row[k + 2] : 0.0, q1 = k + 3 < Nz ? row[k + 3] : 0.0, q2 = k + 4 < Nz ? row[k + 4] : 0.0,
           q3 = k + 5 < Nz ? row[k + 5] : 0.0, q4 = k + 6 < Nz ? row[k + 6] : 0.0, q5 = k + 7 < Nz ? row[k + 7] : 0.0;
    double2 p23 = z2p[(k + 2) * 4 + 1];
#pragma unroll UNR
    for (int b = k + 2; b < Nz; ++b) {
      const double vb = q0;
      q0 = q1; q1 = q2; q2 = q3; q3 = q4; q4 = q5;
      q5 = (b + 6 < Nz) ? row[b + 6] : 0.0;
      const double2 c23 = p23;
      if (b + 1 < Nz) p23 = z2p[(b + 1) * 4 + 1];
      const double xb = fma(c23.x, xm1, c23.y * vb);       // -Lt[b][b-1]/Lt_bb, 1/Lt_bb
      if (LAST) {
        row[b] = xb;
      } else if (b >= k + 3) {
        const double2 a45 = z2p[(b - 2) * 4 + 2], a67 = z2p[(b - 2) * 4 + 3];
        double u = a67.y * xb;
        u = fma(a67.x, xm1, u);
        u = fma(a45.y, xm2, u);
        u = fma(a45.x, xm3, u);
        row[b - 2] = u;
      }
      xm3 = xm2;
      xm2 = xm1;
      xm1 = xb;
    }
    if (!LAST) {                              // columns Nz-2, Nz-1 (x_{Nz}, x_{Nz+1} = 0)
      const double2 a45 = z2p[(Nz - 2) * 4 + 2], a67 = z2p[(Nz - 2) * 4 + 3];
      double u = a67.x * xm1;
      u = fma(a45.y, xm2, u);
      u = fma(a45.x, xm3, u);
      row[Nz - 2] = u;
      const double2 b45 = z2p[(Nz - 1) * 4 + 2];
      double u1 = b45.y * xm1;
      u1 = fma(b45.x, xm2, u1);
      row[Nz - 1] = u1;
    }
  }
}

// A group of threads that processes one item: the whole CTA (named barrier 0)
// or one of G equal slices of it (named barriers 1 .. G).  In cluster mode
// the item is shared by the nparts CTAs of a thread-block cluster; this CTA
// is part `part` and owns an equal range of the item's columns (radial
// sweeps, right side, expansion) and rows (vertical sweeps).  csync() orders
// the phases whose data cross CTAs: a cluster-wide barrier with release /
// acquire semantics (the item's arrays live in global memory), else the
// group's own barrier.
struct Grp {
  int tid, nth, bar;
  int part = 0, nparts = 1;
  __device__ __forceinline__ void sync() const {
    if (bar == 0) __syncthreads();
    else asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nth) : "memory");
  }
  __device__ __forceinline__ void csync() const {
    if (nparts > 1)
      asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    else
      sync();
  }
  // [lo, hi) of this part's share of n
  __device__ __forceinline__ int lo(int n) const { return (int)((long long)n * part / nparts); }
  __device__ __forceinline__ int hi(int n) const { return (int)((long long)n * (part + 1) / nparts); }
};

// J iterations of Algorithm 1 on one item from X_0 = 0: right side in Fa,
// result in S.  Factor tables of iteration c (counted per group over every
// step and item it processes; c0 = the item's first iteration) arrive in
// buffer c & 1 by TMA bulk copies issued one iteration ahead.
struct AdiShared {
  double *RB0, *ZB0;
  int rlen, zlen;
  unsigned long long *bar;
  double *xs;     // twisted-sweep exchange scratch (TW_SLOTS x xhalf doubles), or NULL
  int xhalf;      // threads per side of a twisted sweep (half the group)
};

// TT: the transposed (adjoint) system's records instead of the forward ones.
template <bool TT>
__device__ __forceinline__ void issue_tables(const AdiShared &sh, const AdiArgs &a, const Item &it, long long c,
                                             long long c0) {
  const int jt = (int)((c - c0) % it.J), buf = (int)(c & 1);
  const int rsz = it.M * RSTRIDE + ((TT ? it.twrT : it.twr) ? RTWIST : 0);
  const int zsz = it.Nz * ZSTRIDE + ((TT ? it.twzT : it.twz) ? ZTWIST : 0);
  const unsigned rbytes = (unsigned)(rsz * sizeof(double));
  const unsigned zbytes = (unsigned)(zsz * sizeof(double));
  const long long roff = TT ? it.roffT : it.roff, zoff = TT ? it.zoffT : it.zoff;
  mbar_expect(&sh.bar[buf], rbytes + zbytes);
  bulk_g2s(sh.RB0 + buf * sh.rlen, a.fac + roff + (size_t)jt * rsz, rbytes, &sh.bar[buf]);
  bulk_g2s(sh.ZB0 + buf * sh.zlen, a.fac + zoff + (size_t)jt * zsz, zbytes, &sh.bar[buf]);
}

// UNR: unroll factor of the sweeps.  Measured on GB300: 2 with the work
// arrays in shared memory; 8 with them in global memory, where more rows in
// flight hide the load latency (1 is 6x slower there, 8 beats 4 by 15 %).
// TW: compiled with the twisted sweeps (items whose tables carry twisted
// solves, twr / twz > 0); without it only the one-sided sweeps are compiled,
// which keeps the register allocation of the plain kernels unchanged.
// OTW: every item of the launch is twisted in both directions (the host
// checks): the one-sided sweeps are not compiled at all, which leaves the
// 128 registers of a 512-thread CTA to the twisted sweeps and their
// six-column queue (measured at 512^3: 0.81 / 0.80 of the FP64 peak, Poisson
// / heat, against 0.78 / 0.77 with the one-sided sweeps compiled in).
template <bool TT, int UNR, bool TW = false, bool OTW = false>
__device__ __forceinline__ void adi_iterations(const Grp &gp, const AdiShared &sh, const AdiArgs &a, const Item &it,
                                               double *S, const double *Fa, int ldF, long long &c, long long c0,
                                               long long c_end, bool &timed_out) {
  const int M = it.M, Nz = it.Nz, nsl = it.nsl, W = nsl * Nz, ld = a.ld, J = it.J;
  // this part's columns (radial chains) and rows (vertical chains)
  const int cb0 = gp.lo(W), cb1 = gp.hi(W), rb0 = gp.lo(nsl * M), rb1 = gp.hi(nsl * M);
  for (int jt = 0; jt < J; ++jt, ++c) {
    const int buf = (int)(c & 1);
    if (gp.tid == 0 && c + 1 < c_end && !a.test_no_tma) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue_tables<TT>(sh, a, it, c + 1, c0);
    }
    if (!mbar_wait(&sh.bar[buf], (unsigned)((c >> 1) & 1), a.wait_limit)) timed_out = true;
    const double *RB = sh.RB0 + buf * sh.rlen;
    const double *ZB = sh.ZB0 + buf * sh.zlen;
    const int xh = sh.xhalf;
    const bool bottom = gp.tid >= xh;
    const int chain = gp.tid - (bottom ? xh : 0);
    const int twr = TT ? it.twrT : it.twr, twz = TT ? it.twzT : it.twz;
    if (OTW || (TW && twr)) {
      const int col = cb0 + chain;
      if (col < cb1) {
        if (jt == 0) radial_tw1<true, UNR>(S + col, Fa + col, ld, RB, M, twr, bottom, sh.xs + chain, xh);
        else radial_tw1<false, UNR>(S + col, Fa + col, ld, RB, M, twr, bottom, sh.xs + chain, xh);
      }
      gp.sync();
      if (col < cb1) radial_tw2<UNR>(S + col, ld, RB, M, twr, bottom, sh.xs + chain, xh);
    } else if constexpr (!OTW) {
      for (int col = cb0 + gp.tid; col < cb1; col += gp.nth) {
        if (jt == 0) radial_sweep<true, UNR>(S + col, Fa + col, ld, RB, M);
        else radial_sweep<false, UNR>(S + col, Fa + col, ld, RB, M);
      }
    }
    gp.csync();
    if (OTW || (TW && twz)) {
      const int r = rb0 + chain;
      const int sl = r / M, aa = r - sl * M;
      double *rowp = S + aa * ld + sl * Nz;
      if (r < rb1) vertical_tw1<UNR>(rowp, ZB, Nz, twz, bottom, sh.xs + chain, xh);
      gp.sync();
      if (r < rb1) {
        if (jt + 1 == J) vertical_tw2<true, UNR>(rowp, ZB, Nz, twz, bottom, sh.xs + chain, xh);
        else vertical_tw2<false, UNR>(rowp, ZB, Nz, twz, bottom, sh.xs + chain, xh);
      }
    } else if constexpr (!OTW) {
      for (int r = rb0 + gp.tid; r < rb1; r += gp.nth) {
        const int sl = r / M, aa = r - sl * M;
        if (jt + 1 == J) vertical_sweep<true, UNR>(S + aa * ld + sl * Nz, ZB, Nz);
        else vertical_sweep<false, UNR>(S + aa * ld + sl * Nz, ZB, Nz);
      }
    }
    gp.csync();
  }
  (void)ldF;
}

__device__ __forceinline__ void init_bars(const Grp &gp, unsigned long long *bar) {
  if (gp.tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  gp.sync();
}

// Every BDF1 step of one item (see adi_kernel): right side, ADI, expansion.
template <int UNR, bool TW = false, bool OTW = false>
__device__ __forceinline__ void process_item_forward(const Grp &gp, const AdiArgs &a, const Item &it,
                                                     const AdiShared &sh, double *S, double *Fa, long long &c,
                                                     bool &timed_out) {
  const int tid = gp.tid, nth = gp.nth;
  const int M = it.M, Nz = it.Nz, nsl = it.nsl, W = nsl * Nz;
  const int cb0 = gp.lo(W), Wp = gp.hi(W) - cb0;    // this part's columns of the item
  const int ld = a.ld;
  const int m = it.m, n = it.n;
  const long long slice = (long long)m * n;
  const double *r2 = a.fac + it.r2off;
  const double *c02 = a.fac + it.c02off;
  const long long c0 = c, c_end = c0 + (long long)a.nsteps * it.J;
  if (tid == 0 && !a.test_no_tma) issue_tables<false>(sh, a, it, c0, c0);
  const bool ring = a.hist_b > 0;
  const double *Xsrc = ring ? nullptr : a.Xin + it.xoff;
  double *Xout = ring ? nullptr : a.Xout + it.xoff;
  const double *lift = a.lift ? a.lift + it.xoff : nullptr;
  const double *Gbase = a.G ? a.G + it.xoff : nullptr;
  int base = a.hist_base;
  for (int step = 0; step < a.nsteps; ++step) {
    const double *Gs = Gbase ? Gbase + (size_t)step * a.gstride : nullptr;
    const double *hs[4] = {nullptr, nullptr, nullptr, nullptr};
    if (ring) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (i < a.order) hs[i] = a.hist + (size_t)((base + i) % a.hist_b) * a.hist_stride + it.xoff;
      Xout = a.hist + (size_t)((base + a.hist_b - 1) % a.hist_b) * a.hist_stride + it.xoff;
    }
    // Right side of eq. HelmholtzMatEqn, E = trunc(R_2 (delta X + kappa g) C02^T), in two
    // banded passes: T1 = (delta X + kappa g) C02^T on the class rows, then E = R_2 T1
    // (delta X = X_n for BDF1, sum_i beta_i X_{n-i} from the history ring otherwise).
    for (int e = tid; e < it.Mfull * Wp; e += nth) {
      const int ap = e / Wp, cc = cb0 + (e - ap * Wp);
      const int sl = cc / Nz, b = cc - sl * Nz;
      const int i = it.pr + 2 * ap, j = it.pz + 2 * b;
      const size_t row = (size_t)(it.s0 + sl) * slice + (size_t)i * n;
      double acc = 0.0;
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        const int jj = j + 2 * t;
        if (jj < n) {
          double z;
          if (ring) {
            z = 0.0;
#pragma unroll
            for (int h = 0; h < 4; ++h)
              if (h < a.order) z = fma(a.beta[h], hs[h][row + jj], z);
          } else {
            z = Xsrc[row + jj];
          }
          if (Gs) z = fma(a.kappa, Gs[row + jj], z);
          acc = fma(c02[b * C02STRIDE + t], z, acc);
        }
      }
      S[ap * ld + cc] = acc;
    }
    gp.sync();
    const double *corr = a.corr ? a.corr + it.xoff : nullptr;
    for (int e = tid; e < M * Wp; e += nth) {
      const int aa = e / Wp, cc = cb0 + (e - aa * Wp);
      double acc = 0.0;
#pragma unroll
      for (int s = -1; s <= 3; ++s) {
        const int q = aa + s;
        if (q >= 0 && q < it.Mfull) acc = fma(r2[aa * R2STRIDE + s + 1], S[q * ld + cc], acc);
      }
      if (corr) {
        const int sl = cc / Nz, b = cc - sl * Nz;
        acc += corr[(size_t)(it.s0 + sl) * slice + (size_t)(it.pr + 2 * aa) * n + it.pz + 2 * b];
      }
      Fa[aa * ld + cc] = acc;
    }
    gp.sync();

    adi_iterations<false, UNR, TW, OTW>(gp, sh, a, it, S, Fa, ld, c, c0, c_end, timed_out);

    // X = S_r Y S_z^T on this item's class rows / columns (phi_j = T_{j+2} - T_j).
    const int Wf = nsl * it.Nzfull, f0 = gp.lo(Wf), Wfp = gp.hi(Wf) - f0;
    const bool do_ck = a.ckpt && ((step + 1) % a.ckpt_every == 0);
    double *ck = do_ck ? a.ckpt + it.xoff + (size_t)((step + 1) / a.ckpt_every) * (size_t)a.p * slice : nullptr;
    for (int e = tid; e < it.Mfull * Wfp; e += nth) {
      const int ap = e / Wfp, cc = f0 + (e - ap * Wfp);
      const int sl = cc / it.Nzfull, b = cc - sl * it.Nzfull;
      const double *Ys = S + sl * Nz;
      const bool r0 = ap - 1 >= 0, r1 = ap < M, c0b = b - 1 >= 0, c1 = b < Nz;
      double x = 0.0;
      if (r0 && c0b) x += Ys[(ap - 1) * ld + b - 1];
      if (r0 && c1) x -= Ys[(ap - 1) * ld + b];
      if (r1 && c0b) x -= Ys[ap * ld + b - 1];
      if (r1 && c1) x += Ys[ap * ld + b];
      const size_t o = (size_t)(it.s0 + sl) * slice + (size_t)(it.pr + 2 * ap) * n + it.pz + 2 * b;
      if (lift) x += lift[o];
      Xout[o] = x;
      if (ck) ck[o] = x;
    }
    if (a.zero_other) {
      const int po = 1 - it.pr, Mo = (m - po + 1) / 2;
      for (int e = tid; e < Mo * Wfp; e += nth) {
        const int ap = e / Wfp, cc = f0 + (e - ap * Wfp);
        const int sl = cc / it.Nzfull, b = cc - sl * it.Nzfull;
        const size_t o = (size_t)(it.s0 + sl) * slice + (size_t)(po + 2 * ap) * n + it.pz + 2 * b;
        const double x = lift ? lift[o] : 0.0;
        Xout[o] = x;
        if (ck) ck[o] = x;
      }
    }
    gp.csync();
    Xsrc = Xout;
    if (ring) base = (base + a.hist_b - 1) % a.hist_b;
  }
}

// One CTA per item.  S_SMEM / F_SMEM place the item's iterate (S) and right
// side (Fa) in shared memory, else in the per-item global work area.
template <bool S_SMEM, bool F_SMEM, int MAXT, bool TW, bool OTW = false>
__global__ void __launch_bounds__(MAXT, 1) adi_kernel(const AdiArgs a) {
  extern __shared__ __align__(16) double sm[];
  __shared__ __align__(8) unsigned long long bar[2];
  const Item it = a.items[blockIdx.x];
  const Grp gp{(int)threadIdx.x, (int)blockDim.x, 0};
  AdiShared sh;
  sh.rlen = a.maxM * RSTRIDE + RTWIST;
  sh.zlen = a.maxNz * ZSTRIDE + ZTWIST;
  sh.RB0 = sm;
  sh.ZB0 = sm + 2 * sh.rlen;
  sh.bar = bar;
  double *smem_next = sh.ZB0 + 2 * sh.zlen;
  double *gw = a.gwork + (size_t)blockIdx.x * a.gwork_per_item;
  double *S = S_SMEM ? smem_next : gw;
  if (S_SMEM) smem_next += (size_t)a.smem_rows * a.ld;
  double *Fa = F_SMEM ? smem_next : gw + (S_SMEM ? 0 : (size_t)a.smem_rows * a.ld);
  if (F_SMEM) smem_next += (size_t)a.maxM * a.ld;
  sh.xs = a.twist_half ? smem_next : nullptr;
  sh.xhalf = a.twist_half ? a.twist_half : gp.nth;
  init_bars(gp, bar);
  bool timed_out = false;
  long long c = 0;
  process_item_forward<S_SMEM ? 2 : 8, TW, OTW>(gp, a, it, sh, S, Fa, c, timed_out);
  if (timed_out && a.err) atomicExch(a.err, (int)CYL_ERR_TIMEOUT);
}

// Cluster mode, for items whose work arrays fit no SM's shared memory (grids
// of about 220 points per axis and more): the a.cluster CTAs of a
// thread-block cluster share one item, whose iterate S and right side Fa
// stay in the item's global work area.  Each CTA owns at most 128 chains of
// every sweep and runs them as twisted solves (two threads per chain, 256
// threads, two warps per SM sub-partition); the phases that read other
// CTAs' results meet at cluster barriers.  Only (resident CTAs / a.cluster)
// items are live at a time, so their work arrays stay in L2 (at 512^3: 38
// items x 2.1 MB) instead of streaming through DRAM every ADI iteration.
template <int UNR>
__global__ void __launch_bounds__(256, 1) adi_cluster_kernel(const AdiArgs a) {
  extern __shared__ __align__(16) double sm[];
  __shared__ __align__(8) unsigned long long bar[2];
  const int item = blockIdx.x / a.cluster;
  const Item it = a.items[item];
  Grp gp{(int)threadIdx.x, (int)blockDim.x, 0};
  gp.part = blockIdx.x - item * a.cluster;            // rank in the cluster (clusters tile the grid along x)
  gp.nparts = a.cluster;
  AdiShared sh;
  sh.rlen = a.maxM * RSTRIDE + RTWIST;
  sh.zlen = a.maxNz * ZSTRIDE + ZTWIST;
  sh.RB0 = sm;
  sh.ZB0 = sm + 2 * sh.rlen;
  sh.bar = bar;
  sh.xs = sh.ZB0 + 2 * sh.zlen;
  sh.xhalf = a.twist_half;
  double *gw = a.gwork + (size_t)item * a.gwork_per_item;
  double *S = gw, *Fa = gw + (size_t)a.smem_rows * a.ld;
  init_bars(gp, bar);
  bool timed_out = false;
  long long c = 0;
  process_item_forward<UNR, true>(gp, a, it, sh, S, Fa, c, timed_out);
  if (timed_out && a.err) atomicExch(a.err, (int)CYL_ERR_TIMEOUT);
}

size_t adi_cluster_smem_bytes(int maxM, int maxNz, int twist_half) {
  const size_t d = 2 * ((size_t)maxM * RSTRIDE + RTWIST + (size_t)maxNz * ZSTRIDE + ZTWIST) +
                   (size_t)TW_SLOTS * twist_half;
  return d * sizeof(double);
}

cudaError_t launch_adi_cluster(const AdiArgs &a, int threads, size_t smem, cudaStream_t st) {
  if (a.cluster < 2 || a.cluster > 8 || threads > 256 || a.twist_half * 2 != threads) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(adi_cluster_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.nitems * a.cluster), 1, 1);
  cfg.blockDim = dim3((unsigned)threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)a.cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, adi_cluster_kernel<8>, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// Persistent batch kernel: the CTA is split into G groups of blockDim.x / G
// threads; each group pulls items (largest first) from a queue and runs every
// step of each.  S lives in the group's shared-memory slice, Fa in the
// group's global work area.
template <int G, bool TW, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) adi_batch_kernel(const AdiArgs a, int *queue) {
  extern __shared__ __align__(16) double sm[];
  __shared__ __align__(8) unsigned long long bar[2 * G];
  __shared__ int next_item[G];
  const int gsize = blockDim.x / G, g = threadIdx.x / gsize;
  const Grp gp{(int)threadIdx.x - g * gsize, gsize, G == 1 ? 0 : 1 + g};
  // every group's slice starts on a 256-byte boundary (TMA destinations and
  // double2 loads of the factor tables need 16-byte alignment)
  double *base = sm + (size_t)g * (size_t)a.group_doubles;
  AdiShared sh;
  sh.rlen = a.maxM * RSTRIDE + (TW ? RTWIST : 0);
  sh.zlen = a.maxNz * ZSTRIDE + (TW ? ZTWIST : 0);
  sh.RB0 = base;
  sh.ZB0 = base + 2 * sh.rlen;
  sh.bar = bar + 2 * g;
  double *S = sh.ZB0 + 2 * sh.zlen;
  sh.xs = TW ? S + (size_t)a.smem_rows * a.ld : nullptr;   // twisted-sweep exchange, after S
  sh.xhalf = TW ? a.twist_half : gsize;
  double *Fa = a.gwork + ((size_t)blockIdx.x * G + g) * a.gwork_per_item;
  init_bars(gp, sh.bar);
  bool timed_out = false;
  long long c = 0;
  for (;;) {
    if (gp.tid == 0) next_item[g] = atomicAdd(queue, 1);
    gp.sync();
    const int idx = next_item[g];
    gp.sync();
    if (idx >= a.nitems) break;
    const Item it = a.items[idx];
    process_item_forward<2, TW>(gp, a, it, sh, S, Fa, c, timed_out);
  }
  if (timed_out && a.err) atomicExch(a.err, (int)CYL_ERR_TIMEOUT);
}

// One group's shared-memory slice: double-buffered tables, S, and (twisted
// groups) the interface maps and the exchange scratch; a multiple of 32
// doubles so every group's slice starts 256-byte aligned.
size_t batch_group_doubles(int ld, int smem_rows, int maxM, int maxNz, int twist_half) {
  const size_t tails = twist_half ? (size_t)(RTWIST + ZTWIST) : 0;
  const size_t d = (size_t)2 * (maxM * RSTRIDE + maxNz * ZSTRIDE + tails) + (size_t)smem_rows * ld +
                   (size_t)TW_SLOTS * twist_half;
  return (d + 31) / 32 * 32;
}

size_t batch_smem_bytes(int G, int ld, int smem_rows, int maxM, int maxNz, int twist_half) {
  return batch_group_doubles(ld, smem_rows, maxM, maxNz, twist_half) * G * sizeof(double);
}

template <int G, bool TW>
static cudaError_t launch_batch_t(const AdiArgs &a, int *queue, int threads, int blocks, size_t smem,
                                  cudaStream_t st) {
  // CTAs of at most 256 threads get the full register budget (no spills in the sweeps)
  if (threads <= 256) {
    cudaError_t e = cudaFuncSetAttribute(adi_batch_kernel<G, TW, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    adi_batch_kernel<G, TW, 256><<<blocks, threads, smem, st>>>(a, queue);
  } else {
    cudaError_t e = cudaFuncSetAttribute(adi_batch_kernel<G, TW, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    adi_batch_kernel<G, TW, 512><<<blocks, threads, smem, st>>>(a, queue);
  }
  return cudaGetLastError();
}

cudaError_t launch_batch(const AdiArgs &a, int *queue, int G, int threads, int blocks, size_t smem,
                         cudaStream_t st) {
  if (a.nitems <= 0 || a.nsteps <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  const bool tw = a.twist_half > 0;
  switch (G) {
    case 1: return tw ? launch_batch_t<1, true>(a, queue, threads, blocks, smem, st)
                      : launch_batch_t<1, false>(a, queue, threads, blocks, smem, st);
    case 2: return tw ? launch_batch_t<2, true>(a, queue, threads, blocks, smem, st)
                      : launch_batch_t<2, false>(a, queue, threads, blocks, smem, st);
    case 4: return tw ? launch_batch_t<4, true>(a, queue, threads, blocks, smem, st)
                      : launch_batch_t<4, false>(a, queue, threads, blocks, smem, st);
    default: return cudaErrorInvalidValue;
  }
}

// Adjoint of the BDF1 steps n = n_hi-1 .. n_lo for one item (the transpose of
// adi_kernel's map, step by step in reverse):
//   mu = S_r^T lam S_z;  Lambda = (A^T . B + C^T . D)^-1 mu by ADI;
//   lam <- R_2^T Lambda C02 (class rows < m, class columns < n);
//   dL/dg_n = kappa lam;  dL/dalpha += <lam, X_{n+1} - X_n - kappa g_n> / alpha
// (the last identity follows from A Y B^T + C Y D^T = E, A = C - kappa alpha L,
// D = -kappa alpha D2:  d/dalpha of the solve is (E - C Y B^T) / alpha).
// The transposed Sylvester solve is the forward-form system of the flipped
// transposes J A^T J, ... on index-reversed arrays (J reverses the class
// rows and, per slice, the class columns), so mu is written and Lambda read
// in reversed order and the forward sweeps (twisted where the records are)
// do the iterations with the transposed records.  Work arrays as adi_kernel.
template <bool S_SMEM, bool F_SMEM, int MAXT, bool TW, bool OTW = false>
__global__ void __launch_bounds__(MAXT, 1) adi_adjoint_kernel(const AdiArgs a, AdjointArgs g) {
  extern __shared__ __align__(16) double sm[];
  __shared__ __align__(8) unsigned long long bar[2];
  __shared__ double red[32];
  const Item it = a.items[blockIdx.x];
  const int tid = threadIdx.x, nth = blockDim.x;
  const int M = it.M, Nz = it.Nz, nsl = it.nsl, W = nsl * Nz, Wf = nsl * it.Nzfull;
  const int ld = a.ld;
  const int m = it.m, n = it.n;
  const long long slice = (long long)m * n, Ntot = (long long)a.p * slice;
  AdiShared sh;
  sh.rlen = a.maxM * RSTRIDE + RTWIST;
  sh.zlen = a.maxNz * ZSTRIDE + ZTWIST;
  sh.RB0 = sm;
  sh.ZB0 = sm + 2 * sh.rlen;
  sh.bar = bar;
  double *smem_next = sh.ZB0 + 2 * sh.zlen;
  double *gw = a.gwork + (size_t)blockIdx.x * a.gwork_per_item;
  double *S = S_SMEM ? smem_next : gw;
  if (S_SMEM) smem_next += (size_t)a.smem_rows * ld;
  double *Fa = F_SMEM ? smem_next : gw + (S_SMEM ? 0 : (size_t)a.smem_rows * ld);
  if (F_SMEM) smem_next += (size_t)a.maxM * ld;
  sh.xs = a.twist_half ? smem_next : nullptr;
  sh.xhalf = a.twist_half ? a.twist_half : nth;
  const Grp gp{tid, nth, 0};
  init_bars(gp, bar);
  const double *r2 = a.fac + it.r2off;
  const double *c02 = a.fac + it.c02off;
  const int nst = g.n_hi - g.n_lo;
  const long long total_it = (long long)nst * it.J;
  if (tid == 0 && !a.test_no_tma) issue_tables<true>(sh, a, it, 0, 0);
  bool timed_out = false;
  double apart = 0.0;
  double *lam = g.lam;
  const bool ring = g.lam_ring != nullptr;
  long long c = 0;
  for (int n_step = g.n_hi - 1; n_step >= g.n_lo; --n_step) {
    double *lin = ring ? g.lam_ring + (size_t)((n_step + 1 + g.jofs) % g.R) * Ntot : lam;
    // mu[a][b] = lam[a][b] - lam[a][b+1] - lam[a+1][b] + lam[a+1][b+1] (class indices), stored reversed
    for (int e = tid; e < M * W; e += nth) {
      const int aa = e / W, cc = e - aa * W;
      const int sl = cc / Nz, b = cc - sl * Nz;
      const size_t o = (size_t)(it.s0 + sl) * slice + (size_t)(it.pr + 2 * aa) * n + it.pz + 2 * b;
      Fa[(M - 1 - aa) * ld + sl * Nz + (Nz - 1 - b)] = lin[o] - lin[o + 2] - lin[o + 2 * n] + lin[o + 2 * n + 2];
    }
    __syncthreads();
    adi_iterations<true, S_SMEM ? 2 : 8, TW, OTW>(gp, sh, a, it, S, Fa, ld, c, 0, total_it, timed_out);
    // T1 = Lambda C02 on nsl * Nzfull columns: T1[a][b'] = sum_t Lambda[a][b' - t] C02[b' - t][t]
    for (int e = tid; e < M * Wf; e += nth) {
      const int aa = e / Wf, cc = e - aa * Wf;
      const int sl = cc / it.Nzfull, bp = cc - sl * it.Nzfull;
      double acc = 0.0;
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        const int b = bp - t;
        if (b >= 0 && b < Nz) acc = fma(c02[b * C02STRIDE + t], S[(M - 1 - aa) * ld + sl * Nz + (Nz - 1 - b)], acc);
      }
      Fa[aa * ld + cc] = acc;
    }
    __syncthreads();
    // lam_n = R_2^T T1 on all class rows; forcing gradient and alpha term
    const double *Gn = g.G ? g.G + (size_t)n_step * g.gstride : nullptr;
    double *dgn = g.dg ? g.dg + (size_t)n_step * g.dg_stride : nullptr;
    const double *Xn = (g.traj && !ring) ? g.traj + (size_t)(n_step - g.n_lo) * Ntot : nullptr;
    double *lout[4] = {nullptr, nullptr, nullptr, nullptr};
    const double *xr[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};   // X_{s+1}, X_s, .., X_{s-3}
    if (ring) {
#pragma unroll
      for (int h = 0; h < 4; ++h)
        if (h < g.order) lout[h] = g.lam_ring + (size_t)((n_step - h + g.jofs) % g.R) * Ntot;
      if (g.traj) {
#pragma unroll
        for (int h = 0; h < 5; ++h)
          if (h <= g.order) xr[h] = g.traj + (size_t)(g.traj_K - (n_step + 1 - h)) * Ntot;
      }
    }
    for (int e = tid; e < it.Mfull * Wf; e += nth) {
      const int ap = e / Wf, cc = e - ap * Wf;
      const int sl = cc / it.Nzfull, bp = cc - sl * it.Nzfull;
      double acc = 0.0;
#pragma unroll
      for (int s = -1; s <= 3; ++s) {
        const int q = ap - s;
        if (q >= 0 && q < M) acc = fma(r2[q * R2STRIDE + s + 1], Fa[q * ld + cc], acc);
      }
      const size_t o = (size_t)(it.s0 + sl) * slice + (size_t)(it.pr + 2 * ap) * n + it.pz + 2 * bp;
      if (ring) {
#pragma unroll
        for (int h = 0; h < 4; ++h)
          if (h < g.order) lout[h][o] = fma(g.beta[h], acc, lout[h][o]);
      } else {
        lam[o] = acc;
      }
      if (dgn) {
        if (g.dg_stride == 0) dgn[o] += g.kappa * acc;
        else dgn[o] = g.kappa * acc;
      }
      if (Xn) {
        double d = Xn[o + Ntot] - Xn[o];
        if (Gn) d = fma(-g.kappa, Gn[o], d);
        apart = fma(acc, d, apart);
      }
      if (xr[0]) {
        double d = xr[0][o];
#pragma unroll
        for (int h = 0; h < 4; ++h)
          if (h < g.order) d = fma(-g.beta[h], xr[h + 1][o], d);
        if (Gn) d = fma(-g.kappa, Gn[o], d);
        apart = fma(acc, d, apart);
      }
    }
    if (a.zero_other) {
      const int po = 1 - it.pr, Mo = (m - po + 1) / 2;
      for (int e = tid; e < Mo * Wf; e += nth) {
        const int ap = e / Wf, cc = e - ap * Wf;
        const int sl = cc / it.Nzfull, b = cc - sl * it.Nzfull;
        const size_t o = (size_t)(it.s0 + sl) * slice + (size_t)(po + 2 * ap) * n + it.pz + 2 * b;
        if (!ring) lam[o] = 0.0;
        if (dgn && g.dg_stride != 0) dgn[o] = 0.0;
      }
    }
    if (ring) {
      // lam_{s+1} is consumed: clear this item's positions of its slot (it becomes lam_{s-order})
      const int nclass = a.zero_other ? 2 : 1;
      for (int q = 0; q < nclass; ++q) {
        const int pq = q == 0 ? it.pr : 1 - it.pr, Mq = (m - pq + 1) / 2;
        for (int e = tid; e < Mq * Wf; e += nth) {
          const int ap = e / Wf, cc = e - ap * Wf;
          const int sl = cc / it.Nzfull, b = cc - sl * it.Nzfull;
          lin[(size_t)(it.s0 + sl) * slice + (size_t)(pq + 2 * ap) * n + it.pz + 2 * b] = 0.0;
        }
      }
    }
    __syncthreads();
  }
  if (g.alpha_part) {
    for (int off = 16; off > 0; off >>= 1) apart += __shfl_down_sync(0xffffffffu, apart, off);
    if ((tid & 31) == 0) red[tid >> 5] = apart;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int w = 0; w < (nth + 31) / 32; ++w) s += red[w];
      g.alpha_part[blockIdx.x] += s;
    }
  }
  if (timed_out && a.err) atomicExch(a.err, (int)CYL_ERR_TIMEOUT);
}

// Dirichlet data by lifting (reading of the unstated boundary conditions):
// W = transfinite blend of the boundary nodes of bc (linear in r between the
// faces r = -1, +1, plus linear in z between z = -1, +1, minus the bilinear
// corner term), evaluated on every grid node.
__global__ void lift_values_kernel(const double *__restrict__ bc, double *__restrict__ Wv, int p, int m, int n) {
  const long long total = (long long)p * m * n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e % n);
    const int j = (int)((e / n) % m);
    const long long l = e / ((long long)m * n);
    const double r = cospi((double)(m - 1 - j) / (double)(m - 1));
    const double z = cospi((double)(n - 1 - k) / (double)(n - 1));
    const double *B = bc + l * m * n;
    const double r0 = B[(size_t)0 * n + k], r1 = B[(size_t)(m - 1) * n + k];
    const double z0 = B[(size_t)j * n + 0], z1 = B[(size_t)j * n + n - 1];
    const double c00 = B[0], c01 = B[n - 1], c10 = B[(size_t)(m - 1) * n], c11 = B[(size_t)(m - 1) * n + n - 1];
    const double pr = 0.5 * (1.0 - r) * r0 + 0.5 * (1.0 + r) * r1;
    const double pz = 0.5 * (1.0 - z) * z0 + 0.5 * (1.0 + z) * z1;
    const double prz = 0.25 * ((1.0 - r) * (1.0 - z) * c00 + (1.0 - r) * (1.0 + z) * c01 +
                               (1.0 + r) * (1.0 - z) * c10 + (1.0 + r) * (1.0 + z) * c11);
    Wv[e] = pr + pz - prz;
  }
}

// Right-side correction of the lifted problem on every item's class block:
// corr = c1 (L_k W C02^T + R_2 W D2^T) - c0 R_2 W C02^T (tau rows), i.e. minus
// the left operator of the step (c0 = 1, c1 = kappa alpha) or of the Poisson
// problem (c0 = 0, c1 = 1) applied to W.  One CTA per item.
__global__ void lift_correction_kernel(const AdiArgs a, const double *__restrict__ Wc, double *__restrict__ corr,
                                       double c0, double c1) {
  const Item it = a.items[blockIdx.x];
  const int m = it.m, n = it.n, M = it.M, Nz = it.Nz, nsl = it.nsl;
  const long long slice = (long long)m * n;
  const double *r2 = a.fac + it.r2off, *c02 = a.fac + it.c02off, *lk = a.fac + it.lkoff, *d2 = a.fac + it.d2off;
  const double *Wb = Wc + it.xoff;
  double *Cb = corr + it.xoff;
  for (int e = threadIdx.x; e < M * nsl * Nz; e += blockDim.x) {
    const int aa = e / (nsl * Nz), cc = e - aa * (nsl * Nz);
    const int sl = cc / Nz, b = cc - sl * Nz;
    const int i = it.pr + 2 * aa, j = it.pz + 2 * b;
    const double *Ws = Wb + (size_t)(it.s0 + sl) * slice;
    // row-wise z passes of W at radial class row q: (W C02^T)[q][j], (W D2^T)[q][j]
    auto zc = [&](int q) {
      const double *row = Ws + (size_t)(it.pr + 2 * q) * n;
      double s = 0.0;
#pragma unroll
      for (int t = 0; t < 3; ++t)
        if (j + 2 * t < n) s = fma(c02[b * C02STRIDE + t], row[j + 2 * t], s);
      return s;
    };
    auto zd = [&](int q) {
      const double *row = Ws + (size_t)(it.pr + 2 * q) * n;
      return (j + 2 < n) ? d2[b] * row[j + 2] : 0.0;
    };
    double acc = 0.0;
#pragma unroll
    for (int s = -1; s <= 3; ++s) {       // R_2 (c1 W D2^T - c0 W C02^T)
      const int q = aa + s;
      if (q >= 0 && q < it.Mfull) acc = fma(r2[aa * R2STRIDE + s + 1], c1 * zd(q) - c0 * zc(q), acc);
    }
#pragma unroll
    for (int t = 0; t <= 2; ++t) {        // c1 L_k W C02^T
      const int q = aa + t;
      if (q < it.Mfull) acc = fma(c1 * lk[aa * 3 + t], zc(q), acc);
    }
    Cb[(size_t)(it.s0 + sl) * slice + (size_t)i * n + j] = acc;
  }
}

cudaError_t launch_lift_values(const double *bc, double *Wv, int p, int m, int n, cudaStream_t st) {
  const long long N = (long long)p * m * n;
  lift_values_kernel<<<(int)std::min<long long>((N + 255) / 256, 152LL * 16), 256, 0, st>>>(bc, Wv, p, m, n);
  return cudaGetLastError();
}

// corr is written (and later read) only at the items' class positions
cudaError_t launch_lift_correction(const AdiArgs &a, const double *Wc, double *corr, double c0, double c1, int threads,
                                   cudaStream_t st) {
  lift_correction_kernel<<<a.nitems, threads, 0, st>>>(a, Wc, corr, c0, c1);
  return cudaGetLastError();
}

// Horizontal (disk) Poisson, Section 4 eq. ptpoisson: one thread per
// (slice, z-coefficient) column of an item (k, radial class); right side
// R_2 f on the tau rows, LU solve with -L_k, recombination X = S_r Y, all in
// one pass over the column (in place: f may alias u, the right side reads f
// through a register window ahead of the writes).
__global__ void disk_poisson_kernel(const Item *__restrict__ items, const double *__restrict__ fac,
                                    const double *F, double *U, int n, long long slice, int zero_other) {
  const Item it = items[blockIdx.x];
  const int M = it.M, Mf = it.Mfull, W = it.nsl * n;
  const double *H = fac + it.roff, *r2 = fac + it.r2off;
  const size_t st = 2 * (size_t)n;
  for (int cidx = threadIdx.x; cidx < W; cidx += blockDim.x) {
    const int sl = cidx / n, j = cidx - sl * n;
    const size_t base = (size_t)(it.s0 + sl) * slice + (size_t)it.pr * n + j;
    const double *Fc = F + base;
    double *Uc = U + base;
    double f0 = 0.0, f1 = Fc[0];
    double f2 = Mf > 1 ? Fc[st] : 0.0, f3 = Mf > 2 ? Fc[2 * st] : 0.0, f4 = Mf > 3 ? Fc[3 * st] : 0.0;
    double w1 = 0.0, w2 = 0.0;
    for (int a = 0; a < M; ++a) {
      const double *rr = r2 + a * R2STRIDE;
      const double *h = H + a * HSTRIDE;
      double e = rr[0] * f0;
      e = fma(rr[1], f1, e);
      e = fma(rr[2], f2, e);
      e = fma(rr[3], f3, e);
      e = fma(rr[4], f4, e);
      const double fnext = (a + 4 < Mf) ? Fc[(a + 4) * st] : 0.0;
      const double w = fma(h[0], w1, fma(h[1], w2, e));
      Uc[a * st] = w;
      f0 = f1; f1 = f2; f2 = f3; f3 = f4; f4 = fnext;
      w2 = w1;
      w1 = w;
    }
    double y1 = 0.0, y2 = 0.0, y3 = 0.0;
    for (int a = M - 1; a >= 0; --a) {
      const double *h = H + a * HSTRIDE;
      double y = h[5] * Uc[a * st];
      y = fma(h[4], y3, y);
      y = fma(h[3], y2, y);
      y = fma(h[2], y1, y);
      Uc[a * st] = y;
      y3 = y2; y2 = y1; y1 = y;
    }
    // x_a = y_{a-1} - y_a (phi_a = T_{pr+2a+2} - T_{pr+2a}), top down so y_{a-1} is still intact
    for (int a = Mf - 1; a >= 0; --a) {
      const double ya = a < M ? Uc[a * st] : 0.0;
      const double yb = a >= 1 ? Uc[(a - 1) * st] : 0.0;
      Uc[a * st] = yb - ya;
    }
    if (zero_other) {
      double *Uo = U + (size_t)(it.s0 + sl) * slice + (size_t)(1 - it.pr) * n + j;
      const int Mo = (it.m - (1 - it.pr) + 1) / 2;
      for (int a = 0; a < Mo; ++a) Uo[a * st] = 0.0;
    }
  }
}

cudaError_t launch_disk_poisson(const Item *items, int nitems, const double *fac, const double *F, double *U,
                                int n, long long slice, int zero_other, int threads, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  disk_poisson_kernel<<<nitems, threads, 0, st>>>(items, fac, F, U, n, slice, zero_other);
  return cudaGetLastError();
}

// Slot permutation of up to 5 N-element arrays: dst slot k = src slot
// map.src[k] (a negative entry writes zeros).  Each thread owns one element
// position of every slot and reads before it writes, so dst may equal src
// (the history rotation of a BDF run, the adjoint's ring set-up and read-out).
__global__ void permute_slots_kernel(double *dst, const double *src, long long N, int nd, SlotMap map) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
    double v[kMaxSlots];
#pragma unroll
    for (int k = 0; k < kMaxSlots; ++k)
      if (k < nd) v[k] = map.src[k] >= 0 ? src[(size_t)map.src[k] * N + e] : 0.0;
#pragma unroll
    for (int k = 0; k < kMaxSlots; ++k)
      if (k < nd) dst[(size_t)k * N + e] = v[k];
  }
}

cudaError_t launch_permute_slots(double *dst, const double *src, long long N, int nd, const SlotMap &map,
                                 cudaStream_t st) {
  if (nd < 1 || nd > kMaxSlots) return cudaErrorInvalidValue;
  permute_slots_kernel<<<(int)std::min<long long>((N + 255) / 256, 152LL * 16), 256, 0, st>>>(dst, src, N, nd, map);
  return cudaGetLastError();
}

__global__ void sum_partials_kernel(const double *part, int n, double scale, double *out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += part[i];
    *out = s * scale;
  }
}

cudaError_t launch_sum_partials(const double *part, int n, double scale, double *out, cudaStream_t st) {
  sum_partials_kernel<<<1, 32, 0, st>>>(part, n, scale, out);
  return cudaGetLastError();
}

template <bool S_SMEM, bool F_SMEM, int MAXT, bool TW, bool OTW = false>
static cudaError_t launch_adjoint_t(const AdiArgs &a, const AdjointArgs &g, int threads, size_t smem,
                                    cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(adi_adjoint_kernel<S_SMEM, F_SMEM, MAXT, TW, OTW>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  adi_adjoint_kernel<S_SMEM, F_SMEM, MAXT, TW, OTW><<<a.nitems, threads, smem, st>>>(a, g);
  return cudaGetLastError();
}

template <bool S_SMEM, bool F_SMEM>
static cudaError_t launch_adjoint_level(const AdiArgs &a, const AdjointArgs &g, int threads, size_t smem,
                                        cudaStream_t st) {
  if (a.twist_half > 0) {   // twisted records: 2 x 128 threads, or 2 x 256 with Fa in global memory
    if (threads <= 128) return launch_adjoint_t<S_SMEM, F_SMEM, 128, true>(a, g, threads, smem, st);
    if (threads <= 256) return launch_adjoint_t<S_SMEM, F_SMEM, 256, true>(a, g, threads, smem, st);
    if constexpr (!S_SMEM && !F_SMEM) {
      if (a.all_twisted) return launch_adjoint_t<false, false, 512, true, true>(a, g, threads, smem, st);
    }
    if constexpr (!F_SMEM) return launch_adjoint_t<S_SMEM, false, 512, true>(a, g, threads, smem, st);
    else return cudaErrorInvalidValue;
  }
  return threads <= 256 ? launch_adjoint_t<S_SMEM, F_SMEM, 256, false>(a, g, threads, smem, st)
                        : launch_adjoint_t<S_SMEM, F_SMEM, 512, false>(a, g, threads, smem, st);
}

// Instantiations by work-array placement, as the forward kernel; CTAs of at
// most 256 threads get the full register budget.
cudaError_t launch_adjoint(const AdiArgs &a, const AdjointArgs &g, int threads, size_t smem, cudaStream_t st) {
  if (a.nitems <= 0 || g.n_hi <= g.n_lo) return cudaSuccess;
  if (threads > 512) return cudaErrorInvalidValue;
  if (a.use_smem == 2) return launch_adjoint_level<true, true>(a, g, threads, smem, st);
  if (a.use_smem == 1) return launch_adjoint_level<true, false>(a, g, threads, smem, st);
  return launch_adjoint_level<false, false>(a, g, threads, smem, st);
}

template <bool S_SMEM, bool F_SMEM, int MAXT, bool TW, bool OTW = false>
static cudaError_t launch_adi_t(const AdiArgs &a, int threads, size_t smem, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(adi_kernel<S_SMEM, F_SMEM, MAXT, TW, OTW>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  adi_kernel<S_SMEM, F_SMEM, MAXT, TW, OTW><<<a.nitems, threads, smem, st>>>(a);
  return cudaGetLastError();
}

template <bool S_SMEM, bool F_SMEM>
static cudaError_t launch_adi_level(const AdiArgs &a, int threads, size_t smem, cudaStream_t st) {
  if (a.twist_half > 0) {   // twisted plans: 2 x 128 threads, or 2 x 256 with Fa in global memory
    if (threads <= 128) return launch_adi_t<S_SMEM, F_SMEM, 128, true>(a, threads, smem, st);
    if (threads <= 256) return launch_adi_t<S_SMEM, F_SMEM, 256, true>(a, threads, smem, st);
    if constexpr (!S_SMEM && !F_SMEM) {
      if (a.all_twisted) return launch_adi_t<false, false, 512, true, true>(a, threads, smem, st);
    }
    if constexpr (!F_SMEM) return launch_adi_t<S_SMEM, false, 512, true>(a, threads, smem, st);
    else return cudaErrorInvalidValue;
  }
  return threads <= 128   ? launch_adi_t<S_SMEM, F_SMEM, 128, false>(a, threads, smem, st)
         : threads <= 256 ? launch_adi_t<S_SMEM, F_SMEM, 256, false>(a, threads, smem, st)
                          : launch_adi_t<S_SMEM, F_SMEM, 512, false>(a, threads, smem, st);
}

// Blocks of at most 128 and 256 threads get instantiations with a register
// budget of 255 per thread; the twisted sweeps get instantiations of their own.
cudaError_t launch_adi(const AdiArgs &a, int threads, size_t smem, cudaStream_t st) {
  if (a.nitems <= 0 || a.nsteps <= 0) return cudaSuccess;
  if (a.cluster > 1) return launch_adi_cluster(a, threads, smem, st);
  if (threads > 512) return cudaErrorInvalidValue;
  if (a.use_smem == 2) return launch_adi_level<true, true>(a, threads, smem, st);
  if (a.use_smem == 1) return launch_adi_level<true, false>(a, threads, smem, st);
  return launch_adi_level<false, false>(a, threads, smem, st);
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
