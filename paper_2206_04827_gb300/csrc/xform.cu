// Value <-> coefficient transforms of Section 2 in O(L log L) per line:
// the DCT-I in r and in z (Chebyshev points, any length L) and the DFT in
// theta (half-complex coefficients), each as a chirp-z (Bluestein) product.
//
// Every transform here has the form
//     out_j = post_j * sum_a pre_a x_a exp(i sigma pi (j a) / D)
// (j, a ranging over consecutive integers, possibly negative), and with
// j a = (j^2 + a^2 - (j - a)^2) / 2 and c_t = exp(i sigma pi t^2 / (2 D))
// the kernel factors as c_j c_a conj(c_{j-a}).  So out = post' * (u (*) h)
// with u_a = pre_a c_a x_a and h_t = conj(c_t): a linear convolution, done
// as a circular one of a power-of-two length P through two FFTs and one
// pointwise product with the precomputed spectrum of h.
//
//   DCT-I forward (Section 2: c_j = (2/N) w_j sum_a w_a f_a T_j(x_a), N = L-1,
//     x_a = cos((N - a) pi / N), w = 1/2 at both ends): T_j(x_a) =
//     (-1)^j cos(pi j a / N), so sigma = +1, D = N, pre = w_a,
//     post = (2/N) w_j (-1)^j, real part.  One real line per complex FFT.
//   DCT-I inverse (f_a = sum_j c_j T_j(x_a)): pre = (-1)^j, post = 1.
//   DFT forward (c_w = (1/p) sum_l f_l exp(-i w theta_l), theta_l =
//     (2l - p) pi / p, so exp(-i w theta_l) = (-1)^w exp(-2 pi i w l / p)):
//     sigma = -1, D = p/2, outputs w = -(p/2-1) .. p/2.  Two real lines
//     ride in one complex FFT (x = f + i g); their spectra separate by
//     F_w = (Z_w + conj Z_{-w}) / 2, G_w = (Z_w - conj Z_{-w}) / (2i).
//   DFT inverse (f_l = sum_w C_w exp(i w theta_l) over w = -p/2 .. p/2-1,
//     C Hermitian): sigma = +1, D = p/2, pre = (-1)^w; two lines as
//     X_w = A_w + i B_w, f = Re, g = Im of the result.
//
// FFT: radix-2, decimation in frequency for the forward transform (natural
// order in, bit-reversed out), pointwise product with the kernel spectrum
// stored in bit-reversed order (scaled by 1/P), decimation in time with
// conjugate twiddles for the inverse (bit-reversed in, natural out): no
// permutation pass.  G complex FFTs of one CTA live in shared memory.
//
// FP64 work per complex FFT: P/2 log2 P butterflies of 8 operations (4 in
// the two stages whose twiddles are 1 and -i); the transforms are bound by
// the FP64 pipe (GB300's FP64 rate is far below its memory bandwidth), not by
// HBM.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/cyl.h"
#include "kernels.cuh"

namespace cyl {

namespace {

constexpr double kPi = 3.14159265358979323846;

int bitrev(int k, int logP) {
  int r = 0;
  for (int b = 0; b < logP; ++b) r |= ((k >> b) & 1) << (logP - 1 - b);
  return r;
}

// (cos, sin)(pi * num / den) for 0 <= num < 2 den, reduced exactly to [0, pi/4]
// so that the rounding of pi enters only through a small argument.
void cis_pi(long long num, long long den, double &c, double &s) {
  num %= 2 * den;
  if (num < 0) num += 2 * den;
  // angle = pi num / den in [0, 2 pi): quadrant q = floor(4 num / (2 den))... reduce by halves
  double sgn_c = 1.0, sgn_s = 1.0;
  if (num >= den) {               // angle - pi
    num -= den;
    sgn_c = -sgn_c;
    sgn_s = -sgn_s;
  }
  bool swap = false;
  if (2 * num > den) {            // pi - angle in [0, pi/2)
    num = den - num;
    sgn_c = -sgn_c;
  }
  if (4 * num > den) {            // pi/2 - angle in [0, pi/4]
    // cos(x) = sin(pi/2 - x), sin(x) = cos(pi/2 - x); pi/2 - pi num/den = pi (den - 2 num) / (2 den)
    const double a = kPi * (double)(den - 2 * num) / (2.0 * (double)den);
    c = sgn_c * std::sin(a);
    s = sgn_s * std::cos(a);
    swap = true;
  }
  if (!swap) {
    const double a = kPi * (double)num / (double)den;
    c = sgn_c * std::cos(a);
    s = sgn_s * std::sin(a);
  }
}

// c_t = exp(i sigma pi t^2 / (2 D)) (period 4D in t^2)
void chirp(long long t, long long D, int sigma, double &re, double &im) {
  const long long r = (t * t) % (4 * D);
  double c, s;
  cis_pi(r, 2 * D, c, s);
  re = c;
  im = sigma * s;
}

}  // namespace

std::vector<double> xform_tables(int kind, int L, XformDesc &d) {
  // kind 0 DCT-I forward, 1 DCT-I inverse (length L >= 2), 2 DFT forward, 3 DFT inverse (L = p even)
  d = XformDesc{};
  d.kind = kind;
  d.L = L;
  long long D;
  int sigma;
  int ia0, jb0;
  if (kind <= 1) {
    D = L - 1;
    sigma = +1;
    d.A = d.B = L;
    ia0 = jb0 = 0;
  } else {
    D = L / 2;
    d.A = d.B = L;
    if (kind == 2) {
      sigma = -1;
      ia0 = 0;
      jb0 = -(L / 2 - 1);
    } else {
      sigma = +1;
      ia0 = -(L / 2);
      jb0 = 0;
    }
  }
  d.ia0 = ia0;
  d.jb0 = jb0;
  const long long tmin = (long long)jb0 - (ia0 + d.A - 1), tmax = (long long)jb0 + d.B - 1 - ia0;
  int P = 1, logP = 0;
  while (P < tmax - tmin + 1) {
    P <<= 1;
    ++logP;
  }
  if (P < 2) {
    P = 2;
    logP = 1;
  }
  d.P = P;
  d.logP = logP;
  // layout of the table block (doubles): pre [2A], post [2B], Hbr [2P], tw [P]
  d.pre_off = 0;
  d.post_off = 2LL * d.A;
  d.H_off = d.post_off + 2LL * d.B;
  d.tw_off = d.H_off + 2LL * P;
  std::vector<double> t((size_t)(d.tw_off + P), 0.0);
  const long long N = L - 1;
  for (int a = 0; a < d.A; ++a) {
    const long long ia = ia0 + a;
    double alpha = 1.0;
    if (kind == 0) alpha = (ia == 0 || ia == N) ? 0.5 : 1.0;
    if (kind == 1 || kind == 3) alpha = (ia % 2 == 0) ? 1.0 : -1.0;
    double cr, ci;
    chirp(ia, D, sigma, cr, ci);
    t[d.pre_off + 2 * a] = alpha * cr;
    t[d.pre_off + 2 * a + 1] = alpha * ci;
  }
  for (int b = 0; b < d.B; ++b) {
    const long long jb = jb0 + b;
    double beta = 1.0;
    if (kind == 0) beta = (2.0 / (double)N) * ((jb == 0 || jb == N) ? 0.5 : 1.0) * ((jb % 2 == 0) ? 1.0 : -1.0);
    if (kind == 2) beta = (((jb % 2) + 2) % 2 == 0 ? 1.0 : -1.0) / (double)L;
    double cr, ci;
    chirp(jb, D, sigma, cr, ci);
    t[d.post_off + 2 * b] = beta * cr;
    t[d.post_off + 2 * b + 1] = beta * ci;
  }
  // h at circular positions, then its DFT (direct sum, exact twiddle indices), bit-reversed / P
  std::vector<double> hr(P, 0.0), hi(P, 0.0), cs(P), sn(P);
  for (long long tt = tmin; tt <= tmax; ++tt) {
    double cr, ci;
    chirp(tt, D, sigma, cr, ci);
    const long long s = ((tt % P) + P) % P;
    hr[s] = cr;
    hi[s] = -ci;                  // conj(c_t)
  }
  for (int k = 0; k < P; ++k) cis_pi(2LL * k, P, cs[k], sn[k]);   // exp(2 pi i k / P)
  for (int k = 0; k < P; ++k) {
    double sr = 0.0, si = 0.0;
    for (int s = 0; s < P; ++s) {
      const int q = (int)(((long long)k * s) % P);
      // h_s exp(-2 pi i k s / P)
      sr += hr[s] * cs[q] + hi[s] * sn[q];
      si += hi[s] * cs[q] - hr[s] * sn[q];
    }
    const int kb = bitrev(k, logP);
    t[d.H_off + 2 * kb] = sr / P;
    t[d.H_off + 2 * kb + 1] = si / P;
  }
  for (int k = 0; k < P / 2; ++k) {         // forward twiddles exp(-2 pi i k / P)
    t[d.tw_off + 2 * k] = cs[k];
    t[d.tw_off + 2 * k + 1] = -sn[k];
  }
  return t;
}

namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

// G complex FFT buffers of length P in shared memory, radix-2 stages fused
// in pairs: each thread takes a quad of elements through two stages in
// registers (half the shared-memory passes and barriers of one stage at a
// time, the same operations in the same order).  The two stages of span 1
// and 2 need no multiplication: their twiddles are tw[0] = 1 and
// tw[P/4] = -i, which the host tables hold exactly, so (a, b) * -i is
// (b, -a) and the results equal those of the full complex products.
// DIF forward: natural -> bit-reversed.  DIT inverse with conjugate
// twiddles: bit-reversed -> natural.
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

// one DIF stage of span h = 2^lh over all G buffers
__device__ __forceinline__ void dif_stage(double2 *buf, int G, int P, int lh, const double2 *__restrict__ tw) {
  const int half = P >> 1, h = 1 << lh, tstep = half >> lh;
  for (int b = threadIdx.x; b < G * half; b += blockDim.x) {
    const int g = b / half, r = b - g * half;
    const int pos = r & (h - 1), grp = r >> lh;
    double2 *x = buf + (size_t)g * P + grp * 2 * h + pos;
    const double2 x0 = x[0], x1 = x[h];
    x[0] = cadd(x0, x1);
    x[h] = cmul(csub(x0, x1), __ldg(tw + pos * tstep));
  }
  __syncthreads();
}

__device__ __forceinline__ void fft_dif(double2 *buf, int G, int P, int logP, const double2 *__restrict__ tw) {
  const int quarter = P >> 2;
  int lh = logP - 1;
  // stage pairs (lh, lh - 1), spans H and H/2, on quads pos, pos + H/2, pos + H, pos + 3H/2 of a 2H block
  for (; lh >= 3; lh -= 2) {
    const int H2 = 1 << (lh - 1), ts1 = (P >> 1) >> lh, ts2 = 2 * ts1;
    for (int b = threadIdx.x; b < G * quarter; b += blockDim.x) {
      const int g = b / quarter, q = b - g * quarter;
      const int pos = q & (H2 - 1), blk = q >> (lh - 1);
      double2 *x = buf + (size_t)g * P + blk * 4 * H2 + pos;
      const double2 a0 = x[0], a1 = x[H2], a2 = x[2 * H2], a3 = x[3 * H2];
      const double2 w1 = __ldg(tw + pos * ts1), w1b = __ldg(tw + (pos + H2) * ts1), w2 = __ldg(tw + pos * ts2);
      const double2 b0 = cadd(a0, a2), b2 = cmul(csub(a0, a2), w1);
      const double2 b1 = cadd(a1, a3), b3 = cmul(csub(a1, a3), w1b);
      x[0] = cadd(b0, b1);
      x[H2] = cmul(csub(b0, b1), w2);
      x[2 * H2] = cadd(b2, b3);
      x[3 * H2] = cmul(csub(b2, b3), w2);
    }
    __syncthreads();
  }
  if (lh == 2) {
    dif_stage(buf, G, P, 2, tw);
    lh = 1;
  }
  if (lh == 1) {      // spans 2 and 1 on quads of consecutive elements: twiddles 1 and -i, then 1
    for (int b = threadIdx.x; b < G * quarter; b += blockDim.x) {
      double2 *x = buf + (size_t)4 * b;
      const double2 a0 = x[0], a1 = x[1], a2 = x[2], a3 = x[3];
      const double2 b0 = cadd(a0, a2), b2 = csub(a0, a2);
      const double2 b1 = cadd(a1, a3), d13 = csub(a1, a3);
      const double2 b3 = make_double2(d13.y, -d13.x);
      x[0] = cadd(b0, b1);
      x[1] = csub(b0, b1);
      x[2] = cadd(b2, b3);
      x[3] = csub(b2, b3);
    }
    __syncthreads();
  } else if (lh == 0) {
    dif_stage(buf, G, P, 0, tw);
  }
}

// one DIT stage (conjugate twiddles) of span h = 2^lh
__device__ __forceinline__ void dit_stage(double2 *buf, int G, int P, int lh, const double2 *__restrict__ tw) {
  const int half = P >> 1, h = 1 << lh, tstep = half >> lh;
  for (int b = threadIdx.x; b < G * half; b += blockDim.x) {
    const int g = b / half, r = b - g * half;
    const int pos = r & (h - 1), grp = r >> lh;
    double2 *x = buf + (size_t)g * P + grp * 2 * h + pos;
    const double2 x0 = x[0];
    const double2 t = cmul(x[h], cconj(__ldg(tw + pos * tstep)));
    x[0] = cadd(x0, t);
    x[h] = csub(x0, t);
  }
  __syncthreads();
}

__device__ __forceinline__ void fft_dit_inv(double2 *buf, int G, int P, int logP, const double2 *__restrict__ tw) {
  const int quarter = P >> 2;
  int lh = 0;
  if (logP >= 2) {    // spans 1 and 2 on quads of consecutive elements: twiddles 1, then 1 and +i
    for (int b = threadIdx.x; b < G * quarter; b += blockDim.x) {
      double2 *x = buf + (size_t)4 * b;
      const double2 a0 = x[0], a1 = x[1], a2 = x[2], a3 = x[3];
      const double2 b0 = cadd(a0, a1), b1 = csub(a0, a1);
      const double2 b2 = cadd(a2, a3), b3 = csub(a2, a3);
      const double2 t3 = make_double2(-b3.y, b3.x);
      x[0] = cadd(b0, b2);
      x[2] = csub(b0, b2);
      x[1] = cadd(b1, t3);
      x[3] = csub(b1, t3);
    }
    __syncthreads();
    lh = 2;
  }
  // stage pairs (lh, lh + 1), spans h and 2h, on quads pos, pos + h, pos + 2h, pos + 3h of a 4h block
  for (; lh + 1 < logP; lh += 2) {
    const int h = 1 << lh, tsA = (P >> 1) >> lh, tsB = tsA >> 1;
    for (int b = threadIdx.x; b < G * quarter; b += blockDim.x) {
      const int g = b / quarter, q = b - g * quarter;
      const int pos = q & (h - 1), blk = q >> lh;
      double2 *x = buf + (size_t)g * P + blk * 4 * h + pos;
      const double2 a0 = x[0], a1 = x[h], a2 = x[2 * h], a3 = x[3 * h];
      const double2 wA = cconj(__ldg(tw + pos * tsA));
      const double2 wB = cconj(__ldg(tw + pos * tsB)), wBb = cconj(__ldg(tw + (pos + h) * tsB));
      const double2 t1 = cmul(a1, wA), t3 = cmul(a3, wA);
      const double2 b0 = cadd(a0, t1), b1 = csub(a0, t1);
      const double2 b2 = cadd(a2, t3), b3 = csub(a2, t3);
      const double2 u2 = cmul(b2, wB), u3 = cmul(b3, wBb);
      x[0] = cadd(b0, u2);
      x[2 * h] = csub(b0, u2);
      x[h] = cadd(b1, u3);
      x[3 * h] = csub(b1, u3);
    }
    __syncthreads();
  }
  if (lh < logP) dit_stage(buf, G, P, lh, tw);
}

// KIND 0: DCT-I (forward or inverse by its tables), one real line per FFT.
// KIND 2: DFT forward, values -> half-complex, two lines per FFT.
// KIND 3: DFT inverse, half-complex -> values, two lines per FFT.
// Lines: line q = (o, i), o = q / inner, i = q % inner; element a of line q
// at o * L * inner + a * inner + i.  in may equal out (each CTA reads all
// its lines before it writes them).
template <int KIND>
__global__ void __launch_bounds__(256, 6) chirp_xform_kernel(const double *in, double *out, const double *tab,
                                                          XformDesc d, long long outer, long long inner, int G) {
  extern __shared__ __align__(16) double2 xbuf[];
  const double2 *pre = reinterpret_cast<const double2 *>(tab + d.pre_off);
  const double2 *post = reinterpret_cast<const double2 *>(tab + d.post_off);
  const double2 *Hbr = reinterpret_cast<const double2 *>(tab + d.H_off);
  const double2 *tw = reinterpret_cast<const double2 *>(tab + d.tw_off);
  const int P = d.P, L = d.L;
  constexpr int LPF = KIND == 0 ? 1 : 2;                  // real lines per complex FFT
  const long long nlines = outer * inner;
  const long long nfft = (nlines + LPF - 1) / LPF;
  const int Pm = P - 1;
  __shared__ long long lbase[2 * kMaxXformFfts];     // first element of each line of this FFT group, or -1
  for (long long f0 = (long long)blockIdx.x * G; f0 < nfft; f0 += (long long)gridDim.x * G) {
    const int Gc = (int)min((long long)G, nfft - f0);     // FFTs in this group
    const long long q0 = f0 * LPF;
    const int nl = (int)min((long long)Gc * LPF, nlines - q0);
    for (int e = threadIdx.x; e < Gc * LPF; e += blockDim.x) {
      const long long q = q0 + e;
      long long b = -1;
      if (e < nl) {
        const long long o = q / inner;
        b = o * L * inner + (q - o * inner);
      }
      lbase[e] = b;
    }
    for (int e = threadIdx.x; e < Gc * P; e += blockDim.x) xbuf[e] = make_double2(0.0, 0.0);
    __syncthreads();
    // ---- load: u_a = pre_a x_a at circular slot (ia0 + a) mod P
    for (int e = threadIdx.x; e < Gc * d.A; e += blockDim.x) {
      int g, a;
      if (inner == 1) { g = e / d.A; a = e - g * d.A; }
      else { a = e / Gc; g = e - a * Gc; }
      const int slot = (d.ia0 + a) & Pm;
      double2 x;
      if (KIND == 0) {
        x = make_double2(in[lbase[g] + a * inner], 0.0);
      } else {
        const long long ba = lbase[2 * g], bb = lbase[2 * g + 1];
        if (KIND == 2) {
          x = make_double2(in[ba + a * inner], bb >= 0 ? in[bb + a * inner] : 0.0);
        } else {
          // X_w = A_w + i B_w from the half-complex slots, w = a - p/2
          const int w = a - L / 2;
          const int v = w < 0 ? -w : w;
          auto hc = [&](long long base) -> double2 {
            if (base < 0) return make_double2(0.0, 0.0);
            if (v == 0) return make_double2(in[base], 0.0);
            if (v == L / 2) return make_double2(in[base + (long long)(L - 1) * inner], 0.0);
            const double re = in[base + (long long)(2 * v - 1) * inner], im = in[base + (long long)(2 * v) * inner];
            return make_double2(re, w < 0 ? -im : im);
          };
          const double2 Aw = hc(ba), Bw = hc(bb);
          x = make_double2(Aw.x - Bw.y, Aw.y + Bw.x);
        }
      }
      xbuf[(size_t)g * P + slot] = cmul(__ldg(pre + a), x);
    }
    __syncthreads();
    fft_dif(xbuf, Gc, P, d.logP, tw);
    for (int e = threadIdx.x; e < Gc * P; e += blockDim.x) xbuf[e] = cmul(xbuf[e], __ldg(Hbr + (e & Pm)));
    __syncthreads();
    fft_dit_inv(xbuf, Gc, P, d.logP, tw);
    // ---- store
    if (KIND == 0) {
      for (int e = threadIdx.x; e < nl * d.B; e += blockDim.x) {
        int g, b;
        if (inner == 1) { g = e / d.B; b = e - g * d.B; }
        else { b = e / nl; g = e - b * nl; }
        const double2 y = xbuf[(size_t)g * P + ((d.jb0 + b) & Pm)];
        const double2 c = __ldg(post + b);
        out[lbase[g] + b * inner] = fma(c.x, y.x, -c.y * y.y);
      }
    } else if (KIND == 2) {
      // half-complex slot s of line gl: s = 0 -> w 0; s = 2w-1 / 2w -> Re / Im of w; s = L-1 -> w = L/2
      for (int e = threadIdx.x; e < nl * L; e += blockDim.x) {
        int gl, s;
        if (inner == 1) { gl = e / L; s = e - gl * L; }
        else { s = e / nl; gl = e - s * nl; }
        const int g = gl >> 1, part = gl & 1;
        const double2 *Y = xbuf + (size_t)g * P;
        int w;
        if (s == 0) w = 0;
        else if (s == L - 1) w = L / 2;
        else w = (s + 1) >> 1;
        const int bw = w - d.jb0;
        const double2 Zw = cmul(__ldg(post + bw), Y[(d.jb0 + bw) & Pm]);
        double val;
        if (w == 0 || w == L / 2) {
          val = part == 0 ? Zw.x : Zw.y;
        } else {
          const int bm = -w - d.jb0;
          const double2 Zm = cmul(__ldg(post + bm), Y[(d.jb0 + bm) & Pm]);
          const bool im = (s & 1) == 0;
          if (part == 0) val = im ? 0.5 * (Zw.y - Zm.y) : 0.5 * (Zw.x + Zm.x);
          else val = im ? 0.5 * (Zm.x - Zw.x) : 0.5 * (Zw.y + Zm.y);
        }
        out[lbase[gl] + s * inner] = val;
      }
    } else {
      for (int e = threadIdx.x; e < nl * L; e += blockDim.x) {
        int gl, l;
        if (inner == 1) { gl = e / L; l = e - gl * L; }
        else { l = e / nl; gl = e - l * nl; }
        const int g = gl >> 1, part = gl & 1;
        const double2 y = cmul(__ldg(post + l), xbuf[(size_t)g * P + ((d.jb0 + l) & Pm)]);
        out[lbase[gl] + l * inner] = part == 0 ? y.x : y.y;
      }
    }
    __syncthreads();
  }
}

}  // namespace

// 32 KB of FFT buffers per CTA (8 FFTs of 256 points): seven 256-thread CTAs per SM, so that the
// FFT groups of a pass spread over the resident CTAs in nearly whole waves.
int xform_ffts_per_cta(int P) {
  int G = (int)(32768 / (16 * (long long)P));
  return G < 1 ? 1 : (G > kMaxXformFfts ? kMaxXformFfts : G);
}


template <int KIND>
static cudaError_t launch_xform_t(const double *in, double *out, const double *tab, const XformDesc &d,
                                  long long outer, long long inner, int G, long long groups, int sms, cudaStream_t st) {
  const size_t smem = (size_t)G * d.P * 16;
  cudaError_t e = cudaFuncSetAttribute(chirp_xform_kernel<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, chirp_xform_kernel<KIND>, 256, smem);
  if (e != cudaSuccess) return e;
  // one CTA per FFT group while they fit the resident CTAs, else the resident CTAs loop (grid stride)
  const long long blocks = std::max(1LL, std::min(groups, (long long)sms * std::max(1, per_sm)));
  chirp_xform_kernel<KIND><<<(int)blocks, 256, smem, st>>>(in, out, tab, d, outer, inner, G);
  return cudaGetLastError();
}

cudaError_t launch_xform(const double *in, double *out, const double *tab, const XformDesc &d, long long outer,
                         long long inner, int sms, cudaStream_t st) {
  const long long nlines = outer * inner;
  if (nlines <= 0) return cudaSuccess;
  const int G = xform_ffts_per_cta(d.P);
  const long long nfft = d.kind <= 1 ? nlines : (nlines + 1) / 2;
  const long long groups = (nfft + G - 1) / G;
  switch (d.kind) {
    case 0:
    case 1: return launch_xform_t<0>(in, out, tab, d, outer, inner, G, groups, sms, st);
    case 2: return launch_xform_t<2>(in, out, tab, d, outer, inner, G, groups, sms, st);
    default: return launch_xform_t<3>(in, out, tab, d, outer, inner, G, groups, sms, st);
  }
}

}  // namespace cyl

extern "C" cyl_status cyl_xform_table(int kind, int L, int *info, double *table) {
  if (!info || kind < 0 || kind > 3 || L < 2 || L > 4096 || (kind >= 2 && (L & 1))) return CYL_EINVAL;
  cyl::XformDesc d;
  std::vector<double> t;
  try {
    t = cyl::xform_tables(kind, L, d);
  } catch (...) {
    return CYL_ENOMEM;
  }
  const long long v[11] = {d.P, d.logP, d.A, d.B, d.ia0, d.jb0, d.pre_off, d.post_off, d.H_off, d.tw_off,
                           (long long)t.size()};
  for (int i = 0; i < 11; ++i) info[i] = (int)v[i];
  if (table) std::memcpy(table, t.data(), t.size() * sizeof(double));
  return CYL_OK;
}
