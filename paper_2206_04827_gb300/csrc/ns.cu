// Kernels of the Navier-Stokes step in poloidal-toroidal form (Section 4):
// spectral derivatives on CCF coefficients, and the grid-value operations of
// the pseudo-spectral nonlinear term curl(v x omega).  The step itself is
// orchestrated by cyl_ns_step (api.cu) from these, the value <-> coefficient
// transforms, the Poisson and horizontal Poisson solves and the heat step.
//
// All of it is memory-bound elementwise / per-line work next to the
// transforms and ADI solves of the step.
#include <algorithm>

#include "kernels.cuh"

namespace cyl {

namespace {

// d/dtheta on half-complex slices: slice 2w-1 (Re c_w) <- -w Im c_w, slice 2w
// (Im c_w) <- w Re c_w; zero on slice 0 and on the Nyquist slice (whose
// derivative vanishes on the grid).
__global__ void deriv_theta_kernel(const double *__restrict__ in, double *__restrict__ out, int p, long long mn) {
  const long long total = (long long)p * mn;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(e / mn);
    const long long q = e - (long long)s * mn;
    double v = 0.0;
    if (s != 0 && s != p - 1) {
      const int w = (s + 1) >> 1;
      v = (s & 1) ? -w * in[(long long)(s + 1) * mn + q] : w * in[(long long)(s - 1) * mn + q];
    }
    out[e] = v;
  }
}

// d/dx of Chebyshev T-series along lines (o, i), element a at
// o * L * inner + a * inner + i:  c'_{L-1} = 0, c'_{a-1} = c'_{a+1} + 2 a c_a
// (a = L-1 .. 1), then c'_0 halved.  One thread per line, in != out.
__global__ void deriv_cheb_kernel(const double *__restrict__ in, double *__restrict__ out, long long outer, int L,
                                  long long inner) {
  const long long nl = outer * inner;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nl;
       q += (long long)gridDim.x * blockDim.x) {
    const long long o = q / inner, i = q - o * inner;
    const double *x = in + o * L * inner + i;
    double *y = out + o * L * inner + i;
    double d1 = 0.0, d2 = 0.0;                  // c'_{a}, c'_{a+1}
    y[(long long)(L - 1) * inner] = 0.0;
    for (int a = L - 1; a >= 1; --a) {
      const double d0 = fma(2.0 * a, x[(long long)a * inner], d2);   // c'_{a-1}
      y[(long long)(a - 1) * inner] = (a == 1) ? 0.5 * d0 : d0;
      d2 = d1;
      d1 = d0;
    }
  }
}

// dst = (init ? 0 : dst) + coef r_j^rpow src on grid values [p][m][n],
// r_j the radial grid (table of m radii), rpow in {0, -1, -2}.
__global__ void accum_r_kernel(double *__restrict__ dst, const double *__restrict__ src,
                               const double *__restrict__ radius, int m, int n, long long total, double coef, int rpow,
                               int init) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)((e / n) % m);
    double w = coef;
    if (rpow <= -1) w /= radius[j];
    if (rpow <= -2) w /= radius[j];
    const double v = w * src[e];
    dst[e] = init ? v : dst[e] + v;
  }
}

// N = V x W (cylindrical components, grid values).
__global__ void cross_kernel(const double *__restrict__ vr, const double *__restrict__ vt,
                             const double *__restrict__ vz, const double *__restrict__ wr,
                             const double *__restrict__ wt, const double *__restrict__ wz, double *__restrict__ nr,
                             double *__restrict__ nt, double *__restrict__ nz, long long total) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const double a = vr[e], b = vt[e], c = vz[e], x = wr[e], y = wt[e], z = wz[e];
    nr[e] = fma(b, z, -c * y);
    nt[e] = fma(c, x, -a * z);
    nz[e] = fma(a, y, -b * x);
  }
}

int grid_for(long long work, int sms) {
  const long long b = (work + 255) / 256;
  return (int)std::max(1LL, std::min(b, (long long)sms * 16));
}

}  // namespace

cudaError_t launch_deriv_theta(const double *in, double *out, int p, long long mn, int sms, cudaStream_t st) {
  deriv_theta_kernel<<<grid_for((long long)p * mn, sms), 256, 0, st>>>(in, out, p, mn);
  return cudaGetLastError();
}

cudaError_t launch_deriv_cheb(const double *in, double *out, long long outer, int L, long long inner, int sms,
                              cudaStream_t st) {
  deriv_cheb_kernel<<<grid_for(outer * inner, sms), 256, 0, st>>>(in, out, outer, L, inner);
  return cudaGetLastError();
}

cudaError_t launch_accum_r(double *dst, const double *src, const double *radius, int p, int m, int n, double coef,
                           int rpow, bool init, int sms, cudaStream_t st) {
  const long long total = (long long)p * m * n;
  accum_r_kernel<<<grid_for(total, sms), 256, 0, st>>>(dst, src, radius, m, n, total, coef, rpow, init ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_cross(const double *const V[3], const double *const W[3], double *const Nout[3], long long total,
                         int sms, cudaStream_t st) {
  cross_kernel<<<grid_for(total, sms), 256, 0, st>>>(V[0], V[1], V[2], W[0], W[1], W[2], Nout[0], Nout[1], Nout[2],
                                                      total);
  return cudaGetLastError();
}

}  // namespace cyl
