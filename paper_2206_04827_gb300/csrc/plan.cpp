// Host plan of libcyl: operators, spectral intervals, Zolotarev shifts,
// banded factors and transform matrices.  Everything here runs once per plan
// on the host, in float64.
//
// Paper passages restated here (arXiv 2206.04827):
//   Section 2, Definition "grid" and interpolant f*   -> transform matrices
//   Section 3, operator list (C01, C12, C02, R, R_2, D1, D2) -> band builders
//   Section 3, eq. HelmholtzMatEqn                     -> A, B, C, D per mode
//   Section 3, shift paragraph below Algorithm 1       -> zolotarev()
#include "plan.hpp"

#include <algorithm>
#include <cmath>
#include <cstdio>

namespace cyl {
namespace {

const double PI = 3.14159265358979323846;

// ---------------------------------------------------------------- operators
// Section 3 operators as m x m bands, from the classical three-term relations
// (Abramowitz-Stegun normalisation of C^(1) = U and C^(2)).

Band op_C01(int m) {   // T -> U: T_0 = U_0, T_j = (U_j - U_{j-2}) / 2
  Band B(m, 0, 2);
  B.at(0, 0) = 1.0;
  for (int j = 1; j < m; ++j) {
    B.at(j, j) = 0.5;
    if (j >= 2) B.at(j - 2, j) = -0.5;
  }
  return B;
}

Band op_C12(int m) {   // U -> C^(2): U_j = (C2_j - C2_{j-2}) / (j + 1)
  Band B(m, 0, 2);
  for (int j = 0; j < m; ++j) {
    B.at(j, j) = 1.0 / (j + 1.0);
    if (j >= 2) B.at(j - 2, j) = -1.0 / (j + 1.0);
  }
  return B;
}

Band op_R(int m) {     // x C2_j = ((j+1) C2_{j+1} + (j+3) C2_{j-1}) / (2j + 4)
  Band B(m, 1, 1);
  for (int j = 0; j < m; ++j) {
    if (j + 1 < m) B.at(j + 1, j) = (j + 1.0) / (2.0 * j + 4.0);
    if (j >= 1) B.at(j - 1, j) = (j + 3.0) / (2.0 * j + 4.0);
  }
  return B;
}

Band op_D1(int m) {    // d/dx T_j = j U_{j-1}
  Band B(m, 0, 1);
  for (int j = 1; j < m; ++j) B.at(j - 1, j) = (double)j;
  return B;
}

Band op_D2(int m) {    // d^2/dx^2 T_j = 2 j C2_{j-2}
  Band B(m, 0, 2);
  for (int j = 2; j < m; ++j) B.at(j - 2, j) = 2.0 * j;
  return B;
}

Band mul(const Band &A, const Band &B) {
  Band C(A.n, A.lo + B.lo, A.hi + B.hi);
  for (int i = 0; i < A.n; ++i)
    for (int l = std::max(0, i - A.lo); l <= std::min(A.n - 1, i + A.hi); ++l) {
      const double a = A.get(i, l);
      if (a == 0.0) continue;
      for (int j = std::max(0, l - B.lo); j <= std::min(B.n - 1, l + B.hi); ++j) C.at(i, j) += a * B.get(l, j);
    }
  return C;
}

Band axpby(double x, const Band &A, double y, const Band &B) {
  Band C(A.n, std::max(A.lo, B.lo), std::max(A.hi, B.hi));
  for (int i = 0; i < A.n; ++i)
    for (int j = std::max(0, i - C.lo); j <= std::min(A.n - 1, i + C.hi); ++j)
      C.at(i, j) = x * A.get(i, j) + y * B.get(i, j);
  return C;
}

// Dirichlet recombination and tau truncation: P X S with S[j][j] = -1,
// S[j+2][j] = 1 (phi_j = T_{j+2} - T_j), P keeping the first m-2 rows.
Band recomb(const Band &X) {
  const int n2 = X.n - 2;
  Band Y(n2, X.lo + 2, X.hi);
  for (int i = 0; i < n2; ++i)
    for (int j = std::max(0, i - Y.lo); j <= std::min(n2 - 1, i + Y.hi); ++j)
      Y.at(i, j) = -X.get(i, j) + X.get(i, j + 2);
  return Y;
}

// Parity block of a band whose offsets are all even: rows/cols i = par + 2a.
Band block(const Band &Y, int par) {
  const int nb = (Y.n - par + 1) / 2;
  Band B(std::max(nb, 0), Y.lo / 2, Y.hi / 2);
  for (int a = 0; a < B.n; ++a)
    for (int b = std::max(0, a - B.lo); b <= std::min(B.n - 1, a + B.hi); ++b)
      B.at(a, b) = Y.get(par + 2 * a, par + 2 * b);
  return B;
}

// In-place LU without pivoting (L unit lower, multipliers stored below the diagonal).
bool lu_inplace(Band &A) {
  for (int c = 0; c < A.n; ++c) {
    const double piv = A.get(c, c);
    if (!(std::fabs(piv) > 0.0) || !std::isfinite(piv)) return false;
    for (int r = c + 1; r <= std::min(A.n - 1, c + A.lo); ++r) {
      const double l = A.get(r, c) / piv;
      A.at(r, c) = l;
      for (int j = c + 1; j <= std::min(A.n - 1, c + A.hi); ++j) A.at(r, j) -= l * A.get(c, j);
    }
  }
  return true;
}

void lu_solve(const Band &LU, std::vector<double> &x) {
  const int n = LU.n;
  for (int i = 0; i < n; ++i)
    for (int l = std::max(0, i - LU.lo); l < i; ++l) x[i] -= LU.get(i, l) * x[l];
  for (int i = n - 1; i >= 0; --i) {
    for (int l = i + 1; l <= std::min(n - 1, i + LU.hi); ++l) x[i] -= LU.get(i, l) * x[l];
    x[i] /= LU.get(i, i);
  }
}

// UL factorization without pivoting, eliminating from the bottom up:
// A = Ut Lt with Ut unit upper (its multipliers stored in the strict upper
// band) and Lt lower (stored on and below the diagonal).
bool ul_inplace(Band &A) {
  for (int c = A.n - 1; c >= 0; --c) {
    const double piv = A.get(c, c);
    if (!(std::fabs(piv) > 0.0) || !std::isfinite(piv)) return false;
    for (int r = c - 1; r >= std::max(0, c - A.hi); --r) {
      const double u = A.get(r, c) / piv;
      A.at(r, c) = u;
      for (int j = std::max(0, c - A.lo); j < c; ++j)
        if (A.in(r, j)) A.at(r, j) -= u * A.get(c, j);
    }
  }
  return true;
}

// Solve the dense n x n system K X = B (row-major, B n x nr) in place by
// Gaussian elimination with partial pivoting; false if K is singular.
static bool dense_solve(std::vector<double> K, int n, std::vector<double> &B, int nr) {
  for (int c = 0; c < n; ++c) {
    int pv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(K[r * n + c]) > std::fabs(K[pv * n + c])) pv = r;
    if (!(std::fabs(K[pv * n + c]) > 0.0)) return false;
    if (pv != c) {
      for (int j = 0; j < n; ++j) std::swap(K[c * n + j], K[pv * n + j]);
      for (int j = 0; j < nr; ++j) std::swap(B[c * nr + j], B[pv * nr + j]);
    }
    for (int r = c + 1; r < n; ++r) {
      const double f = K[r * n + c] / K[c * n + c];
      if (f == 0.0) continue;
      for (int j = c; j < n; ++j) K[r * n + j] -= f * K[c * n + j];
      for (int j = 0; j < nr; ++j) B[r * nr + j] -= f * B[c * nr + j];
    }
  }
  for (int c = n - 1; c >= 0; --c)
    for (int j = 0; j < nr; ++j) {
      double s = B[c * nr + j];
      for (int l = c + 1; l < n; ++l) s -= K[c * n + l] * B[l * nr + j];
      B[c * nr + j] = s / K[c * n + c];
    }
  return true;
}

// Interface block of a twisted banded solve T z = s * rhs (s = scale): the
// top rows are LU rows (U z = s w), the bottom rows UL rows (Lt z = s v).
// Unknowns z_{k-lo} .. z_{k+w+hi-1} (w = max(lo, hi) interface rows k ..
// k+w-1); equations: U rows k-lo .. k-1, T rows k .. k+w-1, Lt rows k+w ..
// k+w+hi-1.  Returns the rows of the solution map for z_k .. z_{k+nout-1}
// (nout x neq, row-major), scaled by s.
static bool twist_interface(const Band &T, const Band &LU, const Band &UL, int k, int nout, double s,
                            std::vector<double> &R) {
  const int lo = T.lo, hi = T.hi, w = std::max(lo, hi), n0 = k - lo, neq = lo + w + hi;
  std::vector<double> K((size_t)neq * neq, 0.0), E((size_t)neq * neq, 0.0);
  for (int r = 0; r < neq; ++r) {
    const int i = n0 + r;
    for (int cidx = 0; cidx < neq; ++cidx) {
      const int j = n0 + cidx;
      double v;
      if (r < lo) v = (j >= i) ? LU.get(i, j) : 0.0;          // U row
      else if (r < lo + w) v = T.get(i, j);                   // equation row
      else v = (j <= i) ? UL.get(i, j) : 0.0;                 // Lt row
      K[(size_t)r * neq + cidx] = v;
    }
    E[(size_t)r * neq + r] = 1.0;
  }
  if (!dense_solve(K, neq, E, neq)) return false;             // E = K^-1
  R.assign((size_t)nout * neq, 0.0);
  for (int o = 0; o < nout; ++o)
    for (int cidx = 0; cidx < neq; ++cidx) R[(size_t)o * neq + cidx] = s * E[(size_t)(lo + o) * neq + cidx];
  return true;
}

std::vector<double> matvec(const Band &A, const std::vector<double> &x) {
  std::vector<double> y(A.n, 0.0);
  for (int i = 0; i < A.n; ++i)
    for (int j = std::max(0, i - A.lo); j <= std::min(A.n - 1, i + A.hi); ++j) y[i] += A.get(i, j) * x[j];
  return y;
}

double norm2(const std::vector<double> &x) {
  double s = 0;
  for (double v : x) s += v * v;
  return std::sqrt(s);
}

// Extreme eigenvalues of the pencil K = -Den^-1 Num (real and positive for the
// radial and vertical Laplacian pencils of this method): power iteration for
// the largest, inverse iteration for the smallest.
bool pencil_extremes(const Band &Num, const Band &Den, double &lmin, double &lmax) {
  const int n = Num.n;
  if (n == 1) {
    lmin = lmax = -Num.get(0, 0) / Den.get(0, 0);
    return lmin > 0;
  }
  Band LD = Den, LN = Num;
  if (!lu_inplace(LD) || !lu_inplace(LN)) return false;
  auto start = [n]() {
    std::vector<double> x(n);
    for (int i = 0; i < n; ++i) x[i] = 1.0 + 0.37 * std::sin(1.7 * i + 0.3);
    return x;
  };
  std::vector<double> x = start();
  double nx = norm2(x), est = 0, prev = -1;
  for (double &v : x) v /= nx;
  for (int it = 0; it < 4000; ++it) {
    std::vector<double> y = matvec(Num, x);
    for (double &v : y) v = -v;
    lu_solve(LD, y);
    est = norm2(y);
    if (!(est > 0) || !std::isfinite(est)) return false;
    for (int i = 0; i < n; ++i) x[i] = y[i] / est;
    if (it > 60 && std::fabs(est - prev) <= 1e-12 * est) break;
    prev = est;
  }
  lmax = est;
  x = start();
  nx = norm2(x);
  for (double &v : x) v /= nx;
  prev = -1;
  for (int it = 0; it < 2000; ++it) {
    std::vector<double> y = matvec(Den, x);
    lu_solve(LN, y);
    for (double &v : y) v = -v;
    est = norm2(y);
    if (!(est > 0) || !std::isfinite(est)) return false;
    for (int i = 0; i < n; ++i) x[i] = y[i] / est;
    if (it > 30 && std::fabs(est - prev) <= 1e-13 * est) break;
    prev = est;
  }
  lmin = 1.0 / est;
  return lmin > 0 && lmax >= lmin;
}

// ------------------------------------------------------ Zolotarev-type shifts
// Section 3, paragraph below Algorithm 1: with spec(C^-1 A) in [a,b] and the
// vertical spectrum in [c,d], gamma = |c-a||d-b| / (|c-b||d-a|),
// alpha_Z = -1 + 2 gamma + 2 sqrt(gamma^2 - gamma), modulus k = sqrt(1 - 1/alpha_Z^2),
// T the Moebius map {-alpha_Z, -1, 1, alpha_Z} -> {a, b, c, d}, and the shift pair
// of iteration j is T(-+ alpha_Z dn((2j+1) K(k) / (2J), k)).  The point in
// [a,b] goes into the vertical solve and the point in [c,d] into the radial
// solve (the error factor of one sweep is (P - q)(P - p)^-1 on the radial
// side, so p must lie away from spec(P)).  J follows the Zolotarev-number
// bound of the cited theorem, J = ceil(log(16 gamma) log(4/tol) / pi^2).

struct Moebius {
  double z1, z2, z3, w1, w2, w3;
  double operator()(double z) const {
    const double s = (z - z1) * (z2 - z3) / ((z - z3) * (z2 - z1));
    return (w1 * (w2 - w3) - s * w3 * (w2 - w1)) / ((w2 - w3) - s * (w2 - w1));
  }
};

bool zolotarev(double a, double b, double c, double d, double tol, Shifts &S) {
  S.a = a; S.b = b; S.c = c; S.d = d;
  const double gam = std::fabs(c - a) * std::fabs(d - b) / (std::fabs(c - b) * std::fabs(d - a));
  if (!(gam > 1.0) || !std::isfinite(gam)) return false;
  const double al = -1.0 + 2.0 * gam + 2.0 * std::sqrt(gam * gam - gam);
  const double kp = 1.0 / al;
  const double K = ellip_K(kp);
  int J = (int)std::ceil(std::log(16.0 * gam) * std::log(4.0 / tol) / (PI * PI));
  J = std::max(J, 1);
  const Moebius T{-al, -1.0, 1.0, a, b, c};
  const double d4 = T(al);
  if (!(std::fabs(d4 - d) <= 1e-6 * std::fabs(d) + 1e-300)) return false;
  S.J = J;
  S.p.resize(J);
  S.q.resize(J);
  for (int j = 0; j < J; ++j) {
    const double dn = jacobi_dn((2.0 * j + 1.0) * K / (2.0 * J), kp);
    S.q[j] = T(-al * dn);
    S.p[j] = T(al * dn);
  }
  return true;
}

}  // namespace

// ---------------------------------------------------------- elliptic functions
// K(k) = pi / (2 AGM(1, k')) (DLMF 19.8.5).  dn(u | k) by the descending
// arithmetic-geometric mean scheme (DLMF 22.20.1, A&S 16.4): a_0 = 1,
// b_0 = k', c_0 = k; phi_N = 2^N a_N u; phi_{n-1} = (phi_n + asin(c_n sin(phi_n) / a_n)) / 2;
// dn = cos(phi_0) / cos(phi_1 - phi_0).  For u > K/2 the reflection
// dn(u) = k' / dn(K - u) (DLMF 22.4) keeps full relative accuracy when dn is small.

double ellip_K(double kprime) {
  double a = 1.0, b = kprime;
  for (int it = 0; it < 64 && std::fabs(a - b) > 1e-16 * a; ++it) {
    const double an = 0.5 * (a + b);
    b = std::sqrt(a * b);
    a = an;
  }
  return PI / (2.0 * a);
}

static double dn_agm(double u, double kprime) {
  const double k = std::sqrt((1.0 - kprime) * (1.0 + kprime));
  double a[64], c[64];
  a[0] = 1.0;
  double b = kprime;
  c[0] = k;
  int N = 0;
  while (N < 60 && std::fabs(c[N]) > 1e-17 * a[N]) {
    a[N + 1] = 0.5 * (a[N] + b);
    c[N + 1] = 0.5 * (a[N] - b);
    b = std::sqrt(a[N] * b);
    ++N;
  }
  double phi = std::ldexp(a[N] * u, N);
  double phi_prev = phi;
  for (int n = N; n >= 1; --n) {
    phi_prev = phi;
    phi = 0.5 * (phi + std::asin(c[n] * std::sin(phi) / a[n]));
  }
  if (N == 0) return 1.0;
  return std::cos(phi) / std::cos(phi_prev - phi);
}

double jacobi_dn(double u, double kprime) {
  const double K = ellip_K(kprime);
  if (u < 0) u = -u;
  u = std::fmod(u, 2.0 * K);
  if (u > K) u = 2.0 * K - u;          // dn is even and 2K-periodic
  if (u > 0.5 * K) return kprime / dn_agm(K - u, kprime);
  return dn_agm(u, kprime);
}

// ------------------------------------------------------------ block operators
static Band full_R2(int m) { Band R = op_R(m); return mul(mul(R, R), mul(op_C12(m), op_C01(m))); }
static Band full_C02(int m) { return mul(op_C12(m), op_C01(m)); }
static Band full_L(int m, int k) {   // R C12 D1 + R^2 D2 - k^2 C02   (eq. HelmholtzMatEqn)
  Band R = op_R(m);
  Band t1 = mul(R, mul(op_C12(m), op_D1(m)));
  Band t2 = mul(mul(R, R), op_D2(m));
  return axpby(1.0, axpby(1.0, t1, 1.0, t2), -(double)k * k, full_C02(m));
}

Band HostPlan::Cblk(int pr) const { return block(recomb(full_R2(m)), pr); }
Band HostPlan::Lblk(int k, int pr) const { return block(recomb(full_L(m, k)), pr); }
Band HostPlan::Bblk(int pz) const { return block(recomb(full_C02(n)), pz); }
Band HostPlan::D2blk(int pz) const { return block(recomb(op_D2(n)), pz); }

// Pad a block band to fixed offsets [-lo, hi] (so kernels use fixed strides).
static Band widen(const Band &B, int lo, int hi) {
  Band W(B.n, lo, hi);
  for (int i = 0; i < B.n; ++i)
    for (int j = std::max(0, i - B.lo); j <= std::min(B.n - 1, i + B.hi); ++j)
      if (W.in(i, j)) W.at(i, j) = B.get(i, j);
  return W;
}

// b-th order BDF (Section 3: BDF 1, BDF 4 and the kappa^(b), delta^(b)
// definitions), normalised so that y_{n+1} - kappa y'_{n+1} = sum_i beta_i y_{n-i}.
// Orders 2 and 3 are the same backward-difference family as the printed
// BDF 4: sum_{j<=b} (1/j) nabla^j y_{n+1} = h y'_{n+1}.
double bdf_kappa(int b) {
  static const double k[kMaxBdf + 1] = {0.0, 1.0, 2.0 / 3.0, 6.0 / 11.0, 12.0 / 25.0};
  return (b >= 1 && b <= kMaxBdf) ? k[b] : 0.0;
}

void bdf_beta(int b, double beta[kMaxBdf]) {
  static const double t[kMaxBdf + 1][kMaxBdf] = {{0, 0, 0, 0},
                                                 {1.0, 0, 0, 0},
                                                 {4.0 / 3.0, -1.0 / 3.0, 0, 0},
                                                 {18.0 / 11.0, -9.0 / 11.0, 2.0 / 11.0, 0},
                                                 {48.0 / 25.0, -36.0 / 25.0, 16.0 / 25.0, -3.0 / 25.0}};
  for (int i = 0; i < kMaxBdf; ++i) beta[i] = (b >= 1 && b <= kMaxBdf) ? t[b][i] : 0.0;
}

// J T^T J (J the index reversal): the transpose read in reverse order, with the
// band offsets of T itself.
static Band flip_transpose(const Band &T) {
  Band R(T.n, T.lo, T.hi);
  for (int i = 0; i < T.n; ++i)
    for (int j = std::max(0, i - T.lo); j <= std::min(T.n - 1, i + T.hi); ++j) R.at(i, j) = T.get(T.n - 1 - j, T.n - 1 - i);
  return R;
}

// Radial records of Algorithm 1 (layout in plan.hpp) for the radial matrices
// (A, Cm), band offsets -2 .. 3, shifts S, twisted split kr (0: one-sided).
static std::string emit_radial(std::vector<double> &F, const Band &A, const Band &Cm, const Shifts &S, int M,
                               int kr) {
  for (int j = 0; j < S.J; ++j) {
    const double pj = S.p[j], qj = S.q[j], s = qj - pj;
    Band LU = axpby(1.0, A, -pj, Cm);
    if (!lu_inplace(LU)) return "radial LU failed (zero pivot)";
    Band UL;
    if (kr) {
      UL = axpby(1.0, A, -pj, Cm);
      if (!ul_inplace(UL)) return "radial UL failed (zero pivot)";
    }
    for (int i = 0; i < M; ++i) {
      for (int o = -2; o <= 3; ++o)
        F.push_back((i + o >= 0 && i + o < M) ? (A.get(i, i + o) - qj * Cm.get(i, i + o)) / s : 0.0);
      if (kr == 0 || i < kr) {            // LU row (top of a twisted solve)
        F.push_back(i >= 1 ? -LU.get(i, i - 1) : 0.0);
        F.push_back(i >= 2 ? -LU.get(i, i - 2) : 0.0);
        const double dpiv = s / LU.get(i, i);
        for (int o = 1; o <= 3; ++o) F.push_back(i + o < M ? -LU.get(i, i + o) / s * dpiv : 0.0);
        F.push_back(dpiv);
      } else if (i < kr + 3) {            // interface row: apply band only
        for (int o = 0; o < 6; ++o) F.push_back(0.0);
      } else {                            // UL row (bottom of a twisted solve)
        for (int o = 1; o <= 3; ++o) F.push_back(i + o < M ? -UL.get(i, i + o) : 0.0);
        const double dpiv = s / UL.get(i, i);
        F.push_back(-UL.get(i, i - 1) / s * dpiv);
        F.push_back(-UL.get(i, i - 2) / s * dpiv);
        F.push_back(dpiv);
      }
    }
    if (kr) {                             // interface map (3 x 8), scaled by q - p
      Band T = axpby(1.0, A, -pj, Cm);
      std::vector<double> R;
      if (!twist_interface(T, LU, UL, kr, 3, s, R)) return "radial interface solve failed";
      F.insert(F.end(), R.begin(), R.end());
    }
  }
  return std::string();
}

// Vertical records (layout in plan.hpp) for the vertical matrices (D, Bm),
// band offsets -1 .. 2, shifts S, twisted split kz (0: one-sided).
static std::string emit_vertical(std::vector<double> &F, const Band &D, const Band &Bm, const Shifts &S, int Nz,
                                 int kz) {
  for (int j = 0; j < S.J; ++j) {
    Band T = axpby(1.0, D, S.q[j], Bm);
    Band LU = T;
    if (!lu_inplace(LU)) return "vertical LU failed (zero pivot)";
    Band UL;
    if (kz) {
      UL = T;
      if (!ul_inplace(UL)) return "vertical UL failed (zero pivot)";
    }
    const bool last = (j + 1 == S.J);
    const double pn = last ? 0.0 : S.p[j + 1];
    for (int cc = 0; cc < Nz; ++cc) {
      if (kz == 0 || cc < kz) {           // LU column (top of a twisted solve)
        const double dz = 1.0 / LU.get(cc, cc);
        F.push_back(cc >= 1 ? -LU.get(cc, cc - 1) : 0.0);
        F.push_back(cc + 1 < Nz ? -LU.get(cc, cc + 1) * dz : 0.0);
        F.push_back(cc + 2 < Nz ? -LU.get(cc, cc + 2) * dz : 0.0);
        F.push_back(dz);
      } else if (cc < kz + 2) {           // interface column: apply band only
        for (int o = 0; o < 4; ++o) F.push_back(0.0);
      } else {                            // UL column (bottom of a twisted solve)
        const double dz = 1.0 / UL.get(cc, cc);
        F.push_back(cc + 1 < Nz ? -UL.get(cc, cc + 1) : 0.0);
        F.push_back(cc + 2 < Nz ? -UL.get(cc, cc + 2) : 0.0);
        F.push_back(-UL.get(cc, cc - 1) * dz);
        F.push_back(dz);
      }
      for (int o = -1; o <= 2; ++o) {
        const int l = cc + o;
        F.push_back((!last && l >= 0 && l < Nz) ? D.get(cc, l) + pn * Bm.get(cc, l) : 0.0);
      }
    }
    if (kz) {                             // interface map (3 x 5), padded to 16
      std::vector<double> R;
      if (!twist_interface(T, LU, UL, kz, 3, 1.0, R)) return "vertical interface solve failed";
      F.insert(F.end(), R.begin(), R.end());
      F.push_back(0.0);
    }
  }
  return std::string();
}

std::string build_host_plan(HostPlan &hp, int m, int n, int p, double alpha, double dt, double tol,
                            unsigned flags, int bdf_order, int twist) {
  if (bdf_order < 1 || bdf_order > kMaxBdf) return "BDF order out of range";
  hp.m = m; hp.n = n; hp.p = p; hp.alpha = alpha; hp.dt = dt; hp.tol = tol; hp.flags = flags;
  hp.bdf_order = bdf_order;
  for (int c = 0; c < 2; ++c) {
    hp.Mc[c] = std::max(0, (m - 2 - c + 1) / 2);
    hp.Mfull[c] = (m - c + 1) / 2;
    hp.Nc[c] = std::max(0, (n - 2 - c + 1) / 2);
    hp.Nfull[c] = (n - c + 1) / 2;
  }
  const int h = p / 2;
  const bool both = flags & 4u;
  // vertical pencil spectrum per parity: nu = eig(-B^-1 D2) > 0
  for (int pz = 0; pz < 2; ++pz) {
    if (hp.Nc[pz] == 0) continue;
    if (!pencil_extremes(hp.D2blk(pz), hp.Bblk(pz), hp.nu_min[pz], hp.nu_max[pz]))
      return "vertical pencil eigenvalue estimate failed";
  }
  double nu_lo = 1e300, nu_hi = 0;
  for (int pz = 0; pz < 2; ++pz)
    if (hp.Nc[pz] > 0) { nu_lo = std::min(nu_lo, hp.nu_min[pz]); nu_hi = std::max(nu_hi, hp.nu_max[pz]); }
  nu_lo *= 0.95;
  nu_hi *= 1.05;
  // radial pencil spectrum per (k, parity): mu = eig(-C^-1 L_k) > 0
  hp.mu_min.assign((h + 1) * 2, 0.0);
  hp.mu_max.assign((h + 1) * 2, 0.0);
  std::vector<Band> Cb(2), Bb(2), D2b(2);
  for (int c = 0; c < 2; ++c) {
    if (hp.Mc[c] > 0) Cb[c] = widen(hp.Cblk(c), 2, 3);
    if (hp.Nc[c] > 0) { Bb[c] = widen(hp.Bblk(c), 1, 2); D2b[c] = widen(hp.D2blk(c), 1, 2); }
  }
  for (int k = 0; k <= h; ++k)
    for (int pr = 0; pr < 2; ++pr) {
      if (hp.Mc[pr] == 0 || (!both && pr != (k & 1))) continue;
      double lo, hi;
      if (!pencil_extremes(hp.Lblk(k, pr), Cb[pr], lo, hi)) return "radial pencil eigenvalue estimate failed";
      hp.mu_min[k * 2 + pr] = lo * 0.95;
      hp.mu_max[k * 2 + pr] = hi * 1.05;
    }

  hp.factors.clear();
  auto &F = hp.factors;
  // right-hand-side bands, shared by both kinds
  long long r2off[2] = {0, 0}, c02off[2] = {0, 0}, d2off[2] = {0, 0};
  {
    Band R2 = full_R2(m), C02 = full_C02(n);
    for (int pr = 0; pr < 2; ++pr) {
      r2off[pr] = (long long)F.size();
      for (int a = 0; a < hp.Mc[pr]; ++a)
        for (int s = -1; s <= 3; ++s) {
          const int i = pr + 2 * a, j = i + 2 * s;
          F.push_back((j >= 0 && j < m) ? R2.get(i, j) : 0.0);
        }
      if (F.size() & 1) F.push_back(0.0);
    }
    for (int pz = 0; pz < 2; ++pz) {
      c02off[pz] = (long long)F.size();
      for (int b = 0; b < hp.Nc[pz]; ++b)
        for (int t = 0; t <= 2; ++t) {
          const int i = pz + 2 * b, j = i + 2 * t;
          F.push_back(j < n ? C02.get(i, j) : 0.0);
        }
      if (F.size() & 1) F.push_back(0.0);
    }
    Band D2z = op_D2(n);   // D2[j][j+2] (lifting correction)
    for (int pz = 0; pz < 2; ++pz) {
      d2off[pz] = (long long)F.size();
      for (int b = 0; b < hp.Nc[pz]; ++b) {
        const int i = pz + 2 * b;
        F.push_back(i + 2 < n ? D2z.get(i, i + 2) : 0.0);
      }
      if (F.size() & 1) F.push_back(0.0);
    }
  }
  // radial operator L_k = R C12 D1 + R^2 D2 - k^2 C02 per (k, class): L_k[i][i+2t], t = 0..2
  std::vector<long long> lkoff((h + 1) * 2, -1);
  for (int k = 0; k <= h; ++k)
    for (int pr = 0; pr < 2; ++pr) {
      if (hp.Mc[pr] == 0 || (!both && pr != (k & 1))) continue;
      Band Lf = full_L(m, k);
      lkoff[k * 2 + pr] = (long long)F.size();
      for (int a = 0; a < hp.Mc[pr]; ++a)
        for (int t = 0; t <= 2; ++t) {
          const int i = pr + 2 * a, j = i + 2 * t;
          F.push_back(j < m ? Lf.get(i, j) : 0.0);
        }
      if (F.size() & 1) F.push_back(0.0);
    }

  hp.r2off[0] = r2off[0];
  hp.r2off[1] = r2off[1];
  // horizontal (disk) Poisson: LU of -L_k per (k, class) (flag CYL_WITH_DISK)
  hp.disk_off.assign((h + 1) * 2, -1);
  if (flags & 256u) {
    for (int k = 0; k <= h; ++k)
      for (int pr = 0; pr < 2; ++pr) {
        if (hp.Mc[pr] == 0 || (!both && pr != (k & 1))) continue;
        Band A = axpby(-1.0, widen(hp.Lblk(k, pr), 2, 3), 0.0, Cb[pr]);
        if (!lu_inplace(A)) return "disk LU failed (zero pivot)";
        hp.disk_off[k * 2 + pr] = (long long)F.size();
        const int M = hp.Mc[pr];
        for (int i = 0; i < M; ++i) {
          const double d = 1.0 / A.get(i, i);
          F.push_back(i >= 1 ? -A.get(i, i - 1) : 0.0);
          F.push_back(i >= 2 ? -A.get(i, i - 2) : 0.0);
          for (int o = 1; o <= 3; ++o) F.push_back(i + o < M ? -A.get(i, i + o) * d : 0.0);
          F.push_back(d);
        }
      }
  }
  // twisted solves only where both sweeps' chains (two slices x class size) fit kTwistMaxChains:
  // there the second half of the threads doubles the warps per SM sub-partition
  const int maxclass = std::max(std::max(hp.Mc[0], hp.Mc[1]), std::max(hp.Nc[0], hp.Nc[1]));
  // twist == 3 (cluster plans): every item, each CTA of its cluster owning at most kTwistMaxChains chains;
  // twist == 4 (work arrays in global memory): every item, one slice per item
  if (twist == 4 && maxclass > kTwistMaxChainsGlobal) return "twisted single-slice items need class sizes <= 256";
  const bool tw_ok = (twist == 1 && 2 * maxclass <= kTwistMaxChains) || (twist == 2 && maxclass <= kTwistMaxChains) ||
                     twist == 3 || twist == 4;
  for (int kind = 0; kind < kNumKinds; ++kind) {
    KindTables &KT = hp.kind[kind];
    KT = KindTables();
    if (!(flags & (kind == 0 ? 1u : 2u)) || kind > bdf_order) continue;
    const double ka = (kind >= 1) ? alpha * dt * bdf_kappa(kind) : 1.0;   // kappa alpha (heat), 1 (Poisson)
    KT.shifts.assign((h + 1) * 2, Shifts());
    // [c, d]: vertical spectrum of Qhat = -(B^-1 D)^T, union over vertical parities
    const double c = -ka * nu_hi, d = -ka * nu_lo;
    for (int k = 0; k <= h; ++k)
      for (int pr = 0; pr < 2; ++pr) {
        if (hp.Mc[pr] == 0 || (!both && pr != (k & 1))) continue;
        const double mlo = hp.mu_min[k * 2 + pr], mhi = hp.mu_max[k * 2 + pr];
        const double a = (kind >= 1) ? 1.0 + ka * mlo : mlo;
        const double b = (kind >= 1) ? 1.0 + ka * mhi : mhi;
        Shifts &S = KT.shifts[k * 2 + pr];
        if (!zolotarev(a, b, c, d, tol, S)) return "shift computation failed";
        KT.Jmax = std::max(KT.Jmax, S.J);
        const int M = hp.Mc[pr];
        // radial matrices A = -L (Poisson) or C - kappa alpha L (heat)
        Band L = widen(hp.Lblk(k, pr), 2, 3);
        Band A = (kind >= 1) ? axpby(1.0, Cb[pr], -ka, L) : axpby(-1.0, L, 0.0, L);
        const long long roff = (long long)F.size();
        const int kr = (tw_ok && M >= kTwistMinM) ? (M - 3) / 2 : 0;   // twisted split of the radial solve
        std::string e = emit_radial(F, A, Cb[pr], S, M, kr);
        if (!e.empty()) return e;
        // adjoint (heat): the transposed system A^T X B + C^T X D = E is the forward-form system of the
        // flipped transposes J A^T J, J C^T J, J B^T J, J D^T J on index-reversed arrays; its records
        // have the forward layout (one-sided in cluster plans, whose adjoint runs one CTA per item)
        long long roffT = -1;
        const int krT = (twist == 3) ? 0 : kr;
        if (kind >= 1) {
          roffT = (long long)F.size();
          e = emit_radial(F, flip_transpose(A), flip_transpose(Cb[pr]), S, M, krT);
          if (!e.empty()) return "transposed " + e;
        }
        // vertical factors per vertical parity; items
        for (int pz = 0; pz < 2; ++pz) {
          const int Nz = hp.Nc[pz];
          if (Nz == 0) continue;
          Band D = axpby(-ka, D2b[pz], 0.0, D2b[pz]);
          const long long zoff = (long long)F.size();
          const int kz = (tw_ok && Nz >= kTwistMinN) ? (Nz - 2) / 2 : 0;   // twisted split of the vertical solve
          std::string ev = emit_vertical(F, D, Bb[pz], S, Nz, kz);
          if (!ev.empty()) return ev;
          long long zoffT = -1;
          const int kzT = (twist == 3) ? 0 : kz;
          if (kind >= 1) {
            zoffT = (long long)F.size();
            ev = emit_vertical(F, flip_transpose(D), flip_transpose(Bb[pz]), S, Nz, kzT);
            if (!ev.empty()) return "transposed " + ev;
          }
          // one item per slice group
          auto add_item = [&](int s0, int nsl) {
            Item it{};
            it.s0 = s0; it.nsl = nsl; it.k = k; it.pr = pr; it.pz = pz;
            it.M = M; it.Mfull = hp.Mfull[pr]; it.Nz = Nz; it.Nzfull = hp.Nfull[pz];
            it.J = S.J; it.roff = roff; it.zoff = zoff; it.r2off = r2off[pr]; it.c02off = c02off[pz];
            it.roffT = roffT; it.zoffT = zoffT;
            it.m = m; it.n = n; it.xoff = 0;
            it.lkoff = lkoff[k * 2 + pr]; it.d2off = d2off[pz];
            it.twr = kr; it.twz = kz; it.twrT = krT; it.twzT = kzT;
            KT.items.push_back(it);
          };
          if (k == 0) add_item(0, 1);
          else if (k == h) add_item(p - 1, 1);
          else if (twist == 4) { add_item(2 * k - 1, 1); add_item(2 * k, 1); }
          else add_item(2 * k - 1, 2);
        }
      }
    // largest first (J x class block x slices): with more items than resident CTAs the
    // hardware hands out CTAs in launch order, so the longest items start first
    std::stable_sort(KT.items.begin(), KT.items.end(), [](const Item &x, const Item &y) {
      return (double)x.J * x.M * x.Nz * x.nsl > (double)y.J * y.M * y.Nz * y.nsl;
    });
    KT.built = true;
  }
  return std::string();
}

}  // namespace cyl
