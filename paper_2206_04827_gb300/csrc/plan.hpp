// Internal plan representation of libcyl (host side).  Not part of the ABI.
//
// Notation (Section 3): per wavenumber k the BDF step / Poisson problem is the
// generalised Sylvester equation  A Y B^T + C Y D^T = E  on the Dirichlet
// recombined coefficients Y (X = S_r Y S_z^T, phi_j = T_{j+2} - T_j).  Every
// operator has even bandwidth offsets, so the equation splits into parity
// blocks ("class" indices a = (i - parity) / 2).  Block bands:
//   radial  A, C : offsets -2 .. +3        vertical  B : -1 .. +2,  D : 0 .. +1
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace cyl {

// Square banded matrix: entry (i, j) stored when j - i lies in [-lo, hi].
struct Band {
  int n = 0, lo = 0, hi = 0;
  std::vector<double> v;
  Band() = default;
  Band(int n_, int lo_, int hi_) : n(n_), lo(lo_), hi(hi_), v((size_t)n_ * (lo_ + hi_ + 1), 0.0) {}
  int w() const { return lo + hi + 1; }
  bool in(int i, int j) const { return i >= 0 && j >= 0 && i < n && j < n && j - i >= -lo && j - i <= hi; }
  double get(int i, int j) const { return in(i, j) ? v[(size_t)i * w() + (j - i + lo)] : 0.0; }
  double &at(int i, int j) { return v[(size_t)i * w() + (j - i + lo)]; }
};

// Factors per row of one shifted radial matrix (A - p C) for iteration j,
// pre-scaled so that one sweep computes Z = (A - pC)^-1 [(q-p) E + (A - qC) U]:
//   [0..5]  (A - qC)[i][i+o] / (q-p),  o = -2 .. 3
//   [6..7]  -L[i][i-1], -L[i][i-2]               (unit lower factor)
//   [8..10] -U[i][i+o] / U[i][i],  o = 1 .. 3     (upper factor, pivot folded in)
//   [11]    (q-p) / U[i][i]
// so that Z_i = [11] * y_i + [10] Z_{i+3} + [9] Z_{i+2} + [8] Z_{i+1}: the loop-carried
// recurrence is a single fused multiply-add per row.
constexpr int RSTRIDE = 12;
// The transposed system of the adjoint, A^T X B + C^T X D = E, equals the
// forward-form system of the flipped transposes J A^T J, J C^T J, J B^T J,
// J D^T J (J the index reversal, which keeps the band offsets) on
// index-reversed arrays; its records have exactly the forward layout below,
// built from those matrices with the same shifts.
// Factors per column of one vertical matrix (D + qB) and the next apply band:
//   [0]     -L[c][c-1]
//   [1..2]  -U[c][c+1] / U[c][c], -U[c][c+2] / U[c][c]   (pivot folded in)
//   [3]     1 / U[c][c]
//   [4..7]  (D + p' B)[c][c+o], o = -1 .. 2      (p' = next radial shift)
constexpr int ZSTRIDE = 8;
// Right-hand-side bands: R_2[i][i+2s] (s = -1..3) per radial class row and
// C02[j][j+2t] (t = 0..2) per vertical class column.
// Twisted solves (forward tables only).  With split row k the radial table
// holds LU records for rows < k, apply-only records for the interface rows
// k .. k+2, and UL records for rows > k+2:
//   [0..5] apply band as above, [6..8] -Ut[i][i+1..i+3] (unit upper of
//   A - pC = Ut Lt), [9..10] -Lt[i][i-1], -Lt[i][i-2] over Lt[i][i], [11] (q-p)/Lt[i][i],
// followed by RTWIST doubles: the 3 x 8 map from (w_{k-2}, w_{k-1}, y_k,
// y_{k+1}, y_{k+2}, v_{k+3}, v_{k+4}, v_{k+5}) to z_k .. z_{k+2}.  The vertical
// table (split column k) holds LU records for columns < k, apply-only for
// k, k+1, and UL records [0..1] -Ut[c][c+1..c+2], [2] -Lt[c][c-1]/Lt[c][c],
// [3] 1/Lt[c][c] beyond, followed by ZTWIST doubles: the 3 x 5 map from
// (w_{k-1}, z_k, z_{k+1}, v_{k+2}, v_{k+3}) to x_k .. x_{k+2} (one pad).
constexpr int RTWIST = 24;
constexpr int ZTWIST = 16;
constexpr int kTwistMinM = 10, kTwistMinN = 8;
constexpr int kTwistMaxChains = 128;
// twisted sweeps with the work arrays in global memory (twist mode 4): one
// CTA of 2 x 256 threads per single-slice item
constexpr int kTwistMaxChainsGlobal = 256;
// Horizontal (disk) Poisson: LU records of -L_k (recombined, tau rows) per
// class row: [0..1] -L[i][i-1], -L[i][i-2]; [2..4] -U[i][i+1..i+3]/U[i][i];
// [5] 1/U[i][i].
constexpr int HSTRIDE = 6;
constexpr int R2STRIDE = 5;
constexpr int C02STRIDE = 3;

// One unit of ADI work: one or two half-complex slices (Re/Im of the same
// wavenumber share every operator) x one radial class x one vertical class.
struct Item {
  int s0, nsl;        // first slice, number of slices (1 or 2; slice s0+1 when 2)
  int k, pr, pz;      // |wavenumber|, radial and vertical parity class
  int M, Mfull;       // unknown rows (class rows < m-2), class rows < m
  int Nz, Nzfull;     // unknown cols (class cols < n-2), class cols < n
  int J;              // ADI iterations
  int m, n;           // grid of the item's problem (n_r, n_z)
  long long xoff;     // offset (doubles) of the problem's arrays in a batch (0 for one problem)
  long long roff;     // offset (doubles) of the radial factors  [J][M][RSTRIDE]
  long long zoff;     // offset (doubles) of the vertical factors [J][Nz][ZSTRIDE]
  long long r2off;    // offset of the R_2 band table   [M][R2STRIDE]
  long long c02off;   // offset of the C02 band table   [Nz][C02STRIDE]
  long long roffT;    // transposed radial factors (adjoint), heat only, else -1
  long long zoffT;    // transposed vertical factors (adjoint), heat only, else -1
  long long lkoff;    // radial operator L_k bands [M][3] (lifting of boundary data)
  long long d2off;    // vertical D2 band [Nz] (lifting of boundary data)
  int twr, twz;       // twisted split rows of the radial / vertical solves (0: plain)
  int twrT, twzT;     // the same for the transposed (adjoint) records
};

struct Shifts {
  int J = 0;
  double a = 0, b = 0, c = 0, d = 0;
  std::vector<double> p, q;   // p in [c,d] (radial solve), q in [a,b] (vertical solve)
};

// Problem kinds: 0 = Poisson, b = 1..4 = one step of the b-th order BDF
// (kappa^(b) = h * bdf_kappa(b)).
constexpr int kNumKinds = 5;
constexpr int kMaxBdf = 4;
double bdf_kappa(int b);                       // kappa^(b) / h
void bdf_beta(int b, double beta[kMaxBdf]);    // delta^(b) coefficients (zero-padded)

struct KindTables {             // one per problem kind
  bool built = false;
  // per (k, pr): shifts; index k * 2 + pr
  std::vector<Shifts> shifts;
  std::vector<Item> items;
  int Jmax = 0;
};

struct HostPlan {
  int m = 0, n = 0, p = 0;
  double alpha = 0, dt = 0, tol = 0;
  unsigned flags = 0;
  // radial class sizes and vertical class sizes
  int Mc[2] = {0, 0}, Mfull[2] = {0, 0}, Nc[2] = {0, 0}, Nfull[2] = {0, 0};
  // spectra of the unscaled pencils: mu (radial, per k, parity) and nu (vertical, per parity)
  std::vector<double> mu_min, mu_max;   // index k * 2 + pr
  double nu_min[2] = {0, 0}, nu_max[2] = {0, 0};
  int bdf_order = 1;                    // highest BDF order built (heat)
  std::vector<long long> disk_off;      // per (k, pr): HSTRIDE records of -L_k, or -1
  long long r2off[2] = {0, 0};          // R_2 band tables per radial class
  KindTables kind[kNumKinds];           // 0 = Poisson, 1..bdf_order = BDF 1..b
  std::vector<double> factors;          // all radial and vertical factor rows + rhs bands

  // radial block operators per k (lazily usable by introspection)
  Band Cblk(int pr) const;
  Band Lblk(int k, int pr) const;
  Band Bblk(int pz) const;
  Band D2blk(int pz) const;
};

// Build everything on the host.  Returns an empty string on success, else a message.
// twist: 0 = one-sided sweeps only; 1 = twisted (two-sided) solves where both
// sweeps of a two-slice item have at most kTwistMaxChains chains; 2 = where
// one slice has (batch plans, which split twisted pairs into single slices);
// 3 = every item (cluster plans: each CTA of an item's cluster owns at most
// kTwistMaxChains chains of every sweep); 4 = every item, with single-slice
// items (grids whose work arrays leave shared memory: one CTA of two threads
// per chain, at most kTwistMaxChainsGlobal chains per sweep).
std::string build_host_plan(HostPlan &hp, int m, int n, int p, double alpha, double dt, double tol,
                            unsigned flags, int bdf_order = 1, int twist = 1);

double ellip_K(double kprime);
double jacobi_dn(double u, double kprime);

}  // namespace cyl
