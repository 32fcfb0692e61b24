// Launch wrappers of the libcyl device kernels (internal header).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "plan.hpp"

namespace cyl {

// Arguments of one fused ADI launch (one CTA per Item, every step of the run).
struct AdiArgs {
  const Item *items;       // device item table
  int nitems;
  const double *fac;       // device factor / band tables
  const double *Xin;       // T-basis coefficients read by the first step ([p][m][n])
  double *Xout;            // T-basis coefficients written by every step
  const double *G;         // forcing coefficients (heat) or NULL
  double kappa;            // F = R_2 (X + kappa g) C02^T
  long long gstride;       // per-step stride of G (0 = constant)
  int nsteps;
  double *ckpt;            // NULL or checkpoint slots of N doubles
  int ckpt_every;
  int m, n, p;
  int zero_other;          // write zeros into the non-solved radial parity rows
  double *gwork;           // global work arrays when the item does not fit in shared memory
  long long gwork_per_item;
  int use_smem;            // 2: S and Fa in shared memory, 1: S only, 0: neither
  int ld;                  // leading dimension of the work arrays (odd)
  int smem_rows;           // rows of the S array (max Mfull)
  int maxM, maxNz;         // band table sizes in shared memory
  int *err;                // device status word (CYL_ERR_TIMEOUT on a bounded-wait timeout)
  long long group_doubles; // batch kernel: shared-memory slice per thread group (multiple of 32)
  long long wait_limit;    // SM clock cycles a bounded wait may spin (about 1 s normally)
  // BDF history ring (hist_b > 0 replaces Xin / Xout): slot i at hist + i *
  // hist_stride; at the launch's first step the newest state is in slot
  // hist_base and X_{n-i} in slot (hist_base + i) % hist_b; each step writes
  // the new state over the oldest slot.  The right side of every step of the
  // launch is delta^(order) X_n + kappa g_n = sum_{i<order} beta[i] X_{n-i} + kappa g_n.
  double *hist;
  long long hist_stride;
  int hist_b, hist_base, order;
  double beta[4];
  int twist_half;          // > 0: twisted sweeps, threads [0, h) top chains, [h, 2h) bottom chains
  const double *lift;      // coefficients of the lifting W of the boundary data, or NULL
  const double *corr;      // right-side correction of the lifted problem (class positions), or NULL
  int test_no_tma;         // failure-detection test: never start table copies, so waits run out
  int cluster;             // > 1: CTAs of a thread-block cluster per item (work arrays in global memory)
  int all_twisted;         // every item's records (of the system this launch solves) twisted both ways
};

constexpr int CYL_ERR_TIMEOUT = 4;

// Extra arguments of one adjoint launch (steps n_hi-1 down to n_lo).
struct AdjointArgs {
  double *lam;             // adjoint state, in: dL/dX_{n_hi}, out: dL/dX_{n_lo} ([p][m][n])
  const double *G;         // forcing (for the alpha term) or NULL
  long long gstride;
  double *dg;              // dL/dg output or NULL
  long long dg_stride;     // 0: accumulate into one array; else per-step stride
  const double *traj;      // X_{n_lo} .. X_{n_hi} (N each) or NULL (no alpha term)
  double *alpha_part;      // per-item partial sums of <lam, X_{n+1} - X_n - kappa g_n>, or NULL
  double kappa;
  int n_lo, n_hi;
  // multistep (BDF b) mode when lam_ring != NULL (lam unused): lam_j is slot
  // (j + jofs) % R of lam_ring (slots N apart); step s reads lam_{s+1}, adds
  // beta[h] * w into lam_{s-h} (h < order) and clears lam_{s+1}'s slot for
  // reuse.  traj then holds X_j at traj + (traj_K - j) * N (reverse time
  // order) and the alpha term is <w, X_{s+1} - sum_h beta_h X_{s-h} - kappa g_s>.
  double *lam_ring;
  int R, jofs, order;
  double beta[4];
  long long traj_K;
};

cudaError_t launch_adjoint(const AdiArgs &a, const AdjointArgs &g, int threads, size_t smem, cudaStream_t st);
cudaError_t launch_lift_values(const double *bc, double *Wv, int p, int m, int n, cudaStream_t st);
cudaError_t launch_lift_correction(const AdiArgs &a, const double *Wc, double *corr, double c0, double c1, int threads,
                                   cudaStream_t st);
cudaError_t launch_disk_poisson(const Item *items, int nitems, const double *fac, const double *F, double *U,
                                int n, long long slice, int zero_other, int threads, cudaStream_t st);
constexpr int kMaxSlots = 5;
struct SlotMap {
  int src[kMaxSlots];
};
cudaError_t launch_permute_slots(double *dst, const double *src, long long N, int nd, const SlotMap &map,
                                 cudaStream_t st);
cudaError_t launch_sum_partials(const double *part, int n, double scale, double *out, cudaStream_t st);

constexpr int TW_SLOTS = 11;   // exchange doubles per chain of a twisted sweep
size_t adi_smem_bytes(int ld, int smem_rows, int maxM, int maxNz, int level, int twist_half);
size_t batch_group_doubles(int ld, int smem_rows, int maxM, int maxNz, int twist_half);
size_t batch_smem_bytes(int G, int ld, int smem_rows, int maxM, int maxNz, int twist_half);
cudaError_t launch_batch(const AdiArgs &a, int *queue, int G, int threads, int blocks, size_t smem,
                         cudaStream_t st);

cudaError_t launch_adi(const AdiArgs &a, int threads, size_t smem, cudaStream_t st);
// cluster mode (a.cluster CTAs per item, 2 x twist_half threads, twisted tables)
size_t adi_cluster_smem_bytes(int maxM, int maxNz, int twist_half);
cudaError_t launch_adi_cluster(const AdiArgs &a, int threads, size_t smem, cudaStream_t st);

// Chirp-z (Bluestein) line transforms of Section 2 (xform.cu): kind 0 DCT-I
// forward, 1 DCT-I inverse (line length L = the number of Chebyshev
// points), 2 DFT forward to half-complex, 3 DFT inverse from half-complex
// (L = p).  The table block (doubles) holds pre [2A] and post [2B]
// multipliers, the bit-reversed kernel spectrum scaled by 1/P [2P] and the
// FFT twiddles exp(-2 pi i k / P), k < P/2 [P].
struct XformDesc {
  int kind = 0, L = 0, P = 0, logP = 0, A = 0, B = 0, ia0 = 0, jb0 = 0;
  long long pre_off = 0, post_off = 0, H_off = 0, tw_off = 0;
};
constexpr int kMaxXformFfts = 16;     // complex FFTs per CTA
constexpr int kMaxXformP = 8192;      // largest FFT length (shared memory: 16 P bytes per FFT)
std::vector<double> xform_tables(int kind, int L, XformDesc &d);
int xform_ffts_per_cta(int P);
// Lines along one axis: outer x inner lines of L elements, element a of line
// (o, i) at o * L * inner + a * inner + i (in may equal out).
cudaError_t launch_xform(const double *in, double *out, const double *tab, const XformDesc &d, long long outer,
                         long long inner, int sms, cudaStream_t st);

// Navier-Stokes step kernels (ns.cu): d/dtheta on half-complex slices, the
// Chebyshev derivative along lines (o, i) of L elements (element a at
// o * L * inner + a * inner + i; in != out), dst = (init ? 0 : dst) + coef
// r^rpow src on grid values (radius: the m radial grid points), N = V x W.
cudaError_t launch_deriv_theta(const double *in, double *out, int p, long long mn, int sms, cudaStream_t st);
cudaError_t launch_deriv_cheb(const double *in, double *out, long long outer, int L, long long inner, int sms,
                              cudaStream_t st);
cudaError_t launch_accum_r(double *dst, const double *src, const double *radius, int p, int m, int n, double coef,
                           int rpow, bool init, int sms, cudaStream_t st);
cudaError_t launch_cross(const double *const V[3], const double *const W[3], double *const Nout[3], long long total,
                         int sms, cudaStream_t st);

// out[o][j][i] = sum_t W[j][t] in[o][t][i]  (dense transform along one axis)
cudaError_t launch_axis_matvec(const double *in, double *out, const double *W, long long outer, int L,
                               long long inner, cudaStream_t st);

}  // namespace cyl
