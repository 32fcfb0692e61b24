// C ABI of libcyl (see include/cyl.h for the contract of every entry point).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/cyl.h"
#include "kernels.cuh"
#include "plan.hpp"

using cyl::HostPlan;
using cyl::Item;

struct cyl_plan_s {
  HostPlan hp;
  cudaStream_t st = nullptr;
  bool host_only = false;
  int device = 0;
  double *d_fac = nullptr;
  Item *d_items[2] = {nullptr, nullptr};
  int nitems[2] = {0, 0};
  int threads[2] = {0, 0};
  size_t smem[2] = {0, 0};
  int use_smem[2] = {1, 1};
  int ld = 1, smem_rows = 0, maxM = 0, maxNz = 0;
  long long gwork_per_item = 0;
  double *d_gwork = nullptr;
  double *d_W[6] = {};          // Wr_f, Wr_i, Wz_f, Wz_i, Wt_f, Wt_i
  double *d_tmp[3] = {};        // N-element scratch arrays
  int *d_err = nullptr;         // device status word written by bounded waits
  double *d_apart = nullptr;    // per-item partial sums of the alpha gradient
  size_t N = 0;
};

namespace {

constexpr size_t kSmemLimit = 227 * 1024 - 1024;   // opt-in limit minus static shared memory

template <class T>
cudaError_t upload(T **dst, const T *src, size_t count) {
  *dst = nullptr;
  if (count == 0) return cudaSuccess;
  cudaError_t e = cudaMalloc((void **)dst, count * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice);
}

void free_device(cyl_plan_s *P) {
  cudaFree(P->d_fac);
  for (auto &p : P->d_items) cudaFree(p);
  cudaFree(P->d_gwork);
  for (auto &p : P->d_W) cudaFree(p);
  for (auto &p : P->d_tmp) cudaFree(p);
  cudaFree(P->d_err);
  cudaFree(P->d_apart);
}

cyl_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return CYL_OK;
  if (e == cudaErrorMemoryAllocation) return CYL_ENOMEM;
  return CYL_ECUDA;
}

cyl_status vals2coeffs_impl(cyl_plan_s *P, const double *vals, double *coeffs) {
  const HostPlan &h = P->hp;
  const long long m = h.m, n = h.n, p = h.p;
  cudaError_t e;
  if ((e = cyl::launch_axis_matvec(vals, P->d_tmp[0], P->d_W[2], p * m, (int)n, 1, P->st)) != cudaSuccess)
    return from_cuda(e);
  if ((e = cyl::launch_axis_matvec(P->d_tmp[0], P->d_tmp[1], P->d_W[0], p, (int)m, n, P->st)) != cudaSuccess)
    return from_cuda(e);
  return from_cuda(cyl::launch_axis_matvec(P->d_tmp[1], coeffs, P->d_W[4], 1, (int)p, m * n, P->st));
}

cyl_status coeffs2vals_impl(cyl_plan_s *P, const double *coeffs, double *vals) {
  const HostPlan &h = P->hp;
  const long long m = h.m, n = h.n, p = h.p;
  cudaError_t e;
  if ((e = cyl::launch_axis_matvec(coeffs, P->d_tmp[0], P->d_W[5], 1, (int)p, m * n, P->st)) != cudaSuccess)
    return from_cuda(e);
  if ((e = cyl::launch_axis_matvec(P->d_tmp[0], P->d_tmp[1], P->d_W[1], p, (int)m, n, P->st)) != cudaSuccess)
    return from_cuda(e);
  return from_cuda(cyl::launch_axis_matvec(P->d_tmp[1], vals, P->d_W[3], p * m, (int)n, 1, P->st));
}

cyl::AdiArgs adi_args(cyl_plan_s *P, int kind) {
  cyl::AdiArgs a{};
  a.items = P->d_items[kind];
  a.nitems = P->nitems[kind];
  a.fac = P->d_fac;
  a.m = P->hp.m;
  a.n = P->hp.n;
  a.p = P->hp.p;
  a.zero_other = (P->hp.flags & CYL_BOTH_PARITIES) ? 0 : 1;
  a.gwork = P->d_gwork;
  a.gwork_per_item = P->gwork_per_item;
  a.use_smem = P->use_smem[kind];
  a.ld = P->ld;
  a.smem_rows = P->smem_rows;
  a.maxM = P->maxM;
  a.maxNz = P->maxNz;
  a.err = P->d_err;
  a.ckpt_every = 1;
  return a;
}

cyl_status run_adi(cyl_plan_s *P, int kind, const double *Xin, double *Xout, const double *G, double kappa,
                   long long gstride, int nsteps, double *ckpt, int ckpt_every) {
  cyl::AdiArgs a{};
  a.items = P->d_items[kind];
  a.nitems = P->nitems[kind];
  a.fac = P->d_fac;
  a.Xin = Xin;
  a.Xout = Xout;
  a.G = G;
  a.kappa = kappa;
  a.gstride = gstride;
  a.nsteps = nsteps;
  a.ckpt = ckpt;
  a.ckpt_every = ckpt_every > 0 ? ckpt_every : 1;
  a.m = P->hp.m;
  a.n = P->hp.n;
  a.p = P->hp.p;
  a.zero_other = (P->hp.flags & CYL_BOTH_PARITIES) ? 0 : 1;
  a.transpose = 0;
  a.gwork = P->d_gwork;
  a.gwork_per_item = P->gwork_per_item;
  a.use_smem = P->use_smem[kind];
  a.ld = P->ld;
  a.smem_rows = P->smem_rows;
  a.maxM = P->maxM;
  a.maxNz = P->maxNz;
  a.err = P->d_err;
  return from_cuda(cyl::launch_adi(a, P->threads[kind], P->smem[kind], P->st));
}

}  // namespace

extern "C" {

const char *cyl_status_string(cyl_status s) {
  switch (s) {
    case CYL_OK: return "CYL_OK";
    case CYL_EINVAL: return "CYL_EINVAL: invalid argument";
    case CYL_ENOMEM: return "CYL_ENOMEM: allocation failed";
    case CYL_ECUDA: return "CYL_ECUDA: CUDA runtime error";
    case CYL_ETIMEOUT: return "CYL_ETIMEOUT: bounded device wait ran out";
    case CYL_ESTATE: return "CYL_ESTATE: plan not built for this operation";
  }
  return "CYL_UNKNOWN";
}

double cyl_ellip_K(double kprime) { return cyl::ellip_K(kprime); }
double cyl_jacobi_dn(double u, double kprime) { return cyl::jacobi_dn(u, kprime); }

cyl_status cyl_plan(cyl_plan_t *plan, int n_r, int n_z, int n_theta, double alpha, double dt, double adi_tol,
                    unsigned flags, void *stream) {
  if (!plan) return CYL_EINVAL;
  *plan = nullptr;
  if (n_r < 4 || n_z < 4 || n_theta < 2 || (n_theta & 1)) return CYL_EINVAL;
  if (!(adi_tol > 0.0) || adi_tol > 1e-2) return CYL_EINVAL;
  if (!(flags & (CYL_WITH_POISSON | CYL_WITH_HEAT))) return CYL_EINVAL;
  if (flags & ~(unsigned)(CYL_WITH_POISSON | CYL_WITH_HEAT | CYL_BOTH_PARITIES | CYL_HOST_ONLY | CYL_FORCE_GLOBAL))
    return CYL_EINVAL;
  if ((flags & CYL_WITH_HEAT) && !(alpha > 0.0 && dt > 0.0)) return CYL_EINVAL;
  if ((long long)n_r * n_z * n_theta > (1LL << 40)) return CYL_EINVAL;
  cyl_plan_s *P = new (std::nothrow) cyl_plan_s();
  if (!P) return CYL_ENOMEM;
  try {
    std::string err = cyl::build_host_plan(P->hp, n_r, n_z, n_theta, alpha, dt, adi_tol, flags);
    if (!err.empty()) {
      delete P;
      return CYL_EINVAL;
    }
  } catch (const std::bad_alloc &) {
    delete P;
    return CYL_ENOMEM;
  } catch (...) {
    delete P;
    return CYL_EINVAL;
  }
  P->host_only = (flags & CYL_HOST_ONLY) != 0;
  P->st = (cudaStream_t)stream;
  P->N = (size_t)n_r * n_z * n_theta;
  const HostPlan &h = P->hp;
  // launch geometry shared by both kinds
  P->maxM = std::max(h.Mc[0], h.Mc[1]);
  P->maxNz = std::max(h.Nc[0], h.Nc[1]);
  P->smem_rows = std::max(h.Mfull[0], h.Mfull[1]);
  int maxW = 0;
  for (int kind = 0; kind < 2; ++kind)
    for (const Item &it : h.kind[kind].items) maxW = std::max(maxW, it.nsl * it.Nzfull);
  P->ld = std::max(1, maxW) | 1;
  for (int kind = 0; kind < 2; ++kind) {
    int thr = 32;
    for (const Item &it : h.kind[kind].items) thr = std::max(thr, std::max(it.nsl * it.Nz, it.nsl * it.M));
    P->threads[kind] = (thr + 31) / 32 * 32;
    const bool fits = !(flags & CYL_FORCE_GLOBAL) &&
                      cyl::adi_smem_bytes(P->ld, P->smem_rows, P->maxM, P->maxNz, true) <= kSmemLimit;
    P->use_smem[kind] = fits ? 1 : 0;
    P->smem[kind] = cyl::adi_smem_bytes(P->ld, P->smem_rows, P->maxM, P->maxNz, fits);
  }
  if (P->threads[0] > 512 || P->threads[1] > 512) {
    delete P;
    return CYL_EINVAL;
  }
  if (P->host_only) {
    *plan = P;
    return CYL_OK;
  }
  cudaError_t e = cudaGetDevice(&P->device);
  if (e == cudaSuccess) e = upload(&P->d_fac, h.factors.data(), h.factors.size());
  for (int kind = 0; kind < 2 && e == cudaSuccess; ++kind) {
    P->nitems[kind] = (int)h.kind[kind].items.size();
    e = upload(&P->d_items[kind], h.kind[kind].items.data(), h.kind[kind].items.size());
  }
  const std::vector<double> *Ws[6] = {&h.Wr_f, &h.Wr_i, &h.Wz_f, &h.Wz_i, &h.Wt_f, &h.Wt_i};
  for (int i = 0; i < 6 && e == cudaSuccess; ++i) e = upload(&P->d_W[i], Ws[i]->data(), Ws[i]->size());
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaMalloc((void **)&P->d_tmp[i], P->N * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void **)&P->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(P->d_err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void **)&P->d_apart, std::max(1, P->nitems[1]) * sizeof(double));
  if (e == cudaSuccess && !(P->use_smem[0] && P->use_smem[1])) {
    P->gwork_per_item = ((long long)P->smem_rows * P->ld + (long long)P->maxM * P->ld + 31) / 32 * 32;
    const int maxItems = std::max(P->nitems[0], P->nitems[1]);
    e = cudaMalloc((void **)&P->d_gwork, (size_t)P->gwork_per_item * maxItems * sizeof(double));
  }
  if (e != cudaSuccess) {
    free_device(P);
    delete P;
    cudaGetLastError();
    return from_cuda(e);
  }
  *plan = P;
  return CYL_OK;
}

cyl_status cyl_destroy(cyl_plan_t P) {
  if (!P) return CYL_OK;
  if (!P->host_only) free_device(P);
  delete P;
  return CYL_OK;
}

cyl_status cyl_vals2coeffs(cyl_plan_t P, const double *vals, double *coeffs) {
  if (!P || !vals || !coeffs) return CYL_EINVAL;
  if (P->host_only) return CYL_ESTATE;
  return vals2coeffs_impl(P, vals, coeffs);
}

cyl_status cyl_coeffs2vals(cyl_plan_t P, const double *coeffs, double *vals) {
  if (!P || !vals || !coeffs) return CYL_EINVAL;
  if (P->host_only) return CYL_ESTATE;
  return coeffs2vals_impl(P, coeffs, vals);
}

cyl_status cyl_poisson(cyl_plan_t P, const double *f, double *u, int space) {
  if (!P || !f || !u || (space != CYL_VALUES && space != CYL_COEFFS)) return CYL_EINVAL;
  if (P->host_only || !P->hp.kind[0].built) return CYL_ESTATE;
  if (space == CYL_COEFFS) return run_adi(P, 0, f, u, nullptr, 0.0, 0, 1, nullptr, 1);
  cyl_status s = vals2coeffs_impl(P, f, P->d_tmp[2]);
  if (s != CYL_OK) return s;
  s = run_adi(P, 0, P->d_tmp[2], P->d_tmp[2], nullptr, 0.0, 0, 1, nullptr, 1);
  if (s != CYL_OK) return s;
  return coeffs2vals_impl(P, P->d_tmp[2], u);
}

cyl_status cyl_heat_step(cyl_plan_t P, double *T, const double *g, long long g_step_stride, int nsteps,
                         double *ckpt, int ckpt_every) {
  if (!P || !T || nsteps < 0 || g_step_stride < 0) return CYL_EINVAL;
  if (g_step_stride != 0 && (size_t)g_step_stride < P->N) return CYL_EINVAL;
  if (ckpt && ckpt_every < 1) return CYL_EINVAL;
  if (P->host_only || !P->hp.kind[1].built) return CYL_ESTATE;
  if (nsteps == 0) return CYL_OK;
  if (ckpt) {
    cudaError_t e = cudaMemcpyAsync(ckpt, T, P->N * sizeof(double), cudaMemcpyDeviceToDevice, P->st);
    if (e != cudaSuccess) return from_cuda(e);
  }
  return run_adi(P, 1, T, T, g, P->hp.dt, g ? g_step_stride : 0, nsteps, ckpt, ckpt_every);
}

static size_t adjoint_workspace_doubles(const cyl_plan_s *P, int nsteps, int ckpt_every, bool need_alpha) {
  if (!need_alpha || nsteps <= 0) return 0;
  const long long c = std::min(ckpt_every, nsteps);
  const long long nseg = (nsteps + c - 1) / c;
  // checkpoints X_0, X_c, ..., one segment of states X_{s c} .. X_{s c + c}, one work state
  return (size_t)(nseg + (c + 1) + 1) * P->N;
}

cyl_status cyl_heat_adjoint_workspace(cyl_plan_t P, int nsteps, int ckpt_every, int need_alpha, size_t *bytes) {
  if (!P || !bytes || nsteps < 0 || ckpt_every < 1) return CYL_EINVAL;
  *bytes = adjoint_workspace_doubles(P, nsteps, ckpt_every, need_alpha != 0) * sizeof(double);
  return CYL_OK;
}

cyl_status cyl_heat_adjoint(cyl_plan_t P, const double *T0, const double *g, long long g_step_stride, int nsteps,
                            int ckpt_every, const double *dL_dTN, double *dL_dT0, double *dL_dg,
                            double *dL_dalpha, void *workspace, size_t workspace_bytes) {
  if (!P || !dL_dTN || !dL_dT0 || nsteps < 0 || ckpt_every < 1 || g_step_stride < 0) return CYL_EINVAL;
  if (g_step_stride != 0 && (size_t)g_step_stride < P->N) return CYL_EINVAL;
  if (dL_dalpha && !T0) return CYL_EINVAL;
  if (P->host_only || !P->hp.kind[1].built) return CYL_ESTATE;
  const size_t need = adjoint_workspace_doubles(P, nsteps, ckpt_every, dL_dalpha != nullptr);
  if (need && (!workspace || workspace_bytes < need * sizeof(double))) return CYL_EINVAL;
  const size_t N = P->N;
  const double kappa = P->hp.dt;
  cudaError_t e = cudaMemcpyAsync(dL_dT0, dL_dTN, N * sizeof(double), cudaMemcpyDeviceToDevice, P->st);
  if (e == cudaSuccess && dL_dg && g_step_stride == 0) e = cudaMemsetAsync(dL_dg, 0, N * sizeof(double), P->st);
  if (e == cudaSuccess && dL_dalpha)
    e = cudaMemsetAsync(P->d_apart, 0, std::max(1, P->nitems[1]) * sizeof(double), P->st);
  if (e != cudaSuccess) return from_cuda(e);
  if (nsteps == 0) {
    if (dL_dalpha) return from_cuda(cudaMemsetAsync(dL_dalpha, 0, sizeof(double), P->st));
    return CYL_OK;
  }
  cyl::AdiArgs a = adi_args(P, 1);
  cyl::AdjointArgs adj{};
  adj.lam = dL_dT0;
  adj.G = g;
  adj.gstride = g ? g_step_stride : 0;
  adj.dg = dL_dg;
  adj.dg_stride = g_step_stride;
  adj.kappa = kappa;
  if (!dL_dalpha) {
    // the stepping map is linear in (X_0, g): no forward states are needed
    adj.n_lo = 0;
    adj.n_hi = nsteps;
    return from_cuda(cyl::launch_adjoint(a, adj, P->threads[1], P->smem[1], P->st));
  }
  const int c = std::min(ckpt_every, nsteps);
  const int nseg = (nsteps + c - 1) / c;
  double *ck = static_cast<double *>(workspace);       // nseg slots
  double *seg = ck + (size_t)nseg * N;                  // c + 1 slots
  double *work = seg + (size_t)(c + 1) * N;             // 1 slot
  e = cudaMemcpyAsync(ck, T0, N * sizeof(double), cudaMemcpyDeviceToDevice, P->st);
  if (e != cudaSuccess) return from_cuda(e);
  cyl_status s;
  if (nseg > 1) {                                       // checkpoints X_c, X_2c, ... (ck slot s = X_{s c})
    s = run_adi(P, 1, T0, work, g, kappa, g ? g_step_stride : 0, (nseg - 1) * c, ck, c);
    if (s != CYL_OK) return s;
  }
  adj.traj = seg;
  adj.alpha_part = P->d_apart;
  for (int sgi = nseg - 1; sgi >= 0; --sgi) {
    const int n_lo = sgi * c, n_hi = std::min(n_lo + c, nsteps);
    e = cudaMemcpyAsync(seg, ck + (size_t)sgi * N, N * sizeof(double), cudaMemcpyDeviceToDevice, P->st);
    if (e != cudaSuccess) return from_cuda(e);
    const double *gseg = g ? g + (size_t)n_lo * g_step_stride : nullptr;
    s = run_adi(P, 1, seg, work, gseg, kappa, g ? g_step_stride : 0, n_hi - n_lo, seg, 1);
    if (s != CYL_OK) return s;
    adj.n_lo = n_lo;
    adj.n_hi = n_hi;
    e = cyl::launch_adjoint(a, adj, P->threads[1], P->smem[1], P->st);
    if (e != cudaSuccess) return from_cuda(e);
  }
  return from_cuda(cyl::launch_sum_partials(P->d_apart, P->nitems[1], 1.0 / P->hp.alpha, dL_dalpha, P->st));
}

cyl_status cyl_sync(cyl_plan_t P) {
  if (!P) return CYL_EINVAL;
  if (P->host_only) return CYL_OK;
  cudaError_t e = cudaStreamSynchronize(P->st);
  if (e != cudaSuccess) return from_cuda(e);
  int flag = 0;
  e = cudaMemcpy(&flag, P->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return from_cuda(e);
  if (flag != 0) {
    cudaMemset(P->d_err, 0, sizeof(int));
    return (cyl_status)flag;
  }
  return CYL_OK;
}

cyl_status cyl_grid(cyl_plan_t P, double *r, double *z, double *theta) {
  if (!P) return CYL_EINVAL;
  const HostPlan &h = P->hp;
  const double pi = 3.14159265358979323846;
  if (r)
    for (int j = 0; j < h.m; ++j) r[j] = std::cos((h.m - 1 - j) * pi / (h.m - 1));
  if (z)
    for (int k = 0; k < h.n; ++k) z[k] = std::cos((h.n - 1 - k) * pi / (h.n - 1));
  if (theta)
    for (int l = 0; l < h.p; ++l) theta[l] = (2.0 * l - h.p) * pi / h.p;
  return CYL_OK;
}

cyl_status cyl_plan_shifts(cyl_plan_t P, int which, int k, int parity, int *J, double *interval4,
                           double *p_shift, double *q_shift) {
  if (!P || !J || which < 0 || which > 1 || k < 0 || k > P->hp.p / 2 || parity < 0 || parity > 1)
    return CYL_EINVAL;
  const auto &KT = P->hp.kind[which];
  if (!KT.built) return CYL_ESTATE;
  const cyl::Shifts &S = KT.shifts[k * 2 + parity];
  if (S.J == 0) return CYL_ESTATE;
  *J = S.J;
  if (interval4) {
    interval4[0] = S.a; interval4[1] = S.b; interval4[2] = S.c; interval4[3] = S.d;
  }
  if (p_shift) std::memcpy(p_shift, S.p.data(), S.J * sizeof(double));
  if (q_shift) std::memcpy(q_shift, S.q.data(), S.J * sizeof(double));
  return CYL_OK;
}

cyl_status cyl_plan_operator(cyl_plan_t P, int op, int which, int k, int parity, int *dim, double *out) {
  if (!P || !dim || op < 0 || op > 3 || which < 0 || which > 1 || parity < 0 || parity > 1 || k < 0 ||
      k > P->hp.p / 2)
    return CYL_EINVAL;
  const HostPlan &h = P->hp;
  if (which == 1 && !(h.alpha > 0 && h.dt > 0)) return CYL_ESTATE;
  const double ka = which == 1 ? h.alpha * h.dt : 1.0;
  cyl::Band B;
  if (op == 0) {
    cyl::Band L = h.Lblk(k, parity), C = h.Cblk(parity);
    B = cyl::Band(L.n, 2, 3);
    for (int i = 0; i < L.n; ++i)
      for (int j = std::max(0, i - 2); j <= std::min(L.n - 1, i + 3); ++j)
        B.at(i, j) = which == 1 ? C.get(i, j) - ka * L.get(i, j) : -L.get(i, j);
  } else if (op == 1) {
    B = h.Cblk(parity);
  } else if (op == 2) {
    B = h.Bblk(parity);
  } else {
    cyl::Band D2 = h.D2blk(parity);
    B = cyl::Band(D2.n, D2.lo, D2.hi);
    for (size_t i = 0; i < D2.v.size(); ++i) B.v[i] = -ka * D2.v[i];
  }
  *dim = B.n;
  if (out)
    for (int i = 0; i < B.n; ++i)
      for (int j = 0; j < B.n; ++j) out[(size_t)i * B.n + j] = B.get(i, j);
  return CYL_OK;
}

}  // extern "C"
