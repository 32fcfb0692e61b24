// C ABI of libcyl (see include/cyl.h for the contract of every entry point).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <thread>
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
  // per kind: 0 = Poisson, b = 1..4 = BDF b step
  Item *d_items[cyl::kNumKinds] = {};
  int nitems[cyl::kNumKinds] = {};
  int threads[cyl::kNumKinds] = {};
  size_t smem[cyl::kNumKinds] = {};
  int use_smem[cyl::kNumKinds] = {1, 1, 1, 1, 1};
  int twist_half[cyl::kNumKinds] = {};   // > 0: the kind's tables hold twisted solves
  int all_tw[cyl::kNumKinds] = {};       // every item twisted both ways (forward / transposed records)
  int all_twT[cyl::kNumKinds] = {};
  int cluster = 0;                        // > 1: CTAs per item of the cluster-mode ADI launch
  int ld = 1, smem_rows = 0, maxM = 0, maxNz = 0;
  long long gwork_per_item = 0;
  double *d_gwork = nullptr;
  // chirp-z transform tables (csrc/xform.cu): z forward / inverse, r forward / inverse, theta forward / inverse
  cyl::XformDesc xd[6];
  long long xoff[6] = {};
  double *d_xtab = nullptr;
  double *d_radius = nullptr;   // radial grid points r_j (Definition "grid"), Navier-Stokes step
  int sms = 152;
  double *d_tmp[3] = {};        // N-element scratch arrays
  // batch plans (cyl_plan_batch): several problems, two persistent launch classes
  bool is_batch = false;
  int nprob = 0;
  std::vector<long long> offsets;   // prefix offsets (doubles) of each problem's arrays
  std::vector<Item> bitems;         // all items, largest first
  struct BatchClass {
    Item *d_items = nullptr;
    int nitems = 0, G = 1, threads = 128, blocks = 0, ld = 1, smem_rows = 0, maxM = 0, maxNz = 0;
    int twist_half = 0;
    size_t smem = 0;
    long long gwork_per_item = 0;
    double *d_gwork = nullptr;
    int *d_queue = nullptr;
  } bc[2];
  int threshold = 0;                // items with max(M, Nz) > threshold go to class 0
  int chains_per_thread = 1;        // one-sided classes: chains each thread sweeps in turn
  cudaStream_t aux = nullptr;       // second stream for the concurrent class
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int *d_err = nullptr;         // device status word written by bounded waits
  double *d_apart = nullptr;    // per-item partial sums of the alpha gradient
  Item *d_disk_items = nullptr;  // horizontal (disk) Poisson items (k, radial class), CYL_WITH_DISK
  int ndisk = 0, disk_threads = 0;
  double *d_lift = nullptr;     // coefficients of the lifting W of the boundary data
  double *d_corr = nullptr;     // right-side correction of the lifted problem
  size_t N = 0;
};

namespace {

constexpr size_t kSmemLimit = 227 * 1024 - 1024;   // opt-in limit minus static shared memory
constexpr long long kWaitCycles = 2000000000LL;     // bounded device waits: about 1 s at 2 GHz
constexpr long long kTestWaitCycles = 2000000LL;    // about 1 ms under CYL_TEST_NO_TMA

template <class T>
cudaError_t upload(T **dst, const T *src, size_t count) {
  *dst = nullptr;
  if (count == 0) return cudaSuccess;
  cudaError_t e = cudaMalloc((void **)dst, count * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice);
}

void free_batch(cyl_plan_s *P) {
  for (auto &c : P->bc) {
    if (!P->host_only) {
      cudaFree(c.d_items);
      cudaFree(c.d_gwork);
      cudaFree(c.d_queue);
    }
    c = cyl_plan_s::BatchClass();
  }
}

void free_device(cyl_plan_s *P) {
  free_batch(P);
  if (P->aux) cudaStreamDestroy(P->aux);
  if (P->ev_fork) cudaEventDestroy(P->ev_fork);
  if (P->ev_join) cudaEventDestroy(P->ev_join);
  cudaFree(P->d_fac);
  for (auto &p : P->d_items) cudaFree(p);
  cudaFree(P->d_gwork);
  cudaFree(P->d_xtab);
  cudaFree(P->d_radius);
  for (auto &p : P->d_tmp) cudaFree(p);
  cudaFree(P->d_err);
  cudaFree(P->d_apart);
  cudaFree(P->d_lift);
  cudaFree(P->d_corr);
  cudaFree(P->d_disk_items);
}

cyl_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return CYL_OK;
  if (e == cudaErrorMemoryAllocation) return CYL_ENOMEM;
  return CYL_ECUDA;
}

// Section 2: DCT-I along z, then r, then the DFT along theta (chirp-z line transforms).
cyl_status vals2coeffs_impl(cyl_plan_s *P, const double *vals, double *coeffs) {
  const HostPlan &h = P->hp;
  const long long m = h.m, n = h.n, p = h.p;
  const double *T = P->d_xtab;
  cudaError_t e;
  if ((e = cyl::launch_xform(vals, P->d_tmp[0], T + P->xoff[0], P->xd[0], p * m, 1, P->sms, P->st)) != cudaSuccess)
    return from_cuda(e);
  if ((e = cyl::launch_xform(P->d_tmp[0], P->d_tmp[1], T + P->xoff[2], P->xd[2], p, n, P->sms, P->st)) != cudaSuccess)
    return from_cuda(e);
  return from_cuda(cyl::launch_xform(P->d_tmp[1], coeffs, T + P->xoff[4], P->xd[4], 1, m * n, P->sms, P->st));
}

cyl_status coeffs2vals_impl(cyl_plan_s *P, const double *coeffs, double *vals) {
  const HostPlan &h = P->hp;
  const long long m = h.m, n = h.n, p = h.p;
  const double *T = P->d_xtab;
  cudaError_t e;
  if ((e = cyl::launch_xform(coeffs, P->d_tmp[0], T + P->xoff[5], P->xd[5], 1, m * n, P->sms, P->st)) != cudaSuccess)
    return from_cuda(e);
  if ((e = cyl::launch_xform(P->d_tmp[0], P->d_tmp[1], T + P->xoff[3], P->xd[3], p, n, P->sms, P->st)) != cudaSuccess)
    return from_cuda(e);
  return from_cuda(cyl::launch_xform(P->d_tmp[1], vals, T + P->xoff[1], P->xd[1], p * m, 1, P->sms, P->st));
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
  a.twist_half = P->twist_half[kind];
  a.cluster = P->cluster;
  a.all_twisted = P->cluster > 1 ? 0 : P->all_tw[kind];
  a.ckpt_every = 1;
  a.test_no_tma = (P->hp.flags & CYL_TEST_NO_TMA) ? 1 : 0;
  a.wait_limit = a.test_no_tma ? kTestWaitCycles : kWaitCycles;
  return a;
}

// Boundary data by lifting: W = coefficients of the blend of bc's boundary
// nodes (into d_lift) and the right-side correction of the kind's equation
// applied to W (into d_corr).  Uses d_tmp[0], d_tmp[1] as transform scratch.
cyl_status prepare_lift(cyl_plan_s *P, int kind, const double *bc) {
  cudaError_t e = cudaSuccess;
  if (!P->d_lift) e = cudaMalloc((void **)&P->d_lift, P->N * sizeof(double));
  if (e == cudaSuccess && !P->d_corr) e = cudaMalloc((void **)&P->d_corr, P->N * sizeof(double));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return from_cuda(e);
  }
  cyl::AdiArgs a = adi_args(P, kind);
  // step operator of BDF b (kind b >= 1): c0 = 1, c1 = kappa^(b) alpha; Poisson: c0 = 0, c1 = 1
  const double c0 = kind >= 1 ? 1.0 : 0.0;
  const double c1 = kind >= 1 ? P->hp.alpha * P->hp.dt * cyl::bdf_kappa(kind) : 1.0;
  // W's grid values go to d_corr (free until the correction overwrites it), its coefficients to d_lift
  cudaError_t e2 = cyl::launch_lift_values(bc, P->d_corr, P->hp.p, P->hp.m, P->hp.n, P->st);
  if (e2 != cudaSuccess) return from_cuda(e2);
  cyl_status s = vals2coeffs_impl(P, P->d_corr, P->d_lift);
  if (s != CYL_OK) return s;
  return from_cuda(cyl::launch_lift_correction(a, P->d_lift, P->d_corr, c0, c1, std::min(P->threads[kind], 256), P->st));
}

cyl::AdiArgs step_args(cyl_plan_s *P, int kind, const double *Xin, double *Xout, const double *G, double kappa,
                       long long gstride, int nsteps, double *ckpt, int ckpt_every, bool lifted) {
  cyl::AdiArgs a = adi_args(P, kind);
  a.Xin = Xin;
  a.Xout = Xout;
  a.G = G;
  a.kappa = kappa;
  a.gstride = gstride;
  a.nsteps = nsteps;
  a.ckpt = ckpt;
  a.ckpt_every = ckpt_every > 0 ? ckpt_every : 1;
  a.lift = lifted ? P->d_lift : nullptr;
  a.corr = lifted ? P->d_corr : nullptr;
  return a;
}

cyl_status run_adi(cyl_plan_s *P, int kind, const double *Xin, double *Xout, const double *G, double kappa,
                   long long gstride, int nsteps, double *ckpt, int ckpt_every, bool lifted = false) {
  cyl::AdiArgs a = step_args(P, kind, Xin, Xout, G, kappa, gstride, nsteps, ckpt, ckpt_every, lifted);
  return from_cuda(cyl::launch_adi(a, P->threads[kind], P->smem[kind], P->st));
}

constexpr int kBatchThreads = 128;      // smallest CTA of the persistent batch kernel
constexpr int kBatchMaxThreads = 512;
constexpr int kBatchDefaults[][2] = {{63, 4}, {63, 2}, {47, 4}, {31, 4}, {95, 2}, {0, 1}};   // (threshold, groups)

// Split a batch's items into two launch classes (threshold on max(M, Nz)) and
// build their device tables and work areas.  Pairs of Re/Im slices whose
// shared-memory footprint exceeds a group's budget are split into two items.
cyl_status configure_batch(cyl_plan_s *P, int threshold, int G_small, int cpt = 1) {
  free_batch(P);
  P->threshold = threshold;
  P->chains_per_thread = cpt;
  int sms = 152;
  if (!P->host_only) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P->device);
  for (int cls = 0; cls < 2; ++cls) {
    auto &C = P->bc[cls];
    C.G = cls == 0 ? 1 : G_small;
    const size_t budget = kSmemLimit / C.G / sizeof(double) - 32;   // doubles per group
    std::vector<Item> cand;
    int cM = 0, cNz = 0, cRows = 0, cW1 = 0;
    for (const Item &it0 : P->bitems) {
      const bool big = std::max(it0.M, it0.Nz) > threshold;
      if ((cls == 0) != big) continue;
      cand.push_back(it0);
      cM = std::max(cM, it0.M);
      cNz = std::max(cNz, it0.Nz);
      cRows = std::max(cRows, it0.Mfull);
      cW1 = std::max(cW1, it0.Nzfull);
    }
    std::vector<Item> items;
    if (!cand.empty()) {
      // widest row the group's slice can hold next to the double-buffered tables
      bool ctw = false;
      for (const Item &it0 : cand) ctw = ctw || it0.twr || it0.twz;
      const long long bands = 2LL * (cM * cyl::RSTRIDE + cNz * cyl::ZSTRIDE);
      const int tw_cap = std::min(cyl::kTwistMaxChains, kBatchMaxThreads / C.G / 2);
      const long long extra =                    // interface maps and exchange scratch of twisted groups
          ctw ? 2LL * (cyl::RTWIST + cyl::ZTWIST) + (long long)cyl::TW_SLOTS * tw_cap : 0;
      const long long ldmax = ((long long)budget - bands - extra) / cRows;
      if (ldmax < (cW1 | 1)) return CYL_EINVAL;
      const int chains_max = 4 * (kBatchMaxThreads / C.G);   // a twisted item: two threads per chain
      for (const Item &it0 : cand) {
        const bool tw = it0.twr || it0.twz;
        const bool pair_ok = it0.nsl == 2 && ((2 * it0.Nzfull) | 1) <= ldmax &&
                             2 * std::max(it0.M, it0.Nz) <= (tw ? tw_cap : chains_max);
        if (it0.nsl == 2 && !pair_ok) {
          Item a1 = it0, a2 = it0;
          a1.nsl = a2.nsl = 1;
          a2.s0 = it0.s0 + 1;
          items.push_back(a1);
          items.push_back(a2);
        } else {
          items.push_back(it0);
        }
      }
    }
    std::stable_sort(items.begin(), items.end(), [](const Item &x, const Item &y) {
      return (double)x.J * x.M * x.Nz * x.nsl > (double)y.J * y.M * y.Nz * y.nsl;
    });
    C.nitems = (int)items.size();
    if (C.nitems == 0) continue;
    for (const Item &it : items) {
      C.maxM = std::max(C.maxM, it.M);
      C.maxNz = std::max(C.maxNz, it.Nz);
      C.smem_rows = std::max(C.smem_rows, it.Mfull);
      C.ld = std::max(C.ld, it.nsl * it.Nzfull);
    }
    C.ld |= 1;
    // one thread per chain of the widest item (two warps per SM sub-partition for the
    // large items, whose shared memory admits one CTA per SM), at most 512 per CTA
    int chains = 32;
    bool tw = false;
    for (const Item &it : items) {
      chains = std::max(chains, it.nsl * std::max(it.M, it.Nz));
      tw = tw || it.twr || it.twz;
    }
    const int half = (chains + 31) / 32 * 32;
    if (tw && (half > cyl::kTwistMaxChains || 2 * half * C.G > kBatchMaxThreads)) return CYL_EINVAL;
    C.twist_half = tw ? half : 0;            // twisted groups: top chains, then bottom chains
    // one-sided groups: ceil(chains / cpt) threads, each sweeping cpt chains in turn
    const int half_cpt = ((chains + cpt - 1) / cpt + 31) / 32 * 32;
    const int per_group = tw ? 2 * half : std::min(kBatchMaxThreads / C.G, half_cpt);
    C.threads = std::max(kBatchThreads, C.G * per_group);
    C.smem = cyl::batch_smem_bytes(C.G, C.ld, C.smem_rows, C.maxM, C.maxNz, C.twist_half);
    if (C.smem > kSmemLimit) return CYL_EINVAL;
    C.blocks = std::min(C.nitems, sms * std::max(1, (int)(kSmemLimit / std::max<size_t>(C.smem, 1))));
    C.blocks = std::max(1, std::min(C.blocks, 4 * sms));
    C.gwork_per_item = ((long long)C.maxM * C.ld + 31) / 32 * 32;
    if (P->host_only) continue;              // configuration only (host-side checks)
    cudaError_t e = upload(&C.d_items, items.data(), items.size());
    if (e == cudaSuccess)
      e = cudaMalloc((void **)&C.d_gwork, (size_t)C.gwork_per_item * C.blocks * C.G * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void **)&C.d_queue, sizeof(int));
    if (e != cudaSuccess) return from_cuda(e);
  }
  return CYL_OK;
}

cyl_status run_batch(cyl_plan_s *P, double *T, const double *g, int nsteps) {
  bool two = P->bc[0].nitems > 0 && P->bc[1].nitems > 0;
  cudaError_t e = cudaSuccess;
  if (two) {
    e = cudaEventRecord(P->ev_fork, P->st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(P->aux, P->ev_fork, 0);
    if (e != cudaSuccess) return from_cuda(e);
  }
  for (int cls = 0; cls < 2; ++cls) {
    auto &C = P->bc[cls];
    if (C.nitems == 0) continue;
    cyl::AdiArgs a{};
    a.items = C.d_items;
    a.nitems = C.nitems;
    a.fac = P->d_fac;
    a.Xin = T;
    a.Xout = T;
    a.G = g;
    a.kappa = P->hp.dt;
    a.gstride = 0;
    a.nsteps = nsteps;
    a.ckpt_every = 1;
    a.zero_other = (P->hp.flags & CYL_BOTH_PARITIES) ? 0 : 1;
    a.gwork = C.d_gwork;
    a.gwork_per_item = C.gwork_per_item;
    a.use_smem = 1;
    a.ld = C.ld;
    a.smem_rows = C.smem_rows;
    a.maxM = C.maxM;
    a.maxNz = C.maxNz;
    a.err = P->d_err;
    a.wait_limit = kWaitCycles;
    a.group_doubles = (long long)cyl::batch_group_doubles(C.ld, C.smem_rows, C.maxM, C.maxNz, C.twist_half);
    a.twist_half = C.twist_half;
    if (a.group_doubles % 32 != 0 || (size_t)a.group_doubles * C.G * sizeof(double) > C.smem) return CYL_EINVAL;
    cudaStream_t st = (two && cls == 1) ? P->aux : P->st;
    e = cyl::launch_batch(a, C.d_queue, C.G, C.threads, C.blocks, C.smem, st);
    if (e != cudaSuccess) return from_cuda(e);
  }
  if (two) {
    e = cudaEventRecord(P->ev_join, P->aux);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(P->st, P->ev_join, 0);
  }
  return from_cuda(e);
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
  return cyl_plan_bdf(plan, n_r, n_z, n_theta, alpha, dt, adi_tol, 1, flags, stream);
}

cyl_status cyl_plan_bdf(cyl_plan_t *plan, int n_r, int n_z, int n_theta, double alpha, double dt,
                        double adi_tol, int bdf_order, unsigned flags, void *stream) {
  if (!plan) return CYL_EINVAL;
  *plan = nullptr;
  if (n_r < 4 || n_z < 4 || n_theta < 2 || (n_theta & 1)) return CYL_EINVAL;
  if (n_r > 4096 || n_z > 4096 || n_theta > 4096) return CYL_EINVAL;   // transform FFT length <= 8192
  if (!(adi_tol > 0.0) || adi_tol > 1e-2) return CYL_EINVAL;
  if (!(flags & (CYL_WITH_POISSON | CYL_WITH_HEAT | CYL_WITH_DISK))) return CYL_EINVAL;
  if (flags & ~(unsigned)(CYL_WITH_POISSON | CYL_WITH_HEAT | CYL_BOTH_PARITIES | CYL_HOST_ONLY | CYL_FORCE_GLOBAL |
                          CYL_TEST_NO_TMA | CYL_WITH_BC | CYL_PLAIN_SWEEPS | CYL_WITH_DISK | CYL_FORCE_CLUSTER))
    return CYL_EINVAL;
  if ((flags & CYL_WITH_HEAT) && !(alpha > 0.0 && dt > 0.0)) return CYL_EINVAL;
  if (bdf_order < 1 || bdf_order > cyl::kMaxBdf) return CYL_EINVAL;
  if ((long long)n_r * n_z * n_theta > (1LL << 40)) return CYL_EINVAL;
  // Cluster mode (CYL_FORCE_CLUSTER): C CTAs per item, each with at most kTwistMaxChains chains per
  // sweep (two slices per item when n_theta >= 4, class sizes (n_r - 1) / 2 and (n_z - 1) / 2).
  // Measured on GB300 at 512^2 x 256 it reaches 0.44 of the FP64 peak against 0.59 for one CTA per
  // item with the work arrays in global memory (the twisted sweeps' registers allow one 256-thread
  // CTA per SM, too few warps to hide the L2 latency of the shared work arrays), so it is not the
  // default for any grid.
  int cluster = 0;
  if ((flags & CYL_FORCE_CLUSTER) && !(flags & (CYL_FORCE_GLOBAL | CYL_PLAIN_SWEEPS))) {
    const int maxM = std::max(0, (n_r - 1) / 2), maxNz = std::max(0, (n_z - 1) / 2);
    const int nsl = n_theta >= 4 ? 2 : 1;
    const int chains = nsl * std::max(maxM, maxNz);
    const int C = std::max(2, (chains + cyl::kTwistMaxChains - 1) / cyl::kTwistMaxChains);
    if (C <= 8) cluster = C;
  }
  // Sweep layout.  Where the work arrays of two-slice items fit no SM's shared memory (or with
  // CYL_FORCE_GLOBAL), items hold one slice and every solve is twisted (twist mode 4): one CTA of
  // two threads per chain keeps four warps per SM sub-partition on half the live work area per SM
  // (at 512^3: 1 MB per SM, 152 MB in all, against 2.1 MB and 320 MB for two-slice items with
  // one-sided sweeps); measured on GB300 at 512^3: 0.68 of the FP64 peak against 0.60.
  int twist = (flags & CYL_PLAIN_SWEEPS) ? 0 : 1;
  if (cluster) {
    twist = 3;
  } else if (twist) {
    const int maxM = std::max(0, (n_r - 1) / 2), maxNz = std::max(0, (n_z - 1) / 2);
    const int rows = (n_r + 1) / 2, nsl = n_theta >= 4 ? 2 : 1;
    const int ld2 = (nsl * ((n_z + 1) / 2)) | 1;
    const bool fits = cyl::adi_smem_bytes(ld2, rows, maxM, maxNz, 1, 0) <= kSmemLimit;
    if ((!fits || (flags & CYL_FORCE_GLOBAL)) && std::max(maxM, maxNz) <= cyl::kTwistMaxChainsGlobal) twist = 4;
  }
  cyl_plan_s *P = new (std::nothrow) cyl_plan_s();
  if (!P) return CYL_ENOMEM;
  try {
    std::string err = cyl::build_host_plan(P->hp, n_r, n_z, n_theta, alpha, dt, adi_tol, flags, bdf_order, twist);
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
  for (int kind = 0; kind < cyl::kNumKinds; ++kind)
    for (const Item &it : h.kind[kind].items) maxW = std::max(maxW, it.nsl * it.Nzfull);
  P->ld = std::max(1, maxW) | 1;
  for (int kind = 0; kind < cyl::kNumKinds; ++kind) {
    int thr = 32;
    bool tw = false;
    for (const Item &it : h.kind[kind].items) {
      thr = std::max(thr, std::max(it.nsl * it.Nz, it.nsl * it.M));
      tw = tw || it.twr || it.twz;
    }
    // twisted solves: one thread per chain and side (top chains in the first half)
    const int half = (thr + 31) / 32 * 32;
    P->twist_half[kind] = tw ? half : 0;
    bool all = !h.kind[kind].items.empty(), allT = all;
    for (const Item &it : h.kind[kind].items) {
      all = all && it.twr > 0 && it.twz > 0;
      allT = allT && it.twrT > 0 && it.twzT > 0 && it.roffT >= 0 && it.zoffT >= 0;
    }
    P->all_tw[kind] = all ? 1 : 0;
    P->all_twT[kind] = allT ? 1 : 0;
    // one-sided sweeps: one thread per chain up to 512; the threads loop over further chains
    P->threads[kind] = tw ? 2 * half : std::min(half, 512);
    const int th = P->twist_half[kind];
    int level = 0;
    if (!(flags & CYL_FORCE_GLOBAL)) {
      if (cyl::adi_smem_bytes(P->ld, P->smem_rows, P->maxM, P->maxNz, 2, th) <= kSmemLimit) level = 2;
      else if (cyl::adi_smem_bytes(P->ld, P->smem_rows, P->maxM, P->maxNz, 1, th) <= kSmemLimit) level = 1;
      if (level == 2 && P->threads[kind] > 256) level = 1;   // 2 x 256 twisted threads: Fa in global memory
    }
    P->use_smem[kind] = level;
    P->smem[kind] = cyl::adi_smem_bytes(P->ld, P->smem_rows, P->maxM, P->maxNz, level, th);
    if (cluster) {
      // 256 threads (128 chains x 2 sides) per CTA, work arrays in global memory; at least 120 KB of
      // shared memory keeps one CTA per SM, so that only (SMs / cluster) items are live in L2
      P->threads[kind] = 2 * cyl::kTwistMaxChains;
      P->twist_half[kind] = cyl::kTwistMaxChains;
      P->use_smem[kind] = 0;
      P->smem[kind] = std::max<size_t>(cyl::adi_cluster_smem_bytes(P->maxM, P->maxNz, cyl::kTwistMaxChains),
                                       120 * 1024);
    }
  }
  P->cluster = cluster;
  for (int kind = 0; kind < cyl::kNumKinds; ++kind)
    if (P->threads[kind] > 512) {
      delete P;
      return CYL_EINVAL;
    }
  if (P->host_only) {
    *plan = P;
    return CYL_OK;
  }
  cudaError_t e = cudaGetDevice(&P->device);
  if (e == cudaSuccess) e = upload(&P->d_fac, h.factors.data(), h.factors.size());
  for (int kind = 0; kind < cyl::kNumKinds && e == cudaSuccess; ++kind) {
    P->nitems[kind] = (int)h.kind[kind].items.size();
    e = upload(&P->d_items[kind], h.kind[kind].items.data(), h.kind[kind].items.size());
  }
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&P->sms, cudaDevAttrMultiProcessorCount, P->device);
  if (e == cudaSuccess) {
    // transform tables: z forward / inverse (DCT-I, n points), r (m points), theta (DFT, p points)
    std::vector<double> xt;
    const int kinds[6] = {0, 1, 0, 1, 2, 3}, lens[6] = {n_z, n_z, n_r, n_r, n_theta, n_theta};
    for (int i = 0; i < 6; ++i) {
      std::vector<double> t = cyl::xform_tables(kinds[i], lens[i], P->xd[i]);
      P->xoff[i] = (long long)xt.size();
      xt.insert(xt.end(), t.begin(), t.end());
      if (xt.size() & 1) xt.push_back(0.0);          // keep every block 16-byte aligned
    }
    e = upload(&P->d_xtab, xt.data(), xt.size());
  }
  if (e == cudaSuccess) {
    std::vector<double> rad(n_r);
    for (int j = 0; j < n_r; ++j) rad[j] = std::cos((n_r - 1 - j) * 3.14159265358979323846 / (n_r - 1));
    e = upload(&P->d_radius, rad.data(), rad.size());
  }
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaMalloc((void **)&P->d_tmp[i], P->N * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void **)&P->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(P->d_err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void **)&P->d_apart, std::max(1, P->nitems[1]) * sizeof(double));
  if (e == cudaSuccess && (flags & CYL_WITH_DISK)) {
    std::vector<Item> di;
    const int hh = n_theta / 2;
    for (int k = 0; k <= hh; ++k)
      for (int pr = 0; pr < 2; ++pr) {
        const long long off = h.disk_off[k * 2 + pr];
        if (off < 0) continue;
        Item it{};
        it.k = k; it.pr = pr; it.M = h.Mc[pr]; it.Mfull = h.Mfull[pr];
        it.m = n_r; it.n = n_z; it.roff = off; it.r2off = h.r2off[pr];
        it.s0 = k == 0 ? 0 : (k == hh ? n_theta - 1 : 2 * k - 1);
        it.nsl = (k == 0 || k == hh) ? 1 : 2;
        di.push_back(it);
      }
    P->ndisk = (int)di.size();
    P->disk_threads = std::min(256, std::max(32, (2 * n_z + 31) / 32 * 32));
    e = upload(&P->d_disk_items, di.data(), di.size());
  }
  if (e == cudaSuccess && (flags & CYL_WITH_BC)) e = cudaMalloc((void **)&P->d_lift, P->N * sizeof(double));
  if (e == cudaSuccess && (flags & CYL_WITH_BC)) e = cudaMalloc((void **)&P->d_corr, P->N * sizeof(double));
  bool all_smem = true;
  for (int kind = 0; kind < cyl::kNumKinds; ++kind) all_smem = all_smem && P->use_smem[kind] == 2;
  if (e == cudaSuccess && !all_smem) {
    P->gwork_per_item = ((long long)P->smem_rows * P->ld + (long long)P->maxM * P->ld + 31) / 32 * 32;
    const int maxItems = *std::max_element(P->nitems, P->nitems + cyl::kNumKinds);
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
  if (P->host_only || P->is_batch) return CYL_ESTATE;
  return vals2coeffs_impl(P, vals, coeffs);
}

cyl_status cyl_coeffs2vals(cyl_plan_t P, const double *coeffs, double *vals) {
  if (!P || !vals || !coeffs) return CYL_EINVAL;
  if (P->host_only || P->is_batch) return CYL_ESTATE;
  return coeffs2vals_impl(P, coeffs, vals);
}

cyl_status cyl_poisson(cyl_plan_t P, const double *f, const double *bc, double *u, int space) {
  if (!P || !f || !u || (space != CYL_VALUES && space != CYL_COEFFS)) return CYL_EINVAL;
  if (P->host_only || P->is_batch || !P->hp.kind[0].built) return CYL_ESTATE;
  const double *F = f;
  cyl_status s;
  if (space == CYL_VALUES) {
    if ((s = vals2coeffs_impl(P, f, P->d_tmp[2])) != CYL_OK) return s;
    F = P->d_tmp[2];
  }
  if (bc && (s = prepare_lift(P, 0, bc)) != CYL_OK) return s;
  double *U = space == CYL_VALUES ? P->d_tmp[2] : u;
  if ((s = run_adi(P, 0, F, U, nullptr, 0.0, 0, 1, nullptr, 1, bc != nullptr)) != CYL_OK) return s;
  return space == CYL_VALUES ? coeffs2vals_impl(P, P->d_tmp[2], u) : CYL_OK;
}

cyl_status cyl_disk_poisson(cyl_plan_t P, const double *f, double *u, int space) {
  if (!P || !f || !u || (space != CYL_VALUES && space != CYL_COEFFS)) return CYL_EINVAL;
  if (P->host_only || P->is_batch || !P->d_disk_items) return CYL_ESTATE;
  const int zero_other = (P->hp.flags & CYL_BOTH_PARITIES) ? 0 : 1;
  const long long slice = (long long)P->hp.m * P->hp.n;
  if (space == CYL_COEFFS)
    return from_cuda(cyl::launch_disk_poisson(P->d_disk_items, P->ndisk, P->d_fac, f, u, P->hp.n, slice, zero_other,
                                              P->disk_threads, P->st));
  cyl_status s = vals2coeffs_impl(P, f, P->d_tmp[2]);
  if (s != CYL_OK) return s;
  cudaError_t e = cyl::launch_disk_poisson(P->d_disk_items, P->ndisk, P->d_fac, P->d_tmp[2], P->d_tmp[2], P->hp.n,
                                           slice, zero_other, P->disk_threads, P->st);
  if (e != cudaSuccess) return from_cuda(e);
  return coeffs2vals_impl(P, P->d_tmp[2], u);
}

cyl_status cyl_heat_step(cyl_plan_t P, double *T, const double *g, long long g_step_stride, int nsteps,
                         double *ckpt, int ckpt_every) {
  return cyl_heat_step_bc(P, T, g, g_step_stride, nsteps, nullptr, ckpt, ckpt_every);
}

cyl_status cyl_heat_step_bc(cyl_plan_t P, double *T, const double *g, long long g_step_stride, int nsteps,
                            const double *bc, double *ckpt, int ckpt_every) {
  if (!P || !T || nsteps < 0 || g_step_stride < 0) return CYL_EINVAL;
  if (P->is_batch) return CYL_ESTATE;
  if (g_step_stride != 0 && (size_t)g_step_stride < P->N) return CYL_EINVAL;
  if (ckpt && ckpt_every < 1) return CYL_EINVAL;
  if (P->host_only || !P->hp.kind[1].built) return CYL_ESTATE;
  if (nsteps == 0) return CYL_OK;
  if (ckpt) {
    cudaError_t e = cudaMemcpyAsync(ckpt, T, P->N * sizeof(double), cudaMemcpyDeviceToDevice, P->st);
    if (e != cudaSuccess) return from_cuda(e);
  }
  if (bc) {
    cyl_status s = prepare_lift(P, 1, bc);
    if (s != CYL_OK) return s;
  }
  return run_adi(P, 1, T, T, g, P->hp.dt, g ? g_step_stride : 0, nsteps, ckpt, ckpt_every, bc != nullptr);
}

// nsteps BDF steps on a history ring of ring_len slots (slot (base + i) % ring_len
// holds X_{n-i}; v states known).  Start-up steps (v < order) run one launch
// each at order v; the rest run in one launch.  g + (s0 + s) * gstride drives
// step s.  Updates base and v; lifted_kind tracks which order's lifting
// correction the plan's lifting arrays hold.
cyl_status bdf_forward(cyl_plan_s *P, double *ring, int ring_len, int &base, int &v, int s0, int nsteps,
                       const double *g, long long gstride, const double *bc, int &lifted_kind) {
  const int order = P->hp.bdf_order;
  for (int s = 0; s < nsteps;) {
    const int b = std::min(order, v);                  // start-up through lower orders
    const int cnt = b < order ? 1 : nsteps - s;
    if (bc && lifted_kind != b) {
      cyl_status st = prepare_lift(P, b, bc);
      if (st != CYL_OK) return st;
      lifted_kind = b;
    }
    const double *Gs = g ? g + (size_t)(s0 + s) * (size_t)gstride : nullptr;
    cyl::AdiArgs a = step_args(P, b, nullptr, nullptr, Gs, P->hp.dt * cyl::bdf_kappa(b), g ? gstride : 0, cnt,
                               nullptr, 1, bc != nullptr);
    a.hist = ring;
    a.hist_stride = (long long)P->N;
    a.hist_b = ring_len;
    a.hist_base = base;
    a.order = b;
    cyl::bdf_beta(b, a.beta);
    cudaError_t e = cyl::launch_adi(a, P->threads[b], P->smem[b], P->st);
    if (e != cudaSuccess) return from_cuda(e);
    base = ((base - cnt) % ring_len + ring_len) % ring_len;
    v = std::min(order, v + cnt);
    s += cnt;
  }
  return CYL_OK;
}

// dst slot i = src slot (base + i) % b, i < b (canonical order of a ring).
cudaError_t copy_canonical(double *dst, const double *src, size_t N, int b, int base, cudaStream_t st) {
  cyl::SlotMap map{};
  for (int i = 0; i < b; ++i) map.src[i] = (base + i) % b;
  return cyl::launch_permute_slots(dst, src, (long long)N, b, map, st);
}

cyl_status cyl_heat_step_bdf(cyl_plan_t P, double *hist, int nvalid, const double *g, long long g_step_stride,
                             int nsteps, const double *bc) {
  if (!P || !hist || nsteps < 0 || g_step_stride < 0) return CYL_EINVAL;
  if (P->is_batch || P->host_only) return CYL_ESTATE;
  const int order = P->hp.bdf_order;
  if (nvalid < 1 || nvalid > order) return CYL_EINVAL;
  if (g_step_stride != 0 && (size_t)g_step_stride < P->N) return CYL_EINVAL;
  for (int b = 1; b <= order; ++b)
    if (!P->hp.kind[b].built) return CYL_ESTATE;
  int base = 0, v = nvalid, lifted_kind = -1;
  cyl_status s = bdf_forward(P, hist, order, base, v, 0, nsteps, g, g_step_stride, bc, lifted_kind);
  if (s != CYL_OK) return s;
  if (base != 0) return from_cuda(copy_canonical(hist, hist, P->N, order, base, P->st));
  return CYL_OK;
}

static size_t bdf_adjoint_workspace_doubles(const cyl_plan_s *P, int nsteps, int ckpt_every, bool need_alpha) {
  const size_t order = P->hp.bdf_order;
  size_t d = (order + 1) * P->N;                        // adjoint ring lam_j
  if (need_alpha && nsteps > 0) {
    const long long c = std::min(ckpt_every, nsteps);
    const long long nseg = (nsteps + c - 1) / c;
    d += (size_t)nseg * order * P->N;                   // history checkpoints
    d += (size_t)(c + order) * P->N;                    // one recomputed segment (reverse time order)
  }
  return d;
}

cyl_status cyl_heat_adjoint_bdf_workspace(cyl_plan_t P, int nsteps, int ckpt_every, int need_alpha,
                                          size_t *bytes) {
  if (!P || !bytes || nsteps < 0 || ckpt_every < 1) return CYL_EINVAL;
  *bytes = bdf_adjoint_workspace_doubles(P, nsteps, ckpt_every, need_alpha != 0) * sizeof(double);
  return CYL_OK;
}

cyl_status cyl_heat_adjoint_bdf(cyl_plan_t P, const double *hist0, int nvalid, const double *g,
                                long long g_step_stride, int nsteps, const double *bc, int ckpt_every,
                                const double *dL_dhistN, double *dL_dhist0, double *dL_dg, double *dL_dalpha,
                                void *workspace, size_t workspace_bytes) {
  if (!P || !dL_dhistN || !dL_dhist0 || nsteps < 0 || ckpt_every < 1 || g_step_stride < 0) return CYL_EINVAL;
  if (P->is_batch || P->host_only) return CYL_ESTATE;
  const int order = P->hp.bdf_order, R = order + 1, jofs = order;
  if (nvalid < 1 || nvalid > order) return CYL_EINVAL;
  if (g_step_stride != 0 && (size_t)g_step_stride < P->N) return CYL_EINVAL;
  if (dL_dalpha && !hist0) return CYL_EINVAL;
  for (int b = 1; b <= order; ++b)
    if (!P->hp.kind[b].built) return CYL_ESTATE;
  const size_t need = bdf_adjoint_workspace_doubles(P, nsteps, ckpt_every, dL_dalpha != nullptr);
  if (!workspace || workspace_bytes < need * sizeof(double)) return CYL_EINVAL;
  const size_t N = P->N;
  double *ring = static_cast<double *>(workspace);
  cudaError_t e = cudaSuccess;
  // lam_{nsteps - i} = dL/dhist_N slot i for the known final slots; every other ring slot zero
  {
    cyl::SlotMap map{};
    for (int k = 0; k < R; ++k) map.src[k] = -1;
    const int keep = std::min(order, nvalid + nsteps);
    for (int i = 0; i < keep; ++i) map.src[(nsteps - i + jofs) % R] = i;
    e = cyl::launch_permute_slots(ring, dL_dhistN, (long long)N, R, map, P->st);
  }
  if (e == cudaSuccess && dL_dg && g_step_stride == 0) e = cudaMemsetAsync(dL_dg, 0, N * sizeof(double), P->st);
  if (e == cudaSuccess && dL_dalpha)
    e = cudaMemsetAsync(P->d_apart, 0, std::max(1, P->nitems[1]) * sizeof(double), P->st);
  if (e != cudaSuccess) return from_cuda(e);
  // reverse steps [lo, hi): launches of one order each (start-up steps alone)
  auto reverse = [&](int lo, int hi, const double *traj, long long trajK) -> cyl_status {
    for (int s_hi = hi; s_hi > lo;) {
      const int s_top = s_hi - 1;
      const int b = std::min(order, nvalid + s_top);
      const int s_lo = b < order ? s_top : std::max(lo, order - nvalid);
      cyl::AdjointArgs adj{};
      adj.lam_ring = ring;
      adj.R = R;
      adj.jofs = jofs;
      adj.order = b;
      cyl::bdf_beta(b, adj.beta);
      adj.G = g;
      adj.gstride = g ? g_step_stride : 0;
      adj.dg = dL_dg;
      adj.dg_stride = g_step_stride;
      adj.kappa = P->hp.dt * cyl::bdf_kappa(b);
      adj.traj = traj;
      adj.traj_K = trajK;
      adj.alpha_part = traj ? P->d_apart : nullptr;
      adj.n_lo = s_lo;
      adj.n_hi = s_hi;
      cyl::AdiArgs a = adi_args(P, b);
      a.all_twisted = P->cluster > 1 ? 0 : P->all_twT[b];
      cudaError_t err = cyl::launch_adjoint(a, adj, P->threads[b], P->smem[b], P->st);
      if (err != cudaSuccess) return from_cuda(err);
      s_hi = s_lo;
    }
    return CYL_OK;
  };
  cyl_status s = CYL_OK;
  if (!dL_dalpha) {
    s = reverse(0, nsteps, nullptr, 0);
  } else if (nsteps > 0) {
    const int c = std::min(ckpt_every, nsteps);
    const int nseg = (nsteps + c - 1) / c;
    double *ck = ring + (size_t)R * N;                  // nseg histories, canonical order
    double *traj = ck + (size_t)nseg * order * N;       // c + order states
    int lifted_kind = -1;
    e = cudaMemcpyAsync(ck, hist0, (size_t)order * N * sizeof(double), cudaMemcpyDeviceToDevice, P->st);
    if (e != cudaSuccess) return from_cuda(e);
    if (nseg > 1) {                                     // histories at c, 2c, ... (traj's first slots as the ring)
      e = cudaMemcpyAsync(traj, hist0, (size_t)order * N * sizeof(double), cudaMemcpyDeviceToDevice, P->st);
      if (e != cudaSuccess) return from_cuda(e);
      int base = 0, v = nvalid;
      for (int k = 1; k < nseg; ++k) {
        s = bdf_forward(P, traj, order, base, v, (k - 1) * c, c, g, g_step_stride, bc, lifted_kind);
        if (s != CYL_OK) return s;
        e = copy_canonical(ck + (size_t)k * order * N, traj, N, order, base, P->st);
        if (e != cudaSuccess) return from_cuda(e);
      }
    }
    for (int k = nseg - 1; k >= 0; --k) {
      const int n_lo = k * c, n_hi = std::min(n_lo + c, nsteps), len = n_hi - n_lo;
      // X_j at traj + (n_hi - j) N: the checkpoint history fills slots len .. len + order - 1
      e = cudaMemcpyAsync(traj + (size_t)len * N, ck + (size_t)k * order * N, (size_t)order * N * sizeof(double),
                          cudaMemcpyDeviceToDevice, P->st);
      if (e != cudaSuccess) return from_cuda(e);
      int base = len, v = std::min(order, nvalid + n_lo);
      s = bdf_forward(P, traj, len + order, base, v, n_lo, len, g, g_step_stride, bc, lifted_kind);
      if (s != CYL_OK) return s;
      s = reverse(n_lo, n_hi, traj, n_hi);
      if (s != CYL_OK) return s;
    }
  }
  if (s != CYL_OK) return s;
  // dL/dhist_0 slot i = lam_{-i} for the known initial states, zero beyond
  {
    cyl::SlotMap map{};
    for (int i = 0; i < cyl::kMaxSlots; ++i) map.src[i] = -1;
    for (int i = 0; i < nvalid; ++i) map.src[i] = (-i + jofs) % R;
    e = cyl::launch_permute_slots(dL_dhist0, ring, (long long)N, order, map, P->st);
    if (e != cudaSuccess) return from_cuda(e);
  }
  if (dL_dalpha)
    return from_cuda(cyl::launch_sum_partials(P->d_apart, P->nitems[1], 1.0 / P->hp.alpha, dL_dalpha, P->st));
  return CYL_OK;
}

// need_alpha: 0 none, 1 with the library's own checkpoints, 2 with the caller's (cyl_heat_step's ckpt)
static size_t adjoint_workspace_doubles(const cyl_plan_s *P, int nsteps, int ckpt_every, int need_alpha) {
  if (!need_alpha || nsteps <= 0) return 0;
  const long long c = std::min(ckpt_every, nsteps);
  const long long nseg = (nsteps + c - 1) / c;
  // checkpoints X_0, X_c, ... (unless the caller's), one segment of states X_{s c} .. X_{s c + c}, one work state
  return (size_t)((need_alpha == 2 ? 0 : nseg) + (c + 1) + 1) * P->N;
}

cyl_status cyl_heat_adjoint_workspace(cyl_plan_t P, int nsteps, int ckpt_every, int need_alpha, size_t *bytes) {
  if (!P || !bytes || nsteps < 0 || ckpt_every < 1) return CYL_EINVAL;
  if (need_alpha < 0 || need_alpha > 2) return CYL_EINVAL;
  *bytes = adjoint_workspace_doubles(P, nsteps, ckpt_every, need_alpha) * sizeof(double);
  return CYL_OK;
}

cyl_status cyl_heat_adjoint(cyl_plan_t P, const double *T0, const double *g, long long g_step_stride, int nsteps,
                            int ckpt_every, const double *dL_dTN, double *dL_dT0, double *dL_dg,
                            double *dL_dalpha, void *workspace, size_t workspace_bytes) {
  return cyl_heat_adjoint_bc(P, T0, g, g_step_stride, nsteps, nullptr, ckpt_every, nullptr, dL_dTN, dL_dT0,
                             dL_dg, dL_dalpha, workspace, workspace_bytes);
}

cyl_status cyl_heat_adjoint_bc(cyl_plan_t P, const double *T0, const double *g, long long g_step_stride,
                               int nsteps, const double *bc, int ckpt_every, const double *ckpt, const double *dL_dTN,
                               double *dL_dT0, double *dL_dg, double *dL_dalpha, void *workspace,
                               size_t workspace_bytes) {
  if (!P || !dL_dTN || !dL_dT0 || nsteps < 0 || ckpt_every < 1 || g_step_stride < 0) return CYL_EINVAL;
  if (g_step_stride != 0 && (size_t)g_step_stride < P->N) return CYL_EINVAL;
  if (dL_dalpha && !T0) return CYL_EINVAL;
  if (P->host_only || P->is_batch || !P->hp.kind[1].built) return CYL_ESTATE;
  const size_t need = adjoint_workspace_doubles(P, nsteps, ckpt_every, !dL_dalpha ? 0 : (ckpt ? 2 : 1));
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
  a.all_twisted = P->cluster > 1 ? 0 : P->all_twT[1];
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
  // checkpoints (slot s = X_{s c}): the caller's, written by cyl_heat_step with the same ckpt_every,
  // or computed here by a forward pass
  double *own_ck = ckpt ? nullptr : static_cast<double *>(workspace);          // nseg slots
  const double *ck = ckpt ? ckpt : own_ck;
  double *seg = ckpt ? static_cast<double *>(workspace) : own_ck + (size_t)nseg * N;   // c + 1 slots
  double *work = seg + (size_t)(c + 1) * N;             // 1 slot
  cyl_status s;
  // the data enter the run affinely: only the recomputed states see them
  if (bc && (s = prepare_lift(P, 1, bc)) != CYL_OK) return s;
  const bool lifted = bc != nullptr;
  if (!ckpt) {
    e = cudaMemcpyAsync(own_ck, T0, N * sizeof(double), cudaMemcpyDeviceToDevice, P->st);
    if (e != cudaSuccess) return from_cuda(e);
    if (nseg > 1) {                                     // checkpoints X_c, X_2c, ...
      s = run_adi(P, 1, T0, work, g, kappa, g ? g_step_stride : 0, (nseg - 1) * c, own_ck, c, lifted);
      if (s != CYL_OK) return s;
    }
  }
  adj.traj = seg;
  adj.alpha_part = P->d_apart;
  for (int sgi = nseg - 1; sgi >= 0; --sgi) {
    const int n_lo = sgi * c, n_hi = std::min(n_lo + c, nsteps);
    e = cudaMemcpyAsync(seg, ck + (size_t)sgi * N, N * sizeof(double), cudaMemcpyDeviceToDevice, P->st);
    if (e != cudaSuccess) return from_cuda(e);
    const double *gseg = g ? g + (size_t)n_lo * g_step_stride : nullptr;
    s = run_adi(P, 1, seg, work, gseg, kappa, g ? g_step_stride : 0, n_hi - n_lo, seg, 1, lifted);
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

cyl_status cyl_plan_flops(cyl_plan_t P, int which, int nsteps, int transposed, double *flops) {
  if (!P || !flops || which < 0 || which >= cyl::kNumKinds || nsteps < 0) return CYL_EINVAL;
  const std::vector<Item> &items = P->is_batch ? P->bitems : P->hp.kind[which].items;
  if (P->is_batch && which != 1) return CYL_ESTATE;
  double f = 0.0;
  for (const Item &it : items) {
    const double W = (double)it.nsl * it.Nz, M = it.M;
    double per_step;
    if (!transposed) {
      per_step = 3.0 * it.Mfull * W + 5.0 * M * W + (12.0 * it.J - 6.0 + 8.0 * it.J - 4.0) * M * W +
                 1.5 * it.Mfull * it.nsl * it.Nzfull;
    } else {
      const double Wf = (double)it.nsl * it.Nzfull;
      per_step = 1.5 * M * W + (12.0 * it.J - 6.0 + 8.0 * it.J - 4.0) * M * W + 3.0 * M * Wf +
                 5.0 * it.Mfull * Wf;
    }
    // BDF b > 1: delta^(b) X_n, b - 1 further fused multiply-adds per class element
    if (!transposed && which >= 2) per_step += (which - 1.0) * it.Mfull * it.nsl * it.Nzfull;
    f += 2.0 * per_step * nsteps;   // 2 flops per fused multiply-add
  }
  *flops = f;
  return CYL_OK;
}

cyl_status cyl_grid(cyl_plan_t P, double *r, double *z, double *theta) {
  if (!P) return CYL_EINVAL;
  if (P->is_batch) return CYL_ESTATE;
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
  if (!P || !J || which < 0 || which >= cyl::kNumKinds || k < 0 || k > P->hp.p / 2 || parity < 0 || parity > 1)
    return CYL_EINVAL;
  if (P->is_batch) return CYL_ESTATE;
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

cyl_status cyl_plan_launch_info(cyl_plan_t P, int which, int *info) {
  if (!P || !info || which < 0 || which >= cyl::kNumKinds) return CYL_EINVAL;
  if (P->is_batch) return CYL_ESTATE;
  const auto &KT = P->hp.kind[which];
  int nsl = 0;
  for (const Item &it : KT.items) nsl = std::max(nsl, it.nsl);
  info[0] = (int)KT.items.size();
  info[1] = P->threads[which];
  info[2] = P->twist_half[which];
  info[3] = P->use_smem[which];
  info[4] = (int)P->smem[which];
  info[5] = P->cluster > 1 ? P->cluster : 1;
  info[6] = nsl;
  info[7] = KT.built ? 1 : 0;
  info[8] = (P->cluster > 1 || !KT.built) ? 0 : P->all_tw[which];
  return CYL_OK;
}

cyl_status cyl_plan_item_tables(cyl_plan_t P, int which, int item, int j, int transposed, int *info,
                                double *radial, double *vertical) {
  if (!P || !info || which < 0 || which >= cyl::kNumKinds || item < 0 || j < 0) return CYL_EINVAL;
  if (P->is_batch) return CYL_ESTATE;
  const auto &KT = P->hp.kind[which];
  if (!KT.built) return CYL_ESTATE;
  if (item >= (int)KT.items.size()) return CYL_EINVAL;
  const Item &it = KT.items[item];
  if (j >= it.J) return CYL_EINVAL;
  const int twr = transposed ? it.twrT : it.twr, twz = transposed ? it.twzT : it.twz;
  info[0] = it.M; info[1] = it.Nz; info[2] = it.J; info[3] = twr; info[4] = twz;
  info[5] = it.k; info[6] = it.pr; info[7] = it.pz;
  if (transposed && (it.roffT < 0 || it.zoffT < 0)) return CYL_ESTATE;
  const size_t rs = (size_t)it.M * cyl::RSTRIDE + (twr ? cyl::RTWIST : 0);
  const size_t zs = (size_t)it.Nz * cyl::ZSTRIDE + (twz ? cyl::ZTWIST : 0);
  const double *F = P->hp.factors.data();
  const long long ro = transposed ? it.roffT : it.roff, zo = transposed ? it.zoffT : it.zoff;
  if (radial) std::memcpy(radial, F + ro + (size_t)j * rs, rs * sizeof(double));
  if (vertical) std::memcpy(vertical, F + zo + (size_t)j * zs, zs * sizeof(double));
  return CYL_OK;
}

cyl_status cyl_plan_operator(cyl_plan_t P, int op, int which, int k, int parity, int *dim, double *out) {
  if (!P || !dim || op < 0 || op > 3 || which < 0 || which >= cyl::kNumKinds || parity < 0 || parity > 1 || k < 0 ||
      k > P->hp.p / 2)
    return CYL_EINVAL;
  if (P->is_batch) return CYL_ESTATE;
  const HostPlan &h = P->hp;
  if (which >= 1 && !(h.alpha > 0 && h.dt > 0)) return CYL_ESTATE;
  const double ka = which >= 1 ? h.alpha * h.dt * cyl::bdf_kappa(which) : 1.0;
  cyl::Band B;
  if (op == 0) {
    cyl::Band L = h.Lblk(k, parity), C = h.Cblk(parity);
    B = cyl::Band(L.n, 2, 3);
    for (int i = 0; i < L.n; ++i)
      for (int j = std::max(0, i - 2); j <= std::min(L.n - 1, i + 3); ++j)
        B.at(i, j) = which >= 1 ? C.get(i, j) - ka * L.get(i, j) : -L.get(i, j);
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

namespace {

constexpr int kNsArrays = 12;   // workspace arrays of N doubles of cyl_ns_step

// One Navier-Stokes step (Section 4) on the vorticity PT state (lw, gw); see
// include/cyl.h: cyl_ns_step.  W[0] gamma_v; W[1..3] v, then N = v x omega
// (grid values); W[4..6] omega values, then N's coefficients; W[7], W[8]
// coefficient scratch; W[9] value scratch; W[10], W[11] s1 / s2, then
// gamma_a / lambda_a.
cyl_status ns_one_step(cyl_plan_s *P, double *lw, double *gw, double *const W[kNsArrays]) {
  const HostPlan &h = P->hp;
  const int m = h.m, n = h.n, p = h.p;
  const long long mn = (long long)m * n, N = (long long)p * mn;
  const int sms = P->sms;
  cudaStream_t st = P->st;
  cyl_status s;
  cudaError_t e = cudaSuccess;
  // derivative of coefficients `in` into `out`: 'r', 'z' or 't' (theta)
  auto d = [&](char ax, const double *in, double *out) -> cudaError_t {
    if (ax == 't') return cyl::launch_deriv_theta(in, out, p, mn, sms, st);
    if (ax == 'r') return cyl::launch_deriv_cheb(in, out, p, m, n, sms, st);
    return cyl::launch_deriv_cheb(in, out, (long long)p * m, n, 1, sms, st);
  };
  // dst (grid values) (+)= coef r^rpow values(C)
  auto acc = [&](double *dst, const double *C, double coef, int rpow, bool init) -> cyl_status {
    cyl_status q = coeffs2vals_impl(P, C, W[9]);
    if (q != CYL_OK) return q;
    return from_cuda(cyl::launch_accum_r(dst, W[9], P->d_radius, p, m, n, coef, rpow, init, sms, st));
  };
#define NS_TRY(x) do { if ((e = (x)) != cudaSuccess) return from_cuda(e); } while (0)
#define NS_S(x) do { if ((s = (x)) != CYL_OK) return s; } while (0)
  // PT components of curl(lam z) + curl curl(gam z) into (Vr, Vt, Vz), grid values (eq. pt).  The
  // values of d_r lam are kept in dr_lam_out when given; dr_gam_in, when given, holds the values of
  // d_r gam (the velocity's lambda is the vorticity's gamma, so the second call reuses the first's).
  auto pt_field = [&](const double *lam, const double *gam, double *Vr, double *Vt, double *Vz, double *dr_lam_out,
                      const double *dr_gam_in) -> cyl_status {
    cyl_status q;
    cudaError_t ee;
    if ((ee = d('t', lam, W[7])) != cudaSuccess) return from_cuda(ee);          // V_r = r^-1 d_th lam + d_r d_z gam
    if ((q = acc(Vr, W[7], 1.0, -1, true)) != CYL_OK) return q;
    if ((ee = d('z', gam, W[7])) != cudaSuccess || (ee = d('r', W[7], W[8])) != cudaSuccess) return from_cuda(ee);
    if ((q = acc(Vr, W[8], 1.0, 0, false)) != CYL_OK) return q;
    if ((ee = d('r', lam, W[7])) != cudaSuccess) return from_cuda(ee);          // V_th = -d_r lam + r^-1 d_th d_z gam
    if (dr_lam_out) {
      if ((q = coeffs2vals_impl(P, W[7], dr_lam_out)) != CYL_OK) return q;
      if ((ee = cyl::launch_accum_r(Vt, dr_lam_out, P->d_radius, p, m, n, -1.0, 0, true, sms, st)) != cudaSuccess)
        return from_cuda(ee);
    } else if ((q = acc(Vt, W[7], -1.0, 0, true)) != CYL_OK) {
      return q;
    }
    if ((ee = d('z', gam, W[7])) != cudaSuccess || (ee = d('t', W[7], W[8])) != cudaSuccess) return from_cuda(ee);
    if ((q = acc(Vt, W[8], 1.0, -1, false)) != CYL_OK) return q;
    if ((ee = d('r', gam, W[7])) != cudaSuccess || (ee = d('r', W[7], W[8])) != cudaSuccess) return from_cuda(ee);
    if ((q = acc(Vz, W[8], -1.0, 0, true)) != CYL_OK) return q;                 // V_z = -Delta_h gam
    if (dr_gam_in) {
      if ((ee = cyl::launch_accum_r(Vz, dr_gam_in, P->d_radius, p, m, n, -1.0, -1, false, sms, st)) != cudaSuccess)
        return from_cuda(ee);
    } else if ((q = acc(Vz, W[7], -1.0, -1, false)) != CYL_OK) {
      return q;
    }
    if ((ee = d('t', gam, W[7])) != cudaSuccess || (ee = d('t', W[7], W[8])) != cudaSuccess) return from_cuda(ee);
    return acc(Vz, W[8], -1.0, -2, false);
  };
  // 1. velocity potentials (eq. ptcurl): lambda_v = gamma_w, -lap gamma_v = lambda_w, refined once: the
  //    first solution u1 (W[1]) enters as the lifting of a second solve whose right side is the
  //    residual (W[2] = minus the Poisson operator applied to u1), so W[0] = u1 + the correction.  The
  //    nonlinear term differentiates gamma_v up to three times; at 128^3 the ADI's own error (~2e-14
  //    of max|gamma_v|) alone moved a step by ~4e-11.
  NS_S(run_adi(P, 0, lw, W[1], nullptr, 0.0, 0, 1, nullptr, 1));
  {
    cyl::AdiArgs a = step_args(P, 0, lw, W[0], nullptr, 0.0, 0, 1, nullptr, 1, false);
    NS_TRY(cyl::launch_lift_correction(a, W[1], W[2], 0.0, 1.0, std::min(P->threads[0], 256), st));
    a.lift = W[1];
    a.corr = W[2];
    NS_TRY(cyl::launch_adi(a, P->threads[0], P->smem[0], st));
  }
  // 2. v and omega on the grid (eq. pt); W[10] carries the values of d_r gamma_w from one to the other
  NS_S(pt_field(gw, W[0], W[1], W[2], W[3], W[10], nullptr));
  NS_S(pt_field(lw, gw, W[4], W[5], W[6], nullptr, W[10]));
  // 3. N = v x omega (in place of v)
  {
    const double *V[3] = {W[1], W[2], W[3]}, *Om[3] = {W[4], W[5], W[6]};
    double *No[3] = {W[1], W[2], W[3]};
    NS_TRY(cyl::launch_cross(V, Om, No, N, sms, st));
  }
  for (int c = 0; c < 3; ++c) NS_S(vals2coeffs_impl(P, W[1 + c], W[4 + c]));
  // 4. right sides of eq. ptpoisson for a = curl N:
  //    s1 = d_r N_th + N_th / r - r^-1 d_th N_r
  NS_TRY(d('r', W[5], W[7]));
  NS_S(acc(W[10], W[7], 1.0, 0, true));
  NS_TRY(cyl::launch_accum_r(W[10], W[2], P->d_radius, p, m, n, 1.0, -1, false, sms, st));
  NS_TRY(d('t', W[4], W[7]));
  NS_S(acc(W[10], W[7], -1.0, -1, false));
  NS_S(vals2coeffs_impl(P, W[10], W[10]));
  //    s2 = d_z (d_r N_r + N_r / r + r^-1 d_th N_th) - Delta_h N_z
  NS_TRY(d('r', W[4], W[7]));
  NS_S(acc(W[11], W[7], 1.0, 0, true));
  NS_TRY(cyl::launch_accum_r(W[11], W[1], P->d_radius, p, m, n, 1.0, -1, false, sms, st));
  NS_TRY(d('t', W[5], W[7]));
  NS_S(acc(W[11], W[7], 1.0, -1, false));
  NS_S(vals2coeffs_impl(P, W[11], W[8]));
  NS_TRY(d('z', W[8], W[7]));                      // the two r^0 terms combined in coefficients:
  NS_TRY(d('r', W[6], W[8]));                      // W[7] = d_z div_h - d_r^2 N_z, one transform
  NS_TRY(d('r', W[8], W[9]));
  NS_TRY(cyl::launch_accum_r(W[7], W[9], P->d_radius, p, m, n, -1.0, 0, false, sms, st));
  NS_S(coeffs2vals_impl(P, W[7], W[11]));
  NS_S(acc(W[11], W[8], -1.0, -1, false));
  NS_TRY(d('t', W[6], W[7]));
  NS_TRY(d('t', W[7], W[8]));
  NS_S(acc(W[11], W[8], -1.0, -2, false));
  NS_S(vals2coeffs_impl(P, W[11], W[11]));
  //    horizontal solves: gamma_a from s1, lambda_a from s2 (in place)
  const int zero_other = (h.flags & CYL_BOTH_PARITIES) ? 0 : 1;
  NS_TRY(cyl::launch_disk_poisson(P->d_disk_items, P->ndisk, P->d_fac, W[10], W[10], n, mn, zero_other,
                                  P->disk_threads, st));
  NS_TRY(cyl::launch_disk_poisson(P->d_disk_items, P->ndisk, P->d_fac, W[11], W[11], n, mn, zero_other,
                                  P->disk_threads, st));
  // 5. eq. NSrewrite, IMEX BDF1: one heat step each with alpha = 1/Re and forcing (lambda_a, gamma_a)
  NS_S(run_adi(P, 1, lw, lw, W[11], h.dt, 0, 1, nullptr, 1));
  NS_S(run_adi(P, 1, gw, gw, W[10], h.dt, 0, 1, nullptr, 1));
#undef NS_TRY
#undef NS_S
  (void)N;
  return CYL_OK;
}

}  // namespace

extern "C" {

cyl_status cyl_ns_workspace(cyl_plan_t P, size_t *bytes) {
  if (!P || !bytes) return CYL_EINVAL;
  if (P->is_batch) return CYL_ESTATE;
  *bytes = (size_t)kNsArrays * P->N * sizeof(double);
  return CYL_OK;
}

cyl_status cyl_ns_step(cyl_plan_t P, double *lam_w, double *gam_w, int nsteps, void *workspace,
                       size_t workspace_bytes) {
  if (!P || !lam_w || !gam_w || nsteps < 0) return CYL_EINVAL;
  if (P->is_batch || P->host_only || !P->hp.kind[0].built || !P->hp.kind[1].built || !P->d_disk_items)
    return CYL_ESTATE;
  if (P->hp.m % 2) return CYL_EINVAL;
  if (!workspace || workspace_bytes < (size_t)kNsArrays * P->N * sizeof(double)) return CYL_EINVAL;
  double *W[kNsArrays];
  for (int i = 0; i < kNsArrays; ++i) W[i] = static_cast<double *>(workspace) + (size_t)i * P->N;
  for (int s = 0; s < nsteps; ++s) {
    cyl_status st = ns_one_step(P, lam_w, gam_w, W);
    if (st != CYL_OK) return st;
  }
  return CYL_OK;
}

}  // extern "C"

extern "C" {

cyl_status cyl_plan_batch(cyl_plan_t *plan, int nprob, const int *n_r, const int *n_z, const int *n_theta,
                          const double *alpha, double dt, double adi_tol, unsigned flags, void *stream) {
  if (!plan) return CYL_EINVAL;
  *plan = nullptr;
  if (nprob < 1 || !n_r || !n_z || !n_theta || !alpha || !(dt > 0.0)) return CYL_EINVAL;
  if (!(adi_tol > 0.0) || adi_tol > 1e-2) return CYL_EINVAL;
  if (!(flags & CYL_WITH_HEAT) ||
      (flags & ~(unsigned)(CYL_WITH_HEAT | CYL_BOTH_PARITIES | CYL_PLAIN_SWEEPS | CYL_HOST_ONLY)))
    return CYL_EINVAL;
  for (int i = 0; i < nprob; ++i)
    if (n_r[i] < 4 || n_z[i] < 4 || n_theta[i] < 2 || (n_theta[i] & 1) || !(alpha[i] > 0.0) ||
        n_r[i] > 256 || n_z[i] > 256)
      return CYL_EINVAL;
  cyl_plan_s *P = new (std::nothrow) cyl_plan_s();
  if (!P) return CYL_ENOMEM;
  P->is_batch = true;
  P->nprob = nprob;
  P->st = (cudaStream_t)stream;
  // host plans in parallel (independent problems)
  std::vector<HostPlan> hps(nprob);
  std::vector<std::string> errs(nprob);
  const int nth = std::max(1u, std::min(std::thread::hardware_concurrency(), 64u));
  std::vector<std::thread> pool;
  for (int t = 0; t < nth; ++t)
    pool.emplace_back([&, t]() {
      for (int i = t; i < nprob; i += nth) {
        try {
          // twisted solves per single slice (configure_batch splits twisted pairs)
          errs[i] = cyl::build_host_plan(hps[i], n_r[i], n_z[i], n_theta[i], alpha[i], dt, adi_tol,
                                         (flags & CYL_BOTH_PARITIES) | CYL_WITH_HEAT, 1,
                                         (flags & CYL_PLAIN_SWEEPS) ? 0 : 2);
        } catch (...) {
          errs[i] = "host plan failed";
        }
      }
    });
  for (auto &th : pool) th.join();
  for (int i = 0; i < nprob; ++i)
    if (!errs[i].empty()) {
      delete P;
      return CYL_EINVAL;
    }
  // merge factor tables and items
  P->offsets.assign(nprob + 1, 0);
  size_t ftotal = 0;
  for (int i = 0; i < nprob; ++i) {
    P->offsets[i + 1] = P->offsets[i] + (long long)n_r[i] * n_z[i] * n_theta[i];
    ftotal += hps[i].factors.size();
  }
  P->N = (size_t)P->offsets[nprob];
  std::vector<double> fac;
  fac.reserve(ftotal);
  for (int i = 0; i < nprob; ++i) {
    const long long base = (long long)fac.size();
    fac.insert(fac.end(), hps[i].factors.begin(), hps[i].factors.end());
    for (Item it : hps[i].kind[1].items) {
      it.roff += base; it.zoff += base; it.r2off += base; it.c02off += base;
      it.lkoff += base; it.d2off += base;
      if (it.roffT >= 0) it.roffT += base;
      if (it.zoffT >= 0) it.zoffT += base;
      it.xoff = P->offsets[i];
      P->bitems.push_back(it);
    }
  }
  P->hp.flags = flags;
  P->hp.dt = dt;
  P->hp.tol = adi_tol;
  P->hp.kind[1].built = true;
  P->host_only = (flags & CYL_HOST_ONLY) != 0;
  if (P->host_only) {                        // host tables and the batch configuration only
    cyl_status s = CYL_EINVAL;
    for (const auto &d : kBatchDefaults)
      if ((s = configure_batch(P, d[0], d[1])) == CYL_OK) break;
    if (s != CYL_OK) {
      delete P;
      return s;
    }
    *plan = P;
    return CYL_OK;
  }
  cudaError_t e = cudaGetDevice(&P->device);
  if (e == cudaSuccess) e = upload(&P->d_fac, fac.data(), fac.size());
  if (e == cudaSuccess) e = cudaMalloc((void **)&P->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(P->d_err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P->aux, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming);
  cyl_status s = from_cuda(e);
  if (s == CYL_OK)                           // first feasible default (the autotuner refines it)
    for (const auto &d : kBatchDefaults)
      if ((s = configure_batch(P, d[0], d[1])) == CYL_OK) break;
  if (s != CYL_OK) {
    free_device(P);
    delete P;
    cudaGetLastError();
    return s;
  }
  *plan = P;
  return CYL_OK;
}

cyl_status cyl_batch_layout(cyl_plan_t P, int *nprob, long long *offsets) {
  if (!P || !P->is_batch) return CYL_EINVAL;
  if (nprob) *nprob = P->nprob;
  if (offsets) std::memcpy(offsets, P->offsets.data(), (P->nprob + 1) * sizeof(long long));
  return CYL_OK;
}

cyl_status cyl_heat_step_batch(cyl_plan_t P, double *T, const double *g, int nsteps) {
  if (!P || !T || nsteps < 0) return CYL_EINVAL;
  if (!P->is_batch || P->host_only) return CYL_ESTATE;
  if (nsteps == 0) return CYL_OK;
  return run_batch(P, T, g, nsteps);
}

cyl_status cyl_batch_set_config(cyl_plan_t P, int threshold, int groups, int chains_per_thread) {
  if (!P || !P->is_batch || (groups != 1 && groups != 2 && groups != 4) || threshold < 0) return CYL_EINVAL;
  if (chains_per_thread != 1 && chains_per_thread != 2) return CYL_EINVAL;
  return configure_batch(P, threshold, groups, chains_per_thread);
}

cyl_status cyl_batch_get_config(cyl_plan_t P, int *threshold, int *groups, int *chains_per_thread,
                                int *items_per_class) {
  if (!P || !P->is_batch) return CYL_EINVAL;
  if (threshold) *threshold = P->threshold;
  if (groups) *groups = P->bc[1].G;
  if (chains_per_thread) *chains_per_thread = P->chains_per_thread;
  if (items_per_class) {
    items_per_class[0] = P->bc[0].nitems;
    items_per_class[1] = P->bc[1].nitems;
  }
  return CYL_OK;
}

cyl_status cyl_batch_autotune(cyl_plan_t P, const double *T, const double *g, int nsteps, double *best_ms) {
  if (!P || !P->is_batch || !T || nsteps < 1) return CYL_EINVAL;
  if (P->host_only) return CYL_ESTATE;
  double *work = nullptr;
  cudaError_t e = cudaMalloc((void **)&work, P->N * sizeof(double));
  if (e != cudaSuccess) return from_cuda(e);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int thresholds[] = {0, 31, 47, 63, 95};
  const int groups[] = {1, 2, 4};
  float best = 1e30f;
  int bt = 63, bg = 4, bc = 1;
  cyl_status s = CYL_OK;
  for (int th : thresholds)
    for (int G : groups)
      for (int cpt = 1; cpt <= 2; ++cpt) {
      if (th == 0 && G != 1) continue;
      s = configure_batch(P, th, G, cpt);
      if (s != CYL_OK) { s = CYL_OK; continue; }
      float ms = 0;
      for (int rep = 0; rep < 2 && s == CYL_OK; ++rep) {
        cudaMemcpyAsync(work, T, P->N * sizeof(double), cudaMemcpyDeviceToDevice, P->st);
        cudaEventRecord(e0, P->st);
        s = run_batch(P, work, g, nsteps);
        cudaEventRecord(e1, P->st);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
      }
      if (s != CYL_OK) break;
      if (ms < best) { best = ms; bt = th; bg = G; bc = cpt; }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(work);
  if (s != CYL_OK) return s;
  if (best_ms) *best_ms = best;
  return configure_batch(P, bt, bg, bc);
}

}  // extern "C"
