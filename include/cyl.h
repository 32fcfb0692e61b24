/*
 * cyl.h -- C ABI of libcyl, a GB300-native (sm_103a) FP64 implementation of the
 * Chebyshev-Chebyshev-Fourier (CCF) solver for the heat and Poisson equations in
 * the closed cylinder r <= 1, z in [-1, 1] (Darrow, arXiv 2206.04827).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid sizes follow Section 2: m = n_r radial, n = n_z vertical, p = n_theta
 * angular points of the doubled grid (Definition "grid"); N = m n p unknowns.
 *
 * Array layout (values and coefficients alike): row-major [p][m][n] float64,
 * i.e. index (l, j, k) at offset (l * m + j) * n + k, z fastest.
 *   * Values are samples on the doubled grid of Definition "grid".
 *   * Coefficients are those of the unique CCF interpolant (Section 2,
 *     interpolant f*), stored half-complex along theta: slice 0 holds c_0,
 *     slices 2w-1 and 2w hold Re c_w and Im c_w (w = 1 .. p/2-1), slice p-1
 *     holds the (real) Nyquist coefficient c_{-p/2}.  Negative wavenumbers are
 *     implied by c_{-w} = conj(c_w); only real fields are represented.
 *
 * Boundary data: homogeneous Dirichlet at r = +-1 (the doubled radius: r = -1
 * is the physical wall at theta + pi) and z = +-1.  The paper does not state
 * its boundary conditions; this is the reading the library implements.
 *
 * Radial parity: a real field on the doubled grid has c_{j,k,w} = 0 unless
 * j = w (mod 2), and every operator couples only equal parities.  By default
 * the solvers compute the physical parity block and write zeros in the other;
 * CYL_BOTH_PARITIES solves both blocks (inputs that are not real fields).
 *
 * Pointers: unless stated otherwise every array argument is a caller-owned
 * DEVICE pointer to float64 of N elements, valid on the plan's device.  The
 * plan owns its operator tables, ADI factors and scratch.  Calls that take
 * device pointers are asynchronous on the plan's CUDA stream and make no host
 * synchronisation and no allocation.
 *
 * Errors: every entry point returns a cyl_status; no C++ exception crosses the
 * ABI.  On error the contents of output arrays are unspecified.
 */
#ifndef CYL_H
#define CYL_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cyl_plan_s *cyl_plan_t;

typedef enum {
  CYL_OK = 0,
  CYL_EINVAL = 1,   /* invalid size, parameter, flag or NULL pointer          */
  CYL_ENOMEM = 2,   /* host or device allocation failed                       */
  CYL_ECUDA = 3,    /* a CUDA runtime call failed                             */
  CYL_ETIMEOUT = 4, /* a bounded device-side wait ran out                      */
  CYL_ESTATE = 5    /* the plan was not built for this operation              */
} cyl_status;

/* plan flags */
#define CYL_WITH_POISSON   1u  /* build the Poisson factors                     */
#define CYL_WITH_HEAT      2u  /* build the BDF1 heat factors (needs alpha, dt) */
#define CYL_BOTH_PARITIES  4u  /* solve both radial parity blocks                */
#define CYL_HOST_ONLY      8u  /* host tables only: no device memory, no kernels */
#define CYL_FORCE_GLOBAL  16u  /* keep ADI work arrays in global memory          */
/* Failure-detection test only: the ADI kernels never start their factor-table
 * copies, so every bounded device wait runs out (after about 1 ms) and
 * cyl_sync reports CYL_ETIMEOUT; the results of such a plan are garbage. */
#define CYL_TEST_NO_TMA   32u
/* allocate the two N-element lifting arrays of non-zero Dirichlet data at
 * plan time (otherwise the first call with bc != NULL allocates them, which
 * a stream capture does not allow) */
#define CYL_WITH_BC       64u
/* plain LU sweeps only: no twisted (two-sided) solves, which otherwise run
 * where every sweep of a two-slice item has at most 128 chains (grids up to
 * about 130) and, with single-slice items, where two-slice work arrays leave
 * shared memory (grids of about 220 to 514 points per axis); the results
 * then match the persistent batch kernel bit for bit */
#define CYL_PLAIN_SWEEPS 128u
/* build the horizontal (disk) Poisson tables for cyl_disk_poisson */
#define CYL_WITH_DISK    256u
/* cluster mode: the CTAs of a thread-block cluster share each work item
 * through its global work area, each with at most 128 chains per sweep,
 * solved as twisted two-thread chains (at most 8 CTAs per item: grids up
 * to about 1024 points per axis).  Off by default: on GB300 it is slower
 * than one CTA per item for the grids whose work arrays leave shared memory.
 * CYL_FORCE_GLOBAL or CYL_PLAIN_SWEEPS override it. */
#define CYL_FORCE_CLUSTER 512u

/* space selector of cyl_poisson */
#define CYL_VALUES 0
#define CYL_COEFFS 1

/*
 * cyl_plan -- build a solver plan for one grid.
 *
 * Section 3: the per-mode matrix equation (eq. HelmholtzMatEqn) and its
 * Poisson analogue; Algorithm 1 (ADI); the shift choice below Algorithm 1
 * (Zolotarev-type shifts from K(k), dn and a Moebius map).
 *
 *   n_r, n_z   4 .. 4096;  n_theta even, 2 .. 4096 (the doubled grid needs theta + pi).
 *   alpha, dt  > 0 when CYL_WITH_HEAT is set (diffusivity; BDF1 step kappa = dt).
 *   adi_tol    in (0, 1e-2]: target relative accuracy of the Zolotarev bound;
 *              the iteration count per mode is J = ceil(log(16 gamma) log(4/tol) / pi^2).
 *   flags      CYL_WITH_POISSON and/or CYL_WITH_HEAT, optionally
 *              CYL_BOTH_PARITIES, CYL_HOST_ONLY, CYL_FORCE_GLOBAL, CYL_WITH_BC,
 *              CYL_PLAIN_SWEEPS, CYL_FORCE_CLUSTER; CYL_WITH_DISK (alone or
 *              with the others).
 *   stream     cudaStream_t on which every device call of this plan runs
 *              (NULL = legacy default stream).  Ignored with CYL_HOST_ONLY.
 *
 * Builds the banded operators from the three-term relations, estimates the
 * spectral intervals of both pencils per wavenumber, computes the shifts,
 * factors every shifted banded matrix (LU without pivoting, reciprocal
 * pivots) and uploads everything.  Allocates host and device memory; not
 * for use inside stream capture.  *plan is set to NULL on error.
 */
cyl_status cyl_plan(cyl_plan_t *plan, int n_r, int n_z, int n_theta, double alpha,
                    double dt, double adi_tol, unsigned flags, void *stream);

/*
 * cyl_plan_bdf -- cyl_plan for runs of the b-th order BDF, b = bdf_order in
 * 1..4 (Section 3: BDF 1, BDF 4, and the kappa^(b), delta^(b) definitions;
 * orders 2 and 3 from the same backward-difference family:
 * kappa^(b)/h = 1, 2/3, 6/11, 12/25).  With CYL_WITH_HEAT the plan holds the
 * factors of every order 1..b (the first steps of a run use lower orders, see
 * cyl_heat_step_bdf), so it needs about b times the factor memory of
 * cyl_plan.  cyl_plan(...) is cyl_plan_bdf(..., 1, ...).
 */
cyl_status cyl_plan_bdf(cyl_plan_t *plan, int n_r, int n_z, int n_theta, double alpha,
                        double dt, double adi_tol, int bdf_order, unsigned flags, void *stream);

/* Release a plan and all memory it owns (NULL is accepted). */
cyl_status cyl_destroy(cyl_plan_t plan);

/*
 * cyl_vals2coeffs -- Section 2, the DCT-I in r, DCT-I in z and DFT in theta
 * that take grid values to interpolation coefficients.  vals and coeffs are
 * device arrays of N float64 ([p][m][n]); they may alias.
 */
cyl_status cyl_vals2coeffs(cyl_plan_t plan, const double *vals, double *coeffs);

/* cyl_coeffs2vals -- inverse of cyl_vals2coeffs (evaluation of f* on the grid). */
cyl_status cyl_coeffs2vals(cyl_plan_t plan, const double *coeffs, double *vals);

/*
 * Dirichlet data (bc arguments).  The paper's problem statement (Section 1)
 * poses the wall condition u = 0; non-zero data are applied by lifting:
 * u = u0 + W, where W is the transfinite blend of the data (linear in r
 * between the faces r = -1, +1 of the doubled grid, plus linear in z between
 * z = -1, +1, minus the bilinear corner term), u0 has zero data and solves
 * the same equation with the left operator applied to W moved to the right
 * side.  bc is a device array of N float64 GRID VALUES in the [p][m][n]
 * layout of which only the boundary nodes (radial index 0 or m-1, vertical
 * index 0 or n-1) are read; the interior is ignored.  Without
 * CYL_BOTH_PARITIES the data must be a field on the doubled grid
 * (value at (-r, z, theta) = value at (r, z, theta + pi)), as f must.
 * bc = NULL means zero data.  The first call with bc != NULL allocates two
 * N-element plan arrays unless the plan was made with CYL_WITH_BC.
 */

/*
 * cyl_poisson -- solve -lap u = f with Dirichlet data bc (the Poisson solves
 * of Section 4, with the Section 3 discretisation without its identity
 * term).  f and u are device arrays of N float64; space = CYL_VALUES (both
 * are grid values) or CYL_COEFFS (both are half-complex coefficients); bc is
 * NULL (u = 0 on the wall) or grid values as described above, in either
 * space.  f and u may alias.  Needs CYL_WITH_POISSON.
 */
cyl_status cyl_poisson(cyl_plan_t plan, const double *f, const double *bc, double *u, int space);

/*
 * cyl_disk_poisson -- the horizontal Poisson solve -Delta_h u = f,
 * Delta_h = lap - d_z^2 (Section 4, eq. ptpoisson: the toroidal and poloidal
 * potentials of the poloidal-toroidal decomposition), "diagonalised in theta
 * and z": z enters as a parameter, so every (half-complex slice,
 * z-coefficient) column is one banded radial tau solve of the r^2-multiplied
 * operator -L_k of eq. HelmholtzMatEqn with u = 0 at r = -1 and r = +1 (the
 * boundary conditions are unstated; no condition in z, as Delta_h has no z
 * derivative).  f and u: device arrays of N float64 in the given space
 * (CYL_VALUES or CYL_COEFFS); they may alias.  One launch in coefficient
 * space (plus the transforms in value space).  Needs CYL_WITH_DISK.
 */
cyl_status cyl_disk_poisson(cyl_plan_t plan, const double *f, double *u, int space);

/*
 * cyl_heat_step -- advance (d_t - alpha lap) T = g by nsteps BDF1 steps
 * (Section 3, BDF 1 and eq. HelmholtzMatEqn with kappa = dt, delta X = X_n;
 * the forcing of step n -> n+1 is g at level n).
 *
 *   T              device, N float64 coefficients; in: T_0, out: T_nsteps.
 *   g              device coefficients, or NULL for g = 0.
 *   g_step_stride  0: the same g every step; otherwise step n reads
 *                  g + n * g_step_stride (elements, >= N).
 *   ckpt           NULL, or device array of (nsteps / ckpt_every + 1) * N
 *                  float64 that receives T_0, T_c, T_2c, ... (c = ckpt_every).
 *   ckpt_every     >= 1 when ckpt is given.
 * Needs CYL_WITH_HEAT.
 */
cyl_status cyl_heat_step(cyl_plan_t plan, double *T, const double *g, long long g_step_stride,
                         int nsteps, double *ckpt, int ckpt_every);

/* cyl_heat_step_bc -- cyl_heat_step with time-constant Dirichlet data bc
 * (grid values, see above; NULL = zero data): every step returns
 * T_{n+1} = u0 + W with u0 of zero data.  T_0 itself need not meet the data. */
cyl_status cyl_heat_step_bc(cyl_plan_t plan, double *T, const double *g, long long g_step_stride,
                            int nsteps, const double *bc, double *ckpt, int ckpt_every);

/*
 * cyl_heat_step_bdf -- nsteps steps of the b-th order BDF (b = the plan's
 * bdf_order): eq. HelmholtzMatEqn with kappa = kappa^(b) and right side
 * R_2 (delta^(b) X_n + kappa g_n) C02^T, delta^(b) X_n = sum_i beta_i X_{n-i}.
 *
 *   hist     device, b * N float64 coefficients; slot i (hist + i * N) holds
 *            X_{n-i}, i = 0 the newest.  In/out: on return slot i holds
 *            X_{n+nsteps-i}.
 *   nvalid   1..b: how many slots hold known states on entry.  While fewer
 *            than b states are known a step uses BDF v (v = states known),
 *            one launch per such start-up step; slots beyond
 *            min(b, nvalid + nsteps) are unspecified on return.
 *   g, g_step_stride, bc   as for cyl_heat_step_bc (g + s * stride drives
 *            step s; bc: time-constant Dirichlet data or NULL).
 * The history is a ring inside the kernels (each step overwrites the oldest
 * slot); one elementwise pass at the end restores the slot order above.
 * Needs a plan from cyl_plan_bdf with CYL_WITH_HEAT.
 */
cyl_status cyl_heat_step_bdf(cyl_plan_t plan, double *hist, int nvalid, const double *g,
                             long long g_step_stride, int nsteps, const double *bc);

/*
 * cyl_heat_adjoint_bdf -- reverse-mode derivatives of a scalar loss of the
 * final history of the run cyl_heat_step_bdf(hist0, nvalid, g, g_step_stride,
 * nsteps, bc) computes (not in the paper: the transpose of that multistep
 * map).  Backward through the steps, with lam_j = dL/dX_j accumulated:
 * w = (step map of BDF b)^T lam_{s+1}; lam_{s-i} += beta_i w; dL/dg_s =
 * kappa^(b) w; dL/dalpha += <w, X_{s+1} - delta^(b) X_s - kappa^(b) g_s> / alpha
 * (the BDF b analogue of the identity of cyl_heat_adjoint, on the lifted
 * states when bc != NULL).  Start-up steps use their own order, as forward.
 *
 *   hist0, nvalid, g, g_step_stride, nsteps, bc   as for cyl_heat_step_bdf
 *               (hist0 is not modified; may be NULL when dL_dalpha is NULL).
 *   dL_dhistN   device, b * N float64: dL/d(final history), slot i = dL/dX_{N-i}
 *               (slots beyond min(b, nvalid + nsteps) are ignored).
 *   dL_dhist0   device, b * N float64 output, slot i = dL/dX_{-i} for
 *               i < nvalid, zero beyond (may alias dL_dhistN).
 *   dL_dg, dL_dalpha, ckpt_every   as for cyl_heat_adjoint (checkpoints hold
 *               whole histories: b states every ckpt_every steps).
 *   workspace   device memory of at least cyl_heat_adjoint_bdf_workspace()
 *               bytes (always needed: the adjoint ring of b + 1 states).
 * Needs a plan from cyl_plan_bdf with CYL_WITH_HEAT.
 */
cyl_status cyl_heat_adjoint_bdf(cyl_plan_t plan, const double *hist0, int nvalid, const double *g,
                                long long g_step_stride, int nsteps, const double *bc, int ckpt_every,
                                const double *dL_dhistN, double *dL_dhist0, double *dL_dg,
                                double *dL_dalpha, void *workspace, size_t workspace_bytes);

/* Bytes of device workspace cyl_heat_adjoint_bdf needs. */
cyl_status cyl_heat_adjoint_bdf_workspace(cyl_plan_t plan, int nsteps, int ckpt_every, int need_alpha,
                                          size_t *bytes);

/*
 * cyl_heat_adjoint -- reverse-mode derivatives of a scalar loss L(T_N) of the
 * BDF1 run that cyl_heat_step(T0, g, g_step_stride, nsteps) computes.  Not in
 * the paper: the exact transpose of that linear stepping map, i.e. the
 * transposed Sylvester solves (ADI on A^T X B + C^T X D = E with the same
 * shifts) run backward through the steps.  dL/dalpha uses the forward states,
 * recomputed segment by segment from checkpoints every ckpt_every steps:
 * dL/dalpha = sum_n <dL/dT_n, T_{n+1} - T_n - dt g_n> / alpha, an identity of
 * the BDF1 step (the alpha-derivative of the solve is (E - C Y B^T) / alpha).
 *
 *   T0, g, g_step_stride, nsteps   as for cyl_heat_step (T0 is not modified;
 *               T0 may be NULL when dL_dalpha is NULL).
 *   dL_dTN      device, N float64: dL/dT_N (coefficient layout).
 *   dL_dT0      device, N float64 output (may alias dL_dTN).
 *   dL_dg       NULL, or device output shaped like g: N float64 when
 *               g_step_stride = 0 (summed over steps), else nsteps arrays at
 *               stride g_step_stride.
 *   dL_dalpha   NULL, or device pointer to ONE float64 output.
 *   ckpt_every  >= 1; states are recomputed in segments of this length
 *               (a value >= nsteps stores every state of the run).
 *   workspace   device memory of at least cyl_heat_adjoint_workspace() bytes
 *               (none is needed when dL_dalpha is NULL).
 * Cost: one forward pass for the checkpoints, one for the recomputation and
 * one transposed pass (only the last without dL_dalpha).  Needs CYL_WITH_HEAT.
 */
cyl_status cyl_heat_adjoint(cyl_plan_t plan, const double *T0, const double *g,
                            long long g_step_stride, int nsteps, int ckpt_every,
                            const double *dL_dTN, double *dL_dT0, double *dL_dg,
                            double *dL_dalpha, void *workspace, size_t workspace_bytes);

/* cyl_heat_adjoint_bc -- cyl_heat_adjoint of the run cyl_heat_step_bc(T0, g,
 * g_step_stride, nsteps, bc) computes.  The data enter that run affinely, so
 * dL/dT0 and dL/dg are those of the zero-data run; the alpha identity holds
 * on the lifted states, which the recomputation produces with bc.
 *   ckpt   NULL, or the checkpoints that forward run wrote (its ckpt argument
 *          with the same ckpt_every): the adjoint then reads them instead of
 *          recomputing them in a forward pass of its own (one forward pass
 *          fewer), and needs the smaller workspace of need_alpha = 2. */
cyl_status cyl_heat_adjoint_bc(cyl_plan_t plan, const double *T0, const double *g,
                               long long g_step_stride, int nsteps, const double *bc, int ckpt_every,
                               const double *ckpt, const double *dL_dTN, double *dL_dT0, double *dL_dg,
                               double *dL_dalpha, void *workspace, size_t workspace_bytes);

/* Bytes of device workspace cyl_heat_adjoint needs: need_alpha 0 (no dL/dalpha)
 * needs none, 1 the checkpoints and one recomputed segment, 2 (dL/dalpha with
 * the caller's checkpoints, cyl_heat_adjoint_bc) one recomputed segment. */
cyl_status cyl_heat_adjoint_workspace(cyl_plan_t plan, int nsteps, int ckpt_every, int need_alpha,
                                      size_t *bytes);

/* ---------------------------------------------------------------------------
 * Batches of independent cylinders (not in the paper: many problems of
 * uneven grids and every Fourier mode of each in one persistent launch).
 * ------------------------------------------------------------------------- */

/*
 * cyl_plan_batch -- one plan for nprob independent heat problems on grids
 * n_r[i] x n_z[i] x n_theta[i] (each 4 <= n_r, n_z <= 256, n_theta even >= 2),
 * diffusivities alpha[i] > 0, one step dt > 0 and one ADI tolerance.  flags:
 * CYL_WITH_HEAT (required), optionally CYL_BOTH_PARITIES, CYL_PLAIN_SWEEPS
 * (one-sided sweeps only; otherwise items of at most 128 chains per slice use
 * twisted solves, two threads per chain), CYL_HOST_ONLY (host tables and the
 * batch configuration only: cyl_batch_set_config / get_config work, the
 * device calls return CYL_ESTATE).  The per-problem
 * host plans are built in parallel threads.  The batch arrays are the
 * problems' [p][m][n] coefficient arrays concatenated in problem order
 * (offsets from cyl_batch_layout).  Every (problem, wavenumber, parity) work
 * item goes into a queue sorted by work, largest first; items whose
 * max(radial, vertical) block size exceeds a threshold run one per CTA, the
 * others run G per CTA (thread groups with named barriers); the two classes
 * are two persistent launches on two streams.  Allocates; not for use inside
 * stream capture.
 */
cyl_status cyl_plan_batch(cyl_plan_t *plan, int nprob, const int *n_r, const int *n_z,
                          const int *n_theta, const double *alpha, double dt, double adi_tol,
                          unsigned flags, void *stream);

/* Number of problems and nprob + 1 prefix offsets (in doubles) of each
 * problem's array inside the batch arrays (host output; either may be NULL). */
cyl_status cyl_batch_layout(cyl_plan_t plan, int *nprob, long long *offsets);

/*
 * cyl_heat_step_batch -- nsteps BDF1 steps of every problem of the batch
 * (per problem exactly the arithmetic of cyl_heat_step).  T: device batch
 * array, in/out; g: device batch array of forcings constant in time, or NULL.
 * No allocation, no host synchronisation: capturable in a CUDA graph.
 */
cyl_status cyl_heat_step_batch(cyl_plan_t plan, double *T, const double *g, int nsteps);

/* Launch configuration of a batch plan: threshold on max(M, Nz) between the
 * one-item-per-CTA class and the G-items-per-CTA class, G in {1, 2, 4}, and
 * the chains each thread of a one-sided (not twisted) class sweeps in turn,
 * 1 or 2 (twisted classes always run two threads per chain).  Setting it
 * reallocates the plan's work areas (not during capture). */
cyl_status cyl_batch_set_config(cyl_plan_t plan, int threshold, int groups, int chains_per_thread);
cyl_status cyl_batch_get_config(cyl_plan_t plan, int *threshold, int *groups, int *chains_per_thread,
                                int *items_per_class);

/*
 * cyl_batch_autotune -- time every candidate configuration (thresholds
 * 0/31/47/63/95 x G = 1/2/4 x chains per thread 1/2) for nsteps steps on
 * copies of the caller's T and
 * g, keep the fastest and return its time per call in *best_ms (nullable).
 * T is not modified.  Allocates a temporary batch array; host-synchronising.
 */
cyl_status cyl_batch_autotune(cyl_plan_t plan, const double *T, const double *g, int nsteps,
                              double *best_ms);

/*
 * cyl_sync -- wait for every call queued on the plan's stream, then report
 * device-side failures of those calls: CYL_ETIMEOUT when a bounded wait inside
 * a kernel ran out (the affected outputs are then unspecified; the flag is
 * cleared), CYL_ECUDA for a CUDA error.  Host-synchronising; not for use
 * inside stream capture.  Not in the paper.
 */
cyl_status cyl_sync(cyl_plan_t plan);

/*
 * cyl_vals2coeffs_noalloc -- the values -> coefficients transform of
 * cyl_vals2coeffs without a plan and without any allocation.  The paper has
 * no counterpart; this entry point exists for callers that cannot allocate
 * device memory: hosts whose own pool owns all device memory and forbids
 * other allocations, and loops that must never enter an allocator.
 * cyl_plan allocates, so such callers cannot use the planned entry points.
 *
 *   n_r, n_z     >= 2; n_theta even and >= 2.
 *   vals, coeffs caller-owned device arrays of n_r*n_z*n_theta float64
 *                ([p][m][n] layout as above); they may alias.
 *   stream       cudaStream_t to run on (NULL = legacy default stream).
 *
 * Scratch comes from one fixed array of CYL_NOALLOC_SCRATCH_DOUBLES float64
 * (64 MiB) that every device context loading the library holds until the
 * process exits.  A call needs 2 N + n_r^2 + n_z^2 + n_theta^2 doubles of it
 * (N = n_r n_z n_theta; e.g. 160^3 fits, 170^3 does not); larger problems
 * return CYL_EINVAL and launch nothing.  The first call in each CUDA context
 * looks up the array's device address (cudaGetSymbolAddress, with the device
 * current) and caches it under the context's unique ID; after
 * cudaDeviceReset the device's new context gets its own lookup on the next
 * call.  Every call uses the same array and fully rewrites what it reads, so
 * nothing needs clearing between calls, but calls whose kernels overlap on
 * the GPU (different streams, or different host threads) race on the array
 * and give wrong results: serialise them.  A launch error left pending by the
 * caller's earlier work is returned as CYL_ECUDA before anything is
 * launched.  Calls no cudaMalloc or cudaFree.
 */
#define CYL_NOALLOC_SCRATCH_DOUBLES (1 << 23)
cyl_status cyl_vals2coeffs_noalloc(int n_r, int n_z, int n_theta, const double *vals, double *coeffs,
                                   void *stream);

/*
 * cyl_ns_step -- nsteps time steps of the incompressible Navier-Stokes
 * equations in vorticity form (Section 4, eq. ns) on the poloidal-toroidal
 * (PT) decomposition (eq. pt) of the vorticity, omega = curl(lam_w z) +
 * curl curl(gam_w z), Re = 1 / alpha of the plan.  Each step: lambda_v =
 * gam_w and -lap gamma_v = lam_w (eq. ptcurl, one Poisson solve); v and
 * omega on the grid (eq. pt; derivatives on coefficients, the factors 1/r on
 * grid values); N = v x omega pointwise; the PT decomposition (lambda_a,
 * gamma_a) of curl N from eq. ptpoisson (right sides z . curl N and
 * z . curl curl N, two horizontal Poisson solves); then eq. NSrewrite by the
 * first-order implicit-explicit BDF: one BDF1 heat step each for lam_w and
 * gam_w with forcing lambda_a, gamma_a.  Boundary data (reading of the
 * unstated no-slip conditions): homogeneous Dirichlet in every scalar solve
 * (gamma_v on the whole wall, gamma_a and lambda_a at r = +-1, lam_w, gam_w
 * on the whole wall).
 *
 *   plan       from cyl_plan with CYL_WITH_POISSON | CYL_WITH_HEAT |
 *              CYL_WITH_DISK, alpha = 1 / Re, dt the step; n_r even (no grid
 *              point on the axis, where the factors 1/r are applied).
 *   lam_w, gam_w  device coefficient arrays of N float64 (in / out).
 *   workspace  caller-owned device memory of cyl_ns_workspace bytes.
 *
 * CYL_ESTATE when the plan lacks one of the three solvers, CYL_EINVAL for an
 * odd n_r, a short workspace or NULL pointers.  Asynchronous on the plan's
 * stream; allocates nothing.
 */
cyl_status cyl_ns_workspace(cyl_plan_t plan, size_t *bytes);
cyl_status cyl_ns_step(cyl_plan_t plan, double *lam_w, double *gam_w, int nsteps, void *workspace,
                       size_t workspace_bytes);

/*
 * cyl_xform_table -- host copy of the table block of one chirp-z line
 * transform (Section 2: the DCT-I in r and z, the DFT in theta), as the
 * plans build it.  kind: 0 = DCT-I forward, 1 = DCT-I inverse (L = number of
 * Chebyshev points, 2..4096), 2 = DFT forward to half-complex, 3 = DFT
 * inverse (L = n_theta, even, 2..4096).  info (11 ints, host): FFT length
 * P, log2 P, input count A, output count B, first input index, first output
 * index, offsets (doubles) of the pre-multipliers (A complex), the
 * post-multipliers (B complex), the bit-reversed kernel spectrum scaled by
 * 1/P (P complex), the FFT twiddles exp(-2 pi i k / P), k < P/2 (P/2
 * complex), and the block's total length.  table: host array of that length,
 * or NULL to query.  No device access.  CYL_EINVAL for bad arguments.
 */
cyl_status cyl_xform_table(int kind, int L, int *info, double *table);

/* Human-readable name of a status code (static string). */
const char *cyl_status_string(cyl_status s);

/*
 * cyl_fp64_fma_probe -- measurement of the machine, not of the method (the
 * paper has no counterpart): the FP64 fused multiply-add throughput that the
 * FP64 roofline of the ADI kernels divides by.  Launches blocks x threads
 * threads on `stream`, each running 8 independent FMA chains for `iters`
 * iterations, and stores in *flops (host) the launch's FP64 flops (2 per
 * FMA).  The caller times the launch (CUDA events on `stream`) and divides.
 *
 *   blocks >= 1; threads a multiple of 32 in 32..1024; iters >= 1.
 *   sink   device array of blocks*threads float64; never written for the
 *          probe's arguments, it only keeps the chains from being removed.
 *
 * CYL_EINVAL for bad arguments, CYL_ECUDA when the launch fails.  Allocates
 * nothing.
 */
cyl_status cyl_fp64_fma_probe(int blocks, int threads, long long iters, double *sink, double *flops,
                              void *stream);

/* ---------------------------------------------------------------------------
 * Host-side introspection (no device access; valid on CYL_HOST_ONLY plans).
 * ------------------------------------------------------------------------- */

/* which: 0 = Poisson, b = 1..4 = the BDF b step (1 = the BDF1 heat step;
 * 2..4 only on plans from cyl_plan_bdf).  k = |wavenumber| in 0 .. n_theta/2;
 * parity = radial parity block (0 or 1).
 * Returns J and, when the pointers are non-NULL, the spectral interval
 * [a, b] of the radial pencil, [c, d] of the vertical pencil (Section 3, the
 * intervals below Algorithm 1) and the J shift pairs: p_shift[j] (used in
 * the radial solve, lies in [c, d]) and q_shift[j] (used in the vertical
 * solve, lies in [a, b]).  p_shift / q_shift must hold J doubles; call once
 * with NULL to learn J. */
cyl_status cyl_plan_shifts(cyl_plan_t plan, int which, int k, int parity, int *J,
                           double *interval4, double *p_shift, double *q_shift);

/* Copy the parity block (class index rows/cols) of one plan operator to a
 * dense row-major host array.  op: 0 = A (radial, per k), 1 = C (radial),
 * 2 = B (vertical), 3 = D (vertical); which as above; parity selects the
 * radial (op 0, 1) or vertical (op 2, 3) parity class.  *dim receives the
 * block size; out (dim*dim doubles) may be NULL to query the size. */
cyl_status cyl_plan_operator(cyl_plan_t plan, int op, int which, int k, int parity, int *dim,
                             double *out);

/* Launch layout of one kind's ADI kernel (which as above; plans only, not
 * batch plans: CYL_ESTATE).  info[9] receives {items, threads per CTA,
 * twisted half (threads per side of a twisted solve, 0: one-sided sweeps),
 * placement (2: iterate and right side in shared memory, 1: iterate only,
 * 0: both in the per-item global work area), dynamic shared memory bytes,
 * CTAs per item (1, or the cluster size in cluster mode), slices per item
 * (the largest), built (0 when the kind was not built), all twisted (1 when
 * every item's forward solves are twisted both ways: with the work arrays in
 * global memory the launch then uses a kernel compiled without the
 * one-sided sweeps)}.  Items whose two
 * slices leave shared memory are split into single-slice items with twisted
 * solves on two threads per chain (up to 2 x 256 threads), unless
 * CYL_PLAIN_SWEEPS or cluster mode is given. */
cyl_status cyl_plan_launch_info(cyl_plan_t plan, int which, int *info);

/* Host copy of one work item's factor records for ADI iteration j (the
 * tables the kernels read; layout in the library's plan header: radial
 * records of 12 doubles per class row, vertical records of 8 per class
 * column, plus the interface maps of twisted solves).  transposed = 1 gives
 * the records of the transposed system A^T X B + C^T X D = E the adjoint
 * kernels solve (heat kinds only, else CYL_ESTATE): the records, in the
 * forward layout, of the flipped transposes J A^T J, J C^T J, J B^T J,
 * J D^T J (J reverses the index order), which solve the transposed system
 * on index-reversed arrays; twisted where the forward records are, except in
 * cluster plans.  info[8] receives {M, Nz, J, twr, twz, k, parity_r,
 * parity_z}; twr / twz are the split rows of the requested records' twisted
 * radial / vertical solves (0: plain LU sweep).  radial needs M*12 + (twr ?
 * 24 : 0) doubles, vertical Nz*8 + (twz ? 16 : 0); either may be NULL.  Items
 * are numbered as the plan lists them (which as above). */
cyl_status cyl_plan_item_tables(cyl_plan_t plan, int which, int item, int j, int transposed, int *info,
                                double *radial, double *vertical);

/* Grid of Definition "grid" (Section 2) into caller-owned HOST arrays:
 * r[m] = cos((m-1-j) pi / (m-1)), z[n] likewise, theta[p] = (2l - p) pi / p.
 * Any pointer may be NULL. */
cyl_status cyl_grid(cyl_plan_t plan, double *r, double *z, double *theta);

/* Algorithmic FP64 flops of nsteps steps of the fused ADI kernel (which: 0
 * Poisson, b heat BDF b; transposed: 0 forward, 1 adjoint), counting 2 per fused
 * multiply-add: the right side (3 + 5 per element), Algorithm 1 (radial
 * sweep 12 and vertical sweep 8 per element and iteration, minus the radial
 * apply of the first and the vertical apply of the last iteration) and the
 * Dirichlet expansion.  Host only; valid for batch plans (which = 1). */
cyl_status cyl_plan_flops(cyl_plan_t plan, int which, int nsteps, int transposed, double *flops);

/* Complete elliptic integral K as a function of the complementary modulus
 * k' (so that k = sqrt(1 - k'^2) never loses precision), and the Jacobi
 * function dn(u | k) with the same argument convention (DLMF 19.8, 22.20). */
double cyl_ellip_K(double kprime);
double cyl_jacobi_dn(double u, double kprime);

#ifdef __cplusplus
}
#endif

#endif /* CYL_H */
