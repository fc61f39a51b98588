/*
 * lbm.h -- C ABI of the GB300 (sm_103a) axisymmetric MRT lattice Boltzmann solver
 * for thermal flow in porous media at the REV scale (Liu, He & Li, arXiv 1409.5929).
 *
 * The paper states its problem (Sec. 4.2-4.4, Fig. 3) as: a vertical annulus
 * r_i <= r <= r_o, 0 <= z <= H, filled with a porous medium of porosity phi
 * (Eq. 8); parameters Ra, Da, Pr, J, lambda, F_phi (Eq. 9); a hot inner wall, a cold
 * outer wall, adiabatic top and bottom, no slip; fluid initially at rest; the
 * average Nusselt numbers of Eq. 42 as the result.  This interface follows that
 * statement: create a problem, give it a porosity field, step it, read the fields,
 * the Nusselt numbers and the convergence residual.
 *
 * One time step (Sec. 3.1-3.2) at every node is: pull streaming (Eq. 22, 33);
 * non-equilibrium extrapolation at wall nodes (Sec. 4, ref. [47]); T (Eq. 38),
 * rho (Eq. 26), u from the quadratic drag relation (Eq. 28-30); body force
 * (Eq. 6-7), axisymmetric force a_r (Eq. 25) and moment-space source (Eq. 24);
 * MRT relaxation in moment space (Eq. 21, 23) and f+ = M^-1 m+ (Eq. 22); the D2Q5
 * temperature update with its axisymmetric source (Eq. 33-37).
 *
 * Grid and units (lattice units, delta_t = delta_r = 1, c = 1, rho0 = 1):
 *   nodes (kr, kz), 0 <= kr < nr, 0 <= kz < nz; z is the fastest index of every
 *   nr*nz array this interface reads or writes (row-major [kr][kz]).
 *   Annulus: walls are the outermost nodes; L = nr - 1, H = nz - 1,
 *   r_i = L / (R* - 1), r(kr) = r_i + kr.  Corners belong to the side walls.
 *   Pipe (periodic z): the axis lies half a cell below row 0, r(kr) = kr + 1/2,
 *   row nr - 1 is the no-slip wall, L = nr - 1/2.
 *
 * Conventions for every entry point:
 *   - Returns LBM_OK (0) or a positive LBM_ERR_* code; lbm_last_error() then gives
 *     a message (thread-local, valid until the next call on that thread).
 *   - No exception or longjmp crosses the interface.
 *   - A handle owns all its device memory; it is not thread-safe (one thread at a
 *     time per handle).  Input arrays are copied; the caller keeps ownership of
 *     every pointer it passes.
 *   - Device work is queued on the handle's stream (lbm_set_stream); calls that
 *     return host data synchronise that stream.
 *   - on_device = 1: the pointer is CUDA device memory on the handle's device;
 *     on_device = 0: ordinary (or pinned) host memory.
 */
#ifndef LBM_H
#define LBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define LBM_OK 0
#define LBM_ERR_INVALID 1   /* bad argument or parameter (tau <= 1/2, phi outside (0, 1], ...) */
#define LBM_ERR_CUDA 2      /* a CUDA runtime call failed */
#define LBM_ERR_OOM 3       /* device or pinned host allocation failed */
#define LBM_ERR_DIVERGED 4  /* NaN or Inf found in the fields */
#define LBM_ERR_TIMEOUT 5   /* a bounded device wait ran out */

/* geometry */
#define LBM_ANNULUS 0             /* Fig. 3: walls on all four sides */
#define LBM_ANNULUS_PERIODIC_Z 1  /* side walls only, periodic in z */
#define LBM_PIPE_PERIODIC_Z 2     /* axis (specular image row) + outer wall, periodic in z */
#define LBM_PIPE_INFLOW 3         /* Fig. 1 (Sec. 4.1): axis + wall (T_cold), inlet row z = 0
                                     (u = (0, u_in), T_hot), outlet row z = H (zero gradient of u
                                     and T, density held at 1); inlet and outlet own their corners */

/* collision of the flow populations */
#define LBM_MRT 0
#define LBM_BGK 1

/* storage type of the distributions between steps (arithmetic is always FP32) */
#define LBM_F32 0
#define LBM_F16 1
#define LBM_BF16 2

/* node classes written by lbm_node_class */
#define LBM_FLUID 0
#define LBM_WALL_IN 1
#define LBM_WALL_OUT 2
#define LBM_BOTTOM 3
#define LBM_TOP 4
#define LBM_AXIS 5
#define LBM_INLET 6
#define LBM_OUTLET 7

typedef struct lbm_params {
    int32_t nr, nz;          /* grid; both >= 3 */
    int32_t geometry;        /* LBM_ANNULUS, LBM_ANNULUS_PERIODIC_Z, LBM_PIPE_PERIODIC_Z, LBM_PIPE_INFLOW */
    int32_t storage;         /* LBM_F32, LBM_F16, LBM_BF16 */
    double radius_ratio;     /* R* = r_o / r_i > 1 (annulus geometries) */
    double Ra, Da, Pr, J, lambda;  /* Eq. 9; the paper uses J = lambda = 1 (Sec. 4) */
    double Ma;               /* Mach number of Eq. 39 (0.1 in the paper); unused if tau_nu > 0 */
    double tau_nu;           /* > 0: viscous relaxation time given; <= 0: from Eq. 39 */
    double F_eps;            /* < 0: Ergun F_phi per node (Eq. 8); 0: no Forchheimer drag; > 0: constant */
    double eps_mean;         /* porosity that, with Da, fixes the particle diameter of Eq. 8;
                                1 = no solid matrix (K = Da L^2 everywhere) */
    double T_hot, T_cold;    /* inner and outer wall temperatures (pipe with inlet: inlet and wall
                                temperatures); T0 = (T_hot + T_cold) / 2 */
    double body_accel_z;     /* z component of the external acceleration a of Eq. 7 */
    double init_noise;       /* cold start: T = T0 + init_noise * U(-1, 1) on non-wall nodes */
    uint64_t seed;           /* SplitMix64 seed of that noise (draw number kr*nz + kz) */
    double u_in;             /* LBM_PIPE_INFLOW: inlet velocity U_in (Re = r_i U_in / nu, Sec. 4.1),
                                0 <= u_in < 1/2 (lattice units; a low-Mach model wants u_in << c_s) */
    double heater_len;       /* annulus geometries: > 0 puts an isoflux discrete heater of length
                                heater_len * H on the inner wall (Sec. 4.4, Fig. 7) with
                                q' L / k = T_hot - T_cold, insulates the rest of the inner wall
                                and sets T0 = T_cold; 0: inner wall held at T_hot */
    double heater_center;    /* heater centre h / H in [0, 1] (node kz is heated when
                                |kz - h H| <= l H / 2); heater_len <= 1 */
    int32_t collision;       /* LBM_MRT (Eq. 21 with the rates of Sec. 4) or LBM_BGK (every rate
                                1/tau_nu: the BGK limit of Sec. 3.1) */
    int32_t inplace;         /* 0: two state buffers (A/B, read one, write the other);
                                1: one state buffer updated in place (AA pattern: the
                                populations alternate between two layouts from step to
                                step), half the state memory for the same bytes per
                                step; lbm_create only (lbm_batch_create rejects it),
                                lbm_residual then returns LBM_ERR_INVALID (no previous
                                state is kept; lbm_run works); one node per thread for
                                every storage type */
} lbm_params;

/* Derived lattice constants (Eq. 9, 31, 39), for checks and reporting. */
typedef struct lbm_info {
    double L, H, r0;         /* characteristic length, height, r(kr = 0) */
    double tau_nu, tau_T;    /* relaxation times (Eq. 39) */
    double nu_e, nu;         /* effective and fluid kinematic viscosity (Eq. 31, J) */
    double gbeta;            /* g * beta from U = Ma c_s = sqrt(g beta dT L) */
    double T0;               /* reference temperature */
    double Ma;
    double Kbar;             /* Da * L^2 */
    int64_t steps;           /* steps taken since the last (re)initialisation */
    int64_t bytes_per_step;  /* algorithmic HBM bytes of one step: read + write of every
                                population, one FP32 porosity, the FP16 temperature
                                reference and (16-bit storage) the 4 x FP16 flow
                                reference (lbm_rebase) read per node */
} lbm_info;

typedef struct lbm_handle lbm_handle;

/* Fill *p with the porous-annulus defaults (48 x 96, R* = 2, eps = 0.6, Da = 1e-2,
 * Ra = 1e3, Pr = 1, J = lambda = 1, Ma = 0.1, Ergun F_eps, T_hot = 1, T_cold = 0,
 * noise 1e-3, seed 1, FP32 storage, no discrete heater, heater centre 0.5). */
void lbm_params_default(lbm_params *p);

/* Validate *p and derive the lattice constants without touching a GPU. */
int lbm_derive(const lbm_params *p, lbm_info *out);

/* Allocate a problem on the current CUDA device: two state buffers (A/B),
 * the porosity field (uniform eps_mean) and scratch; cold start (rho = 1, u = 0,
 * noisy T).  *out receives the handle.  LBM_ERR_OOM if memory runs out. */
int lbm_create(const lbm_params *p, lbm_handle **out);

/* Queue all further device work of h on `stream` (a cudaStream_t, e.g. from
 * torch.cuda.Stream.cuda_stream); NULL = the legacy default stream.  Work queued on the
 * new stream starts after the work already queued on the old one. */
int lbm_set_stream(lbm_handle *h, void *stream);

/* Replace the porosity field by phi[nr*nz] (each value in (0, 1]).  Takes effect
 * from the next step; the state is not re-initialised (call lbm_init_fields). */
int lbm_set_porosity(lbm_handle *h, const float *phi, int on_device);

/* Storage detail with no counterpart in the paper: the porosity upload of lbm_set_porosity
 * without its synchronisation.  phi (nr*nz floats, host memory; pinned memory lets the
 * copy run asynchronously) is copied on a copy stream of the handle into one of two
 * alternating staging buffers.  The next call that reads the field (a step, the fields,
 * the residual, a re-initialisation) converts it on the handle's stream, after the work
 * queued before it: steps queued before this call see the old field, and the copy overlaps
 * them and any call that does not read the field (the Nusselt numbers of Eq. 42).  An
 * upload that no reader has seen is replaced by the next one.  phi must stay unchanged until
 * a synchronising call that follows the next reader of the field (or lbm_destroy).  Values
 * outside (0, 1] are counted when the field is converted, not rejected: lbm_porosity_errors
 * reports them.  Returns at once. */
int lbm_set_porosity_async(lbm_handle *h, const float *phi);

/* Number of porosity values outside (0, 1] seen by lbm_set_porosity_async since the last
 * clear (clear = 1 resets the count).  Synchronises. */
int lbm_porosity_errors(lbm_handle *h, uint32_t *count, int clear);

/* (Re)initialise the state from the fields (u_r, u_z, T), each nr*nz, or pass three
 * NULLs for the cold start.  The populations are f = M^-1(m_eq - S/2) (Eq. 19-20,
 * 24, so that Eq. 29 returns the given u at rest), g = g_eq(T, u) (Eq. 35), after
 * one collision; wall nodes take u = 0 and their wall temperature.  Resets the
 * step count. */
int lbm_init_fields(lbm_handle *h, const float *ur, const float *uz, const float *T, int on_device);

/* Advance nsteps >= 0 time steps (asynchronous on the handle's stream). */
int lbm_step(lbm_handle *h, int64_t nsteps);

/* Fields of the current state (what the next step's pull sees, after the wall
 * rebuild) into caller-owned float arrays of nr*nz: rho (Eq. 26), u_r, u_z
 * (Eq. 28; 0 on walls), T (Eq. 38; the wall temperature on walls).  Any pointer
 * may be NULL.  Synchronises when on_device = 0. */
int lbm_moments(lbm_handle *h, float *rho, float *ur, float *uz, float *T, int on_device);

/* Average Nusselt numbers of Eq. 42 on the inner and outer wall of the current
 * state: one-sided second-order dT/dr at the wall, trapezoid rule over the nz wall
 * nodes, H = nz - 1, dT = T_hot - T_cold.  FP64 reduction.  Synchronises.  The
 * inner value is NaN for the pipes; both are NaN for LBM_PIPE_INFLOW (lbm_pipe_nusselt)
 * and with the discrete heater (lbm_heater_nusselt). */
int lbm_nusselt(lbm_handle *h, double *nu_inner, double *nu_outer);

/* lbm_nusselt without the synchronisation: enqueues the reduction of the current state
 * and the transfer of (Nu_inner, Nu_outer) into out[0..1] (host memory) on the handle's
 * stream and returns.  Pinned (page-locked, mapped) memory is written by the device
 * directly; other host memory takes an ordinary copy.  out must stay allocated until the values are there,
 * after the next synchronising call (lbm_sync).  NaN entries as for lbm_nusselt. */
int lbm_nusselt_async(lbm_handle *h, double *out);

/* Wait for all work queued on the handle (its compute and copy streams). */
int lbm_sync(lbm_handle *h);

/* Discrete heater (heater_len > 0) only: Eq. 44 at every heated inner-wall node,
 * Nu(z) = q' L / (k (T_h - T_o)) = (T_hot - T_cold) / (T_h(z) - T_cold), and its mean
 * over the heater (Eq. 43, heated nodes weighted equally) into *nu_mean.  nu_z (may be
 * NULL) receives nz values, NaN off the heater.  The heater wall temperature solves the
 * one-sided second-order difference of q' = -k dT/dr with the next two nodes inward.
 * FP64.  Synchronises. */
int lbm_heater_nusselt(lbm_handle *h, double *nu_mean, double *nu_z);

/* LBM_PIPE_INFLOW only: local wall Nusselt number of Eq. 40 at every column,
 * Nu(z) = D (dT/dr)_w / (T_w - T_b), D = 2 r_i, into nu[0 .. nz-1] (host memory).
 * T_b is the mixing-cup temperature int u_z r T dr / int u_z r dr: Eq. 41 as printed
 * leaves out u_z, which would put the no-porous pipe at Nu = 5.3 instead of the 3.674
 * of Table 1.  Trapezoid rule on r = 0, 1/2, 3/2, ..., r_i; (dT/dr)_w one-sided,
 * second order.  FP64.  The inlet column gives NaN (T_w = T_b there).  Synchronises. */
int lbm_pipe_nusselt(lbm_handle *h, double *nu, int32_t nz);

/* Stokes stream function of the current state (Table 3 lists its largest magnitude,
 * |psi|max, without defining psi; this is the standard form for the continuity
 * equation Eq. 1): r u_z = d psi/dr, r u_r = -d psi/dz, i.e.
 *   psi(r, z) = integral of r' u_z(r', z) dr' from r_s to r,
 * with r_s the inner wall (annulus; psi = 0 there) or the axis (pipes; the first
 * trapezoid panel runs from r = 0 to the first row at r = 1/2).  Trapezoid rule over
 * the rows, FP64 accumulation, lattice units (divide by alpha L or nu L for the
 * dimensionless forms).  psi (may be NULL): nr*nz floats, z fastest, in device memory
 * when on_device != 0, else host memory; *psi_max (may be NULL) receives max |psi|
 * over the grid.  Synchronises. */
int lbm_stream_function(lbm_handle *h, float *psi, int on_device, double *psi_max);

/* Convergence residual between the current state n and the previous state n - 1:
 * max(|u^n - u^(n-1)|_2 / |u^n|_2, |T^n - T^(n-1)|_2 / |T^n|_2) over non-wall
 * nodes, and the mass sum over all nodes of r * rho (= sum_i f_i), both in FP64.
 * Needs at least one step since initialisation (LBM_ERR_INVALID otherwise).
 * Returns LBM_ERR_DIVERGED if a field holds NaN or Inf.  Synchronises. */
int lbm_residual(lbm_handle *h, double *res, double *mass);

/* Step until steady or max_steps.  Every check_every steps the mean change per step
 * over the interval, max(|u^n - u^(n-k)|_2 / |u^n|_2, |T^n - T^(n-k)|_2 / |T^n|_2) / k
 * over non-wall nodes (FP64), is compared with tol; it averages out the rounding
 * jitter of an FP32 or 16-bit state, which keeps the consecutive-step residual of
 * lbm_residual near 1e-8 - 1e-7 however long the run.  Before every interval the
 * temperature reference is refreshed (lbm_rebase).  *steps_done and *res (either
 * may be NULL) receive the steps taken and the last value.  LBM_ERR_DIVERGED on
 * NaN/Inf.  Synchronises at every check. */
int lbm_run(lbm_handle *h, int64_t max_steps, int64_t check_every, double tol, int64_t *steps_done,
            double *res);

/* Storage detail with no counterpart in the paper.  The thermal populations are
 * stored as deviations from w_i (T0 + R(x)), R(x) a per-node FP16 offset set from the
 * start temperature; this call sets R(x) to the current T(x) - T0 (rounded to FP16)
 * and re-expresses the stored deviations against it.  With 16-bit storage the flow
 * populations are likewise stored against a per-node reference equilibrium (the
 * deviation part of Eq. 32's f_eq from a per-node FP16 quad: r (rho - 1), r rho u and
 * 1 / (r rho phi)), which this call refreshes in the same pass.  Every field and
 * population is unchanged up to the storage rounding of the re-encoded values; what
 * changes is the size of the stored numbers, and so the rounding of later steps:
 * without refreshes, FP32 rounding stops slow thermal modes once their change per step
 * drops below the rounding of |T - T0 - R| (a spread of about 1e-3 in Nu on slowly
 * converging annuli), and 16-bit rounding of deviations from the rest state jitters the
 * flow by about 4e-4 per step.  lbm_run refreshes before every check interval; with
 * 16-bit storage lbm_step also refreshes every 1024 steps since the last refresh.
 * With in-place storage after an odd number of steps, boundary nodes whose outgoing
 * populations that layout drops (they leave the domain) keep their old references.
 * Asynchronous on the handle's stream. */
int lbm_rebase(lbm_handle *h);

/* Node classes (LBM_FLUID ... LBM_AXIS) into out[nr*nz] (host memory). */
int lbm_node_class(lbm_handle *h, uint8_t *out);

/* Export the current state's post-collision populations of rows
 * [row0, row0 + nrows) in FP64, undoing the storage encoding: f[i][row][kz]
 * (9 planes of nrows*nz) and g[i][row][kz] (5 planes), host memory, r-weighted
 * as in Eq. 17.  For checks against an FP64 reference and for inspection.
 * With in-place storage after an odd number of steps, populations that leave the
 * domain from boundary nodes are not kept and export as NaN (no step reads them).
 * Synchronises. */
int lbm_export_populations(lbm_handle *h, int32_t row0, int32_t nrows, double *f, double *g);

/* Derived constants and step count of h. */
int lbm_get_info(lbm_handle *h, lbm_info *out);

/* Bounded waits of the staged 16-bit bulk kernel (not an operation of the paper).  With
 * 16-bit storage, even nz and grids of at least 16 blocks per SM, the bulk step copies
 * each row's source segments into shared memory with bulk copies whose completion every
 * thread awaits for at most `rounds` polls (default a few seconds).
 * A wait that runs out marks the handle: the block drains its copies in flight and
 * stops, so that step's results are invalid.  lbm_wait_status synchronises the handle's
 * stream and returns LBM_ERR_TIMEOUT if any wait ran out since the last clear (clear = 1
 * resets the mark), else LBM_OK; lbm_run checks it at every residual check.
 * lbm_set_wait_limit sets `rounds` (< 0: the default; 0 makes every wait run out at
 * once, for tests of the error path). */
int lbm_set_wait_limit(lbm_handle *h, int rounds);
int lbm_wait_status(lbm_handle *h, int clear);
/* enable = 0 runs the 16-bit bulk step on global loads everywhere (the update and its
 * arithmetic are the same; the staged kernel only moves the loads); 1 (default) stages
 * where it applies. */
int lbm_set_staging(lbm_handle *h, int enable);

/* Per-launch timing of the step kernels with CUDA events on the handle's stream.
 * enable = 1 starts recording (and clears the totals), 0 stops.  lbm_kernel_times
 * synchronises and returns the summed milliseconds and launch counts of the bulk
 * step kernel and of the wall-node kernel since timing was enabled. */
int lbm_set_timing(lbm_handle *h, int enable);
int lbm_kernel_times(lbm_handle *h, double *bulk_ms, int64_t *bulk_launches, double *wall_ms,
                     int64_t *wall_launches);

/* Allocation-free residual (the paper has no counterpart: this is a service for
 * callers that cannot allocate device memory when they need the check, e.g. a host
 * framework whose own allocator owns all device memory, or a monitoring path that
 * must not trigger the device-wide synchronisation cudaMalloc / cudaFree can cause).
 * Same result as lbm_residual, computed from two field snapshots the caller supplies:
 *   cur:  device floats, 4 planes of nr*nz at stride field_stride: rho, u_r, u_z, T
 *         of state n (the layout lbm_moments writes when given plane pointers);
 *   prev: the same 4 planes of state n - 1 (its rho plane is not read);
 *   each must point into device (or managed) memory of the current device whose
 *   allocation holds 3*field_stride + nr*nz floats from the pointer on; a host pointer,
 *   another device's memory or a shorter allocation is rejected with LBM_ERR_INVALID
 *   before anything is launched (cudaPointerGetAttributes and the driver's
 *   cuMemGetAddressRange, neither of which allocates; the extent check is skipped if
 *   the driver does not offer that call);
 *   geometry, nr, nz: as in lbm_params; r0 = r(kr = 0) (lbm_info.r0);
 *   *res, *mass: host doubles receiving the residual and sum of r * rho (FP64).
 * It calls no cudaMalloc, cudaFree or other allocating routine: the reduction's
 * partial sums live in a file-scope static device array of 1025 x 6 doubles (49 KB),
 * held by every GPU that loads the library until the process exits.  Every call looks
 * up that array's address in the current device's context (cudaGetSymbolAddress); the
 * first call on a device may also load the library's device code there, so make that
 * first call before any stream capture.  All calls share the array and each overwrites
 * it: calls that overlap on the GPU (other streams, other threads) race.  Limits:
 * 3 <= nr, nz <= 65535 and nr*nz < 2^31, nr*nz <= field_stride <= 2^40 (LBM_ERR_INVALID
 * beyond).  Work runs on `stream` (NULL = legacy default) and the call synchronises it.
 * LBM_ERR_DIVERGED if cur holds NaN or Inf. */
int lbm_field_residual_noalloc(int32_t geometry, int32_t nr, int32_t nz, double r0, const float *cur,
                               const float *prev, int64_t field_stride, double *res, double *mass,
                               void *stream);

/* ------------------------------------------------------------------ batches --
 * Many independent problems of uneven size advanced by the same kernel launches.
 * Every step of every active instance is the step of lbm_step (same kernels, same
 * arithmetic); the batch only shares launches, a CUDA graph and the checks.  All
 * instances must use the same storage type.  Instance indices are 0 .. n-1.  The
 * batch owns one stream (lbm_batch_set_stream replaces it; the legacy default stream
 * cannot be captured and is rejected).  Not thread-safe. */
typedef struct lbm_batch lbm_batch;

/* Allocate and cold-start n instances with parameters p[0..n-1] (validated as in
 * lbm_create); each gets uniform porosity eps_mean. */
int lbm_batch_create(const lbm_params *p, int32_t n, lbm_batch **out);
int lbm_batch_set_stream(lbm_batch *b, void *stream);
/* Porosity field of instance i (nr_i * nz_i values in (0, 1], copied). */
int lbm_batch_set_porosity(lbm_batch *b, int32_t i, const float *phi, int on_device);
/* (Re)initialise instance i as lbm_init_fields does; a stopped instance becomes
 * active again. */
int lbm_batch_init_fields(lbm_batch *b, int32_t i, const float *ur, const float *uz, const float *T, int on_device);
/* nsteps steps of every active instance (two launches per step for the whole batch). */
int lbm_batch_step(lbm_batch *b, int64_t nsteps);
/* Step until every instance is steady (criterion of lbm_run, per instance, checked
 * every check_every steps; check_every must be even) or max_steps.  The steps of one
 * check interval are captured once in a CUDA graph and replayed; instances that meet
 * tol stop stepping.  steps[n], res[n] (either may be NULL) receive the steps each
 * instance took and its last criterion value.  LBM_ERR_DIVERGED names an instance that
 * produced NaN or Inf (it is stopped; the others have run to that check). */
int lbm_batch_run(lbm_batch *b, int64_t max_steps, int64_t check_every, double tol, int64_t *steps, double *res);
/* lbm_rebase for every instance (lbm_batch_run refreshes the active instances before
 * every check interval).  Asynchronous on the batch's stream. */
int lbm_batch_rebase(lbm_batch *b);
/* Eq. 42 of every instance: nu_inner[n], nu_outer[n] (host). */
int lbm_batch_nusselt(lbm_batch *b, double *nu_inner, double *nu_outer);
/* Fields of instance i, as lbm_moments. */
int lbm_batch_moments(lbm_batch *b, int32_t i, float *rho, float *ur, float *uz, float *T, int on_device);
/* lbm_pipe_nusselt of instance i (LBM_PIPE_INFLOW), nu[0 .. nz-1] in host memory.
 * Synchronises. */
int lbm_batch_pipe_nusselt(lbm_batch *b, int32_t i, double *nu, int32_t nz);
/* Autotuner: times `steps` steps for each bulk tile shape (columns x rows per block x
 * rows per thread; twelve shapes of at most 256 threads) and keeps the fastest; *cols and
 * *rows receive the tile's columns and rows, *ms_per_step its time per step.  The state
 * advances by the steps the tuning ran (2 warm-up steps + `steps` per shape; the batch's
 * step count in lbm_batch_get_info includes them). */
int lbm_batch_tune(lbm_batch *b, int32_t steps, int32_t *cols, int32_t *rows, float *ms_per_step);
/* lbm_set_wait_limit and lbm_wait_status for the batch's staged 16-bit bulk kernel
 * (instances with even nz; the tuned tile shape then serves the odd-nz instances and the
 * reference refresh).  lbm_batch_run checks the status after every check interval. */
int lbm_batch_set_wait_limit(lbm_batch *b, int rounds);
int lbm_batch_wait_status(lbm_batch *b, int clear);
int lbm_batch_set_staging(lbm_batch *b, int enable);
/* Derived constants of instance i; steps = steps taken by the batch. */
int lbm_batch_get_info(lbm_batch *b, int32_t i, lbm_info *out);
int lbm_batch_destroy(lbm_batch *b);

/* Free everything h owns.  h may be NULL. */
int lbm_destroy(lbm_handle *h);

/* Message of the last failed call on this thread ("" if none). */
const char *lbm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
