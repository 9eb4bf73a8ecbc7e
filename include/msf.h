/*
 * msf.h -- C ABI of the GB300 (sm_103a) implementation of the conservative
 * sharp-interface method for compressible multi-material flows of
 * Pan, Han, Hu & Adams (arXiv:1704.00519).
 *
 * One context owns one CUDA device's worth of state for n_instances
 * independent problems on uniform Cartesian grids (1D, 2D or 3D) with up to
 * MSF_MAXMAT materials, each a stiffened gas. Every call returns an
 * msf_status; nothing aborts, exits or throws across this boundary. Pointer
 * arguments are plain host or device pointers as stated per call; the caller
 * keeps ownership of everything it passes in. All arrays are dense, C order,
 * interior cells only, with x the fastest index.
 *
 * Threading: a context is used by one host thread at a time.
 * Streams: work is issued on msf_options.stream (a cudaStream_t, or NULL for
 * the legacy default stream).
 */
#ifndef MSF_H
#define MSF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MSF_MAXMAT 8
#define MSF_NSTATS 8

typedef struct msf_ctx msf_ctx; /* opaque; created by msf_create, freed by msf_destroy */

typedef enum {
  MSF_OK = 0,
  MSF_EINVAL = 1,     /* invalid argument (checked on the host before any launch) */
  MSF_ENOMEM = 2,     /* device allocation failed */
  MSF_ECUDA = 3,      /* a CUDA runtime call failed */
  MSF_ENONFINITE = 4, /* a non-finite conserved value was produced */
  MSF_ENEGATIVE = 5,  /* density <= 0 or p + pinf <= 0 met in a state that was used */
  MSF_EBAND = 6,      /* a flux stencil reached a cell without a state of that material */
  MSF_ETIMEOUT = 7,   /* reserved */
  MSF_ESTATE = 8,     /* context unusable after an earlier device-detected error */
  MSF_EUNSUPPORTED = 9
} msf_status;

typedef enum { MSF_BC_TRANSMISSIVE = 0, MSF_BC_REFLECTIVE = 1, MSF_BC_INFLOW = 2 } msf_bc;
typedef enum { MSF_HOST = 0, MSF_DEVICE = 1 } msf_mem;
typedef enum { MSF_FP64 = 0, MSF_FP32_BULK = 1 } msf_precision;

/* Grid of one instance (Sec. 2.3: uniform Cartesian cells).
 *   dim          1, 2 or 3; n[d] interior cells on axis d (n[d] = 1 for d >= dim)
 *   lo, hi       domain box; h_d = (hi_d - lo_d) / n_d
 *   bc[d][side]  msf_bc for the low (0) and high (1) side of axis d
 *   inflow_prim  primitive (rho, u_0..u_{dim-1}, p) imposed on an inflow side
 *   inflow_mat   material of the inflow state
 *   geom         MSF_GEOM_CARTESIAN (0), or MSF_GEOM_CYLINDRICAL (1): a grid of
 *                one dimension whose x is the radius of an axisymmetric flow
 *                (Sec. 3, Case II; lo[0] >= 0). Cell i has volume r_i h and
 *                its faces areas r_f; the radial momentum gains p alpha / r_i;
 *                totals weight each cell by its volume.
 *   free_surface 0, or 1: material fs_mat is an ambient that is not solved
 *                (Sec. 3, Case II). Its state is held at (fs_rho, 0, p(t)) and
 *                the interfaces of the other materials with it carry the
 *                pressure p(t) = fs_p0 for t <= fs_t0, falling linearly to
 *                fs_p1 at fs_t1 and fs_p1 after; the interface velocity comes
 *                from the two-shock wave curve of the solved side. Requires
 *                fs_rho > 0 and fs_t1 > fs_t0. The tape and adjoint entry points
 *                refuse a grid with geom != 0 or free_surface != 0
 *                (MSF_EUNSUPPORTED). */
typedef struct {
  int32_t dim;
  int32_t n[3];
  double lo[3], hi[3];
  int32_t bc[3][2];
  double inflow_prim[3][2][5];
  int32_t inflow_mat[3][2];
  int32_t geom;
  int32_t free_surface, fs_mat;
  double fs_rho, fs_p0, fs_t0, fs_t1, fs_p1;
} msf_grid;
typedef enum { MSF_GEOM_CARTESIAN = 0, MSF_GEOM_CYLINDRICAL = 1 } msf_geom;

/* Equation of state of one material (Sec. 2.1).
 * kind MSF_EOS_STIFFENED (0): stiffened gas p = (gamma - 1) rho e - gamma pinf
 *   (pinf = 0 is the ideal gas); sound speed c^2 = gamma (p + pinf) / rho.
 * kind MSF_EOS_TAIT (1): Tait's equation p = B (rho/rho0)^gamma - B + p0 with
 *   gamma, tait_B > 0, tait_rho0 > 0, tait_p0 (pinf is ignored). The pressure
 *   does not depend on the internal energy; the energy of a state given by
 *   (rho, u, p) and the sound speed are those of the stiffened gas with
 *   pinf = B - p0, whose isentrope through (rho0, p0) is Tait's curve; in the
 *   HLLC wave speeds (Sec. 2.3.2) Psi = c^2 and Upsilon = 0.
 * The adjoint step and msf_cfl_dt_noalloc take stiffened gases only. */
#define MSF_EOS_STIFFENED 0
#define MSF_EOS_TAIT 1
typedef struct {
  double gamma, pinf;
  int32_t kind;
  double tait_B, tait_rho0, tait_p0;
} msf_eos;

/* Run options. Zero-initialise and call msf_default_options() first.
 *   precision    MSF_FP64: all arithmetic in FP64.
 *                MSF_FP32_BULK: WENO5 fluxes, primitive recovery, ghost states,
 *                HLLC and the CFL bound in FP32; conserved storage, flux
 *                accumulation, geometry, conservation correction, level set,
 *                mixing, scale separation and totals in FP64.
 *   cfl          CFL number (Sec. 3: 0.6)
 *   weno_eps     WENO5 smoothness epsilon (1e-6)
 *   mix_alpha    cells of a material with 0 < alpha < mix_alpha are mixed (0.5)
 *   ext_sweeps   Jacobi sweeps of the ghost-state extension (dim + 3)
 *   vel_sweeps   Jacobi sweeps of the interface-velocity extension (6)
 *   reinit_iters Godunov iterations of the band distance maintenance (6)
 *   scale_sep    1: interface scale separation once per step (Sec. 2.3.3)
 *   reinit       1: distance maintenance once per step
 *   scale_eps_h  epsilon of the scale separation in units of h_min; 0 selects
 *                0.5 (1D), 0.75 (2D), 0.9 (3D) (Sec. 2.3.3)
 *   phi_cap_h    the unsigned distance is clamped at phi_cap_h * h_min (8)
 *   use_graph    1: replay each step as a captured CUDA graph
 *   profile      1: record CUDA events around the flux-update kernel of each
 *                stage (read back with msf_profile_read)
 *   batch_mode   for n_instances > 1 of dimension 1: 0 = one persistent launch
 *                per msf_step call, one CTA per instance (largest first, CTA
 *                size autotuned on the first steps); 1 = the per-instance
 *                kernel sequence of a single instance, instance after instance
 *   stream       cudaStream_t for all work of this context
 *   rk_stages    3: three-stage TVD Runge-Kutta (default); 2: the two-stage
 *                TVD Runge-Kutta the paper uses (Sec. 3), beta_s = (0, 1/2)
 *                in the form of Eq. local-advection
 *   literal_reduced  0 (default): in a cut cell the interface state of the
 *                heaviest pair acts on the boundary of every other present
 *                material m through its area vector S^m (pointing into m),
 *                and the heavier material R of the pair takes minus their
 *                sum (sum_m X^m = 0; with two materials X^R = -X^L exactly as
 *                in Sec. 2.3.2). 1: the reduced model as printed in Sec. 2.3.2,
 *                only the pair exchanges, X^R = [0, p* S^R, p* u* n.S^R],
 *                X^L = -X^R, the other materials get nothing (for comparison:
 *                a resting junction then does not stay at rest)
 *   literal_normal   1: each area vector S^m replaced by |S^m| n^m, the
 *                material's own level-set normal (the printed form of the
 *                exchange flux of Sec. 2.3.2); 0 (default): S^m itself
 *   positivity   1: every face flux is limited towards the first-order
 *                Lax-Friedrichs flux just enough that the density and
 *                p + pinf of the two half states it feeds stay positive
 *                (Hu, Adams & Shu, J. Comput. Phys. 242, 2013), for long runs
 *                that reach near-vacuum states; 0 (default): the plain
 *                WENO5-LLF flux of Sec. 3 (the paper has no positivity
 *                treatment)
 * Tapes and the adjoint step refuse contexts with a literal option or the
 * positivity limiter set (MSF_EUNSUPPORTED). */
typedef struct {
  int32_t precision;
  double cfl, weno_eps, mix_alpha;
  int32_t ext_sweeps, vel_sweeps, reinit_iters;
  int32_t scale_sep, reinit;
  double scale_eps_h, phi_cap_h;
  int32_t use_graph, profile, batch_mode;
  void* stream;
  int32_t rk_stages;
  int32_t literal_reduced, literal_normal;
  int32_t positivity;
} msf_options;

/* Fill opt with the defaults above for a grid of dimension dim. */
msf_status msf_default_options(int32_t dim, msf_options* opt);

/* Create a context for n_instances grids with n_mat materials each.
 *   grids  [n_instances] host array; every instance must have the same dim
 *   eos    [n_instances * n_mat] host array, instance-major
 *   opt    host pointer
 *   out    receives the context
 * Allocates all device memory of the context (freed by msf_destroy).
 * Errors: MSF_EINVAL (bad sizes, n_mat outside [1, MSF_MAXMAT], gamma <= 1,
 * pinf < 0, non-finite box, options out of range), MSF_ENOMEM, MSF_ECUDA. */
msf_status msf_create(const msf_grid* grids, int32_t n_instances, int32_t n_mat, const msf_eos* eos,
                      const msf_options* opt, msf_ctx** out);

/* Free every resource of the context. NULL is accepted. */
msf_status msf_destroy(msf_ctx* ctx);

/* Initial data of one instance (Sec. 2.2: regional level set (phi, chi)).
 *   phi   [cells] unsigned distance to the interface network, phi >= 0
 *   chi   [cells] material indicator in [0, n_mat)
 *   prim  [n_mat][dim + 2][cells] primitive state (rho, u_d, p) of each
 *         material, used where that material has a non-zero sub-volume
 *   mem   MSF_HOST or MSF_DEVICE: where the three arrays live
 * Computes the cut-cell geometry with the conservation correction and sets the
 * conserved state alpha * U of every material; resets t, the ledger and the
 * counters. Errors: MSF_EINVAL for phi < 0 or non-finite, chi out of range,
 * rho <= 0 or p + pinf <= 0 or non-finite prim (host inputs are checked on
 * the host; device inputs on the device before use). */
msf_status msf_set_levelset(msf_ctx* ctx, int32_t instance, const double* phi, const int32_t* chi,
                            const double* prim, int32_t mem);

/* Advance every instance by up to n_steps full TVD-RK3 steps (three stages of
 * Eq. discretized_equ with the beta_s weights of Eq. local-advection), or
 * until t_end: the last time step is clipped so that t lands on t_end; an
 * instance already at t_end does nothing. The time step is
 * cfl / max over the cells of sum_d (|u_d| + c) / h_d over the materials
 * present (Sec. 3), on a grid with a free surface also over |u*| / h of its
 * cut cells (the surface moves at the u* of its wave curve). The stages are
 * those of opt.rk_stages (3, or the 2 of Sec. 3). Work is enqueued on
 * opt.stream.
 * sync = 1: wait and report device-detected errors (MSF_ENONFINITE,
 * MSF_ENEGATIVE, MSF_EBAND); sync = 0: return after enqueueing (errors are
 * reported by the next synchronising call). After a device-detected error the
 * context returns MSF_ESTATE until msf_set_levelset or msf_set_state. */
msf_status msf_step(msf_ctx* ctx, int32_t n_steps, double t_end, int32_t sync);

/* FP64 totals of one instance (Sec. 2.3.1, Eq. sum_equ): totals[m][v] =
 * sum over interior cells of alpha^m U^m_v times the cell volume, and the
 * accumulated net boundary inflow ledger[m][v] of the same quantity, so that
 * totals(t) - totals(0) - ledger(t) vanishes to round-off (per material for
 * mass; summed over materials for momentum and energy, which the interface
 * exchange moves between materials). Host arrays [n_mat][dim + 2]. Synchronises. */
msf_status msf_totals(msf_ctx* ctx, int32_t instance, double* totals, double* ledger);

/* ---------------------------------------------------------------------------
 * Differentiation at frozen interface evolution (single-instance contexts).
 *
 * A tape records one step: the time t and time step dt of the step, the
 * conserved state Q^n, and the level set (phi, chi) after the boundary fill at
 * the start of each of the three stages and after the level-set stage of the
 * last stage. Replaying a tape advances the current conserved state by one
 * step with the interface evolution frozen to the tape: the level set of each
 * stage is the recorded one instead of the advected one (Sec. 2.2), the time
 * step is the recorded one, band maintenance and scale separation are left
 * out, and every discrete choice made from the state (interface pair, the
 * correction's material of Eq. vol_corr2, small cells and mixing targets) is
 * re-made from the replayed state. What the replay computes from the
 * conserved state and the EOS parameters is the flow part of the step
 * (Sec. 2.3: primitive recovery, ghost extension, reduced interface exchange,
 * aperture-weighted WENO5-LLF fluxes, the RK combination of Eq.
 * local-advection, mixing); the adjoint step is its exact reverse-mode
 * derivative (up to the discrete choices, which it holds fixed).
 * Tape memory is device memory owned by the caller, 256-byte aligned, of
 * msf_tape_bytes bytes; a tape is independent of the context that wrote it
 * (a context with the same grid and options but other EOS parameters or
 * inflow states may replay it).
 * ------------------------------------------------------------------------- */

/* Bytes of one tape. MSF_EUNSUPPORTED for several instances. */
msf_status msf_tape_bytes(const msf_ctx* ctx, int64_t* bytes);

/* One full step (as msf_step with n_steps = 1, sync = 1) that also writes its
 * tape. MSF_EINVAL if t >= t_end (no step) or the tape pointer is not aligned. */
msf_status msf_step_taped(msf_ctx* ctx, void* tape, double t_end);

/* One step from the current conserved state (see msf_set_conserved) with the
 * interface evolution frozen to the tape. Sets t = tape t + tape dt; phi and
 * chi end as the tape's level set after the last level-set stage. Synchronises. */
msf_status msf_replay_step(msf_ctx* ctx, const void* tape);

/* Replace the conserved state of the interior cells (SoA [n_mat][dim+2][cells],
 * x fastest; host or device per mem), keeping phi, chi, t, ledger, counters. */
msf_status msf_set_conserved(msf_ctx* ctx, int32_t instance, const double* Q, int32_t mem);

/* Adjoint of the replayed step of a tape: given lam_out = dJ/dQ^{n+1} (device,
 * SoA [n_mat][dim+2][cells] of the interior cells), writes lam_in = dJ/dQ^n
 * (device, same layout; may not alias lam_out) and ADDS dJ/d(gamma_m, pinf_m)
 * to d_eos[m][2] and dJ/d(inflow primitive state) to d_inflow[3][2][5] (host
 * arrays; either may be NULL), for J(Q^{n+1}) and the replay map
 * Q^{n+1}(Q^n, gamma, pinf, inflow). Recomputes the stages from the tape
 * (stage checkpointing), then pulls lam back through mixing, the RK
 * combination, fluxes and exchange, boundary states, stencil states,
 * extension sweeps and primitive recovery of each stage in reverse order.
 * Leaves the context at the tape's starting state (Q^n, phi, chi, t of the
 * tape). Synchronises. Errors: MSF_EINVAL (alignment, empty tape),
 * MSF_EUNSUPPORTED (several instances), device errors as msf_step. */
msf_status msf_adjoint_step(msf_ctx* ctx, const void* tape, const double* lam_out, double* lam_in, double* d_eos,
                            double* d_inflow);

/* Copy one instance's state out (all outputs optional, NULL skips):
 *   Q [n_mat][dim+2][cells] conserved alpha U, alpha [n_mat][cells] volume
 *   fractions of the current geometry, phi [cells], chi [cells], t [1].
 * mem says where Q, alpha, phi and chi live; t is always a host pointer. Synchronises. */
msf_status msf_get_state(msf_ctx* ctx, int32_t instance, double* Q, double* alpha, double* phi, int32_t* chi,
                         double* t, int32_t mem);

/* Replace one instance's state (Q, phi, chi as in msf_get_state; t host value);
 * recomputes the geometry and clears a device-detected error. */
msf_status msf_set_state(msf_ctx* ctx, int32_t instance, const double* Q, const double* phi, const int32_t* chi,
                         double t, int32_t mem);

/* Event counters summed over instances since msf_set_levelset: cut cells,
 * cells with >= 3 materials, corrected cells, small (mixed) cells, mixing
 * failures, merges, oddball cells, steps. counters: host [MSF_NSTATS]. Synchronises. */
msf_status msf_stats(msf_ctx* ctx, int64_t* counters);

/* Time step of the last step taken (host value). Synchronises. */
msf_status msf_last_dt(msf_ctx* ctx, int32_t instance, double* dt);

/* Intermediate fields of the last stage of one instance, for testing:
 * which = 0 alpha [n_mat][cells], 1 stencil state [n_mat][dim+2][cells],
 * 2 exchange flux [n_mat][dim+2][cells], 3 interface velocity [3][cells],
 * 4 mixed-cell flag [cells], 5 step material mask [cells]. out: host double array.
 * Cells outside the narrow band hold 0 for fields 1-3. Synchronises. */
msf_status msf_debug_field(msf_ctx* ctx, int32_t instance, int32_t which, double* out);

/* Progress of one instance: simulated time t, steps taken since
 * msf_set_levelset, and the device-detected error of that instance
 * (MSF_OK, MSF_ENONFINITE, MSF_ENEGATIVE or MSF_EBAND). Host outputs, any may
 * be NULL. Synchronises. An instance with an error stops stepping; the
 * others continue. */
msf_status msf_instance_info(msf_ctx* ctx, int32_t instance, double* t, int64_t* steps, int32_t* status);

/* CTA size the batched persistent kernel uses (0 before the first batched
 * step or when the context does not run batched). */
msf_status msf_batch_block_size(msf_ctx* ctx, int32_t* block_size);

/* Number of kernel launches one step enqueues (all instances). */
msf_status msf_launches_per_step(msf_ctx* ctx, int64_t* n);

/* With opt.profile = 1: device time in ms of the flux-update kernel of each of
 * the three stages of the last step of instance 0 (flux_ms: host [3]).
 * Synchronises. MSF_EINVAL when profiling is off. */
msf_status msf_profile_read(msf_ctx* ctx, double* flux_ms);

/* Largest state msf_cfl_dt_noalloc accepts: its scratch holds one partial
 * maximum per 256 cells, 16384 doubles (128 KiB) on every device. */
#define MSF_NOALLOC_MAX_CELLS 4194304

/* CFL time step of a single-material state, for callers that must not
 * allocate device memory. The paper has no counterpart: this is a service of
 * the library, the same bound msf_step applies to a cell with one material
 * (dt = cfl / max over cells of sum_d (|u_d| + c) / h_d, c^2 = gamma (p + pinf) / rho).
 *   U       device [dim + 2][cells] conservative state (rho, rho u_d, rho E)
 *   cells   1 .. MSF_NOALLOC_MAX_CELLS (larger: MSF_EINVAL)
 *   eos     host pointer, the material; h host [dim] cell sizes
 *   dt_out  device pointer to one double, written asynchronously; NaN when
 *           any cell has rho <= 0, c^2 <= 0 (p + pinf <= 0) or a non-finite
 *           value (the states msf_step reports as MSF_ENEGATIVE or
 *           MSF_ENONFINITE), so a bad state never yields a finite step
 *   stream  cudaStream_t for the two kernels (NULL: legacy default stream)
 * Calls no cudaMalloc/cudaFree and no allocating library routine: its scratch
 * is a fixed array compiled into the library, present on every device that
 * loads it until the process exits. The first call on a device looks up that
 * array's device address (cudaGetSymbolAddress) with the device current;
 * later calls look it up again unless their stream is being captured, when
 * the address of the last call outside capture is used, so make the first
 * call on each device before any stream capture (a capturing first call
 * returns MSF_ESTATE). Every call shares the array and writes every slot it
 * reads, so nothing needs clearing between calls; calls that overlap on the
 * GPU (other streams, other threads) race on it and must be ordered by the
 * caller. Errors: MSF_EINVAL (message via msf_last_error(NULL)), MSF_ECUDA,
 * MSF_ESTATE. */
msf_status msf_cfl_dt_noalloc(const double* U, int64_t cells, int32_t dim, const msf_eos* eos, const double* h,
                              double cfl, double* dt_out, void* stream);

/* FMA throughput of the CUDA cores of the current device, in flop/s (two
 * flops per fused multiply-add): precision MSF_FP64 measures FP64, any other
 * valid precision (MSF_FP32_BULK) FP32. The paper has no counterpart: this is
 * a measurement service, the denominator of the arithmetic roofline of the
 * flux kernels. Runs independent FMA chains on every SM (best of five
 * launches, CUDA events on `stream`), synchronises, allocates nothing.
 * Errors: MSF_EINVAL (message via msf_last_error(NULL)), MSF_ECUDA. */
msf_status msf_fma_peak(int32_t precision, double* flops_per_s, void* stream);

/* Human-readable message for the last non-OK status of this context
 * (or of msf_create when ctx is NULL). Never NULL. */
const char* msf_last_error(const msf_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
