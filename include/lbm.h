/*
 * lbm.h -- C ABI of the GB300 (sm_103a) two-distribution D2Q9 multiphase lattice Boltzmann
 * library.
 *
 * The method (Li, Luo & Gao, "Additional interfacial force in lattice Boltzmann models for
 * incompressible multiphase flows"):
 *   - an order-parameter distribution f_a whose zeroth moment phi tracks the interface by the
 *     convective Cahn-Hilliard equation (Eq. 2) with chemical potential
 *     mu = theta'(phi) - kappa lap(phi), theta = beta (phi^2 - phi*^2)^2 (Eq. 1);
 *   - a pressure distribution gbar_a (g_a = cs2 f_a + psi w_a, psi = p - rho cs2) that solves
 *     the pressure and velocity by Eq. 8 with forcing (e_a - u).K, K = (F_s + G) omega_a(u)
 *     - (omega_a(u) - omega_a(0)) grad(psi), discretised to second order;
 *   - density rho = rho_B + (phi + phi*)/(2 phi*) (rho_A - rho_B) (Eq. 4);
 *   - a per-run flag that removes the additional interfacial force
 *     F_a = -u [d_t rho + div(rho u)] (Eq. 12) by adding -F_a to the forcing.
 * Surface tension force F_s = -phi grad(mu), gravity G = (0, -rho g); derivatives are isotropic
 * central differences over the D2Q9 neighbours.
 *
 * Conventions
 *   - Lattice units, dx = dt = 1, cs2 = 1/3.  Fields exchanged with the caller are row-major
 *     float32 arrays of nx*ny values, index y*nx + x, x in [0,nx), y in [0,ny).
 *   - Every call returns LBM_OK (0) or a negative LBM_ERR_* code; no exception crosses the ABI.
 *     lbm_last_error() gives a thread-local message for the last failure.
 *   - The library owns all device state of a simulation; the caller owns every buffer it
 *     passes in.  Pointers to fields may be host or device memory (detected per call).
 *   - Work is queued on the CUDA stream given at creation (NULL = legacy default stream).
 *     lbm_step is asynchronous; lbm_moments and lbm_diagnostics synchronise that stream.
 *   - One simulation must not be used from two host threads at once; different simulations
 *     may be stepped from different host threads concurrently.
 *   - One GPU per process: the library measures the device it first runs on (multiprocessor
 *     count, occupancy, shared-memory limits) once and sizes every later launch by it.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define LBM_API __attribute__((visibility("default")))
#else
#define LBM_API
#endif

/* boundary types */
#define LBM_PERIODIC 0
#define LBM_WALL 1 /* no-slip wall half a cell outside the first/last row or column */

/* population storage */
#define LBM_FP32 0     /* 4-byte populations */
#define LBM_FP16_DEV 1 /* 2-byte fp16 deviations from the lattice-weight baseline, FP32 math */
#define LBM_BF16_DEV 2 /* 2-byte bf16 deviations, FP32 math; gbar stored by stochastic rounding
                          (unbiased, deterministic for a given value and place) */

/* step kernel (lbm_set_kernel) */
#define LBM_KERNEL_AUTO 0  /* the 2-D tile kernel where it applies on grids of at most 262144
                              cells, else the row march */
#define LBM_KERNEL_ROWS 1  /* strips marching rows: every configuration */
#define LBM_KERNEL_TILES 2 /* 2-D tiles in four shared-memory passes: s_form 0, f_form 0 */
#define LBM_KERNEL_RESIDENT 3 /* the 2-D tiles kept resident: one launch per lbm_step call */

/* return codes */
#define LBM_OK 0
#define LBM_ERR_INVALID_ARG (-1)
#define LBM_ERR_OOM (-2)
#define LBM_ERR_BUDGET (-3)
#define LBM_ERR_DIVERGED (-4)
#define LBM_ERR_TIMEOUT (-5)
#define LBM_ERR_CUDA (-6)

/* Scheme parameters (lattice units).
 *   beta, kappa   free-energy coefficients of Eq. 1 (> 0); see lbm_params_from_sigma_W.
 *   phi_star      equilibrium order parameter (> 0); phase A (heavy) is +phi*, B is -phi*.
 *   theta_M       Cahn-Hilliard mobility of Eq. 2 (>= 0).
 *   tau_f         relaxation time of f (> 1/2).
 *   tau_g_A/B     relaxation time of gbar in pure phase A / B (> 1/2); in the interface the
 *                 dynamic viscosity rho cs2 (tau - 1/2) is interpolated linearly in the liquid
 *                 fraction c = (phi + phi*)/(2 phi*) clamped to [0, 1].
 *   rho_A, rho_B  phase densities (> 0), Eq. 4.
 *   gravity       magnitude g of the body force G = (0, -rho g).
 *   bc_x, bc_y    LBM_PERIODIC or LBM_WALL.
 *   remove_Fa     0: scheme as first stated (Eq. 8 with F_s + G);
 *                 1: additional interfacial force removed (forcing F_s + G + u s with
 *                    s = rho' theta_M lap(mu) = d_t rho + div(rho u) by Eq. 5).
 *   storage       LBM_FP32, LBM_FP16_DEV or LBM_BF16_DEV.
 *   ch_conservative  0 (default): the f collision adds w_a phi div(u) (div by the isotropic
 *                 central differences), so the recovered Cahn-Hilliard equation is Eq. 2's
 *                 convective form d_t phi + u.grad(phi) = div(theta_M grad mu) even where the
 *                 weakly compressible flow has div(u) != 0;
 *                 1: no source, the conservative form d_t phi + div(phi u) = ... (the f
 *                 collision conserves phi locally).
 *   fs_form       0 (default): surface-tension force F_s = -phi grad(mu) (the solved p is the
 *                 modified pressure p_h - phi mu); 1: F_s = mu grad(phi) (p is p_h).
 *   s_form        mass defect s = d_t rho + div(rho u) used with remove_Fa:
 *                 0 (default): Eq. 5, s = rho' theta_M lap(mu);
 *                 1: directly from the previous step, s^t = (rho^t - rho^{t-1}) +
 *                    div(rho u)^{t-1} (isotropic divergence); the simulation then keeps rho and
 *                    div(rho u) in two more planes per state buffer (8 B per cell each,
 *                    lbm_sim_device_bytes counts them; at t = 0 the initial fields stand for
 *                    t = -1).
 *   f_form        order-parameter LBE (the paper uses a Cahn-Hilliard LBE it does not print):
 *                 0 (default): BGK towards an equilibrium whose second moment carries the
 *                 chemical potential; 1: forced form, relaxing to phi omega_a(u) with the
 *                 forcing (e_a - u).grad(phi) omega_a(u) and the mobility source
 *                 theta_M lap(mu) omega_a(u).  1 needs FP32 storage (its populations are O(phi))
 *                 and cannot join a batch; both are rejected with LBM_ERR_INVALID_ARG. */
typedef struct {
    double beta, kappa, phi_star, theta_M, tau_f, tau_g_A, tau_g_B, rho_A, rho_B, gravity;
    int bc_x, bc_y, remove_Fa, storage;
    int ch_conservative, fs_form;
    int s_form, f_form;
} lbm_params;

/* FP64 diagnostics of the current state (reductions in a fixed order: bitwise reproducible).
 *   sum_phi         sum of phi over the grid (conserved, Eq. 5 integrated)
 *   liquid_area     sum of c = clamp((phi + phi*)/(2 phi*), 0, 1)
 *   centroid_x/y    sum(c x)/sum(c), sum(c y)/sum(c)
 *   vel_x/y         sum(c u)/sum(c)
 *   spread_radius   half of the largest row sum of c (half the widest liquid chord)
 *   max_u           max |u|
 *   p_liquid/p_gas  mean pressure over phi > 0.9 phi* / phi < -0.9 phi*
 *   finite          0 if sum_phi or max_u is not finite (the run has diverged) */
typedef struct {
    long long step;
    double sum_phi, liquid_area, centroid_x, centroid_y, vel_x, vel_y;
    double spread_radius, max_u, p_liquid, p_gas;
    int finite, pad;
} lbm_diag;

typedef struct lbm_sim lbm_sim;

/* kappa = 3 sigma W / (8 phi*^2), beta = 3 sigma / (4 W phi*^4): the planar equilibrium of
 * Eq. 1 is phi* tanh(2x/W) with surface tension sigma.  Returns LBM_ERR_INVALID_ARG unless
 * sigma, W, phi_star > 0. */
LBM_API int lbm_params_from_sigma_W(double sigma, double W, double phi_star, double* beta, double* kappa);

/* BGK relaxation time of a kinematic viscosity: tau = nu / cs2 + 1/2. */
LBM_API double lbm_tau_from_nu(double nu);

/* Device bytes one simulation of nx x ny holds (both population buffers, field scratch and
 * reduction scratch) for the given storage. */
LBM_API size_t lbm_device_bytes(int nx, int ny, int storage);

/* Device bytes held by an existing simulation (lbm_device_bytes plus the s_form = 1 planes). */
LBM_API size_t lbm_sim_device_bytes(const lbm_sim* sim);

/* Create a simulation on the current CUDA device.  nx, ny >= 3 (>= 4 along a walled axis),
 * and ny * pitch * 76 B < 2 GiB (pitch = nx rounded up to 32: about 28 M cells); parameters
 * are validated (tau > 1/2, densities, beta, kappa, phi* > 0, theta_M >= 0).
 * cuda_stream: a cudaStream_t (may be NULL).  On success *out owns its device state: stream-ordered
 * allocations from the device's default memory pool on cuda_stream (no device-wide
 * synchronisation, so a simulation can be created while others run), returned to the pool by
 * lbm_destroy.
 * Errors: LBM_ERR_INVALID_ARG, LBM_ERR_OOM (device allocation failed), LBM_ERR_CUDA. */
LBM_API int lbm_create(int nx, int ny, const lbm_params* params, void* cuda_stream, lbm_sim** out);

/* Set the state at t = 0 from phi0, ux0, uy0, p0 (nx*ny float32 each, host or device; ux0,
 * uy0 and p0 may be NULL for zero): f = f^eq(phi0, mu0, u0), gbar = g^eq(p0, rho0, u0).
 * Asynchronous for device inputs; host inputs are copied before return, and the initialisation
 * kernels stay queued on the simulation's stream behind those copies. */
LBM_API int lbm_init_fields(lbm_sim* sim, const float* phi0, const float* ux0, const float* uy0,
                    const float* p0);

/* Advance n >= 0 time steps (asynchronous, queued on the simulation's stream). */
LBM_API int lbm_step(lbm_sim* sim, int n);

/* Macroscopic fields of the current state (phi, rho, ux, uy, p; any pointer may be NULL),
 * row-major nx*ny float32 each, host or device.  Synchronises the stream.  When nx is a multiple
 * of 32, device outputs are written by the moment kernel itself; the others are copied from the
 * simulation's work planes. */
LBM_API int lbm_moments(lbm_sim* sim, float* phi, float* rho, float* ux, float* uy, float* p);

/* The same two calls with every field in one caller-owned block, so that a transfer is one copy
 * instead of one per field (no counterpart in the paper: a transfer-cost measure).
 * lbm_init_fields_packed: `fields` holds phi0, ux0, uy0, p0 one after the other (4 nx*ny
 *   float32, row-major; host or device); otherwise as lbm_init_fields (host memory is consumed
 *   before return).
 * lbm_moments_packed: writes phi, rho, ux, uy, p of the current state one after the other into
 *   `fields` (5 nx*ny float32, host or device) and synchronises the stream.
 * Errors: LBM_ERR_INVALID_ARG for NULL arguments, LBM_ERR_CUDA for launch or copy failures. */
LBM_API int lbm_init_fields_packed(lbm_sim* sim, const float* fields);
LBM_API int lbm_moments_packed(lbm_sim* sim, float* fields);

/* The additional interfacial force of the current state (Eq. 12: F_a = -u [d_t rho + div(rho u)],
 * evaluated as -u s with u the state's velocity and s the mass defect by the simulation's s_form:
 * Eq. 5's rho' theta_M lap(mu), or the direct form from the stored density and flux), whether or
 * not the scheme removes it; the paper's Fig. 3 shows its y component.  fa_x, fa_y: row-major
 * nx*ny float32, host or device, either may be NULL.  Synchronises the stream.  Errors:
 * LBM_ERR_INVALID_ARG for a NULL sim, LBM_ERR_CUDA for launch or copy failures. */
LBM_API int lbm_interfacial_force(lbm_sim* sim, float* fa_x, float* fa_y);

/* FP64 diagnostics of the current state into *out (host).  Returns LBM_ERR_DIVERGED (and
 * fills *out, finite = 0) when the state is no longer finite.  Synchronises the stream. */
LBM_API int lbm_diagnostics(lbm_sim* sim, lbm_diag* out);

/* Free the simulation's device state (synchronises its stream first). */
LBM_API int lbm_destroy(lbm_sim* sim);

/* Number of time steps taken since lbm_init_fields. */
LBM_API long long lbm_step_count(const lbm_sim* sim);

/* Checkpoint / resume (no counterpart in the paper: it lets a server evict a simulation's
 * device state to host memory and resume it later bitwise).  A checkpoint is a 64-byte header
 * (magic "LBMC", version 2, nx, ny, row pitch, storage, step count, payload size) followed by
 * the raw population buffer of the current state; it holds no parameters.  Version 2 is the
 * blocked population layout: each row is pitch / 32 blocks of 32 cells, a block holding every
 * population plane of its cells in turn (FP32: f_0..f_8, gbar_0..gbar_8, f_0lo, 128 B each;
 * 16-bit: the FP32 rest plane, then 17 planes of 64 B); with s_form = 1 two FP32 planes
 * [rho, div(rho u)] of ny rows x pitch follow the populations.  Version 1 checkpoints (plain
 * planes) are rejected.
 * lbm_checkpoint_bytes: size of the checkpoint of `sim` (0 if sim is NULL).
 * lbm_checkpoint: writes it to `buf` (host or device memory, at least checkpoint_bytes long,
 *   caller-owned); synchronous.  A batch member must be removed from its batch first.
 * lbm_restore: replaces the state of `sim` (same nx, ny and storage; its parameters and stream
 *   are its own) by the checkpoint in `buf`, including the step count; synchronous.
 * Errors: LBM_ERR_INVALID_ARG for NULL arguments, a short buffer, a batch member, a bad header
 * or a size/storage mismatch (the state is then left unchanged); LBM_ERR_CUDA for copy
 * failures. */
LBM_API size_t lbm_checkpoint_bytes(const lbm_sim* sim);
LBM_API int lbm_checkpoint(lbm_sim* sim, void* buf, size_t bytes);
LBM_API int lbm_restore(lbm_sim* sim, const void* buf, size_t bytes);

/* Replace the stream the simulation queues its work on (cudaStream_t, may be NULL).  The previous
 * stream is synchronised first (the state's allocation and earlier work are ordered on it). */
LBM_API int lbm_set_stream(lbm_sim* sim, void* cuda_stream);

/* Tile shape of the fused step kernel: threads per CTA (64, 128 or 256; the CTA covers
 * threads - 6 interior columns) and rows per CTA (>= 1).  0 keeps the current value.  A new
 * simulation has 128 threads and as many rows per CTA as make one wave of resident CTAs
 * (at least 8 rows). */
LBM_API int lbm_set_tile(lbm_sim* sim, int threads, int seg_rows);

/* Step kernel of the simulation (no counterpart in the paper; both kernels compute every cell
 * bitwise alike): LBM_KERNEL_AUTO (default), LBM_KERNEL_ROWS, LBM_KERNEL_TILES or
 * LBM_KERNEL_RESIDENT.  The row march
 * streams large grids at the memory system's pace; on small grids its per-segment pipeline is
 * latency-bound, and the tile kernel (one load round and four short passes per step) is faster.
 * LBM_KERNEL_TILES and LBM_KERNEL_RESIDENT need s_form 0 and f_form 0 (else
 * LBM_ERR_INVALID_ARG).  Takes effect at the
 * next lbm_step; batches always run their own kernel. */
LBM_API int lbm_set_kernel(lbm_sim* sim, int kernel);
/* LBM_KERNEL_RESIDENT (same scope as LBM_KERNEL_TILES) runs lbm_step(sim, n >= 2) as ONE launch
 * whose CTAs stay on the device for all n steps (a cooperative launch of at most one wave, each
 * CTA stepping its tiles in turn).  Before a step, a tile waits only until the tiles within 4
 * cells of it (the farthest a step reads) have finished the previous step; the result is bitwise
 * that of LBM_KERNEL_TILES.  n = 1 runs the tile kernel.
 *
 * lbm_set_wait_limit: every such wait gives up after timeout_ns nanoseconds (default 1e9, > 0);
 *   the launch then ends early and leaves the state undefined, later resident launches do
 *   nothing, and the next lbm_step_status or lbm_diagnostics returns LBM_ERR_TIMEOUT (which
 *   re-arms the waits; lbm_init_fields or lbm_restore then gives a defined state again).
 *   hold_tile >= 0 is a test hook: that tile (row-major 16 x 8 tiles) never announces a finished
 *   step, so the waits of its neighbours run out; -1 (default) disables it.
 * lbm_step_status: synchronises the simulation's stream; LBM_ERR_TIMEOUT if a resident launch
 *   gave up since the status was last read, else LBM_OK.
 * Errors: LBM_ERR_INVALID_ARG for a NULL sim or timeout_ns <= 0; LBM_ERR_CUDA. */
LBM_API int lbm_set_wait_limit(lbm_sim* sim, long long timeout_ns, int hold_tile);
/* The kernel lbm_step runs for this simulation under its current choice: LBM_KERNEL_ROWS,
 * LBM_KERNEL_TILES or LBM_KERNEL_RESIDENT (AUTO resolved; a resident choice runs the tile kernel
 * for single steps); LBM_ERR_INVALID_ARG for a NULL sim. */
LBM_API int lbm_active_kernel(const lbm_sim* sim);
LBM_API int lbm_step_status(lbm_sim* sim);

/* Kernel launches issued by this simulation since creation (step, init, moments,
 * reductions). */
LBM_API long long lbm_launch_count(const lbm_sim* sim);

/* Static description of an error code. */
LBM_API const char* lbm_strerror(int code);

/* Message of the last failed call on this host thread ("" if none). */
LBM_API const char* lbm_last_error(void);

/* Allocation-free FP64 diagnostics of fields the caller already holds on the device.
 * The paper has no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- a host application that owns the whole device-memory budget (for example a
 * server whose pools have reserved it), or a loop that must not take the device-wide
 * synchronisation of a fresh allocation.  It allocates nothing: the per-row partial sums live
 * in one fixed file-scope device array of the library (8192 rows x 12 doubles plus the result,
 * 768 KB, held by every GPU that loads the library until the process exits).
 *   phi, ux, uy, p  row-major nx*ny float32 each (caller-owned, read only), in device memory of
 *                   the current device or in managed memory (anything else: LBM_ERR_INVALID_ARG);
 *   ny <= 8192 (larger grids: LBM_ERR_INVALID_ARG with a message), nx >= 1, phi_star > 0;
 *   step            copied into out->step;
 *   cuda_stream     stream the two reduction kernels run on (NULL: legacy default stream);
 *   out             host or device lbm_diag; a host record is filled before return (the stream
 *                   is synchronised) and LBM_ERR_DIVERGED is returned if the fields are not
 *                   finite; a device record is written asynchronously.  Synchronising is not
 *                   possible on a stream under capture: there a host out is refused with
 *                   LBM_ERR_INVALID_ARG, and a device out must be passed.
 * The reduction is the one lbm_diagnostics performs (same partials, order and result).  The
 * first call on a device looks up the array's device address with that device current; make
 * that first call before any stream capture.  All calls share the array: nothing in it has to
 * start at zero (every partial read is written first by the same call), but two calls whose
 * kernels overlap on the GPU race on it. */
LBM_API int lbm_diagnostics_fields_noalloc(const float* phi, const float* ux, const float* uy, const float* p,
                                           int nx, int ny, double phi_star, long long step, void* cuda_stream,
                                           lbm_diag* out);

/* ------------------------------------------------------------------ ragged batches
 * A batch advances many independent simulations (different sizes and parameters) with one
 * launch per time step over a work list of tiles from all of them.  Simulations stay owned by
 * the caller; the batch references them.  budget_bytes caps the summed lbm_device_bytes of
 * its members (0 = no cap).  lbm_batch_step(k) advances every member by k steps (replays of one
 * 16-step CUDA graph captured per membership, the rest launched directly); members keep stepping
 * on the batch's stream. */
typedef struct lbm_batch lbm_batch;

LBM_API int lbm_batch_create(size_t budget_bytes, void* cuda_stream, lbm_batch** out);
/* Add a simulation (it must not be in another batch).  LBM_ERR_BUDGET if it does not fit. */
LBM_API int lbm_batch_add(lbm_batch* b, lbm_sim* sim, int* slot);
LBM_API int lbm_batch_remove(lbm_batch* b, int slot);
LBM_API int lbm_batch_step(lbm_batch* b, int k);
/* Tile shape of the batch kernel (threads per CTA 64/128/256; rows per tile for members that
 * did not set their own, >= 1); 0 keeps the current value.  Takes effect at the next step. */
LBM_API int lbm_batch_set_tile(lbm_batch* b, int threads, int seg_rows);
/* Members, device bytes in use. */
LBM_API int lbm_batch_size(const lbm_batch* b);
LBM_API size_t lbm_batch_bytes(const lbm_batch* b);
LBM_API int lbm_batch_destroy(lbm_batch* b);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
