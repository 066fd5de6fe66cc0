/*
 * lbm.h - C ABI of the GB300 D3Q19 lattice Boltzmann solver with the adaptive
 * volumetric-flux boundary condition of McClure, Li, Sheppard and Miller,
 * "An adaptive volumetric flux boundary condition for lattice Boltzmann
 * methods" (arXiv:1806.10589).
 *
 * The library owns its device memory.  Every call returns an lbm_status and
 * never aborts; after a CUDA failure the context is poisoned (every later call
 * returns LBM_ECUDA) and lbm_last_error() says what failed.  A context is used
 * by one host thread at a time; separate contexts are independent.
 *
 * Conventions shared by all calls:
 *   - voxel arrays are laid out [z][y][x] with x fastest, nx*ny*nz entries;
 *   - the flow axis is z; the inlet is the plane z = 0 (face LBM_FACE_ZMIN),
 *     the outlet the plane z = nz-1 (face LBM_FACE_ZMAX); the four lateral faces
 *     are no-flow walls (Section 2 allows periodic or no-flow; this library
 *     implements no-flow);
 *   - lattice units throughout: rho0 = 1, c_s^2 = 1/3, nu = (tau - 1/2)/3.
 */
#ifndef GB300_LBM_H
#define GB300_LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx; /* opaque, created by lbm_create, freed by lbm_destroy */

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = -1,       /* bad argument (message in lbm_last_error) */
    LBM_ENOMEM = -2,       /* device or host allocation failed */
    LBM_ECUDA = -3,        /* CUDA runtime error; sticky for the context */
    LBM_EUNSUPPORTED = -4, /* valid request this library does not implement */
    LBM_EUNSTABLE = -5,    /* NaN or |u| > 0.1 found by lbm_get_monitors */
    LBM_ETIMEOUT = -6      /* reserved for bounded device waits */
} lbm_status;

/* Collision operator.  LBM_MODEL_MRT is Appendix A's multiple-relaxation-time
 * operator with s_e = s_eps = s_pi = s_nu = 1/tau and s_q = s_m =
 * 8(2 - s_nu)/(8 - s_nu); because every D3Q19 moment is even or odd in xi and
 * the rates split the same way, it is evaluated as the equivalent
 * two-relaxation-time update (s+ = s_nu, s- = s_q). */
/* LBM_MODEL_COLOR names the two-fluid colour model, which has its own context
 * (lbm_color_create below); lbm_create rejects it as an unknown model (LBM_EINVAL). */
enum { LBM_MODEL_BGK = 0, LBM_MODEL_MRT = 1, LBM_MODEL_COLOR = 2 };

/* Storage of the 19 distributions in device memory (arithmetic is FP64 for
 * LBM_PREC_FP64 and FP32 otherwise).  The 16-bit formats store the scaled
 * deviation (f_q / w_q - 1 - r(z)) * 2^10 from the rest-state weight w_q and a
 * linear reference density r(z) between the inlet and outlet densities
 * (refreshed every 1024 steps).  Steps round these stores stochastically (zero
 * mean error, reproducible: the random bits hash the step, node and direction),
 * so a steady state carries no rounding bias. */
enum { LBM_PREC_FP64 = 0, LBM_PREC_FP32 = 1, LBM_PREC_FP16DEV = 2, LBM_PREC_BF16DEV = 3 };

/* Faces.  Only z faces are open (the paper derives the z-inlet condition). */
enum { LBM_FACE_ZMIN = 4, LBM_FACE_ZMAX = 5 };

/* Create a solver.  Cites: Eq. (d3q19), Eq. (LBE), Appendix A.
 *   mask       host, nx*ny*nz bytes [z][y][x]: 0 = pore, 1 = solid; copied, the
 *              caller keeps ownership.  Any other byte value is LBM_EINVAL.
 *   nx, ny     1..2047;  nz 3..1023.
 *   tau        > 0.5, the relaxation time (nu = (tau - 1/2)/3).
 *   model      LBM_MODEL_*;  precision LBM_PREC_*.
 *   out        receives the new context.
 * The planes z = 0 and z = nz-1 must each hold at least one pore node
 * (LBM_EINVAL otherwise).  Cells are initialised at rest, f = f^eq(rho=1, u=0).
 * Defaults: inlet flux Q = 0, outlet density rho_out = 1, default CUDA stream. */
int lbm_create(const uint8_t* mask, int nx, int ny, int nz, double tau, int model,
               int precision, lbm_ctx** out);

/* Prescribe the volumetric flux Q (lattice units, lu^3/lt) through the inlet,
 * Eq. (flux).  Every step the inlet density is then set from Eq. (potential),
 * rho_in = (rho0 Q + sum over inlet pore nodes of the known sum of Eq. inlet)/A,
 * A = number of inlet pore nodes, and imposed with the Hecht-Harting pressure
 * closure of Appendix B, so that the sum of u_z over the inlet equals Q to
 * rounding.  face must be LBM_FACE_ZMIN; LBM_FACE_ZMAX returns
 * LBM_EUNSUPPORTED (Section 2: a flux condition at both ends is neither needed
 * nor advantageous).  Takes effect at the next step. */
int lbm_set_flux_bc(lbm_ctx* ctx, int face, double Q);

/* Prescribe a fixed density (pressure p = rho/3, Eq. pressure) on a face with the
 * Appendix B closure.  LBM_FACE_ZMAX sets the outlet density (default 1.0);
 * LBM_FACE_ZMIN switches the inlet from the flux condition to this fixed
 * density until lbm_set_flux_bc is called again.  rho must be > 0. */
int lbm_set_pressure_bc(lbm_ctx* ctx, int face, double rho);

/* Use this CUDA stream (a cudaStream_t passed as void*, e.g. a PyTorch stream
 * handle) for all later device work of this context.  NULL = default stream.
 * A variant-3 state left in the in-place layout is swapped back on the
 * previous stream first. */
int lbm_set_stream(lbm_ctx* ctx, void* cuda_stream);

/* Select the step-kernel variant.  Every variant computes the same step:
 * variants 0-2 bit for bit in FP64/FP32; the AA pattern to rounding (its
 * kernels may contract products into FMAs differently); with the 16-bit formats
 * within the storage rounding.  0 = one thread per pore node (the default); 1 = persistent kernel
 * whose neighbour ids and pulled values are staged in shared memory by cp.async
 * one 256-node tile ahead; 2 = the same with 128-node tiles; 3 = AA pattern:
 * ONE distribution buffer updated in place (the second buffer is freed, so the
 * state needs half the memory), alternating a gather-scatter step and a
 * node-local step; every storage format.  On
 * variant 3 the first lbm_step call swaps the buffer into the in-place layout
 * (one launch), and the buffer stays in that layout across lbm_step calls,
 * which continue the alternation where the last call left it.  Any other call
 * on the context swaps it back first, on the context's stream (one launch, two
 * after an odd number of steps); 16-bit formats also swap back at every
 * reference-profile refresh.  So every call that reads or writes the state
 * sees it exactly as with the other variants.  Leaving variant 3 allocates the second buffer again
 * (LBM_ENOMEM if that fails; the context stays on variant 3).  Unknown
 * variants return LBM_EINVAL.  Synchronises. */
int lbm_set_kernel(lbm_ctx* ctx, int variant);

/* Advance n >= 0 time steps, asynchronously on the context's stream.  One step
 * follows Section 2's order: pull streaming with halfway bounce-back at solid
 * voxels, the inlet density reduction (Eq. potential), the pressure closures at
 * inlet and outlet (Appendix B), then collision (Appendix A) at every pore node.
 * Runs of 64 steps are replayed from captured CUDA graphs.  On variant 3 the
 * buffer is left in the AA pattern's in-place layout (see lbm_set_kernel).
 * Stream capture of the context's stream: runs of 64 steps launch the
 * library's own graphs, which a capturing stream rejects (LBM_ECUDA).  The
 * host-side buffer parity, layout and step count advance when a call is made,
 * not when recorded work replays.  So on variant 3 a call made while the
 * stream captures keeps the pull layout at its start and end, and a buffer left
 * in the in-place layout by an earlier call makes it, and every other call that
 * would swap the layout back inside the capture, return LBM_EINVAL instead of
 * recording a swap; make any other call on the context (e.g. lbm_set_stream)
 * before the capture begins. */
int lbm_step(lbm_ctx* ctx, int n);

/* Measured flux through a face: Q = sum of u_z over the face's pore nodes of the
 * current state, in FP64, and the density imposed on that face at the last step
 * (rho_in from Eq. potential for the inlet, rho_out for the outlet).  Either
 * pointer may be NULL.  Synchronises the context's stream. */
int lbm_get_flux(lbm_ctx* ctx, int face, double* Q, double* rho_bc);

/* FP64 monitors of the current state: total mass sum(rho) over pore nodes,
 * inlet and outlet fluxes, and max |u|.  Returns LBM_EUNSTABLE when a value is
 * NaN or max |u| > 0.1 (Section 3.2's stability rule of thumb), else LBM_OK.
 * Any pointer may be NULL.  Synchronises. */
int lbm_get_monitors(lbm_ctx* ctx, double* mass, double* q_in, double* q_out, double* u_max);

/* Steady-state criterion of Section 3.1 (Eq. stopping_criterion):
 *   residual = sum_x |u(x,t) - u(x,t')| / sum_x |u(x,t)|
 * over pore nodes (|.| the Euclidean norm per node, FP64 sums), where t' is the
 * state at the previous call; the paper uses a lag t - t' of 1000 steps and
 * stops at residual <= 1e-6.  The first call only stores the snapshot (it
 * allocates 24 bytes per pore node once) and returns +infinity.  Synchronises. */
int lbm_steady_residual(lbm_ctx* ctx, double* residual);

/* Macroscopic fields rho = sum f (Eq. m0), u = sum f xi / rho0 (Eq. m357) of the
 * current state into caller-owned HOST arrays of nx*ny*nz doubles each ([z][y][x]);
 * solid voxels are written as 0.  Any pointer may be NULL.  Synchronises. */
int lbm_get_fields(lbm_ctx* ctx, double* rho, double* ux, double* uy, double* uz);

/* The same fields as FP32 into caller-owned DEVICE buffers: rho (nx*ny*nz floats)
 * and u (3*nx*ny*nz floats, components ux, uy, uz as three consecutive
 * [z][y][x] blocks).  Asynchronous on the context's stream. */
int lbm_get_fields_device(lbm_ctx* ctx, float* rho, float* u);

/* Reset every pore node to f^eq(rho, u) from caller-owned HOST arrays of nx*ny*nz
 * doubles ([z][y][x]; solid entries ignored), e.g. for a warm start.  A NULL
 * velocity component means 0; NULL rho means 1.  Synchronises. */
int lbm_set_fields(lbm_ctx* ctx, const double* rho, const double* ux, const double* uy,
                   const double* uz);

/* Copy all 19 distributions of the current state to/from a caller-owned HOST
 * array of 19*nx*ny*nz doubles laid out [q][z][y][x], q in the order of
 * Eq. (d3q19) (7..18 as fixed by Appendix B).  get writes 0 at solid voxels; set
 * ignores them and encodes into the storage precision.  Synchronises. */
int lbm_get_distributions(lbm_ctx* ctx, double* f);
int lbm_set_distributions(lbm_ctx* ctx, const double* f);

/* Sizes: number of pore nodes, inlet pore nodes (A), outlet pore nodes, steps
 * taken since creation or the last set_* call.  Any pointer may be NULL. */
int lbm_get_info(const lbm_ctx* ctx, int64_t* n_pore, int64_t* a_in, int64_t* a_out,
                 int64_t* steps);

/* Profiling aid: run n >= 1 steps as individual kernel launches on the context's
 * stream, with CUDA events around each step launch.  Returns the mean device time
 * in milliseconds of the step kernel.  On variant 3 that is the mean over the
 * alternating gather-scatter and node-local launches; with n = 1 it is the
 * gather-scatter launch alone.  The layout swaps around the launches are not
 * timed.  The second output is 0, because the inlet reduction runs inside the
 * step kernel.  Either pointer may be NULL.  Advances the state by n steps exactly
 * like lbm_step(ctx, n).  Synchronises. */
int lbm_time_kernels(lbm_ctx* ctx, int n, float* ms_step_kernel, float* ms_inlet_kernel);

/* Inlet density for callers that cannot allocate device memory at the point of
 * the call -- a process whose device memory is reserved up front by another
 * allocator (a framework's caching pool leaves no room for a second one), or
 * real-time code that sizes all of its memory before it starts and must not
 * stall in the allocator later.  The paper has no counterpart: this is a
 * library-interface addition.  It computes, from the context's current distributions and the
 * prescribed Q, the inlet density rho_in of Eq. (potential) that the next step
 * imposes in flux mode, and writes it as one double to the caller-owned DEVICE
 * pointer rho_in_device, asynchronously on the context's stream.
 *   - Allocates nothing: its reduction scratch is a fixed static device array
 *     of 16.6 KB that every GPU loading the library keeps until process exit;
 *     the first call on a device looks up that array's device address, so make
 *     it before any stream capture.
 *   - Inlets of at most 524,288 pore nodes; larger ones return LBM_EINVAL.
 *   - All calls share the scratch array: calls whose kernels overlap on the GPU
 *     (other streams, other host threads, other contexts) race and must be
 *     serialised by the caller.
 *   - The array's device address is cached per device for the life of the
 *     process; after a cudaDeviceReset on that device the cached address is
 *     stale, so the entry point must not be called there again. */
int lbm_inlet_density_noalloc(lbm_ctx* ctx, double* rho_in_device);

/* Free all device and host memory of the context.  NULL is accepted. */
int lbm_destroy(lbm_ctx* ctx);

/* ---------------------------------------------------------------------------
 * Batched ensemble: n_members independent sub-volumes (each its own voxel box,
 * mask and inlet flux target, same tau/model/precision), advanced together by
 * one kernel launch per step; runs of 64 steps replay a captured CUDA graph.
 * Per member the problem is exactly the single-lattice one above (Section 2:
 * flux inlet by Eq. potential + Appendix B closures, pressure outlet rho = 1,
 * no-flow lateral faces, Appendix A collision).
 * ------------------------------------------------------------------------- */
typedef struct lbm_batch lbm_batch; /* opaque */

/* masks: n_members host pointers to uint8 [z][y][x] masks (copied); dims: 3 ints
 * per member (nx, ny, nz) with the single-lattice limits; every member needs
 * pore nodes on its inlet and outlet planes.  Members start at rest with Q = 0. */
int lbm_batch_create(int n_members, const uint8_t* const* masks, const int* dims, double tau, int model,
                     int precision, lbm_batch** out);
/* Inlet flux Q of one member (Eq. flux), as lbm_set_flux_bc.  Synchronises. */
int lbm_batch_set_flux_bc(lbm_batch* b, int member, double Q);
int lbm_batch_set_stream(lbm_batch* b, void* cuda_stream);
/* Advance all members n >= 0 steps, asynchronously on the batch's stream. */
int lbm_batch_step(lbm_batch* b, int n);
/* As lbm_get_flux for one member (sum of u_z over the face, FP64; imposed density). */
int lbm_batch_get_flux(lbm_batch* b, int member, int face, double* Q, double* rho_bc);
/* One member's distributions to/from a host array of 19*nx*ny*nz doubles [q][z][y][x]. */
int lbm_batch_get_distributions(lbm_batch* b, int member, double* f);
int lbm_batch_set_distributions(lbm_batch* b, int member, const double* f);
/* One member's rho and u (as lbm_get_fields) into host arrays of nx*ny*nz doubles. */
int lbm_batch_get_fields(lbm_batch* b, int member, double* rho, double* ux, double* uy, double* uz);
/* Total pore nodes, 256-node tiles of the launch, steps taken.  NULLs allowed. */
int lbm_batch_get_info(const lbm_batch* b, int64_t* n_pore, int64_t* n_tiles, int64_t* steps);
/* Profiling aid: n >= 1 single-step launches with CUDA events around each on the
 * batch's stream; mean device milliseconds per step.  Advances the state. */
int lbm_batch_time_step(lbm_batch* b, int n, float* ms);

/* Launch configurations of lbm_batch_step.  All compute the same steps; they differ
 * in launch form and register cap.
 *   LBM_BATCH_GRAPH (default): one launch per step, with one 256-node tile per block.
 *     Runs of 64 steps replay a captured CUDA graph.
 *   LBM_BATCH_PERSISTENT: one cooperative launch carries all steps of a call.  The
 *     call is split at the 16-bit reference refreshes.  Blocks walk the tiles with
 *     a grid stride, and a grid barrier separates the steps.  That barrier's wait
 *     is bounded (2^31 SM cycles, about 1 s).  If a wait runs out, the call returns
 *     LBM_ETIMEOUT and the state it leaves is incomplete.  The call synchronises
 *     the stream to read that status.
 *   LBM_BATCH_AA: the AA pattern of lbm_set_kernel variant 3 on the shared store.
 *     Steps alternate a gather-scatter and a node-local launch under a captured
 *     graph, with in-place layout swaps around each call.  Both buffers stay
 *     allocated.
 *   *_CAPPED: the same launch compiled for 5 resident 256-thread blocks per SM
 *     (48 registers) instead of 4 (64 registers).  There is no cap for FP64.
 * lbm_batch_set_config selects a configuration.  lbm_batch_autotune measures
 * them for you.  For every configuration it runs trial_steps steps untimed, then
 * trial_steps timed steps, restoring the state after each run.  The restore uses
 * a temporary device copy of the state (LBM_ENOMEM if there is no room).  It then
 * selects the fastest: *best receives it, and ms_per_step[LBM_BATCH_NCONFIG] (may
 * be NULL) the per-step times.  On return, the state, step count and boundary
 * values are those before the call.  Both calls synchronise. */
enum {
    LBM_BATCH_GRAPH = 0,
    LBM_BATCH_GRAPH_CAPPED = 1,
    LBM_BATCH_PERSISTENT = 2,
    LBM_BATCH_PERSISTENT_CAPPED = 3,
    LBM_BATCH_AA = 4,
    LBM_BATCH_AA_CAPPED = 5,
    LBM_BATCH_NCONFIG = 6
};
int lbm_batch_set_config(lbm_batch* b, int config);
int lbm_batch_autotune(lbm_batch* b, int trial_steps, int* best, float* ms_per_step);
/* Diagnostic of the persistent launch's grid barrier (no effect on the state).
 * Four blocks meet at a barrier expecting four arrivals (*completes = 1 if it
 * completed), then at one expecting five, whose bounded wait must run out after
 * about timeout_ms (0 < timeout_ms <= 2000) and be reported (*times_out = 1).
 * The context stays usable either way.  Synchronises. */
int lbm_batch_check_barrier(lbm_batch* b, double timeout_ms, int* completes, int* times_out);
int lbm_batch_destroy(lbm_batch* b);
const char* lbm_batch_last_error(const lbm_batch* b);

/* Message of the last error on ctx (or of the last failed lbm_create when
 * ctx is NULL).  The string is owned by the library and valid until the next
 * call on the same context. */
const char* lbm_last_error(const lbm_ctx* ctx);

/* ---------------------------------------------------------------------------
 * Two-fluid colour model (Appendix A) with the flux inlet of Section 2.
 * Momentum: D3Q19 as above, with the interfacial equilibrium terms
 * m1 += alpha|C|, m9 += alpha|C|/2 (2nx^2 - ny^2 - nz^2), m11 += alpha|C|/2 (ny^2 - nz^2),
 * m13/m14/m15 += alpha|C|/2 nx ny / ny nz / nx nz, C = grad phi, n = C/|C|.
 * Phases: D3Q7 A and B (w0 = 1/3, w1..6 = 1/9) with the recolouring update
 * A_q(x + xi_q) = w_q N_A [1 + 9/2 u.xi_q + beta N_B n.xi_q] (B with -beta N_A),
 * phi = (N_A - N_B)/(N_A + N_B).  Readings of the silent points: C is the
 * isotropic D3Q19 stencil 3 sum_q w_q xi_q phi(x + xi_q), a solid voxel
 * contributes phi_s (wetting: +1 = the solid looks like phase A), a neighbour
 * outside the box (any face) the node's own phi, so the box faces are
 * wetting-neutral walls (they still bounce momentum and phases back); the inlet plane holds the injected composition
 * (N_A = (1 + phi_in)/2, N_B = (1 - phi_in)/2 at the reference density 1, set on
 * the value that entered through the inlet), the outlet lets both phases leave with their local
 * composition.  FP64 or FP32
 * storage.  A mask whose z = 0 (z = nz-1) plane is all solid has no inlet
 * (outlet) condition, so closed boxes are allowed.
 * ------------------------------------------------------------------------- */
typedef struct lbm_color lbm_color; /* opaque */
int lbm_color_create(const uint8_t* mask, int nx, int ny, int nz, double tau, double alpha, double beta,
                     double phi_s, int precision, lbm_color** out);
int lbm_color_set_stream(lbm_color* c, void* cuda_stream);
/* Inlet flux Q (Eq. flux, Eq. potential) and the phase phi_in of the injected fluid. */
int lbm_color_set_flux_bc(lbm_color* c, double Q, double phi_in);
/* Rest state with a phase field: host phi (nx*ny*nz doubles in [-1, 1]) and optional
 * rho (NULL = 1): f = f^eq(rho, 0), A = w7 rho (1 + phi)/2, B = w7 rho (1 - phi)/2. */
int lbm_color_set_phase(lbm_color* c, const double* phi, const double* rho);
/* Whole state from/to host arrays [q][z][y][x]: f 19, A 7 and B 7 planes of nx*ny*nz doubles. */
int lbm_color_set_state(lbm_color* c, const double* f, const double* A, const double* B);
int lbm_color_get_state(lbm_color* c, double* f, double* A, double* B);
int lbm_color_step(lbm_color* c, int n);
/* rho, u and phi of the current state (host, nx*ny*nz doubles each; NULLs allowed; 0 at solids). */
int lbm_color_get_fields(lbm_color* c, double* rho, double* ux, double* uy, double* uz, double* phi);
/* Sum of u_z over the inlet or outlet pore nodes, and the face density. */
int lbm_color_get_flux(lbm_color* c, int face, double* Q, double* rho_bc);
int lbm_color_destroy(lbm_color* c);
const char* lbm_color_last_error(const lbm_color* c);

/* ---------------------------------------------------------------------------
 * Learned warm start (not in the paper; a library addition).  A 3-D U-Net
 * with `levels` resolution levels and base * 2^l channels at level l (the
 * specified network: levels = 4, base = 32, i.e. 32/64/128/256 channels, 15
 * convolutions; every channel count must be 32, 64, 128 or 256), 3x3x3
 * convolutions, ReLU, 2x2x2 mean pooling, nearest upsampling and additive
 * skips, maps a voxel geometry to 4 steady-state fields: the velocity divided
 * by the superficial velocity u_D = Q / (nx ny), and the pressure gradient
 * G = -(p(z+1) - p(z)) / (nu u_D), p = rho / 3, nu = (tau - 1/2) / 3.  The convolutions (forward, data
 * gradient, weight gradient) run on the tcgen05 tensor cores with BF16
 * weights and activations and FP32 accumulation; pooling, upsampling, loss
 * and Adam run in this library's CUDA kernels; the master parameters and Adam
 * state are FP32.  All volumes have sides divisible by 2^(levels-1); masks are
 * uint8 [z][y][x], 1 = solid (as for lbm_create); fields are float32
 * [c][z][y][x] with c = u_x, u_y, u_z, G; a NaN target entry has no target
 * (it adds nothing to the loss).  Parameters are stored layer by layer
 * (forward order) as W[cout][27][cin] (taps dz, dy, dx each in -1, 0, 1, then
 * the input channel) followed by b[cout]; they start at 0 until set.  A
 * tensor-core pipeline wait that runs out (bounded at about one second)
 * returns LBM_ETIMEOUT instead of hanging.
 * ------------------------------------------------------------------------- */
typedef struct lbm_wsnet lbm_wsnet; /* opaque */
int lbm_wsnet_create(int levels, int base, lbm_wsnet** out);   /* LBM_EINVAL for an unsupported shape */
int lbm_wsnet_num_params(const lbm_wsnet* net, int64_t* n);
int lbm_wsnet_set_stream(lbm_wsnet* net, void* cuda_stream);
int lbm_wsnet_set_params(lbm_wsnet* net, const float* params);   /* host, num_params floats; resets Adam */
int lbm_wsnet_get_params(lbm_wsnet* net, float* params);         /* host, num_params floats */
/* Masked mean squared error over pore voxels of `batch` samples (host arrays:
 * masks batch*nz*ny*nx bytes, targets batch*4*nz*ny*nx floats; divided by
 * 4 * the pore count) and its gradient
 * w.r.t. the parameters (host, num_params floats; may be NULL). */
int lbm_wsnet_loss_grad(lbm_wsnet* net, const uint8_t* masks, const float* targets, int batch, int nx, int ny,
                        int nz, double* loss, float* grad);
/* Adam training (beta 0.9 / 0.999, eps 1e-8): `epochs` passes over n_samples
 * host samples in mini-batches of `batch`, visiting samples in the caller's
 * order (epochs*n_samples indices); mean loss per epoch into loss_history
 * (epochs floats, may be NULL).  Synchronises.  Deterministic: the weight and
 * bias gradients are summed per row split and the splits added in a fixed
 * order (no floating-point atomics), so the same inputs give bitwise the same
 * parameters on the same GPU model (also for lbm_wsnet_loss_grad's gradient;
 * the reported losses are FP64 sums whose order, and so whose last bits, may
 * vary).  The partial sums take up to 8.5e7 bytes of device memory more,
 * freed by lbm_wsnet_release_buffers. */
int lbm_wsnet_train(lbm_wsnet* net, const uint8_t* masks, const float* targets, int n_samples, int nx, int ny,
                    int nz, int epochs, int batch, float lr, const int* order, float* loss_history);
/* Predicted fields (host, 4*nz*ny*nx floats) of one geometry; 0 at solids. */
int lbm_wsnet_predict(lbm_wsnet* net, const uint8_t* mask, int nx, int ny, int nz, float* y);
/* Free the activation buffers kept between calls (sized for the last batch and volume). */
int lbm_wsnet_release_buffers(lbm_wsnet* net);
int lbm_wsnet_destroy(lbm_wsnet* net);
const char* lbm_wsnet_last_error(const lbm_wsnet* net);

/* One 3x3x3 convolution of the network on the tensor cores, on caller-owned
 * DEVICE buffers in the network's activation layout: BF16, channels last,
 * [batch][nz+2][ny+2][nx+2][c] with a one-voxel border that must hold zeros
 * (the layer's zero padding).  cin, cout in {32, 64, 128, 256}; w is BF16
 * [cout][27][cin] (taps dz, dy, dx in -1..1).  Asynchronous work on `stream`,
 * then a synchronisation of it.
 *   op 0, forward:  out[v][co] = act(bias[co] + sum_t sum_ci w[co][t][ci] in[v + t][ci])
 *         (in: cin channels; out: BF16, cout channels, border rows written 0;
 *          bias FP32 [cout] or NULL; act = ReLU if relu, else identity)
 *   op 1, data gradient:  out[v][ci] = sum_t sum_co w[co][t][ci] in[v - t][co]
 *         (in: the output gradient, cout channels; out: BF16, cin channels,
 *          border rows written 0)
 *   op 2, weight gradient:  out[co][t][ci] += sum_v aux[v][co] in[v + t][ci]
 *         (in: the layer input, cin channels; aux: the output gradient, cout
 *          channels, zero on border rows; out: FP32 [cout][27][cin], added to
 *          with FP32 atomics, one per row split: the order of those additions,
 *          and so the last bits, may vary between calls)
 * Returns LBM_EINVAL for bad arguments, LBM_ECUDA for a CUDA error and
 * LBM_ETIMEOUT if a pipeline wait ran out. */
int lbm_conv3d_bf16(int op, const void* in, const void* aux, const void* w, const float* bias, int relu, void* out,
                    int batch, int nx, int ny, int nz, int cin, int cout, void* cuda_stream);
/* The same convolution launched `reps` times back to back on `cuda_stream`,
 * bracketed by CUDA events on that stream; *ms_per_call = the mean time of
 * one launch.  For op 2 the weight gradient is added `reps` times. */
int lbm_conv3d_bf16_time(int op, const void* in, const void* aux, const void* w, const float* bias, int relu,
                         void* out, int batch, int nx, int ny, int nz, int cin, int cout, int reps,
                         float* ms_per_call, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* GB300_LBM_H */
