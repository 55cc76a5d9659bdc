/*
 * bats.h -- C ABI of libbats: one explicit second-order stage of the
 * ideal-MHD finite-volume update over all blocks of a 2:1 block-adaptive
 * grid (8^3-cell blocks, 2 ghost layers) on one NVIDIA GB300 (sm_103a).
 *
 * Method: arXiv 2501.06717 (BATSRUS GPU), Section 3 and Algorithms 1-2 (the
 * solver loop: face values, face fluxes, sources, update, ghost-cell
 * exchange), Section 4.1-4.2 (ghost layers; copy, restriction and
 * prolongation at resolution changes), Section 5.1 Eqs. 1-5 (ideal MHD with
 * the Powell 8-wave source terms, mu0 = 1), Section 5.2 (two-stage
 * second-order time stepping, inner body, inflow and floating boundaries).
 *
 * Conventions used by every entry point:
 *  - Status: 0 (BATS_OK) on success, a negative BATS_ERR_* code on failure;
 *    bats_last_error() then describes the failure.  No entry point aborts.
 *  - A state array is double [8][n_blocks][8][8][8] (variable, block, k, j, i;
 *    i fastest) of the conservative variables (rho, rho ux, rho uy, rho uz,
 *    B1x, B1y, B1z, e1), with B = B0 + B1 and e1 = p/(gamma-1) + rho u^2/2 +
 *    B1^2/2.  Block order is the leaf order given to bats_create.
 *  - Pointers to caller memory may be host or device (CUDA) pointers; the
 *    library detects which and copies.  The caller keeps ownership of every
 *    buffer it passes; the library owns the handle and all device memory it
 *    allocates, released by bats_destroy.
 *  - All device work is enqueued on the stream given to bats_create.  Entry
 *    points that return data to the host synchronise that stream.
 */
#ifndef BATS_H
#define BATS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define BATS_OK 0
#define BATS_ERR_INVALID_ARG (-1)     /* bad pointer, size, index or descriptor   */
#define BATS_ERR_UNBALANCED_TREE (-2) /* leaves overlap, leave gaps, or break 2:1 */
#define BATS_ERR_OUT_OF_MEMORY (-3)   /* device or host allocation failed         */
#define BATS_ERR_CUDA (-4)            /* a CUDA runtime call or launch failed      */
#define BATS_ERR_NONPHYSICAL (-5)     /* rho <= 0, p <= 0 or NaN after an update   */
#define BATS_ERR_TIMEOUT (-6)         /* a bounded device wait ran out             */
#define BATS_ERR_NOT_TRAINED (-7)     /* learned form requested without weights    */

/* ---- enumerations ------------------------------------------------------ */
enum { BATS_BC_PERIODIC = 0, BATS_BC_OUTFLOW = 1, BATS_BC_INFLOW = 2 };
enum { BATS_LIM_MINMOD = 0, BATS_LIM_MC = 1, BATS_LIM_NONE = 2 };
enum { BATS_RK_MIDPOINT = 0, BATS_RK_SSP2 = 1, BATS_RK_EULER = 2 };
enum { BATS_FP64 = 0, BATS_MIXED = 1 };
enum { BATS_B0_NONE = 0, BATS_B0_UNIFORM = 1, BATS_B0_DIPOLE = 2, BATS_B0_LINEAR = 3 };
enum { BATS_FLUX_RUSANOV = 0, BATS_FLUX_HLL = 1, BATS_FLUX_LINDE = 2 };
enum { BATS_PHASE_STAGE = 0, BATS_PHASE_DT = 1, BATS_PHASE_TOTAL = 2, BATS_NUM_PHASES = 3 };

typedef struct bats bats_t;

/* One grid (Section 2: a tree of equal-size blocks; 8^3 cells per block).
 *  lo, hi     domain corners; the domain is root[a] * 8 * 2^level cells per axis
 *  root       root blocks per axis (level 0)
 *  leaves     n_leaves x 4 int32 (level, i, j, k): block coordinates at that
 *             level; read during bats_create only
 *  bc         per domain face (-x, +x, -y, +y, -z, +z): BATS_BC_*; periodic
 *             must be set on both faces of an axis.  Outflow copies the nearest
 *             interior cell (zero gradient, the paper's "floating" boundary,
 *             Section 5.2); inflow holds the fixed state `inflow`.
 *  inflow     primitive state (rho, u, B1, p) of inflow faces
 *  body_r     cells whose centre lies within body_r of the origin are held
 *             at the primitive state `body` (Section 5.2 inner boundary); 0 = none */
typedef struct {
  double lo[3], hi[3];
  int32_t root[3];
  int32_t n_leaves;
  const int32_t* leaves;
  int32_t bc[6];
  double inflow[8];
  double body_r;
  double body[8];
} bats_grid_desc;

/* Physics and launch form, shared by all grids of a handle.
 *  gamma          ratio of specific heats (Eq. 5)
 *  limiter        BATS_LIM_MINMOD or BATS_LIM_MC (limited linear reconstruction
 *                 of primitives, Algorithm 1 "calc_face_value"), or BATS_LIM_NONE
 *                 (first order: face values are the cell values)
 *  rk             BATS_RK_MIDPOINT (default), BATS_RK_SSP2, or BATS_RK_EULER (the
 *                 one-stage scheme of Section 5.2's time-accurate session)
 *  precision      BATS_FP64: every step in FP64.  BATS_MIXED: reconstruction,
 *                 fluxes and sources in FP32; pressure recovery and the state
 *                 accumulation in FP64.
 *  b0, b0_param   background field B0 (split field): UNIFORM (B0 = p[0..2]),
 *                 DIPOLE (moment p[0..2] at the origin), LINEAR (B0 = p[0..2] +
 *                 G x, G = p[3..11] row-major)
 *  powell         1 = add the Powell 8-wave div-B source terms (Eqs. 2-4)
 *  learned        1 = add the MLP flux correction (needs bats_set_mlp)
 *  persistent     1 = one persistent launch per stage (grid = SMs x occupancy)
 *  blocks_per_cta blocks processed per work item in the persistent launch (>= 1)
 *  ctas_per_sm    persistent CTAs per SM (0 = the occupancy limit)
 *  use_graph      1 = replay whole bats_step calls from a CUDA graph
 *  local_dt       1 = local time stepping (Section 5.2's steady-state session):
 *                 with a CFL number, every cell advances with its own
 *                 dt_i = cfl / sum_d (|u_d| + c_f,d) / dx_d of the step's initial
 *                 state, in every stage; the elapsed time advances by the global
 *                 dt.  Ignored by bats_step_dt (fixed dt).
 *  reflux         1 = conservative flux correction at resolution changes: the
 *                 flux through a coarse face that borders a refined region is
 *                 replaced, for the coarse cell, by the mean of the 4 fine
 *                 fluxes through it, so every conserved variable is conserved to
 *                 round-off on periodic grids without sources.  Not with
 *                 `learned` (BATS_ERR_INVALID_ARG).
 *  flux           numerical face flux: BATS_FLUX_RUSANOV (Algorithm 1's
 *                 "calc_face_flux" with the Rusanov flux, the default),
 *                 BATS_FLUX_HLL, the two-state Harten-Lax-van Leer flux with
 *                 the wave-speed bounds S_L = min(un_L - cf_L, un_R - cf_R),
 *                 S_R = max(un_L + cf_L, un_R + cf_R), or BATS_FLUX_LINDE, the
 *                 flux of Section 5.1's runs (Linde 2002, cited without its
 *                 formula): HLL with the contact wave restored,
 *                 F = F_HLL - delta alpha S_L S_R / (S_R - S_L) r with
 *                 alpha = minmod((rho_R - rho_L) - (p_R - p_L) / c^2,
 *                 rho_R - rho_L) (the density jump no pressure jump carries,
 *                 at most the density jump itself),
 *                 delta = c / (c + |u_n|), r = (1, u, 0, |u|^2 / 2), u, rho, p
 *                 the means of the two face states and c^2 = gamma p / rho.
 *                 Neither HLL nor Linde is available with `learned` (the
 *                 correction is clipped by the Rusanov dissipation):
 *                 BATS_ERR_INVALID_ARG.
 *  learned_last_only  learned form: 1 = apply the correction in the last
 *                 stage of each two-stage step only (the stage whose fluxes
 *                 make U^{n+1}, and the one whose fine fluxes the training
 *                 target is made of); the first stage then takes the plain
 *                 Rusanov flux.  0 (the default) = both stages. */
typedef struct {
  double gamma;
  int32_t limiter, rk, precision, b0;
  double b0_param[12];
  int32_t powell, learned, persistent, blocks_per_cta;
  int32_t ctas_per_sm, use_graph;
  int32_t local_dt;
  int32_t reflux;
  int32_t flux;
  int32_t learned_last_only;
} bats_physics;

/* Create a solver for n_grids independent grids advanced together (batched
 * launch).  Validates every tree (exact tiling, full face/edge/corner 2:1
 * balance through periodic wraps), builds the per-block neighbour table and
 * the per-level block maps on the host once (the paper's memory-map idea,
 * Section 4.4), and allocates device memory.  cuda_stream: a cudaStream_t, or
 * NULL for a blocking stream owned by the handle (ordered with the legacy
 * default stream).  On success *out owns everything; on failure
 * *out is NULL and the return code says why.  The state is undefined until
 * bats_set_state is called for every grid. */
int bats_create(const bats_grid_desc* grids, int n_grids, const bats_physics* phys, void* cuda_stream,
                bats_t** out);

/* Release the handle and all its device memory.  NULL is ignored. */
void bats_destroy(bats_t* h);

/* Message of the last failure on this handle ("" if none).  With h == NULL,
 * the message of the last failed bats_create in this process. */
const char* bats_last_error(const bats_t* h);

/* Copy the state of grid `grid` from U (host or device; n = 8 * 512 *
 * n_blocks doubles, layout above) and recompute its CFL speed bound.
 * Resets the grid's elapsed time to 0. */
int bats_set_state(bats_t* h, int grid, const double* U, size_t n);

/* Copy the state of grid `grid` into U (host or device, n doubles). */
int bats_get_state(bats_t* h, int grid, double* U, size_t n);

/* All grids at once: U holds every grid's state back to back in grid order,
 * each in the layout above (n = 8 * 512 * total blocks doubles), host or
 * device.  One transfer each way instead of one per grid; the effect is that
 * of bats_set_state / bats_get_state on every grid (elapsed times reset to 0,
 * CFL bounds recomputed).  Both return after the copy has completed. */
int bats_set_states(bats_t* h, const double* U, size_t n);
int bats_get_states(bats_t* h, double* U, size_t n);

/* Advance every grid by n steps of the two-stage scheme (Section 5.2) with
 * dt = cfl / max over non-body cells of sum_d (|u_d| + c_f,d)/dx_d, per grid,
 * from the state at the start of each step.  Each stage fills ghost cells,
 * reconstructs, computes Rusanov fluxes, adds sources and updates
 * (Algorithms 1-2).  The time step never leaves the device.  Returns after the
 * stream is synchronised once at the end; *t_out (nullable) receives grid 0's
 * elapsed time.  BATS_ERR_NONPHYSICAL if any update produced rho <= 0,
 * p <= 0 or NaN (the state is then that of the failing step). */
int bats_step(bats_t* h, int n, double cfl, double* t_out);

/* As bats_step with a fixed dt for every grid. */
int bats_step_dt(bats_t* h, int n, double dt, double* t_out);

/* Time step the next bats_step(cfl) would take for grid `grid`. */
int bats_get_dt(bats_t* h, int grid, double cfl, double* dt);

/* Elapsed simulated time of grid `grid` since its last bats_set_state. */
int bats_get_time(bats_t* h, int grid, double* t);

/* Milliseconds of device time of the last bats_step call, by phase
 * (BATS_PHASE_*), from CUDA events on the handle's stream: ms[0] the stage
 * kernels (events bracket the two stage launches of each step, the mixed
 * form's ghost pre-pass included; beyond 256 steps the first 256 are
 * scaled), ms[1] everything else (time-step bookkeeping kernels), ms[2]
 * total.  Under CUDA-graph replay the stage events are event nodes of the
 * graph, recorded by every replay.  n = entries in ms. */
int bats_get_timings(bats_t* h, double* ms, int n);

/* Debug view of the ghost fill (Section 4.1-4.2) for the current state:
 * writes the padded tiles double [8][n_blocks][12][12][12] of grid `grid`
 * into T (host or device; n doubles).  Only the interior and the six face
 * slabs (the cells the stencil reads) are defined; edge and corner cells are
 * set to 0. */
int bats_debug_fill_ghosts(bats_t* h, int grid, double* T, size_t n);

/* Mixed form (BATS_MIXED handles only, else BATS_ERR_INVALID_ARG): the same
 * view of the FP32 ghost fill, as primitives (rho, u, B1, p) widened to
 * double, same layout.  At resolution changes these are the restriction (the
 * conservative mean of the 8 children) and the prolongation of Section 4.2
 * written in primitive form from the FP32 primitive copies. */
int bats_debug_fill_ghosts_w(bats_t* h, int grid, double* T, size_t n);

/* Debug view of one stage: R = dU/dt of the current state of grid `grid`
 * (fluxes, sources; body cells 0), double [8][n_blocks][8][8][8]. */
int bats_debug_residual(bats_t* h, int grid, double* R, size_t n);

/* Test hook for the bounded device waits (the stage kernel's waits on its
 * bulk-copy barrier give up after about 1 s and report instead of hanging):
 * one CTA waits on a barrier that nothing completes.  Returns
 * BATS_ERR_TIMEOUT after about 1 s; the handle stays usable. */
int bats_debug_wait_timeout(bats_t* h);

/* Launch-form controls (the autotuner's knobs): persistent launch on/off,
 * blocks per work item, CTAs per SM, CUDA-graph replay of whole steps. */
int bats_set_launch(bats_t* h, int persistent, int blocks_per_cta, int ctas_per_sm, int use_graph);

/* Staging layout of the mixed form's plain stage kernel (an autotuner knob;
 * the result is the same either way, bit for bit).  The kernel stages each
 * block's padded stencil (Section 4.1's ghost cells around the block's own
 * cells) in shared memory: the block's 512 cells by one tensor copy (TMA),
 * the face slabs at resolution changes from their precomputed buffer by bulk
 * copies, and the same-level face slabs, with tma = 1 (the default), by one
 * tensor copy each of the neighbour's cells nearest the face, or with
 * tma = 0 gathered by the kernel's threads.  BATS_ERR_INVALID_ARG for other
 * values.  bats_get_staging returns the current value (-1 for NULL). */
int bats_set_staging(bats_t* h, int tma);
int bats_get_staging(const bats_t* h);

/* Measurement helper, no counterpart in the paper: the FP64 FMA throughput of
 * the current device in GFLOP/s (2 flops per FMA), the ceiling of the FP64
 * form's stage kernel, whose FP64 pipe is its bound.  Runs a kernel of
 * independent FMA chains (eight per thread, 8 CTAs of 256 threads per SM)
 * four times on cuda_stream (NULL: the legacy default stream) and returns the
 * best of the last three (CUDA events).  Allocates and frees 8 bytes of
 * device memory.  BATS_ERR_CUDA on a CUDA failure (message: bats_last_error
 * with NULL). */
int bats_fp64_fma_rate(void* cuda_stream, double* gflops);

/* Number of kernels launched by the last bats_step call. */
int bats_get_launch_count(bats_t* h, long long* n);

/* Learned form: number of block-stages, since bats_create, whose learned
 * update left a non-physical cell (rho <= 0, p <= 0 or not finite) and were
 * therefore recomputed with the plain Rusanov flux, the method's own flux
 * (the network only corrects it).  0 for the plain forms.  The count is read
 * back at the end of each bats_step/bats_step_dt call. */
int bats_get_fallbacks(bats_t* h, long long* n);

/* Self-check of the mixed form's integer-only number conversions (no paper
 * counterpart: on GB300 the FP32<->FP64 conversion instructions run on the
 * FP64 unit, so the kernels convert with integer operations instead).  For n
 * host values, f2d_out[i] = the kernels' conversion of f[i] to double and
 * d2f_out[i] = the kernels' conversion of d[i] to float, for comparison with
 * the compiler's conversions.  Allocates and frees its own device buffers. */
int bats_debug_check_conversions(const float* f, const double* d, int n, double* f2d_out, float* d2f_out);

/* Self-check of the network's activation (the learned correction's GELU,
 * tanh form, Hendrycks & Gimpel): y[i] = the kernels' GELU of x[i] as they
 * compute it for the hidden activations -- two values at a time in packed
 * FP32 around tanh.approx.f32, the result rounded to BF16.  variant 0: the
 * fused learned stage and the trainer; variant 1: the inference kernel,
 * which rounds twice the GELU (its next layer's weights halved), returned
 * halved (exact).  n host values; allocates and frees its own device
 * buffers; BATS_ERR_INVALID_ARG for another variant. */
int bats_debug_gelu(const float* x, int n, int variant, float* y);

/* ---- learned flux correction (a small MLP on tensor cores) -------------
 * Network: 40 inputs -> 64 -> 64 -> 8 outputs, tanh-form GELU after the two
 * hidden layers, BF16 weights and activations with FP32 accumulation.
 * Parameters (BATS_MLP_NPARAM floats, row-major [out][in]): W1 [64][40],
 * b1 [64], W2 [64][64], b2 [64], W3 [8][64], b3 [8].
 * Inputs of a face (in the face frame: normal component first, then the next
 * two axes cyclically): the primitives (rho, u, B1, p) of the four cells
 * around the face and the mean of the two reconstructed face states, scaled
 * by rho_ref (mean stencil density) and c_ref (the Rusanov speed cmax):
 * rho/rho_ref, u/c_ref, B1/(sqrt(rho_ref) c_ref), p/(rho_ref c_ref^2).
 * Outputs: the flux correction in the face frame in units of
 * (rho_ref c_ref, rho_ref c_ref^2, sqrt(rho_ref) c_ref^2, rho_ref c_ref^3);
 * each component is clipped to the Rusanov dissipation |cmax (UR - UL)/2| of
 * that face and added to the Rusanov flux.  With all-zero weights the method
 * is the plain Rusanov scheme. */
#define BATS_MLP_NPARAM 7304

/* Install network weights in a solver (host or device pointer, copied) and
 * turn the learned form on for its next steps; params == NULL turns it off.
 * Each stage then runs three launches: face inputs, the network, the fused
 * stage with the correction.  BATS_ERR_INVALID_ARG on a handle created with
 * refluxing or the HLL flux (the correction is defined on the Rusanov flux). */
int bats_set_mlp(bats_t* h, const float* params);

/* Training-data view of grid `grid`: for every face of every block (index
 * ((block * 3 + d) * 576 + line * 9 + f), line = a + 8 b over the two
 * transverse cell indices in increasing axis order, f = 0..8 the face on the
 * low side of cell f along d) the 40 network inputs X (float, host or device,
 * n_faces x 40; nullable) and F (double, n_faces x 10): the plain Rusanov flux
 * (8, x/y/z components) and the face's rho_ref and c_ref, of the current
 * state (stage_input 0) or of the midpoint
 * stage-2 input U* = U + (dt/2) R(U) (stage_input 1, dt > 0).  The state is
 * not changed.  n_faces = 1728 * n_blocks of the grid.  Rusanov handles only
 * (the fluxes are the learned correction's targets): BATS_ERR_INVALID_ARG
 * with BATS_FLUX_HLL. */
int bats_debug_face_data(bats_t* h, int grid, int stage_input, double dt, float* X, double* F, size_t n_faces);

/* Trainer: FP32 master weights, Adam state, GPU forward and backward. */
typedef struct bats_mlp bats_mlp_t;
/* params NULL: seeded initialisation (hidden layers N(0, 1/fan_in), biases and
 * the output layer zero, so the initial network is the plain scheme). */
int bats_mlp_create(const float* params, uint64_t seed, void* cuda_stream, bats_mlp_t** out);
void bats_mlp_destroy(bats_mlp_t* m);
int bats_mlp_set_params(bats_mlp_t* m, const float* params);
int bats_mlp_get_params(bats_mlp_t* m, float* params);
/* Y (n x 8) = network(X (n x 40)); host or device pointers.  The inputs are
 * rounded to BF16; the network runs on the tensor cores (tcgen05, FP32
 * accumulation in tensor memory).  BATS_ERR_TIMEOUT if a bounded device wait
 * ran out (the handle stays usable). */
int bats_mlp_forward(bats_mlp_t* m, const float* X, int64_t n, float* Y);
/* Y (n x 8 floats) = network(Xb), Xb the inputs already rounded to BF16:
 * n rows of 24 words, word j holding inputs 2j (low half) and 2j + 1 (high
 * half), words 20..23 zero -- the layout bats_debug_face_data's inputs take
 * once rounded.  Device pointers, 16-byte aligned, else
 * BATS_ERR_INVALID_ARG.  Queued on the handle's stream without a
 * synchronisation; bats_mlp_sync reports its errors. */
int bats_mlp_forward_bf16(bats_mlp_t* m, const uint32_t* Xb, int64_t n, float* Y);
/* Waits for the handle's stream; BATS_ERR_TIMEOUT if a bounded device wait of
 * a kernel queued since the last check ran out, BATS_ERR_INVALID_ARG for a
 * sample index outside its training set (both cleared). */
int bats_mlp_sync(bats_mlp_t* m);
/* Loss L = (1/(8n)) sum (y - t)^2 over n samples (X n x 40, T n x 8) and its
 * gradient (grad nullable, BATS_MLP_NPARAM floats); inputs are rounded to
 * BF16 as in inference.  Forward and backward products run on the tensor
 * cores (tcgen05, the weight gradients with the samples as the contracted
 * dimension); each CTA (one per SM at most, 128 samples per tile) writes a
 * partial sum and the partials are added in CTA order, so the result is the
 * same bit for bit from call to call on one GPU. */
int bats_mlp_loss_grad(bats_mlp_t* m, const float* X, const float* T, int64_t n, float* grad, double* loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with learning rate lr on
 * the batch; *loss (nullable) receives the loss before the step. */
int bats_mlp_train_step(bats_mlp_t* m, const float* X, const float* T, int64_t n, float lr, double* loss);
/* One epoch of minibatch Adam steps on a training set already on the device:
 * step s (s = 0 .. n_perm / batch - 1) uses samples perm[s * batch] ..
 * perm[s * batch + batch - 1], each a row of X (n x 40 floats) and T (n x 8
 * floats); a ragged rest of perm is not used.  X, T and perm (int64 row
 * indices in [0, n)) are device pointers, else BATS_ERR_INVALID_ARG, as for
 * batch < 1, n_perm < batch or lr < 0.  The steps are queued on the handle's
 * stream and synchronised once, at the end; *mean_loss (nullable) receives the
 * mean over the steps of each step's loss before its update.  An index
 * outside [0, n) contributes nothing and makes the call return
 * BATS_ERR_INVALID_ARG after the epoch (the steps still ran). */
int bats_mlp_train_epoch(bats_mlp_t* m, const float* X, const float* T, int64_t n, const int64_t* perm,
                         int64_t n_perm, int64_t batch, float lr, double* mean_loss);

/* ---- stepping without device allocation --------------------------------
 * No counterpart in the paper: an addition for callers that cannot allocate
 * device memory when they step -- code whose device memory is owned by an
 * external manager, or a runtime that forbids cudaMalloc after start-up.
 * bats_create allocates the state, stage buffers and tables of a handle;
 * bats_step_noalloc instead advances one grid held in the caller's own
 * buffer, and keeps everything else it needs (a block-major copy of the
 * state, the intermediate stage state, the block and level tables, the
 * time-step and error words) in one fixed array in device memory that the
 * library reserves when it is loaded, about 8 MB, held by every GPU that
 * loads the library until the process exits.  It allocates nothing: no
 * device memory and no host heap (the tables are built in about 80 KB of the
 * caller's stack).
 *
 * Limits: at most BATS_NOALLOC_MAX_BLOCKS blocks, and the per-level block
 * maps (sum over levels 0..max of the number of block positions,
 * root[0]*root[1]*root[2]*8^level) at most BATS_NOALLOC_MAX_MAP_ENTRIES;
 * larger grids are rejected with BATS_ERR_INVALID_ARG and a message.  FP64
 * form only (phys->precision must be BATS_FP64, learned 0).  The refluxing
 * and local-time-step options need buffers this entry point does not keep:
 * phys->reflux or phys->local_dt set is rejected with BATS_ERR_INVALID_ARG
 * (never silently ignored).  All three schemes (midpoint, SSP-RK2 and the
 * one-stage BATS_RK_EULER) and all limiters are supported.  The launch
 * fields of phys (persistent, blocks_per_cta, ctas_per_sm, use_graph) are
 * ignored: one CTA per block, eager launches.
 *
 * Arguments: grid, phys as for bats_create (one grid); U the state, host or
 * device, n = 8 * 512 * n_leaves doubles in the layout above, read and then
 * overwritten with the state after `steps` steps; cfl > 0 selects the CFL
 * time step, otherwise the fixed dt > 0 is used; *t_out (nullable) receives
 * the elapsed time; cuda_stream a cudaStream_t or NULL (legacy default
 * stream); err/err_len (nullable) receive a message on failure.  Returns after
 * synchronising the stream.
 *
 * The first call on a device (per process) looks up the device address of
 * the array and sets the stage kernel's shared-memory limit; make that first
 * call before any CUDA stream capture.  If that set-up fails, the call
 * returns BATS_ERR_CUDA and the next call tries the set-up again.  All calls share the one array, which
 * keeps the previous call's contents (each call rewrites what it reads first
 * and clears its counters), so calls whose GPU work overlaps -- from two
 * threads, or on two streams without ordering -- race and corrupt each
 * other's results: serialise them. */
#define BATS_NOALLOC_MAX_BLOCKS 128
#define BATS_NOALLOC_MAX_MAP_ENTRIES 16384
int bats_step_noalloc(const bats_grid_desc* grid, const bats_physics* phys, double* U, size_t n, int steps,
                      double cfl, double dt, double* t_out, void* cuda_stream, char* err, size_t err_len);

#ifdef __cplusplus
}
#endif
#endif /* BATS_H */
