/*
 * lbm.h -- C ABI of the GB300 (sm_103a) coupled lattice Boltzmann solver for
 * N-phase flows with liquid-solid phase change.
 *
 * Method: Huang, Zhan, Chai, Huang, Liu, "A diffuse-interface model for N-phase
 * flows with liquid-solid phase change", arXiv 2603.22902.  Section 2 defines the
 * model (mixture rule eq. 2, continuity with mass source, enthalpy equation and
 * the enthalpy -> (f_l, T) map eq. H, N-phase conservative Allen-Cahn equation
 * with the pairwise source R_p, reduction-consistent free energy, chemical
 * potentials and the surface force F_s); Section 3 the three coupled lattice
 * Boltzmann equations (pressure-based flow LBE with source S and penalty force,
 * total-enthalpy LBE, N phase-field LBEs) on a D2Q9 lattice, c_s^2 = 1/3,
 * dx = dt = 1.
 *
 * Conventions
 *  - Every call returns an int status: LBM_OK (0) or a negative LBM_E* code.
 *    lbm_last_error() returns a message for the last failing call on a handle.
 *  - Fields are row-major [ny][nx] float64 (x fastest), whatever the internal
 *    precision; phi is N such planes, contiguous ([N][ny][nx]).
 *  - where = LBM_HOST: pointers are host memory (pinned or pageable); the call
 *    copies and returns when the data is in place.  where = LBM_DEVICE: pointers
 *    are device memory of the handle's device; the work is queued on the handle's
 *    stream and the call returns without synchronising.
 *  - The handle owns all device memory it allocates; the caller owns every buffer
 *    it passes.  Calls on one handle are not thread-safe; work is stream-ordered.
 *  - No CPU fallback: without a CUDA device every call that needs one fails with
 *    LBM_ECUDA.
 *  - Tracing: the calls that put work on the GPU (lbm_step, lbm_set_fields,
 *    lbm_get_fields, lbm_get_diagnostics, lbm_save_state / lbm_load_state, the batch,
 *    slab and adjoint calls) are NVTX ranges named after the call, in the NVTX domain
 *    "lbm"; a profiler can select a call's kernels by them.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_MAXN 4

/* status codes */
#define LBM_OK 0
#define LBM_EINVAL (-1)    /* invalid argument or parameter set */
#define LBM_ENOMEM (-2)    /* device or host allocation failed */
#define LBM_ECUDA (-3)     /* CUDA runtime error (no device, launch failure, ...) */
#define LBM_EUNSTABLE (-4) /* a non-finite value was found by the diagnostics */
#define LBM_ETIMEOUT (-5)  /* a bounded device-side wait gave up */
#define LBM_ESTATE (-6)    /* call out of order (e.g. step before set_fields) */

/* boundary kinds per side; sides are 0 = x-min, 1 = x-max, 2 = y-min, 3 = y-max */
#define LBM_BC_PERIODIC 0 /* both sides of an axis must be periodic, or neither */
#define LBM_BC_WALL 1     /* half-way bounce-back, no-slip, wetting ghost for phi */
#define LBM_BC_OUTFLOW 2  /* y sides only: incoming populations copied along the boundary row */
#define LBM_T_ADIABATIC 0
#define LBM_T_DIRICHLET 1 /* y-side walls only: non-equilibrium extrapolation (Section 4.1) */

/* arithmetic / storage precision of the populations */
#define LBM_FP64 0  /* FP64 storage and arithmetic (the parity path) */
#define LBM_FP32 1  /* FP32 storage and arithmetic */
#define LBM_FP16S 2 /* FP16 storage of shifted populations, FP32 arithmetic */
#define LBM_BF16S 3 /* BF16 storage of shifted populations, FP32 arithmetic */
#define LBM_DF64 4  /* double-word (FP32 pair, ~48-bit) storage and arithmetic on the FP32
                       pipes, the enthalpy map in FP64 where it decides f_l; held to the
                       FP64 parity bar; 32x8 tiles only (batches too) */

#define LBM_HOST 0
#define LBM_DEVICE 1

typedef struct lbm_handle lbm_handle;

typedef struct {
    int nx, ny; /* lattice size, >= 3 each */
} lbm_grid;

/* Liquid and solid properties of one phase (eq. 2: density, viscosity, thermal
 * conductivity, heat capacity) and its specific latent heat (Section 2, H = C_p T +
 * L f_l); latent = 0 marks a phase that never changes phase (ambient, impurities). */
typedef struct {
    double rho_l, rho_s;
    double mu_l, mu_s;
    double lambda_l, lambda_s;
    double cp_l, cp_s;
    double latent;
} lbm_phase;

/* Thermal and body-force parameters.  T_sol <= T_liq are the solidus and liquidus
 * temperatures of eq. H; rho_ref and cp_ref the reference density and heat capacity
 * of the enthalpy LBE (Section 3; cp_ref = 0 selects 2 c_s c_l / (c_s + c_l) of
 * phase 0); u_solid the solid velocity u_s of the penalty force; accel a body
 * acceleration (the body force G = rho accel). */
typedef struct {
    double T_sol, T_liq;
    double rho_ref, cp_ref;
    double u_solid[2];
    double accel[2];
} lbm_thermal;

/* Boundary description.  wet_cos[side][p*LBM_MAXN+q] = cos(theta_pq) of the wall on
 * that side (antisymmetric in p, q; 0 = neutral wetting); it enters the ghost value
 * of phi_p beyond the wall: phi_p + (4/eps) sum_q cos(theta_pq) phi_p phi_q. */
typedef struct {
    int kind[4];
    int tkind[4];
    double T_wall[4];
    double wet_cos[4][LBM_MAXN * LBM_MAXN];
} lbm_bc;

/* Numerical parameters: interface width eps and mobility M (Section 3:
 * M = c_s^2 (tau_g - 1/2)); pairwise surface tensions sigma[p*LBM_MAXN+q] (symmetric,
 * zero diagonal; beta_pq = 3 sigma_pq / eps, k_pq = -3 eps sigma_pq / 4, Section 2);
 * precision = LBM_FP64 / LBM_FP32 / LBM_FP16S / LBM_BF16S / LBM_DF64; diag_every = K > 0 makes
 * lbm_step run the non-finite check every K steps (0 = only when asked). */
typedef struct {
    double eps, mobility;
    double sigma[LBM_MAXN * LBM_MAXN];
    int precision;
    int diag_every;
} lbm_numerics;

/* Diagnostics of the current state: per-phase volume sum_x phi_p, per-phase solid
 * volume sum_x f_s phi_p, max_x |sum_p phi_p - 1|, count of non-finite cells. */
typedef struct {
    double mass[LBM_MAXN];
    double solid[LBM_MAXN];
    double max_sum_dev;
    long long nonfinite;
    long long steps;
} lbm_diag;

/* Create a solver for N phases (2 <= N <= LBM_MAXN) on the current CUDA device.
 * Checks the parameters (tau_f, tau_g, tau_h > 1/2 for every phase, sigma symmetric
 * with zero diagonal, boundary combinations), derives beta_pq, k_pq and c_p,ref on
 * the host and allocates two population sets of 9 (N + 2) planes and two sets of
 * 3 + 2N lagged planes.  *out is set to NULL on failure.  The state is undefined
 * until lbm_set_fields. */
int lbm_create(const lbm_grid* grid, int N, const lbm_phase* phases, const lbm_thermal* thermal,
               const lbm_bc* bc, const lbm_numerics* numerics, lbm_handle** out);

/* Queue all later work of the handle on `stream` (a cudaStream_t; NULL = default).
 * A service of the library: the paper has no counterpart. */
int lbm_set_stream(lbm_handle* h, void* stream);

/* Initial state at t = 0 from phi [N][ny][nx], T, ux, uy (ux / uy may be NULL = 0):
 * rho H from the inverse of eq. H (a cell at or above T_liq is liquid), p = 0,
 * every population at its equilibrium, mdot' = Q' = 0, psi' = psi, (phi u)' = phi u.
 * Resets the step counter. */
int lbm_set_fields(lbm_handle* h, const double* phi, const double* T, const double* ux,
                   const double* uy, int where);

/* Advance nsteps fused time steps (one kernel launch per step on the handle's
 * stream; asynchronous unless diag_every > 0, which synchronises every K steps and
 * returns LBM_EUNSTABLE when a non-finite value appears). */
int lbm_step(lbm_handle* h, long nsteps);

/* Macroscopic fields of the current state (NULL = skip): phi [N][ny][nx], T,
 * specific enthalpy H = (rho H) / rho, liquid fraction f_l, velocity u and pressure p
 * (computed from the current populations exactly as the step computes them). */
int lbm_get_fields(lbm_handle* h, double* phi, double* T, double* H, double* fl, double* ux,
                   double* uy, double* p, int where);

/* Diagnostics of the current state (synchronises the handle's stream): the quantities
 * behind the paper's conservation claims, measured on the lattice.  Per-phase volume
 * sum_x phi_p: conserved to round-off without phase change (the conservative Allen-Cahn
 * LBE of Section 3 with the source phi_p mdot, Section 2; mass conservation of the
 * N-phase model stated in the Conclusions), and its change on freezing the volume change
 * of Section 4.1 (Table 1: h_f / h_0 = rho_l / rho_s).  Per-phase solid volume
 * sum_x f_s phi_p: the frozen amount (eq. H, f_s = 1 - f_l).  max_x |sum_p phi_p - 1|: the
 * constraint sum_p phi_p = 1 that the pairwise R_p keeps (Section 2, reduction
 * consistency).  Non-finite count: a cell whose sum_p phi_p, rho H or f_0 is not finite. */
int lbm_get_diagnostics(lbm_handle* h, lbm_diag* out);

/* Raw state (a service of the library for checkpoint and restart; the paper has no
 * counterpart): *bytes receives the size of the checkpoint; buf may be NULL to query.
 * lbm_save_state copies populations, lagged planes and the step counter to host
 * memory; lbm_load_state restores them on a handle created with the same grid, N and
 * precision. */
int lbm_save_state(lbm_handle* h, void* buf, size_t* bytes);
int lbm_load_state(lbm_handle* h, const void* buf, size_t bytes);

/* Steps taken since lbm_set_fields / lbm_load_state. */
long long lbm_get_steps(const lbm_handle* h);

/* Bounds-check record of a library built with -DLBM_CHECK_BOUNDS (every global load
 * and store of the kernels checks its index against its buffer; a violation is counted
 * and skipped, never trapped): out3 = {violations, site code of the first, its index}.
 * Synchronises the handle's stream.  Returns LBM_EINVAL in normal builds. */
int lbm_debug_bounds(lbm_handle* h, long long* out3);

/* Tile shape (bx, by) of the fused step kernel; 0, 0 restores the default (32x8).  The
 * shape must be one of the compiled variants, 32x8, 32x4, 64x4 or 16x16, and 32x8 for
 * an LBM_DF64 handle (LBM_EINVAL otherwise).  Results of different shapes agree to
 * rounding, not bit for bit (each shape is compiled on its own). */
int lbm_set_tile(lbm_handle* h, int bx, int by);


/* Step with its inputs staged in shared memory by the tensor-memory accelerator: one
 * block per 32x8 tile, whose thread 0 copies the tile's populations and lagged values
 * (tile and ring) with six tensor copies; the tile is then computed from shared memory
 * (the arithmetic is that of lbm_step, cell by cell, bit for bit); positions beyond the
 * lattice are filled with zeros by the copies and, across a periodic side, read again
 * from the cells they wrap to.  A service of the library for LBM_FP16S and LBM_BF16S
 * handles with N = 2 or 3, nx a multiple of 8 and the 32x8 tile, where it is on from
 * lbm_create (a handle whose tensor maps cannot be encoded runs the
 * one-launch form).  on = 0 returns to the one-launch form, on = 1 asks for the staged one
 * (LBM_EINVAL where it does not apply, LBM_ECUDA when the tensor maps cannot be encoded);
 * lbm_set_tile with another shape turns it off.  Every wait for the copies is bounded; a
 * wait that gave up is reported as LBM_ETIMEOUT by the next lbm_step with diag_every > 0
 * or lbm_get_diagnostics, with the state undefined. */
int lbm_set_staging(lbm_handle* h, int on);

/* Diagnostics sums without any allocation, for callers that cannot allocate device
 * memory when they need them: a host that owns all device memory through its own arena
 * or pool and forbids other allocators, a service whose device memory is fixed when it
 * starts, a timed loop that forbids allocation latency.
 * (The paper has no counterpart: this is a service of the library.)
 * Inputs are caller-owned device fields of one lattice: phi [N][ny][nx] and the liquid
 * fraction fl [ny][nx] (as written by lbm_get_fields with LBM_DEVICE); out is a
 * caller-owned device array of 2N + 2 doubles that receives, as lbm_get_diagnostics does,
 * sum_x phi_p (N values), sum_x (1 - fl) phi_p (N values), max_x |sum_p phi_p - 1| and the
 * count of non-finite cells.  That count looks only at the fields passed in: a cell counts
 * when fl or sum_p phi_p is not finite (lbm_get_diagnostics also looks at rho H and the rest
 * population of f, which are not inputs here).  The work is queued on `stream` (a cudaStream_t, NULL = the
 * default stream) and the call returns without synchronising.
 * The block partial sums live in a fixed array of 608 x 10 doubles (48.6 KiB) in the
 * library's device image, which every GPU that loads the library holds until the process
 * exits; any lattice up to 2^31 cells fits in it (a grid-stride loop caps the number of
 * blocks at 608).  N > LBM_MAXN, a lattice beyond 2^31 cells or a NULL pointer is
 * rejected with LBM_EINVAL and a message in lbm_last_error(NULL).  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  All calls share the array, so
 * calls whose work overlaps on the GPU (other streams, other host threads) race; calls
 * on one stream are ordered and safe.  The looked-up address holds for the life of the
 * device's primary context: do not use this call across a cudaDeviceReset.  A CUDA error
 * already pending from earlier work makes the call return LBM_ECUDA without launching
 * (the error is left pending for its owner).  No cudaMalloc, cudaFree or allocating
 * library routine is called. */
int lbm_field_sums_noalloc(const double* phi, const double* fl, int nx, int ny, int N, double* out,
                           void* stream);

/* Measured FP64 instruction rate of the current device, the roofline of the FP64 step
 * (bound by the FP64 pipe, not by HBM): eight independent chains of FP64 fused
 * multiply-adds per thread, 8 blocks of 256 threads per SM, timed with CUDA events, the
 * best of 5 launches after 3 untimed ones.  *ginst_per_s receives FP64 thread-instructions
 * per second in units of 1e9 (one FMA = 2 flop), *ms (may be NULL) the best launch time.
 * Allocates and frees a small device buffer; synchronises the device.  A measurement
 * service of the library (the paper has no counterpart). */
int lbm_measure_fp64_rate(double* ginst_per_s, double* ms);

/* Message of the last failing call on h.  With h = NULL: the message of the calling
 * thread's last failing call that has no handle (lbm_create, lbm_field_sums_noalloc);
 * each host thread keeps its own.  Never NULL. */
const char* lbm_last_error(const lbm_handle* h);

void lbm_destroy(lbm_handle* h);

/* ---- y slabs: one lattice as bands of rows, one handle per band -------------------------
 * The fused step (Section 3) is a one-cell stencil in every field, so a lattice cut into
 * bands of rows steps exactly like the whole lattice when, after every step, each cut is
 * crossed by two messages per direction:
 *   phase 1: the populations that the step pushed across the cut (the three directions
 *            with c_y across it, of every species: 3 (N + 2) rows of nx values);
 *   phase 2: the boundary row's phase-field and enthalpy populations (all nine directions,
 *            9 (N + 1) rows) and its lagged mdot' and Q' (2 rows): the inputs from which
 *            the next step's stencil ring recomputes phi_p, rho and psi.
 * A slab handle holds rows [y0, y1) plus one ghost row beyond each cut side; the ghost
 * rows are stepped too, and the exchange overwrites what they get wrong.  The same calls
 * serve two handles on one GPU (a device-to-device copy of the message) and handles on
 * different GPUs (NCCL send / receive of the packed buffers).  The paper solves one
 * lattice on one machine; this is a service of the library for lattices that do not fit
 * one GPU. */

/* A handle for rows [y0, y1) of the lattice `grid` with the global parameters.  A side
 * of the band is a cut where another band continues the lattice: y0 > 0, y1 < ny, or
 * either when the y sides are periodic.  A cut side gets a ghost row and is declared an
 * adiabatic, neutrally wetting wall of the band's own lattice (it touches only the ghost
 * row); the other side keeps the global boundary rule.  The band's lattice has
 * (y1 - y0) + ghosts rows, at least 3.  lbm_set_fields takes that lattice's fields: global
 * rows y0 - 1 .. y1 (wrapped when periodic, without the rows beyond a global side).
 * lbm_get_fields returns them, ghost rows included; lbm_slab_sums gives the diagnostics
 * sums over the band's own rows (lbm_get_diagnostics would count the ghost rows).  Errors
 * as lbm_create; y0, y1 out of range or a band without a cut is LBM_EINVAL. */
int lbm_slab_create(const lbm_grid* grid, int y0, int y1, int N, const lbm_phase* phases,
                    const lbm_thermal* thermal, const lbm_bc* bc, const lbm_numerics* numerics,
                    lbm_handle** out);

/* out4 = {rows of the band's lattice, ghost row below (0/1), ghost row above (0/1), y0}. */
int lbm_slab_geometry(const lbm_handle* h, int* out4);

/* Bytes of one message of `phase` (1 or 2) through one cut (rows padded to 16 bytes);
 * -1 for a handle that is not a slab or a bad phase. */
long long lbm_slab_message_bytes(const lbm_handle* h, int phase);

/* Pack the message of `phase` that the handle sends through its cut side `side` (2 = y-min,
 * 3 = y-max) into the device buffer msg; unpack the message that arrives through that
 * side.  Per step, in this order: lbm_step on every band; phase 1 packs of every cut, then
 * the transfers, then phase 1 unpacks; the same for phase 2.  The message that a band
 * packs on its y-max side is unpacked by the band above on its y-min side, and the other
 * way round.  Queued on the handle's stream; no synchronisation.  A side that is not a cut
 * is LBM_EINVAL. */
int lbm_slab_pack(lbm_handle* h, int side, int phase, void* msg);
int lbm_slab_unpack(lbm_handle* h, int side, int phase, const void* msg);

#define LBM_SLAB_INNER 1   /* tile rows clear of the band's first two and last two rows */
#define LBM_SLAB_EDGE 2    /* the other tile rows; completes the step */
/* One step of a slab handle in two launches, for overlapping the halo exchange with the
 * step: part LBM_SLAB_INNER steps the tile rows whose rows and one-cell ring avoid the
 * band's first two and last two rows (the ghost and boundary rows that the exchange
 * writes), part LBM_SLAB_EDGE the other tile rows, and then the step is complete (as one
 * lbm_step: ping-pong sets flipped, step count + 1).  Each destination slot of the step is
 * written by one cell, so the two parts together equal lbm_step bit for bit.  The
 * exchange of step t reads and writes only the band's edge rows of the set that step t
 * wrote, which the inner part of step t + 1 neither reads nor writes: the order per step
 * may be inner part of step t + 1, exchange of step t (on another stream, after the edge
 * part of step t), edge part of step t + 1 (after the exchange).  Calls out of order
 * (LBM_SLAB_EDGE without LBM_SLAB_INNER, two LBM_SLAB_INNER, lbm_step between them) are
 * LBM_ESTATE; a handle that is not a slab or another part is LBM_EINVAL.  Queued on the
 * handle's stream; no synchronisation. */
int lbm_slab_step_part(lbm_handle* h, int part);

/* The diagnostics of lbm_get_diagnostics over the band's own rows, into host memory
 * out[2N + 2]: sum phi_p (N), sum (1 - f_l) phi_p (N), max |sum_p phi_p - 1| and the count of
 * non-finite cells.  Adding the sums and counts and taking the maximum of the deviation
 * over all bands gives the lattice's diagnostics.  Synchronises the stream. */
int lbm_slab_sums(lbm_handle* h, double* out);

/* ---- gradients: the adjoint of the FP64 step -------------------------------------------
 * Loss of the liquid fraction after nsteps steps from given initial fields:
 *     L = sum_x w(x) (phi_pcm(x) f_l(x) - f_target(x))^2,  w = 1 when weight is NULL,
 * where phi_pcm = sum_p phi_p over the phases with latent > 0: the liquid fraction of
 * the phase-changing material (f_l itself jumps from 1 to 0 across a band of width
 * ~phi_pcm in rho H, so unweighted it has no useful derivative where phi_pcm -> 0);
 * and its gradient with respect to the parameters of the run: the Dirichlet wall
 * temperatures (Section 4.1), the latent heat per volume rho_l^p L_p of each phase
 * (through eq. H; the Stefan number sets L_p = c_p,s (T_m - T_w,ref) / Ste), and the
 * liquid and solid conductivities of each phase (eq. 2, through tau_h of the enthalpy
 * LBE, Section 3). */
typedef struct {
    double loss;
    double T_wall[4];                  /* dL / dT_wall[side] (sides without a Dirichlet wall: 0) */
    double rhoL[LBM_MAXN];             /* dL / d(rho_l^p L_p) */
    double lambda_s[LBM_MAXN];         /* dL / d lambda_s^p */
    double lambda_l[LBM_MAXN];         /* dL / d lambda_l^p */
} lbm_fl_grad;

/* Run the handle from phi0, T0, ux0, uy0 (as lbm_set_fields; ux0 / uy0 may be NULL)
 * for nsteps steps, then evaluate L and its gradient by the hand-written reverse of
 * the fused step (discrete adjoint).
 * - The kinks of eq. H take the derivative of the branch the forward step took.
 * - The forward run keeps a copy of the state every checkpoint_every steps. The
 *   reverse sweep recomputes one segment at a time from its checkpoint, stores its
 *   states, and steps the adjoint back through them.
 * - Device memory: (nsteps / checkpoint_every + checkpoint_every + 2) states plus
 *   20 + 11 N planes of doubles, allocated for the duration of the call.
 * - FP64 handles only (LBM_EINVAL otherwise). fl_target and weight are [ny][nx] like
 *   the fields, in host or device memory per `where`.
 * - On return the handle holds the state after nsteps steps. Synchronises. */
int lbm_adjoint_fl_loss(lbm_handle* h, const double* phi0, const double* T0, const double* ux0,
                        const double* uy0, const double* fl_target, const double* weight, int where,
                        long nsteps, int checkpoint_every, lbm_fl_grad* out);

/* ---- batches of independent cases ----------------------------------------------------
 * Many independent problems, each created by lbm_create (its own grid, phase properties,
 * thermal parameters and boundary spec, Section 4), advanced together.  The paper solves
 * one problem at a time; this is a throughput service of the library.
 * - Every tile of every case is one item of a flat work list, so cases of uneven sizes
 *   fill the GPU together.
 * - The per-cell arithmetic is that of lbm_step.
 * - Each case keeps its own handle. Fields, diagnostics and state I/O go through the
 *   lbm_* calls on that handle.
 * - A handle may also be stepped alone between batch steps.
 * - The batch does not own the handles. They must outlive it. */
typedef struct lbm_batch lbm_batch;

#define LBM_BATCH_PERSISTENT 0 /* one cooperative launch per tile-shape group and call;
                                  grid barrier between steps */
#define LBM_BATCH_PER_STEP 1   /* one launch per tile-shape group and step */
#define LBM_BATCH_STAGED 2     /* the per-step form, with every tile of a 32x8-tile group
                                  computed from a TMA-staged copy of its inputs (the staged
                                  step of lbm_set_staging) where the group allows it: policy
                                  LBM_FP16S or LBM_BF16S, N = 2 or 3, every case's nx a multiple
                                  of 8; other groups run the per-step form.  Its
                                  arithmetic is the per-step form's; the kernels are separate
                                  instantiations, so a stored 16-bit value may differ by one
                                  unit of the format. */
/* Every form: the launches of a call are captured into a CUDA graph the first time a
 * call of that length runs, and the graph is replayed by later calls of that length. */

/* Size classes of a case, by cells nx * ny: <= 128^2, <= 256^2, <= 384^2, larger. */
#define LBM_BATCH_CLASSES 4

typedef struct {
    int mode;                          /* LBM_BATCH_PERSISTENT, LBM_BATCH_PER_STEP or LBM_BATCH_STAGED */
    int blocks_per_sm;                 /* persistent grid: resident blocks per SM, 0 = all that fit */
    int tile[LBM_BATCH_CLASSES][2];    /* tile (bx, by) per size class: 32x8, 64x4 or 16x16 */
    int graph;                         /* out: 1 when the calls replay a CUDA graph */
} lbm_batch_plan;

/* Build a batch over ncases handles, owned by the caller.
 * - All handles live on the current device and share N and the precision policy
 *   (LBM_DF64 batches use 32x8 tiles only: lbm_batch_set_plan refuses other shapes).
 * - Every handle must have been given fields (lbm_set_fields).
 * - The initial plan is persistent, 32x8 tiles for every class, all blocks that fit.
 * - Errors: LBM_EINVAL for mixed N or precision, a NULL or repeated handle, or
 *   ncases < 1; LBM_ESTATE when a handle has no fields; LBM_ENOMEM.
 * - Messages are in lbm_batch_last_error(NULL). */
int lbm_batch_create(int ncases, lbm_handle* const* cases, lbm_batch** out);

/* Stream of the batch's launches (a cudaStream_t; NULL = the legacy default stream). */
int lbm_batch_set_stream(lbm_batch* b, void* stream);

/* Replace the plan. A tile shape that is not 32x8, 64x4 or 16x16 is LBM_EINVAL. */
int lbm_batch_set_plan(lbm_batch* b, const lbm_batch_plan* plan);
int lbm_batch_get_plan(const lbm_batch* b, lbm_batch_plan* plan);

/* Advance every case by nsteps steps (Section 3), queued on the batch stream, without
 * synchronising.
 * - Each handle's step count and current state follow.
 * - Work queued on a handle's own stream must be ordered with the batch stream by the
 *   caller (the same stream for both is simplest).
 * - In the persistent mode a step waits for every block of its launch. A wait gives up
 *   after 2^21 polls (about a second; more for groups above 16M cells), and the next
 *   lbm_batch_sync reports LBM_ETIMEOUT. */
int lbm_batch_step(lbm_batch* b, long nsteps);

/* Bound of every grid-barrier wait of the persistent form, in polls (0 = the default:
 * 2^21 polls, or one per 8 cells of the largest group).  A service for tests of the
 * timeout path and for callers that want a step to fail fast rather than wait about a
 * second: with a bound of a few polls the first wait gives up, every block of the launch
 * leaves at its next barrier, the state of the cases is left partly stepped (undefined)
 * and the next lbm_batch_sync returns LBM_ETIMEOUT and resets the barrier.  Waits for the
 * batch's queued work first.  polls < 0 is LBM_EINVAL. */
int lbm_batch_set_wait_limit(lbm_batch* b, long long polls);

/* Wait for the batch's queued work. Returns LBM_OK, LBM_ETIMEOUT (a grid-barrier wait of
 * the persistent form, or a wait of the staged form for its tensor copies, gave up; the
 * barrier is reset, the state undefined) or LBM_ECUDA. */
int lbm_batch_sync(lbm_batch* b);

/* Tune the plan on the current state and set the best one (also written to *best
 * when best is not NULL).
 * - Candidates: each launch mode (LBM_BATCH_STAGED where a group allows it); each tile
 *   shape per size class present; fewer resident blocks per SM.
 * - Each candidate is timed over trial_steps steps (>= 1) with CUDA events, after one
 *   untimed call of the same length.
 * - The state of every case, and its step count, are restored afterwards.
 * - Allocates a copy of all states for the duration of the call. Synchronises. */
int lbm_batch_autotune(lbm_batch* b, int trial_steps, lbm_batch_plan* best);

/* Message of the last failing call on b (or of lbm_batch_create when b is NULL). */
const char* lbm_batch_last_error(const lbm_batch* b);

void lbm_batch_destroy(lbm_batch* b);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
