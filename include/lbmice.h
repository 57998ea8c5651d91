/*
 * lbmice.h -- C ABI of the GB300 (sm_103a) coupled lattice-Boltzmann ice-crystal step.
 *
 * Method: Tan, Hosseini, Seidel-Morgenstern, Thevenin, Lorenz, "Modeling ice crystal growth
 * using the lattice Boltzmann method" (arXiv 2101.07163), Sec. 2.2. One call of
 * lbmice_step(h, 1) advances, in one fused CUDA kernel, the three D2Q9 lattices of one grid:
 *   - flow f (Sec. 2.2.1): BGK collision towards the second-order Hermite equilibrium at the
 *     solid-damped velocity u* = (1 - phi)/2 u, plus the solid drag
 *     F = -h eta_f (1 + phi)^2 (1 - phi) u / (4 W0^2), h = 2.757, by Guo forcing;
 *   - vapour supersaturation g (Sec. 2.2.2): advection-diffusion BGK with
 *     g^eq = w U (1 + c.u* / c_s^2), tau_g = D q(phi)/c_s^2 + 1/2, q = 1 - phi, and the
 *     phase-change source -w (L_sat/2) d(phi)/dt;
 *   - phase field h (Sec. 2.2.3, Eq. (d), Eq. (e)): the modified LB update with the a_s^2
 *     time factor, source Q = phi - phi^3 + lambda U (1 - phi^2)^2, and anisotropy
 *     a_s = 1 + eps cos(6 theta) from the E4 isotropic gradient of phi (Sec. 3.1.1,
 *     Table 1).
 * Options (lbmice_params): the gradient stencil E2, E4, E6 or E8 (Sec. 3.1.1), the four-fold
 * anisotropy of the validation system (Sec. 3.1.2), and FP16 or BF16 storage of the
 * populations as deviations from their FP32 moments (arithmetic stays FP32).
 * Unit conventions: W0, tau0, dx, dt and D share one unit system (the paper's validation
 * units are W0 = tau0 = 1, dx = 0.4, dt = 0.008, Sec. 3.1.2); u_in and nu are in lattice
 * units (dx/dt, dx^2/dt).
 *
 * Conventions of every entry point:
 *   - Return LBMICE_OK (0) on success, a negative LBMICE_E* code on failure; no C++
 *     exception crosses the ABI. lbmice_strerror() names a code.
 *   - The handle owns all device memory it allocates; the caller owns every buffer it
 *     passes in. Pointers marked "device" must be CUDA device pointers on the handle's
 *     device; "host" pointers may be pageable or pinned.
 *   - All GPU work is enqueued on the stream given to lbmice_create (0 = the legacy default
 *     stream). Calls that return data to host memory synchronise that stream; the others
 *     are asynchronous unless stated.
 *   - A handle is not thread-safe: one host thread at a time per handle.
 *   - Fields are row-major float arrays of ny rows and nx columns (element (x, y) at
 *     y * nx + x), unless stated otherwise.
 *   - D2Q9 order of populations: c = (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1)
 *     (1,-1).
 */
#ifndef LBMICE_H_
#define LBMICE_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ----------------------------------------------------------------------- */
#define LBMICE_OK 0
#define LBMICE_EINVAL (-1)     /* bad argument: null pointer, size, range, buffer length */
#define LBMICE_ECUDA (-2)      /* a CUDA runtime call or kernel launch failed */
#define LBMICE_ENOMEM (-3)     /* device or pinned host allocation failed */
#define LBMICE_ENONFINITE (-4) /* a NaN or Inf was found in phi, U or rho */
#define LBMICE_EUNSTABLE (-5)  /* derived relaxation time <= 1/2 or inflow >= sound speed */
#define LBMICE_ETIMEOUT (-6)   /* a bounded device-side wait gave up */
#define LBMICE_ENOTSUP (-7)    /* the call needs the checked build (LBMICE_CHECKED)         */

/* ---- boundary kinds of the four faces (Sec. 3.1.3, Sec. 3.2.2) --------------------------
 * PERIODIC: wrap (must be set on both faces of an axis).
 * INLET:    ghost nodes hold vapour (phi = -1, a_s = 1) at U_in, with the flow equilibrium
 *           at the adjacent node's density and velocity u_in along the inward normal.
 * OUTLET:   zero-gradient: ghost nodes copy the adjacent node.
 * FREESLIP: specular wall: ghost nodes are the mirror image of the adjacent node.        */
#define LBMICE_BC_PERIODIC 0
#define LBMICE_BC_INLET 1
#define LBMICE_BC_OUTLET 2
#define LBMICE_BC_FREESLIP 3

/* ---- field selectors of lbmice_fields / lbmice_load ------------------------------------ */
#define LBMICE_FIELD_PHI 0      /* phi = sum h (Sec. 2.2.3)                   float[ny][nx] */
#define LBMICE_FIELD_U 1        /* U = sum g (Sec. 2.2.2)                     float[ny][nx] */
#define LBMICE_FIELD_RHO 2      /* rho = sum f (Sec. 2.2.1); 1 without flow   float[ny][nx] */
#define LBMICE_FIELD_UX 3       /* u*_x = (1-phi)/2 j_x/(rho + k/2)           float[ny][nx] */
#define LBMICE_FIELD_UY 4       /* u*_y                                       float[ny][nx] */
#define LBMICE_FIELD_PHI_PREV 5 /* phi one step earlier (d(phi)/dt history)   float[ny][nx] */
#define LBMICE_FIELD_POPS 6     /* populations, planes h0..h8, g0..g8 and, with flow,
                                   f0..f8: float[18 or 27][ny][nx] (decoded to float for
                                   16-bit storage)                                         */
#define LBMICE_FIELD_STATE 7    /* the whole state in its storage format, opaque bytes
                                   (lbmice_state_bytes); loading it restores a run exactly */

/* ---- storage of the populations (16-bit forms halve the traffic; arithmetic is FP32) ---
 * F32:  every population as float (224 B moved per node update with all three lattices).
 * F16, BF16: per lattice the zeroth moment (phi, U, rho) as float and the 8 moving
 *       populations as 16-bit deviations p_a - w_a M from the local rest state; the rest
 *       population is rebuilt as w_0 M - sum of deviations, so the moments are stored
 *       exactly (124 B moved per node update with all three lattices).                   */
#define LBMICE_STORAGE_F32 0
#define LBMICE_STORAGE_F16 1
#define LBMICE_STORAGE_BF16 2

#define LBMICE_NSTATS 6

/* ---- parameters (Sec. 2.1, Sec. 2.2, Sec. 3) -------------------------------------------- */
typedef struct lbmice_params {
  int32_t nx, ny;       /* grid nodes, each >= 4, with pitch * ny < 2^31 (pitch = nx rounded
                           up to 32); larger offsets are 64-bit throughout                 */
  double dx, dt;        /* grid and time step (default 0.4, 0.008)                         */
  double W0, tau0;      /* interface width and time (default 1, 1)                         */
  double D;             /* vapour diffusivity (default 2)                                  */
  double lambda;        /* coupling; <= 0 selects tau0 D / (a2 W0^2), a2 = 0.6267 (beta = 0)*/
  double L_sat;         /* vapour absorption rate at the interface (default 1)             */
  double eps;           /* six-fold anisotropy strength eps_xy, 0 <= eps < 1 (default 0.05)*/
  double kappa_N;       /* factor of the anisotropic flux: 1 = a_s da_s/d(grad phi)
                           (default), 2 = the printed d(a_s^2)/d(grad phi)                 */
  double U_in;          /* supersaturation carried in by an INLET face                     */
  double u_in;          /* inflow speed, lattice units, along the inlet's inward normal    */
  double nu;            /* kinematic viscosity, lattice units (default 0.016)              */
  int32_t bc[4];        /* faces -x, +x, -y, +y: LBMICE_BC_*                               */
  int32_t flow;         /* 1: evolve the flow lattice f; 0: fluid at rest, f not stored    */
  int32_t check_every;  /* lbmice_step checks for NaN/Inf every this many steps (0: never) */
  int32_t storage;      /* LBMICE_STORAGE_* (default F32)                                  */
  int32_t stencil;      /* gradient of phi (Sec. 3.1.1): 2 central difference, 4, 6 or 8 the
                           isotropic stencils of Table 1 (default 4; 0 also means 4)       */
  int32_t fold;         /* anisotropy symmetry: 6 (ice, Sec. 2.1, default; 0 also) or 4 (the
                           four-fold validation system)                                    */
} lbmice_params;

typedef struct lbmice_ctx lbmice_t;

/* Fill *p with the defaults above for an nx x ny periodic grid without flow.
 * Returns LBMICE_EINVAL if p is null. */
int lbmice_params_default(lbmice_params* p, int32_t nx, int32_t ny);

/* Validate *p, derive the lattice constants (Sec. 2.1 beta = 0 lambda, Sec. 2.2.1
 * tau_f = nu/c_s^2 + 1/2), allocate the state on the current CUDA device and return a
 * handle in *out. stream: a cudaStream_t (0 = legacy default stream); all work of the
 * handle runs on it. Errors: EINVAL (null, size, face kinds, unpaired PERIODIC, eps range),
 * EUNSTABLE (tau_f <= 1/2 with flow, |u_in| >= 1/sqrt(3)), ENOMEM, ECUDA. On error *out is
 * set to NULL and nothing is leaked. The state is zero until an init call. */
int lbmice_create(const lbmice_params* p, void* stream, lbmice_t** out);

/* Initial condition of Sec. 3.1.2 / Sec. 3.2: circular seed of radius R0 cells centred at
 * (cx, cy) (node coordinates), phi = tanh((R0 - r) dx / (sqrt(2) W0)), uniform U = U0,
 * rho = 1, velocity u_in along the inlet normal times the liquid fraction (1 - phi)/2
 * (zero without an inlet). Populations are set to the equilibria of these moments and the
 * phi history to phi. Asynchronous. Errors: EINVAL, ECUDA. */
int lbmice_init_seed(lbmice_t* h, double cx, double cy, double R0, double U0);

/* Initial condition from moment fields: double arrays [ny][nx] (host or device, per
 * on_device). phi and U are required; rho (default 1), ux, uy (default 0) may be NULL and
 * are ignored when params.flow = 0 (the fluid is at rest).
 * Populations become the equilibria of (phi, U, rho, u) -- h^eq of Eq. (e) with the
 * anisotropic flux of phi's E4 gradient, g^eq of Sec. 2.2.2, f^eq of Sec. 2.2.1 -- and the
 * phi history is set to sum h. Host arrays are copied before the call returns (the stream
 * is synchronised); device arrays are read asynchronously. Errors: EINVAL, ENOMEM, ECUDA. */
int lbmice_set_fields(lbmice_t* h, const double* phi, const double* U, const double* rho,
                      const double* ux, const double* uy, int32_t on_device);

/* Advance nsteps >= 0 time steps (one fused kernel per step; chunks of steps are replayed
 * as CUDA graphs). Asynchronous unless params.check_every > 0, in which case the stream is
 * synchronised every check_every steps and LBMICE_ENONFINITE is returned as soon as a NaN or
 * Inf appears in phi, U or rho. Errors: EINVAL, ECUDA, ENONFINITE. */
int lbmice_step(lbmice_t* h, int64_t nsteps);

/* Copy one field (LBMICE_FIELD_*) of the current state into dst, which holds bytes bytes
 * (must be at least the field's size: 4 nx ny, 4 nx ny times 18 or 27 for POPS,
 * lbmice_state_bytes for STATE).
 * dst_on_device: 1 = device pointer (asynchronous), 0 = host pointer (the call
 * synchronises the stream before returning). Errors: EINVAL, ECUDA. */
int lbmice_fields(lbmice_t* h, int32_t which, void* dst, size_t bytes, int32_t dst_on_device);

/* Overwrite the state from a checkpoint: which = LBMICE_FIELD_POPS (layout as in
 * lbmice_fields; phi, and with 16-bit storage U and rho, are recomputed as the sums),
 * LBMICE_FIELD_PHI_PREV, or LBMICE_FIELD_STATE (bytes from lbmice_fields(STATE) of a handle
 * with the same parameters). src holds bytes bytes, on the device (1) or host (0). Loading
 * POPS and PHI_PREV restores an F32 state exactly; STATE restores any storage exactly.
 * Errors: EINVAL, ECUDA. */
int lbmice_load(lbmice_t* h, int32_t which, const void* src, size_t bytes,
                int32_t src_on_device);

/* FP64 reductions of the current state into out[LBMICE_NSTATS] (host):
 *   out[0] solid area   sum (1 + phi)/2 dx^2
 *   out[1] flow mass    sum rho                 (exactly conserved without inlet/outlet)
 *   out[2] vapour invariant sum U + (L_sat/2) sum phi_prev (exact with periodic faces)
 *   out[3] sum phi
 *   out[4] number of nodes where phi, U or rho is NaN or Inf
 *   out[5] time steps taken since the last init
 * Synchronises the stream. Errors: EINVAL, ECUDA. */
int lbmice_stats(lbmice_t* h, double out[LBMICE_NSTATS]);

/* Tip positions (Sec. 3.1.2 measures the tip speed V as the rate of the phi = 0 crossing;
 * Sec. 3.2.2 compares the tips facing and leaving the inflow), computed on the device from
 * the current phi, so a long run tracks its tips without exporting the field. For each of
 * nrays directions angles_deg[i] (degrees, counter-clockwise from +x; host array), radii[i]
 * (host) receives the distance in cells from (cx, cy) (node coordinates) to the first
 * crossing of phi from > 0 to <= 0 along the ray: phi is sampled at r = k step, k = 0, 1, ...
 * by bilinear interpolation of the four surrounding nodes (in double), and the crossing is
 * placed by linear interpolation between the two samples around it. NaN when phi <= 0 at the
 * centre, or when the ray reaches x < 0, y < 0, x > nx - 2 or y > ny - 2 first. 1 <= nrays
 * <= LBMICE_MAX_RAYS, step > 0. Synchronises the stream. Errors: EINVAL, ECUDA. */
#define LBMICE_MAX_RAYS 1024
int lbmice_tips(lbmice_t* h, double cx, double cy, double step, int32_t nrays,
                const double* angles_deg, double* radii);

/* Size in bytes of the LBMICE_FIELD_STATE blob of this handle (0 for a null handle). */
size_t lbmice_state_bytes(const lbmice_t* h);

/* Wait for the handle's stream and report any pending asynchronous CUDA error. */
int lbmice_sync(lbmice_t* h);

/* Number of time steps taken since the last init (host counter, no synchronisation). */
int64_t lbmice_steps_done(const lbmice_t* h);

/* Release the handle and all device memory it owns (synchronises the stream first).
 * Null is accepted. */
int lbmice_destroy(lbmice_t* h);

/* Static description of an error code. */
const char* lbmice_strerror(int code);

/* Name of the CUDA error behind the last LBMICE_ECUDA / LBMICE_ENOMEM returned on the calling
 * thread ("none" if there was none); a static string. */
const char* lbmice_last_error(void);

/* ---- checked build -------------------------------------------------------------------------
 * The same sources compiled with -DLBMICE_CHECKED (liblbmice_checked.so; the Python binding
 * loads it when the environment sets LBMICE_CHECKED=1) test every global and shared-memory
 * index of the step kernels -- single-grid and batched -- against the extent of its buffer
 * before the access: population regions (nodes < pstride), [ny][pitch] planes, and the
 * shared-memory phi and source tiles. A violation sets a bit of a device word (1
 * population region, 2 plane, 4 shared memory) and the access is skipped, a load giving 0;
 * nothing traps. It stands in for a memory checker and costs speed; the normal library
 * compiles the tests away.
 *
 * lbmice_debug_flags waits for the device (cudaDeviceSynchronize), writes the word to *flags
 * and, if clear is 1, resets it. lbmice_debug_set_margin makes the tests use extents shrunk by
 * margin elements (>= 0; 0 restores them), so that accesses near the end of a buffer, still
 * inside it, are reported and skipped: a self-test of the checks. Both are process-wide for
 * the current device. Errors: EINVAL (null flags, clear not 0/1, negative margin), ECUDA; in
 * the normal library they return LBMICE_ENOTSUP (flags 0). */
int lbmice_debug_flags(uint32_t* flags, int32_t clear);
int lbmice_debug_set_margin(int64_t margin);

/* Self-test of the bounded device-side waits (both builds). The march's phi-ring waits poll
 * their mbarrier for about a second at most; one that gives up sets a device word that the
 * next health check (check_every, lbmice_stats) reports as LBMICE_ETIMEOUT. This call runs
 * one CTA whose wait cannot be satisfied (an mbarrier phase that expects 16 bytes no copy
 * brings, nothing in flight), waits for the device, reads and clears the word: it returns
 * LBMICE_ETIMEOUT when the wait gave up and was reported, LBMICE_OK if it was not. The
 * context stays usable. Errors: ECUDA. */
int lbmice_debug_wait_selftest(void);

/* ---- many grids in one launch --------------------------------------------------------------
 * A batch advances many independent grids -- different sizes, supersaturations,
 * anisotropies, inflows and faces -- with one kernel launch per time step for every shape
 * in use (and per LBMICE_BATCH_MAX_PER_LAUNCH members of that shape), captured in CUDA graphs
 * of 60 steps, instead of one launch per grid. Each launch carries its members' constants
 * and buffer roles in its kernel parameters (no device-side list). The march shape is one
 * wave of persistent CTAs over the concatenated column strips of its members (each CTA an
 * equal share of their rows); a tile shape is one CTA per tile of the concatenated member
 * tilings. Every shape collides a node with the same arithmetic, so a member's results do
 * not depend on its shape, and equal those of lbmice_step bit for bit. Members are ordinary
 * handles: initialise, read and check them with the single-grid calls through
 * lbmice_batch_member. All members share the flow flag and the storage, and advance in
 * lockstep: lbmice_batch_step refuses (EINVAL) once a member was stepped on its own
 * (re-initialising every member restarts them together). There is no device-side wait in
 * the batched path.                                                                         */
typedef struct lbmice_batch lbmice_batch_t;

/* Shapes the batched step can use for a member (autotuned per grid size): the column march
 * of the single-grid step, or a 2D tile of 256 threads that collides its tile plus a
 * one-node ring. */
#define LBMICE_SHAPE_MARCH 0
#define LBMICE_SHAPE_32x8 1
#define LBMICE_SHAPE_64x4 2
#define LBMICE_SHAPE_16x16 3
/* Members one batched launch can carry (its parameter block, one 352-byte descriptor per
 * member, stays under the 32 KB kernel-parameter limit). */
#define LBMICE_BATCH_MAX_PER_LAUNCH 64

/* Create count member grids from params[0..count-1] on stream (as lbmice_create each), all
 * with the march shape. The batched step is the default scheme only: every member takes the
 * E4 gradient and the six-fold anisotropy (stencil 0 or 4, fold 0 or 6). Errors: EINVAL
 * (count < 1, null, mixed flow or storage, another stencil or fold, any member's
 * parameters), EUNSTABLE, ENOMEM, ECUDA; nothing is leaked on error. */
int lbmice_batch_create(const lbmice_params* params, int32_t count, void* stream,
                        lbmice_batch_t** out);

/* Number of members, and a borrowed handle of member i (owned by the batch; do not
 * destroy it, do not step it on its own). */
int32_t lbmice_batch_size(const lbmice_batch_t* b);
lbmice_t* lbmice_batch_member(lbmice_batch_t* b, int32_t i);

/* Advance every member by nsteps: per step, one launch per shape in use and per
 * LBMICE_BATCH_MAX_PER_LAUNCH members of that shape. Errors: EINVAL (members out of
 * lockstep), ECUDA. Asynchronous. */
int lbmice_batch_step(lbmice_batch_t* b, int64_t nsteps);

/* Autotuner: for each distinct grid size, time steps_per_trial steps of those members with
 * each shape (CUDA events) and keep the fastest. Every member is advanced by the same
 * number of steps (written to *steps_taken), so the batch stays in lockstep; initialise the
 * members again afterwards if the run must start from its initial state. shapes (optional,
 * host, count entries) receives the chosen shape of each member. Synchronises the stream.
 * Errors: EINVAL, ECUDA. */
int lbmice_batch_autotune(lbmice_batch_t* b, int32_t steps_per_trial, int32_t* shapes,
                          int64_t* steps_taken);

/* Set the shape of member i (LBMICE_SHAPE_*); launches already queued keep the shapes
 * they were given. Errors: EINVAL. */
int lbmice_batch_set_shape(lbmice_batch_t* b, int32_t i, int32_t shape);

/* Destroy the batch and all its members. Null is accepted. */
int lbmice_batch_destroy(lbmice_batch_t* b);

/* ---- gradients: checkpointed tape and the discrete adjoint of the step ----------------------
 * Reverse-mode derivatives of a run with respect to the parameters eps, D and lambda and to
 * the initial moment fields, for the loss L a caller builds from the final phi and U fields:
 * the adjoint of every step (Sec. 2.2 collisions, Eq. (d) pull, E4 gradient of Sec. 3.1.1,
 * anisotropy of Sec. 2.1) is hand-derived from the FP32 step and runs on the GPU.
 * A tape records a grid that was initialised by lbmice_set_fields or lbmice_init_seed (an
 * equilibrium state, step 0) and is then advanced only through lbmice_tape_record; it keeps
 * the state every `every` steps (lbmice_state_bytes each, on the device). The reverse sweep
 * restores each checkpoint, recomputes that segment's states and runs backwards through them
 * (work space: every + 1 population buffers and every + 2 phi planes, allocated by the first
 * backward). Supported: FP32 storage, periodic faces on all four sides (EINVAL otherwise).
 * Non-differentiable points are taken as the branch the step takes: below the |grad phi|^2
 * threshold the anisotropy does not depend on the gradient or on eps; q(phi) = 1 - phi has
 * zero slope where its clamp to [0, 2] is active.                                             */
typedef struct lbmice_tape lbmice_tape_t;

/* Start a tape on grid h (borrowed; it must outlive the tape), keeping a checkpoint every
 * `every` >= 1 steps. The reverse step adds the pull's own-population term inside the
 * collision adjoint when the reverse working set (about 464 bytes per node) exceeds the L2,
 * else in a separate pass; the environment variable LBMICE_ADJ_FUSED=1 or 0, read here,
 * forces one form (both give the same bits). Errors: EINVAL (null, every < 1, h not at step
 * 0, storage other than FP32, a face that is not periodic), ENOMEM, ECUDA. */
int lbmice_tape_create(lbmice_t* h, int32_t every, lbmice_tape_t** out);

/* Advance the grid by nsteps through lbmice_step, keeping checkpoints. Errors: EINVAL (the
 * grid was stepped outside the tape), ENONFINITE (check_every), ENOMEM, ECUDA. */
int lbmice_tape_record(lbmice_tape_t* t, int64_t nsteps);

/* Steps recorded so far, -1 for a null tape. */
int64_t lbmice_tape_steps(const lbmice_tape_t* t);

/* Reverse sweep from the seeds phi_bar = dL/dphi_T and U_bar = dL/dU_T ([ny][nx] float32,
 * host or device, either may be null = 0) at the recorded final step. grads (host, 3
 * doubles, may be null) receives dL/d eps, dL/d D (through D dt/dx^2 and, when lambda is not
 * given, through the beta = 0 lambda = tau0 D / (a2 W0^2) of Sec. 2.1) and dL/d lambda (lambda
 * alone). phi0_bar, U0_bar, rho0_bar, ux0_bar, uy0_bar ([ny][nx] float32, host or device, each
 * may be null) receive dL/d of the initial moment fields (rho0 and u0 are zero without the
 * flow lattice). Synchronises the grid's stream. The tape may be swept again. Errors: EINVAL
 * (the grid was stepped outside the tape), ENOMEM, ECUDA. */
int lbmice_tape_backward(lbmice_tape_t* t, const float* phi_bar, const float* U_bar,
                         double grads[3], float* phi0_bar, float* U0_bar, float* rho0_bar,
                         float* ux0_bar, float* uy0_bar);

/* Free the tape (checkpoints and work space); the grid is untouched. Null is accepted. */
int lbmice_tape_destroy(lbmice_tape_t* t);

/* ---- diagnostics without allocation -------------------------------------------------------
 * The paper has no counterpart: this is a service of the library, not a step of the method.
 * Some callers cannot allocate device memory when they want diagnostics -- for example an
 * application whose device memory is reserved up front by its own pool allocator, or a
 * time-critical loop that cannot accept the device synchronisation and latency of
 * cudaMalloc. lbmice_stats_noalloc computes the first five values of lbmice_stats
 * (solid area, flow mass, vapour invariant, sum phi, non-finite count) from state buffers the
 * caller owns, and allocates nothing: its per-block partial sums live in a fixed 80 KB
 * __device__ array that every GPU loading this library holds until the process exits.
 *   pops:     device, planes h0..h8, g0..g8[, f0..f8] of [ny][pitch] floats (plane stride
 *             pitch * ny), as exported by lbmice_fields(LBMICE_FIELD_POPS) with pitch = nx;
 *   phi, phi_prev: device, [ny][pitch] floats;  flow: 1 if the f planes are present;
 *   dx, L_sat: as in lbmice_params;  out: device, 5 doubles, written by the call;
 *   stream:   cudaStream_t the work is enqueued on (asynchronous; nothing is synchronised).
 * Grids of more than LBMICE_NOALLOC_MAX_NODES nodes are rejected with LBMICE_EINVAL, as are
 * null pointers and pitch < nx. The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and caches it per device ordinal for the
 * life of the process; make that first call before any stream capture. The cached address
 * belongs to the device's primary context as it was then: after cudaDeviceReset (or anything
 * else that destroys and recreates that context) it is stale and this entry point must not
 * be called again in the process. Every call uses the same array, which keeps the last call's partial sums (no element
 * needs to start at zero): calls that overlap on the GPU -- on different streams, or from
 * different threads -- race on it and must be serialised by the caller.
 * Errors: EINVAL, ECUDA. */
#define LBMICE_NOALLOC_MAX_NODES (2048LL * 8192LL)
int lbmice_stats_noalloc(const float* pops, const float* phi, const float* phi_prev,
                         int32_t nx, int32_t ny, int32_t pitch, int32_t flow, double dx,
                         double L_sat, double* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LBMICE_H_ */
