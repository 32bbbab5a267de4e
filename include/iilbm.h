/*
 * iilbm.h -- C ABI of the GB300 (sm_103a) immersed interface–lattice Boltzmann
 * time step (II-LBM; Qin, Kolahdouz & Griffith, arXiv 2003.12186).
 *
 * One handle = one D2Q9 lattice, its populations, and at most one immersed
 * interface (a closed, counter-clockwise marker polygon).  All device memory is
 * allocated and owned by the library; every call is asynchronous on the handle's
 * CUDA stream unless stated otherwise.  Pointers marked "host or device" are
 * classified with cudaPointerGetAttributes and copied with cudaMemcpyAsync.
 *
 * Error behaviour: every entry point returns IILBM_OK (0) or a negative
 * iilbm_status.  Argument errors are detected on the host before any work is
 * queued and leave the handle unchanged.  Device-side faults of the method
 * (non-finite populations, a marker polygon that leaves its valid region, a
 * cut-link list beyond capacity) are latched in a device status word and
 * returned by the next call that synchronises (iilbm_get_*, iilbm_synchronize).
 *
 * Paper citations give the section / equation that defines each operation.
 */
#ifndef IILBM_H
#define IILBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct iilbm_lattice *iilbm_t;

typedef enum {
  IILBM_OK = 0,
  IILBM_ERR_INVALID_ARG = -1,   /* bad size, rate, enum or NULL where required */
  IILBM_ERR_OOM = -2,           /* device allocation failed */
  IILBM_ERR_CUDA = -3,          /* a CUDA runtime call failed */
  IILBM_ERR_DEVICE_TIMEOUT = -4,/* a bounded device wait gave up */
  IILBM_ERR_NONFINITE = -5,     /* a NaN / Inf appeared in the populations */
  IILBM_ERR_INTERFACE = -6,     /* marker polygon invalid (segment too long, outside region) */
  IILBM_ERR_CAPACITY = -7,      /* a fixed-size resource is too small: cut-link list,
                                   forcing kernel's shared memory, or the no-allocation
                                   read-out's staging array */
  IILBM_ERR_NO_DEVICE = -8      /* no CUDA device, or not a compute capability 10.3 device */
} iilbm_status;

enum { IILBM_SRT = 0, IILBM_MRT = 1 };
/* Storage precision of the shifted populations df_i = f_i - w_i rho0.  Arithmetic
 * is FP64 for IILBM_F64 and FP32 for the others. */
enum { IILBM_F64 = 0, IILBM_F32 = 1, IILBM_F16 = 2, IILBM_BF16 = 3 };
/* Boundaries: periodic box; walls at y = -1/2, ny - 1/2 (halfway bounce-back) and
 * periodic x; channel = walls plus parabolic inflow at x = 0 and outflow at nx - 1;
 * the boxes of the paper's section 4 (4.1: open, 4.2: no-slip walls), whose edge nodes
 * are set every step by non-equilibrium extrapolation from their inward neighbour
 * (diagonal at a corner): BOX_OUTFLOW rho = rho0 with the neighbour's velocity,
 * BOX_WALL u = 0 with the neighbour's density.  A box is not batched. */
enum { IILBM_BC_PERIODIC = 0, IILBM_BC_WALLS_Y = 1, IILBM_BC_CHANNEL = 2,
       IILBM_BC_BOX_OUTFLOW = 3, IILBM_BC_BOX_WALL = 4 };
/* Force term of the lattice Boltzmann equation: Guo's (Eqs. 21-22, velocity Eq. 24,
 * the default) or the simple external force term (Eq. 16, velocity sum e f / rho), the
 * one the paper's II-LBM uses outside its section 4.2.  Direct forcing needs Guo's. */
enum { IILBM_FORCE_GUO = 0, IILBM_FORCE_SIMPLE = 1 };
/* Lagrangian force models: Eq. 19 spring; rest-length spring; a prescribed force;
 * direct forcing Eq. 18 (iterated). */
enum { IILBM_SPRING = 0, IILBM_SPRING_REST = 1, IILBM_PRESCRIBED = 2, IILBM_DIRECT = 3 };

typedef struct {
  int32_t nx, ny;       /* lattice nodes; node (i, j) sits at coordinate (i, j); 4 <= n <= 32768 */
  int32_t collision;    /* IILBM_SRT (Eq. 14 + Eq. 21) or IILBM_MRT (Eq. 15 + Eq. 22) */
  int32_t storage;      /* IILBM_F64 / F32 / F16 / BF16 */
  int32_t bc;           /* IILBM_BC_* */
  int32_t jump;         /* 1: II-LBM (normal force through the jump of Eq. 32, tangential
                           part spread, Eq. 46); 0: IB-LBM with Guo forcing (whole G spread) */
  int32_t storage_scale_log2; /* stored value = df * 2^k (exact); 0 for F32/F64 */
  int32_t force;        /* IILBM_FORCE_GUO or IILBM_FORCE_SIMPLE */
  double tau;           /* relaxation time lambda, nu = c_s^2 (lambda - 1/2) (Eq. 7); > 0.5 */
  double s[9];          /* MRT rates in the Lallemand-Luo moment order
                           (rho, e, eps, jx, qx, jy, qy, pxx, pxy) */
  double rho0;          /* reference density of the shifted storage */
  double u_max;         /* channel centre-line inflow speed */
  double body[2];       /* uniform body force density added to g */
  void *stream;         /* cudaStream_t to run on; NULL: the library creates one */
} iilbm_config;

typedef struct {
  int32_t model;        /* IILBM_SPRING / SPRING_REST / PRESCRIBED / DIRECT */
  int32_t moves;        /* 1: markers advected, X += U (Eq. 20); 0: fixed */
  double stiffness;     /* kappa of Eq. 19 (or of the rest-length spring) */
  double dX;            /* Lagrangian spacing Delta X (Eq. 17) */
  double rest_length;   /* l0 of the rest-length spring */
  double eta;           /* direct-forcing gain of Eq. 18 */
  int32_t mdf_iters;    /* direct forcing: maximum passes */
  int32_t curve;        /* interface of the jump: 0 the marker polygon (Fn linear along each
                           segment); m = 1..16 the periodic cubic spline through the markers
                           (end of section 3.2): normals and |X_s| from its tangent, Fn along
                           it from the spline of the markers' Fn, crossings on m chords per
                           segment.  Not for DIRECT (a rigid body keeps the polygon). */
  double mdf_tol;       /* direct forcing: stop when max_k |U^D - U_k| < tol (0: all passes) */
} iilbm_interface_params;

/* Create a lattice (section 2.2.1: D2Q9, Eq. 9 weights), populations at rest
 * (df = 0).  cfg is copied; *out receives the handle.  Allocates all device memory
 * of the lattice.  Errors: INVALID_ARG, OOM, CUDA, NO_DEVICE. */
int iilbm_create_lattice(iilbm_t *out, const iilbm_config *cfg);

/* Release the handle and all its device memory (synchronises its stream). */
int iilbm_destroy(iilbm_t h);

/* Install (replace) the immersed interface: n markers, xy[n][2] FP64, closed and
 * counter-clockwise (host or device).  aux[n][2] is the prescribed force G
 * (PRESCRIBED) or the desired velocity U^D (DIRECT), else ignored (may be NULL).
 * The markers are copied; the caller keeps ownership.  Every segment must be
 * shorter than 16 lattice units and every marker at least 3 nodes from a
 * non-periodic edge.  DIRECT needs a fixed body (moves = 0), eta > 0, Guo's force term,
 * and a body whose band (every node of a marker's 4 x 4 stencil and every candidate
 * destination of its cut links) fits the forcing kernel's shared memory: 12 values per
 * band node plus 29 per marker, at most 227 KB (a D = 80 cylinder of 251 markers: 200 KB
 * in FP64, 108 KB in FP32).  n = 0 removes the interface.
 * Sections 2.2.2 (Eqs. 17-20) and 3 (Eqs. 31-32, 46-47).
 * Errors: INVALID_ARG, INTERFACE, OOM, CUDA. */
int iilbm_set_interface(iilbm_t h, const double *xy, int32_t n,
                        const iilbm_interface_params *p, const double *aux);

/* Set the state to the equilibrium (Eq. 23) of rho(x), u(x) ([ny][nx] FP64 each,
 * host or device; NULL means rho0 / zero). */
int iilbm_init_equilibrium(iilbm_t h, const double *rho, const double *ux, const double *uy);

/* Set / read the state: df[9][ny][nx] FP64 shifted populations f_i - w_i rho0 in
 * natural (pull) layout, host or device, streamed populations without the jump of
 * the current interface.  Converted to / from the storage precision. */
int iilbm_set_populations(iilbm_t h, const double *df);
int iilbm_get_populations(iilbm_t h, double *df);

/* Advance n >= 0 time steps of section 3.2 (Eq. 47 with Eqs. 17-24): Lagrangian
 * force, normal split, jump on cut links, tangential spreading, interpolation,
 * fused stream-collide, marker update.  Asynchronous.  Unless IILBM_OPT_CUDA_GRAPH is
 * off, steps are replayed from CUDA graphs for any n: the first replaying call
 * captures graphs of 32, 16, 8, 4, 2 and 1 steps from an even time level and of one
 * step from an odd level (make that first call outside any stream capture of your
 * own), and each call then launches one odd step where the level is odd and the
 * binary decomposition of the rest.  A directly forced body is captured too: each
 * captured step begins with its force iteration. */
int iilbm_step(iilbm_t h, int32_t n);

/* Macroscopic fields of the current state ([ny][nx] FP64 each, host or device,
 * any may be NULL): drho = rho - rho0 (Eq. 11 less rho0) and u of Eq. 24, computed
 * from the populations plus the current interface's jump and force -- the values
 * the next collision will use.  Synchronises. */
int iilbm_get_macros(iilbm_t h, double *drho, double *ux, double *uy);

/* Markers (each [n][2] FP64 except Fn [n]; host or device; any may be NULL):
 * current positions X, the most recent Lagrangian force G and jump strength
 * Fn = G.n/|X_s| (Eq. 32), and the velocity U interpolated in the most recent step
 * (Eq. 20).  Synchronises. */
int iilbm_get_markers(iilbm_t h, double *X, double *G, double *U, double *Fn);

/* Direct forcing: force updates of the most recent body-force computation and its
 * final residual max_k |U^D - U_k| (Eq. 18 repeated).  Synchronises. */
int iilbm_get_mdf_stats(iilbm_t h, int32_t *iters, double *residual);

/* Direct forcing: the warm start G^(0) [n][2] of the force iteration (host or device;
 * NULL = zero, the plain iteration).  Kept until replaced; first used by the next force
 * iteration (that of the current state unless a read-out has already run it). */
int iilbm_set_warm_start(iilbm_t h, const double *G0);

/* Direct forcing: where the force iteration of each step starts.
 *   IILBM_WS_GIVEN     the G^(0) of iilbm_set_warm_start (zero unless set: the plain
 *                      iteration);
 *   IILBM_WS_PREVIOUS  the force the iteration reached in the previous step (zero at
 *                      the first step after iilbm_set_interface).
 * The stopping rule (mdf_iters, mdf_tol) is the same in every mode.  INVALID_ARG for an
 * unknown mode or a batched lattice. */
enum { IILBM_WS_GIVEN = 0, IILBM_WS_PREVIOUS = 1, IILBM_WS_MLP = 2 };
int iilbm_set_warm_start_mode(iilbm_t h, int32_t mode);

/* Direct forcing: U*_k [n][2], the velocity interpolated at the markers from the state
 * without the body's force (u* of Eq. 18 before the first update), as recorded by the
 * most recent force iteration.  Host or device pointer; synchronises.  INVALID_ARG
 * unless the interface is a directly forced body. */
int iilbm_get_unforced_velocity(iilbm_t h, double *Ustar);

/* Force of the fluid on the body, F = -sum_k G_k dX (Eq. 25 without the internal
 * inertia term), from the most recent Lagrangian force.  Drag and
 * lift coefficients follow as 2 F / (rho U^2 D) (Eqs. 52-53).  Synchronises. */
int iilbm_get_body_force(iilbm_t h, double *F);

/* A rigid body carrying the directly forced interface (section 2.3).  The current
 * markers become the body's reference shape: its centre X_c0 is their mean and each
 * marker keeps its offset from it at angle 0.  After every step the library reduces the
 * step's Lagrangian force G to
 *   F_ext = -sum_k G_k dX + rho0 V_s (U_c(t) - U_c(t-1))                      (Eq. 25)
 *   T_ext = -sum_k (X_k - X_c) x G_k dX + (rho0 V_s / m) I_s (W(t) - W(t-1))   (Eq. 26)
 * moves the body, places every marker rigidly (X_k = X_c + R(theta) X0_k) and gives it
 * the body's velocity as its desired velocity, U^D_k = U_c + W x (X_k - X_c).  The force
 * iteration then rebuilds its band of nodes and cut links in every step.
 *   IILBM_BODY_PRESCRIBED_X  harmonic translation in x (section 4.4):
 *       X_c(t) = X_c0 - amplitude sin(u_max t / amplitude), U_c(t) = -u_max cos(u_max t /
 *       amplitude), t the lattice's time level (U_c(0) = -u_max).
 *   IILBM_BODY_FREE          on each degree of freedom set in dof (1 x, 2 y, 4 rotation)
 *       a spring k = spring[d] about the start and a damper c = damping[d] (the
 *       oscillator of section 4.5):  m a(t+1) = F_ext - k (X_c - X_c0) - c U_c,
 *       I_s w(t+1) = T_ext - k theta - c W (Eq. 27); U_c(t+1) = U_c(t) + a(t+1) (Eq. 28);
 *       X_c(t+1) = X_c(t) + U_c(t) + (a(t) + a(t+1)) / 2 (Eq. 29), the same for theta.
 * mass m > 0, inertia I_s > 0 (FREE; ignored when PRESCRIBED_X), volume V_s >= 0 the
 * body's area.  The explicit scheme is unstable for a light body (mass below about 2.6
 * rho0 V_s in a resting fluid).  The body stays until iilbm_set_interface replaces the
 * interface.  Synchronises.  Errors: INVALID_ARG (no directly forced interface, batched
 * lattice, bad mode or parameters), CAPACITY (the moving band's shared memory exceeds
 * 227 KB), OOM, CUDA. */
enum { IILBM_BODY_PRESCRIBED_X = 1, IILBM_BODY_FREE = 2 };
typedef struct {
  int32_t mode;         /* IILBM_BODY_PRESCRIBED_X or IILBM_BODY_FREE */
  int32_t dof;          /* FREE: free degrees of freedom, bits 1 x, 2 y, 4 rotation */
  double amplitude;     /* PRESCRIBED_X: A > 0 */
  double u_max;         /* PRESCRIBED_X: peak velocity */
  double mass;          /* FREE: m */
  double inertia;       /* FREE: I_s */
  double volume;        /* V_s, the body's area (internal-fluid inertia of Eqs. 25-26) */
  double spring[3];     /* FREE: k per degree of freedom (x, y, rotation) */
  double damping[3];    /* FREE: c per degree of freedom */
} iilbm_body_params;
int iilbm_set_rigid_body(iilbm_t h, const iilbm_body_params *bp);

/* The body's state after the most recent step: state[9] = X_c, Y_c, theta, U_x, U_y, W,
 * F_x, F_y, T (the last F_ext, T_ext of Eqs. 25-26; host pointer).  Synchronises.
 * INVALID_ARG without a body. */
int iilbm_get_rigid_body(iilbm_t h, double *state);

/* The jump of the current state's interface on the streamed populations (Eq. 47 with
 * Eq. 32): J[i-1][y][x] = the sum of s w_i/c_s^2 Fn(crossing) over the crossings of the
 * link x - e_i -> x, i = 1..8, [8][ny][nx] FP64 (host or device), zero off the cut
 * links.  Runs the current state's interface phase if it has not run.  Synchronises.
 * Errors: INVALID_ARG (NULL), OOM, CUDA, latched device status. */
int iilbm_get_jump(iilbm_t h, double *J);

/* Number of cut-link crossings of the current state's interface (Eq. 47). */
int iilbm_get_cut_link_count(iilbm_t h, int32_t *count);

/* Kernel timing (diagnostic).  enable = 1 starts recording a CUDA event pair around
 * every launch of the lean stream-collide (all tiles without a jump or force) on the
 * handle's stream and counting every kernel the library launches; enable = 0 stops.
 * iilbm_get_timing synchronises, returns the summed lean stream-collide device time
 * (ms), its launch count, the number of library kernels launched, and the number of
 * flagged tiles (128 x 8 nodes each, handed to the forced kernel instead) summed over
 * the interface phases run since timing was enabled, then resets them. */
int iilbm_set_timing(iilbm_t h, int32_t enable);
int iilbm_get_timing(iilbm_t h, double *stream_collide_ms, int32_t *stream_collide_launches,
                     int64_t *kernel_launches, int64_t *flagged_tiles);

/* Execution options (on by default but the TMA kernel; for A/B measurements and tests):
 *  IILBM_OPT_CUDA_GRAPH     replay steps from captured CUDA graphs (iilbm_step);
 *  IILBM_OPT_OVERLAP        run the forced stream-collide, then the interpolation
 *                           fused with the next step's interface phase (one kernel),
 *                           on a second, high-priority stream while the lean
 *                           stream-collide runs (direct forcing: the forced
 *                           stream-collide and the interpolation only);
 *  IILBM_OPT_VECTOR_KERNEL  vectorised stream-collide (else one node per thread);
 *  IILBM_OPT_TMA_KERNEL     FP32 storage: the lean stream-collide of interior tiles moves
 *                           its populations with bulk tensor copies through shared
 *                           memory (the other tiles keep the vectorised kernel);
 *                           value 1 every step, 2 odd steps only, 0 never (the default:
 *                           on GB300 it runs as fast as the vectorised kernel alone and
 *                           slower beside the side stream's kernels);
 *  IILBM_OPT_FORCED_BLOCKS  blocks of the forced stream-collide, which stride over the
 *                           flagged tiles (value > 0; 0 restores the default, two per
 *                           SM): fewer blocks hold fewer of the SMs' registers while the
 *                           lean stream-collide runs beside them.
 * Results agree either way up to the order of floating-point atomic additions.
 * Synchronises the handle's stream. */
enum { IILBM_OPT_CUDA_GRAPH = 0, IILBM_OPT_OVERLAP = 1, IILBM_OPT_VECTOR_KERNEL = 2,
       IILBM_OPT_FORCED_BLOCKS = 3, IILBM_OPT_TMA_KERNEL = 4 };
int iilbm_set_option(iilbm_t h, int32_t option, int32_t value);

/* No-allocation read-out (the paper has no counterpart; this is a service of the
 * library).  Same results as iilbm_get_macros, for callers that must not allocate
 * device memory at this point: code whose device memory is owned by a caching
 * allocator or a fixed budget (a cudaMalloc there can fail or fragment the pool), and
 * latency-bound loops, where cudaMalloc / cudaFree would synchronise the device.  The
 * fields are staged in a static device array of IILBM_NOALLOC_MAX_CELLS nodes x 3
 * doubles (6 MiB) that every device loading the library keeps until exit; a lattice
 * with more nodes gets IILBM_ERR_CAPACITY.  The first call on a device looks up the
 * array's device address, so make it before any stream capture.  All calls share the
 * array: calls whose GPU work overlaps in time race.  Outputs as iilbm_get_macros
 * (host or device, any may be NULL).  Synchronises. */
#define IILBM_NOALLOC_MAX_CELLS (1 << 18)
int iilbm_get_macros_noalloc(iilbm_t h, double *drho, double *ux, double *uy);

/* ---------------------------------------------------------------- batches
 * A batch advances many independent lattices together: every phase of a time step is
 * one launch for all of them (a flattened list of tiles for the stream-collide, of
 * markers for the interface phase and the interpolation, one CTA per fixed body for
 * direct forcing), replayed from CUDA graphs.  It is built from existing lattice
 * handles that share storage (F32, F16 or BF16), collision model and boundary kind,
 * have nx a multiple of 4 and the same step parity, and whose interfaces (if any) are
 * marker polygons (curve = 0); sizes, rates, interfaces and force models may differ.  The lattices stay owned by the caller.  While batched,
 * iilbm_step, iilbm_set_interface, iilbm_init_equilibrium, iilbm_set_populations,
 * iilbm_set_option and iilbm_destroy on them return INVALID_ARG; read-outs run on the
 * batch's stream after its work.  Destroy the batch before its lattices.
 * Errors of create: INVALID_ARG (mixed kinds, F64, a repeated or batched lattice), OOM,
 * CUDA. */
typedef struct iilbm_batch *iilbm_batch_t;
int iilbm_create_batch(iilbm_batch_t *out, const iilbm_t *lattices, int32_t count, void *stream);
int iilbm_destroy_batch(iilbm_batch_t b);
/* Advance every lattice of the batch by n time steps (asynchronous). */
int iilbm_batch_step(iilbm_batch_t b, int32_t n);
/* Stream-collide variant of the lean (unforced) tiles: nodes per thread NPT, resident
 * blocks per SM that the registers are budgeted for, and grid (one block per work item
 * of 4 tiles of 128 x 8 nodes, or a persistent grid striding over the items):
 *   0 / 1  NPT 4, 3 blocks, per item / persistent     2 / 3  NPT 4, 2 blocks
 *   4 / 5  NPT 2, 3 blocks                            6 / 7  NPT 2, 2 blocks
 *   8 / 9  NPT 1, 3 blocks
 *   10 / 11  NPT 4, 3 blocks in the even step and 2 in the odd one
 * Results agree to rounding (the arithmetic is the same; contraction may differ). */
int iilbm_batch_set_variant(iilbm_batch_t b, int32_t variant);
/* Autotuner: time every variant for `steps` (rounded up to whole graph replays) real
 * steps of the batch and keep the fastest; the lattices advance by those steps.
 * Returns the variant chosen and its time per step (us). */
int iilbm_batch_autotune(iilbm_batch_t b, int32_t steps, int32_t *chosen, double *us_per_step);
/* Lean stream-collide timing of eager batch steps (as iilbm_set_timing). */
int iilbm_batch_set_timing(iilbm_batch_t b, int32_t enable);
int iilbm_batch_get_timing(iilbm_batch_t b, double *stream_collide_ms, int32_t *launches,
                           int64_t *kernel_launches);
/* Wait for the batch's streams; returns any latched device status of its lattices. */
int iilbm_batch_synchronize(iilbm_batch_t b);

/* ------------------------------------------------------- learned warm start
 * A small network proposes the starting force G^(0)_k of the direct-forcing iteration
 * from each marker's local features; the iteration with its stopping rule still
 * decides the answer.  Features of marker k (30, FP32): for j = k-2 .. k+2 (cyclic)
 *   U^D_j - U*_j (2), the outward unit normal (2), the signed curvature
 *   -(X_{j+1} - 2 X_j + X_{j-1}) . n_j / dX^2 (1), and Re (1).
 * Network: x -> (x - in_mean) * in_istd -> 3 x [64, GELU (erf form)] -> 2 ->
 * * out_scale + out_mean.  Parameters packed as W1 [64][30], b1 [64], W2 [64][64], b2,
 * W3 [64][64], b3, W4 [2][64], b4 [2] (10434 FP32 values, weights [out][in]).
 * Training: mean squared error of the normalised outputs over a batch, Adam. */
typedef struct iilbm_mlp *iilbm_mlp_t;
enum { IILBM_MLP_PARAMS = 10434, IILBM_MLP_FEATURES = 30 };
/* Create a network on the current device (parameters zero, identity normalisation);
 * stream may be NULL (the network makes its own).  Errors: NO_DEVICE, OOM. */
int iilbm_mlp_create(iilbm_mlp_t *out, void *stream);
/* Destroy it (detach it from every lattice first). */
int iilbm_mlp_destroy(iilbm_mlp_t m);
/* Packed parameters in / out (host or device, FP32); setting them resets Adam. */
int iilbm_mlp_set_params(iilbm_mlp_t m, const float *params);
int iilbm_mlp_get_params(iilbm_mlp_t m, float *params);
/* Input normalisation (30 means, 30 reciprocal deviations) and output scaling (2, 2);
 * host pointers.  INVALID_ARG for a zero or non-finite output scale. */
int iilbm_mlp_set_normalization(iilbm_mlp_t m, const float *in_mean, const float *in_istd,
                                const float *out_mean, const float *out_scale);
/* Y [N][2] = network(X [N][30]); host or device pointers; synchronises. */
int iilbm_mlp_forward(iilbm_mlp_t m, const float *X, int32_t N, float *Y);
/* Gradient [10434] and value of the loss over all N samples (targets T [N][2]). */
int iilbm_mlp_gradient(iilbm_mlp_t m, const float *X, const float *T, int32_t N, float *grad,
                       float *loss);
/* `steps` Adam steps; step s uses the samples order[s * batch .. (s+1) * batch - 1]
 * (indices into X, T; host or device; each in [0, N)).  losses [steps] (nullable)
 * receives each step's batch loss before its update.  Errors: INVALID_ARG, OOM, CUDA. */
int iilbm_mlp_train(iilbm_mlp_t m, const float *X, const float *T, int32_t N,
                    const int32_t *order, int32_t steps, int32_t batch, float lr, float beta1,
                    float beta2, float eps, float *losses);
/* Start every force iteration of lattice h from the network's proposal (mode
 * IILBM_WS_MLP) with Reynolds-number feature re; the network must outlive the setting
 * (iilbm_set_warm_start_mode detaches it).  INVALID_ARG unless h carries a directly
 * forced body on the network's device; CAPACITY if the forcing kernel's shared memory
 * would exceed 227 KB. */
int iilbm_set_warm_start_mlp(iilbm_t h, iilbm_mlp_t mlp, double re);
/* The raw features F [n][30] of every marker from the U* of the most recent force
 * iteration (what the network sees before normalisation).  Synchronises. */
int iilbm_get_df_features(iilbm_t h, double re, float *F);

/* Wait for the handle's stream and return any latched device status. */
int iilbm_synchronize(iilbm_t h);

/* Static description of a status code. */
const char *iilbm_error_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* IILBM_H */
