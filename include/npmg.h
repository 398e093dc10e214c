/*
 * npmg.h -- C ABI of the GB300 multigrid pressure-Poisson library.
 *
 * The library solves the discrete pressure-Poisson system of the Neural
 * Physics projection method (Chen, Heaney & Pain, arXiv 2402.17913):
 *
 *     A_h x = b,   A_h = -Laplacian_h
 *
 * where A_h is the paper's fixed-weight diffusion filter with unit
 * coefficient (Sec. 2.1 and App. A: the 2D 5-point filter
 * [0 -1 0; -1 4 -1; 0 -1 0] / h^2 and the 3D 7-point filter with centre 6),
 * applied as a cross-correlation (Eq. define_convolution) over an L x M (x N)
 * grid whose padding ring holds the boundary values (Sec. 2.1: zero padding =
 * Dirichlet 0; Sec. 2.3: copy padding = zero normal derivative).  The solver
 * is the multigrid cycle of Sec. 2.2 (Jacobi smoothing, Eq. Jacobi-1-relax;
 * 2x2(x2) average restriction; copy prolongation; filters re-discretised per
 * level, App. B) used as the preconditioner of conjugate gradients, inside an
 * iterative-refinement loop whose solution accumulator and outer residual are
 * float64.  ns_step() runs one projection step of Algorithm 1.
 *
 * Conventions for every entry point
 * ---------------------------------
 *  * Arrays are dense, row-major with x fastest: index = (z*ny + y)*nx + x.
 *    shape[] and spacing[] are given in the order (x, y, z); bc[] lists the
 *    faces x-, x+, y-, y+, z-, z+ (MG_BC_DIRICHLET or MG_BC_NEUMANN).
 *  * Pointers named d_* are DEVICE pointers owned by the caller; h_* are host
 *    pointers.  The library owns only what it allocates in *_create and
 *    frees in *_destroy.  Solves and steps allocate nothing.
 *  * `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls enqueue work on it; a call that returns statistics
 *    (non-NULL out-stats pointer) synchronises that stream before returning.
 *  * Every call returns an mg_status.  On MG_ERR_* the message is available
 *    from mg_last_error() (thread-local, valid until the next failing call
 *    on the same thread).  MG_NOT_CONVERGED / MG_DIVERGED still leave the
 *    best iterate in the output buffer.
 *  * Handles are not thread-safe; use one handle per host thread.  All
 *    handles work on the CUDA device that was current at *_create.
 *  * Solid cells (mask byte 1) are not unknowns: they are returned as 0, and
 *    a fluid/solid face is a zero-normal-derivative face.
 */
#ifndef NPMG_H
#define NPMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MG_OK = 0,
  MG_ERR_INVALID = 1,     /* bad argument; nothing was enqueued          */
  MG_ERR_CUDA = 2,        /* a CUDA call failed; see mg_last_error()     */
  MG_ERR_OOM = 3,         /* device allocation failed in *_create        */
  MG_NOT_CONVERGED = 4,   /* iteration limit reached before rel_tol      */
  MG_DIVERGED = 5,        /* residual became non-finite or grew > 1e3x   */
  MG_TIMEOUT = 6          /* a bounded device-side wait gave up          */
} mg_status;

enum { MG_BC_DIRICHLET = 0, MG_BC_NEUMANN = 1 };

/* Storage of the cycle's level arrays (Sec. 2.2 smoothing, restriction and
 * prolongation): the iterate, right-hand side and correction of every level
 * but the finest.  The CG vectors (residual, preconditioned residual,
 * search direction, A p, inner correction) stay float32 and the refinement
 * loop's residual and iterate float64 at every setting; arithmetic is
 * float32 throughout. */
typedef enum {
  MG_FP32 = 0,        /* level arrays float32                              */
  MG_MIXED_FP16 = 1,  /* level arrays float16                              */
  MG_MIXED_BF16 = 2   /* level arrays bfloat16                             */
} mg_precision;

typedef struct {
  int pre;              /* Jacobi sweeps before restriction (default 2)        */
  int post;             /* Jacobi sweeps after prolongation (default 2)        */
  double omega;         /* Jacobi relaxation, Eq. Jacobi-1-relax (2/3)         */
  double coarse_scale;  /* factor s on every coarse correction (1.0)           */
  int levels;           /* grid levels, 0 = coarsen until the smallest side
                           is 4 (e.g. 256^2 -> 7 levels)                       */
  int krylov;           /* 1 = cycle preconditions CG (default); 0 = plain
                           stationary cycles                                    */
  int max_inner;        /* CG iterations per refinement step (default 200)     */
  int max_outer;        /* refinement steps (default 12)                       */
  mg_precision prec;    /* level-array storage (default MG_FP32)               */
  double inner_floor;   /* smallest relative tolerance asked of one inner
                           solve; 0 = default (1e-4)                           */
  int cycle;            /* MG_CYCLE_V (default): pre sweeps, residual
                           restriction, exact coarsest solve, post sweeps;
                           MG_CYCLE_SAWTOOTH: the paper's cycle (App. B
                           recursion): the residual restricted down with no
                           smoothing, and on every level from the coarsest up
                           one Jacobi step from zero r / d plus coarse_scale
                           times the prolonged correction, then `post` sweeps
                           (no exact coarsest solve; `pre` is ignored).  With
                           the re-discretised coarse levels the stationary
                           sawtooth needs coarse_scale ~ 0.5.                 */
  int refine;           /* arithmetic of the refinement loop's iterate and
                           outer residual (Sec. 4 item (4), mixed precision
                           with iterative refinement): MG_REFINE_FP64
                           (default) keeps the iterate in float64 and forms
                           r = b - A x in float64; MG_REFINE_FF keeps it as
                           float-float pairs (hi + lo float32, about 48
                           significant bits) and forms r with error-free
                           float32 products (faster where float64 is slow).  */
} mg_options;

enum { MG_CYCLE_V = 0, MG_CYCLE_SAWTOOTH = 1 };
enum { MG_REFINE_FP64 = 0, MG_REFINE_FF = 1 };

typedef struct {
  int status;           /* mg_status of the solve                             */
  int iters;            /* CG iterations (cycles when krylov = 0), all steps   */
  int outer;            /* refinement steps taken                             */
  int levels;           /* grid levels used                                   */
  double relres0;       /* ||b - A x0|| / ||b|| of the initial guess (float64) */
  double relres;        /* final ||b - A x|| / ||b||, x = float64 iterate      */
  double bnorm;         /* ||b||_2                                            */
  float ms;             /* device time of the solve, milliseconds             */
  double history[32];   /* relres after each refinement step (first `outer`+1) */
  double guess_relres;  /* relres of the caller's initial guess (= relres0
                           unless the guess was rejected)                     */
  int guess_rejected;   /* 1 when a checked guess (ns_step with a learned
                           guess) had relres > 1 and the solve restarted
                           from zero                                          */
} mg_stats;

typedef struct mg_handle_s* mg_handle;
typedef struct ns_handle_s* ns_handle;

/* Fill *opt with the defaults listed above. */
void mg_default_options(mg_options* opt);

/* Thread-local text of the last error (never NULL). */
const char* mg_last_error(void);

/*
 * mg_create: build the level hierarchy of A_h (Sec. 2.2 / App. B: level k
 * has half the cells of level k-1 per axis and spacing 2^k h).
 *   dim        2 or 3.
 *   shape      cells per axis (x, y[, z]); each must be divisible by
 *              2^(levels-1) and the coarsest side must be >= 2.
 *   spacing    h per axis (x, y[, z]), > 0.
 *   bc         2*dim face types (x-, x+, y-, y+[, z-, z+]).
 *   d_solid    device uint8 array of shape cells (1 = solid) or NULL.  Read
 *              during the call only.  Every fluid component must touch a
 *              Dirichlet face (otherwise A_h is singular).
 *   opt        NULL = defaults.
 * Allocates the workspace (hierarchy, CG vectors, float64 accumulator,
 * coarsest-level inverse) on the current device and factors the coarsest
 * level.  Errors: MG_ERR_INVALID (bad shape/bc/options), MG_ERR_OOM,
 * MG_ERR_CUDA.  *out is NULL on error.
 */
mg_status mg_create(mg_handle* out, int dim, const int64_t shape[3],
                    const double spacing[3], const int bc[6],
                    const uint8_t* d_solid, const mg_options* opt,
                    void* stream);

/*
 * mg_solve: solve A_h x = b until ||b - A_h x||_2 <= rel_tol * ||b||_2.  The
 * iterate is kept in float64 and the refinement residual is evaluated in
 * float64 (or both in float-float with opt->refine = MG_REFINE_FF).
 *   d_b   device float32 right-hand side (values on solid cells ignored),
 *         16-byte aligned.
 *   d_x   device float32, 16-byte aligned: initial guess on entry, solution
 *         on exit (the iterate rounded to float32 once; fetch the iterate
 *         as float64 with mg_get_solution_f64).
 *   rel_tol  > 0.
 *   out   host stats or NULL.
 * Synchronises the stream.  After the first residual the refinement loop
 * runs on the device as one CUDA graph with conditional while nodes (4 CG
 * iterations per inner body, both loops bounded by counts as well as by the
 * convergence flags); where that graph cannot be built, or with the
 * environment variable NPMG_NO_DEVICE_LOOP set when the handle first
 * solves, the host launches graphs of 4 CG iterations and reads the device
 * control block between them (the same kernels in the same order; kernels
 * inside graphs with conditional nodes are not visible to ncu).  The
 * device loop reads a copy of the right-hand side in the handle's
 * workspace; the graphs are built on the first solve.  Returns MG_OK,
 * MG_NOT_CONVERGED, MG_DIVERGED, or an error (MG_ERR_INVALID for NULL or
 * misaligned pointers or rel_tol <= 0).
 */
mg_status mg_solve(mg_handle h, const float* d_b, float* d_x, double rel_tol,
                   void* stream, mg_stats* out);

/* Copy the float64 iterate of the last solve into d_x64 (device, cells). */
mg_status mg_get_solution_f64(mg_handle h, double* d_x64, void* stream);

/* Number of levels and cells per axis of level k (host ints). */
mg_status mg_level_shape(mg_handle h, int k, int64_t shape_out[3]);
int mg_num_levels(mg_handle h);

/*
 * Building blocks, one kernel each, on caller-provided float32 device
 * arrays of level k's shape.  They use the operator of level k scaled by
 * (h_0x / h_kx)^2 ... i.e. the coefficients w_a = h_0x^2 / h_{k,a}^2 (the
 * finest x-spacing squared times the paper's filter), which is the form the
 * solver iterates on; multiply by 1/h_0x^2 to get A_h itself.
 *   mg_apply_operator: d_y = A'_k d_x (0 on solid cells).
 *   mg_smooth: `sweeps` weighted-Jacobi sweeps of A'_k x = b in place.
 *   mg_residual_restrict: d_bc (level k+1) = R (b - A'_k x).
 *   mg_prolong_correct: x += s * P e (e on level k+1), 0 on solid cells.
 *   mg_precondition: d_z = one cycle of the preconditioner on r, level 0.
 * Every array must be 16-byte aligned (the kernels move float4 vectors);
 * a NULL or misaligned array returns MG_ERR_INVALID with nothing enqueued.
 */
mg_status mg_apply_operator(mg_handle h, int k, const float* d_x, float* d_y,
                            void* stream);
mg_status mg_smooth(mg_handle h, int k, float* d_x, const float* d_b,
                    int sweeps, void* stream);
mg_status mg_residual_restrict(mg_handle h, int k, const float* d_x,
                               const float* d_b, float* d_bc, void* stream);
mg_status mg_prolong_correct(mg_handle h, int k, const float* d_e, float* d_x,
                             void* stream);
mg_status mg_precondition(mg_handle h, const float* d_r, float* d_z,
                          void* stream);

mg_status mg_destroy(mg_handle h);

/*
 * mg_vcycle_noalloc: the cycle of mg_precondition (d_z = M d_r, level 0 =
 * the whole grid) for callers that cannot allocate device memory -- code
 * running inside someone else's stream capture, plugins given a fixed memory
 * budget, real-time loops that must never enter the allocator.  It needs no
 * handle and allocates nothing: the arguments are those of mg_create plus
 * the input r and output z (float32, device, cells, 16-byte aligned);
 * opt->prec must be MG_FP32.  All temporaries (mask hierarchy, level
 * vectors, coarsest-level inverse, rebuilt on every call) live in one
 * static device array of 8 MiB that every GPU loading the library keeps
 * until exit.  Limits: at most 2^18 cells (e.g. 512^2 or 64^3) and at most
 * 256 cells on the coarsest level; larger problems return MG_ERR_INVALID
 * with a message.  The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress) and caches it, so make that first
 * call before any stream capture.  Every call uses the same array: calls
 * that overlap on the GPU (other streams, other host threads) race and must
 * be serialised by the caller.  The paper has no counterpart; it is an
 * interface convenience.
 */
mg_status mg_vcycle_noalloc(int dim, const int64_t shape[3], const double spacing[3], const int bc[6],
                            const uint8_t* d_solid, const mg_options* opt, const float* d_r, float* d_z,
                            void* stream);

/*
 * Instrumentation (no counterpart in the paper).  With profiling on, every
 * kernel launch of the handle (solves, and the projection steps of the
 * ns_handle that owns it) is bracketed by CUDA events on its stream and the
 * solve runs without its CUDA graph; mg_profile_read adds up the event
 * times per kernel class (milliseconds) and launch counts into the caller's
 * host arrays of MG_K_COUNT entries, synchronising the handle's last stream.
 * mg_kernel_launches counts every kernel the handle has launched (the nodes
 * of each graph launch included) whether or not profiling is on.
 */
typedef enum {
  MG_K_DOWN_FINE = 0,   /* smoothing + residual + restriction, finest level  */
  MG_K_UP_FINE = 1,     /* prolongation + correction + smoothing, finest     */
  MG_K_DOWN = 2,        /* the same on the other multi-block levels          */
  MG_K_UP = 3,
  MG_K_COARSE = 4,      /* single-block cycle of the coarse levels (2D
                           float32 V(2,2): with the middle levels, one
                           thread-block-cluster launch)                     */
  MG_K_P_UPDATE = 5,    /* CG: p = z + beta p, Ap, (p, Ap)                   */
  MG_K_XR_UPDATE = 6,   /* CG: d += alpha p, r -= alpha Ap, ||r||            */
  MG_K_OUTER = 7,       /* float64 refinement residual                       */
  MG_K_INIT_FINISH = 8,
  MG_K_MOMENTUM = 9,
  MG_K_DIVERGENCE = 10,
  MG_K_CORRECT = 11,
  MG_K_CLUSTER_PCG = 12, /* a small 2D grid's whole CG solve after the first
                            residual, one thread-block-cluster launch        */
  MG_K_COUNT = 13
} mg_kernel_class;
mg_status mg_profile_enable(mg_handle h, int on);
mg_status mg_profile_read(mg_handle h, double* h_ms, int64_t* h_launches, int reset);
int64_t mg_kernel_launches(mg_handle h);

/*
 * mg_probe_l2_read (instrumentation, no counterpart in the paper): the
 * roof for kernels whose working set stays in L2.  One kernel launch on
 * `stream` reads the n floats of d_buf (device, 16-byte aligned, n a
 * multiple of 4) `reps` times with coalesced 16-byte loads over 4 blocks per
 * SM, and writes one partial sum per block into d_sink (device, at least
 * 4 x the SM count floats).  With d_buf smaller than L2, the caller's CUDA
 * events around the call give the L2 read bandwidth (n * 4 * reps bytes /
 * time).  Errors: MG_ERR_INVALID (bad sizes or alignment), MG_ERR_CUDA.
 */
mg_status mg_probe_l2_read(const float* d_buf, int64_t n, int reps, float* d_sink, int sink_len, void* stream);

/*
 * Projection step (Algorithm 1) on a staggered grid of cells (x, y[, z])
 * with spacing h in every direction.  Pressure at cell centres (cells);
 * u on x-faces (nx+1, ny[, nz]), v on y-faces (nx, ny+1[, nz]), w on z-faces
 * (nx, ny, nz+1), each x fastest.  Boundaries: x- inflow (u = u_inflow,
 * tangential 0), x+ outflow (zero-gradient velocity, p = 0), other faces
 * free-slip walls.  d_solid (cells, 1 = solid, nullable) marks the body:
 * faces touching it get the implicit absorption sigma (Eq. Tn+1); its cells
 * are not pressure unknowns.
 *
 * ns_create: allocates the pressure hierarchy (Neumann except x+ Dirichlet)
 *   and the momentum workspace.  sigma: absorption on solid faces (1e8).
 * ns_step: momentum predictor + corrector (Sec. 2.3 two-pass scheme with
 *   frozen time-n advecting velocity), b = -(1/dt) D q*, pressure correction
 *   solve A_h dp = b from dp = 0 to rel_tol, q -= dt G dp, p += dp.  u, v,
 *   (w), p are updated in place.  out: stats of the pressure solve or NULL.
 */
mg_status ns_create(ns_handle* out, int dim, const int64_t cells[3], double h,
                    const uint8_t* d_solid, double sigma,
                    const mg_options* opt, void* stream);
mg_status ns_step(ns_handle ns, float* d_u, float* d_v, float* d_w,
                  float* d_p, double dt, double nu, double u_inflow,
                  double rel_tol, void* stream, mg_stats* out);
/*
 * ns_set_stencils: the filters of the momentum step (Alg. 1 step 1) for
 * every later ns_step / ns_momentum on ns.  NS_STENCIL_FD (the default of
 * ns_create): the 5-point (2D) / 7-point (3D) diffusion filter and central
 * differences (App. A, Eq. AAA).  NS_STENCIL_FE: the finite-element filters
 * of App. A: 9-point / 27-point diffusion, 1/(4 h^2) [-1 -2 -1; -2 12 -2;
 * -1 -2 -1] and 1/(26 h^2) (88 centre, -6 face, -3 edge, -2 corner), and
 * advection along each axis by the central difference smoothed with weights
 * (1, 4, 1) across the other axes (1/(12 h), 1/(72 h)); the printed z
 * filters, whose sign is opposite to the x and y ones, are taken with the
 * +d/dz sign of those.  Neighbours outside the face array follow the
 * padding rule of every axis they leave.  MG_ERR_INVALID for a NULL handle
 * or another value.
 */
enum { NS_STENCIL_FD = 0, NS_STENCIL_FE = 1 };
mg_status ns_set_stencils(ns_handle ns, int stencil);
/* Step 1 only: q* from q^n and p^n into d_us, d_vs, d_ws (face arrays),
   with the filters chosen by ns_set_stencils. */
mg_status ns_momentum(ns_handle ns, const float* d_u, const float* d_v,
                      const float* d_w, const float* d_p, float* d_us,
                      float* d_vs, float* d_ws, double dt, double nu,
                      double u_inflow, void* stream);
/* Step 2 RHS only: d_b = -(1/dt) D q* on fluid cells, 0 on solid cells. */
mg_status ns_divergence_rhs(ns_handle ns, const float* d_us, const float* d_vs,
                            const float* d_ws, double dt, float* d_b,
                            void* stream);
/* Steps 3-5 only: q -= dt G dp (faces that G corrects), p += dp. */
mg_status ns_correct(ns_handle ns, float* d_u, float* d_v, float* d_w,
                     float* d_p, const float* d_dp, double dt, void* stream);
/*
 * Batched solves: `count` independent 2D problems A_h x = b of different
 * sizes (each the operator of mg_create), all solved to rel_tol by ONE
 * persistent cooperative launch that a CUDA graph replays.  The launch walks
 * the phases of the refinement / MG-PCG algorithm in lockstep over the
 * instances (work items: (instance, tile) pairs per level, or whole
 * instances), with grid-wide barriers between phases; converged instances
 * drop out of the work lists.  Barrier waits are bounded: a barrier that
 * cannot complete within the timeout makes the solve return MG_TIMEOUT.
 *
 * mg_create_batched:
 *   shapes    count x 2 int64 (nx, ny) per instance; multiples of 4 with
 *             more than 1024 cells each.
 *   spacing   count x 2 doubles (hx, hy).
 *   bc        4 face types shared by all instances (x-, x+, y-, y+).
 *   d_masks   host array of `count` device uint8 pointers (1 = solid), each
 *             may be NULL; or NULL for no masks.  Read during the call.
 *   opt       only MG_FP32; pre/post give the initial sweep depth.
 *   Allocates all instances' workspace.  A tile shape and sweep depth found
 *   earlier by mg_tune_batched for the same GPU and batch (cache file
 *   $NPMG_TUNE_CACHE, default ~/.cache/npmg_batched_tune.txt) is reused.
 * mg_solve_batched: d_rhs / d_x are host arrays of `count` device pointers
 *   (float32, instance-shaped; d_x = initial guess in, solution out).  `out`
 *   = host array of `count` stats or NULL.  Synchronises the stream.  Returns
 *   MG_OK when every instance converged, else the first non-OK status.
 * mg_tune_batched: the autotuner.  Solves the given batch with every tile
 *   shape (64x16, 32x16, 128x8, 64x32, 128x16) and sweep depth (1, 2, 3
 *   Jacobi sweeps per level and leg), each solve starting from the guesses
 *   d_x holds on entry (copied once to a temporary device buffer), keeps the
 *   fastest time to rel_tol, writes it to the cache and reports it (host
 *   ints, each nullable).  d_x is overwritten with the last solve's result.
 * mg_batched_config: set the tile shape, sweep depth, barrier timeout
 *   (seconds) and a test hook: with withhold_first_arrival != 0 one block
 *   never arrives at the first barrier, so the solve must end in MG_TIMEOUT.
 */
typedef struct mg_batch_s* mg_batch;
mg_status mg_create_batched(mg_batch* out, int count, const int64_t* shapes, const double* spacing, const int bc[4],
                            const uint8_t* const* d_masks, const mg_options* opt, void* stream);
mg_status mg_solve_batched(mg_batch b, const float* const* d_rhs, float* const* d_x, double rel_tol, void* stream,
                           mg_stats* out);
mg_status mg_tune_batched(mg_batch b, const float* const* d_rhs, float* const* d_x, double rel_tol, void* stream,
                          int* out_tile_x, int* out_tile_y, int* out_sweeps);
mg_status mg_batched_config(mg_batch b, int tile_x, int tile_y, int sweeps, double barrier_timeout_s,
                            int withhold_first_arrival);
mg_status mg_destroy_batched(mg_batch b);

/*
 * Learned initial guess (the warm start of the pressure solve).
 *
 * A bias-free 3D U-Net with 3 resolutions and 16 channels maps the
 * divergence right-hand side b and the previous pressure p^n of a
 * projection step (Algorithm 1) to a guess of the pressure increment dp that
 * the solve then refines; multigrid from the guess still runs to the same
 * tolerance and, in ns_step, restarts from zero when the guess is worse than
 * zero (relres > 1).  Sec. 1 and Sec. 5 of the paper motivate coupling such
 * networks with the solver; the network and its training are defined here:
 *   x = (b / rms(b), p^n / rms(p^n))  (2 channels, rms over the sample)
 *   e1 = R(W1 x), e1 = R(W2 e1)        full resolution
 *   e2 = R(W3 P e1), e2 = R(W4 e2)     half           (P = 2x2x2 average)
 *   e3 = R(W5 P e2), e3 = R(W6 e3)     quarter
 *   d2 = R(W7 (U e3 + e2))             half           (U = copy upsampling)
 *   d1 = R(W8 (U d2 + e1))             full
 *   dp_guess = rms(b) * W9 d1          (1 channel)
 * with R = ReLU and Wk 3x3x3 cross-correlations with zero padding.  Weights
 * are FP32 masters; activations and tensor-core operands are BF16 with FP32
 * accumulation.  Training minimises 0.5 * mean((net(x) - dp / rms(b))^2)
 * (GN_LOSS_L2) or the residual of the guess, 0.5 * sum over interior
 * fluid cells of (A_crop y - b / rms(b))^2 / size (GN_LOSS_RESIDUAL; A_crop
 * = the 7-point pressure operator of the crop with spacing h, links only
 * between fluid cells inside the crop), with Adam (beta1 0.9, beta2 0.999,
 * eps 1e-8) on 3D crops of solver runs.
 *
 * Weights on the host are the 9 layers back to back, layer k as
 * [27 taps][c_in][c_out] float32, tap t = (dz+1)*9 + (dy+1)*3 + (dx+1),
 * (c_in, c_out) = (2,16), (16,16) x 7, (16,1): GN_NUM_WEIGHTS floats.
 * Device fields are float32 [n][z][y][x] (x fastest), 16-byte aligned; every
 * cell count must be divisible by 4.  Calls are asynchronous on `stream`
 * unless they return host values.
 *
 * gn_create: weights from h_weights (required); allocates the FP32 masters,
 *   Adam moments and packed operands.  Activation workspaces are allocated
 *   on first use of a shape and kept.
 * gn_forward: d_out[n] = dp_guess for samples (d_b[n], d_p[n]).
 * gn_gradients: loss and gradient (host, weight layout; nullable) under
 *   loss_mode: targets d_t (the solver's dp) for GN_LOSS_L2; fluid flags
 *   d_fluid (float 1/0, NULL = all fluid) and spacing h for
 *   GN_LOSS_RESIDUAL; synchronises.
 * gn_adam_step: one Adam step with h_grad (weight layout) or, when NULL,
 *   the last gn_gradients result; lr > 0.
 * gn_dataset_reserve: room for `capacity` crops of size crop (x, y, z)
 *   of a grid with spacing h.
 * gn_dataset_add: cuts full fields (cells) into non-overlapping crops and
 *   appends (b, p^n = d_p_next - d_dp, dp, fluid) for each until full;
 *   d_solid = uint8 solid flags of the grid or NULL.
 * gn_train: `steps` Adam steps on minibatches of `batch` crops drawn with a
 *   seeded generator under loss_mode, the learning rate decaying from lr to
 *   lr / 20 along a half cosine; a minibatch's inputs b and p^n are scaled
 *   by their rms over the whole minibatch (so the residual loss is the
 *   minibatch's squared relative residual / 2); h_losses (nullable)
 *   receives each step's loss; synchronises.
 * gn_conv3d (building block): one convolution of a BF16 NDHWC16 tensor
 *   d_x ([n][z][y][x][16]) with FP32 weights d_w ([27][16][16], device).
 *   mode GN_CONV_F32: d_y = float [..][16]; GN_CONV_RELU: bf16 ReLU output;
 *   GN_CONV_DGRAD: float output of the data gradient (mirrored taps,
 *   transposed channels); GN_CONV_LIN: bf16 linear output.
 *   d_scratch: device, GN_CONV_SCRATCH_BYTES, 256-byte aligned; synchronises.
 * gn_conv3d_wgrad (building block): d_dw[t][ci][co] = sum over voxels of
 *   x[v + o_t][ci] * g[v][co]; d_scratch >= GN_WGRAD_SCRATCH_MIN bytes (more
 *   bytes = more blocks); synchronises.
 * ns_set_guess: attach (g != NULL) or detach the guess network of ns_step;
 *   ns does not own g.
 * Errors: MG_ERR_INVALID (bad shape, NULL, misaligned), MG_ERR_OOM,
 * MG_ERR_CUDA, MG_TIMEOUT (a tile load or MMA that did not complete in its
 * bounded wait).
 */
#define GN_NUM_WEIGHTS 49680
#define GN_CONV_SCRATCH_BYTES 28160
#define GN_WGRAD_SCRATCH_MIN (256 + 27 * 16 * 16 * 4)
enum { GN_CONV_F32 = 0, GN_CONV_RELU = 1, GN_CONV_DGRAD = 2, GN_CONV_LIN = 3 };
enum { GN_LOSS_L2 = 0, GN_LOSS_RESIDUAL = 1 };
typedef struct gn_handle_s* gn_handle;
mg_status gn_create(gn_handle* out, const float* h_weights, void* stream);
mg_status gn_set_weights(gn_handle g, const float* h_weights);
mg_status gn_get_weights(gn_handle g, float* h_weights);
mg_status gn_forward(gn_handle g, int n, const int64_t cells[3], const float* d_b, const float* d_p, float* d_out,
                     void* stream);
mg_status gn_gradients(gn_handle g, int n, const int64_t cells[3], const float* d_b, const float* d_p,
                       const float* d_t, const float* d_fluid, int loss_mode, double h, double* h_loss,
                       float* h_grad, void* stream);
mg_status gn_adam_step(gn_handle g, const float* h_grad, double lr, void* stream);
mg_status gn_dataset_reserve(gn_handle g, const int64_t crop[3], int capacity, double h);
mg_status gn_dataset_add(gn_handle g, const int64_t cells[3], const float* d_b, const float* d_p_next,
                         const float* d_dp, const uint8_t* d_solid, void* stream);
int gn_dataset_size(gn_handle g);
mg_status gn_train(gn_handle g, int steps, int batch, uint64_t seed, double lr, int loss_mode, double* h_losses,
                   void* stream);
mg_status gn_conv3d(const void* d_x, const float* d_w, void* d_y, int n, const int64_t cells[3], int mode,
                    void* d_scratch, void* stream);
mg_status gn_conv3d_wgrad(const void* d_x, const void* d_g, float* d_dw, int n, const int64_t cells[3],
                          void* d_scratch, size_t scratch_bytes, void* stream);
/* Kernels the guess network's calls have launched so far (process-wide). */
int64_t gn_kernel_launches(void);
mg_status gn_destroy(gn_handle g);
mg_status ns_set_guess(ns_handle ns, gn_handle g);
/* ns_set_guess_level: as ns_set_guess, with the network run on the grid
 * coarsened `level` times (0, 1 or 2).  ns_step then restricts b and p^n
 * by 2x2x2 averages, runs g there and interpolates its dp back trilinearly
 * level by level (0 on solid cells): 1/8 or 1/64 of the network's work, for
 * the smooth part of dp that the cycles are slowest to remove.  g must be
 * trained on fields coarsened the same way (ns_coarse_fields) with the
 * coarse spacing 2^level h.  Sides divisible by 4 * 2^level; MG_ERR_OOM when
 * the coarse buffers cannot be allocated. */
mg_status ns_set_guess_level(ns_handle ns, gn_handle g, int level);
/* Device pointers (owned by ns, valid until the next ns_step) of the last
   step's right-hand side b and pressure increment dp (cells each). */
mg_status ns_last_fields(ns_handle ns, const float** d_b, const float** d_dp);
/* ns_coarse_fields: the last step's b and dp and the given pressure d_p
 * (cells each), restricted `level` times (1 or 2) by 2x2x2 averages into
 * caller buffers of cells / 8^level floats, and the solid mask coarsened as
 * often (a coarse cell is solid when all its children are) into d_solid_c
 * (cells / 8^level bytes); 3D grids with sides divisible by 2^level.
 * Enqueued on stream; the first call allocates the handle's coarse buffers
 * (MG_ERR_OOM if that fails). */
mg_status ns_coarse_fields(ns_handle ns, int level, const float* d_p, float* d_b_c, float* d_p_c, float* d_dp_c,
                           uint8_t* d_solid_c, void* stream);

/*
 * Implicit advection-diffusion step (Sec. 2.2, Eq. BE-advection-concise;
 * Sec. 3.2 "Multigrid solver for the advection-diffusion equation").
 *
 * One backward-Euler step of dT/dt + u dT/dx + v dT/dy - nu Lap T = 0 on an
 * nx x ny node grid of spacing h with zero padding (Sec. 2.1):
 *   A T^{n+1} = T^n,  A = I + dt (u D_x + v D_y - nu Lap_h),
 * D_x the central difference (Eq. A) or the first-order upwind difference
 * (backward for u >= 0, forward for u < 0; the printed Eq. A-up holds the
 * forward differences, the upwind scheme of a velocity along -x and -y),
 * Lap_h the 5-point filter of App. A.  A is nonsymmetric, so the solve is
 * the cycle as a stationary iteration x <- x + M (b - A x) (no CG), with a
 * float64 iterate, a float64 residual and the cycle in float32.
 *
 * Levels: nodes halved per level (2x2 average restriction, copy
 * prolongation); the coarse stencils re-discretised at spacing 2^k h
 * (AD_COARSE_REDISCRETISE, App. B) or the Galerkin product R A P
 * (AD_COARSE_GALERKIN: the re-discretised stencil with the diffusion term
 * times 2^k).  Cycle MG_CYCLE_V: `pre` relaxed Jacobi sweeps from zero,
 * residual restricted, recursion, `coarse_scale` times the copied
 * correction, `post` sweeps; the coarsest level (<= 256 nodes) by a dense
 * inverse computed at create.  MG_CYCLE_SAWTOOTH: the paper's cycle (the
 * residual restricted without smoothing, r / c plus the scaled correction
 * on the way up, then `post` sweeps; its alpha = 1 and one sweep are
 * omega = 1, post = 1).
 *
 * ad_create: cells = {nx, ny} (8 .. 65536, divisible by 2^(levels-1));
 *   h, dt > 0; nu >= 0; scheme AD_UPWIND or AD_CENTRAL; opt NULL = defaults.
 *   Allocates every buffer; MG_ERR_INVALID / MG_ERR_OOM / MG_ERR_CUDA.
 * ad_solve: d_b = T^n, d_x0 = initial guess or NULL (= T^n, the previous
 *   time level, Sec. 3.2), d_x = T^{n+1} out (nx * ny float32 device
 *   arrays, [y][x], x fastest; d_x may alias d_x0).  Stops when
 *   ||b - A x||_2 / ||b||_2 <= rel_tol (checked before every cycle), when
 *   the L1 norm of one cycle's change of x is <= l1_tol (the paper's gauge;
 *   0 disables it), or after opt.max_cycles cycles (MG_NOT_CONVERGED);
 *   MG_DIVERGED when the residual grows 1000-fold.  Enqueued on stream and
 *   synchronised every 8 cycles.
 */
enum { AD_UPWIND = 0, AD_CENTRAL = 1 };
enum { AD_COARSE_REDISCRETISE = 0, AD_COARSE_GALERKIN = 1 };
typedef struct {
  int cycle;            /* MG_CYCLE_V (default) or MG_CYCLE_SAWTOOTH          */
  int pre;              /* V: Jacobi sweeps before restriction, 0..2 (2)     */
  int post;             /* sweeps after the correction, 0..2 (2)              */
  double omega;         /* Jacobi relaxation (2/3)                            */
  double coarse_scale;  /* factor on every coarse correction (1)              */
  int coarse_op;        /* AD_COARSE_REDISCRETISE (default) or _GALERKIN      */
  int levels;           /* 0 = halve while both sides stay even and >= 4      */
  int max_cycles;       /* (1000)                                             */
} ad_options;
typedef struct {
  int status;           /* mg_status of the solve                             */
  int cycles;           /* cycles run                                         */
  double relres0;       /* relres of the initial guess                        */
  double relres;        /* relres of the returned iterate (float64)           */
  double l1_first;      /* L1 norm of the first cycle's change of x           */
  double l1_last;       /* L1 norm of the last cycle's change of x            */
  float ms;             /* device time of the solve, milliseconds             */
} ad_stats;
typedef struct ad_handle_s* ad_handle;
mg_status ad_default_options(ad_options* opt);
mg_status ad_create(ad_handle* out, const int64_t cells[2], double h, double dt,
                    double nu, double u, double v, int scheme,
                    const ad_options* opt, void* stream);
mg_status ad_solve(ad_handle h, const float* d_b, const float* d_x0, float* d_x,
                   double rel_tol, double l1_tol, void* stream, ad_stats* out);
/* Levels of the hierarchy; the first level handled by the single-block
   kernel; kernels launched so far (0 for NULL). */
int ad_num_levels(ad_handle h);
int ad_coarse_start(ad_handle h);
int64_t ad_kernel_launches(ad_handle h);
mg_status ad_destroy(ad_handle h);

/* The pressure handle inside ns (owned by ns; do not destroy). */
mg_handle ns_pressure_handle(ns_handle ns);
mg_status ns_destroy(ns_handle ns);

#ifdef __cplusplus
}
#endif
#endif /* NPMG_H */
