/*
 * unwrap_lp.h -- C ABI of the GB300 (sm_103a) L^p-norm phase-unwrapping library.
 *
 * Method: Legarda-Saenz, Brito-Loeza, Espinosa-Romero, "On the performance of
 * preconditioned methods to solve L^p-norm phase unwrapping" (arXiv 2203.13675),
 * Algorithm 1: an outer reweighting (IRLS) loop that turns the wrapped-gradient
 * residual into per-edge weights U, V (Eq. UV), around an inner preconditioned
 * conjugate-gradient solve of the weighted 5-point system A(U,V) phi = b
 * (Eq. Axb), with the paper's preconditioners (Sec. 2 list: identity, Jacobi,
 * ILU(0), IC(0), SOR read as SSOR) plus a DCT Poisson preconditioner (the
 * Fourier-basis approach of Sec. 1).
 *
 * Conventions shared by every entry point:
 *  - Grids are H rows (index i, the paper's y) by W columns (index j, the
 *    paper's x); pixel (i,j) is element i*W + j of a contiguous row-major
 *    array.  H >= 2, W >= 2.
 *  - Unless stated otherwise pointers are CUDA DEVICE pointers owned by the
 *    caller; the library never frees them.  Work is enqueued on the given
 *    stream (NULL = legacy default stream) and returns before it finishes
 *    unless the function says it synchronises.
 *  - Return values are ulp_status codes: 0 success, 1 a warning (phi written,
 *    the inner solve hit l_max), negative an error (outputs undefined).
 *    ulp_last_error() returns a message for the calling thread's last error.
 *  - Masks are uint8 arrays (1 = pixel excluded: every edge touching it gets
 *    weight 0 and its phi keeps the initial value); NULL means no mask.
 *  - Every wait inside a kernel is bounded (options.spin_timeout_s); a wait
 *    that runs out makes the call return ULP_ERR_TIMEOUT, never a hang.
 */
#ifndef UNWRAP_LP_H
#define UNWRAP_LP_H

#include <stdint.h>

/* Symbol visibility of the entry points (the library is built with hidden
 * default visibility, so only these names are exported). */
#ifndef ULP_API
#define ULP_API __attribute__((visibility("default")))
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Preconditioner M of Algorithm 1 ("estimate preconditioning matrix M from A").
 * The first five are the paper's list (Sec. 2, items 1-5); DCT is the
 * unweighted Neumann-Poisson pseudo-inverse applied through cosine transforms;
 * LEARNED is a trained network (ulp_unet) applied as M^-1 inside flexible CG;
 * MG is a multigrid cycle (the paper names multigrid among the fast solvers of
 * this system, Sec. 1); RBSSOR and RBILU are items 3-5 with the unknowns in
 * red-black order instead of the natural one (the paper leaves the ordering
 * open), which makes each triangular solve one parallel pass per colour.  DCT,
 * LEARNED, MG, RBSSOR and RBILU run in flexible CG on single-map FP64 plans; MG
 * also on mixed-precision plans and, map by map, on batched plans. */
typedef enum {
  ULP_PRECOND_IDENTITY = 0, /* M = I: PCG becomes CG */
  ULP_PRECOND_JACOBI = 1,   /* M = diag(A) */
  ULP_PRECOND_ILU0 = 2,     /* incomplete LU, no fill, natural row-major order */
  ULP_PRECOND_IC0 = 3,      /* incomplete Cholesky, no fill (same M as ILU0 for symmetric A) */
  ULP_PRECOND_SSOR = 4,     /* symmetric SOR, relaxation options.omega */
  ULP_PRECOND_DCT = 5,      /* s = L^+ r, L the unit-weight Neumann Laplacian */
  ULP_PRECOND_LEARNED = 6,  /* s = D^-1 r + rho N(r / rho, U, V), rho = rms(r); needs ulp_plan_set_unet */
  ULP_PRECOND_MG = 7,       /* one symmetric V-cycle of aggregation multigrid: 2x2 aggregates, Galerkin
                               coarse operators, 2 + 2 damped-Jacobi sweeps (omega 2/3), correction x 1.5 */
  ULP_PRECOND_RBSSOR = 8,   /* SSOR(omega) with the unknowns in red-black order (red: i + j even, first) */
  ULP_PRECOND_RBILU = 9     /* ILU(0) (= IC(0)) with the unknowns in red-black order */
} ulp_precond;

typedef enum {
  ULP_OK = 0,
  ULP_WARN_MAXITER = 1,    /* phi written; some inner solve stopped at l_max */
  ULP_ERR_INVALID = -1,    /* bad argument (sizes, p, eps, non-finite psi, ...) */
  ULP_ERR_CUDA = -2,       /* a CUDA runtime call failed */
  ULP_ERR_BREAKDOWN = -3,  /* d^T A d <= 0 or non-finite inside PCG */
  ULP_ERR_TIMEOUT = -4,    /* an in-kernel wait exceeded options.spin_timeout_s */
  ULP_ERR_NOMEM = -5,      /* device allocation failed */
  ULP_ERR_UNSUPPORTED = -6 /* option combination not built */
} ulp_status;

typedef enum {
  ULP_STOP_RELRES = 0, /* stop when ||r_l||_2 <= tol * ||b||_2 (recurrence residual) */
  ULP_STOP_PAPER = 1   /* Algorithm 1's test: stop when delta_new <= tol^2 delta_0, delta = r^T M^-1 r */
} ulp_stop_mode;

typedef enum {
  ULP_PRECISION_FP64 = 0,  /* every vector, weight and reduction in FP64 */
  ULP_PRECISION_MIXED = 1  /* FP32 vectors/weights/stencil, FP64-accurate dot products and
                              alpha/beta, FP64 phi and true residual every refresh period.
                              Applies to ULP_PRECOND_IDENTITY, ULP_PRECOND_JACOBI (persistent
                              PCG) and ULP_PRECOND_MG (flexible CG, FP32 V-cycle; a stop seen
                              on the FP32 recurrence is confirmed on the FP64 true residual);
                              other preconditioners return ULP_ERR_UNSUPPORTED */
} ulp_precision;

typedef enum {
  ULP_PHI0_ZERO = 0, /* phi^0 = 0 */
  ULP_PHI0_USER = 1  /* phi holds phi^0 on entry (warm start / resume / the paper's random start) */
} ulp_phi0_mode;

typedef struct ulp_options {
  int stop_mode;          /* ulp_stop_mode, default ULP_STOP_RELRES */
  double outer_tol;       /* Algorithm 1 outer test: continue while ||phi^{k+1}-phi^k||/||phi^k|| > outer_tol.
                             Default 1e-6 (the paper's tol).  ||phi^k|| = 0 counts as +infinity. */
  long long refresh;      /* true-residual period of Algorithm 1 (r = b - A phi when l mod period = 0);
                             <= 0: floor(sqrt(H*W)) in FP64, 20 in mixed precision */
  double omega;           /* SSOR relaxation in (0, 2), default 1 */
  int precision;          /* ulp_precision, default ULP_PRECISION_FP64 */
  int phi0_mode;          /* ulp_phi0_mode, default ULP_PHI0_ZERO */
  int tile_rows;          /* rows per warp tile; 0 = autotuned table */
  int blocks_per_sm;      /* resident blocks per SM of the persistent solver; 0 = autotuned */
  double spin_timeout_s;  /* bound on any in-kernel wait, default 2.0 s */
  int profile;            /* 1: record CUDA events around every persistent solver launch (ulp_plan_counters);
                             2: as 1, and the DCT solve runs host-driven (each kernel a host launch) */
  int graph;              /* 1: ulp_unwrap / ulp_unwrap_batched capture their kernel sequence into a CUDA
                             graph on the first call and replay it while the arguments stay the same
                             (ignored when profile = 1) */
  int stall_window;       /* ULP_PRECOND_LEARNED: an inner solve whose ||r|| has not halved within this many
                             iterations (counted from the last time it did), or that meets r^T s <= 0 or
                             d^T A d <= 0, switches to the Jacobi preconditioner for the rest of that solve;
                             default (0) 200 (plain CG and Jacobi PCG on 2^14..2^22-pixel maps halve ||r||
                             every 40-450 iterations) */
} ulp_options;

/* Per-call statistics, written on the host when the call synchronises. */
#define ULP_MAX_OUTER_STATS 64
typedef struct ulp_stats {
  int status;                                 /* ulp_status of the call */
  int outer;                                  /* outer passes run (k at exit) */
  long long inner_total;                      /* sum of inner PCG iterations */
  long long inner[ULP_MAX_OUTER_STATS];       /* l at exit of each inner solve */
  double relres[ULP_MAX_OUTER_STATS];         /* ||r_l|| / ||b|| at exit of each inner solve */
  double outer_err[ULP_MAX_OUTER_STATS];      /* Algorithm 1's error after each pass (inf if ||phi^k|| = 0) */
  int fallbacks;                              /* ULP_PRECOND_LEARNED: inner solves that switched to Jacobi */
  double setup_ms;                            /* device time spent building the preconditioner from A in
                                                 this call (Algorithm 1, "estimate preconditioning matrix
                                                 M from A"; the paper reports its share, Sec. 3): the
                                                 pivot and coefficient phases of the ILU(0)/IC(0)/SSOR
                                                 solvers, always; the coarse grids (multigrid), the mask
                                                 bits (DCT) and the red-black pivots of the flexible-CG
                                                 solves on plans made with options.profile != 0; 0 for
                                                 I and Jacobi, whose D^-1 comes with the system kernel */
} ulp_stats;

/* Fills *opt with the defaults listed above. */
ULP_API void ulp_options_default(ulp_options* opt);

/* Message for the calling thread's most recent error ("" if none). Static storage. */
ULP_API const char* ulp_last_error(void);

/* ---------------------------------------------------------------------------
 * Whole method (Algorithm 1).
 * ------------------------------------------------------------------------- */

/* unwrap_lp: Algorithm 1 with default options except the arguments given.
 *   psi   [H*W]  wrapped phase, values in (-pi, pi] (Eq. wrapped); host OR device
 *                memory (detected with cudaPointerGetAttributes).
 *   p            the L^p exponent, 0 <= p <= 2 (the paper states p < 2; p = 2 is the
 *                unweighted least-squares limit).
 *   eps          tau of Eq. (UV), > 0 (the paper uses 0.01).
 *   precond      ulp_precond.
 *   tol          inner relative-residual tolerance (ULP_STOP_RELRES), > 0.
 *   max_outer    k_max of Algorithm 1 (>= 1); the outer tolerance is 0 here, so
 *                passes continue until phi stops changing or k_max is reached.
 *   max_inner    l_max; <= 0 means 2*H*W (the paper's choice).
 *   phi   [H*W]  output unwrapped phase, same memory kind as psi.  phi^0 = 0.
 * Synchronises the legacy default stream.  Host buffers are copied to and from
 * internal device buffers inside the call.  Allocates and frees its workspace. */
ULP_API int unwrap_lp(const double* psi, int H, int W, double p, double eps, int precond,
              double tol, int max_outer, int max_inner, double* phi);

/* Plans own all device workspace for one grid size (or one batch of sizes) and
 * are reused across calls; creating one allocates, calls on it do not. */
typedef struct ulp_plan_s* ulp_plan;

/* ulp_plan_create: workspace for H x W maps.  opt may be NULL (defaults).
 * Allocates device memory; the current CUDA device is the plan's device. */
ULP_API int ulp_plan_create(int H, int W, const ulp_options* opt, ulp_plan* out);

/* ulp_plan_create_batched: workspace for n maps of sizes H[t] x W[t] solved
 * together by one persistent launch per outer pass (I, Jacobi, ILU/IC/SSOR).
 * 1 <= n <= 256.  With ULP_PRECOND_MG the first batched call also creates one
 * single-map plan per map (the plan owns and destroys them) and runs the maps
 * concurrently on eight streams forked from the call's stream. */
ULP_API int ulp_plan_create_batched(int n, const int* H, const int* W, const ulp_options* opt,
                            ulp_plan* out);

ULP_API void ulp_plan_destroy(ulp_plan plan);

/* ulp_unwrap: Algorithm 1 on the plan's grid, enqueued on cuda_stream.
 *   psi [H*W] device, mask [H*W] device uint8 or NULL, phi [H*W] device
 *   (holds phi^0 on entry when opt.phi0_mode = ULP_PHI0_USER).
 *   stats: host pointer or NULL.  Non-NULL makes the call synchronise the
 *   stream and fill *stats; the return value is then the solve's status.
 *   NULL returns after enqueueing (ULP_OK unless an argument is invalid);
 *   ulp_plan_last_status() reads the outcome later.
 *   With max_outer > 8 (and opt.graph = 0) the call also waits for the GPU
 *   after every 8 passes and enqueues no further pass once every map has left
 *   its outer loop (a pass past the outer stop would do nothing but cost its
 *   launches); the results are the same. */
ULP_API int ulp_unwrap(ulp_plan plan, const double* psi, const uint8_t* mask, double p, double eps,
               int precond, double tol, int max_outer, int max_inner, double* phi,
               void* cuda_stream, ulp_stats* stats);

/* One map of a batch: device pointers as in ulp_unwrap, own p and tau. */
typedef struct ulp_map {
  const double* psi;
  const uint8_t* mask;
  double* phi;
  double p;
  double eps;
} ulp_map;

/* ulp_unwrap_batched: the n maps of a batched plan (sizes in creation order),
 * all outer passes of all maps in max_outer persistent launches; with
 * ULP_PRECOND_MG (FP64 or mixed precision) each map runs the multigrid flexible
 * CG of ulp_unwrap on its own plan, the maps spread over eight streams (largest
 * first, on the least-loaded stream), all forked from and joined back into
 * cuda_stream.  per_map: host array of n stats or NULL (same synchronisation
 * rule as ulp_unwrap).  Returns the worst status over the maps. */
ULP_API int ulp_unwrap_batched(ulp_plan plan, const ulp_map* maps, int precond, double tol,
                       int max_outer, int max_inner, void* cuda_stream, ulp_stats* per_map);

/* Synchronises the plan's last stream and returns its last call's status;
 * fills *stats (first map of a batch) when non-NULL. */
ULP_API int ulp_plan_last_status(ulp_plan plan, ulp_stats* stats);

/* Instrumentation of a plan: kernels it enqueued, and (with options.profile)
 * the summed device duration of its persistent solver launches, timed with
 * CUDA events recorded on the call's stream around each launch.  Reading the
 * durations synchronises those events.  reset != 0 clears after reading. */
typedef struct ulp_counters {
  long long kernel_launches;  /* every kernel the plan enqueued */
  long long solver_launches;  /* persistent PCG launches among them */
  double solver_ms;           /* summed duration of the timed solver launches (profile only) */
  long long timed_launches;   /* solver launches included in solver_ms */
  /* options.profile = 2, flexible-CG solves, run host-driven: summed durations and counts of each
   * phase, [0] A (d = s + beta d, q = A d, d^T q), [1] B (phi, r update), [2] R (true residual),
   * [3] M (s = M^-1 r: the GEMM chain, the network, the red-black passes or the V-cycle), [4] D
   * (r^T s, r^T r, stop test), [5] U (multigrid only: the V-cycle's last kernel, the up step on
   * the map's grid, which also runs D where it can; timed on its own and not included in M) */
  double phase_ms[6];
  long long phase_launches[6];
  /* flexible-CG solves run as a graph whose WHILE body executes once per inner iteration:
   * the kernels of its start and of one body (the body's kernels are not in kernel_launches;
   * an outer pass with l inner iterations runs start + l x body of them) */
  long long graph_start_kernels;
  long long graph_body_kernels;
} ulp_counters;
ULP_API int ulp_plan_counters(ulp_plan plan, int reset, ulp_counters* out);

/* ulp_autotune: picks options.tile_rows and options.blocks_per_sm of the
 * persistent solvers for n maps of sizes H[t] x W[t] by timing, for each
 * candidate, one outer pass of maps (device data, as in ulp_unwrap_batched)
 * capped at iters inner iterations (<= 0: 40) with CUDA events around the
 * solver launch.  precision is ulp_precision.  Writes the fastest into *best
 * (other fields default); when cache_path is non-NULL appends one JSON line
 * (GPU name, precision, preconditioner, a hash of the sizes, the choice and its
 * time).  Allocates and frees a plan per candidate; synchronises the default
 * stream.  No counterpart in the paper: it tunes the launch shape only. */
ULP_API int ulp_autotune(int n, const int* H, const int* W, const ulp_map* maps, int precond, int precision,
                         int iters, const char* cache_path, ulp_options* best);

/* ---------------------------------------------------------------------------
 * Single steps of the method (device pointers, contiguous H*W arrays,
 * enqueued on cuda_stream).  They use the same kernels as the solver.
 * ------------------------------------------------------------------------- */

/* Sec. 2.1: Delta^x_{i,j} = W(psi_{i,j+1} - psi_{i,j}) for j <= W-2 and
 * Delta^y_{i,j} = W(psi_{i+1,j} - psi_{i,j}) for i <= H-2, with W the wrapping
 * operator of Eq. (wrapped) onto (-pi, pi]; the last column of dx and the last
 * row of dy are 0 (they only multiply zero boundary weights). */
ULP_API int ulp_wrapped_diffs(const double* psi, int H, int W, double* dx, double* dy, void* cuda_stream);

/* Eq. (UV) and Eq. (Axb): U_{i,j} = tau / (|phi_{i,j+1} - phi_{i,j} - dx_{i,j}|^(2-p) + tau),
 * V likewise along i (0 on edges leaving the grid or touching a masked pixel), and the
 * right-hand side b_{i,j} = dx_{i,j-1}U_{i,j-1} - dx_{i,j}U_{i,j} + dy_{i-1,j}V_{i-1,j} - dy_{i,j}V_{i,j}.
 * b may be NULL. */
ULP_API int ulp_weights(const double* phi, const double* dx, const double* dy, const uint8_t* mask,
                int H, int W, double p, double eps, double* U, double* V, double* b,
                void* cuda_stream);

/* Eq. (Axb) left-hand side: y = A(U,V) x, with
 * (A x)_{i,j} = (U_{i,j-1}+U_{i,j}+V_{i-1,j}+V_{i,j}) x_{i,j}
 *              - U_{i,j} x_{i,j+1} - U_{i,j-1} x_{i,j-1} - V_{i,j} x_{i+1,j} - V_{i-1,j} x_{i-1,j}. */
ULP_API int ulp_matvec(const double* U, const double* V, const double* x, int H, int W, double* y,
               void* cuda_stream);

/* One application s = M^{-1} r of the preconditioner built from A(U,V)
 * (Algorithm 1, "estimate preconditioning matrix M from A").  omega is used by
 * SSOR only.  mask is used by the DCT preconditioner only (s = 0 on masked pixels). */
ULP_API int ulp_precond_apply(int precond, const double* U, const double* V, const uint8_t* mask,
                      int H, int W, double omega, const double* r, double* s, void* cuda_stream);

/* The inner PCG of Algorithm 1 on A(U,V) phi = b, warm-started from phi
 * (overwritten with the result).  stats (host, nullable) receives inner[0],
 * relres[0] and the status; non-NULL synchronises. */
ULP_API int ulp_pcg(const double* U, const double* V, const double* b, int H, int W, int precond,
            double tol, int max_inner, const ulp_options* opt, double* phi, void* cuda_stream,
            ulp_stats* stats);

/* ---------------------------------------------------------------------------
 * Allocation-free inner solve.  The paper has no counterpart: this entry point
 * exists for callers of this library that cannot allocate device memory --
 * a caller whose device memory is already held by another allocator (a
 * framework's caching pool, where cudaMalloc would fail or force the pool to
 * release memory), or a caller on a latency-bound loop that cannot pay for
 * cudaMalloc/cudaFree (cudaFree waits for the whole device) or risk an
 * out-of-memory failure mid-run.  ulp_pcg allocates and frees a workspace on
 * every call; this variant allocates nothing.
 * ------------------------------------------------------------------------- */

/* ulp_pcg_noalloc: the same solve and results as ulp_pcg with default options
 * and precond ULP_PRECOND_IDENTITY or ULP_PRECOND_JACOBI (others return
 * ULP_ERR_UNSUPPORTED); U, V, b, phi are caller-owned device arrays as there.
 *   Workspace: one static device array of 8 MiB inside the library, which
 *   every GPU that loads the library holds until the process exits.  Grids are
 *   limited to H * round_up(W, 64) <= 65536 elements (e.g. 256 x 256);
 *   larger grids return ULP_ERR_INVALID with a message in ulp_last_error().
 *   No cudaMalloc, cudaFree or other allocating routine is called.
 *   Set-up: the first call on each device (with that device current) looks up
 *   the array's device address; make that first call before any stream
 *   capture.
 *   Sharing: all calls on a device use the same array and leave their
 *   contents in it; each call clears what it needs before use.  Calls whose
 *   work overlaps on the GPU (different streams or host threads) race on the
 *   array: the caller must serialise them.
 *   stats (host, nullable) as in ulp_pcg; non-NULL synchronises the stream
 *   and returns the solve's status (a negative one also sets ulp_last_error());
 *   NULL returns after enqueueing, without reading the solve's status. */
ULP_API int ulp_pcg_noalloc(const double* U, const double* V, const double* b, int H, int W,
                            int precond, double tol, int max_inner, double* phi, void* cuda_stream,
                            ulp_stats* stats);


/* ---------------------------------------------------------------------------
 * Learned preconditioner.  The paper compares fixed algebraic preconditioners
 * (Sec. 2, items 1-5); this extension replaces the application s = M^-1 r of
 * Algorithm 1 by a trained network, used inside flexible CG because it is not
 * a fixed linear operator.  Network: a four-level U-Net on NHWC BF16
 * activations, widths 16/32/64/128, 3x3 convolutions with ReLU, 2x2 average
 * pooling and nearest-neighbour upsampling with skip concatenations, and a
 * linear 1x1 head:
 *   e0: 3->16 at HxW, e1: 16->32 at H/2, e2: 32->64 at H/4, b3: 64->128 at H/8,
 *   d2: [e2 | up(b3)] 192->64, d1: [e1 | up(d2)] 96->32, d0: [e0 | up(d1)] 48->16,
 *   y = w_h . d0 + b_h.
 * Input per pixel: (r / rho, U, V) with rho = sqrt(mean(r^2)); the
 * application is the Jacobi step plus the learned correction,
 * s = D^-1 r + rho * y (D the diagonal of A(U,V); 0 on masked pixels).
 * Parameters (FP32, canonical order): for e0 e1 e2 b3 d2 d1 d0 the weight
 * [Cout][Cin][3][3] then the bias [Cout]; then the head weight [16] and bias.
 * All device pointers; calls on one network must not overlap on the GPU (they
 * share its workspace).
 * ------------------------------------------------------------------------- */
typedef struct ulp_unet_s* ulp_unet;

/* number of parameters (242721) */
ULP_API int ulp_unet_param_count(void);
/* new network on the current device: He-uniform weights from splitmix64(seed), zero biases */
ULP_API int ulp_unet_create(unsigned long long seed, ulp_unet* out);
ULP_API void ulp_unet_destroy(ulp_unet net);
/* copy the canonical parameter vector from / to host memory (set resets the optimizer state) */
ULP_API int ulp_unet_set_params(ulp_unet net, const float* params);
ULP_API int ulp_unet_get_params(ulp_unet net, float* params);
/* binary parameter file: "ULPUNET1", int64 count, count FP32 values */
ULP_API int ulp_unet_save(ulp_unet net, const char* path);
ULP_API int ulp_unet_load(const char* path, ulp_unet* out);

/* One preconditioner application on an H x W map (contiguous FP64 planes r, U,
 * V, s; mask uint8 or NULL): s = D^-1 r + rho N(r / rho, U, V), 0 on masked
 * pixels.  The network runs on the map zero-padded to multiples of 128. */
ULP_API int ulp_unet_apply(ulp_unet net, const double* r, const double* U, const double* V,
                           const uint8_t* mask, int H, int W, double* s, void* cuda_stream);

/* Network output y = N(r / rho, U, V) (FP32 [B][H][W]) for B images stored one
 * after another in r, U, V ([B][H][W] FP64); H, W multiples of 128, B <= 64. */
ULP_API int ulp_unet_forward(ulp_unet net, int B, int H, int W, const double* r, const double* U,
                             const double* V, float* y, void* cuda_stream);

/* Training loss and its gradient with respect to the parameters (canonical
 * order, FP32 device array of ulp_unet_param_count() values, NULL to skip).
 * Per image, with x = r / rho, e~ = e / rho (e the error of a PCG iterate,
 * A e = r) and the direction s~ = D^-1 x + y:
 *   L = 1 - (s~^T x)^2 / ((s~^T A s~)(e~^T x)),
 * the A-norm fraction of the error that one exact line search along s~ leaves;
 * the loss is the mean over the B images.  Layout as ulp_unet_forward; loss
 * (host, nullable) synchronises. */
ULP_API int ulp_unet_loss_grad(ulp_unet net, int B, int H, int W, const double* r, const double* U,
                               const double* V, const double* e, double* loss, float* grad,
                               void* cuda_stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on the loss
 * of B training pairs: pair b is r + pair_idx[b]*H*W, e + pair_idx[b]*H*W with
 * the weights U + sys_idx[b]*H*W, V + sys_idx[b]*H*W (host index arrays).
 * loss (host, nullable) receives the batch loss before the step and synchronises. */
ULP_API int ulp_unet_train_step(ulp_unet net, int B, const long long* pair_idx, const int* sys_idx,
                                int H, int W, const double* r, const double* e, const double* U,
                                const double* V, float lr, double* loss, void* cuda_stream);

/* Training pairs from the inner PCG of Algorithm 1 on A(U,V) phi = b: phi* is
 * the solution to relative residual tol_star (from 0; solved with the multigrid
 * flexible CG, which reaches it in tens of iterations), and for each k < n,
 * phi_l is the iterate of the PCG with precond (identity or Jacobi) after
 * iters[k] iterations from 0; writes r_out[k] = b - A phi_l and
 * e_out[k] = phi* - phi_l ([n][H][W] FP64).  Allocates one plan and a workspace
 * of 3 H W doubles for the call.  Synchronises. */
ULP_API int ulp_unet_harvest(const double* U, const double* V, const double* b, int H, int W, int precond,
                             double tol_star, int n, const int* iters, double* r_out, double* e_out,
                             void* cuda_stream);

/* Network used by ULP_PRECOND_LEARNED on a single-map FP64 plan (NULL detaches).
 * The plan does not own it: keep it alive while the plan may use it. */
ULP_API int ulp_plan_set_unet(ulp_plan plan, ulp_unet net);

#ifdef __cplusplus
}
#endif
#endif /* UNWRAP_LP_H */
