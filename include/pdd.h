/*
 * pdd.h -- C ABI of libpdd.so: the Monte Carlo nodal stage of Probabilistic
 * Domain Decomposition (Bernal & Acebron, "A multigrid-like algorithm for
 * probabilistic domain decomposition"), on one NVIDIA GB300 (sm_103a).
 *
 * For each interfacial node x0 the library simulates many Euler-Maruyama
 * paths of dX = b dt + sigma dW (Sec. 2.1, eq. F:SDE) until the first exit
 * from the unit box [0,1]^D, with the Gobet-Menozzi shrunken-boundary test or
 * the naive test (Algorithm 1).  Along each path it accumulates the
 * Feynman-Kac weights of eq. F:Dynkin / eq. F:VR_Milstein_sys,
 *     Y_{k+1} = Y_k (1 - h c(X_k))       (or Y_k exp(-h c(X_k))),
 *     Z_{k+1} = Z_k - h Y_k f(X_k),
 * and the pathwise control variate of eq. F:xiControlVariate,
 *     xi_{k+1} = xi_k - Y_k (sigma^T grad v(X_k)) . dW_k,
 * where v is a previous, more accurate iterate given on a control grid
 * (Sec. 3.1: "a D-dimensional array holding pointwise values").  The scores
 * are phi = g(Pi X_tau) Y_tau + Z_tau and the controlled score phi + xi
 * (eqs. F:Statistics_VR, F:Combining_method).  Per node it returns sample
 * means, variances (N - 1), the covariance and Pearson correlation of
 * (phi, xi) (eq. F:Rho), standard errors sqrt(V/N) (eq. F:Statistical_error),
 * the variance ratio V[phi+xi]/V[phi] (eq. F:Variance_Reduction) and the
 * predicted speedup V[phi] / (kappa V[phi+xi]) from the nodal cost model
 * (eqs. F:Pointwise_cost and F:VR_Pointwise_cost), and the mean number of
 * steps nu = E[tau]/h (eq. F:nu).
 *
 * PDE sign convention: 1/2 sum_ij a_ij d_ij u + b . grad u - c u = f with
 * c >= 0 (the paper writes +c with c <= 0).
 *
 * Conventions of every call:
 *   - Every function returns a pdd_status (or void for destructors).  No call
 *     aborts, throws or exits; on a non-OK status pdd_last_error() returns a
 *     message (thread-local, valid until the next call on the same thread).
 *   - The library owns the opaque handles and all device memory it allocates.
 *     The caller owns every input and output buffer; the library never frees
 *     or retains them beyond the call (or, with PDD_FLAG_ASYNC, beyond the
 *     completion of the work enqueued on the context's stream).
 *   - Results are deterministic functions of (problem, grid contents, node
 *     coordinates, node index, n_paths, dt, seed, stream_tag): sums are kept
 *     in exact fixed-point integer arithmetic, so the order in which the GPU
 *     finishes paths does not change a single bit.
 *   - Random numbers: Philox4x32-10 (Salmon et al., SC'11) with key
 *     (seed_lo32, stream_tag) and counter (block, path, node, seed_hi32);
 *     normal number i of a path is Box-Muller output i % 4 of block i / 4;
 *     step k uses normals D k .. D k + D - 1.
 */
#ifndef PDD_H
#define PDD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PDD_ABI_VERSION 1

typedef enum {
  PDD_OK = 0,
  PDD_ERR_INVALID = -1,   /* bad argument; nothing was enqueued */
  PDD_ERR_NOMEM = -2,     /* device allocation failed or memory budget exceeded */
  PDD_ERR_CUDA = -3,      /* a CUDA runtime call failed (message has the CUDA error) */
  PDD_ERR_TIMEOUT = -4,   /* a bounded wait ran out */
  PDD_ERR_BUSY = -5,      /* admission queue full / resource in use; retry later */
  PDD_ERR_NOT_READY = -6, /* poll: request still running */
  PDD_ERR_CANCELLED = -7, /* poll: request was cancelled */
  PDD_ERR_OVERFLOW = -8,  /* a score left the fixed-point range |score| < 32768 */
  PDD_ERR_BOUNDS = -9,    /* bounds-checked build only: a kernel index left its buffer
                             (the message names the checks that failed)               */
  PDD_ERR_DEADLINE = -10, /* submit: the request cannot finish within the server's
                             deadline after the work already queued and running       */
  PDD_WARN_TRUNCATED = 1, /* results valid, but some paths hit max_steps */
  PDD_WARN_NOT_CONVERGED = 2 /* pdd_mlmc: results valid, stopping test not met */
} pdd_status;

/* Built-in problems on the unit box [0,1]^D (the synthetic workloads).     */
typedef enum {
  /* D=2, b = (sin y / 2, cos x / 2), c = 1 + x^2 + y^2, sigma = I,
     u = e^{x+y} cos(x-y), f from the PDE, g = u.                          */
  PDD_PROBLEM_CFG0_2D = 0,
  /* D=2, A = (1 + sin(2 pi x)/2) [[1, 1/2], [1/2, 1]], sigma its lower
     Cholesky factor, b, c, u as CFG0_2D, f from the PDE.                  */
  PDD_PROBLEM_ANISO_2D = 1,
  /* D=3, b = 0, c = 1, sigma = I, u = e^x sin y cos z + x y z.            */
  PDD_PROBLEM_CUBE_3D = 2,
  /* D=2, b = c = f = 0, sigma = I, g = u = x^2 - y^2 (harmonic).          */
  PDD_PROBLEM_HARMONIC_2D = 3,
  /* D=2, the paper's example (Sec. 6, eq. F:PDE_ejemplo): sigma = sqrt(2) I,
     b = cos(x+y) [1,1] / (1.1 + sin(x+y)), c = (x^2+y^2) / (1.1 + sin(x+y)),
     u = 2 cos(2 (y-2) x) + sin(3 (x-2) y) + 3.1, f from the PDE, g = u.   */
  PDD_PROBLEM_PAPER_EX_2D = 4
} pdd_problem_kind;

typedef enum {
  PDD_EXIT_GOBET_MENOZZI = 0, /* finish when d(X_k) >= -0.5826 |sigma^T N| sqrt(h) (Algorithm 1) */
  PDD_EXIT_NAIVE = 1          /* finish when d(X_k) >= 0 (weak order 1/2, Sec. 2.3) */
} pdd_exit_rule;

typedef enum {
  PDD_Y_EULER = 0, /* Y_{k+1} = Y_k (1 - h c_k), as in Algorithm 1 */
  PDD_Y_EXP = 1    /* Y_{k+1} = Y_k exp(-h c_k) */
} pdd_y_rule;

typedef enum {
  PDD_PATH_FP32 = 0, /* path arithmetic in FP32 (compensated Z and xi sums) */
  PDD_PATH_FP64 = 1  /* path arithmetic in FP64 */
} pdd_path_precision;

typedef enum { PDD_GRID_VALUES = 0, PDD_GRID_GRADIENT = 1 } pdd_grid_kind;
typedef enum { PDD_DTYPE_F32 = 0, PDD_DTYPE_F64 = 1 } pdd_dtype;

#define PDD_CV_NONE (-1)     /* plain estimator only (xi = 0) */
#define PDD_CV_EXACT (-2)    /* control variate from the analytic grad u (the "exact" CV) */
#define PDD_MAX_GRIDS 8      /* control-grid slots per problem */
#define PDD_FLAG_EMIT_PATHS 1u /* also write per-path phi, xi, steps */
#define PDD_FLAG_ASYNC 2u      /* device inputs/outputs only: return once enqueued */
#define PDD_FLAG_GRAPH 4u      /* pdd_estimate_levels: capture the launch sequence in a CUDA
                                  graph and replay it while the arguments repeat */
#define PDD_MAX_LEVELS 128     /* levels (or batches) per pdd_estimate_levels call */

typedef struct pdd_ctx pdd_ctx;
typedef struct pdd_problem pdd_problem;
typedef struct pdd_server pdd_server;

typedef struct {
  int32_t kind;      /* pdd_problem_kind */
  int32_t exit_rule; /* pdd_exit_rule */
  int32_t y_rule;    /* pdd_y_rule */
  int32_t precision; /* pdd_path_precision */
  int64_t max_steps; /* per-path cap; <= 0 means ceil(100 / dt) per estimate */
} pdd_problem_desc;

/* A control grid: n points per axis on [0,1]^D, spacing 1/(n-1), x index
   fastest.  VALUES: n^D samples of v (the library takes centred differences
   inside and second-order one-sided differences on the edges, in FP64, and
   stores the gradient in FP32).  GRADIENT: n^D * D interleaved components.   */
typedef struct {
  int32_t n;         /* points per axis, 3 <= n <= 4097 (2D) / 513 (3D) */
  int32_t kind;      /* pdd_grid_kind */
  int32_t dtype;     /* pdd_dtype */
  int32_t on_device; /* data is a device pointer */
  const void* data;
} pdd_grid_desc;

typedef struct {
  int64_t n_nodes;          /* 0 <= n_nodes < 2^32 (0: nothing to do) */
  const float* coords[3];   /* SoA node coordinates x[], y[], z[] (D used) */
  int32_t coords_on_device; /* coords are device pointers */
  int32_t grid_id;          /* PDD_CV_NONE, PDD_CV_EXACT, or a grid slot */
  int64_t n_paths;          /* paths per node, 1 <= n_paths < 2^32 */
  double dt;                /* time step h > 0 */
  double kappa;             /* per-step cost ratio CV/plain for pred_speedup; <= 0: 1 */
  uint64_t seed;
  uint32_t stream_tag;      /* Philox key word 1 (cascade level or request tag) */
  uint32_t flags;           /* PDD_FLAG_* */
  float* path_phi;          /* EMIT_PATHS: device, n_nodes * n_paths, node-major */
  float* path_xi;           /* EMIT_PATHS: device, same layout */
  int32_t* path_steps;      /* EMIT_PATHS: device, same layout */
} pdd_estimate_args;

/* Caller-owned per-node outputs (SoA, n_nodes entries each).  Any pointer may
   be NULL (not written).  on_device selects device or host pointers.        */
typedef struct {
  int32_t on_device;
  int32_t reserved;
  double* mean_phi;     /* E[phi] estimate */
  double* var_phi;      /* V[phi] (N - 1) */
  double* mean_cv;      /* E[phi + xi] */
  double* var_cv;       /* V[phi + xi] */
  double* cov_phi_xi;   /* Cov[phi, xi] */
  double* var_xi;       /* V[xi] */
  double* rho;          /* Pearson rho[phi, xi]; NaN without a control variate */
  double* se_phi;       /* sqrt(V[phi] / N) */
  double* se_cv;        /* sqrt(V[phi + xi] / N) */
  double* vr;           /* V[phi + xi] / V[phi] */
  double* pred_speedup; /* V[phi] / (kappa V[phi + xi]) */
  double* mean_steps;   /* E[tau_h] / h */
  uint64_t* n_paths;    /* paths accumulated */
  uint64_t* n_truncated;/* paths stopped by max_steps */
} pdd_node_stats;

/* Library ABI version (PDD_ABI_VERSION of the build). */
int pdd_abi_version(void);

/* Thread-local message for the last non-OK status returned on this thread. */
const char* pdd_last_error(void);

/* Create a context on CUDA device `device`.  cuda_stream: a cudaStream_t to
   enqueue on (e.g. torch.cuda.current_stream().cuda_stream), or NULL for a
   stream the context creates and owns.  mem_budget: cap in bytes on the
   context's workspace (0 = no cap).  *out receives the handle.              */
int pdd_ctx_create(int device, void* cuda_stream, size_t mem_budget, pdd_ctx** out);
void pdd_ctx_destroy(pdd_ctx* ctx);
/* Switch the stream; waits for the previous stream's pending work first. */
int pdd_ctx_set_stream(pdd_ctx* ctx, void* cuda_stream);
/* Kernel timing: when enabled, every path-kernel launch is bracketed by CUDA
   events on the launching stream.  pdd_ctx_kernel_time waits for them and
   returns the summed milliseconds and the number of timed launches since the
   previous call; per_launch_ms (nullable, `capacity` entries) receives the
   individual durations in launch order.  The event list is then cleared.   */
int pdd_ctx_set_timing(pdd_ctx* ctx, int enable);
int pdd_ctx_kernel_time(pdd_ctx* ctx, double* total_ms, int64_t* launches, double* per_launch_ms,
                        int64_t capacity);
/* Number of library kernels launched by this context since creation. */
int pdd_ctx_launch_count(pdd_ctx* ctx, int64_t* launches);
/* Number of CUDA graphs captured by PDD_FLAG_GRAPH calls on this context. */
int pdd_ctx_graph_count(pdd_ctx* ctx, int64_t* captures);
/* Launch shape of the path kernels: block_threads (multiple of 32 in
   [32, 512]; 0 = 128) and a cap on the grid size (0 = occupancy x SM count).
   The shape changes only the speed: the results are exact sums keyed by
   (node, path), identical for every shape.                                  */
int pdd_ctx_set_launch(pdd_ctx* ctx, int block_threads, int max_blocks);
/* Euler steps a path kernel takes per iteration, between lane refills (the
   scheduling quantum): PDD_ITER_SHORT = 2 in 2D / 4 in 3D, PDD_ITER_LONG =
   4 (8 without a control variate) in 2D / 8 in 3D (FP32 paths; FP64 paths
   always take the short one), PDD_ITER_AUTO
   (the default) = long when the segments with time steps above 2e-3 hold at
   most 5 % of the launch's expected path-steps (n_nodes x n_paths / h), short
   otherwise.  Longer iterations pay the refill and exit bookkeeping once per
   more steps; a lane whose path ends early in an iteration idles for the rest
   of it.  Like the launch shape, the choice changes only the speed (results
   are exact sums keyed by node and path).  pdd_autotune sets it too.
   pdd_ctx_get_launch reads the context's shape and iteration choice (any
   output may be NULL).                                                     */
#define PDD_ITER_AUTO 0
#define PDD_ITER_SHORT 1
#define PDD_ITER_LONG 2
int pdd_ctx_set_iteration(pdd_ctx* ctx, int mode);
int pdd_ctx_get_launch(pdd_ctx* ctx, int* block_threads, int* max_blocks, int* iteration);
/* Paths per lane a warp claims from a launch's path cursor at once (one
   atomic per 32 x paths_per_lane consecutive path indices; the warp's lanes
   then run them one at a time as they finish): 0 (the default) = automatic,
   4 when the launch's paths are short (the segments with time steps of at
   most 2e-3 hold at most 5 % of its expected path-steps) and it has at least
   4 x 32 paths for every warp that can be resident, 1 otherwise; or a power
   of two in [1, 64].  Larger claims hit the
   cursor less often (it matters for paths of ~10 steps) but leave more
   unstarted paths with one warp at the end of a launch.  Like the launch
   shape, the claim changes only the speed.  PDD_ERR_INVALID for other values.
   pdd_autotune searches it (1, 4, 16 against automatic).
   pdd_ctx_get_claim reads the setting (0 = automatic).                       */
int pdd_ctx_set_claim(pdd_ctx* ctx, int paths_per_lane);
int pdd_ctx_get_claim(pdd_ctx* ctx, int* paths_per_lane);
/* Stops the work in flight on the context (no counterpart in the paper):
   callable from any thread, also while another thread waits inside an
   estimate on this context.  The kernels take no further paths (a copy on a
   stream of the context's own moves the launch's path cursor past its last
   path; nothing on the device waits for it), the paths already running end
   normally, and the call in flight returns PDD_ERR_CANCELLED with the
   statistics of the paths that ran (n_paths per node tells how many).
   Calls that start after pdd_ctx_abort returns are not affected.  If the call
   in flight was about to finish it may report PDD_ERR_CANCELLED with every
   path run.  Applies to pdd_estimate_nodes / _levels, pdd_accumulate, the
   coupled calls and what runs on them (fit, MLMC); not to the
   allocation-free call or to servers (use pdd_cancel).  It allocates
   nothing: the context made its stream, event and 16 page-locked bytes.    */
int pdd_ctx_abort(pdd_ctx* ctx);

int pdd_create_problem(pdd_ctx* ctx, const pdd_problem_desc* desc, pdd_problem** out);
int pdd_destroy_problem(pdd_problem* problem);

/* Copy a control grid into slot grid_id (0 <= grid_id < PDD_MAX_GRIDS) and
   build its FP32 gradient table on the device (Sec. 3.1 lookup table; the
   gradient that enters F = -sigma^T grad v, eq. F:ExactF).  The caller may
   free `data` on return.  Waits for the context's stream before replacing
   an existing grid.                                                         */
int pdd_set_control_grid(pdd_problem* problem, int grid_id, const pdd_grid_desc* desc);

/* Estimate all nodes: n_nodes x n_paths paths of Algorithm 1.  Synchronous
   unless PDD_FLAG_ASYNC (allowed only with device coords and device outputs).
   Returns PDD_WARN_TRUNCATED (synchronous calls) when any path hit
   max_steps, PDD_ERR_OVERFLOW when a score left |score| < 32768.          */
int pdd_estimate_nodes(pdd_problem* problem, const pdd_estimate_args* args, pdd_node_stats* out);

/* Several levels -- e.g. the levels of the multigrid-like cascade (Sec. 1,
   Algorithm 5), each with its own nodes, n_paths, dt, control grid, seed,
   stream_tag and outputs -- in ONE persistent launch: the paths of all levels
   form one work list, levels with the smallest dt (the longest paths) first,
   so short paths fill the tail of long ones.  Results are bit-identical to one
   pdd_estimate_nodes call per level.  levels[l].flags may hold
   PDD_FLAG_EMIT_PATHS; `flags` (the call's) may hold PDD_FLAG_ASYNC and
   PDD_FLAG_GRAPH (both need device coordinates and outputs).  With
   PDD_FLAG_GRAPH the clear / path-kernel / finalise sequence is captured once
   into a CUDA graph (kept by the context) and replayed by later calls with
   identical arguments; different arguments re-capture.  Levels may mix
   control grids with plain levels (grid_id = PDD_CV_NONE) but not with
   PDD_CV_EXACT.  n_levels in [1, PDD_MAX_LEVELS]; outs[l] receives level l. */
int pdd_estimate_levels(pdd_problem* problem, int n_levels, const pdd_estimate_args* levels,
                        pdd_node_stats* outs, uint32_t flags);

/* Exact node records, for checkpoint / resume and for merging runs.  A node
   record is PDD_RECORD_WORDS uint64 words of exact integer sums (128-bit sums
   of the fixed-point scores, their squares and product, the exit indices and
   their squares, the path count and the truncation count).  Records add
   element-wise with carries (pdd_records_merge), so paths can be split over
   calls, processes or GPUs in any way and merged into the same bits.
   pdd_accumulate runs paths path_offset .. path_offset + args->n_paths - 1 of
   every node (same random streams as pdd_estimate_nodes) and adds their sums
   into `records` (device, n_nodes x PDD_RECORD_WORDS, zeroed by the caller
   before the first call); synchronous unless args->flags has PDD_FLAG_ASYNC.
   pdd_finalize_records turns records (device) into the statistics of
   pdd_estimate_nodes (out: host or device per out->on_device).
   pdd_records_merge adds n_nodes host records `src` into host records `dst`. */
#define PDD_RECORD_WORDS 16
int pdd_accumulate(pdd_problem* problem, const pdd_estimate_args* args, uint64_t path_offset,
                   uint64_t* records);
int pdd_finalize_records(pdd_ctx* ctx, const uint64_t* records, int64_t n_nodes, double kappa,
                         pdd_node_stats* out);
int pdd_records_merge(uint64_t* dst, const uint64_t* src, int64_t n_nodes);

/* Multilevel coupling (the multilevel Monte Carlo variant the paper names as
   future work, Sec. 1 and Sec. 7), 2D and 3D problems with FP32 paths.  For
   every (node, path) the library runs a FINE path at h/2 = args->dt / 2 on
   the path's own random stream (the same path pdd_estimate_nodes runs at
   dt/2) and a COARSE path at h = args->dt driven by the sums of pairs of fine
   increments, dW_c(k) = dW_f(2k) + dW_f(2k+1); each path has its own exit.
   out_fine receives the statistics of the fine level (as pdd_estimate_nodes
   at dt/2); out_diff those of the level difference: mean_phi / var_phi of
   phi_f - phi_c, mean_cv / var_cv of (phi_f + xi_f) - (phi_c + xi_c),
   mean_steps of the coarse path.  The difference has a small variance, so
   E[phi_h/2] - E[phi_h] is cheap to resolve (the multilevel telescoping sum).
   Coordinates and outputs are device pointers; with PDD_FLAG_EMIT_PATHS the
   per-path arrays hold 2 x n_nodes x n_paths entries, fine first.
   pdd_accumulate_coupled runs pairs path_offset .. path_offset + n_paths - 1
   and adds their exact sums into rec_fine / rec_diff (device, n_nodes x
   PDD_RECORD_WORDS each, zeroed by the caller before the first call), the
   records pdd_finalize_records turns into the two statistics above.        */
int pdd_estimate_coupled(pdd_problem* problem, const pdd_estimate_args* args,
                         pdd_node_stats* out_fine, pdd_node_stats* out_diff);
int pdd_accumulate_coupled(pdd_problem* problem, const pdd_estimate_args* args,
                           uint64_t path_offset, uint64_t* rec_fine, uint64_t* rec_diff);

/* Multilevel Monte Carlo estimate of the nodal values (the MLMC variant the
   paper leaves to future work, Sec. 1 and Sec. 7; the level-adaptive
   sample allocation is Giles' standard one).  Level 0 is Algorithm 1 at
   h_0 = dt0; level l >= 1 is the coupled difference phi_{h_l} - phi_{h_(l-1)},
   h_l = dt0 / 2^l (pdd_accumulate_coupled with dt = h_(l-1)); level l draws
   stream_tag_base + l.  With a control grid (or PDD_CV_EXACT) every level
   uses the controlled score phi + xi.  Starting from min_levels levels with
   n_pilot paths each, the driver repeats:
     1. run the missing paths of every level (path indices continue, so the
        result equals one run with the final counts);
     2. from the records: per node the level mean m_l,i and variance v_l,i,
        and the cost c_l,i (mean exit index, fine + coarse for l >= 1);
        Vbar_l, Cbar_l = their node means;
     3. N_l = ceil(2 eps^-2 sqrt(Vbar_l / Cbar_l) sum_k sqrt(Vbar_k Cbar_k))
        (pdd_mlmc_allocate: least total cost with node-mean variance
        sum_l Vbar_l / N_l <= eps^2 / 2);
     4. when every level has its N_l: the bias estimate
        b = max(r_L, r_(L-1) / 2^alpha) / (2^alpha - 1), where r_l is the
        node-RMS of m_l,i with the sampling noise v_l,i / N_l removed; stop
        if b <= eps / sqrt(2), else add a level (up to max_levels).  With
        min_levels == max_levels the levels are fixed (a bias model chose
        them) and b is only reported.
   Per node: estimate = sum_l m_l,i, variance = sum_l v_l,i / N_l, and the
   Talay-Tubaro (Richardson) extrapolation on the finest pair,
   extrapolated = estimate + m_L,i / (2^alpha - 1), with its variance
   sum_(l<L) v_l,i / N_l + (2^alpha / (2^alpha - 1))^2 v_L,i / N_L.
   Output arrays are host arrays of n_nodes (any may be NULL).  Returns
   PDD_OK when converged, PDD_WARN_NOT_CONVERGED when max_levels, the round
   cap (64) or the 2^32 path limit stopped it first (outputs valid), or an
   error status.                                                            */
#define PDD_MLMC_MAX_LEVELS 16
typedef struct {
  int64_t n_nodes;
  const float* coords[3];     /* device SoA coordinates */
  int32_t grid_id;            /* control grid, PDD_CV_NONE or PDD_CV_EXACT */
  int32_t min_levels;         /* 2 .. max_levels */
  int32_t max_levels;         /* min_levels .. PDD_MLMC_MAX_LEVELS */
  int32_t reserved;
  double dt0;                 /* step of level 0 */
  int64_t n_pilot;            /* first paths of every level, >= 2 */
  double target_rmse;         /* eps > 0: node-mean MSE against u <= eps^2 */
  double alpha;               /* weak order (1 with the Gobet-Menozzi test) */
  uint64_t seed;
  uint32_t stream_tag_base;
  uint32_t reserved2;
} pdd_mlmc_args;
typedef struct {
  double* estimate;           /* n_nodes (host, nullable) */
  double* variance;           /* n_nodes */
  double* extrapolated;       /* n_nodes: Talay-Tubaro on the finest pair */
  double* extrap_variance;    /* n_nodes */
  int32_t n_levels;           /* levels used, L + 1 */
  int32_t rounds;             /* passes of steps 1-4 */
  int64_t n_paths[PDD_MLMC_MAX_LEVELS];   /* N_l */
  double var_mean[PDD_MLMC_MAX_LEVELS];   /* Vbar_l */
  double cost_mean[PDD_MLMC_MAX_LEVELS];  /* Cbar_l, path-steps per sample */
  double corr_rms[PDD_MLMC_MAX_LEVELS];   /* r_l */
  double bias_estimate;       /* b of the last test */
  int64_t path_steps;         /* path-steps of all levels (exit indices summed) */
} pdd_mlmc_out;
int pdd_mlmc_allocate(int n_levels, const double* var_mean, const double* cost_mean,
                      double target_rmse, int64_t* n_paths);
int pdd_mlmc(pdd_problem* problem, const pdd_mlmc_args* args, pdd_mlmc_out* out);

/* Fast fit of nodal constants (Algorithm 3, Sec. 5 H5).  For every node the
   library runs n_paths realisations of Algorithm 1 at each of n_h equispaced
   time steps h_max = h_1 > ... > h_{n_h} = h_min (the "cloud"), drawing the
   auxiliary variate psi = -int Y sigma^T grad(w) . dW alongside, where grad(w)
   is control grid `grid_id` (PDD_CV_NONE: no auxiliary variate), all (node, h)
   pairs in persistent launches of up to PDD_MAX_LEVELS time steps each
   (stream_tag_base + j keys time step j).  Per node it then fits
     first moments  E[eta_h] = E[eta_0] + B h^delta    (normal noise, identity
                    link: ordinary least squares) for eta = phi, tau, phi psi;
     variances      E[V[eta_h]] = V[eta_0] + B h^delta (gamma noise, identity
                    link: iteratively reweighted least squares) for phi, psi;
   and returns E[phi], beta, V[phi], alpha, E[tau], K = 4 q^2 E[tau]
   (2|beta|)^(1/delta) (eq. F:Pointwise_cost), Cov[phi,psi], V[psi] and
   rho[phi,psi].  Output arrays are host arrays of n_nodes (any may be NULL);
   `cloud` (nullable, host, n_nodes x n_h x 6) receives h, E[phi_h],
   V[phi_h], E[tau_h], Cov[phi_h,psi_h], V[psi_h].                          */
typedef struct {
  int64_t n_nodes;
  const float* coords[3];   /* device SoA coordinates */
  int32_t grid_id;          /* grid of grad(w) for psi, or PDD_CV_NONE */
  int32_t n_h;              /* time steps in the cloud, 2 .. 4096 */
  double h_min, h_max;      /* 0 < h_min < h_max */
  int64_t n_paths;          /* realisations per (node, h) */
  double delta;             /* weak order: 1 (Gobet-Menozzi), 0.5 (naive test) */
  double q;                 /* confidence factor of the balanced simulation (eq. F:N_y_h) */
  uint64_t seed;
  uint32_t stream_tag_base;
  uint32_t reserved;
} pdd_fit_args;

typedef struct {
  double *E_phi, *beta, *V_phi, *alpha, *E_tau, *K, *cov_phi_psi, *V_psi, *rho_phi_psi;
  double* cloud;
} pdd_fit_out;

int pdd_fit_constants(pdd_problem* problem, const pdd_fit_args* args, pdd_fit_out* out);

/* Scheduling of the tolerance sequence (Algorithm 4, with the sensitivity
   formula eq. F:Sensitivity_formula).  Host computation, no GPU.  Inputs per
   node i (arrays of n_nodes): K_i, beta_i, alpha_i, V_i[phi], V_i[psi],
   rho_i[phi, psi] (as fitted by pdd_fit_constants), and delta, kappa and the
   nodal target tolerance a0.  Step j solves
     a_{j+1} = argmin_{a > a_j} sum_i K_i V_i[phi] ( kappa (1 - r_i^2(a)
               + |alpha_i r_i(a) / beta_i| a_j) + (a_j / a)^{2 + 1/delta} ),
     r_i^2(a) = 1 - V_i[psi] a^2 (1 - rho_i^2) / (4 V_i[phi])  (clamped at 0),
   by a log-spaced scan and golden-section refinement on (a_j, a_max], a_max
   the largest a with some r_i^2 > 0, and stops when the predicted speedup
   S_j = sum_i K_i V_i[phi] / (minimum value) falls below min_speedup (the
   paper stops at 1.5) or after max_levels levels.  Outputs: a[0] = a0,
   a[1..J] the coarser tolerances (a has room for max_levels + 1 values),
   speedup[j] = S_j of step j (speedup[J] is the rejected step's, NaN when
   no step was tried; room for max_levels + 1 values); *n_levels = J.        */
typedef struct {
  int64_t n_nodes;
  const double *K, *beta, *alpha, *V_phi, *V_psi, *rho_phi_psi;
  double delta, kappa, a0, min_speedup;
} pdd_schedule_args;

int pdd_schedule(const pdd_schedule_args* args, double* a, double* speedup, int max_levels,
                 int* n_levels);

/* Balanced simulation per node (Definition "Balanced MC simulation",
   eq. F:N_y_h): at tolerance a with confidence factor q and weak order delta,
     h_i = (a / (2 |beta_i|))^(1/delta)   (bias = a/2),
     N_i = ceil(4 q^2 V_i / a^2)           (statistical error = a/2),
   h_i clamped to [h_min, h_max] (beta_i = 0 gives h_max) and N_i to
   [n_min, n_max].  V_i is the variance of the score the level runs: V[phi]
   for a plain level, V[phi + xi] with a control variate.  Host computation,
   no GPU; host arrays of n_nodes (beta, var in; h, n_paths out).
   PDD_ERR_INVALID on bad arguments.                                         */
int pdd_balanced_plan(int64_t n_nodes, double a, double q, double delta, const double* beta,
                      const double* var, double h_min, double h_max, int64_t n_min,
                      int64_t n_max, double* h, int64_t* n_paths);

/* The scheduling model's prediction for one level of the cascade (Algorithm 4
   objective, eq. F:Sensitivity_formula): the level at tolerance aj that uses
   the control variate of the coarser level at tolerance a (a <= 0: a plain
   level).  Per node i, with r_i^2(a) as in pdd_schedule:
     rho2[i] = max(r_i^2(a) - |alpha_i r_i(a) / beta_i| aj, 0), the predicted
               rho^2[phi_h, xi_h] (0 for a plain level);
     cost[i] = K_i V_i[phi] w_i / aj^(2 + 1/delta), the predicted path-steps
               (eq. F:Pointwise_cost), w_i = 1 - r_i^2(a) + |alpha_i r_i(a) /
               beta_i| aj for a controlled level (multiply by kappa for its
               cost in plain-step units) and 1 for a plain one.
   Host computation; host arrays of s->n_nodes.  PDD_ERR_INVALID on bad
   arguments.                                                               */
int pdd_schedule_predict(const pdd_schedule_args* s, double a, double aj, double* rho2,
                         double* cost);

/* Autotuner: runs `sample` (device coordinates) under candidate launch shapes
   (128/256/512 threads per block, full and half occupancy) with the automatic
   iteration and claim, then the fastest shape with the short and the long
   iteration (pdd_ctx_set_iteration; FP32 paths), then with claims of 1, 4 and
   16 paths per lane (pdd_ctx_set_claim), times each with CUDA events on the
   context's stream, and keeps the fastest as the context's launch shape,
   iteration and claim.  Outputs (nullable): the chosen shape and its time
   (pdd_ctx_get_launch gives the iteration, pdd_ctx_get_claim the claim).
   Results of later calls do not depend on the choice.                       */
int pdd_autotune(pdd_problem* problem, const pdd_estimate_args* sample, int* best_threads,
                 int* best_max_blocks, double* best_ms);

/* ---- Serving: continuous batching of estimate requests -------------------
   A server admits requests (one pdd_estimate_args each: nodes, n_paths, dt,
   grid, seed, stream_tag) while a slot of the running batch and room in its
   device arena are free, and runs the admitted requests together: every
   scheduler iteration is one persistent launch that carries slices of paths
   of up to max_active requests (requests of the same problem and
   control-variate class share a launch; `policy` decides the slices), so
   requests arriving while others run join the next launch.  Results are bit-identical to pdd_estimate_nodes
   on the same arguments (exact sums keyed by node and path).  A scheduler
   thread owned by the server issues launches on two streams of its own and
   polls CUDA events; nothing on the device waits.                          */
typedef struct {
  int32_t max_active;          /* requests in the running batch, 1..128 (0: 32) */
  int32_t max_queue;           /* pending requests before PDD_ERR_BUSY (0: 256) */
  int64_t quantum_path_steps;  /* target path-steps per launch (0: 8e9) */
  size_t device_arena_bytes;   /* device memory for admitted requests (0: 256 MiB);
                                  a request takes about 252 B per node */
  int32_t policy;              /* how a launch's path-steps are shared among the batch:
                                  PDD_SERVE_FAIR (0): equal shares; PDD_SERVE_SHORTEST (1):
                                  requests with the least remaining work first, each up to
                                  all its remaining paths, until the quantum is spent (less
                                  latency for small requests; large ones wait under overload);
                                  PDD_SERVE_EARLIEST_DEADLINE (2): the same fill in submission
                                  order (every request has the relative deadline deadline_s),
                                  under which the deadline admission bounds every admitted
                                  request's completion by deadline_s, as far as the predicted
                                  work and rate hold */
  int32_t reserved;            /* 0 */
  double deadline_s;           /* > 0: admission by predicted work -- pdd_submit refuses
                                  (PDD_ERR_DEADLINE) a request whose predicted path-steps,
                                  added to the predicted remaining path-steps of every
                                  queued and running request, would take longer than
                                  0.8 x deadline_s at the server's measured rate (the rest
                                  is a margin for the error of the predicted work and rate;
                                  a guarantee under PDD_SERVE_EARLIEST_DEADLINE as far as the
                                  predictions hold, an estimate under the other policies);
                                  0: no deadline */
  double rate_hint;            /* path-steps/s assumed until the server has measured its own
                                  rate over retired launches (0: 1e11) */
} pdd_server_desc;
#define PDD_SERVE_FAIR 0
#define PDD_SERVE_SHORTEST 1
#define PDD_SERVE_EARLIEST_DEADLINE 2

typedef struct {
  int64_t submitted, admitted, rejected_busy, rejected_invalid, rejected_nomem;
  int64_t completed, cancelled, failed, launches, pending, active;
  int64_t path_steps;  /* Euler steps executed by retired launches, whether or not
                          their requests later completed */
  int64_t rejected_deadline;      /* refused by the deadline (PDD_ERR_DEADLINE) */
  int64_t completed_path_steps;   /* Euler steps of completed requests (their results'
                                     mean exit index x paths): goodput = this / path_steps */
  int64_t backlog_path_steps;     /* predicted path-steps still to run for queued and
                                     running requests */
  int64_t rate_path_steps_per_s;  /* the rate admission currently assumes */
} pdd_server_stats;

int pdd_server_create(pdd_ctx* ctx, const pdd_server_desc* desc, pdd_server** out);
/* Copies the request (coordinates from host or device memory, read before the
   call returns) and queues it.  Its predicted work is n_nodes x n_paths x
   (expected exit index at its dt); the expected exit index of each (problem,
   dt) comes from a pilot launch (64 paths from each of up to 128 of the
   request's nodes, plain estimator) that the first request with that pair
   runs before this call returns -- the only time pdd_submit waits for the
   GPU -- and is refined with the exit indices of every completed request.
   PDD_ERR_BUSY when max_queue requests are pending (retry or shed),
   PDD_ERR_DEADLINE when desc.deadline_s is set and the request's predicted
   work would not finish within it after the backlog, PDD_ERR_NOMEM when the
   request can never fit the arena, PDD_ERR_INVALID for malformed requests
   (EMIT_PATHS is not served).  Each refusal is counted apart in the
   statistics.  *ticket identifies the request.                             */
int pdd_submit(pdd_server* server, pdd_problem* problem, const pdd_estimate_args* args,
               uint64_t* ticket);
/* Waits up to timeout_us (0: do not wait) for the request.  PDD_OK: results
   copied into *out (host or device per out->on_device) and the ticket is
   released; PDD_ERR_NOT_READY / PDD_ERR_TIMEOUT: still running (ticket kept);
   PDD_ERR_CANCELLED: cancelled (ticket released); other errors: the request
   failed (ticket released) -- PDD_ERR_OVERFLOW (or PDD_ERR_BOUNDS in the
   bounds-checked build) fails every request with a slice in the launch whose
   error word was set.                                                       */
int pdd_poll(pdd_server* server, uint64_t ticket, pdd_node_stats* out, int timeout_us);
/* Stops issuing the request's paths; its memory is released once no launch
   in flight uses it; pdd_poll then returns PDD_ERR_CANCELLED.               */
int pdd_cancel(pdd_server* server, uint64_t ticket);
int pdd_server_get_stats(pdd_server* server, pdd_server_stats* out);
/* Test hook, host side only: 1 = the next admission fails as if the arena
   allocation failed (that request ends with PDD_ERR_NOMEM); 2 = the next
   scheduled request is dropped as if the worker running it died (it ends
   with PDD_ERR_CANCELLED).  Other requests are unaffected.                 */
int pdd_server_inject_fault(pdd_server* server, int fault);
/* Cancels queued and running requests, waits for launches in flight (they
   end by themselves) and frees the server.                                  */
void pdd_server_destroy(pdd_server* server);

/* ---- Allocation-free estimate (the paper has no counterpart) -------------
   The same estimate as pdd_estimate_nodes, for callers that cannot let the
   library allocate device memory: for example an application whose own pool
   allocator has reserved the device memory, or a latency-critical loop that
   must not pay for cudaMalloc/cudaFree and the device-wide synchronisation
   they can cause.  Instead of the context's workspace, its scratch (path
   cursor, error bits and the per-node exact sums) is one fixed device array
   of 256 + 128 * PDD_NOALLOC_MAX_NODES bytes (about 512 KiB), which every GPU
   that loads the library holds until the process exits.  The call performs
   no cudaMalloc, cudaFree or other allocating call.
   - n_nodes <= PDD_NOALLOC_MAX_NODES, else PDD_ERR_INVALID with a message.
   - Coordinates, outputs and EMIT_PATHS buffers must be device pointers
     (host buffers would need device staging memory).
   - Control grids are loaded beforehand with pdd_set_control_grid (which
     allocates, so it belongs to set-up).
   - The first call on each device looks up and caches the array's device
     address (cudaGetSymbolAddress); make that first call before any stream
     capture.
   - With CUDA's lazy module loading (the default), the first launch of each
     kernel variant -- one per (problem kind, path precision, control-variate
     mode: none, grid or exact) -- loads that kernel, and loading can reserve
     device memory.  Warm up once per variant (any call, e.g. with few paths)
     before relying on the call allocating nothing.
   - The launch settings are the context's (shape, iteration and claim:
     pdd_ctx_set_launch / _set_iteration / _set_claim / pdd_autotune), as for
     pdd_estimate_nodes; the caller's current device is left unchanged.
   - Every call uses the same array, which keeps the previous call's contents
     (each call clears what must start at zero).  Calls that can overlap on
     the GPU -- different streams or different contexts -- race on it and give
     wrong results: serialise them.  Calls on one context are serialised.
   Flags, statuses and outputs are those of pdd_estimate_nodes.             */
#define PDD_NOALLOC_MAX_NODES 4096
int pdd_estimate_nodes_noalloc(pdd_problem* problem, const pdd_estimate_args* args,
                               pdd_node_stats* out);

#ifdef __cplusplus
}
#endif
#endif /* PDD_H */
