/*
 * phsvds.h -- C ABI of the GB300 (sm_103a) implementation of PHSVDS.
 *
 * PHSVDS (Wu & Stathopoulos, "A preconditioned hybrid SVD method for computing
 * accurately singular triplets of large matrices", arXiv 1408.5535) computes the
 * k smallest (or largest) singular triplets (sigma_i, u_i, v_i) of a sparse
 * A in R^{m x n}, m >= n, full column rank (Section 1, eq. 1.1), in two stages:
 *   stage 1 (Algorithm 1): block GD+k on C = A^T A to the accuracy the normal
 *           equations allow (Section 3.1, the dynamic tolerance delta_C);
 *   stage 2 (Algorithm 2): Jacobi-Davidson-type outer loop on the augmented
 *           B = [0 A^T; A 0] with the refined projection (Section 3.2),
 * until sqrt(||r_u||^2 + ||r_v||^2) <= tol * ||A|| (Section 5).
 *
 * Conventions for every entry point:
 *  - All matrices are dense column-major unless stated otherwise; CSR arrays
 *    are 0-based with row_ptr[0] = 0 and row_ptr[m] = nnz, column indices of a
 *    row strictly increasing (validated; violation -> PHSVDS_ERR_INVALID).
 *  - The caller owns every pointer it passes; the library never frees them.
 *    Pointers are host pointers unless the argument says "device" or the
 *    call's ptr_on_device flag is 1.
 *  - The library owns its device copies and workspaces; they live until
 *    phsvds_destroy (or until the next solve on the same handle).  The device
 *    memory they took stays reserved in the handle's own memory pool until
 *    phsvds_destroy, so that repeated solves do not map it again.
 *  - Errors: every call returns a phsvds_status.  On error nothing is written to
 *    the output arrays except what the status documents; phsvds_last_error()
 *    returns a one-line description of the last failure on this handle.
 *  - A handle is not thread-safe; use one handle per host thread.
 */
#ifndef PHSVDS_H
#define PHSVDS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct phsvds_ctx* phsvds_handle;

typedef enum {
    PHSVDS_OK = 0,
    PHSVDS_ERR_INVALID = 1,        /* bad argument, CSR structure, m < n, k out of range */
    PHSVDS_ERR_NOT_CONVERGED = 2,  /* max_restarts reached (Section 5: 10000 restarts) */
    PHSVDS_ERR_BREAKDOWN = 3,      /* orthogonalisation could not extend the basis */
    PHSVDS_ERR_NAN = 4,            /* a NaN/Inf appeared in A or in the iteration */
    PHSVDS_ERR_TIMEOUT = 5,        /* wall-clock limit (opts.time_limit_s) reached */
    PHSVDS_ERR_CUDA = 6,           /* a CUDA runtime call failed */
    PHSVDS_ERR_OOM = 7             /* device allocation failed */
} phsvds_status;

typedef enum { PHSVDS_SMALLEST = 0, PHSVDS_LARGEST = 1 } phsvds_target;

/* Correction operator of stage 1 (Section 4): identity (plain GD+k), or the
 * Jacobi preconditioner M = (diag(C) - theta I)^{-1}, diag(C)_j = ||A e_j||^2,
 * applied in the Olsen form t = M r - e M x, e = x^T M r / x^T M x, or the
 * learned correction network (no counterpart in the paper: a 3-layer 3x3
 * convolution network on the grid of a grid-structured operator, mapping
 * [r / ||r|| * sqrt(n), feature channels] to the correction t; opts.learned_*),
 * or a preconditioner M ~ A given by the caller (Sec. 4, square A, M diagonal:
 * opts.precond_M): M^{-1} M^{-T} for C in stage 1 and [0 M^{-1}; M^{-T} 0]
 * for B in stage 2, both in the Olsen form. */
typedef enum { PHSVDS_PREC_NONE = 0, PHSVDS_PREC_JACOBI = 1, PHSVDS_PREC_LEARNED = 2,
               PHSVDS_PREC_GIVEN = 3 } phsvds_precond;

/* Parameters of the learned correction network: 3024 BF16 values, layer-major
 * (16x4x3x3, 16x16x3x3, 1x16x3x3), each [out][in][row][col]. */
#define PHSVDS_CNN_NPARAM 3024
/* Floats of the workspace of phsvds_cnn_forward / _backward for a batch of B
 * images of npix pixels (8-byte aligned). */
#define PHSVDS_CNN_WORK_FLOATS(B, npix) (65 * (int64_t)(B) * (int64_t)(npix) + 2 * PHSVDS_CNN_NPARAM + 2 * (int64_t)(B))

/* PHSVDS_FP64: every step in FP64.  PHSVDS_MIXED: stage 1 first runs with FP32
 * storage, FP32 SpMM and Gram products (FP64 reduction across thread blocks) to
 * the FP32-attainable tolerance, then continues in FP64 from that basis; the
 * projected eigenproblems, stage 2 and the final residuals are FP64. */
typedef enum { PHSVDS_FP64 = 0, PHSVDS_MIXED = 1 } phsvds_precision;

/* SpMM schedule for C X = A^T (A X): fused single pass with L2 atomics, or two
 * phases (Z = A X kept in L2, then A^T Z from a CSC copy), or picked by timing. */
typedef enum { PHSVDS_SPMM_AUTO = 0, PHSVDS_SPMM_FUSED_ATOMIC = 1, PHSVDS_SPMM_TWO_PHASE = 2 } phsvds_spmm_schedule;

typedef struct {
    int block_size;        /* stage-1 block size b (1..8), default 1 */
    int max_basis;         /* maxBasisSize, default 35 (Section 5); max_basis + 8 <= 64 */
    int min_restart;       /* minRestartSize, default 21 (Section 5); 2 b <= min_restart and
                              min_restart + b <= max_basis, b = min(block_size, k) */
    int max_restarts;      /* per stage, default 10000 (Section 5) */
    double eps_factor;     /* delta_C floor = eps_factor * eps (O(||C|| eps), Sec. 3.1), default 4 */
    phsvds_precision precision;
    phsvds_spmm_schedule spmm;
    int stage2;            /* 1 = automatic switch (Sec. 3.1), 0 = stage 1 only */
    int rayleigh_ritz;     /* 1 = Algorithm 1 step 3 before stage 2, default 1 */
    uint64_t seed;         /* SplitMix64 seed of the random vectors the method draws */
    double time_limit_s;   /* 0 = none */
    int profile;           /* 1 = time kernel classes with CUDA events (stats.t_*_ms), default 0 */
    /* PHSVDS_PREC_LEARNED: host pointers, copied at the start of the solve.
     * learned_params: PHSVDS_CNN_NPARAM BF16 values; learned_features: 3 planes
     * of n floats (log diffusion, beta_x, beta_y per grid cell); the grid is
     * grid_nx x grid_ny = n, cell (x, y) = column y*grid_nx + x of A. */
    const void* learned_params;
    const float* learned_features;
    int grid_nx, grid_ny;
    /* learned correction falls back (to Jacobi, else none) when a window of
     * this many stage-1 iterations neither locks a vector nor halves the
     * smallest target residual; default 200, 0 = never */
    int stall_window;
    /* recording of the plain method's residuals (training data of the learned
     * correction): every record_every-th FP64 stage-1 iteration, the residual
     * of the first target is written to host record_r + i*n (record_max
     * vectors at most); stats.recorded counts them.  NULL = off. */
    double* record_r;
    int record_max;
    int record_every;
    /* projected eigensolver of stage 1: 0 = FP64 Jacobi spread over an 8-CTA
     * cluster; 1 = one-CTA FP64 Jacobi with each round's work compacted to
     * its rotating pairs; 2 (default) = an FP32 Jacobi pass, the exact FP64
     * frame rebuilt from it, and an FP64 Jacobi clean-up of the pairs touching
     * the targets, whenever the last targets were >= 1e-5 theta_max (FP32
     * resolves them; GB300's FP64 latency is ~14x its FP32 latency), else 0 */
    int projected_solver;
    /* optional initial guess of stage 1 (the hand-off between runs of
     * Sec. 3.3: e.g. the right singular vectors of an earlier solve): host
     * pointer to init_nv columns of length n, column-major, that replace the
     * default start (ones(n,1)/sqrt(n) plus random columns, Sec. 5); they are
     * copied at the start of the solve and orthonormalised on the device.
     * NULL = default start; init_nv = 0 means k columns; 0 <= init_nv <=
     * max_basis. */
    const double* init_V;
    int init_nv;
    /* PHSVDS_MIXED only: how the FP64 continuation of stage 1 expands its
     * basis.  0 = plain GD+k (the residual); 1 (default) = the Jacobi-Davidson
     * correction of the JDQMR form (Sec. 4): for each targeted Ritz pair
     * (theta, x) an approximate solution t of (I - QQ^T)(C - theta I)
     * (I - QQ^T) t = r, Q = [locked vectors, x], by MINRES in FP32 with the
     * FP32 copy of A, at most inner_maxit steps (default 60) or until its
     * residual falls by inner_tol (default 1e-3).  2: the FP32 stage too
     * (FP32 outer Rayleigh-Ritz, FP32 MINRES): faster where the FP32 stage
     * runs long on ill-conditioned smallest targets, but near the FP32
     * floor the FP32 correction is rounding noise and the stage can stall
     * (as on the largest triplets of a matrix with ||A|| ~ 3e4), so it is
     * not the default.  With PHSVDS_PREC_JACOBI
     * the system is preconditioned by D = diag(C), solved symmetrically in
     * y = D^{1/2} t with Q = [locked vectors, the block's Ritz vectors]
     * (this replaces the Olsen-Jacobi correction of the FP64 continuation).
     * The Rayleigh-Ritz step, the convergence test and the orthogonalisation
     * stay in FP64, so the accuracy is that of the FP64 method. */
    int mixed_inner;
    int inner_maxit;
    double inner_tol;
    /* 1: stage 2 of a SMALLEST solve corrects with the preconditioner that
     * Sec. 4 builds for B from a preconditioner M ~ C^{-1} of stage 1,
     * [0 A M; M A^T 0], here with M = diag(C)^{-1} (the unshifted Jacobi
     * preconditioner of C), in the Olsen form t = P r - e P x,
     * e = x^T P r / x^T P x (two products with A and two with A^T per
     * iteration); 0 (default): t = r. */
    int stage2_precond;
    /* PHSVDS_PREC_GIVEN: host pointer to the n diagonal entries of M ~ A
     * (square A, m = n; every entry finite and nonzero), copied at the start
     * of the solve. */
    const double* precond_M;
    /* the correction of stage 2: 0 (default) t = r (GD, the PHSVDS(GD+k)
     * variant); 1 = the JDQMR form (Sec. 4): t an inexact solution of
     * (I - QQ^T)(B - theta1 I)(I - QQ^T) t = -r, Q = [locked vectors, x], by
     * MINRES in FP64; after each inner step z = x + t is scored by its
     * eigen-residual ||B z - rho(z) z|| / ||z|| (B t carried by the
     * recurrence, no extra products), the steps stop once that falls below
     * tol ||A|| / sqrt(2), or after inner2_patience steps (default 25) without
     * a 10% gain, or at inner2_maxit (default 300), and the best iterate is
     * used.  With 1 the targets stage 1 resolved are taken first and the tiny
     * ones (sigma~ <= sqrt(eps) ||A||) last, and locking a tiny pair also
     * deflates its mirror [v; -u].  Not with stage2_precond or a given
     * preconditioner. */
    int stage2_inner;
    int inner2_maxit;
    int inner2_patience;
    /* 1: Algorithm 3 (Sec. 4), dynamic switching between GD+k on C and on B
     * under preconditioning (SMALLEST, FP64): runs of at most maxIter
     * iterations alternate between C (with the shift-free form of the
     * preconditioner: diag(C)^{-1} for PHSVDS_PREC_JACOBI, M^{-1} M^{-T} for
     * PHSVDS_PREC_GIVEN, none for PHSVDS_PREC_NONE) and B (targets the
     * positive eigenvalues nearest zero, preconditioner [0 A M; M A^T 0] or
     * [0 M^{-1}; M^{-T} 0]), each from the other's approximations; the faster
     * by the mean log-reduction of the residual per iteration runs again,
     * maxIter = dyn_init_iter (default 50) x 2^j, j raised on a repeat and
     * halved on a switch, at most dyn_max_switch (default 8) times; the end
     * is B's result or the two-stage method from C's vectors
     * (stats.dynamic_route). */
    int dynamic;
    int dyn_init_iter;
    int dyn_max_switch;
    /* 1 (default): a solve repeats bit for bit on the same device and build
     * (every cross-block reduction sums in a fixed order, and the autotuner
     * leaves out the fused SpMM schedule, whose atomics sum in arrival
     * order); 0: the autotuner may take the fused schedule when it is
     * faster (the triplets then vary in the last bits between runs, and the
     * iteration counts a little). */
    int deterministic;
    /* ||A|| of the user requirement ||r|| < delta ||A|| (Sec. 3.1): the
     * switch test after stage 1, the stage-2 test delta ||A|| / sqrt(2) and
     * the tiny-sigma threshold.  0 (default): stage 1's running largest Ritz
     * value (for the smallest triplets it can sit far below ||A||, which only
     * tightens the tests); > 0: the caller's value of ||A|| (PRIMME's aNorm),
     * raised by any larger Ritz value; < 0: the larger of that and the
     * square root of the largest Ritz value of 30 Lanczos steps on C run
     * before stage 1 (FP64, seeded start; a lower bound of ||A||, so the tests
     * stay at least as tight as delta ||A||).  Stage 1's own delta_C keeps
     * its current largest Ritz value, as Algorithm 1 states.
     * stats.norm_A_est reports the value used. */
    double norm_A;
    /* 1: the FP64 method (PHSVDS_FP64, no or the Jacobi preconditioner)
     * expands stage 1 by the Jacobi-Davidson correction of the JDQMR form
     * (Sec. 4) as opts.mixed_inner describes, with the MINRES solves in FP64
     * on the FP64 products with C (the same algorithm as the mixed form's FP64
     * continuation, in one precision); 0 (default): plain GD+k. */
    int stage1_inner;
} phsvds_opts;

typedef struct {
    int64_t matvecs_A;     /* products of one vector with A */
    int64_t matvecs_At;    /* products of one vector with A^T */
    int64_t iters_stage1;  /* outer iterations (all stage-1 passes) */
    int64_t iters_stage1_fp32; /* of which in FP32 (mixed precision) */
    int64_t iters_stage2;
    int64_t restarts;
    int switched;          /* 1 if stage 2 ran */
    double norm_A_est;     /* running ||A|| estimate (largest Ritz value) */
    double t_stage1_ms, t_stage2_ms, t_total_ms;
    int spmm_schedule;     /* schedule used: 1 fused atomic, 2 two-phase */
    int64_t kernel_launches;   /* CUDA kernels this solve launched */
    /* with opts.profile: device time (CUDA events) and call counts per kernel
     * class: [0] fused A^T A SpMM (products with C), [1] Gram / CGS passes,
     * [2] basis transforms and Ritz vectors, [3] the refined vector of stage
     * 2 (inverse iteration on R; also the Jacobi SVD entry point), [4] single
     * products with A or A^T (products with B), [5] the projected
     * eigensolvers (Jacobi, FP64 and FP32 passes); [6 + c] is class c of the
     * FP32-storage launches of the mixed-precision stage 1 ([0..5] FP64),
     * where [9] holds the vector kernels of the FP32 inner solves
     * (opts.mixed_inner) */
    double t_class_ms[12];
    int64_t n_class[12];
    int64_t spmm_c_calls;      /* C-products, each one fused A^T A SpMM launch set */
    double spmm_c_ms;          /* their summed device time (opts.profile) */
    int spmm_c_width;          /* block width of the stage-1 C-products */
    int64_t jacobi_sweeps;     /* stage-1 projected eigensolver: sweeps and rotations */
    int64_t jacobi_rotations;
    int64_t jacobi_calls;      /* its launches, and the sum of their matrix orders j */
    int64_t jacobi_dim_sum;
    int fell_back;             /* 1 if the learned correction was replaced (stall) */
    int64_t fell_back_at;      /* stage-1 iteration of the fallback */
    int64_t recorded;          /* residuals written to opts.record_r */
    int64_t stage1_stagnation_locks;  /* targets locked on their rounding floor, finished by stage 2 */
    int spmm_plan_cached;      /* 1 if the autotuned SpMM schedule came from an earlier solve on this
                                  handle of a matrix with the same m, n, nnz (and block width) */
    /* algorithmic work per kernel class (the classes of t_class_ms): flops,
     * and the bytes the operations must move at least (each operand read
     * once, each result written once); filled with or without opts.profile */
    double class_flops[12];
    double class_bytes[12];
    int64_t inner_solves;      /* Jacobi-Davidson corrections of stage 1 (opts.mixed_inner, opts.stage1_inner):
                                  block inner solves, in every precision the solve used */
    int64_t inner_steps;       /* ... and their MINRES steps (each one product with C of the block, in the
                                  inner solve's precision) */
    int64_t inner2_solves;     /* JDQMR corrections of stage 2 (opts.stage2_inner = 1) */
    int64_t inner2_steps;      /* ... and their MINRES steps (each one product with B) */
    int spmm_schedule_f32;     /* schedule of the FP32 products with C (mixed precision; 0 otherwise) */
    /* opts.dynamic = 1: how Algorithm 3 ended (1 all found on C, then the
     * two-stage method; 2 C faster: the two-stage method from C's vectors;
     * 3 all found on B; 4 B faster: B to the end), its runs and switches */
    int dynamic_route;
    int dynamic_runs;
    int dynamic_switches;
} phsvds_stats;

/* Create a context on CUDA device `device`.  cuda_stream: a cudaStream_t to run
 * on, or NULL to let the library create its own (an ordinary stream, ordered
 * with the legacy default stream like one from cudaStreamCreate, so inputs
 * written there by the caller are complete before the library reads them). */
phsvds_status phsvds_create(phsvds_handle* out, int device, void* cuda_stream);

/* Fill *opts with the defaults listed above. */
phsvds_status phsvds_default_opts(phsvds_opts* opts);

/*
 * k smallest (target = PHSVDS_SMALLEST) or largest singular triplets of A
 * (Section 1, eq. 1.1): stage 1 is Algorithm 1 (GD+k on C = A^T A to the
 * tolerance delta_C of Section 3.1, then the Rayleigh-Ritz step of
 * Algorithm 1 step 3); the switch test of Section 3.1 (delta < eps ||A|| /
 * sigma_i, or a stage-1 residual above the tolerance) decides whether stage 2,
 * Algorithm 2 (the refined projection on B of Section 3.2, initial guesses
 * [v; A v / sigma] / sqrt(2) of Section 3.3), runs; a triplet is accepted
 * when sqrt(||r_u||^2 + ||r_v||^2) <= tol ||A|| (Section 5), with ||A|| the
 * largest Ritz value seen (Algorithm 1).
 *  m, n, nnz     : A is m x n (m >= n >= 1) with nnz stored entries;
 *  row_ptr       : m+1 int64 offsets; col_idx: nnz int32; val: nnz doubles (CSR);
 *  ptr_on_device : 1 if row_ptr/col_idx/val are device pointers, else host;
 *  k             : 1 <= k <= min(n, opts.min_restart - 1);
 *  tol           : delta of the criterion sqrt(||r_u||^2+||r_v||^2) <= delta ||A||;
 *  precond       : stage-1 correction operator;
 *  opts          : NULL for defaults;
 *  sigma[k], U (m x k), V (n x k), resid[k] : host outputs, sigma ascending for
 *                  SMALLEST and descending for LARGEST; resid[i] is the final
 *                  sqrt(||A v_i - s_i u_i||^2 + ||A^T u_i - s_i v_i||^2);
 *                  any of U, V, resid may be NULL;
 *  stats         : may be NULL; filled also on NOT_CONVERGED.
 * The library copies A to the device (and builds its CSC copy) on each call.
 */
phsvds_status phsvds_solve(phsvds_handle h, int64_t m, int64_t n, int64_t nnz,
                           const int64_t* row_ptr, const int32_t* col_idx, const double* val,
                           int ptr_on_device, int k, phsvds_target target, double tol,
                           phsvds_precond precond, const phsvds_opts* opts,
                           double* sigma, double* U, double* V, double* resid,
                           phsvds_stats* stats);

/* One matrix of a batch: CSR as in phsvds_solve. */
typedef struct {
    int64_t m, n, nnz;
    const int64_t* row_ptr;
    const int32_t* col_idx;
    const double* val;
} phsvds_csr;

/* One result of a batch: output buffers provided by the caller (host; sigma
 * and resid k entries, U m x k and V n x k column-major; U, V, resid may be
 * NULL), and what the solve reports. */
typedef struct {
    double* sigma;
    double* U;
    double* V;
    double* resid;
    phsvds_status status;   /* this matrix's status */
    char message[160];      /* its phsvds_last_error() text when status != OK */
    phsvds_stats stats;
} phsvds_result;

/*
 * Batched form of phsvds_solve (the method of Sections 3-5 applied to many
 * independent matrices): the `count` matrices are solved concurrently on the
 * handle's device by `concurrency` worker threads (0 = min(count, 4)), each
 * with its own stream and workspace, taking matrices largest (nnz) first.
 * Every matrix gets the same k, target, tol, precond and opts as phsvds_solve,
 * and its own autotuned SpMM plan.  ptr_on_device applies to every matrix;
 * device inputs are read only after the work already queued on the handle's
 * stream has finished.  Blocks until all solves are done.
 * Returns PHSVDS_OK when every matrix converged, else the status of the first
 * failing matrix in index order (each out[i].status and message tell which);
 * PHSVDS_ERR_INVALID for bad arguments, PHSVDS_ERR_CUDA if no worker could
 * create its context.
 */
phsvds_status phsvds_solve_batched(phsvds_handle h, int count, const phsvds_csr* mats, int ptr_on_device,
                                   int k, phsvds_target target, double tol, phsvds_precond precond,
                                   const phsvds_opts* opts, int concurrency, phsvds_result* out);

/*
 * Inner solve for the training data of the learned correction (no
 * counterpart in the paper; its corrections are Sec. 4's preconditioned
 * ones): x_i = (A^T A - shift I)^{-1} r_i for `count` right-hand sides by
 * conjugate gradients in FP64 on the device, up to 8 in lockstep, each to
 * ||r - (A^T A - shift I) x|| <= rtol ||r|| or maxit iterations.
 * shift must lie below the smallest eigenvalue of A^T A (the system SPD).
 * A as in phsvds_solve; R and X: host, n x count column-major; iters (host,
 * count, may be NULL) receives the iterations each needed.
 * Errors: INVALID (bad arguments), NOT_CONVERGED (some rhs needed more than
 * maxit; X still holds the last iterates), CUDA.
 */
phsvds_status phsvds_normal_cg(phsvds_handle h, int64_t m, int64_t n, int64_t nnz,
                               const int64_t* row_ptr, const int32_t* col_idx, const double* val,
                               int ptr_on_device, double shift, int count, const double* R, double* X,
                               double rtol, int maxit, int* iters);

/*
 * The learned correction network on a batch of grid images (no counterpart in
 * the paper).  All pointers DEVICE.  x: batch x 4 x ny x nx floats (planes:
 * residual, log diffusion, beta_x, beta_y); y: batch x ny x nx floats;
 * params: PHSVDS_CNN_NPARAM BF16; work: PHSVDS_CNN_WORK_FLOATS(batch, nx*ny)
 * floats, 8-byte aligned, which keeps the activations for a following
 * phsvds_cnn_backward.  FP32 arithmetic with the BF16 weights.
 */
phsvds_status phsvds_cnn_forward(phsvds_handle h, int batch, int nx, int ny, const void* params,
                                 const float* x, float* y, float* work);

/*
 * Backward pass after phsvds_cnn_forward(x, y, work) with the same arguments:
 * the loss L = (1/batch) sum_b ||y_b - t_b||^2 / ||t_b||^2 (t: batch x ny x nx
 * targets) is ADDED to *loss (device double) and dL/dparams (FP32, at the
 * BF16 weights) is ADDED to grad (PHSVDS_CNN_NPARAM floats).  DEVICE pointers.
 */
phsvds_status phsvds_cnn_backward(phsvds_handle h, int batch, int nx, int ny, const void* params,
                                  const float* x, const float* y, const float* t, float* work,
                                  float* grad, double* loss);

/*
 * One Adam step (Kingma & Ba) on FP32 master weights w with gradient grad and
 * moments m, v (PHSVDS_CNN_NPARAM floats each, DEVICE), step >= 1 (bias
 * correction), then params (BF16, DEVICE) = round-to-nearest(w); grad is
 * zeroed for the next accumulation.
 */
phsvds_status phsvds_cnn_adam(phsvds_handle h, float* w, float* grad, float* m, float* v, int step,
                              float lr, float beta1, float beta2, float eps, void* params);

/*
 * Kernel-level entry point: Y = A^T (A X) for a block of b vectors (Section 1,
 * C = A^T A), all pointers DEVICE pointers, FP64.  X and Y are n x b ROW-major
 * (the b values of one row contiguous).  row_ptr int32 (nnz < 2^31).
 * schedule 1 = fused single pass with atomics (Y is overwritten: the call zeroes
 * it first), 2 = two phases through Z = A X (z: caller-provided m x b device
 * scratch) using the CSC copy (csc_ptr n+1, csc_row nnz, csc_val nnz).
 * lanes_a: threads per row of A (fused, or the first phase), lanes_at: threads
 * per row of A^T (second phase); each in {1, 2, 4, 8, 16}, or 0 to pick it from
 * the mean row length nnz/m (resp. nnz/n), or the negated width to keep the
 * 32-byte row gathers out of L1.  nnz is used for nothing else.
 * b in {1, 2, 4, 8}.  A 32-byte aligned X with 32-byte rows (b = 4 FP64,
 * b = 8 FP32) is gathered with 256-bit loads.  Runs on the handle's stream;
 * asynchronous (nothing is read back).
 * Errors: PHSVDS_ERR_INVALID (nothing launched) for bad sizes, b, schedule or
 * lanes, or a NULL pointer the schedule reads (col_idx and val when nnz > 0;
 * for schedule 2 also csc_ptr, z, and csc_row and csc_val when nnz > 0);
 * PHSVDS_ERR_CUDA for a failed launch.
 */
phsvds_status phsvds_ata_spmm_f64(phsvds_handle h, int schedule, int lanes_a, int lanes_at, int64_t m, int64_t n,
                                  int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx, const double* val,
                                  const int32_t* csc_ptr, const int32_t* csc_row, const double* csc_val,
                                  int b, const double* X, double* Y, double* z);

/* Same in FP32 (values, X, Y and z float). */
phsvds_status phsvds_ata_spmm_f32(phsvds_handle h, int schedule, int lanes_a, int lanes_at, int64_t m, int64_t n,
                                  int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx, const float* val,
                                  const int32_t* csc_ptr, const int32_t* csc_row, const float* csc_val,
                                  int b, const float* X, float* Y, float* z);

/* Capacity, in doubles, of the fixed scratch of phsvds_ata_spmm_static_f64
 * (2 MiB): m * b may not exceed it. */
#define PHSVDS_STATIC_Z_MAX 262144

/*
 * Allocation-free variant of phsvds_ata_spmm_f64 with the two-phase schedule:
 * Y = A^T (A X) through Z = A X.  The paper has no counterpart to this entry
 * point; it serves callers that cannot allocate device memory while they run
 * it -- a program that has handed all device memory to its own pool, or a
 * latency-critical loop in which a cudaMalloc (which may synchronise the
 * device) is not acceptable -- and so cannot provide the m x b buffer z that
 * phsvds_ata_spmm_f64 needs.  Here Z lives in a fixed array of
 * PHSVDS_STATIC_Z_MAX doubles inside the library's device memory, and no call
 * allocates anything.
 *
 * Arguments as phsvds_ata_spmm_f64 (all DEVICE pointers, X and Y n x b
 * row-major, b in {1, 2, 4, 8}, CSR and CSC copies of A), except: no schedule
 * and no z; nnz is passed by the caller (it picks the lanes per row, and
 * taking it as an argument avoids reading row_ptr[m] back to the host).
 * Errors: PHSVDS_ERR_INVALID, with nothing launched, for bad arguments (a NULL
 * pointer, among them a NULL col_idx, val, csc_row or csc_val when nnz > 0) or
 * when m * b > PHSVDS_STATIC_Z_MAX (use phsvds_ata_spmm_f64 then);
 * PHSVDS_ERR_CUDA when the scratch cannot be located or a launch fails.
 * Runs on the handle's stream; asynchronous.
 *
 * The first call on each device makes that device current and looks up the
 * array's address (cudaGetSymbolAddress), which may also load the library's
 * device code; make this first call before any stream capture begins.  The
 * address is kept for the life of the process: after a cudaDeviceReset of
 * that device the library's device code may be loaded elsewhere, so the
 * entry point must not be called again on that device in the same process.  The
 * scratch needs no clearing, since the first phase writes every entry the
 * second reads.  There is ONE scratch per device, shared by all handles and
 * threads: calls whose executions can overlap (different streams, or handles
 * used from several threads) race on it and give wrong results.  Order them on
 * one stream.
 */
phsvds_status phsvds_ata_spmm_static_f64(phsvds_handle h, int64_t m, int64_t n, int64_t nnz,
                                         const int32_t* row_ptr, const int32_t* col_idx, const double* val,
                                         const int32_t* csc_ptr, const int32_t* csc_row, const double* csc_val,
                                         int b, const double* X, double* Y);

/*
 * Kernel-level entry point: CSR -> CSC transpose on the device (setup step of the
 * two-phase SpMM).  Inputs/outputs are DEVICE pointers: row_ptr (m+1), col_idx,
 * val (nnz); outputs csc_ptr (n+1), csc_row (nnz), csc_val (nnz).  Row indices
 * within each column come out increasing (deterministic).
 */
phsvds_status phsvds_csr_to_csc_f64(phsvds_handle h, int64_t m, int64_t n, int64_t nnz,
                                    const int32_t* row_ptr, const int32_t* col_idx, const double* val,
                                    int32_t* csc_ptr, int32_t* csc_row, double* csc_val);

/*
 * Kernel-level entry point: one-CTA FP64 cyclic Jacobi eigensolver for a
 * symmetric j x j matrix (the projected problem H = V^T C V of the Rayleigh-Ritz
 * step; Algorithm 2 step 7), each round's work compacted to its rotating
 * pairs.  DEVICE pointers.  H (j x j, column-major,
 * overwritten by the rotated matrix, whose diagonal holds the eigenvalues),
 * S (j x j, on entry the accumulated rotation -- identity for a cold start --
 * on exit S * J, so that S^T H_in S = diag(theta) for a cold start), theta (j).
 * 1 <= j <= 64.  Sweeps until every |h_pq| <= tol * max_ij |h_ij| or
 * max_sweeps; *sweeps_out (device int) receives the sweep count.
 */
phsvds_status phsvds_jacobi_eig_f64(phsvds_handle h, int j, double* H, double* S, double* theta,
                                    double tol, int max_sweeps, int* sweeps_out);

/*
 * Kernel-level entry point: the same FP64 cyclic Jacobi eigensolver spread over
 * an 8-CTA thread-block cluster (each CTA keeps a copy of H in shared memory
 * and updates one eighth of each round's 2 x 2 blocks, exchanged through
 * distributed shared memory).  Arguments and results as phsvds_jacobi_eig_f64.
 */
phsvds_status phsvds_jacobi_eig_cluster_f64(phsvds_handle h, int j, double* H, double* S, double* theta,
                                            double tol, int max_sweeps, int* sweeps_out);

/*
 * Kernel-level entry point: one-CTA FP64 one-sided (Hestenes) Jacobi SVD of a
 * j x j matrix G (refined projection, Algorithm 2 step 8: R = U Sigma S^T).
 * The solver itself needs only the smallest right singular vector of R per
 * iteration and computes it by inverse iteration; this entry point gives the
 * whole SVD.  DEVICE pointers.  G (column-major, overwritten by G * J = U Sigma), S (on
 * entry an orthogonal start -- identity for a cold start -- on exit S * J),
 * sig (j) the column norms of the result.  1 <= j <= 64.
 */
phsvds_status phsvds_jacobi_svd_f64(phsvds_handle h, int j, double* G, double* S, double* sig,
                                    double tol, int max_sweeps, int* sweeps_out);

/*
 * Kernel-level entry point: the refined vector of stage 2 (Algorithm 2 step 8,
 * Sec. 3.2), as the solver computes it.  s1 = the right singular vector of
 * the smallest singular value of the j x j upper-triangular R, by inverse
 * iteration (a forward solve with R^T and a back solve with R per step) from
 * x0, stopping once ||R s1|| falls by less than a relative tau or after maxit
 * steps; theta1 = s1^T H s1.  A pivot below 2^-52 max |r_ab| is raised to
 * that value.  DEVICE pointers: R (column-major, leading dimension ldr >= j;
 * its strictly lower triangle is ignored), x0 (j, or NULL for a fixed
 * all-positive start), H (j x j symmetric, leading dimension ldh >= j), s1
 * (j, unit norm on return), out (2 doubles: theta1, ||R s1||), steps_out (1
 * int, or NULL).  1 <= j <= 64, maxit >= 1.  Nothing is allocated.
 */
phsvds_status phsvds_refined_vector_f64(phsvds_handle h, int j, const double* R, int ldr, const double* x0,
                                        const double* H, int ldh, int maxit, double tau, double* s1,
                                        double* out, int* steps_out);

/*
 * Kernel-level entry point: one pass of block classical Gram-Schmidt, the
 * step that orthonormalises the new basis vectors of Algorithms 1 and 2
 * against the locked vectors and the basis (two passes, "CGS2"), and that
 * forms the projected matrix V^T W of the Rayleigh-Ritz step (Algorithm 2
 * step 7).  With P = [P1 | P2] (n x p1 and n x p2, column-major, leading
 * dimensions ld1, ld2 >= n; p = p1 + p2 <= 64) and the block T (n x q,
 * leading dimension ldt >= n, 1 <= q <= 8), in this order:
 *   if Gsub: T <- T - P Gsub      (Gsub p x q, column-major, leading dim p);
 *   if Gout: Gout += P^T T        (p x q, column-major, leading dim p);
 *   if Tout: Tout += T^T T        (q x q, column-major).
 * Gsub, Gout, Tout are FP64 (each may be NULL); Gout and Tout accumulate, so
 * the caller zeroes them first.  Products accumulate per thread in the
 * storage precision and across thread blocks in FP64.  All pointers DEVICE.
 * Asynchronous on the handle's stream.  Errors: PHSVDS_ERR_INVALID (nothing
 * launched) for bad sizes or NULL pointers; PHSVDS_ERR_CUDA for a failed launch.
 */
phsvds_status phsvds_block_cgs_f64(phsvds_handle h, int64_t n, const double* P1, int ld1, int p1,
                                   const double* P2, int ld2, int p2, double* T, int ldt, int q,
                                   const double* Gsub, double* Gout, double* Tout);
/* Same with FP32 storage of P and T (the mixed-precision stage 1). */
phsvds_status phsvds_block_cgs_f32(phsvds_handle h, int64_t n, const float* P1, int ld1, int p1,
                                   const float* P2, int ld2, int p2, float* T, int ldt, int q,
                                   const double* Gsub, double* Gout, double* Tout);

/*
 * Kernel-level entry point: Out = P Y - Xs diag(theta) (the Ritz vectors
 * X = V S and residuals R = W S - X Theta of the targeted pairs, and the basis
 * transforms V <- V Y of thick restart and locking, Algorithm 2 steps 7-10).
 * P n x p (ld ldp >= n, 1 <= p <= 64), Y p x r FP64 (ld ldy >= p,
 * 1 <= r <= 64), Out n x r (ld ldo >= n); theta (r, FP64) and Xs (n x r, ld
 * ldx) may be NULL together (no subtraction); Out may equal P when r <= p (in
 * place).  norms2 (r, FP64, or NULL): norms2[c] += ||Out(:, c)||^2.  All
 * pointers DEVICE; asynchronous.  Errors as phsvds_block_cgs_f64.
 */
phsvds_status phsvds_tall_small_f64(phsvds_handle h, int64_t n, const double* P, int ldp, int p, const double* Y,
                                    int ldy, int r, double* Out, int ldo, const double* Xs, int ldx,
                                    const double* theta, double* norms2);
/* Same with FP32 storage of P, Out and Xs. */
phsvds_status phsvds_tall_small_f32(phsvds_handle h, int64_t n, const float* P, int ldp, int p, const double* Y,
                                    int ldy, int r, float* Out, int ldo, const float* Xs, int ldx,
                                    const double* theta, double* norms2);

/* Synchronise the handle's stream. */
phsvds_status phsvds_sync(phsvds_handle h);

/* One-line description of the last error on this handle ("" if none). */
const char* phsvds_last_error(phsvds_handle h);

const char* phsvds_status_string(phsvds_status s);

void phsvds_destroy(phsvds_handle h);

#ifdef __cplusplus
}
#endif

#endif /* PHSVDS_H */
