/*
 * gadi.h -- C ABI of the GB300 (sm_103a) implementation of three-precision
 * General ADI (GADI) for sparse A x = b, following arXiv 2512.21164.
 *
 * The method (Algorithm 1 of the paper, Sec. 2.3): with the splitting
 * A = M + N (Sec. 3.1, "eq:split"), a regularisation alpha > 0 and an
 * extrapolation omega in [0, 2) (Sec. 1, Lemma 1), repeat
 *     r = b - A x                               in u_r  (FP64 or double-FP64)
 *     solve (alpha I + M) z = r                 in u_s  (FP64, FP32 or BF16)
 *     solve (alpha I + N) y = (2 - omega) alpha z   in u_s
 *     x = x + y                                 in u    (FP64)
 * until ||b - A x|| / ||b - A x_0|| <= tol.  The splitting is HSS:
 * M = (A + A^T)/2, N = (A - A^T)/2, used for every problem class of Sec. 5.
 * The shifted SPD system is solved by CG; the shifted skew system by CG on
 * the normal equations (Sec. 5.1), or exactly and pointwise when alpha I + N
 * is diagonal (the complex class of Sec. 5.4).
 *
 * Precisions (Sec. 3.1 requires u_r <= u <= u_s; Sec. 5.1 variants):
 *   u = FP64 (u_high must be GADI_FP64); u_r = FP64 by default, or double-FP64
 *   (GADI_FP64X2 in gadi_opts.u_r: unit roundoff about u^2, see below);
 *   u_s = u_low: FP64 (GADI-FP64), FP32 (GADI-FP32) or BF16 storage with FP32
 *   arithmetic (GADI-BF16).  Inner vectors are stored in u_s; dot products and
 *   matrix-vector products are carried in FP32 (FP64 when u_s = FP64).
 *
 * Conventions for every entry point below:
 *   - Status: negative values are errors; on an error no output is written.
 *     Positive values (NOT_CONVERGED, STAGNATED, DIVERGED) are non-fatal: x
 *     holds the last iterate and the stats are filled.
 *   - Pointers to vectors may be host or device memory of the current CUDA
 *     device unless stated otherwise; the library detects which.  Host
 *     vectors are staged through device buffers owned by the handle (the
 *     copies are part of the call).
 *   - Vectors have length n doubles for real problems and 2n doubles for the
 *     complex class (interleaved re, im pairs), n = nx*ny(*nz) or the CSR size.
 *   - Grids are row-major with x fastest: index (z*ny + y)*nx + x.
 *   - Device vectors should start on a 16-byte boundary (any cudaMalloc or
 *     PyTorch allocation does); real-valued vectors that do not are handled
 *     by a slower path, complex ones are rejected with GADI_ERR_INVALID.
 *   - Calls on one handle are not thread-safe.  All work is issued on the
 *     stream given in gadi_opts (NULL = the legacy default stream) and the
 *     calls return after that work has finished.
 *   - The library never calls back into Python or PyTorch; device memory for
 *     its own workspace comes from cudaMalloc in gadi_create / first solve.
 */
#ifndef GADI_H
#define GADI_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GADI_OK = 0,              /* converged: relres <= tol                      */
    GADI_NOT_CONVERGED = 1,   /* maxit outer iterations reached                */
    GADI_STAGNATED = 2,       /* relres fell < 1% over the stagnation window   */
    GADI_DIVERGED = 3,        /* relres > 1e6 or not finite                    */
    GADI_ERR_INVALID = -1,    /* bad argument                                  */
    GADI_ERR_NONFINITE = -2,  /* NaN/Inf in an input vector or parameter       */
    GADI_ERR_CUDA = -3,       /* a CUDA runtime call failed                    */
    GADI_ERR_OOM = -4,        /* device allocation failed                      */
    GADI_ERR_TIMEOUT = -5,    /* a device-side grid barrier gave up waiting    */
    GADI_ERR_UNSUPPORTED = -6 /* valid request this build does not implement   */
} gadi_status;

/* GADI_FP64X2 ("double-FP64", u ~ 2^-104 ~ u^2) is a residual precision only
 * (gadi_opts.u_r): r = b - A x is formed with every product exact (a product
 * and its fused-multiply-add error term) and the sum compensated (Knuth's
 * TwoSum, as in the Dot2 algorithm of Ogita, Rump & Oishi, "Accurate sum and
 * dot product", SIAM J. Sci. Comput. 26(6), 2005), giving r as an unevaluated
 * pair hi + lo; r_s is hi + lo rounded to u_s (ties broken by lo in the
 * normal binary32 range; elsewhere hi is rounded), ||r|| is taken from hi. */
typedef enum { GADI_FP64 = 0, GADI_FP32 = 1, GADI_BF16 = 2, GADI_FP64X2 = 3 } gadi_prec;

/* Splittings of Sec. 2.1.  Only HSS is used by the paper's experiments
 * (Sec. 5.2-5.4); the others are reserved. */
typedef enum { GADI_SPLIT_HSS = 0 } gadi_splitting;

/* Problem classes of Sec. 5, plus a general CSR matrix (Sec. 5.1: the
 * paper's own implementation stores A, H and S as sparse matrices). */
typedef enum {
    GADI_STENCIL_2D5 = 0, /* -Lap u + beta.grad u (+ kappa u), 5-point, 5.2   */
    GADI_STENCIL_3D7 = 1, /* 3D convection-diffusion (+ kappa u), 7-point, 5.3 */
    GADI_COMPLEX_2D5 = 2, /* (L + kappa I) + i sigma I, Sec. 5.4              */
    GADI_CSR = 3          /* general A with positive definite (A + A^T)/2     */
} gadi_kind;

/* Operators for gadi_apply. */
typedef enum { GADI_OP_A = 0, GADI_OP_M = 1, GADI_OP_N = 2, GADI_OP_AT = 3 } gadi_op;

/* Problem descriptor (Sec. 5.2-5.4).  Stencil matrices are the centred finite
 * differences scaled by h^2 (entries O(1)):
 *   2D: A = M + N, M: centre 4 + kappa, neighbours -1; N: E +c_x, W -c_x,
 *       N +c_y, S -c_y with c_i = beta_i h / 2 (kappa >= 0: an h^2-scaled
 *       reaction term, as in the problem of Sec. 5.2; 0 for pure
 *       convection-diffusion);
 *   3D: centre 6 + kappa and a third axis;
 *   complex: M = L + kappa I (L the 5-point Laplacian), N = i sigma I.
 *   kappa < 0 is rejected (GADI_ERR_INVALID).
 * h <= 0 means h = 1/(nx+1).  CSR arrays (host memory, 0-based, int32 indices,
 * FP64 values, n rows) are copied by gadi_create; the caller keeps them. */
typedef struct {
    int kind;
    int nx, ny, nz;
    double h;
    double beta[3];
    double kappa, sigma;
    int n;
    const int *rowptr;
    const int *col;
    const double *val;
    /* complex class only (NULL otherwise, or for T = sigma I): a per-point
     * imaginary diagonal T = diag(T_i), HOST array of nx*ny finite doubles
     * in grid order (the random potential V(x) of Sec. 5.4), copied by
     * gadi_create; sigma is then ignored.  S = alpha I + i T stays diagonal
     * (pointwise solve); its T_i are rounded to u_s like stored
     * coefficients. */
    const double *sigma_pt;
} gadi_problem;

/* Solver options.  Defaults (gadi_opts_default): tol_h = tol_s = 1e-3 (1e-2
 * for BF16), maxit_inner = 1000, inner_stag = 10, outer_stag_window = 50,
 * s_pointwise = 1, stream = NULL, max_blocks = 0 (one persistent block set
 * per SM), hist = NULL, batch_group = 0, alpha_restarts = 0, h_resident = 2
 * (1 for BF16, where tensor memory measured slower), u_r = GADI_FP64,
 * s_resident = 1, backward_err = 0, batch_interleave = 0.  The
 * step entry gadi_step_solve_h takes the same h_resident default. */
typedef struct {
    double tol_h;          /* inner CG relative residual tolerance on H     */
    double tol_s;          /* inner CGNR tolerance on S (normal residual)   */
    int maxit_inner;       /* cap on each inner solve (reaching it is fine) */
    int inner_stag;        /* stop an inner solve after this many steps
                              without a new residual minimum (0 = off)      */
    int outer_stag_window; /* STAGNATED if relres fell < 1% over this many
                              outer iterations (0 = off)                    */
    int s_pointwise;       /* complex class: solve the diagonal S exactly   */
    void *stream;          /* cudaStream_t                                  */
    int max_blocks;        /* cap on persistent blocks (0 = automatic)      */
    double *hist;          /* optional HOST array of maxit+1 doubles: relres
                              per outer iteration                           */
    int batch_group;       /* gadi_solve_batched: k > 0 = groups of k blocks
                              for every system size; 0 = sizes chosen per
                              size class by the library's tuner (timed on
                              the device, kept for the process)            */
    int alpha_restarts;    /* Sec. 4.3: on STAGNATED or DIVERGED,
                              double alpha and continue from the last finite
                              iterate, up to this many times (0 = off)      */
    int h_resident;        /* 2D real class, FP32/BF16, 16-byte aligned rows:
                              1 = CG on H keeps its search direction p in
                              shared memory when a block's rows (+2 halo
                              rows) fit without lowering occupancy; 2 = as
                              1, and z and r of the block's rows also stay
                              on chip, in tensor memory (TMEM), when each
                              thread's share fits 16 slots of 16 bytes
                              (e.g. 2048 x 2048, FP32 or BF16, on 152
                              SMs), else as 1; 0 = always
                              stream p through global memory.  Same
                              arithmetic in all three; 1 and 2 give the
                              same bits, 0 differs in the order of the
                              grid-wide sums.  gadi_solve_batched: >= 1 =
                              units keep p in shared memory on their
                              group's blocks (as 1) where every system
                              admits it (an FP64 residual, 16-byte rows,
                              a candidate group size whose row share
                              fits); 0 = streaming.  Other values:
                              INVALID.                                    */
    gadi_prec u_r;         /* residual precision u_r (Sec. 3.1, u_r <= u):
                              GADI_FP64 or GADI_FP64X2; every problem
                              class, single and batched solves             */
    int s_resident;        /* with h_resident = 2 taken: 1 = CGNR on S also
                              keeps its direction p in shared memory (two
                              halo rows each side) and t, y in tensor
                              memory when every block owns two rows or
                              more (S p is recomputed, never stored); 0 =
                              stream it.  Same arithmetic; the grid-wide
                              sums' order differs.  Other values: INVALID. */
    int backward_err;      /* gadi_solve: 0 = off; k > 0 = after the solve,
                              compute the normwise backward error of eq.
                              (3.2), ||b - A x|| / (||A||_2 ||x|| + ||b||),
                              into gadi_stats.backward_err, with ||A||_2
                              from k steps of gadi_norm2_estimate (kept by
                              the handle for the next solve with the same
                              k); outside the timed solve.  < 0: INVALID.  */
    int batch_interleave;  /* gadi_solve_batched with nrhs = 4, FP32 inner
                              solves and an FP64 residual: 1 = the four
                              right-hand sides of a system form one unit,
                              their vectors interleaved as [n][4] (one
                              sweep, barrier and grid sum serve all four;
                              each keeps its own scalars and stopping);
                              0 = one unit per right-hand side (the
                              default: faster on uneven batches whose
                              large systems dominate).  Other values:
                              INVALID.                                   */
} gadi_opts;

typedef struct {
    int outer_its;          /* outer iterations done (x_k with k = outer_its) */
    long long inner_its_h;  /* total CG iterations on H                      */
    long long inner_its_s;  /* total CGNR iterations on S                    */
    double relres;          /* ||b - A x|| / ||b - A x_0|| at exit (FP64)    */
    double r0_norm;         /* ||b - A x_0||                                 */
    double seconds;         /* device time of the solve (CUDA events)        */
    int status;             /* same as the return value                      */
    int blocks;             /* persistent blocks launched                    */
    double alpha;           /* alpha of the last run (after any restarts)    */
    int restarts;           /* alpha restarts taken (Sec. 4.3)               */
    int h_resident;         /* the H-solve taken: 0 streaming, 1 p in shared
                               memory, 2 p in shared and z, r in tensor
                               memory                                        */
    int s_resident;         /* 1 if CGNR on S also ran resident (h_resident
                               = 2 and every block owns >= 2 rows): p in
                               shared memory, t and y in tensor memory       */
    double backward_err;    /* normwise backward error of eq. (3.2) of the
                               returned x (gadi_opts.backward_err > 0), with
                               ||b - A x|| the solve's own final FP64
                               residual norm; -1 if not computed             */
} gadi_stats;

typedef struct gadi_handle gadi_handle;

/* Fill *o with the defaults listed above for precision u_low. */
void gadi_opts_default(gadi_opts *o, gadi_prec u_low);

/* Human-readable name of a status code (static string). */
const char *gadi_status_str(gadi_status s);

/* Description of the last CUDA failure seen by this thread in the library
 * (the failing call, source line and CUDA's message); "" if none.  The
 * string belongs to the library and is overwritten by the next failure. */
const char *gadi_last_error(void);

/* Build the operator set for a problem and a splitting (Sec. 3.1) on the
 * current CUDA device.  Stencils are matrix-free: only scalars are kept.
 * CSR: A, M = (A + A^T)/2 and N = (A - A^T)/2 are formed in FP64 on the host
 * and copied to the device.  Errors: INVALID (sizes <= 0, kind or splitting
 * unknown, CSR pattern out of range), OOM, CUDA.  *out is NULL on error. */
gadi_status gadi_create(const gadi_problem *prob, gadi_splitting split, gadi_handle **out);

/* Release the handle and its device memory.  NULL is a no-op. */
void gadi_destroy(gadi_handle *h);

/* Algorithm 1 (Sec. 2.3) with precisions u = u_r = u_high = FP64 and
 * u_s = u_low.  b: right-hand side (read only); x: initial guess in,
 * final iterate out (the paper uses x_0 = 0).  Stops when
 * ||b - A x_k|| / ||b - A x_0|| <= tol (Sec. 5.1) or after maxit outer
 * iterations.  alpha > 0 and 0 <= omega < 2 (Lemma 1).  opts NULL = defaults;
 * stats may be NULL.  The whole iteration runs in one persistent cooperative
 * kernel; stopping decisions are made on the device.
 * Errors: INVALID (alpha <= 0, omega outside [0,2), u_high != FP64, tol < 0,
 * maxit < 0), NONFINITE (NaN/Inf in b, x, alpha, omega), TIMEOUT, CUDA, OOM. */
gadi_status gadi_solve(gadi_handle *h, const double *b, double *x, double alpha, double omega,
                       gadi_prec u_high, gadi_prec u_low, double tol, int maxit,
                       const gadi_opts *opts, gadi_stats *stats);

/* Many independent systems and right-hand sides in one persistent launch
 * (Algorithm 1 for each).  hs[s] (s < nsys): handles of the 2D 5-point class
 * (other classes: GADI_ERR_UNSUPPORTED); b[s], x[s]: DEVICE arrays of nrhs
 * consecutive vectors of system s ([nrhs][n_s] doubles), x in/out as in
 * gadi_solve; alpha[s]: that system's regularisation; omega, precisions, tol,
 * maxit and opts are shared.  Systems of the same grid form a size class.
 * The grid of persistent blocks is cut into groups, each with a size for its
 * class: opts->batch_group blocks, or (batch_group = 0, the default) the size
 * a tuner picks -- it times outer iterations of each class's units on groups
 * of 1, 2, 4, ... 64 blocks, the whole grid busy with copies of them (once
 * per grid, precision, options and alpha values in the process), starts
 * each class at the size with the fewest block-seconds per outer iteration,
 * gives each class groups in proportion to its work (units x block-seconds
 * per outer iteration x the grid's side), then moves one class at a time to
 * the size that most lowers the estimated finish time of the batch.  Each
 * group takes units from its class's device-side queue, then from the
 * queues of classes of smaller systems (never a larger one, nor one whose
 * rows do not split over the group for the resident H-solve).  A unit is one
 * (system, rhs), or with opts->batch_interleave one system's four right-hand
 * sides; with opts->h_resident >= 1 (FP32 / BF16, see there) the units' CG on
 * H keeps p in shared memory.  per_unit (nullable) gets
 * nsys*nrhs entries in the order s*nrhs + j, with `seconds` the unit's own
 * device time and `blocks` the size of the group that ran it.  Returns
 * GADI_OK if every unit converged, else the first non-OK unit status;
 * errors as gadi_solve. */
gadi_status gadi_solve_batched(gadi_handle *const *hs, int nsys, int nrhs, const double *const *b,
                               double *const *x, const double *alpha, double omega, gadi_prec u_high,
                               gadi_prec u_low, double tol, int maxit, const gadi_opts *opts,
                               gadi_stats *per_unit);

/* Sec. 4.3, the check of eq. 4.1: condition numbers of H = alpha I + M and S = alpha I + N
 * from closed forms, for the stencil classes (host only, no GPU work).
 * M's spectrum is the sum of 1D Dirichlet Laplacian spectra plus kappa, so
 * kappa(H) = (alpha + lmax) / (alpha + lmin) exactly.
 * N is normal with eigenvalues i (sum_i 2 c_i cos(j pi h_i)) (i sigma for the
 * complex class), so kappa(S) <= sqrt(alpha^2 + ||N||^2) / alpha, the value
 * returned (an upper bound; equal when N is singular).  CSR: UNSUPPORTED (no
 * cheap estimate; the check is then skipped, as Sec. 4.3 allows). */
gadi_status gadi_condition_numbers(const gadi_problem *prob, double alpha, double *kappa_h, double *kappa_s);

/* Sec. 4.3, steps 2-3: the smallest alpha_out = alpha0 * 2^k (k >= 0, k <= 60)
 * with kappa(H) kappa(S) u_s < tau (eq. 4.1; tau = 0.01 in the paper), using
 * gadi_condition_numbers and u_s from Table 1 (BF16 3.91e-3, FP32 5.96e-8,
 * FP64 1.11e-16).  Errors: INVALID, UNSUPPORTED (CSR). */
gadi_status gadi_select_alpha(const gadi_problem *prob, double alpha0, gadi_prec u_low, double tau,
                              double *alpha_out);

/* Check of the bounded grid barrier (no counterpart in the paper): launches a
 * small cooperative kernel on `nblocks` blocks in which block 0 never arrives
 * at the barrier, so every other block's wait runs out after timeout_ms; the
 * blocks unwind and the call returns GADI_ERR_TIMEOUT with the device still
 * usable.  It makes no memory access out of bounds and has no other effect.
 * Errors: INVALID (nblocks < 2 or above the co-resident maximum, timeout_ms
 * not in (0, 10000]), CUDA. */
gadi_status gadi_selftest_barrier(int nblocks, double timeout_ms);

/* Timing probe of the grid-wide sum (no counterpart in the paper): runs
 * `iters` grid-wide sums of two FP32 partials per thread on `nblocks`
 * persistent blocks of the solve kernels' size (0 = one per SM), each taken
 * exactly as the inner solves take theirs (block tree, one partial per block,
 * the bounded grid barrier, every block reading all partials), and returns
 * the mean time of one sum in microseconds (device %globaltimer).  CG on H
 * and CGNR on S each take two such sums per iteration, so this is their
 * latency floor.  Synchronous on the legacy default stream.  Errors: INVALID
 * (iters not in [1, 1e6], nblocks above the co-resident maximum), TIMEOUT,
 * CUDA. */
gadi_status gadi_probe_sync(int nblocks, int iters, double *us_per_sum);

/* Timing probe of the FP64 pipe (no counterpart in the paper): one block of
 * the solve kernels' size per SM runs `iters` rounds of 8 independent FP64
 * fused multiply-adds per thread; *gops receives the rate in 10^9 FMA per
 * second (CUDA events), *sm_ops_per_clk (nullable) the same per SM and
 * clock at the device's nominal SM clock.  The rate bounds every FP64 step
 * of the method (the residual, GADI-FP64's inner solves).  Synchronous on
 * the legacy default stream.  Errors: INVALID (iters not in [1, 1e7]), CUDA. */
gadi_status gadi_probe_fp64(int iters, double *gops, double *sm_ops_per_clk);

/* Check of the library's integer-pipe number conversions (no counterpart in
 * the paper): for each of the n doubles at `in` (DEVICE pointer, n >= 0),
 * compares on the device (1) binary64 -> binary32 round-to-nearest-even,
 * (2) binary64 -> BF16 round-to-nearest-even, both against the hardware
 * conversion, and (3) binary32 -> binary64 of the float whose bits are the
 * low 32 bits of the input, against the hardware widening, and (4) that
 * float -> BF16 by the conversion instruction, one value and two values
 * (with the float of the upper 32 bits) per instruction, equals the integer
 * rounding sequence (non-NaN floats) -- all bit for bit.  mismatches (HOST array of
 * 4) receives the count per check.  Synchronous
 * on the legacy default stream.  Errors: INVALID (n < 0, null pointers), CUDA. */
gadi_status gadi_selftest_convert(const double *in, long long n, long long *mismatches);

/* The layout rule of gadi_solve_batched on given timings, host only (no
 * GPU): ncl size classes, largest systems first, class c with count[c] units
 * on a grid of side side[c]; t_outer[c * 7 + i] the seconds per outer
 * iteration of one of its units on a group of 2^i blocks (i = 0..6; <= 0 =
 * not timed / not admitted); fixed > 0 = every class on groups of min(fixed,
 * total) blocks; total = blocks of the grid.  Out: size[c] blocks per group
 * and groups[c] groups of class c (every class >= 1 group, groups[c] <=
 * count[c], sum of size x groups <= total), *estimate the estimated finish
 * time (max over classes of ceil(count / groups) x t(size) x side).
 * Errors: INVALID (bad arguments, a class without a timed size, or more
 * classes than fit in the grid). */
gadi_status gadi_batch_plan(int ncl, const long long *side, const int *count, const double *t_outer, int fixed,
                            int total, int *size, int *groups, double *estimate);

/* y = Op x in FP64 for Op in {A, M, N, A^T} (Sec. 3.1 splitting).  x and y
 * may be host or device memory; stream as in gadi_opts (NULL = default). */
gadi_status gadi_apply(gadi_handle *h, gadi_op op, const double *x, double *y, void *stream);

/* The stencil of Op in {A, M, N, A^T} for a stencil problem, as gadi_create
 * builds it (the operator definition of Sec. 5.2-5.4, h^2-scaled): coef[0]
 * the centre, coef[1..6] the W, E, S, N, B, T neighbours (zero where the
 * class has none), coef[7] the imaginary diagonal of the complex class.  Host
 * only.  Errors: INVALID (CSR, bad sizes or op). */
gadi_status gadi_stencil_coefs(const gadi_problem *prob, gadi_op op, double *coef);

/* ||A||_2 estimate by `iters` steps of power iteration on A^T A in FP64 on
 * the device (a lower bound; used for the backward error of eq. (3.2)). */
gadi_status gadi_norm2_estimate(gadi_handle *h, int iters, double *out, void *stream);

/* ---- single steps of Algorithm 1, for verification of each kernel --------
 * All vectors here are DEVICE pointers.  Vectors in u_s ("u_s vectors") have
 * element type double (FP64), float (FP32) or uint16 BF16 bit patterns
 * (BF16), with the same length as x. */

/* Residual step (Algorithm 1 "r = b - A x" in u_r, fused with the previous
 * update "x = x + y" in u): x_out = x + y (y == NULL: x_out = x),
 * r = b - A x_out in FP64, *rnorm = ||r||_2, rs = fl_{u_s}(r).
 * r_out (nullable) receives r in FP64.  x_out must not alias x. */
gadi_status gadi_step_residual(gadi_handle *h, gadi_prec u_low, const double *b, const double *x,
                               const void *y, double *x_out, double *r_out, void *rs,
                               double *rnorm, void *stream);

/* The same step with the residual precision u_r chosen (GADI_FP64 or
 * GADI_FP64X2, Sec. 3.1): r_out (nullable) receives the FP64 part hi of r,
 * r_lo_out (nullable) the low part lo (zeros for u_r = FP64).  Errors:
 * INVALID (bad u_r or u_low, null b / x / x_out / rs, x aliasing x_out). */
gadi_status gadi_step_residual_ur(gadi_handle *h, gadi_prec u_r, gadi_prec u_low, const double *b,
                                  const double *x, const void *y, double *x_out, double *r_out,
                                  double *r_lo_out, void *rs, double *rnorm, void *stream);

/* H-solve (Algorithm 1, the solve with alpha I + M): CG on (alpha I + M) z = rs in u_s from z = 0,
 * until ||res|| <= tol ||rs|| (tol = 0: exactly maxit steps), or `stag` steps
 * without a new minimum (0 = off).  *its receives the iteration count. */
gadi_status gadi_step_solve_h(gadi_handle *h, double alpha, gadi_prec u_low, const void *rs,
                              void *z, double tol, int maxit, int stag, int *its, void *stream);

/* S-solve (Algorithm 1, the solve with alpha I + N): g = fl_{u_s}((2 - omega) alpha z), then CG on
 * S^T S y = S^T g from y = 0 (t_0 = fl_{u_s}(S^T g)), same stopping rules;
 * pointwise != 0 with the complex class: y = fl_{u_s}(g / (alpha + i sigma)). */
gadi_status gadi_step_solve_s(gadi_handle *h, double alpha, double omega, gadi_prec u_low,
                              const void *z, void *y, double tol, int maxit, int stag,
                              int pointwise, int *its, void *stream);

/* ---- allocation-free variant -------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot call cudaMalloc (code running inside a pre-sized memory pool,
 * a host application that owns every device allocation, or a process that
 * must not grow its device footprint once started).
 *
 * gadi_solve_h_2d_noalloc: the H-solve of the 2D 5-point class -- CG on
 * (alpha I + M) z = rs with M the h^2-scaled 5-point Laplacian (centre 4,
 * neighbours -1) on an nx x ny grid, from z = 0, with the stopping rules of
 * gadi_step_solve_h -- with no handle and no device allocation.  It runs the
 * streaming form of that H-solve (search direction p in global memory, one
 * persistent block per SM), which gadi_step_solve_h also takes on grids with
 * fewer rows than the GPU has SMs; there the two give the same bits.  On
 * taller grids gadi_step_solve_h keeps p on chip and sums in another order,
 * so the results then agree to rounding only.  rs (read) and z (written) are
 * DEVICE u_s vectors of nx*ny elements (double, float or BF16 bits); *its
 * receives the iteration count.
 *   - Scratch: a file-scope device array of about 10.6 MB that every GPU
 *     loading the library holds until exit; the call makes no cudaMalloc,
 *     cudaFree or other allocating call.
 *   - Limit: nx*ny <= 262144 (for example 512 x 512); larger grids are
 *     rejected with GADI_ERR_INVALID and a message in gadi_last_error().
 *   - The first call on each device (and again after the device's context
 *     was rebuilt, e.g. by cudaDeviceReset) looks up the scratch's device
 *     address (cudaGetSymbolAddress) with that device current; make that
 *     first call before any stream capture.
 *   - Synchronous: the call returns after its GPU work has finished.
 *   - Every call shares the one scratch array and leaves its contents
 *     behind (the call clears what must start at zero).  Calls that overlap
 *     on the GPU -- on different streams or host threads -- race on it and
 *     must be serialised by the caller.
 * Errors: INVALID, TIMEOUT, CUDA. */
gadi_status gadi_solve_h_2d_noalloc(int nx, int ny, double alpha, gadi_prec u_low, const void *rs, void *z,
                                    double tol, int maxit, int stag, int *its, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* GADI_H */
