/*
 * eigdc.h -- C-ABI of the GB300 inverse-free spectral divide-and-conquer
 * eigensolver (Ballard, Demmel, Dumitriu, "Minimizing Communication for
 * Eigenproblems and the Singular Value Decomposition", arXiv 1011.3077).
 *
 * Conventions for every entry point
 *   - Matrices are FP64, column-major, with a leading dimension >= rows.
 *     Pointers whose name starts with "d" are DEVICE pointers owned by the
 *     caller (for example from PyTorch); the library never frees them.  A
 *     row-major PyTorch tensor is passed as its transpose.
 *   - All work is stream-ordered on the stream given to eig_create.  Calls
 *     return after the work has completed (they synchronize that stream);
 *     the info structs are filled on return.
 *   - Return value: EIG_OK (0); a negative value is a caller or system error
 *     (arguments are checked before any launch; eig_last_error() gives the
 *     message); a positive value is a numerical outcome (no convergence, no
 *     split, ...), in which case the outputs hold the last iterate.
 *   - Workspace is owned by the handle and grown on demand (cudaMalloc);
 *     eig_workspace_size reports the requirement in advance.
 *   - Orientation: after a split, the leading k columns of the splitter span
 *     the (right) deflating subspace of the eigenvalues of det(A - z B) = 0
 *     outside the unit circle of the mapped pencil, i.e. outside the circle
 *     or right of the line of the region (Sec. 3.1 and 3.2).
 */
#ifndef EIGDC_H
#define EIGDC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct eig_handle_s* eig_handle_t;

/* status codes */
#define EIG_OK 0
#define EIG_ERR_ARG (-1)      /* invalid argument (message in eig_last_error) */
#define EIG_ERR_CUDA (-2)     /* CUDA runtime error */
#define EIG_ERR_NOMEM (-3)    /* workspace allocation failed */
#define EIG_ERR_SCRATCH (-4)  /* eig_gemm_noalloc: the split-K partials exceed its static scratch */
#define EIG_NO_CONVERGENCE 1  /* IRS hit maxit (Algorithm 3), or a leaf solver gave up */
#define EIG_NO_SPLIT 2        /* repeated failure to split a node (Sec. 3.3-3.5) */
#define EIG_NEAR_SINGULAR_PENCIL 3 /* a pencil leaf's factorised matrix is near singular (Sec. 3.5) */
#define EIG_NONFINITE 4       /* NaN/Inf met in an input or an iterate */
#define EIG_TIMEOUT 5         /* eig_server_wait: the request did not finish in time */
#define EIG_CANCELLED 6       /* a server request removed from the queue by eig_server_cancel */

/* arithmetic of the contractions */
#define EIG_FP64 0
/* split precision: the GEMMs of the iteration, the splitter and the similarity
 * run as three-term BF16 products with FP32 accumulation on the tcgen05
 * tensor cores (eig_gemm_split); panels, norms, the R-test, the split test
 * and the rank decision stay FP64.  Defaults then read tau = 1e-5 and
 * split_tol >= 1e-3, and eig_solve(EIG_KIND_SYM) ends with an FP64
 * refinement of the eigenvectors and eigenvalues. */
#define EIG_SPLIT_BF16X3 1
/* FP64-accurate contractions on the tensor cores: the large products of the
 * path (complement products of the squarings, splitter, similarity; every
 * dimension >= 128) split their FP64 operands error-free into nine signed
 * 6-bit digits per row / column (balanced, |digit| <= 32; power-of-two
 * scaled, stored exactly as BF16), multiply the digit pairs of weight levels
 * 0..9 with tcgen05.mma into one FP32 TMEM accumulator per level, exact
 * because each 1792-wide K chunk keeps every partial sum an integer below
 * 2^24, and drain the levels into FP64
 * (eig_gemm_fp64tc).  Error ~ K 2^-53 of max|row| max|column|, like an FP64
 * GEMM; the rank-32 reflector products of the panels stay on the FP64 DFMA
 * kernel, and every other setting (tau, split_tol, no refinement) is that of
 * EIG_FP64. */
#define EIG_FP64_TC 2
/* split precision with unbiased FP32-level products: the error-free split of
 * EIG_FP64_TC cut to four 6-bit digits (24 bits of each row / column maximum)
 * and weight levels 0..3 (10 digit pairs), each level accumulated exactly in
 * FP32 over 960-wide K chunks and drained into FP64 (eig_gemm_fp32tc).  BF16
 * x 3 accumulates every plane product of the whole K range in one FP32
 * accumulator whose additions truncate, a bias that grows with K; here every
 * product of the path (trailing updates and reflector products of the panels
 * included) carries an error of about 2^-24 max|row| max|column| per term
 * with no drift.  Panels, norms, the R-test, the split test and the rank
 * decision stay FP64.  Each node starts at the tier its eigenvalue interval
 * can resolve -- four digits, five digits (30 bits) or the FP64-accurate
 * split of EIG_FP64_TC, chosen from m max(|lo|, |hi|) / (hi - lo), an
 * estimate of how much the split residual amplifies the tier's rounding --
 * and escalates one tier when an attempt finds a true split (0 < rank < m)
 * whose residual stays above split_tol (>= 1e-6).  Symmetric solves end with
 * the FP64 refinement of EIG_SPLIT_BF16X3 when some accepted split ran at an
 * FP32-level tier. */
#define EIG_SPLIT_FP32 3

/* regions (Sec. 3.1 unit circle; Sec. 3.3 line via the Moebius map
 * f(z) = (z - sigma + s)/(z - sigma - s); Sec. 3.5 circles |z - c| = r) */
#define EIG_REGION_UNIT_CIRCLE 0
#define EIG_REGION_CIRCLE 1   /* c_or_sigma = centre c (real), r_or_s = radius r */
#define EIG_REGION_LINE 2     /* c_or_sigma = sigma, r_or_s = scale s > 0 */

/* problem kinds for eig_solve */
#define EIG_KIND_SYM 0        /* RSEP recursion (Algorithm 6, Sec. 3.4) */
#define EIG_KIND_NONSYM 1     /* RNEP recursion (Algorithm 5, Sec. 3.3) */
#define EIG_KIND_PENCIL 2     /* RGNEP recursion (Algorithm 4, Sec. 3.5): eig_pencil_schur */
#define EIG_KIND_CPLANE 3     /* complex-plane recursion (Sec. 3.3): eig_schur_complex */

typedef struct {
  int kind;
  double c_or_sigma;
  double r_or_s;
} eig_region_t;

typedef struct {
  double tau;        /* IRS stopping ratio ||R_j - R_{j-1}||_1 <= tau ||R_{j-1}||_1; <= 0: default.
                        The tensor-core modes also stop once the ratio is below their rounding
                        floor's level (split precision 1e-3, EIG_FP64_TC 1e-10) and fell by
                        less than 4x over the last squaring (EIGDC_VERBOSE=1 prints the
                        ratio of each squaring to stderr) */
  int maxit;         /* IRS runs j = 0..maxit (Algorithm 3, "until j > maxit") */
  double split_tol;  /* accept a split when ||E21||_1/||A||_1 (+ ||F21||_1/||B||_1) <= split_tol;
                        <= 0: max(1e-12, 16 n 2^-53) for a node of size n (the FP64 rounding
                        floor of that ratio grows like n u), pencils max(1e-10, 16 n 2^-53)
                        (two independently computed subspaces; the finished solve's backward
                        error stays 10-50x below the score); BF16 x 3: >= 1e-3;
                        EIG_SPLIT_FP32: >= 1e-6 at the RURV rank */
  int leaf_size;     /* nodes of at most this size go to the leaf solver (<= 64) */
  int prec;          /* EIG_FP64, EIG_SPLIT_BF16X3, EIG_FP64_TC or EIG_SPLIT_FP32 */
  uint64_t seed;     /* Philox key of every draw of the method */
  int max_fail;      /* unproductive attempts per node before EIG_NO_SPLIT */
  int nb;            /* panel width of the blocked QR (0: automatic) */
  int v_draws;       /* Haar redraws per converged IRS (Theorem 2.1 holds w.h.p.) */
  int root_unit_circle; /* eig_solve nonsymmetric: split the root on |z| = 1 */
  int workers;       /* eig_solve: host workers (each with its own CUDA stream) that process
                        independent nodes of the recursion concurrently; 1 = sequential */
  int graphs;        /* 1: capture the repeated launch sequence of the IRS squarings as CUDA
                        graphs (per worker stream, cached on the handle) and replay them; the
                        caller must not synchronize the whole device (cudaDeviceSynchronize)
                        from another thread while the call runs.  0 (default): plain launches */
  int fused_tail;    /* eig_solve symmetric: nodes of at most this many rows (capped at 512; 0,
                        the default, or <= leaf_size: none) are collected and finished by one
                        launch of the fused batched solver (eig_solve_batched_fused), each
                        node's sub-recursion in one CTA with its own node id, interval and
                        depth -- the same decisions as eig_solve takes, FP64 arithmetic on the
                        DFMA pipe.  It replaces the many short launches of small nodes by one
                        launch; a node in one CTA takes about 1e-7 m^3 seconds, so large values
                        lengthen a single solve */
} eig_params_t;

typedef struct {
  int iters;            /* p: squarings performed by IRS */
  double last_ratio;    /* last ||R_j - R_{j-1}||_1 / ||R_{j-1}||_1 */
  int converged;        /* 1 if the R-test fired */
  int k;                /* chosen block size (eig_split) */
  double split_residual;/* ||E21||_1/||A||_1 (+ ||F21||_1/||B||_1) at k */
  int rank;             /* RURV rank: #{|R2_ii| > 1e-8 max|R1_ii|} (1e-5 in split precision,
                           above the FP32-level noise of the iterates), R2 of RURV(A_p), R1
                           of the RQ step on A_p + B_p (A_p measured against A_p + B_p) */
  int draw;             /* Haar draw that was used (0-based) */
} eig_step_info_t;

typedef struct {
  int status;
  int nodes;
  int splits;
  int max_depth;
  int total_iters;      /* squarings summed over all IRS runs */
  int failed_attempts;
  int leaves;
  double flops;         /* algorithmic flops executed (formula counts, see bench) */
} eig_solve_info_t;

/* Host-side fault injection: the next `count` workspace allocations of any
 * handle fail as if cudaMalloc had, so the call returns EIG_ERR_NOMEM (a
 * server request then completes with that status).  0 switches it off.
 * Returns the previous pending count, or EIG_ERR_ARG for count < 0.  No GPU
 * work is involved; for tests of the failure paths. */
int eig_debug_fail_allocations(int count);

/* Defaults: tau = max(1e-14, 4 sqrt(n) 2^-53) at call time, maxit = 60,
 * split_tol = 0 (automatic), leaf_size = 64, seed = 0, max_fail = 8, nb = 0,
 * v_draws = 4, root_unit_circle = 1, workers = 8, graphs = 0, fused_tail = 0. */
void eig_default_params(eig_params_t* p);

/* Create a handle bound to CUDA device `device` and stream `stream`
 * (a cudaStream_t passed as void*; NULL = the legacy default stream). */
int eig_create(eig_handle_t* h, int device, void* stream);
int eig_destroy(eig_handle_t h);
/* Message of the last error on this handle (valid until the next call). */
const char* eig_last_error(eig_handle_t h);
/* Number of CUDA kernels this library has launched in the process so far
 * (instrumentation for benchmarks; no device work). */
unsigned long long eig_kernel_launches(void);
/* Event timing of the FP64 GEMM kernel launches (instrumentation for the
 * roofline of the dominant kernel inside a timed region; no effect on
 * results).  enable != 0: clear and start recording one event pair per
 * launch, on the launch's stream.  enable == 0: stop, wait for the recorded
 * launches and return the summed launch durations (ms), the launch count and
 * the summed algorithmic flops 2mnk (the outputs may be NULL). */
int eig_gemm_timing(int enable, double* total_ms, unsigned long long* launches, double* flops);
/* After eig_gemm_timing(0, ...): the totals of one timed kernel family of the
 * last timed region -- 0 the FP64 DFMA GEMM (work = 2mnk), 1 the FP64-accurate
 * tensor-core split (work = 53 x 2mnk BF16 MMA flops), 2 the FP32-level
 * four- and five-digit splits (10 or 15 x 2mnk), 3 the fused batched solver
 * (work 0).
 * Returns EIG_ERR_ARG for another family. */
int eig_kernel_timing(int family, double* total_ms, unsigned long long* launches, double* work);
/* Device workspace (bytes) the handle needs for calls on size n.  For
 * EIG_KIND_CPLANE: the peak of the stream-ordered allocations of a
 * complex-plane solve with one worker (each further worker adds the scratch
 * of the node it holds). */
int eig_workspace_size(eig_handle_t h, int n, int kind, size_t* bytes);

/* --------------------------------------------------------------- the path */

/* Implicit repeated squaring (Algorithm 3) on the region-mapped pencil.
 * dA (n x n) and dB (n x n, or NULL for B = I) are overwritten with A_p, B_p
 * of the MAPPED pencil.  With params->tau < 0 the R-test never fires and
 * exactly maxit+1 squarings run (used to compare iterates).  Returns
 * EIG_NO_CONVERGENCE if j > maxit without the R-test firing. */
int eig_divide_step(eig_handle_t h, int n, double* dA, int lda, double* dB, int ldb,
                    const eig_region_t* region, const eig_params_t* params,
                    eig_step_info_t* info);

/* R_j of the last squaring of the previous eig_divide_step (upper triangle,
 * diag >= 0) copied to dR (n x n). */
int eig_last_R(eig_handle_t h, int n, double* dR, int ldr);

/* Splitter and split test of one divide step (Algorithms 5 and 6, lines 2-3):
 * Q = GRURV(2, A_p + B_p, A_p, -1, +1) with the Haar draw of (seed, stream,
 * attempt), A^ = Q^T A Q (symmetrised when symmetric != 0), k minimising
 * ||E21||_1 / ||A||_1 (Sec. 4.2.1).  dAp, dBp: converged IRS output; dA: the
 * ORIGINAL matrix, overwritten with A^; dQ (n x n) receives Q.  Redraws V up
 * to params->v_draws times while the split is rejected and 0 < rank < n.
 * Returns EIG_NO_SPLIT when no accepted split exists (outputs hold the last
 * draw). */
int eig_split(eig_handle_t h, int n, const double* dAp, const double* dBp, int ldp,
              double* dA, int lda, double* dQ, int ldq, int symmetric,
              uint64_t stream, int attempt, const eig_params_t* params,
              eig_step_info_t* info);

/* Pencil splitters and split test of one RGNEP step (Algorithm 4, lines 2-5):
 * Q_R = GRURV(2, A_p + B_p, A_p, -1, +1) from the IRS iterates (dApR, dBpR)
 * of the mapped (A, B); Q_L = GRURV(2, A_pL^T, (A_pL + B_pL)^T, +1, -1) from
 * the iterates (dApL, dBpL) of the mapped (A^T, B^T) (Haar draw of purpose 6);
 * A^ = Q_L^T A Q_R, B^ = Q_L^T B Q_R; k minimises ||E21||_1 / ||A||_1 +
 * ||F21||_1 / ||B||_1.  dA, dB: the ORIGINAL pencil, overwritten with A^, B^;
 * dQL, dQR (n x n) receive Q_L, Q_R.  EIG_FP64 or EIG_FP64_TC only (EIG_ERR_ARG
 * otherwise).
 * Returns EIG_NO_SPLIT when no accepted split exists (outputs hold the last
 * draw); the rank reported is that of the right RURV. */
int eig_split_pencil(eig_handle_t h, int n, const double* dApR, const double* dBpR,
                     const double* dApL, const double* dBpL, int ldp, double* dA, int lda,
                     double* dB, int ldb, double* dQL, int ldql, double* dQR, int ldqr,
                     uint64_t stream, int attempt, const eig_params_t* params,
                     eig_step_info_t* info);

/* Generalized real Schur form of a regular pencil (A, B) by the RGNEP
 * recursion (Algorithm 4 with the strategy of Sec. 3.5): the root divides on
 * the unit circle, the group outside continues as the swapped pencil (B, A)
 * (eigenvalues 1/lambda inside the unit disk), later nodes divide on real
 * lines over [-1, 1].  Leaves (<= leaf_size) are solved in the node's
 * orientation (P, Q) = (A, B) or (B, A): M = P Q^{-1}, Hessenberg + Francis
 * on M, then the RQ factor of Q_L^T Q (plus one rotation per complex pair of
 * a swapped leaf, keeping T triangular).  B may be singular (infinite
 * eigenvalues go to the swapped side, where A is factorised).
 * On exit: dA <- S = Q_L^T A Q_R (quasi-upper-triangular, a 2x2 block per
 * complex pair), dB <- T = Q_L^T B Q_R (upper triangular), dQL,
 * dQR <- orthogonal (n x n), and the eigenvalues (alphar + i alphai) / beta
 * (device arrays of n) in block order.  EIG_FP64 or EIG_FP64_TC only (EIG_ERR_ARG
 * otherwise).
 * Status: EIG_NO_SPLIT (no divide found for a node), EIG_NEAR_SINGULAR_PENCIL
 * (the matrix a leaf factorises has max/min |r_ii| > 1e8: an eigenvalue
 * within the leaf's group sits at 0 or infinity of the wrong side, or the
 * pencil is close to singular), EIG_NO_CONVERGENCE (leaf QR iteration),
 * EIG_NONFINITE (NaN/Inf input). */
int eig_pencil_schur(eig_handle_t h, int n, double* dA, int lda, double* dB, int ldb,
                     double* dQL, int ldql, double* dQR, int ldqr, double* dalphar,
                     double* dalphai, double* dbeta, const eig_params_t* params,
                     eig_solve_info_t* info);

/* Full recursive solve (Sec. 3.3 / 3.4 strategies, leaves by cyclic Jacobi or
 * Hessenberg + Francis double-shift QR).
 *   EIG_KIND_SYM:    dA symmetric; dwr <- eigenvalues ascending (n); dU <-
 *                    orthonormal eigenvectors (n x n); dwi unused (may be NULL).
 *   EIG_KIND_NONSYM: dA <- real Schur form T (quasi-upper-triangular, 2x2
 *                    blocks standardised), dU <- Schur vectors with
 *                    A = U T U^T, dwr/dwi <- eigenvalues (block order).
 * dA is overwritten in both cases. */
int eig_solve(eig_handle_t h, int kind, int n, double* dA, int lda, double* dwr,
              double* dwi, double* dU, int ldu, const eig_params_t* params,
              eig_solve_info_t* info);

/* Singular value decomposition through the symmetric eigensolver (RSVD,
 * Sec. 3.2): the embedding H = [[0, A], [A^T, 0]] of order m + n goes through
 * the RSEP recursion (eig_solve, EIG_KIND_SYM, with params); its min(m, n)
 * largest eigenvalues are the singular values, and the two halves of their
 * eigenvectors, times sqrt(2), the left and right singular vectors.
 * dA (m x n) is not modified; dS (min(m, n)) <- singular values descending;
 * dU (m x min(m, n)), dV (n x min(m, n)) <- orthonormal singular vectors
 * (vectors of zero singular values are not determined).  The handle holds
 * 2 (m + n)^2 + (m + n) doubles for H and its eigenvectors. */
int eig_svd(eig_handle_t h, int m, int n, const double* dA, int lda, double* dS, double* dU,
            int ldu, double* dV, int ldv, const eig_params_t* params, eig_solve_info_t* info);

/* Batched solves of independent problems (the units of parallelism of
 * Sec. 4.3, here spread over the handle's host workers, each with its own
 * CUDA stream; problems run largest first, each sequentially inside one
 * worker).  Arrays are HOST arrays of length count; dA[i], dwr[i], dwi[i]
 * (NONSYM) and dU[i] are device pointers with the meaning of eig_solve.
 * status[i] receives each problem's return code and infos[i] (if infos !=
 * NULL) its info.  Returns a negative code only for argument or system
 * errors; numerical outcomes are reported per problem.  Results are
 * identical to separate eig_solve calls with workers = 1. */
int eig_solve_batched(eig_handle_t h, int kind, int count, const int* n, double* const* dA,
                      const int* lda, double* const* dwr, double* const* dwi, double* const* dU,
                      const int* ldu, const eig_params_t* params, int* status,
                      eig_solve_info_t* infos);

/* Fused batched symmetric solves: every problem's whole recursion (the
 * inverse-free iteration of Algorithm 3, the GRURV splitter of Algorithms 1-2,
 * the similarity and split test of Algorithm 6, the median-shift strategy of
 * Sec. 3.4 and Jacobi leaves) runs inside one CTA, and one persistent launch
 * covers the batch: CTAs take the problems largest first from an atomic
 * counter (the independence of Sec. 4.3).  Every product runs on the FP64
 * pipe (params->prec is not used) with the same Philox draws, node ids and
 * decisions as eig_solve, so each problem takes eig_solve's recursion tree.
 *   - Arrays are HOST arrays of length count; n[i] in [1, 512]; dA[i] (lda[i]
 *     >= n[i]) symmetric, overwritten as by eig_solve (EIG_KIND_SYM);
 *     dw[i] <- eigenvalues ascending; dU[i] (ldu[i] >= n[i]) <- eigenvectors.
 *   - status[i] and infos[i] (if infos != NULL) as for eig_solve_batched;
 *     returns a negative code only for argument or system errors.
 *   - The panel width and CTAs per SM are those chosen by the last
 *     eig_fused_autotune on the handle (default: 32-column panels, two CTAs
 *     per SM).  Workspace: about 25 max(n)^2 doubles per CTA, on the handle.
 *   - Synchronizes the handle's stream before returning. */
int eig_solve_batched_fused(eig_handle_t h, int count, const int* n, double* const* dA,
                            const int* lda, double* const* dw, double* const* dU, const int* ldu,
                            const eig_params_t* params, int* status, eig_solve_info_t* infos);

/* One candidate launch shape of the fused batched solver and its time. */
typedef struct {
  int nb;            /* panel width of the blocked QR (16 or 32) */
  int ctas_per_sm;   /* resident CTAs per SM of the persistent launch */
  double ms;         /* CUDA-event time of the launch on the tuning batch */
} eig_fused_config_t;

/* Autotuner of the fused batched solver: draws `samples` symmetric problems
 * (n log-uniform in [nmin, nmax] from `seed`, A = (G + G^T)/2 with Philox
 * Gaussians), times one fused launch over them for each panel width in
 * {16, 32} and each CTAs-per-SM count from 1 to min(3, resident limit), and
 * keeps the fastest on the handle for later eig_solve_batched_fused calls.
 * table (table_cap entries) receives the candidates and *n_table their
 * number; *best the winner.  Allocates (and frees) the sample matrices with
 * cudaMalloc. */
int eig_fused_autotune(eig_handle_t h, int samples, int nmin, int nmax, uint64_t seed,
                       eig_fused_config_t* table, int table_cap, int* n_table,
                       eig_fused_config_t* best);

/* ------------------------------------------------------------- serving
 * A request server: `workers` host threads, each with its own CUDA stream
 * and workspace, take submitted requests in arrival order as soon as a worker
 * is free and the request's device footprint (the workspace eig_solve needs
 * for its n) fits the HBM budget together with the running requests; a
 * request is always admitted when nothing runs.  Requests that arrive while
 * others run are admitted as slots and memory free up, and their work overlaps
 * on the device.  Each request's result is identical to eig_solve with
 * workers = 1 on the same input. */
typedef struct eig_server_s* eig_server_t;
int eig_server_create(eig_server_t* srv, int device, int workers, double hbm_budget_gb);
/* Queue a request (kind, n, buffers as in eig_solve).  The input dA must be
 * complete on the device (the caller synchronizes the stream that wrote it);
 * the buffers stay owned by the caller and must live until the request is
 * done.  *ticket identifies the request. */
int eig_server_submit(eig_server_t srv, int kind, int n, double* dA, int lda, double* dwr,
                      double* dwi, double* dU, int ldu, const eig_params_t* params,
                      uint64_t* ticket);
/* Pencil request (eig_pencil_schur semantics and outputs; EIG_FP64 or
 * EIG_FP64_TC params only, EIG_ERR_ARG otherwise); admission and buffers as for eig_server_submit. */
int eig_server_submit_pencil(eig_server_t srv, int n, double* dA, int lda, double* dB, int ldb,
                             double* dQL, int ldql, double* dQR, int ldqr, double* dalphar,
                             double* dalphai, double* dbeta, const eig_params_t* params,
                             uint64_t* ticket);
/* Complex-plane request (eig_schur_complex semantics and outputs, interleaved
 * complex buffers, no enclosure output; runs on one worker stream).  Admission
 * and buffers as for eig_server_submit. */
int eig_server_submit_complex(eig_server_t srv, int n, const double* dA, int lda, double* dT,
                              int ldt, double* dU, int ldu, double* dw, const eig_params_t* params,
                              int enclose, uint64_t* ticket);
/* *done = 1 once finished; then *status, times[0..2] = queue wait, service,
 * latency (seconds, host steady clock) and *info are filled (each may be NULL). */
int eig_server_poll(eig_server_t srv, uint64_t ticket, int* done, int* status, double* times,
                    eig_solve_info_t* info);
/* Block until the request is done (EIG_TIMEOUT after timeout_s seconds). */
int eig_server_wait(eig_server_t srv, uint64_t ticket, double timeout_s, int* status);
/* Cancel a request that is still queued: it is removed, reported done with
 * status EIG_CANCELLED, and its buffers are not touched.  Returns 1 if it was
 * cancelled, 0 if it had already been admitted (a running solve is not
 * interrupted) or had finished, EIG_ERR_ARG for an unknown ticket. */
int eig_server_cancel(eig_server_t srv, uint64_t ticket);
int eig_server_stats(eig_server_t srv, unsigned long long* completed, unsigned long long* pending,
                     double* reserved_gb, double* peak_reserved_gb);
/* Stop the workers (a running request finishes first, queued ones are
 * dropped) and free everything. */
int eig_server_destroy(eig_server_t srv);

/* ------------------------------------------------------ building blocks
 * The steps of the path, exposed so each can be checked on its own. */

/* Householder QR of dX (m x n, m >= n), R with non-negative diagonal:
 * dQ (m x n, orthonormal columns) and dR (n x n upper; strictly lower part
 * zeroed).  dX is not modified.  (Sec. 3 intro; Sec. 4.2.1 explicit Q.) */
int eig_qr(eig_handle_t h, int m, int n, const double* dX, int ldx, double* dQ,
           int ldq, double* dR, int ldr);

/* rows x cols N(0,1) matrix from Philox4x32-10 + Box-Muller, counter layout
 * (pair index, attempt, purpose, stream), key = seed (Algorithm 1, line 1). */
int eig_gaussian(eig_handle_t h, int rows, int cols, uint64_t seed, int purpose,
                 uint64_t stream, int attempt, double* dG, int ldg);

/* Haar orthogonal V = Q factor (diag R >= 0) of the Gaussian draw
 * (Sec. 2, Algorithm 1, lines 1-2). */
int eig_haar(eig_handle_t h, int n, uint64_t seed, int purpose, uint64_t stream,
             int attempt, double* dV, int ldv);

/* Split test (Sec. 4.2.1): e(k) = max_{j<k} sum_{i>=k} |A_ij| / normA
 * (+ the same for dB / normB when dB != NULL) for k = 1..n-1; *k gets the
 * minimiser (ties: closest to n/2, then smaller k), *e its value.  If
 * hscores != NULL it receives the n-1 values (host memory). */
int eig_split_test(eig_handle_t h, int n, const double* dA, int lda, double normA,
                   const double* dB, int ldb, double normB, int* k, double* e,
                   double* hscores);

/* C = alpha op(A) op(B) + beta C with op = transpose when ta / tb != 0
 * (the FP64 contraction every step uses). */
int eig_gemm(eig_handle_t h, int ta, int tb, int m, int n, int k, double alpha,
             const double* dA, int lda, const double* dB, int ldb, double beta,
             double* dC, int ldc);

/* C = alpha op(A) op(B) + beta C with the FP64-accurate tensor-core split of
 * EIG_FP64_TC (device pointers, column-major; op = transpose when t != 0).
 * Returns EIG_ERR_CUDA if a bounded wait of the kernel timed out. */
int eig_gemm_fp64tc(eig_handle_t h, int ta, int tb, int m, int n, int k, double alpha,
                    const double* dA, int lda, const double* dB, int ldb, double beta, double* dC,
                    int ldc);
/* C = alpha op(A) op(B) + beta C in the split-precision form of the
 * contractions: FP64 operands split into three BF16 planes (hi + mid + lo),
 * the six plane products of weight >= 2^-16 accumulated in FP32 on the
 * tcgen05 tensor cores, FP64 result (FP32-level accuracy, about 2^-22 |A||B|
 * per entry).  The split-precision reading of the trailing-update and
 * complement GEMMs of the inverse-free iteration. */
int eig_gemm_split(eig_handle_t h, int ta, int tb, int m, int n, int k, double alpha,
                   const double* dA, int lda, const double* dB, int ldb, double beta,
                   double* dC, int ldc);

/* C = alpha op(A) op(B) + beta C with the four-digit error-free split of
 * EIG_SPLIT_FP32 on the tcgen05 tensor cores: FP32-level accuracy (error
 * about K 2^-24 max|row of op(A)| max|column of op(B)| in the worst case),
 * exact chunked accumulation, no K-dependent bias. */
int eig_gemm_fp32tc(eig_handle_t h, int ta, int tb, int m, int n, int k, double alpha,
                    const double* dA, int lda, const double* dB, int ldb, double beta,
                    double* dC, int ldc);

/* ------------------------------------------------------ no-allocation GEMM
 * The paper has no counterpart: this entry point serves callers that cannot
 * call cudaMalloc -- for example a process whose device memory is reserved by
 * another allocator's pool, or a latency-critical loop that cannot take the
 * device synchronisation an allocation brings.  It computes what eig_gemm
 * computes, with the same split-K decomposition, but needs no handle and
 * allocates nothing: its K-chunk partials live in a static device array of
 * 2^20 doubles (8 MiB) that every GPU loading the library holds until the
 * process exits.
 *   - stream: a cudaStream_t passed as void* (NULL = legacy default stream);
 *     the call only enqueues work on it and returns.
 *   - All matrix pointers are caller-owned device memory, column-major.
 *   - Returns EIG_ERR_SCRATCH when the split-K partials of this shape
 *     (splits * m * n doubles) exceed 2^20 doubles; shapes that need no
 *     split (large m * n, or small k) never use the array.
 *   - The array's device address is looked up on the first call on each
 *     device (with that device current); make that first call before any
 *     stream capture.  The address is kept for the life of the process: a
 *     device reset (cudaDeviceReset, or the primary context destroyed and
 *     made again) invalidates it, and the entry point must not be called on
 *     that device afterwards.
 *   - All calls share the array; calls that overlap on the GPU race on it.
 */
int eig_gemm_noalloc(void* stream, int ta, int tb, int m, int n, int k, double alpha,
                     const double* dA, int lda, const double* dB, int ldb, double beta,
                     double* dC, int ldc);

/* ------------------------------------------------------ eigenvectors
 * Eigenvectors from the Schur form (the eigenvector section and its blocked
 * form): for A = Q T Q^T as eig_solve (EIG_KIND_NONSYM) returns it -- T
 * quasi-upper-triangular in standard form, wi the imaginary parts -- each
 * 2 x 2 block is made triangular by the unitary whose first column is the
 * block's eigenvector, then Tc X = X diag(Tc) is solved for the upper
 * triangular X (X_jj = 1) by the recurrence
 *   X_ij = (T_ij X_jj + sum_{k=i+1}^{j-1} T_ik X_kj) / (T_jj - T_ii),
 * in blocks of 32 whose off-diagonal right-hand sides are complex GEMMs.
 *   - dT (ldt >= n), dQ (ldq >= n), dwi (n): device, real, not modified.
 *   - dV (ldv >= n): device, complex (interleaved), receives unit 2-norm
 *     eigenvectors, A V = V diag(lam); dlam: device, n complex eigenvalues.
 *   - The recurrence divides by eigenvalue differences; one of modulus below
 *     2^-53 max |T_ii| is replaced by that value, so equal eigenvalues give
 *     large but finite vectors. */
int eig_eigenvectors(eig_handle_t h, int n, const double* dT, int ldt, const double* dQ, int ldq,
                     const double* dwi, double* dV, int ldv, double* dlam);
/* The same from a complex Schur form A = U T U^H (interleaved complex, T upper
 * triangular, as eig_schur_complex returns it): dV receives unit eigenvectors
 * U X, dlam the diagonal of T. */
int eig_eigenvectors_complex(eig_handle_t h, int n, const double* dT, int ldt, const double* dU,
                             int ldu, double* dV, int ldv, double* dlam);

/* ------------------------------------------------------ complex-plane strategy
 * Sec. 3.3: splitting lines at random angles.  The line {z : Re(conj(w) z) = t}
 * (|w| = 1) is mapped to the unit circle by the rotated Moebius map
 * (A - w (t - s) I, A - w (t + s) I); IRS, GRURV, the similarity and the split
 * test then run in complex arithmetic, so eigenvalues that no real line
 * separates (a spectrum along the imaginary axis, conjugate pairs) split too.
 * Complex arrays are interleaved (re, im) FP64 pairs, column-major, with
 * leading dimensions counted in complex elements.
 */
#define EIG_MAX_HALFPLANES 8

/* A convex region {|z - c| <= R} cut by half-planes Re(conj(w_i) z) >= t_i that
 * holds the eigenvalues of a cluster no line could split (the convex
 * enclosures of pseudospectra remarked on in Sec. 3.3).  At most the
 * EIG_MAX_HALFPLANES most recent half-planes are kept; fewer half-planes give
 * a larger region that still holds the cluster. */
typedef struct {
  int offset, size;   /* the cluster's diagonal block T(offset:offset+size, ...) */
  double c_re, c_im, R;
  int nhp;
  double w_re[EIG_MAX_HALFPLANES], w_im[EIG_MAX_HALFPLANES], t[EIG_MAX_HALFPLANES];
} eig_enclosure_t;

/* Complex Schur form A = U T U^H (T upper triangular, w = diag(T)) of an
 * n x n complex matrix by the recursion of Sec. 3.3: a disk holding the
 * spectrum (Gershgorin about tr(A)/n), lines at a random angle and offset
 * within half the radius (Philox purpose 8 of the node and attempt), chops of
 * empty half-planes, the 2-step radius shrink (the next line perpendicular to
 * the chord; the region moves to its enclosing circle, radius at most
 * sin(5 pi/12) R), after a split the smaller of each block's disk
 * |z - c| <= ||A_ii - c I||_F (c its mean eigenvalue) and the enclosing circle
 * of its side, and complex
 * Hessenberg + single-shift QR leaves (leaf_size <= 64).
 *   - dA (lda >= n), dT (ldt >= n), dU (ldu >= n): device, complex; dw: device,
 *     n complex.  dA is not modified.
 *   - params: tau, maxit, split_tol (0: max(1e-12, 16 n 2^-53)), leaf_size,
 *     seed, max_fail, v_draws, workers and prec are used.  Independent nodes
 *     run on `workers` host threads with their own streams; the result does
 *     not depend on the schedule.  EIG_FP64: every contraction
 *     on the FP64 pipe; EIG_FP64_TC: products with every dimension >= 128 (and
 *     m n k >= 2^25) run as four FP64-accurate tensor-core products of the
 *     real and imaginary planes (as eig_gemm_fp64tc); EIG_SPLIT_BF16X3 runs
 *     as EIG_FP64.
 *   - enclose = 1: a node that fails max_fail times is returned as a cluster:
 *     its block is put in Schur form by the leaf solver and its region is
 *     written to enc[i] (up to enc_cap entries; *n_enc = number of clusters).
 *     enclose = 0: such a node stops the solve with EIG_NO_SPLIT.  Clusters
 *     of 65..512 rows use a global-memory form of the leaf solver (one CTA);
 *     a cluster above 512 rows is still written to enc, and the solve
 *     returns EIG_NO_SPLIT.
 *   - Returns EIG_NO_CONVERGENCE if a leaf's QR iteration ran out of steps. */
int eig_schur_complex(eig_handle_t h, int n, const double* dA, int lda, double* dT, int ldt,
                      double* dU, int ldu, double* dw, const eig_params_t* params, int enclose,
                      eig_enclosure_t* enc, int enc_cap, int* n_enc, eig_solve_info_t* info);

/* The single steps of the complex path (interleaved complex, column-major,
 * device pointers; calls synchronize the handle's stream):
 *   eig_zgemm: C = alpha op(A) op(B) + beta C, op = X (0) or X^H (1), DFMA.
 *   eig_zqr: X = Q R for m >= n: Q (m x n, orthonormal columns), R (n x n,
 *     upper triangular with a real non-negative diagonal: the unique QR of a
 *     full-rank X); dR may be NULL.
 *   eig_zhaar: the Haar unitary of (seed, stream, attempt): the Q factor of
 *     G = X + i Y, X and Y the Philox N(0,1) draws of purposes 4 and 7.
 *   eig_zline_step: one step on the line Re(conj(w) z) = t with scale s
 *     (|w| = 1, s > 0): the rotated Moebius map, IRS, the splitter
 *     Q = GRURV(2, A_p + B_p, A_p, -1, +1) with the Haar draws of (seed,
 *     stream, attempt), A^ = Q^H A Q and the split test; dQ and dAhat (either
 *     may be NULL) receive Q and A^, info the iteration count, k, e(k), rank
 *     and draw.  Returns EIG_OK for an accepted split, EIG_NO_SPLIT when IRS
 *     converged without one, EIG_NO_CONVERGENCE when it hit maxit.  Only the
 *     leading k columns of Q are unique (the rest are a basis of the
 *     complementary invariant subspace that rounding picks). */
int eig_zgemm(eig_handle_t h, int ta, int tb, int m, int n, int k, double alpha_re,
              double alpha_im, const double* dA, int lda, const double* dB, int ldb,
              double beta_re, double beta_im, double* dC, int ldc);
int eig_zqr(eig_handle_t h, int m, int n, const double* dX, int ldx, double* dQ, int ldq,
            double* dR, int ldr);
int eig_zhaar(eig_handle_t h, int n, uint64_t seed, uint64_t stream, int attempt, double* dV,
              int ldv);
int eig_zline_step(eig_handle_t h, int n, const double* dA, int lda, double w_re, double w_im,
                   double t, double s, uint64_t stream, int attempt, const eig_params_t* params,
                   double* dQ, int ldq, double* dAhat, int ldah, eig_step_info_t* info);

/* Host-only helpers of the Sec. 3.3 strategy (no GPU or handle needed).
 * eig_cplane_enclosing_circle: a circle (m, r) holding the region
 * {|z - c| <= R} cut by the nhp half-planes Re(conj(w_i) z) >= t_i: the
 * smallest circle through the region's corners when it also holds the
 * region's boundary arcs, else the disk itself.
 * eig_cplane_draw_line: the line (w, t) of attempt `attempt` at node `node`:
 * w = e^{2 pi i u2} (or i * pw when perpendicular != 0), t = R (u1 - 1/2) +
 * Re(conj(w) c), (u1, u2) the Philox pair of purpose 8.  Both return EIG_OK or
 * EIG_ERR_ARG (NULL output, negative count or radius). */
int eig_cplane_enclosing_circle(double c_re, double c_im, double R, int nhp, const double* w_re,
                                const double* w_im, const double* t, double* m_re, double* m_im,
                                double* r);
int eig_cplane_draw_line(uint64_t seed, uint64_t node, int attempt, double c_re, double c_im,
                         double R, int perpendicular, double pw_re, double pw_im, double* w_re,
                         double* w_im, double* t);

#ifdef __cplusplus
}
#endif
#endif /* EIGDC_H */
