// Internal declarations shared by the translation units of libeigdc.
// Host-side launchers for the sm_103a kernels; every launcher enqueues on the
// given stream and returns a cudaError_t from the launch.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/eigdc.h"

namespace eigdc {

// Running count of kernel launches made by this library (all launchers add
// to it); read through eig_kernel_launches().
void note_launches(unsigned long long k);

// NVTX range for the lifetime of a scope (a no-op unless a profiler is attached):
// "eig.solve", "eig.node", "eig.irs", "eig.qr", "eig.split", "eig.leaves", ...
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// ------------------------------------------------------------- api.cu host helpers
// (u1, u2) of Philox pair 0 of (purpose, stream, attempt): u1 in (0, 1), u2 in [0, 1).
void philox_pair_host(uint64_t seed, int purpose, uint64_t stream, int attempt, double* u1,
                      double* u2);
// Philox stream id of child `side` (0 or 1) of a recursion node.
uint64_t child_node_id(uint64_t parent, int side);
// Block size of the smallest score e[k-1], k = 1..n-1 (ties: closest to n/2, then smaller k).
int choose_k_host(const double* e, int n);

// ------------------------------------------------------------- linalg.cu
// C = alpha op(A) op(B) + beta C, column-major FP64.  When splits > 1 the K
// range is cut into `splits` chunks written to `partial` (splits*m*n doubles)
// and reduced in a fixed order (deterministic).
cudaError_t gemm(cudaStream_t s, bool ta, bool tb, int m, int n, int k, double alpha,
                 const double* A, int lda, const double* B, int ldb, double beta,
                 double* C, int ldc, int splits = 1, double* partial = nullptr);
int gemm_choose_splits(int m, int n, int k);
// op(A) B (ta selects op) written as `splits` K-chunk partials in the layout
// partial[z][i + j*m] (ld = m, even for one split); returns the number of
// chunks actually used, or -1 on a launch error.
int gemm_partials(cudaStream_t s, bool ta, int m, int n, int k, const double* A, int lda,
                  const double* B, int ldb, int splits, double* partial);

// Householder panel factorisation of the m x jb panel P (ldp) on a thread-block
// cluster.  In place: R on and above the diagonal, Householder vectors below.
// Writes the explicit unit-lower-trapezoidal V (ldv), tau[jb] and the jb x jb
// upper-triangular T (ldt) of the compact WY form H_0..H_{jb-1} = I - V T V^T.
cudaError_t panel_qr(cudaStream_t s, int m, int jb, double* P, int ldp, double* V,
                     int ldv, double* tau, double* T, int ldt);
int panel_max_width(int m);
void panel_init();   // once per device: picks the largest usable cluster size

// Out = op(T) * (sum_z partial[z]) for a jb x n block (op = T^T if trans).
// With splits == 1 `partial` is read directly; with in_trans the (single)
// input is stored as its n x jb transpose.
cudaError_t reduce_trmm(cudaStream_t s, int jb, int n, const double* partial, int splits,
                        const double* T, int ldt, bool trans, double* out, bool in_trans = false);

// ------------------------------------------------------------- tc_gemm.cu
// Split-BF16 (three-term) GEMM on tcgen05 tensor cores, FP64 in and out,
// FP32-level accuracy.  `ws` must hold tc_gemm_workspace_bytes(m, n, k)
// (the BF16 planes of both operands); *err gets a nonzero bit if a bounded
// wait in the kernel timed out.
size_t tc_gemm_workspace_bytes(int m, int n, int k);
// FP64-accurate GEMM on the tensor cores (error-free split into nine balanced
// digits, exact FP32 accumulation per 1792-wide K chunk, FP64 drain); `ws` must hold
// tcx_gemm_workspace_bytes(m, n, k) bytes; err as for tc_gemm.
size_t tcx_gemm_workspace_bytes(int m, int n, int k);
cudaError_t tcx_gemm(cudaStream_t s, bool ta, bool tb, int m, int n, int k, double alpha,
                     const double* A, int lda, const double* B, int ldb, double beta, double* C,
                     int ldc, void* ws, int* err);
// FP32-level GEMM on the tensor cores: the same error-free split with four
// 6-bit digits (24 bits of each row / column maximum) and levels 0..3 (10
// digit pairs), exact FP32 accumulation per 960-wide K chunk, FP64 drain: no
// accumulation bias, error about 2^-24 max|row| max|column| per product term.
size_t tcx32_gemm_workspace_bytes(int m, int n, int k);
// The same with five digits (30 bits, levels 0..4, 15 digit pairs).
size_t tcx30_gemm_workspace_bytes(int m, int n, int k);
cudaError_t tcx30_gemm(cudaStream_t s, bool ta, bool tb, int m, int n, int k, double alpha,
                       const double* A, int lda, const double* B, int ldb, double beta, double* C,
                       int ldc, void* ws, int* err);
cudaError_t tcx32_gemm(cudaStream_t s, bool ta, bool tb, int m, int n, int k, double alpha,
                       const double* A, int lda, const double* B, int ldb, double beta, double* C,
                       int ldc, void* ws, int* err);
cudaError_t tc_gemm(cudaStream_t s, bool ta, bool tb, int m, int n, int k, double alpha,
                    const double* A, int lda, const double* B, int ldb, double beta, double* C,
                    int ldc, void* ws, int* err);

// ------------------------------------------------------------- misc.cu
cudaError_t fill_identity_block(cudaStream_t s, int rows, int cols, double* Y, int ldy,
                                int diag_row_offset);
cudaError_t region_stack(cudaStream_t s, int n, const double* A, int lda, const double* B,
                         int ldb, int kind, double c_or_sigma, double r_or_s, double* Aj,
                         double* Bj, double* W);
cudaError_t stack_pencil(cudaStream_t s, int n, const double* Aj, const double* Bj, double* W);
// R (upper part of W's top n x n) -> Rcur; accumulates max column sums of
// |Rcur - Rprev| and |Rprev| into sums[0], sums[1] (as ordered bit patterns).
cudaError_t r_extract_diff(cudaStream_t s, int n, const double* W, int ldw, double* Rcur,
                           const double* Rprev, unsigned long long* sums);
cudaError_t copy_matrix(cudaStream_t s, int rows, int cols, const double* A, int lda, double* B,
                        int ldb);
cudaError_t add_matrices(cudaStream_t s, int rows, int cols, const double* A, int lda,
                         const double* B, int ldb, double* C, int ldc);
// Z[i][k] = Y[n-1-k][i]   (Z = (J Y)^T)
cudaError_t reverse_transpose(cudaStream_t s, int n, const double* Y, int ldy, double* Z, int ldz);
// Opt-in event timing of kernel launches (instrumentation): families of
// timed kernels; `work` per launch is its algorithmic flops (FP64 2mnk for the
// GEMMs, BF16 tensor flops 2mnk x digit pairs for the tensor-core splits).
enum { TIMING_DGEMM = 0, TIMING_TCX64 = 1, TIMING_TCX32 = 2, TIMING_FUSED = 3, TIMING_FAMILIES = 4 };
struct TimingToken {
  cudaEvent_t a, b;
  double work;
  int family;
};
TimingToken timing_begin(cudaStream_t s, int family, double work);
void timing_end(cudaStream_t s, const TimingToken& t);
void gemm_timing_start();
// stops timing; totals of every family are kept, the DFMA GEMM's returned
cudaError_t gemm_timing_stop(double* total_ms, unsigned long long* launches, double* flops);
void timing_family(int family, double* total_ms, unsigned long long* launches, double* work);
// B (cols x rows, ldb) = A^T
cudaError_t transpose(cudaStream_t s, int rows, int cols, const double* A, int lda, double* B,
                      int ldb);
// B[:, j] = A[:, n-1-j]
cudaError_t reverse_columns(cudaStream_t s, int rows, int n, const double* A, int lda, double* B,
                            int ldb);
cudaError_t symmetrize(cudaStream_t s, int n, double* A, int lda);
cudaError_t upper_triangle(cudaStream_t s, int n, const double* W, int ldw, double* R, int ldr);
cudaError_t gaussian(cudaStream_t s, int rows, int cols, uint64_t seed, int purpose,
                     uint64_t stream, int attempt, double* G, int ldg);
// column sums of |A| max -> bits in out (atomic max), for ||A||_1
cudaError_t norm1_bits(cudaStream_t s, int rows, int cols, const double* A, int lda,
                       unsigned long long* out);
// One power-iteration normalisation (one CTA): v = y - c x (x null: v = y),
// *est = ||v||_2, xout = v / ||v||_2 (xout may alias x).
cudaError_t power_norm(cudaStream_t s, int n, double c, const double* x, const double* y,
                       double* xout, double* est);
// nonfinite flag (1 if any NaN/Inf) ORed into *flag
cudaError_t nonfinite_check(cudaStream_t s, int rows, int cols, const double* A, int lda,
                            int* flag);
// split test scores e(k) (k = 1..n-1) -> scores[k-1] (accumulates += f(k)/norm)
cudaError_t split_scores(cudaStream_t s, int n, const double* A, int lda, double inv_norm,
                         double* colpart, double* scores, bool accumulate);
cudaError_t diag_gershgorin(cudaStream_t s, int n, const double* A, int lda, double* diag,
                            double* lo_hi);
cudaError_t count_rank(cudaStream_t s, int n, const double* R, int ldr, const double* Sc, int lds,
                       double rel_tol, int* rank);
cudaError_t zero_lower_quasi(cudaStream_t s, int n, double* T, int ldt, const double* wi);
// Split the 2 x 2 blocks of (S, T) marked as complex pairs in wi whose
// generalized eigenvalues are real (rotations applied to S, T, QL, QR; wi
// updated).  scratch: 5n doubles; act: n ints; flag: device int; hflag:
// pinned host int, set to 1 if any block was split.
cudaError_t pencil_split_real_pairs(cudaStream_t s, int n, double* S, int lds, double* T, int ldt,
                                    double* QL, int ldql, double* QR, int ldqr, double* wi,
                                    double* scratch, int* act, int* flag, int* hflag);
// SVD through the symmetric embedding: H = [[0, A], [A^T, 0]]; singular
// triplets from the r = min(m, n) largest eigenpairs of H.
cudaError_t svd_embed(cudaStream_t s, int m, int n, const double* A, int lda, double* H, int ldh);
cudaError_t svd_extract(cudaStream_t s, int m, int n, const double* W, int ldw, const double* w,
                        double* S, double* U, int ldu, double* V, int ldv);
// (alpha_re, alpha_im, beta) of (S, T) in generalized real Schur form; 2 x 2
// blocks of S are marked by wi[i] > 0, wi[i+1] = -wi[i]
cudaError_t pencil_alpha_beta(cudaStream_t s, int n, const double* S, int lds, const double* T,
                              int ldt, const double* wi, double* ar, double* ai, double* be);
// FP64 refinement of a symmetric eigendecomposition (n x n packed operands)
cudaError_t oa_diag(cudaStream_t s, int n, const double* G, const double* S, double* lam,
                    unsigned long long* maxabs);
cudaError_t oa_offmax(cudaStream_t s, int n, const double* G, const double* S,
                      unsigned long long* bits);
cudaError_t oa_correction(cudaStream_t s, int n, const double* G, const double* S,
                          const double* lam, double delta, double* E);
cudaError_t add_inplace(cudaStream_t s, size_t count, double* X, const double* D);

// ------------------------------------------------------------- leaves.cu
// Batched leaves: leaf i is the m_i x m_i block at A + off_i*(lda+1) of the
// global matrix; eigenvectors / Schur vectors go to Z + zoff_i (ldz = 64).
struct LeafDesc {
  int off;      // row/col offset of the leaf in the global matrix
  int m;        // size (<= 64)
  int zoff;     // offset of its 64x64 Z slot in the Z buffer (doubles)
  int swapped = 0;   // pencil leaves: the recursion handled this block as (B, A)
};
cudaError_t jacobi_leaves(cudaStream_t s, int count, const LeafDesc* d_desc, const double* A,
                          int lda, double* w, double* Z, int* status);
cudaError_t francis_leaves(cudaStream_t s, int count, const LeafDesc* d_desc, const double* A,
                           int lda, double* wr, double* wi, double* Z, int* status);
// Pencil leaves, in the leaf's orientation (P, Q) = (A, B), or (B, A) when
// swapped: phase 1 writes M = P Q^{-1} into the leaves' diagonal blocks of
// Mout (status bit 2: Q too ill-conditioned); phase 2 computes the right
// factor QR from Q and the Schur vectors QL of M (slot of ZL), and for a
// swapped leaf rotates the column pair of each complex block (wi) so that
// QL^T B QR stays upper triangular.
cudaError_t pencil_leaves_phase1(cudaStream_t s, int count, const LeafDesc* d_desc, const double* A,
                                 const double* B, int ld, double* Mout, int* status);
cudaError_t pencil_leaves_phase2(cudaStream_t s, int count, const LeafDesc* d_desc, const double* A,
                                 const double* B, int ld, const double* wi, const double* ZL,
                                 double* ZR);
// U[:, off:off+m] = U[:, off:off+m] * Z_i for each leaf (batched, U is n x n)
cudaError_t apply_leaf_vectors(cudaStream_t s, int count, const LeafDesc* d_desc, int n,
                               const double* Uin, int ldu_in, double* Uout, int ldu_out,
                               const double* Z);

// ------------------------------------------------------------- fused.cu
// One problem of the fused batched symmetric solver (device array entry).
struct FusedProblem {
  int n, lda, ldu, pad;
  double* A;   // in: symmetric A; out: the block-diagonal working matrix (as eig_solve)
  double* w;   // out: eigenvalues ascending
  double* U;   // out: eigenvectors
  // has_interval != 0: the problem is a node of a larger recursion -- its
  // Philox node id, eigenvalue interval [lo, hi] and depth continue that
  // recursion; else it is a root (id 1, interval from Gershgorin and the
  // power-iteration estimate, depth 0)
  uint64_t id;
  double lo, hi;
  int depth, has_interval;
};
struct FusedResult {
  int status, nodes, splits, max_depth, total_iters, failed_attempts, leaves, pad;
  double flops;
};
// Device bytes of the per-CTA workspaces for problems up to mx and `ctas` CTAs.
size_t fused_workspace_bytes(int mx, int ctas);
size_t fused_smem_bytes();
int fused_max_n();
// One persistent launch over `count` problems (CTAs take them in `order`
// from an atomic counter); nb = 16 or 32 (panel width).
cudaError_t fused_batched(cudaStream_t s, int count, const FusedProblem* probs, const int* order,
                          FusedResult* results, int* counter, const eig_params_t& p, int nb,
                          int ctas, int mx, void* ws);
// Resident CTAs per SM of the fused kernel (occupancy calculator).
int fused_max_ctas_per_sm();

// ------------------------------------------------------------- cplane.cu
// Complex-plane recursion (Sec. 3.3).  Complex arrays are interleaved (re, im)
// FP64 pairs, column-major, leading dimensions in complex elements.
struct CplaneHalfPlane {
  double wr, wi, t;   // {z : Re(conj(w) z) >= t}
};
struct CplaneCluster {
  int off, m;                          // diagonal block of T
  double cr, ci, R;                    // disk
  std::vector<CplaneHalfPlane> hp;     // half-planes cutting it
};
// Building blocks of the complex path (interleaved complex, column-major):
// QR with explicit Q (m x n) and R (n x n, real non-negative diagonal); the
// Haar unitary of Philox purposes 4 (real) and 7 (imaginary); one step on the
// line Re(conj(w) z) = t with scale sc (EIG_OK: accepted split, EIG_NO_SPLIT:
// converged without one, EIG_NO_CONVERGENCE: IRS hit maxit).
int cplane_qr(cudaStream_t s, int m, int n, const double* dX, int ldx, double* dQ, int ldq,
              double* dR, int ldr, std::string* err);
int cplane_haar(cudaStream_t s, int n, uint64_t seed, uint64_t node, int attempt, double* dV,
                int ldv, std::string* err);
int cplane_step(cudaStream_t s, int n, const double* dA, int lda, double w_re, double w_im,
                double t, double sc, const eig_params_t& p, uint64_t node, int attempt,
                double* dQ, int ldq, double* dAhat, int ldah, eig_step_info_t* info,
                std::string* err);
cudaError_t cplane_zgemm(cudaStream_t s, bool ta, bool tb, int m, int n, int k, double ar,
                         double ai, const double* A, int lda, const double* B, int ldb, double br,
                         double bi, double* C, int ldc);
// Device bytes a complex-plane solve of order n holds at its peak with one
// worker (per-node scratch of the root, node matrices, final products).
size_t cplane_footprint(int n, int prec);
// C = alpha op(A) op(B) + beta C over C (op = X or X^H), DFMA, 64 x 64 tiles.
cudaError_t zgemm(cudaStream_t s, bool ta, bool tb, int m, int n, int k, double2 alpha,
                  const double2* A, int lda, const double2* B, int ldb, double2 beta, double2* C,
                  int ldc);
// A = U T U^H with T upper triangular, w = diag(T).  Returns an EIG_* status;
// on a negative status *err holds the message.
int cplane_schur(cudaStream_t s, int n, const double* dA, int lda, double* dT, int ldt,
                 double* dU, int ldu, double* dw, const eig_params_t& p, bool enclose,
                 std::vector<CplaneCluster>* clusters, eig_solve_info_t* info, std::string* err);

// ------------------------------------------------------------- trevc.cu
// Eigenvectors of A = Q T Q^T from the real Schur form (T quasi-triangular in
// standard form, wi the imaginary parts): V (n x n complex, unit columns) and
// lam (n complex).  Returns an EIG_* status.
// With complex_in, dT and dQ are a complex Schur form (interleaved complex,
// T upper triangular) and dwi is not read.
int trevc(cudaStream_t s, int n, const double* dT, int ldt, const double* dQ, int ldq,
          const double* dwi, double* dV, int ldv, double* dlam, std::string* err,
          bool complex_in = false);

}  // namespace eigdc
