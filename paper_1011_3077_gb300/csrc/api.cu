// C-ABI of libeigdc and the host-side drivers of the divide-and-conquer path
// (Ballard, Demmel, Dumitriu, arXiv 1011.3077):
//   blocked Householder QR (Sec. 3 intro) -> IRS (Algorithm 3) -> GRURV
//   splitters (Algorithm 2 with k = 2; the left one of pencils, Algorithm 4)
//   -> similarity and split test (Algorithms 4-6, Sec. 4.2.1) -> recursion
//   (Sec. 3.3-3.5: lines, the pencil circle search and swap) -> leaves;
//   the SVD through the symmetric embedding (Sec. 3.2).
// Around it: the node-parallel executor (host workers with their own CUDA
// streams), batched solves, CUDA graphs of the squarings, the request
// server, and the precision modes (FP64, the FP64-accurate tensor-core split,
// BF16 x 3 with FP64 refinement).
// Every arithmetic step runs in the sm_103a kernels of linalg.cu, misc.cu,
// leaves.cu, tc_gemm.cu and tcx_gemm.cu; the host only orders launches, reads
// the convergence ratio once per squaring, the chosen k / rank once per
// split, and takes the strategy decisions (shift, interval, circle, swap).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <condition_variable>
#include <chrono>
#include <cstring>
#include <deque>
#include <functional>
#include <mutex>
#include <thread>
#include <string>
#include <vector>

#include "../../include/eigdc.h"
#include "internal.h"

using namespace eigdc;

static std::atomic<unsigned long long> g_launches{0};

void eigdc::note_launches(unsigned long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

namespace {

constexpr int JB_LD_C = 32;   // largest panel width (leading dimension of T)
constexpr int PURPOSE_HAAR = 4;
constexpr int PURPOSE_SHIFT = 5;
constexpr int PURPOSE_HAAR_LEFT = 6;
constexpr uint64_t ROOT_NODE = 1;

}  // namespace

struct eig_handle_s {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  double* lastR = nullptr;
  int lastR_n = 0;
  void* pinned = nullptr;
  size_t pinned_bytes = 0;
  std::vector<eig_handle_s*> workers;   // sub-handles of the node / batch executor
  char* aux = nullptr;                  // caller-level buffers (SVD embedding), grown on demand
  size_t aux_bytes = 0;
  // CUDA graphs of the IRS squaring, keyed by the workspace it runs in
  struct IrsGraph {
    const void* base;
    int n, prec, parity;
    cudaGraphExec_t exec;
    unsigned long long kernels;
  };
  std::vector<IrsGraph> graphs;
  bool graphs_off = false;
  // fused batched solver: panel width and CTAs per SM (0: automatic), set by
  // eig_fused_autotune
  int fused_nb = 32;
  int fused_cps = 0;
};

static void clear_graphs(eig_handle_s* h) {
  for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
  h->graphs.clear();
}

namespace {

// ---------------------------------------------------------------- helpers
struct Fail {
  int code;
};

#define CK(call)                                                              \
  do {                                                                        \
    cudaError_t e__ = (call);                                                 \
    if (e__ != cudaSuccess) {                                                 \
      h->err = std::string("CUDA error: ") + cudaGetErrorString(e__) + " at " \
               + __FILE__ + ":" + std::to_string(__LINE__);                   \
      throw Fail{EIG_ERR_CUDA};                                               \
    }                                                                         \
  } while (0)

#define CK2(hh, call)                                                          \
  do {                                                                         \
    cudaError_t e__ = (call);                                                  \
    if (e__ != cudaSuccess) {                                                  \
      (hh)->err = std::string("CUDA error: ") + cudaGetErrorString(e__) + " at " \
                  + __FILE__ + ":" + std::to_string(__LINE__);                 \
      throw Fail{EIG_ERR_CUDA};                                                \
    }                                                                          \
  } while (0)

static size_t round_up(size_t b) { return (b + 255) & ~(size_t)255; }

// Bump allocator over the handle workspace.  With base == nullptr it only
// measures, so the same carving code gives the size and the pointers.
struct Arena {
  char* base;
  size_t used = 0;
  explicit Arena(char* b) : base(b) {}
  template <class T>
  T* take(size_t count) {
    T* p = base ? reinterpret_cast<T*>(base + used) : nullptr;
    used += round_up(count * sizeof(T));
    return p;
  }
};

// Host-side fault injection: the next g_fail_allocs workspace allocations fail
// as if cudaMalloc had (eig_debug_fail_allocations).
static std::atomic<int> g_fail_allocs{0};

static bool injected_alloc_failure() {
  int v = g_fail_allocs.load();
  while (v > 0)
    if (g_fail_allocs.compare_exchange_weak(v, v - 1)) return true;
  return false;
}

static void ensure_ws(eig_handle_t h, size_t bytes) {
  if (bytes <= h->ws_bytes) return;
  CK(cudaStreamSynchronize(h->stream));
  clear_graphs(h);   // the graphs hold pointers into the old workspace
  if (h->ws) cudaFree(h->ws);
  h->ws = nullptr;
  h->ws_bytes = 0;
  if (injected_alloc_failure() || cudaMalloc(&h->ws, bytes) != cudaSuccess) {
    cudaGetLastError();
    h->ws = nullptr;
    h->err = "workspace allocation of " + std::to_string(bytes) + " bytes failed";
    throw Fail{EIG_ERR_NOMEM};
  }
  h->ws_bytes = bytes;
}

static void* pinned(eig_handle_t h, size_t bytes) {
  if (bytes > h->pinned_bytes) {
    if (h->pinned) cudaFreeHost(h->pinned);
    h->pinned = nullptr;
    h->pinned_bytes = 0;
    if (cudaMallocHost(&h->pinned, bytes) != cudaSuccess) {
      cudaGetLastError();
      h->err = "pinned host allocation failed";
      throw Fail{EIG_ERR_NOMEM};
    }
    h->pinned_bytes = bytes;
  }
  return h->pinned;
}

static size_t gemm_partial_doubles(int m, int n, int k) {
  const int s = gemm_choose_splits(m, n, k);
  return s > 1 ? (size_t)(s + 1) * m * n : 0;
}

// Split-K scratch for the square m x m x m products of every node size m <= n
// (smaller nodes use more K chunks, so the maximum is not at m = n).
static size_t square_partial_doubles(int n) {
  size_t best = 1;
  for (int m = 1; m <= n; ++m) best = std::max(best, gemm_partial_doubles(m, m, m));
  return best;
}

// ---------------------------------------------------------------- QR
struct QRBufs {
  double* W;   int ldw;    // matrix being factorised (in place)
  double* V;   int ldv;    // explicit unit-lower-trapezoidal reflectors
  double* T;   int ldt;    // block T factors, jb x n
  double* tau;
  double* Wk;              // jb x cols product of a block reflector
  double* part;            // split-K partials
  int prec = EIG_FP64;     // arithmetic of the reflector products
  void* tcw = nullptr;     // BF16 planes (split precision)
  int* tcerr = nullptr;    // device flag of the tensor-core kernel
  // two-level form (tensor-core modes): outer blocks of NB2 columns whose
  // aggregated reflector updates the trailing matrix in one tensor-core
  // product pair; TB holds each outer block's NB2 x NB2 T (ld NB2), WB / WB2
  // its NB2 x cols products; cap2 = columns the buffers were carved for
  double* TB = nullptr;
  double* WB = nullptr;
  double* WB2 = nullptr;
  int cap2 = 0;
  bool two_level = false;   // set by geqrf: the last factorisation used it
};

constexpr int NB2 = 256;   // outer block width of the two-level QR

// Internal tier of EIG_SPLIT_FP32 (never passed in by a caller): the
// error-free split with five digits (30 bits), taken by a node whose attempt
// found a true split (0 < rank < n) that the four-digit products could not
// resolve below the split tolerance; the next tier is EIG_FP64_TC.
constexpr int PREC_SPLIT30 = 13;

// First tier of an EIG_SPLIT_FP32 node of size m whose eigenvalues lie in
// [lo, hi].  A split's residual ||E21|| / ||A|| is about the tier's rounding
// level times ||A_node|| over the eigenvalue gap at the line, and the mean gap
// is (hi - lo) / m, so kappa = m max(|lo|, |hi|) / (hi - lo) estimates the
// amplification.  The first tier whose level times kappa stays below the
// 1e-6 split tolerance is taken: four digits at about 2^-20 per unit of
// kappa, five digits at about 2^-27 (fitted to the solver's own log on the
// semicircle at n = 8192: five-digit attempts succeeded up to m ~ 165 near
// the centre of the spectrum, kappa ~ 80, and four-digit ones never did);
// else the FP64-accurate split.  Starting there saves the attempts that
// cannot succeed; a node still escalates when its attempt fails.
static int split_start_tier(int m, double lo, double hi) {
  const double w = hi - lo, a = std::max(std::fabs(lo), std::fabs(hi));
  const double kappa = w > 0.0 ? m * a / w : INFINITY;
  if (kappa * 0x1p-20 <= 1e-6) return EIG_SPLIT_FP32;
  if (kappa * 0x1p-27 <= 1e-6) return PREC_SPLIT30;
  return EIG_FP64_TC;
}

// split precision: FP32-level products on the tensor cores, FP64 panels,
// tests and refinement (BF16 x 3, or the unbiased four- / five-digit split)
static bool split_mode(int prec) {
  return prec == EIG_SPLIT_BF16X3 || prec == EIG_SPLIT_FP32 || prec == PREC_SPLIT30;
}
// contractions on the tensor cores: the split-precision forms or the FP64-accurate split
static bool tc_path(int prec) { return split_mode(prec) || prec == EIG_FP64_TC; }
static bool valid_prec(int prec) {
  return prec == EIG_FP64 || prec == EIG_SPLIT_BF16X3 || prec == EIG_FP64_TC ||
         prec == EIG_SPLIT_FP32;
}

// Plane workspace of a product in `prec`; EIG_SPLIT_FP32 reserves the largest
// of its tiers (four, five and nine digits).
static size_t tc_ws_bytes(int prec, int m, int n, int k) {
  if (prec == EIG_SPLIT_BF16X3) return tc_gemm_workspace_bytes(m, n, k);
  if (prec == EIG_SPLIT_FP32)
    return std::max(std::max(tcx32_gemm_workspace_bytes(m, n, k),
                             tcx30_gemm_workspace_bytes(m, n, k)),
                    tcx_gemm_workspace_bytes(m, n, k));
  if (prec == PREC_SPLIT30) return tcx30_gemm_workspace_bytes(m, n, k);
  if (prec == EIG_FP64_TC) return tcx_gemm_workspace_bytes(m, n, k);
  return 0;
}

// FP32-level tensor-core product of the split-precision form `prec`
static cudaError_t split_gemm(cudaStream_t s, int prec, bool ta, bool tb, int m, int n, int k,
                              double alpha, const double* A, int lda, const double* B, int ldb,
                              double beta, double* C, int ldc, void* ws, int* err) {
  if (prec == EIG_SPLIT_FP32)
    return tcx32_gemm(s, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, ws, err);
  if (prec == PREC_SPLIT30)
    return tcx30_gemm(s, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, ws, err);
  return tc_gemm(s, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, ws, err);
}

// Products that stay on the FP64 DFMA kernel in EIG_FP64_TC mode: the digit
// split costs a pass over both operands and three launches, and a 128 x 48
// tile with nine digit planes per operand needs every dimension of a few
// hundred to pay (measured: 14.9x DFMA at 4096^3 and 12.7x at 2048^3; in its
// first form 3.1x at 1024^3, and slower on the rank-32 reflector products
// 2048 x 32 x 4096 and 4096 x 2048 x 32).
static bool tcx_worth(int m, int n, int k) {
  return m >= 128 && n >= 128 && k >= 128 && (double)m * n * k >= 33554432.0;
}

// C = alpha op(A) op(B) + beta C in the arithmetic of `prec`: BF16 x 3 on the
// tensor cores (split precision), the FP64-accurate tensor-core split for
// large products (EIG_FP64_TC), else the FP64 DFMA kernel with split-K.
static void mm(eig_handle_t h, int prec, void* tcw, int* tcerr, bool ta, bool tb, int m, int n,
               int k, double alpha, const double* A, int lda, const double* B, int ldb,
               double beta, double* C, int ldc, int splits, double* part) {
  if (split_mode(prec))
    CK(split_gemm(h->stream, prec, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, tcw,
                  tcerr));
  else if (prec == EIG_FP64_TC && tcx_worth(m, n, k))
    CK(tcx_gemm(h->stream, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, tcw, tcerr));
  else
    CK(gemm(h->stream, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, splits, part));
}

// BF16 plane scratch of the reflector products of an m x n QR.
static size_t tcw_qr_bytes(int prec, int m, int n) {
  return std::max(tc_ws_bytes(prec, n, JB_LD_C, m), tc_ws_bytes(prec, m, n, JB_LD_C));
}

// The two-level QR runs in the modes whose tensor-core product is the
// error-free digit split (FP64-accurate or the split-precision tiers), on
// factorisations tall and wide enough for NB2-wide outer updates to fill it.
static bool tcx_family(int prec) {
  return prec == EIG_FP64_TC || prec == EIG_SPLIT_FP32 || prec == PREC_SPLIT30;
}
static bool two_level_fits(int m, int n) { return m >= 512 && n >= 2 * NB2; }
// plane scratch of the outer products (NB2 x n x m and m x n x NB2, T products)
static size_t tcw_qr2_bytes(int prec, int m, int n) {
  if (!tcx_family(prec) || !two_level_fits(m, n)) return 0;
  return std::max(std::max(tc_ws_bytes(prec, NB2, n, m), tc_ws_bytes(prec, m, n, NB2)),
                  tc_ws_bytes(prec, NB2, n, NB2));
}

constexpr int JB_LD = 32;

// split-K partials of the jb x cols reflector products (at most 32 K-chunks)
static size_t qr_part_doubles(int m, int cols) { return (size_t)33 * JB_LD * std::max(cols, 1) + 0 * m; }

// Product of an outer block reflector (two-level QR) in the mode's
// tensor-core arithmetic: the split tiers, or the FP64-accurate split where it
// pays (tcx_worth), else the FP64 DFMA kernel.
static void outer_mm(eig_handle_t h, const QRBufs& q, bool ta, bool tb, int m, int n, int k,
                     double alpha, const double* A, int lda, const double* B, int ldb,
                     double beta, double* C, int ldc) {
  if (split_mode(q.prec))
    CK(split_gemm(h->stream, q.prec, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, q.tcw,
                  q.tcerr));
  else if (tcx_worth(m, n, k))
    CK(tcx_gemm(h->stream, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, q.tcw, q.tcerr));
  else
    CK(gemm(h->stream, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc));
}

// C <- (I - V T V^T)^T C for the reflectors of one panel (rows j0.., jb
// columns) on the nc columns of C (mb rows, ldw).
static void panel_update(eig_handle_t h, QRBufs& q, int j0, int jb, int mb, double* C, int nc) {
  cudaStream_t s = h->stream;
  double* Vb = q.V + j0 + (size_t)j0 * q.ldv;
  if (split_mode(q.prec)) {
    // (V^T C)^T = C^T V on the tensor cores (M = nc rows, N = jb)
    CK(split_gemm(s, q.prec, true, false, nc, jb, mb, 1.0, C, q.ldw, Vb, q.ldv, 0.0, q.part,
                  nc, q.tcw, q.tcerr));
    CK(reduce_trmm(s, jb, nc, q.part, 1, q.T + (size_t)j0 * q.ldt, q.ldt, true, q.Wk, true));
    CK(split_gemm(s, q.prec, false, false, mb, nc, jb, -1.0, Vb, q.ldv, q.Wk, jb, 1.0, C,
                  q.ldw, q.tcw, q.tcerr));
  } else {
    int sp = gemm_choose_splits(jb, nc, mb);
    sp = gemm_partials(s, true, jb, nc, mb, Vb, q.ldv, C, q.ldw, sp, q.part);
    if (sp < 0) CK(cudaGetLastError());
    CK(reduce_trmm(s, jb, nc, q.part, sp, q.T + (size_t)j0 * q.ldt, q.ldt, true, q.Wk));
    CK(gemm(s, false, false, mb, nc, jb, -1.0, Vb, q.ldv, q.Wk, jb, 1.0, C, q.ldw));
  }
}

// T of the outer block J0..J0+JB (aggregated from its panels' T factors by
// T_{1:c+jb} = [[T_{1:c}, -T_{1:c} (V_{1:c}^T V_b) T_b], [0, T_b]]) into TB.
static void outer_T(eig_handle_t h, QRBufs& q, int m, int J0, int JB, int jbmax) {
  cudaStream_t s = h->stream;
  double* TBb = q.TB + (size_t)(J0 / NB2) * NB2 * NB2;
  CK(cudaMemsetAsync(TBb, 0, sizeof(double) * NB2 * NB2, s));
  const int mb = m - J0;
  const double* Vo = q.V + J0 + (size_t)J0 * q.ldv;
  for (int c0 = 0; c0 < JB; c0 += jbmax) {
    const int jb = std::min(jbmax, JB - c0);
    const double* Tin = q.T + (size_t)(J0 + c0) * q.ldt;
    CK(copy_matrix(s, jb, jb, Tin, q.ldt, TBb + c0 + (size_t)c0 * NB2, NB2));
    if (c0 == 0) continue;
    // G = V_{1:c}^T V_b (c0 x jb, deterministic split-K over the mb rows)
    CK(gemm(s, true, false, c0, jb, mb, 1.0, Vo, q.ldv, Vo + (size_t)c0 * q.ldv, q.ldv, 0.0, q.WB,
            NB2, gemm_choose_splits(c0, jb, mb), q.part));
    CK(gemm(s, false, false, c0, jb, c0, 1.0, TBb, NB2, q.WB, NB2, 0.0, q.WB2, NB2));
    CK(gemm(s, false, false, c0, jb, jb, -1.0, q.WB2, NB2, Tin, q.ldt, 0.0,
            TBb + (size_t)c0 * NB2, NB2));
  }
}

// Blocked right-looking Householder QR of the m x n matrix in q.W.  In the
// tensor-core modes (two_level_fits), panels of jbmax columns update only
// their NB2-column outer block on the FP64 pipe, and each outer block's
// aggregated reflector then updates the trailing matrix in one tensor-core
// product pair (the rank-NB2 compact-WY update).
static int geqrf(eig_handle_t h, int m, int n, QRBufs& q) {
  cudaStream_t s = h->stream;
  NvtxRange nvtx_("eig.qr");
  const int jbmax = panel_max_width(m);
  if (jbmax <= 0) {
    h->err = "matrix too tall for the on-chip panel factorisation";
    throw Fail{EIG_ERR_ARG};
  }
  q.two_level = q.TB != nullptr && tcx_family(q.prec) && two_level_fits(m, n) && n <= q.cap2 &&
                NB2 % jbmax == 0;
  const int outer = q.two_level ? NB2 : n;
  for (int J0 = 0; J0 < n; J0 += outer) {
    const int JB = std::min(outer, n - J0);
    const int jend = J0 + JB;
    if (q.two_level)   // rows J0.. of the block's reflectors above each panel are zero
      CK(cudaMemset2DAsync(q.V + J0 + (size_t)J0 * q.ldv, sizeof(double) * q.ldv, 0,
                           sizeof(double) * JB, JB, s));
    for (int j0 = J0; j0 < jend; j0 += jbmax) {
      const int jb = std::min(jbmax, jend - j0);
      double* Vb = q.V + j0 + (size_t)j0 * q.ldv;
      CK(panel_qr(s, m - j0, jb, q.W + j0 + (size_t)j0 * q.ldw, q.ldw, Vb, q.ldv, q.tau + j0,
                  q.T + (size_t)j0 * q.ldt, q.ldt));
      const int nc = jend - j0 - jb;
      if (nc > 0) panel_update(h, q, j0, jb, m - j0, q.W + j0 + (size_t)(j0 + jb) * q.ldw, nc);
    }
    if (q.two_level) {
      outer_T(h, q, m, J0, JB, jbmax);
      const int NC = n - jend, mb = m - J0;
      if (NC > 0) {
        const double* Vo = q.V + J0 + (size_t)J0 * q.ldv;
        const double* TBb = q.TB + (size_t)(J0 / NB2) * NB2 * NB2;
        double* C = q.W + J0 + (size_t)jend * q.ldw;
        outer_mm(h, q, true, false, JB, NC, mb, 1.0, Vo, q.ldv, C, q.ldw, 0.0, q.WB, NB2);
        outer_mm(h, q, true, false, JB, NC, JB, 1.0, TBb, NB2, q.WB, NB2, 0.0, q.WB2, NB2);
        outer_mm(h, q, false, false, mb, NC, JB, -1.0, Vo, q.ldv, q.WB2, NB2, 1.0, C, q.ldw);
      }
    }
  }
  return jbmax;
}

// Y <- Q Y for the reflectors of an m x nref factorisation (applied last
// block first).  skip_identity: Y started as [I; 0], so columns left of a
// block's first row are still unit vectors it does not touch.  After a
// two-level factorisation the outer blocks' aggregated reflectors are applied
// with tensor-core products.
static void apply_q(eig_handle_t h, int m, int nref, int jbmax, QRBufs& q, double* Y, int ldy,
                    int ncols, bool skip_identity) {
  cudaStream_t s = h->stream;
  if (q.two_level) {
    const int nout = (nref + NB2 - 1) / NB2;
    for (int b = nout - 1; b >= 0; --b) {
      const int J0 = b * NB2;
      const int JB = std::min(NB2, nref - J0);
      const int mb = m - J0;
      const int c0 = skip_identity ? J0 : 0;
      const int nc = ncols - c0;
      if (nc <= 0) continue;
      double* Yb = Y + J0 + (size_t)c0 * ldy;
      const double* Vo = q.V + J0 + (size_t)J0 * q.ldv;
      const double* TBb = q.TB + (size_t)b * NB2 * NB2;
      outer_mm(h, q, true, false, JB, nc, mb, 1.0, Vo, q.ldv, Yb, ldy, 0.0, q.WB, NB2);
      outer_mm(h, q, false, false, JB, nc, JB, 1.0, TBb, NB2, q.WB, NB2, 0.0, q.WB2, NB2);
      outer_mm(h, q, false, false, mb, nc, JB, -1.0, Vo, q.ldv, q.WB2, NB2, 1.0, Yb, ldy);
    }
    return;
  }
  const int nblocks = (nref + jbmax - 1) / jbmax;
  for (int b = nblocks - 1; b >= 0; --b) {
    const int j0 = b * jbmax;
    const int jb = std::min(jbmax, nref - j0);
    const int mb = m - j0;
    const int c0 = skip_identity ? j0 : 0;
    const int nc = ncols - c0;
    if (nc <= 0) continue;
    double* Yb = Y + j0 + (size_t)c0 * ldy;
    const double* Vb = q.V + j0 + (size_t)j0 * q.ldv;
    if (split_mode(q.prec)) {
      CK(split_gemm(s, q.prec, true, false, nc, jb, mb, 1.0, Yb, ldy, Vb, q.ldv, 0.0, q.part, nc,
                    q.tcw, q.tcerr));
      CK(reduce_trmm(s, jb, nc, q.part, 1, q.T + (size_t)j0 * q.ldt, q.ldt, false, q.Wk, true));
      CK(split_gemm(s, q.prec, false, false, mb, nc, jb, -1.0, Vb, q.ldv, q.Wk, jb, 1.0, Yb, ldy,
                    q.tcw, q.tcerr));
      continue;
    }
    int sp = gemm_choose_splits(jb, nc, mb);
    sp = gemm_partials(s, true, jb, nc, mb, Vb, q.ldv, Yb, ldy, sp, q.part);
    if (sp < 0) CK(cudaGetLastError());
    CK(reduce_trmm(s, jb, nc, q.part, sp, q.T + (size_t)j0 * q.ldt, q.ldt, false, q.Wk));
    CK(gemm(s, false, false, mb, nc, jb, -1.0, Vb, q.ldv, q.Wk, jb, 1.0, Yb, ldy));
  }
}

struct QRWork {
  QRBufs q;
};

static size_t carve_qr(Arena& a, int m, int n, QRWork& w, int prec = EIG_FP64,
                       int outer_prec = EIG_FP64) {
  const size_t start = a.used;
  if (tcx_family(outer_prec) && two_level_fits(m, n)) {
    w.q.TB = a.take<double>((size_t)((n + NB2 - 1) / NB2) * NB2 * NB2);
    w.q.WB = a.take<double>((size_t)NB2 * n);
    w.q.WB2 = a.take<double>((size_t)NB2 * n);
    w.q.cap2 = n;
  }
  w.q.W = a.take<double>((size_t)m * n);
  w.q.ldw = m;
  w.q.V = a.take<double>((size_t)m * n);
  w.q.ldv = m;
  w.q.T = a.take<double>((size_t)JB_LD * n);
  w.q.ldt = JB_LD;
  w.q.tau = a.take<double>(n);
  w.q.Wk = a.take<double>((size_t)JB_LD * n);
  w.q.part = a.take<double>(qr_part_doubles(m, n));
  w.q.prec = prec;
  w.q.tcw = split_mode(prec) ? (void*)a.take<char>(tcw_qr_bytes(prec, m, n)) : nullptr;
  w.q.tcerr = a.take<int>(4);
  return a.used - start;
}

// Explicit Q (m x n) and optionally R (n x n) of X (m x n).
static void qr_explicit(eig_handle_t h, QRWork& w, int m, int n, const double* X, int ldx,
                        double* Q, int ldq, double* R, int ldr) {
  cudaStream_t s = h->stream;
  CK(copy_matrix(s, m, n, X, ldx, w.q.W, w.q.ldw));
  const int jbmax = geqrf(h, m, n, w.q);
  if (R) CK(upper_triangle(s, n, w.q.W, w.q.ldw, R, ldr));
  if (Q) {
    CK(fill_identity_block(s, m, n, Q, ldq, 0));
    apply_q(h, m, n, jbmax, w.q, Q, ldq, n, true);
  }
}

// ---------------------------------------------------------------- IRS
struct IRSWork {
  double *Aj, *Bj, *An, *Bn, *Y, *Rc, *Rp, *gpart;
  unsigned long long* sums;
  int* flag;
  QRWork qr;   // W is the stacked 2n x n matrix
  int prec = EIG_FP64;
  void* tcw = nullptr;
};

static size_t carve_irs(Arena& a, int n, IRSWork& w, int prec = EIG_FP64) {
  const size_t start = a.used;
  const size_t nn = (size_t)n * n;
  w.Aj = a.take<double>(nn);
  w.Bj = a.take<double>(nn);
  w.An = a.take<double>(nn);
  w.Bn = a.take<double>(nn);
  w.Y = a.take<double>(2 * nn);
  w.Rc = a.take<double>(nn);
  w.Rp = a.take<double>(nn);
  w.gpart = a.take<double>(square_partial_doubles(n));
  w.sums = a.take<unsigned long long>(4);
  w.flag = a.take<int>(4);
  w.prec = prec;
  // one plane buffer serves the QR's reflector products and the complement
  // products (they run one after the other on the stream)
  w.tcw = tc_path(prec) ? (void*)a.take<char>(std::max(
                              std::max(tc_ws_bytes(prec, n, n, n),
                                       split_mode(prec) ? tcw_qr_bytes(prec, 2 * n, n) : 0),
                              tcw_qr2_bytes(prec, 2 * n, n)))
                        : nullptr;
  carve_qr(a, 2 * n, n, w.qr, EIG_FP64, prec);
  w.qr.q.prec = prec;
  w.qr.q.tcw = w.tcw;
  return a.used - start;
}

struct IRSOut {
  int iters;
  bool converged;
  double last_ratio;
  double* Ap;
  double* Bp;
  double* Rlast;
};

static double default_tau(int n) { return std::max(1e-14, 4.0 * std::sqrt((double)n) * 0x1p-53); }

// Below this ratio the R-test also stops once the ratio has stopped falling
// quadratically: the rounding floor of the iterates has been reached.  The
// split-precision iterates sit at an FP32-level floor (1e-3); the FP64-
// accurate tensor-core products keep an FP64-level floor that at large n can
// lie a little above default_tau (1e-10); plain FP64 keeps the plain R-test.
static double stall_level(int prec) {
  if (split_mode(prec)) return 1e-3;
  return prec == EIG_FP64_TC ? 1e-10 : 0.0;
}

static bool irs_trace() {
  static const bool on = [] {
    const char* v = std::getenv("EIGDC_VERBOSE");
    return v && v[0] == '1';
  }();
  return on;
}

// stall_below > 0: also stop once the ratio is below stall_below and fell by
// less than 4x over the last squaring (stall_level).
static IRSOut run_irs(eig_handle_t h, IRSWork& w, int n, const double* A, int lda, const double* B,
                      int ldb, const eig_region_t& rg, double tau, int maxit,
                      double stall_below = 0.0, bool use_graphs = false) {
  cudaStream_t s = h->stream;
  NvtxRange nvtx_("eig.irs");
  const size_t nn = (size_t)n * n;
  QRBufs& q = w.qr.q;
  q.ldw = 2 * n;   // the stacked matrix of this (node) size, packed
  q.ldv = 2 * n;
  CK(region_stack(s, n, A, lda, B, ldb, rg.kind, rg.c_or_sigma, rg.r_or_s, w.Aj, w.Bj, q.W));
  double* Aj = w.Aj;
  double* Bj = w.Bj;
  double* An = w.An;
  double* Bn = w.Bn;
  double* Rc = w.Rc;
  double* Rp = w.Rp;
  unsigned long long* hsum = static_cast<unsigned long long*>(pinned(h, 64));
  const int gsplit = gemm_choose_splits(n, n, n);
  CK(cudaMemsetAsync(q.tcerr, 0, sizeof(int), s));
  IRSOut out{0, false, 0.0, nullptr, nullptr, nullptr};
  bool have_prev = false;
  // Device work of one squaring: QR of the stack, R_j (and the R-test sums),
  // the complement [Q12; Q22] = Q [0; I], A_{j+1}, B_{j+1}, the next stack.
  auto squaring = [&](bool prev) {
    const int jbmax = geqrf(h, 2 * n, n, q);
    if (prev) {
      CK(cudaMemsetAsync(w.sums, 0, 2 * sizeof(unsigned long long), s));
      CK(r_extract_diff(s, n, q.W, q.ldw, Rc, Rp, w.sums));
    } else {
      CK(r_extract_diff(s, n, q.W, q.ldw, Rc, nullptr, nullptr));
    }
    CK(fill_identity_block(s, 2 * n, n, w.Y, 2 * n, n));
    apply_q(h, 2 * n, n, jbmax, q, w.Y, 2 * n, n, false);
    mm(h, w.prec, w.tcw, q.tcerr, true, false, n, n, n, 1.0, w.Y, 2 * n, Aj, n, 0.0, An, n, gsplit,
       w.gpart);
    mm(h, w.prec, w.tcw, q.tcerr, true, false, n, n, n, 1.0, w.Y + n, 2 * n, Bj, n, 0.0, Bn, n,
       gsplit, w.gpart);
    CK(stack_pencil(s, n, An, Bn, q.W));
  };
  // From the second squaring on, the launch sequence repeats with the buffer
  // pairs alternating: it is captured once per parity as a CUDA graph (cached
  // on the handle for this workspace and size) and replayed.  Streams that
  // cannot be captured (the legacy default stream) launch eagerly.
  const bool graphs = use_graphs && (s != nullptr) && !h->graphs_off;
  auto run_graph = [&](int parity) {
    for (auto& g : h->graphs) {
      if (g.base == w.Aj && g.n == n && g.prec == w.prec && g.parity == parity) {
        CK(cudaGraphLaunch(g.exec, s));
        note_launches(g.kernels);
        return;
      }
    }
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      h->graphs_off = true;
      squaring(true);
      return;
    }
    try {
      squaring(true);
    } catch (Fail&) {
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(s, &g);
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      throw;
    }
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned long long kernels = 0;   // kernel nodes: the launches of one replay
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    if (e == cudaSuccess && graph) {
      size_t nn = 0;
      e = cudaGraphGetNodes(graph, nullptr, &nn);
      std::vector<cudaGraphNode_t> nodes(nn);
      if (e == cudaSuccess && nn) e = cudaGraphGetNodes(graph, nodes.data(), &nn);
      for (size_t i = 0; e == cudaSuccess && i < nn; ++i) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel)
          ++kernels;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    }
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess || !exec) {
      // capture unavailable here: launch eagerly from now on
      cudaGetLastError();
      h->graphs_off = true;
      squaring(true);
      return;
    }
    if (h->graphs.size() >= 96) clear_graphs(h);
    // the first launch's kernels were counted while capturing; replays add
    // `kernels` each
    h->graphs.push_back({w.Aj, n, w.prec, parity, exec, kernels});
    CK(cudaGraphLaunch(exec, s));
  };
  for (int j = 0;; ++j) {
    if (j == 0 || !graphs) squaring(have_prev);
    else run_graph(j & 1);
    std::swap(Aj, An);
    std::swap(Bj, Bn);
    if (have_prev) {
      CK(cudaMemcpyAsync(hsum, w.sums, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(&hsum[2], q.tcerr, sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (static_cast<int>(hsum[2] & 0xFFFFFFFFull) != 0) {
        h->err = "tensor-core GEMM: a bounded wait timed out";
        throw Fail{EIG_ERR_CUDA};
      }
      double num, den;
      std::memcpy(&num, &hsum[0], 8);
      std::memcpy(&den, &hsum[1], 8);
      const double ratio = den > 0.0 ? num / den : (num == 0.0 ? 0.0 : INFINITY);
      const double prev = out.last_ratio;
      out.last_ratio = ratio;
      const bool stalled = j >= 2 && ratio <= stall_below && ratio > 0.25 * prev;
      if (irs_trace())
        std::fprintf(stderr, "[eigdc] irs n=%d squaring=%d ratio=%.3e tau=%.3e%s\n", n, j + 1,
                     ratio, tau, stalled ? " (stalled)" : "");
      if (ratio <= tau || stalled) {
        out.iters = j + 1;
        out.converged = true;
        out.Rlast = Rc;
        break;
      }
    }
    std::swap(Rc, Rp);
    have_prev = true;
    if (j + 1 > maxit) {
      out.iters = j + 1;
      out.converged = false;
      out.Rlast = Rp;
      break;
    }
  }
  (void)nn;
  out.Ap = Aj;
  out.Bp = Bj;
  return out;
}

// ---------------------------------------------------------------- split
struct SplitWork {
  double *G, *Vh, *X, *U, *R2, *S, *Y, *Z, *Qt, *Ucur, *tmp, *Ahat, *scores, *colpart, *gpart;
  double* QLn = nullptr;    // pencils: left splitter Q_L
  double* Bhat = nullptr;   // pencils: Q_L^T B Q_R
  unsigned long long* nbits;
  int* rank;
  QRWork qr;
  int prec = EIG_FP64;
  void* tcw = nullptr;
};

static size_t carve_split(Arena& a, int n, SplitWork& w, int prec = EIG_FP64,
                          bool pencil = false) {
  const size_t start = a.used;
  const size_t nn = (size_t)n * n;
  if (pencil) {
    w.QLn = a.take<double>(nn);
    w.Bhat = a.take<double>(nn);
  }
  w.G = a.take<double>(nn);
  w.Vh = a.take<double>(nn);
  w.X = a.take<double>(nn);
  w.U = a.take<double>(nn);
  w.R2 = a.take<double>(nn);
  w.S = a.take<double>(nn);
  w.Y = a.take<double>(nn);
  w.Z = a.take<double>(nn);
  w.Qt = a.take<double>(nn);
  w.Ucur = a.take<double>(nn);
  w.tmp = a.take<double>(nn);
  w.Ahat = a.take<double>(nn);
  w.scores = a.take<double>(std::max(n, 1));
  const size_t nrb = (size_t)(n + 31) / 32;
  w.colpart = a.take<double>(nrb * n + n + 8);
  w.gpart = a.take<double>(square_partial_doubles(n));
  w.nbits = a.take<unsigned long long>(4);
  w.rank = a.take<int>(4);
  w.prec = prec;
  w.tcw = tc_path(prec) ? (void*)a.take<char>(std::max(
                              std::max(tc_ws_bytes(prec, n, n, n),
                                       split_mode(prec) ? tcw_qr_bytes(prec, n, n) : 0),
                              tcw_qr2_bytes(prec, n, n)))
                        : nullptr;
  carve_qr(a, n, n, w.qr, EIG_FP64, prec);
  w.qr.q.prec = prec;
  w.qr.q.tcw = w.tcw;
  return a.used - start;
}

// split_tol <= 0: max(1e-12, 16 n u), the rounding floor of ||E21||_1/||A||_1
// after an FP64 step grows about like n u (measured 4-5 n u at n = 2048 and
// 4096); split precision: at least 1e-3 (FP32-level iterates, refined later).
// Pencils: max(1e-10, 16 n u).  The two deflating subspaces are computed
// independently, so their mutual error enters ||F21|| without cancellation,
// concentrated in a few ill-separated columns; the 1-norm score (a column
// maximum) overstates the finished solve's Frobenius backward error 10-50x.
static double effective_split_tol(const eig_params_t& p, int n, bool pencil = false) {
  double t = p.split_tol > 0 ? p.split_tol
                             : std::max(pencil ? 1e-10 : 1e-12, 16.0 * n * 0x1p-53);
  // split precision: FP32-level iterates.  BF16 x 3 accepts up to 1e-3;
  // EIG_SPLIT_FP32 holds its tiers to 1e-6, the coupling the closing FP64
  // refinement resolves pair by pair (measured: splits accepted at 1e-3 left
  // eigenvalue errors of 4e-5 after the refinement at n = 8192, where
  // neighbouring eigenvalues are 2e-4 apart)
  if (p.prec == EIG_SPLIT_BF16X3) t = std::max(t, 1e-3);
  else if (split_mode(p.prec)) t = std::max(t, 1e-6);
  return t;
}

// Tie rule (paper silent): smallest e(k); exact ties -> k closest to n/2,
// then the smaller k.
static int choose_k(const double* e, int n) {
  int best = -1;
  for (int k = 1; k < n; ++k) {
    if (best < 0) {
      best = k;
      continue;
    }
    const double v = e[k - 1], bv = e[best - 1];
    const int d = std::abs(2 * k - n), bd = std::abs(2 * best - n);
    if (v < bv || (v == bv && (d < bd || (d == bd && k < best)))) best = k;
  }
  return best;
}

struct SplitOut {
  int k;
  double e;
  int rank;
  int draw;
  bool accepted;
};

static double device_norm1(eig_handle_t h, int rows, int cols, const double* A, int lda,
                           unsigned long long* dbits) {
  cudaStream_t s = h->stream;
  CK(cudaMemsetAsync(dbits, 0, sizeof(unsigned long long), s));
  CK(norm1_bits(s, rows, cols, A, lda, dbits));
  unsigned long long* hb = static_cast<unsigned long long*>(pinned(h, 64));
  CK(cudaMemcpyAsync(hb, dbits, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  double v;
  std::memcpy(&v, hb, 8);
  return v;
}

// Q_R = GRURV(2, A_p + B_p, A_p, -1, +1) (Algorithms 4-6) into w.Ucur and the
// RURV rank of A_p (relative to max |R1_ii|) into w.rank, for Haar draw `code`.
static void right_splitter(eig_handle_t h, SplitWork& w, int n, const double* Ap,
                           const double* Bp, int ldp, uint64_t seed, uint64_t stream_id,
                           int code, int gsplit) {
  cudaStream_t s = h->stream;
  // Haar V (Algorithm 1, lines 1-2)
  CK(gaussian(s, n, n, seed, PURPOSE_HAAR, stream_id, code, w.G, n));
  qr_explicit(h, w.qr, n, n, w.G, n, w.Vh, n, nullptr, 0);
  // RURV(A_p): [U, R2] = QR(A_p V^T)
  mm(h, w.prec, w.tcw, w.qr.q.tcerr, false, true, n, n, n, 1.0, Ap, ldp, w.Vh, n, 0.0, w.X, n,
     gsplit, w.gpart);
  qr_explicit(h, w.qr, n, n, w.X, n, w.U, n, w.R2, n);
  // RQ(U^T (A_p + B_p)) by reversal: Z = (J Y)^T = Q~ R~, U_cur = Q~ J
  CK(add_matrices(s, n, n, Ap, ldp, Bp, ldp, w.S, n));
  mm(h, w.prec, w.tcw, w.qr.q.tcerr, true, false, n, n, n, 1.0, w.U, n, w.S, n, 0.0, w.Y, n,
     gsplit, w.gpart);
  CK(reverse_transpose(s, n, w.Y, n, w.Z, n));
  qr_explicit(h, w.qr, n, n, w.Z, n, w.Qt, n, w.G, n);   // R~ (diag: R1 reversed) into G
  // rank threshold above the noise floor of the iterates: FP64 rounding, or
  // the FP32 level of the split-precision products
  CK(count_rank(s, n, w.R2, n, w.G, n, split_mode(w.prec) ? 1e-5 : 1e-8, w.rank));
  CK(reverse_columns(s, n, n, w.Qt, n, w.Ucur, n));
}

// Q_L = GRURV(2, A_pL^T, (A_pL + B_pL)^T, +1, -1) (Algorithm 4, left deflating
// subspace) from the IRS iterates of (A^T, B^T), into w.QLn:
//   RULV((A_pL + B_pL)^T ^T): X = (A_pL + B_pL) V_L^T = U L (QL via the QR of
//   the column-reversed X), then Q_L = Q of QR(A_pL^T U).
static void left_splitter(eig_handle_t h, SplitWork& w, int n, const double* ApL,
                          const double* BpL, int ldp, uint64_t seed, uint64_t stream_id, int code,
                          int gsplit) {
  cudaStream_t s = h->stream;
  CK(gaussian(s, n, n, seed, PURPOSE_HAAR_LEFT, stream_id, code, w.G, n));
  qr_explicit(h, w.qr, n, n, w.G, n, w.Vh, n, nullptr, 0);
  CK(add_matrices(s, n, n, ApL, ldp, BpL, ldp, w.S, n));
  mm(h, w.prec, w.tcw, w.qr.q.tcerr, false, true, n, n, n, 1.0, w.S, n, w.Vh, n, 0.0, w.X, n,
     gsplit, w.gpart);
  CK(reverse_columns(s, n, n, w.X, n, w.Z, n));
  qr_explicit(h, w.qr, n, n, w.Z, n, w.Qt, n, nullptr, 0);
  CK(reverse_columns(s, n, n, w.Qt, n, w.U, n));
  mm(h, w.prec, w.tcw, w.qr.q.tcerr, true, false, n, n, n, 1.0, ApL, ldp, w.U, n, 0.0, w.Y, n,
     gsplit, w.gpart);
  qr_explicit(h, w.qr, n, n, w.Y, n, w.QLn, n, nullptr, 0);
}

// Reads the n-1 split scores, the rank and the tensor-core error flag back.
static void read_split(eig_handle_t h, SplitWork& w, int n, std::vector<double>& hscores,
                       int& rank) {
  cudaStream_t s = h->stream;
  const size_t sbytes = sizeof(double) * std::max(n - 1, 1);
  char* hb = static_cast<char*>(pinned(h, sbytes + 64));
  if (n >= 2) CK(cudaMemcpyAsync(hb, w.scores, sizeof(double) * (n - 1), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(hb + sbytes, w.rank, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(hb + sbytes + 8, w.qr.q.tcerr, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  int terr;
  std::memcpy(&terr, hb + sbytes + 8, sizeof(int));
  if (terr != 0) {
    h->err = "tensor-core GEMM: a bounded wait timed out";
    throw Fail{EIG_ERR_CUDA};
  }
  if (n >= 2) std::memcpy(hscores.data(), hb, sizeof(double) * (n - 1));
  std::memcpy(&rank, hb + sbytes, sizeof(int));
}

static void pick_k(SplitOut& out, const std::vector<double>& hscores, int n) {
  if (n >= 2) {
    out.k = choose_k(hscores.data(), n);
    out.e = hscores[out.k - 1];
  } else {
    out.k = 0;
    out.e = 0.0;
  }
}

// Splitter Q = GRURV(2, A_p + B_p, A_p, -1, +1), A^ = Q^T A Q, split test.
// Results stay in w.Ahat / w.Ucur.
static SplitOut run_split(eig_handle_t h, SplitWork& w, int n, const double* Ap,
                          const double* Bp, int ldp, const double* A, int lda, bool symmetric,
                          uint64_t stream_id, int attempt, const eig_params_t& p,
                          bool irs_converged, std::vector<double>& hscores) {
  cudaStream_t s = h->stream;
  NvtxRange nvtx_("eig.split");
  const double normA = device_norm1(h, n, n, A, lda, w.nbits);
  const int gsplit = gemm_choose_splits(n, n, n);
  SplitOut out{0, INFINITY, 0, 0, false};
  const int draws = std::max(1, p.v_draws);
  hscores.assign(std::max(n - 1, 0), 0.0);
  CK(cudaMemsetAsync(w.qr.q.tcerr, 0, sizeof(int), s));
  for (int draw = 0; draw < draws; ++draw) {
    const int code = ((attempt & 0x3F) << 2) | (draw & 3);
    right_splitter(h, w, n, Ap, Bp, ldp, p.seed, stream_id, code, gsplit);
    // similarity and split test
    mm(h, w.prec, w.tcw, w.qr.q.tcerr, false, false, n, n, n, 1.0, A, lda, w.Ucur, n, 0.0, w.tmp,
       n, gsplit, w.gpart);
    mm(h, w.prec, w.tcw, w.qr.q.tcerr, true, false, n, n, n, 1.0, w.Ucur, n, w.tmp, n, 0.0,
       w.Ahat, n, gsplit, w.gpart);
    if (symmetric) CK(symmetrize(s, n, w.Ahat, n));
    if (n >= 2) CK(split_scores(s, n, w.Ahat, n, normA > 0 ? 1.0 / normA : 1.0, w.colpart, w.scores, false));
    int rank;
    read_split(h, w, n, hscores, rank);
    out.rank = rank;
    out.draw = draw;
    pick_k(out, hscores, n);
    if (split_mode(p.prec) && rank > 0 && rank < n) {
      // FP32-level scores sit near the split tolerance, where the argmin can
      // fall on a block size far from the eigenvalue count (measured: k =
      // n - 1 at e = 8.6e-4 for rank 2690 of 4096); the rank-revealed size
      // is the split, and its score is the test
      out.k = rank;
      out.e = hscores[rank - 1];
    }
    out.accepted = irs_converged && out.k > 0 && out.k < n && out.e <= effective_split_tol(p, n);
    if (out.accepted || !irs_converged || rank == 0 || rank == n) break;
  }
  return out;
}

// One RGNEP split (Algorithm 4) from the IRS iterates of (A, B) (right) and
// of (A^T, B^T) (left): Q_R into w.Ucur, Q_L into w.QLn, A^ = Q_L^T A Q_R
// into w.Ahat, B^ = Q_L^T B Q_R into w.Bhat.  The score of k is
// ||E21||_1 / ||A||_1 + ||F21||_1 / ||B||_1.  Acceptance needs both IRS runs
// converged; redraws (v_draws) stop once the right IRS failed or the rank
// shows an empty side.
static SplitOut run_split_pencil(eig_handle_t h, SplitWork& w, int n, const double* ApR,
                                 const double* BpR, const double* ApL, const double* BpL, int ldp,
                                 const double* A, int lda, const double* B, int ldb,
                                 uint64_t stream_id, int attempt, const eig_params_t& p,
                                 bool conv_right, bool conv_left, std::vector<double>& hscores) {
  cudaStream_t s = h->stream;
  NvtxRange nvtx_("eig.split_pencil");
  const double normA = device_norm1(h, n, n, A, lda, w.nbits);
  const double normB = device_norm1(h, n, n, B, ldb, w.nbits);
  const int gsplit = gemm_choose_splits(n, n, n);
  SplitOut out{0, INFINITY, 0, 0, false};
  const int draws = std::max(1, p.v_draws);
  hscores.assign(std::max(n - 1, 0), 0.0);
  CK(cudaMemsetAsync(w.qr.q.tcerr, 0, sizeof(int), s));
  for (int draw = 0; draw < draws; ++draw) {
    const int code = ((attempt & 0x3F) << 2) | (draw & 3);
    right_splitter(h, w, n, ApR, BpR, ldp, p.seed, stream_id, code, gsplit);
    left_splitter(h, w, n, ApL, BpL, ldp, p.seed, stream_id, code, gsplit);
    mm(h, w.prec, w.tcw, w.qr.q.tcerr, false, false, n, n, n, 1.0, A, lda, w.Ucur, n, 0.0, w.tmp,
       n, gsplit, w.gpart);
    mm(h, w.prec, w.tcw, w.qr.q.tcerr, true, false, n, n, n, 1.0, w.QLn, n, w.tmp, n, 0.0,
       w.Ahat, n, gsplit, w.gpart);
    mm(h, w.prec, w.tcw, w.qr.q.tcerr, false, false, n, n, n, 1.0, B, ldb, w.Ucur, n, 0.0, w.tmp,
       n, gsplit, w.gpart);
    mm(h, w.prec, w.tcw, w.qr.q.tcerr, true, false, n, n, n, 1.0, w.QLn, n, w.tmp, n, 0.0,
       w.Bhat, n, gsplit, w.gpart);
    if (n >= 2) {
      CK(split_scores(s, n, w.Ahat, n, normA > 0 ? 1.0 / normA : 1.0, w.colpart, w.scores, false));
      CK(split_scores(s, n, w.Bhat, n, normB > 0 ? 1.0 / normB : 1.0, w.colpart, w.scores, true));
    }
    int rank;
    read_split(h, w, n, hscores, rank);
    out.rank = rank;
    out.draw = draw;
    pick_k(out, hscores, n);
    out.accepted = conv_right && conv_left && out.k > 0 && out.k < n &&
                   out.e <= effective_split_tol(p, n, true);
    if (out.accepted || !conv_right || rank == 0 || rank == n) break;
  }
  return out;
}

// ---------------------------------------------------------------- strategy
static void philox_host(uint32_t c[4], uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)M0 * c[0], p1 = (uint64_t)M1 * c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n1 = lo1, n2 = hi0 ^ c[3] ^ k1, n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    k0 += W0;
    k1 += W1;
  }
}

// u2 of pair 0 of (purpose, stream, attempt): a uniform in [0, 1).
static double philox_uniform(uint64_t seed, int purpose, uint64_t stream, int attempt) {
  uint32_t c[4] = {0u, ((uint32_t)(attempt & 0xFF) << 8) | ((uint32_t)(purpose & 0xFFFF) << 16),
                   (uint32_t)(stream & 0xFFFFFFFFull), (uint32_t)(stream >> 32)};
  philox_host(c, (uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32));
  const uint64_t m2 = ((uint64_t)c[2] << 20) | (c[3] >> 12);
  return (double)m2 * 0x1p-52;
}

// splitmix64 finaliser (Steele, Lea, Flood 2014): child ids of the tree.
static uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static uint64_t child_node(uint64_t parent, int side) {
  return splitmix64(2 * parent + (uint64_t)side + 1);
}


struct Node {
  int off, m;
  double lo, hi;
  uint64_t id;
  int depth;
  bool swapped = false;   // pencils: the node is handled as (B, A) (Sec. 3.5)
};

static void node_diag(eig_handle_t h, const double* Acur, int ld, int off, int m,
                      std::vector<double>& diag) {
  diag.resize(m);
  double* hb = static_cast<double*>(pinned(h, sizeof(double) * (m + 8)));
  CK(cudaMemcpy2DAsync(hb, sizeof(double), Acur + off + (size_t)off * ld, sizeof(double) * (ld + 1),
                       sizeof(double), m, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  std::memcpy(diag.data(), hb, sizeof(double) * m);
}

static void gershgorin_interval(eig_handle_t h, const double* A, int ld, int m, double* dtmp,
                                double& lo, double& hi) {
  CK(diag_gershgorin(h->stream, m, A, ld, dtmp, dtmp + m));
  double* hb = static_cast<double*>(pinned(h, sizeof(double) * (2 * m + 8)));
  CK(cudaMemcpyAsync(hb, dtmp, sizeof(double) * 2 * m, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  lo = INFINITY;
  hi = -INFINITY;
  for (int i = 0; i < m; ++i) {
    lo = std::min(lo, hb[i] - hb[m + i]);
    hi = std::max(hi, hb[i] + hb[m + i]);
  }
}

// Root interval of a symmetric matrix: [c - rho, c + rho] cut to Gershgorin,
// c = tr(A)/n, rho = 1.1 x the estimate of ||A - cI||_2 after POWER_STEPS
// power-iteration steps from the Philox Gaussian vector of purpose 9 (every
// eigenvalue lies within ||A - cI||_2 of c; Gershgorin alone overstates that
// radius by about sqrt(n) for dense matrices, and the line scale of each node
// is its interval's half-width).  dtmp: 2n + 8 doubles; dx, dy: n each.
constexpr int PURPOSE_POWER = 9;
constexpr int POWER_STEPS = 16;
static void spectral_interval(eig_handle_t h, const double* A, int ld, int n, double* dtmp,
                              double* dx, double* dy, uint64_t seed, double& lo, double& hi) {
  cudaStream_t s = h->stream;
  double glo, ghi;
  gershgorin_interval(h, A, ld, n, dtmp, glo, ghi);   // leaves diag in the pinned buffer
  const double* hd = static_cast<const double*>(pinned(h, sizeof(double) * (2 * n + 8)));
  double tr = 0.0;
  for (int i = 0; i < n; ++i) tr += hd[i];
  const double c = tr / n;
  double* dest = dtmp;
  CK(gaussian(s, n, 1, seed, PURPOSE_POWER, ROOT_NODE, 0, dy, n));
  CK(power_norm(s, n, 0.0, nullptr, dy, dx, dest));
  for (int it = 0; it < POWER_STEPS; ++it) {
    CK(gemm(s, false, false, n, 1, n, 1.0, A, ld, dx, n, 0.0, dy, n));
    CK(power_norm(s, n, c, dx, dy, dx, dest));
  }
  double* hb = static_cast<double*>(pinned(h, 64));
  CK(cudaMemcpyAsync(hb, dest, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const double rho = 1.1 * hb[0];
  lo = std::max(glo, c - rho);
  hi = std::min(ghi, c + rho);
  if (!(lo < hi)) {
    lo = glo;
    hi = ghi;
  }
}

static double median_of(std::vector<double> v) {
  std::sort(v.begin(), v.end());
  const size_t n = v.size();
  if (n == 0) return 0.0;
  if (n & 1) return v[n / 2];
  return (v[n / 2 - 1] + v[n / 2]) / 2.0;
}

// Shift of an attempt (first: median of the diagonal plus 1% jitter, later:
// uniform in the middle half of [lo, hi], Sec. 3.4), scale s = half-width.
static void choose_shift(const std::vector<double>& diag, double lo, double hi, uint64_t seed,
                         uint64_t node, int attempt, double& sigma, double& scale) {
  const double c = 0.5 * (lo + hi);
  double R = 0.5 * (hi - lo);
  if (R <= 0.0) R = std::max(std::fabs(c), 1.0) * 1e-3;
  const double xi = philox_uniform(seed, PURPOSE_SHIFT, node, attempt);
  if (attempt == 0) sigma = median_of(diag) + 0.01 * R * (2.0 * xi - 1.0);
  else sigma = c + R * (xi - 0.5);
  sigma = std::min(std::max(sigma, lo + 1e-3 * R), hi - 1e-3 * R);
  scale = R;
}

static double flops_irs_iter(double m) { return 22.0 / 3.0 * m * m * m; }
static double flops_grurv(double m) { return 12.0 * m * m * m; }
static double flops_similarity(double m) { return 4.0 * m * m * m; }

__global__ void permute_columns_kernel(int n, const double* __restrict__ U, int ldu,
                                       const int* __restrict__ perm, double* __restrict__ out,
                                       int ldo) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * n) return;
  const int i = (int)(idx % n), j = (int)(idx / n);
  out[i + (size_t)j * ldo] = U[i + (size_t)perm[j] * ldu];
}

// FP64 refinement of a symmetric eigendecomposition (a12): steps of
// Ogita-Aishima with FP64 GEMMs until the Gram and off-diagonal residuals
// reach the FP64 level (at most 4 steps), then Rayleigh quotients.  G, AU, S,
// E are n x n scratch; lam receives the eigenvalues.  Returns flops executed.
static double refine_symmetric(eig_handle_t h, int n, const double* A, int lda, double* U, int ldu,
                               double* lam, double* G, double* AU, double* S, double* E,
                               unsigned long long* dbits, void* tcw, int* tcerr) {
  cudaStream_t s = h->stream;
  // the n x n products on the tensor cores in the FP64-accurate split (error
  // of an FP64 GEMM) where it pays, else on the DFMA kernel
  auto rmm = [&](bool ta, bool tb, int m_, int n_, int k_, double alpha, const double* X, int ldx,
                 const double* Y, int ldy, double beta, double* Z, int ldz) {
    if (tcw && tcx_worth(m_, n_, k_))
      return tcx_gemm(s, ta, tb, m_, n_, k_, alpha, X, ldx, Y, ldy, beta, Z, ldz, tcw, tcerr);
    return gemm(s, ta, tb, m_, n_, k_, alpha, X, ldx, Y, ldy, beta, Z, ldz);
  };
  if (tcerr) CK(cudaMemsetAsync(tcerr, 0, sizeof(int), s));
  double flops = 0.0;
  const double u = 0x1p-53;
  // one pinned staging area: n eigenvalues, then the residual words
  char* pin = static_cast<char*>(pinned(h, sizeof(double) * ((size_t)n + 16) + 64));
  double* hl = reinterpret_cast<double*>(pin);
  unsigned long long* hb = reinterpret_cast<unsigned long long*>(pin + sizeof(double) * ((size_t)n + 8));
  for (int step = 0; step < 6; ++step) {
    CK(rmm(true, false, n, n, n, 1.0, U, ldu, U, ldu, 0.0, G, n));
    CK(rmm(false, false, n, n, n, 1.0, A, lda, U, ldu, 0.0, AU, n));
    CK(rmm(true, false, n, n, n, 1.0, U, ldu, AU, n, 0.0, S, n));
    flops += 6.0 * (double)n * n * n;
    CK(cudaMemsetAsync(dbits, 0, 3 * sizeof(unsigned long long), s));
    CK(oa_diag(s, n, G, S, lam, &dbits[0]));
    CK(oa_offmax(s, n, G, S, &dbits[1]));
    CK(cudaMemcpyAsync(hb, dbits, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double normA, offS, maxR;
    std::memcpy(&normA, &hb[0], 8);
    std::memcpy(&offS, &hb[1], 8);
    std::memcpy(&maxR, &hb[2], 8);
    const char* venv = std::getenv("EIGDC_VERBOSE");
    if (venv && venv[0] == '1')
      std::fprintf(stderr, "[eigdc] refine step %d: |A| %.3e max|S_offdiag| %.3e max|I - U^T U| %.3e\n",
                   step, normA, offS, maxR);
    const double floor_ = 8.0 * std::sqrt((double)n) * u;
    if (offS <= floor_ * normA && maxR <= floor_) break;
    CK(oa_correction(s, n, G, S, lam, 64.0 * u * normA, E));
    CK(rmm(false, false, n, n, n, 1.0, U, ldu, E, n, 0.0, AU, n));
    flops += 2.0 * (double)n * n * n;
    if (ldu == n) {
      CK(add_inplace(s, (size_t)n * n, U, AU));
    } else {
      CK(add_matrices(s, n, n, U, ldu, AU, n, U, ldu));
    }
  }
  // Clusters: pairs the first-order correction leaves coupled are resolved
  // by diagonalising S = U^T A U on each cluster block (cyclic Jacobi).
  // Order U by the current eigenvalue estimates so clusters are contiguous.
  {
    std::vector<double> lv(n);
    CK(cudaMemcpyAsync(hl, lam, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::memcpy(lv.data(), hl, sizeof(double) * n);
    std::vector<int> perm(n);
    for (int i = 0; i < n; ++i) perm[i] = i;
    std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return lv[a] < lv[b]; });
    int* dperm = reinterpret_cast<int*>(E);
    CK(cudaMemcpyAsync(dperm, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s));
    const size_t t = (size_t)n * n;
    note_launches(1);
    permute_columns_kernel<<<(unsigned)((t + 255) / 256), 256, 0, s>>>(n, U, ldu, dperm, G, n);
    CK(cudaGetLastError());
    CK(copy_matrix(s, n, n, G, n, U, ldu));
    CK(rmm(false, false, n, n, n, 1.0, A, lda, U, ldu, 0.0, AU, n));
    CK(rmm(true, false, n, n, n, 1.0, U, ldu, AU, n, 0.0, S, n));
    flops += 4.0 * (double)n * n * n;
    // lam = diag(S) (the radii output is not used)
    CK(diag_gershgorin(s, n, S, n, lam, E));
    CK(cudaMemsetAsync(dbits, 0, 3 * sizeof(unsigned long long), s));
    CK(oa_offmax(s, n, G, S, &dbits[1]));   // max off-diagonal |S| (the G part is unused)
    CK(cudaMemcpyAsync(hb, dbits, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hl, lam, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double offS;
    std::memcpy(&offS, &hb[1], 8);
    std::memcpy(lv.data(), hl, sizeof(double) * n);
    double normA = 0.0;
    for (double x : lv) normA = std::max(normA, std::fabs(x));
    const double dclu = 64.0 * std::max(offS, (double)n * u * normA);
    std::vector<LeafDesc> clusters;
    for (int i = 0; i < n;) {
      int j = i + 1;
      while (j < n && lv[j] - lv[j - 1] <= dclu && j - i < 64) ++j;
      if (j - i >= 2) clusters.push_back(LeafDesc{i, j - i, (int)clusters.size() * 64 * 64});
      i = j;
    }
    // descriptors in AU, the 64 x 64 vector slots in G (both free here),
    // processed in chunks that fit G
    const size_t cap = std::max<size_t>(1, ((size_t)n * n) / 4096);
    for (size_t c0 = 0; c0 < clusters.size(); c0 += cap) {
      const size_t cnt = std::min(cap, clusters.size() - c0);
      std::vector<LeafDesc> chunk(clusters.begin() + c0, clusters.begin() + c0 + cnt);
      for (size_t q = 0; q < cnt; ++q) chunk[q].zoff = (int)(q * 4096);
      LeafDesc* dd = reinterpret_cast<LeafDesc*>(AU);
      CK(cudaMemcpyAsync(dd, chunk.data(), sizeof(LeafDesc) * cnt, cudaMemcpyHostToDevice, s));
      int* dstat = reinterpret_cast<int*>(&dbits[4]);
      CK(cudaMemsetAsync(dstat, 0, sizeof(int), s));
      CK(jacobi_leaves(s, (int)cnt, dd, S, n, lam, G, dstat));
      CK(apply_leaf_vectors(s, (int)cnt, dd, n, U, ldu, U, ldu, G));
      CK(cudaStreamSynchronize(s));
    }
    const char* venv = std::getenv("EIGDC_VERBOSE");
    if (venv && venv[0] == '1')
      std::fprintf(stderr, "[eigdc] refine clusters: %zu (threshold %.3e, max|S_offdiag| %.3e)\n",
                   clusters.size(), dclu, offS);
  }
  // final orthogonalisation without eigen-corrections (no division by gaps,
  // so no amplification of rounding): X <- X + X (I - X^T X) / 2
  CK(rmm(true, false, n, n, n, 1.0, U, ldu, U, ldu, 0.0, G, n));
  CK(oa_correction(s, n, G, S, lam, INFINITY, E));   // every pair takes r_ij / 2
  CK(rmm(false, false, n, n, n, 1.0, U, ldu, E, n, 0.0, AU, n));
  if (ldu == n) CK(add_inplace(s, (size_t)n * n, U, AU));
  else CK(add_matrices(s, n, n, U, ldu, AU, n, U, ldu));
  flops += 4.0 * (double)n * n * n;
  if (tcerr) {
    int* hf = static_cast<int*>(pinned(h, 64));
    CK(cudaMemcpyAsync(hf, tcerr, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (*hf) {
      h->err = "tensor-core GEMM: a bounded wait timed out";
      throw Fail{EIG_ERR_CUDA};
    }
  }
  return flops;
}

// ---------------------------------------------------------------- solve
// Per-node scratch: IRS and splitter work for a node of size m, and the
// n x m panel of U that the node's splitter updates.
struct NodeWork {
  IRSWork irs;
  SplitWork split;
  double* Unode;
  double* dtmp;
  IRSWork irsL;                      // pencils: IRS of (A^T, B^T)
  double* At = nullptr;              // pencils: node's (A^T, B^T)
  double* Bt = nullptr;
};

static size_t carve_node(Arena& a, int n_total, int m, int prec, NodeWork& w,
                         bool pencil = false) {
  const size_t start = a.used;
  carve_irs(a, m, w.irs, prec);
  carve_split(a, m, w.split, prec, pencil);
  w.Unode = a.take<double>((size_t)n_total * m);
  w.dtmp = a.take<double>(2 * (size_t)m + 8);
  if (pencil) {
    carve_irs(a, m, w.irsL, prec);
    w.At = a.take<double>((size_t)m * m);
    w.Bt = a.take<double>((size_t)m * m);
  }
  return a.used - start;
}

// Solve-level buffers (leaves, sorting, Schur assembly, refinement).
struct SolveMain {
  double *Acur, *wtmp, *Zleaf, *dtmp, *sortbuf, *Tbuf, *gpart;
  double *G, *AU, *S, *E;   // refinement scratch (split precision, symmetric)
  void* rtcw = nullptr;      // refinement: digit planes of its n x n x n products
  int* rtcerr = nullptr;
  unsigned long long* bits;
  int* status;
  LeafDesc* ddesc;
  double* Bcur = nullptr;     // pencils: working B
  double* Zleaf2 = nullptr;   // pencils: right leaf vectors
};

static size_t carve_main(Arena& a, int n, bool refine, SolveMain& w, bool pencil = false) {
  const size_t start = a.used;
  const size_t nn = (size_t)n * n;
  if (pencil) {
    w.Bcur = a.take<double>(nn);
    w.Zleaf2 = a.take<double>((size_t)64 * 64 * std::max(1, n));
  }
  w.Acur = a.take<double>(nn);
  w.wtmp = a.take<double>(2 * (size_t)n + 8);
  w.Zleaf = a.take<double>((size_t)64 * 64 * std::max(1, n));
  w.dtmp = a.take<double>(2 * (size_t)n + 8);
  w.sortbuf = a.take<double>(nn);
  w.Tbuf = a.take<double>(nn);
  w.gpart = a.take<double>(square_partial_doubles(n));
  w.G = refine ? a.take<double>(nn) : nullptr;
  w.AU = refine ? a.take<double>(nn) : nullptr;
  w.S = refine ? a.take<double>(nn) : nullptr;
  w.E = refine ? a.take<double>(nn) : nullptr;
  if (refine) {
    w.rtcw = a.take<char>(tc_ws_bytes(EIG_FP64_TC, n, n, n));
    w.rtcerr = a.take<int>(8);
  }
  w.bits = a.take<unsigned long long>(8);
  w.status = a.take<int>(8);
  w.ddesc = a.take<LeafDesc>(std::max(1, n));
  return a.used - start;
}

// State shared by the workers of one solve.
struct SolveShared {
  int n = 0, ldu = 0, leaf = 64;
  bool sym = true, verbose = false;
  // split precision: some accepted split ran at an FP32-level tier, so the
  // eigendecomposition needs the closing FP64 refinement
  bool low_tier = false;
  // symmetric nodes of at most fused_tail rows (0: none) are not processed
  // here but collected for one launch of the fused batched solver
  int fused_tail = 0;
  std::vector<Node> deferred;
  double* Acur = nullptr;
  double* dU = nullptr;        // pencils: Q_L
  bool pencil = false;
  double* Bcur = nullptr;
  double* dQR = nullptr;
  int ldqr = 0;
  eig_params_t p, pp;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Node> queue;
  int outstanding = 0;
  std::vector<LeafDesc> leaves;
  eig_solve_info_t inf;
  int status = EIG_OK;
  std::string err;
};

// One node of the recursion: attempts (shift, IRS, splitter, split test)
// until a split is accepted; then U and the node's diagonal block are
// updated and the two children are queued.  Runs on the worker handle hw;
// `base` points at scratch of carve_node(n, m) bytes.
static void process_node(eig_handle_t hw, SolveShared& S, Node nd, char* base) {
  cudaStream_t s = hw->stream;
  NvtxRange nvtx_("eig.node");
  const int n = S.n, m = nd.m;
  const eig_params_t& p = S.p;
  double* An = S.Acur + nd.off + (size_t)nd.off * n;
  if (m <= S.leaf) {
    std::lock_guard<std::mutex> lock(S.mu);
    S.inf.nodes++;
    S.inf.max_depth = std::max(S.inf.max_depth, nd.depth);
    S.leaves.push_back(LeafDesc{nd.off, m, (int)S.leaves.size() * 64 * 64});
    return;
  }
  if (m <= S.fused_tail) {
    std::lock_guard<std::mutex> lock(S.mu);
    S.deferred.push_back(nd);
    return;
  }
  Arena arena(base);
  NodeWork w;
  carve_node(arena, n, m, p.prec, w);
  const auto t_node = std::chrono::steady_clock::now();
  std::vector<double> diag, hscores;
  const double tau = p.tau > 0 ? p.tau : -1.0;
  int attempt = 0, fails = 0;
  double flops = 0.0;
  int iters = 0, failed = 0;
  // precision tier of this node's attempts: EIG_SPLIT_FP32 starts at the
  // tier its interval can resolve (split_start_tier) and escalates (five
  // digits, then the FP64-accurate split) when an attempt finds a true split
  // it cannot resolve
  int tier = p.prec == EIG_SPLIT_FP32 ? split_start_tier(m, nd.lo, nd.hi) : p.prec;
  while (true) {
    w.irs.prec = w.irs.qr.q.prec = tier;
    w.split.prec = w.split.qr.q.prec = tier;
    eig_region_t rg;
    if (!S.sym && p.root_unit_circle && nd.id == ROOT_NODE && attempt == 0) {
      rg.kind = EIG_REGION_UNIT_CIRCLE;
      rg.c_or_sigma = 0.0;
      rg.r_or_s = 1.0;
    } else {
      node_diag(hw, S.Acur, n, nd.off, m, diag);
      double sigma, sc;
      choose_shift(diag, nd.lo, nd.hi, p.seed, nd.id, attempt, sigma, sc);
      rg.kind = EIG_REGION_LINE;
      rg.c_or_sigma = sigma;
      rg.r_or_s = sc;
    }
    const double tau_m = tau > 0 ? tau : (split_mode(tier) ? 1e-5 : default_tau(m));
    IRSOut ir = run_irs(hw, w.irs, m, An, n, nullptr, 0, rg, tau_m, p.maxit, stall_level(tier),
                        p.graphs != 0);
    iters += ir.iters;
    flops += ir.iters * flops_irs_iter(m);
    eig_params_t pt = S.pp;
    pt.prec = tier;
    SplitOut so = run_split(hw, w.split, m, ir.Ap, ir.Bp, m, An, n, S.sym, nd.id, attempt, pt,
                            ir.converged, hscores);
    flops += (so.draw + 1) * (flops_grurv(m) + flops_similarity(m));
    if (S.verbose)
      std::fprintf(stderr,
                   "[eigdc] node off=%d m=%d depth=%d attempt=%d region=%d (%.6g, %.6g) "
                   "iters=%d conv=%d ratio=%.3g k=%d e=%.3g rank=%d draw=%d accepted=%d "
                   "t=%.4f s\n",
                   nd.off, m, nd.depth, attempt, rg.kind, rg.c_or_sigma, rg.r_or_s, ir.iters,
                   (int)ir.converged, ir.last_ratio, so.k, so.e, so.rank, so.draw,
                   (int)so.accepted,
                   std::chrono::duration<double>(std::chrono::steady_clock::now() - t_node)
                       .count());
    if (so.accepted) {
      const int k = so.k;
      // U[:, off:off+m] <- U[:, off:off+m] Q ; node block <- A^
      CK2(hw, gemm(s, false, false, n, m, m, 1.0, S.dU + (size_t)nd.off * S.ldu, S.ldu,
                   w.split.Ucur, m, 0.0, w.Unode, n));
      CK2(hw, copy_matrix(s, n, m, w.Unode, n, S.dU + (size_t)nd.off * S.ldu, S.ldu));
      flops += 2.0 * n * (double)m * m;
      CK2(hw, copy_matrix(s, m, m, w.split.Ahat, m, An, n));
      double lo1, hi1, lo2, hi2;
      double* A11 = An;
      double* A22 = An + k + (size_t)k * n;
      if (rg.kind == EIG_REGION_LINE) {
        lo1 = rg.c_or_sigma;
        hi1 = nd.hi;
        lo2 = nd.lo;
        hi2 = rg.c_or_sigma;
      } else {
        gershgorin_interval(hw, A11, n, k, w.dtmp, lo1, hi1);
        gershgorin_interval(hw, A22, n, m - k, w.dtmp, lo2, hi2);
      }
      if (!S.sym) {
        double g1l, g1h, g2l, g2h;
        gershgorin_interval(hw, A11, n, k, w.dtmp, g1l, g1h);
        gershgorin_interval(hw, A22, n, m - k, w.dtmp, g2l, g2h);
        lo1 = std::max(lo1, g1l);
        hi1 = std::min(hi1, g1h);
        lo2 = std::max(lo2, g2l);
        hi2 = std::min(hi2, g2h);
        if (lo1 >= hi1) { lo1 = g1l; hi1 = g1h; }
        if (lo2 >= hi2) { lo2 = g2l; hi2 = g2h; }
      }
      CK2(hw, cudaStreamSynchronize(s));   // children may run on other streams
      std::lock_guard<std::mutex> lock(S.mu);
      if (split_mode(tier)) S.low_tier = true;
      S.inf.nodes++;
      S.inf.splits++;
      S.inf.max_depth = std::max(S.inf.max_depth, nd.depth);
      S.inf.total_iters += iters;
      S.inf.failed_attempts += failed;
      S.inf.flops += flops;
      S.queue.push_back(Node{nd.off, k, lo1, hi1, child_node(nd.id, 0), nd.depth + 1});
      S.queue.push_back(Node{nd.off + k, m - k, lo2, hi2, child_node(nd.id, 1), nd.depth + 1});
      S.outstanding += 2;
      S.cv.notify_all();
      return;
    }
    failed++;
    if (p.prec == EIG_SPLIT_FP32 && tier != EIG_FP64_TC && ir.converged && so.rank > 0 &&
        so.rank < m) {
      // a split exists but the tier's products left ||E21|| above the
      // tolerance: the same attempt (shift and draws) one tier up
      tier = (tier == EIG_SPLIT_FP32) ? PREC_SPLIT30 : EIG_FP64_TC;
      if (S.verbose)
        std::fprintf(stderr, "[eigdc] node off=%d m=%d: precision tier %d\n", nd.off, m, tier);
      continue;
    }
    if (rg.kind == EIG_REGION_LINE && ir.converged) {
      if (so.rank == 0) nd.hi = rg.c_or_sigma;
      else if (so.rank == m) nd.lo = rg.c_or_sigma;
      else fails++;
    } else {
      fails++;
    }
    attempt++;
    if (fails > p.max_fail || attempt > 250) {
      std::lock_guard<std::mutex> lock(S.mu);
      S.inf.nodes++;
      S.inf.total_iters += iters;
      S.inf.failed_attempts += failed;
      S.inf.flops += flops;
      if (S.status == EIG_OK) {
        S.status = EIG_NO_SPLIT;
        S.err = "no split found for a node of size " + std::to_string(m);
      }
      return;
    }
  }
}

// One node of the pencil recursion (RGNEP, Algorithm 4; strategy of Sec.
// 3.5).  The root searches circles |z| = r about the origin: r = 1, then
// r <- r^2 from 1/2 while every eigenvalue is inside, or from 2 while every
// one is outside.  A dividing circle splits the node: the inside group keeps
// its orientation, bounded by r; the outside group (leading k) continues as
// the swapped pencil (B, A), bounded by 1/r.  Running past the last circle
// that held everything inside (outside) makes that circle the node's bound
// (swapping in the second case).  Other nodes divide on real lines Re z =
// sigma over [lo, hi] with the empty-side rule of the symmetric strategy.
// A circle whose IRS fails or whose split is rejected is retried with its
// radius times 2^((2 xi - 1)/4); the search stops at 2^(+-512).  Q_L and Q_R
// of an accepted split update the global left / right Schur vectors and the
// node's blocks of (A, B).
static void process_pencil_node(eig_handle_t hw, SolveShared& S, Node nd, char* base) {
  cudaStream_t s = hw->stream;
  NvtxRange nvtx_("eig.pencil_node");
  const int n = S.n, m = nd.m;
  const eig_params_t& p = S.p;
  double* An = S.Acur + nd.off + (size_t)nd.off * n;
  double* Bn = S.Bcur + nd.off + (size_t)nd.off * n;
  if (m <= S.leaf) {
    std::lock_guard<std::mutex> lock(S.mu);
    S.inf.nodes++;
    S.inf.max_depth = std::max(S.inf.max_depth, nd.depth);
    S.leaves.push_back(LeafDesc{nd.off, m, (int)S.leaves.size() * 64 * 64, nd.swapped ? 1 : 0});
    return;
  }
  Arena arena(base);
  NodeWork w;
  carve_node(arena, n, m, p.prec, w, true);
  const double* P = nullptr;
  const double* Qm = nullptr;
  std::vector<double> hscores;
  const double tau = p.tau > 0 ? p.tau : default_tau(m);
  int attempt = 0, fails = 0, iters = 0, failed = 0;
  double flops = 0.0;
  bool circle = nd.id == ROOT_NODE;
  double r = 1.0, r_prev = 0.0, r_try = 1.0;
  int direction = 0;
  auto orient = [&]() {   // (P, Qm) = (A, B) or (B, A), and their transposes
    P = nd.swapped ? Bn : An;
    Qm = nd.swapped ? An : Bn;
    CK2(hw, transpose(s, m, m, P, n, w.At, m));
    CK2(hw, transpose(s, m, m, Qm, n, w.Bt, m));
  };
  orient();
  while (true) {
    eig_region_t rg;
    if (circle) {
      rg.kind = r_try == 1.0 ? EIG_REGION_UNIT_CIRCLE : EIG_REGION_CIRCLE;
      rg.c_or_sigma = 0.0;
      rg.r_or_s = r_try;
    } else {
      const double c = 0.5 * (nd.lo + nd.hi), R = 0.5 * (nd.hi - nd.lo);
      const double xi = philox_uniform(p.seed, PURPOSE_SHIFT, nd.id, attempt);
      rg.kind = EIG_REGION_LINE;
      rg.c_or_sigma = c + R * (xi - 0.5);
      rg.r_or_s = R;
    }
    const double stall = p.tau > 0 ? 0.0 : stall_level(p.prec);
    IRSOut ir = run_irs(hw, w.irs, m, P, n, Qm, n, rg, tau, p.maxit, stall, p.graphs != 0);
    IRSOut il = run_irs(hw, w.irsL, m, w.At, m, w.Bt, m, rg, tau, p.maxit, stall, p.graphs != 0);
    iters += ir.iters;
    flops += (ir.iters + il.iters) * flops_irs_iter(m);
    SplitOut so = run_split_pencil(hw, w.split, m, ir.Ap, ir.Bp, il.Ap, il.Bp, m, P, n, Qm, n,
                                   nd.id, attempt, S.pp, ir.converged, il.converged, hscores);
    flops += (so.draw + 1) * 2.0 * (flops_grurv(m) + flops_similarity(m));
    if (S.verbose)
      std::fprintf(stderr,
                   "[eigdc] pencil node off=%d m=%d depth=%d swapped=%d attempt=%d region=%d "
                   "(%.6g, %.6g) iters=%d/%d conv=%d/%d k=%d e=%.3g rank=%d draw=%d accepted=%d\n",
                   nd.off, m, nd.depth, (int)nd.swapped, attempt, rg.kind, rg.c_or_sigma,
                   rg.r_or_s, ir.iters, il.iters, (int)ir.converged, (int)il.converged, so.k,
                   so.e, so.rank, so.draw, (int)so.accepted);
    if (so.accepted) {
      const int k = so.k;
      CK2(hw, gemm(s, false, false, n, m, m, 1.0, S.dU + (size_t)nd.off * S.ldu, S.ldu,
                   w.split.QLn, m, 0.0, w.Unode, n));
      CK2(hw, copy_matrix(s, n, m, w.Unode, n, S.dU + (size_t)nd.off * S.ldu, S.ldu));
      CK2(hw, gemm(s, false, false, n, m, m, 1.0, S.dQR + (size_t)nd.off * S.ldqr, S.ldqr,
                   w.split.Ucur, m, 0.0, w.Unode, n));
      CK2(hw, copy_matrix(s, n, m, w.Unode, n, S.dQR + (size_t)nd.off * S.ldqr, S.ldqr));
      flops += 4.0 * n * (double)m * m;
      // the split was computed on (P, Qm); write it back in (A, B) order
      CK2(hw, copy_matrix(s, m, m, w.split.Ahat, m, nd.swapped ? Bn : An, n));
      CK2(hw, copy_matrix(s, m, m, w.split.Bhat, m, nd.swapped ? An : Bn, n));
      double lo1, hi1, lo2, hi2;
      bool sw1, sw2;
      if (circle) {
        const double rr = rg.r_or_s;
        lo1 = -1.0 / rr;
        hi1 = 1.0 / rr;
        lo2 = -rr;
        hi2 = rr;
        sw1 = !nd.swapped;
        sw2 = nd.swapped;
      } else {
        lo1 = rg.c_or_sigma;
        hi1 = nd.hi;
        lo2 = nd.lo;
        hi2 = rg.c_or_sigma;
        sw1 = sw2 = nd.swapped;
      }
      CK2(hw, cudaStreamSynchronize(s));   // children may run on other streams
      std::lock_guard<std::mutex> lock(S.mu);
      S.inf.nodes++;
      S.inf.splits++;
      S.inf.max_depth = std::max(S.inf.max_depth, nd.depth);
      S.inf.total_iters += iters;
      S.inf.failed_attempts += failed;
      S.inf.flops += flops;
      S.queue.push_back(Node{nd.off, k, lo1, hi1, child_node(nd.id, 0), nd.depth + 1, sw1});
      S.queue.push_back(Node{nd.off + k, m - k, lo2, hi2, child_node(nd.id, 1), nd.depth + 1, sw2});
      S.outstanding += 2;
      S.cv.notify_all();
      return;
    }
    failed++;
    const bool empty = ir.converged && (so.rank == 0 || so.rank == m);
    if (circle && empty) {
      const bool inside = so.rank == 0;
      if (inside && direction > 0) {
        // everything outside r_prev and inside r: bounded once swapped
        nd.swapped = !nd.swapped;
        nd.lo = -1.0 / r_prev;
        nd.hi = 1.0 / r_prev;
        circle = false;
        orient();
      } else if (!inside && direction < 0) {
        nd.lo = -r_prev;   // everything inside r_prev and outside r
        nd.hi = r_prev;
        circle = false;
      } else {
        direction = inside ? -1 : 1;
        r_prev = r;
        r = (r == 1.0) ? (inside ? 0.5 : 2.0) : r * r;
        if (std::fabs(std::log2(r)) > 512.0) {
          if (inside) {
            nd.lo = -r_prev;
            nd.hi = r_prev;
          } else {
            nd.swapped = !nd.swapped;
            nd.lo = -1.0 / r_prev;
            nd.hi = 1.0 / r_prev;
            orient();
          }
          circle = false;
        }
      }
      r_try = r;
    } else if (circle) {
      fails++;
      const double xi = philox_uniform(p.seed, PURPOSE_SHIFT, nd.id, attempt);
      r_try = r * std::exp2(0.25 * (2.0 * xi - 1.0));
    } else if (rg.kind == EIG_REGION_LINE && empty) {
      if (so.rank == 0) nd.hi = rg.c_or_sigma;
      else nd.lo = rg.c_or_sigma;
    } else {
      fails++;
    }
    attempt++;
    if (fails > p.max_fail || attempt > 250) {
      std::lock_guard<std::mutex> lock(S.mu);
      S.inf.nodes++;
      S.inf.total_iters += iters;
      S.inf.failed_attempts += failed;
      S.inf.flops += flops;
      if (S.status == EIG_OK) {
        S.status = EIG_NO_SPLIT;
        S.err = "no split found for a pencil node of size " + std::to_string(m);
      }
      return;
    }
  }
}

// Worker loop: take nodes until the tree is finished or a node failed.
// With own_ws the node scratch is grown in hw's workspace per node; else
// `fixed_base` (carved for the root size) is used.
static void worker_loop(eig_handle_t hw, SolveShared& S, bool own_ws, char* fixed_base) {
  if (cudaSetDevice(hw->device) != cudaSuccess) {
    std::lock_guard<std::mutex> lock(S.mu);
    if (S.status == EIG_OK) { S.status = EIG_ERR_CUDA; S.err = "cudaSetDevice failed"; }
    S.cv.notify_all();
    return;
  }
  while (true) {
    Node nd;
    {
      std::unique_lock<std::mutex> lock(S.mu);
      S.cv.wait(lock, [&] { return !S.queue.empty() || S.outstanding == 0 || S.status != EIG_OK; });
      if (S.status != EIG_OK || S.queue.empty()) return;
      nd = S.queue.front();
      S.queue.pop_front();
    }
    try {
      char* base = fixed_base;
      if (own_ws && nd.m > S.leaf) {
        Arena meas(nullptr);
        NodeWork tmp;
        ensure_ws(hw, carve_node(meas, S.n, nd.m, S.p.prec, tmp, S.pencil));
        base = hw->ws;
      }
      if (S.pencil) process_pencil_node(hw, S, nd, base);
      else process_node(hw, S, nd, base);
    } catch (Fail f) {
      std::lock_guard<std::mutex> lock(S.mu);
      if (S.status == EIG_OK) {
        S.status = f.code;
        S.err = hw->err;
      }
    }
    std::lock_guard<std::mutex> lock(S.mu);
    S.outstanding--;
    S.cv.notify_all();
  }
}

static void ensure_workers(eig_handle_t h, int count) {
  while ((int)h->workers.size() < count) {
    eig_handle_t w = new eig_handle_s();
    w->device = h->device;
    if (cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete w;
      h->err = "cudaStreamCreate failed";
      throw Fail{EIG_ERR_CUDA};
    }
    h->workers.push_back(w);
  }
}

size_t fused_run_bytes(eig_handle_t h, int count, int mx, int cps, int* ctas_out);
void fused_run(eig_handle_t h, int count, const int* n, double* const* dA, const int* lda,
               double* const* dw, double* const* dU, const int* ldu, const eig_params_t& p,
               int nb, int cps, int* status, eig_solve_info_t* infos, float* ms,
               const FusedProblem* nodes = nullptr);

// The fused tail of a symmetric solve: every deferred node (at most
// fused_tail rows) is finished by one launch of the fused batched solver on a
// worker handle -- each node's whole sub-recursion in one CTA, continuing the
// node's id, interval and depth, so the tree is the one eig_solve would
// build -- then U[:, off:off+m] <- U[:, off:off+m] Z for each node's
// eigenvectors Z.  Eigenvalues land in wtmp[off..off+m).
static void run_fused_tail(eig_handle_t h, SolveShared& S, double* wtmp, double* dU, int ldu,
                           eig_solve_info_t& inf, int& status) {
  const int cnt = (int)S.deferred.size();
  const int n = S.n;
  // the recursion's last launches (single-worker mode: on h's stream) must
  // have finished before another stream reads the node blocks
  CK(cudaStreamSynchronize(h->stream));
  ensure_workers(h, 1);
  eig_handle_t hw = h->workers[0];
  CK(cudaSetDevice(hw->device));
  std::vector<int> ns(cnt), lds(cnt, n), ldz(cnt), st(cnt);
  std::vector<double*> A(cnt), W(cnt), Z(cnt);
  std::vector<FusedProblem> roots(cnt);
  std::vector<eig_solve_info_t> infos(cnt);
  std::vector<size_t> zoff(cnt);
  size_t zsize = 0;
  int mmax = 1;
  for (int i = 0; i < cnt; ++i) {
    const Node& nd = S.deferred[i];
    ns[i] = nd.m;
    ldz[i] = nd.m;
    A[i] = S.Acur + nd.off + (size_t)nd.off * n;
    W[i] = wtmp + nd.off;
    zoff[i] = zsize;
    zsize += (size_t)nd.m * nd.m;
    mmax = std::max(mmax, nd.m);
    roots[i] = FusedProblem{};
    roots[i].id = nd.id;
    roots[i].lo = nd.lo;
    roots[i].hi = nd.hi;
    roots[i].depth = nd.depth;
    roots[i].has_interval = 1;
  }
  const size_t fb = round_up(fused_run_bytes(hw, cnt, mmax, h->fused_cps, nullptr));
  const size_t zb = round_up(sizeof(double) * zsize);
  ensure_ws(hw, fb + zb + sizeof(double) * (size_t)n * mmax);
  double* zbase = reinterpret_cast<double*>(hw->ws + fb);
  double* tmp = reinterpret_cast<double*>(hw->ws + fb + zb);
  for (int i = 0; i < cnt; ++i) Z[i] = zbase + zoff[i];
  fused_run(hw, cnt, ns.data(), A.data(), lds.data(), W.data(), Z.data(), ldz.data(), S.p,
            h->fused_nb, h->fused_cps, st.data(), infos.data(), nullptr, roots.data());
  cudaStream_t s = hw->stream;
  for (int i = 0; i < cnt; ++i) {
    const Node& nd = S.deferred[i];
    const int m = nd.m;
    CK(gemm(s, false, false, n, m, m, 1.0, dU + (size_t)nd.off * ldu, ldu, Z[i], m, 0.0, tmp,
            n));
    CK(copy_matrix(s, n, m, tmp, n, dU + (size_t)nd.off * ldu, ldu));
    const eig_solve_info_t& r = infos[i];
    if (r.status != EIG_OK && status == EIG_OK) {
      status = r.status;
      h->err = r.status == EIG_NO_SPLIT ? "no split found for a node (fused tail)"
                                        : "a node of the fused tail failed";
    }
    inf.nodes += r.nodes;
    inf.splits += r.splits;
    inf.max_depth = std::max(inf.max_depth, r.max_depth);
    inf.total_iters += r.total_iters;
    inf.failed_attempts += r.failed_attempts;
    inf.leaves += r.leaves;
    inf.flops += r.flops + 2.0 * n * (double)m * m;
  }
  CK(cudaStreamSynchronize(s));
  CK(cudaSetDevice(h->device));
}

static int solve_impl(eig_handle_t h, int kind, int n, double* dA, int lda, double* dwr,
                      double* dwi, double* dU, int ldu, const eig_params_t& p,
                      eig_solve_info_t* info) {
  cudaStream_t s = h->stream;
  NvtxRange nvtx_("eig.solve");
  const bool sym = (kind == EIG_KIND_SYM);
  const bool refine = sym && split_mode(p.prec);
  const int nworkers = std::max(1, std::min(p.workers, 32));
  const char* venv = std::getenv("EIGDC_VERBOSE");
  // scratch: solve-level buffers, plus (single worker) the node scratch for
  // the root size right behind them
  Arena meas(nullptr);
  SolveMain w;
  NodeWork nw;
  carve_main(meas, n, refine, w);
  const size_t main_bytes = meas.used;
  if (nworkers == 1) carve_node(meas, n, n, p.prec, nw);
  ensure_ws(h, meas.used);
  Arena arena(h->ws);
  carve_main(arena, n, refine, w);
  char* node_base = h->ws + main_bytes;
  SolveShared S;
  S.n = n;
  S.ldu = ldu;
  S.leaf = std::max(1, std::min(64, p.leaf_size));
  S.sym = sym;
  S.verbose = venv && venv[0] == '1';
  S.Acur = w.Acur;
  S.dU = dU;
  S.p = p;
  S.fused_tail = (sym && p.fused_tail > S.leaf) ? std::min(p.fused_tail, fused_max_n()) : 0;
  // split precision: FP32-level iterates, so the R-test and the split test
  // are read at that level; the FP64 refinement at the end restores accuracy
  S.pp = p;
  std::memset(&S.inf, 0, sizeof(S.inf));
  // working copy of A; global U = I
  CK(copy_matrix(s, n, n, dA, lda, w.Acur, n));
  CK(fill_identity_block(s, n, n, dU, ldu, 0));
  CK(cudaMemsetAsync(w.status, 0, 8 * sizeof(int), s));
  CK(nonfinite_check(s, n, n, dA, lda, w.status + 2));
  {
    int* hf = static_cast<int*>(pinned(h, 64));
    CK(cudaMemcpyAsync(hf, w.status + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (*hf) {
      h->err = "input contains NaN or Inf";
      S.inf.status = EIG_NONFINITE;
      if (info) *info = S.inf;
      return EIG_NONFINITE;
    }
  }
  double lo0, hi0;
  if (sym && n > S.leaf)
    spectral_interval(h, w.Acur, n, n, w.dtmp, w.wtmp, w.wtmp + n, p.seed, lo0, hi0);
  else
    gershgorin_interval(h, w.Acur, n, n, w.dtmp, lo0, hi0);
  CK(cudaStreamSynchronize(s));
  S.queue.push_back(Node{0, n, lo0, hi0, ROOT_NODE, 0});
  S.outstanding = 1;
  if (nworkers == 1) {
    worker_loop(h, S, false, node_base);
  } else {
    ensure_workers(h, nworkers);
    std::vector<std::thread> threads;
    for (int i = 0; i < nworkers; ++i)
      threads.emplace_back(worker_loop, h->workers[i], std::ref(S), true, nullptr);
    for (auto& t : threads) t.join();
    CK(cudaSetDevice(h->device));
    // a worker that stopped on an error may have left launches in flight
    for (int i = 0; i < nworkers; ++i) CK(cudaStreamSynchronize(h->workers[i]->stream));
  }
  int status = S.status;
  eig_solve_info_t inf = S.inf;
  if (status != EIG_OK) h->err = S.err;
  if (status == EIG_OK) {
    std::vector<LeafDesc>& leaves = S.leaves;
    inf.leaves = (int)leaves.size();
    if (!S.deferred.empty()) run_fused_tail(h, S, w.wtmp, dU, ldu, inf, status);
    NvtxRange nvtx_leaves("eig.leaves");
    CK(cudaMemcpyAsync(w.ddesc, leaves.data(), sizeof(LeafDesc) * leaves.size(),
                       cudaMemcpyHostToDevice, s));
    if (sym) {
      CK(jacobi_leaves(s, (int)leaves.size(), w.ddesc, w.Acur, n, w.wtmp, w.Zleaf, w.status));
    } else {
      CK(francis_leaves(s, (int)leaves.size(), w.ddesc, w.Acur, n, dwr, dwi, w.Zleaf, w.status));
    }
    CK(apply_leaf_vectors(s, (int)leaves.size(), w.ddesc, n, dU, ldu, dU, ldu, w.Zleaf));
    int* hs = static_cast<int*>(pinned(h, 64));
    CK(cudaMemcpyAsync(hs, w.status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hs[0]) {
      status = EIG_NO_CONVERGENCE;
      h->err = "a leaf solver did not converge";
    }
    if (refine && S.low_tier) {
      inf.flops += refine_symmetric(h, n, dA, lda, dU, ldu, w.wtmp, w.G, w.AU, w.S, w.E, w.bits,
                                  w.rtcw, w.rtcerr);
    }
    if (sym) {
      // eigenvalues ascending with their vectors
      std::vector<double> wv(n);
      double* hb = static_cast<double*>(pinned(h, sizeof(double) * (n + 8)));
      CK(cudaMemcpyAsync(hb, w.wtmp, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      std::memcpy(wv.data(), hb, sizeof(double) * n);
      std::vector<int> perm(n);
      for (int i = 0; i < n; ++i) perm[i] = i;
      std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return wv[a] < wv[b]; });
      std::vector<double> ws(n);
      for (int i = 0; i < n; ++i) ws[i] = wv[perm[i]];
      int* dperm = reinterpret_cast<int*>(w.dtmp);
      CK(cudaMemcpyAsync(dperm, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s));
      CK(cudaMemcpyAsync(dwr, ws.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
      const size_t t = (size_t)n * n;
      if (t) {
        note_launches(1);
        permute_columns_kernel<<<(unsigned)((t + 255) / 256), 256, 0, s>>>(n, dU, ldu, dperm, w.sortbuf, n);
        CK(cudaGetLastError());
      }
      CK(copy_matrix(s, n, n, w.sortbuf, n, dU, ldu));
      CK(copy_matrix(s, n, n, w.Acur, n, dA, lda));
      CK(cudaStreamSynchronize(s));
    } else {
      // T = U^T A U with the quasi-triangular pattern of the leaves
      const int gs = gemm_choose_splits(n, n, n);
      CK(gemm(s, false, false, n, n, n, 1.0, dA, lda, dU, ldu, 0.0, w.Tbuf, n, gs, w.gpart));
      CK(gemm(s, true, false, n, n, n, 1.0, dU, ldu, w.Tbuf, n, 0.0, w.sortbuf, n, gs, w.gpart));
      inf.flops += 4.0 * (double)n * n * n;
      CK(zero_lower_quasi(s, n, w.sortbuf, n, dwi));
      CK(copy_matrix(s, n, n, w.sortbuf, n, dA, lda));
      CK(cudaStreamSynchronize(s));
    }
  }
  inf.status = status;
  if (info) *info = inf;
  return status;
}

// Generalized real Schur form of a regular pencil (A, B) by the RGNEP
// recursion (Algorithm 4, Sec. 3.5) and small-pencil leaves (M = A B^{-1},
// Francis on M, RQ of Q_L^T B).  On exit dA <- S = Q_L^T A Q_R
// (quasi-upper-triangular), dB <- T = Q_L^T B Q_R (upper), (ar, ai, be) the
// eigenvalues (ar + i ai) / be in block order.
static int pencil_impl(eig_handle_t h, int n, double* dA, int lda, double* dB, int ldb,
                       double* dQL, int ldql, double* dQR, int ldqr, double* dar, double* dai,
                       double* dbe, const eig_params_t& p, eig_solve_info_t* info) {
  cudaStream_t s = h->stream;
  NvtxRange nvtx_("eig.pencil_solve");
  const int nworkers = std::max(1, std::min(p.workers, 32));
  const char* venv = std::getenv("EIGDC_VERBOSE");
  Arena meas(nullptr);
  SolveMain w;
  NodeWork nw;
  carve_main(meas, n, false, w, true);
  const size_t main_bytes = meas.used;
  if (nworkers == 1) carve_node(meas, n, n, p.prec, nw, true);
  ensure_ws(h, meas.used);
  Arena arena(h->ws);
  carve_main(arena, n, false, w, true);
  char* node_base = h->ws + main_bytes;
  SolveShared S;
  S.n = n;
  S.ldu = ldql;
  S.leaf = std::max(1, std::min(64, p.leaf_size));
  S.sym = false;
  S.pencil = true;
  S.verbose = venv && venv[0] == '1';
  S.Acur = w.Acur;
  S.Bcur = w.Bcur;
  S.dU = dQL;
  S.dQR = dQR;
  S.ldqr = ldqr;
  S.p = p;
  S.pp = p;
  std::memset(&S.inf, 0, sizeof(S.inf));
  CK(copy_matrix(s, n, n, dA, lda, w.Acur, n));
  CK(copy_matrix(s, n, n, dB, ldb, w.Bcur, n));
  CK(fill_identity_block(s, n, n, dQL, ldql, 0));
  CK(fill_identity_block(s, n, n, dQR, ldqr, 0));
  CK(cudaMemsetAsync(w.status, 0, 8 * sizeof(int), s));
  CK(nonfinite_check(s, n, n, dA, lda, w.status + 2));
  CK(nonfinite_check(s, n, n, dB, ldb, w.status + 2));
  {
    int* hf = static_cast<int*>(pinned(h, 64));
    CK(cudaMemcpyAsync(hf, w.status + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (*hf) {
      h->err = "input contains NaN or Inf";
      S.inf.status = EIG_NONFINITE;
      if (info) *info = S.inf;
      return EIG_NONFINITE;
    }
  }
  S.queue.push_back(Node{0, n, -1.0, 1.0, ROOT_NODE, 0, false});
  S.outstanding = 1;
  if (nworkers == 1) {
    worker_loop(h, S, false, node_base);
  } else {
    ensure_workers(h, nworkers);
    std::vector<std::thread> threads;
    for (int i = 0; i < nworkers; ++i)
      threads.emplace_back(worker_loop, h->workers[i], std::ref(S), true, nullptr);
    for (auto& t : threads) t.join();
    CK(cudaSetDevice(h->device));
    // a worker that stopped on an error may have left launches in flight
    for (int i = 0; i < nworkers; ++i) CK(cudaStreamSynchronize(h->workers[i]->stream));
  }
  int status = S.status;
  eig_solve_info_t inf = S.inf;
  if (status != EIG_OK) h->err = S.err;
  if (status == EIG_OK) {
    std::vector<LeafDesc>& leaves = S.leaves;
    const int nl = (int)leaves.size();
    inf.leaves = nl;
    NvtxRange nvtx_leaves("eig.pencil_leaves");
    double* wr = w.wtmp;
    double* wi = w.wtmp + n;
    double* M = w.Tbuf;   // leaves' M = A B^{-1} in the diagonal blocks
    CK(cudaMemcpyAsync(w.ddesc, leaves.data(), sizeof(LeafDesc) * nl, cudaMemcpyHostToDevice, s));
    CK(pencil_leaves_phase1(s, nl, w.ddesc, w.Acur, w.Bcur, n, M, w.status));
    CK(francis_leaves(s, nl, w.ddesc, M, n, wr, wi, w.Zleaf, w.status));
    CK(pencil_leaves_phase2(s, nl, w.ddesc, w.Acur, w.Bcur, n, wi, w.Zleaf, w.Zleaf2));
    CK(apply_leaf_vectors(s, nl, w.ddesc, n, dQL, ldql, dQL, ldql, w.Zleaf));
    CK(apply_leaf_vectors(s, nl, w.ddesc, n, dQR, ldqr, dQR, ldqr, w.Zleaf2));
    int* hs = static_cast<int*>(pinned(h, 64));
    CK(cudaMemcpyAsync(hs, w.status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hs[0] & 2) {
      status = EIG_NEAR_SINGULAR_PENCIL;
      h->err = "a leaf pencil has a near-singular B (max/min |r_ii| > 1e8)";
    } else if (hs[0]) {
      status = EIG_NO_CONVERGENCE;
      h->err = "a leaf solver did not converge";
    }
    // S = Q_L^T A Q_R, T = Q_L^T B Q_R with the leaves' zero patterns
    const int gs = gemm_choose_splits(n, n, n);
    CK(gemm(s, false, false, n, n, n, 1.0, dA, lda, dQR, ldqr, 0.0, w.Tbuf, n, gs, w.gpart));
    CK(gemm(s, true, false, n, n, n, 1.0, dQL, ldql, w.Tbuf, n, 0.0, dA, lda, gs, w.gpart));
    CK(gemm(s, false, false, n, n, n, 1.0, dB, ldb, dQR, ldqr, 0.0, w.Tbuf, n, gs, w.gpart));
    CK(gemm(s, true, false, n, n, n, 1.0, dQL, ldql, w.Tbuf, n, 0.0, dB, ldb, gs, w.gpart));
    inf.flops += 8.0 * (double)n * n * n;
    {
      // 2 x 2 blocks of real generalized eigenvalues become 1 x 1 blocks
      int* hfl = static_cast<int*>(pinned(h, 64));
      CK(pencil_split_real_pairs(s, n, dA, lda, dB, ldb, dQL, ldql, dQR, ldqr, wi, w.sortbuf,
                                 reinterpret_cast<int*>(w.Zleaf2), w.status + 4, hfl));
    }
    CK(zero_lower_quasi(s, n, dA, lda, wi));
    CK(upper_triangle(s, n, dB, ldb, dB, ldb));
    CK(pencil_alpha_beta(s, n, dA, lda, dB, ldb, wi, dar, dai, dbe));
    CK(cudaStreamSynchronize(s));
  }
  inf.status = status;
  if (info) *info = inf;
  return status;
}

static void check_params(eig_handle_t h, const eig_params_t& p) {
  if (p.maxit < 0 || p.leaf_size < 1 || p.v_draws < 1 || p.max_fail < 0 || p.split_tol < 0 ||
      p.fused_tail < 0 || !valid_prec(p.prec)) {
    h->err = "invalid eig_params_t";
    throw Fail{EIG_ERR_ARG};
  }
}

static eig_params_t params_or_default(const eig_params_t* p) {
  eig_params_t q;
  eig_default_params(&q);
  return p ? *p : q;
}

}  // namespace

// Host helpers shared with the complex-plane driver (cplane.cu).
void eigdc::philox_pair_host(uint64_t seed, int purpose, uint64_t stream, int attempt, double* u1,
                             double* u2) {
  uint32_t c[4] = {0u, ((uint32_t)(attempt & 0xFF) << 8) | ((uint32_t)(purpose & 0xFFFF) << 16),
                   (uint32_t)(stream & 0xFFFFFFFFull), (uint32_t)(stream >> 32)};
  philox_host(c, (uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32));
  const uint64_t m1 = ((uint64_t)c[0] << 20) | (c[1] >> 12);
  const uint64_t m2 = ((uint64_t)c[2] << 20) | (c[3] >> 12);
  *u1 = ((double)m1 + 0.5) * 0x1p-52;
  *u2 = (double)m2 * 0x1p-52;
}

uint64_t eigdc::child_node_id(uint64_t parent, int side) { return child_node(parent, side); }

int eigdc::choose_k_host(const double* e, int n) { return choose_k(e, n); }

// =================================================================== C-ABI
extern "C" {

int eig_debug_fail_allocations(int count) {
  if (count < 0) return EIG_ERR_ARG;
  return g_fail_allocs.exchange(count);
}

void eig_default_params(eig_params_t* p) {
  if (!p) return;
  p->tau = 0.0;
  p->maxit = 60;
  p->split_tol = 0.0;
  p->leaf_size = 64;
  p->prec = EIG_FP64;
  p->seed = 0;
  p->max_fail = 8;
  p->nb = 0;
  p->v_draws = 4;
  p->root_unit_circle = 1;
  p->workers = 8;
  p->graphs = 0;
  p->fused_tail = 0;
}

int eig_create(eig_handle_t* out, int device, void* stream) {
  if (!out) return EIG_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return EIG_ERR_CUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return EIG_ERR_CUDA;
  eig_handle_t h = new eig_handle_s();
  h->device = device;
  h->stream = static_cast<cudaStream_t>(stream);
  panel_init();
  *out = h;
  return EIG_OK;
}

int eig_destroy(eig_handle_t h) {
  if (!h) return EIG_ERR_ARG;
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  for (eig_handle_s* w : h->workers) {
    cudaStreamSynchronize(w->stream);
    if (w->ws) cudaFree(w->ws);
    if (w->pinned) cudaFreeHost(w->pinned);
    clear_graphs(w);
    cudaStreamDestroy(w->stream);
    delete w;
  }
  clear_graphs(h);
  if (h->ws) cudaFree(h->ws);
  if (h->aux) cudaFree(h->aux);
  if (h->lastR) cudaFree(h->lastR);
  if (h->pinned) cudaFreeHost(h->pinned);
  delete h;
  return EIG_OK;
}

const char* eig_last_error(eig_handle_t h) { return h ? h->err.c_str() : "null handle"; }

unsigned long long eig_kernel_launches(void) { return g_launches.load(); }

int eig_gemm_timing(int enable, double* total_ms, unsigned long long* launches, double* flops) {
  if (enable) {
    gemm_timing_start();
    return EIG_OK;
  }
  return gemm_timing_stop(total_ms, launches, flops) == cudaSuccess ? EIG_OK : EIG_ERR_CUDA;
}

int eig_kernel_timing(int family, double* total_ms, unsigned long long* launches, double* work) {
  if (family < 0 || family >= TIMING_FAMILIES) return EIG_ERR_ARG;
  timing_family(family, total_ms, launches, work);
  return EIG_OK;
}

int eig_workspace_size(eig_handle_t h, int n, int kind, size_t* bytes) {
  if (!h || !bytes || n < 0) return EIG_ERR_ARG;
  if (kind == EIG_KIND_CPLANE) {   // stream-ordered allocations of one worker, not the handle's
    *bytes = cplane_footprint(n, EIG_FP64_TC);
    return EIG_OK;
  }
  Arena a(nullptr);
  SolveMain w;
  NodeWork nw;
  const bool pencil = (kind == EIG_KIND_PENCIL);
  carve_main(a, n, true, w, pencil);
  // the largest node scratch over the precision modes
  Arena b1(nullptr), b2(nullptr), b3(nullptr);
  NodeWork nw2, nw3;
  carve_node(b1, n, n, EIG_SPLIT_BF16X3, nw, pencil);
  carve_node(b2, n, n, EIG_FP64_TC, nw2, pencil);
  carve_node(b3, n, n, EIG_SPLIT_FP32, nw3, pencil);
  a.used += std::max(std::max(b1.used, b2.used), b3.used);
  *bytes = a.used;
  return EIG_OK;
}

#define API_BEGIN                   \
  if (!h) return EIG_ERR_ARG;       \
  h->err.clear();                   \
  try {                             \
    if (cudaSetDevice(h->device) != cudaSuccess) { h->err = "cudaSetDevice failed"; return EIG_ERR_CUDA; }
#define API_END                     \
  }                                 \
  catch (Fail f) {                  \
    return f.code;                  \
  }

#define REQUIRE(cond, msg)          \
  do {                              \
    if (!(cond)) {                  \
      h->err = msg;                 \
      return EIG_ERR_ARG;           \
    }                               \
  } while (0)

int eig_divide_step(eig_handle_t h, int n, double* dA, int lda, double* dB, int ldb,
                    const eig_region_t* region, const eig_params_t* params,
                    eig_step_info_t* info) {
  API_BEGIN
  REQUIRE(n >= 1, "n must be >= 1");
  REQUIRE(dA && lda >= n, "dA / lda invalid");
  REQUIRE(!dB || ldb >= n, "ldb invalid");
  REQUIRE(region, "region is NULL");
  REQUIRE(region->kind >= 0 && region->kind <= 2, "unknown region kind");
  REQUIRE(region->kind != EIG_REGION_LINE || region->r_or_s > 0, "line scale must be > 0");
  const eig_params_t p = params_or_default(params);
  check_params(h, p);
  Arena meas(nullptr);
  IRSWork w;
  ensure_ws(h, carve_irs(meas, n, w, p.prec));
  Arena a(h->ws);
  carve_irs(a, n, w, p.prec);
  const double tau = p.tau > 0 ? p.tau
                               : (p.tau < 0 ? -1.0 : (split_mode(p.prec) ? 1e-5 : default_tau(n)));
  IRSOut o = run_irs(h, w, n, dA, lda, dB, ldb, *region, tau, p.maxit,
                     p.tau >= 0 ? stall_level(p.prec) : 0.0);
  cudaStream_t s = h->stream;
  CK(copy_matrix(s, n, n, o.Ap, n, dA, lda));
  if (dB) CK(copy_matrix(s, n, n, o.Bp, n, dB, ldb));
  if (h->lastR_n < n) {
    if (h->lastR) cudaFree(h->lastR);
    h->lastR = nullptr;
    if (cudaMalloc(&h->lastR, sizeof(double) * (size_t)n * n) != cudaSuccess) {
      cudaGetLastError();
      h->lastR_n = 0;
      h->err = "allocation for R failed";
      return EIG_ERR_NOMEM;
    }
    h->lastR_n = n;
  }
  CK(copy_matrix(s, n, n, o.Rlast, n, h->lastR, n));
  CK(cudaMemsetAsync(w.flag, 0, sizeof(int), s));
  CK(nonfinite_check(s, n, n, o.Ap, n, w.flag));
  CK(nonfinite_check(s, n, n, o.Bp, n, w.flag));
  int* hf = static_cast<int*>(pinned(h, 64));
  CK(cudaMemcpyAsync(hf, w.flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->iters = o.iters;
    info->last_ratio = o.last_ratio;
    info->converged = o.converged ? 1 : 0;
  }
  if (*hf) {
    h->err = "non-finite iterate";
    return EIG_NONFINITE;
  }
  if (!o.converged) {
    h->err = "IRS did not converge within maxit";
    return EIG_NO_CONVERGENCE;
  }
  return EIG_OK;
  API_END
}

int eig_last_R(eig_handle_t h, int n, double* dR, int ldr) {
  API_BEGIN
  REQUIRE(dR && ldr >= n && n >= 1, "dR / ldr invalid");
  REQUIRE(h->lastR && h->lastR_n >= n, "no R of this size recorded");
  CK(copy_matrix(h->stream, n, n, h->lastR, n, dR, ldr));
  CK(cudaStreamSynchronize(h->stream));
  return EIG_OK;
  API_END
}

int eig_split(eig_handle_t h, int n, const double* dAp, const double* dBp, int ldp, double* dA,
              int lda, double* dQ, int ldq, int symmetric, uint64_t stream, int attempt,
              const eig_params_t* params, eig_step_info_t* info) {
  API_BEGIN
  REQUIRE(n >= 1, "n must be >= 1");
  REQUIRE(dAp && dBp && ldp >= n, "dAp / dBp / ldp invalid");
  REQUIRE(dA && lda >= n, "dA / lda invalid");
  REQUIRE(dQ && ldq >= n, "dQ / ldq invalid");
  const eig_params_t p = params_or_default(params);
  check_params(h, p);
  Arena meas(nullptr);
  SplitWork w;
  ensure_ws(h, carve_split(meas, n, w, p.prec));
  Arena a(h->ws);
  carve_split(a, n, w, p.prec);
  std::vector<double> hs;
  SplitOut so = run_split(h, w, n, dAp, dBp, ldp, dA, lda, symmetric != 0, stream, attempt, p,
                          true, hs);
  cudaStream_t s = h->stream;
  CK(copy_matrix(s, n, n, w.Ahat, n, dA, lda));
  CK(copy_matrix(s, n, n, w.Ucur, n, dQ, ldq));
  CK(cudaStreamSynchronize(s));
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->k = so.k;
    info->split_residual = so.e;
    info->rank = so.rank;
    info->draw = so.draw;
    info->converged = 1;
  }
  if (!so.accepted) {
    h->err = "no acceptable split";
    return EIG_NO_SPLIT;
  }
  return EIG_OK;
  API_END
}

int eig_split_pencil(eig_handle_t h, int n, const double* dApR, const double* dBpR,
                     const double* dApL, const double* dBpL, int ldp, double* dA, int lda,
                     double* dB, int ldb, double* dQL, int ldql, double* dQR, int ldqr,
                     uint64_t stream, int attempt, const eig_params_t* params,
                     eig_step_info_t* info) {
  API_BEGIN
  REQUIRE(n >= 1, "n must be >= 1");
  REQUIRE(dApR && dBpR && dApL && dBpL && ldp >= n, "IRS iterates / ldp invalid");
  REQUIRE(dA && lda >= n && dB && ldb >= n, "dA / dB invalid");
  REQUIRE(dQL && ldql >= n && dQR && ldqr >= n, "dQL / dQR invalid");
  const eig_params_t p = params_or_default(params);
  check_params(h, p);
  REQUIRE(p.prec == EIG_FP64 || p.prec == EIG_FP64_TC,
          "pencils are solved in FP64 (EIG_FP64 or EIG_FP64_TC) only");
  Arena meas(nullptr);
  SplitWork w;
  ensure_ws(h, carve_split(meas, n, w, p.prec, true));
  Arena a(h->ws);
  carve_split(a, n, w, p.prec, true);
  std::vector<double> hs;
  SplitOut so = run_split_pencil(h, w, n, dApR, dBpR, dApL, dBpL, ldp, dA, lda, dB, ldb, stream,
                                 attempt, p, true, true, hs);
  cudaStream_t s = h->stream;
  CK(copy_matrix(s, n, n, w.Ahat, n, dA, lda));
  CK(copy_matrix(s, n, n, w.Bhat, n, dB, ldb));
  CK(copy_matrix(s, n, n, w.QLn, n, dQL, ldql));
  CK(copy_matrix(s, n, n, w.Ucur, n, dQR, ldqr));
  CK(cudaStreamSynchronize(s));
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->k = so.k;
    info->split_residual = so.e;
    info->rank = so.rank;
    info->draw = so.draw;
    info->converged = 1;
  }
  if (!so.accepted) {
    h->err = "no acceptable split";
    return EIG_NO_SPLIT;
  }
  return EIG_OK;
  API_END
}

int eig_pencil_schur(eig_handle_t h, int n, double* dA, int lda, double* dB, int ldb,
                     double* dQL, int ldql, double* dQR, int ldqr, double* dalphar,
                     double* dalphai, double* dbeta, const eig_params_t* params,
                     eig_solve_info_t* info) {
  API_BEGIN
  REQUIRE(n >= 1, "n must be >= 1");
  REQUIRE(dA && lda >= n && dB && ldb >= n, "dA / dB invalid");
  REQUIRE(dQL && ldql >= n && dQR && ldqr >= n, "dQL / dQR invalid");
  REQUIRE(dalphar && dalphai && dbeta, "eigenvalue outputs are NULL");
  const eig_params_t p = params_or_default(params);
  check_params(h, p);
  REQUIRE(p.prec == EIG_FP64 || p.prec == EIG_FP64_TC,
          "pencils are solved in FP64 (EIG_FP64 or EIG_FP64_TC) only");
  return pencil_impl(h, n, dA, lda, dB, ldb, dQL, ldql, dQR, ldqr, dalphar, dalphai, dbeta, p,
                     info);
  API_END
}

int eig_solve(eig_handle_t h, int kind, int n, double* dA, int lda, double* dwr, double* dwi,
              double* dU, int ldu, const eig_params_t* params, eig_solve_info_t* info) {
  API_BEGIN
  REQUIRE(kind == EIG_KIND_SYM || kind == EIG_KIND_NONSYM, "unknown kind");
  REQUIRE(n >= 1, "n must be >= 1");
  REQUIRE(dA && lda >= n, "dA / lda invalid");
  REQUIRE(dwr, "dwr is NULL");
  REQUIRE(kind == EIG_KIND_SYM || dwi, "dwi is NULL");
  REQUIRE(dU && ldu >= n, "dU / ldu invalid");
  const eig_params_t p = params_or_default(params);
  check_params(h, p);
  return solve_impl(h, kind, n, dA, lda, dwr, dwi, dU, ldu, p, info);
  API_END
}

int eig_eigenvectors(eig_handle_t h, int n, const double* dT, int ldt, const double* dQ, int ldq,
                     const double* dwi, double* dV, int ldv, double* dlam) {
  API_BEGIN
  REQUIRE(n >= 1, "n must be >= 1");
  REQUIRE(dT && ldt >= n && dQ && ldq >= n && dwi, "dT / dQ / dwi invalid");
  REQUIRE(dV && ldv >= n && dlam, "dV / dlam invalid");
  std::string err;
  const int rc = trevc(h->stream, n, dT, ldt, dQ, ldq, dwi, dV, ldv, dlam, &err);
  if (rc < 0) h->err = err;
  return rc;
  API_END
}

int eig_eigenvectors_complex(eig_handle_t h, int n, const double* dT, int ldt, const double* dU,
                             int ldu, double* dV, int ldv, double* dlam) {
  API_BEGIN
  REQUIRE(n >= 1, "n must be >= 1");
  REQUIRE(dT && ldt >= n && dU && ldu >= n, "dT / dU invalid");
  REQUIRE(dV && ldv >= n && dlam, "dV / dlam invalid");
  std::string err;
  const int rc = trevc(h->stream, n, dT, ldt, dU, ldu, nullptr, dV, ldv, dlam, &err, true);
  if (rc < 0) h->err = err;
  return rc;
  API_END
}

int eig_zgemm(eig_handle_t h, int ta, int tb, int m, int n, int k, double alpha_re,
              double alpha_im, const double* dA, int lda, const double* dB, int ldb,
              double beta_re, double beta_im, double* dC, int ldc) {
  API_BEGIN
  REQUIRE(m >= 0 && n >= 0 && k >= 0, "negative size");
  REQUIRE(dA && dB && dC, "NULL matrix");
  REQUIRE(lda >= std::max(1, ta ? k : m) && ldb >= std::max(1, tb ? n : k) && ldc >= std::max(1, m),
          "leading dimension too small");
  CK(cplane_zgemm(h->stream, ta != 0, tb != 0, m, n, k, alpha_re, alpha_im, dA, lda, dB, ldb,
                  beta_re, beta_im, dC, ldc));
  CK(cudaStreamSynchronize(h->stream));
  return EIG_OK;
  API_END
}

int eig_zqr(eig_handle_t h, int m, int n, const double* dX, int ldx, double* dQ, int ldq,
            double* dR, int ldr) {
  API_BEGIN
  REQUIRE(m >= 1 && n >= 1 && m >= n, "need m >= n >= 1");
  REQUIRE(dX && ldx >= m && dQ && ldq >= m && (!dR || ldr >= n), "matrix / leading dimension invalid");
  std::string err;
  const int rc = cplane_qr(h->stream, m, n, dX, ldx, dQ, ldq, dR, ldr, &err);
  if (rc < 0) h->err = err;
  return rc;
  API_END
}

int eig_zhaar(eig_handle_t h, int n, uint64_t seed, uint64_t stream, int attempt, double* dV,
              int ldv) {
  API_BEGIN
  REQUIRE(n >= 1 && dV && ldv >= n, "dV / ldv invalid");
  std::string err;
  const int rc = cplane_haar(h->stream, n, seed, stream, attempt, dV, ldv, &err);
  if (rc < 0) h->err = err;
  return rc;
  API_END
}

int eig_zline_step(eig_handle_t h, int n, const double* dA, int lda, double w_re, double w_im,
                   double t, double s, uint64_t stream, int attempt, const eig_params_t* params,
                   double* dQ, int ldq, double* dAhat, int ldah, eig_step_info_t* info) {
  API_BEGIN
  REQUIRE(n >= 2, "n must be >= 2");
  REQUIRE(dA && lda >= n && (!dQ || ldq >= n) && (!dAhat || ldah >= n), "matrix / leading dimension invalid");
  REQUIRE(s > 0.0 && std::fabs(std::hypot(w_re, w_im) - 1.0) <= 1e-12, "need s > 0 and |w| = 1");
  const eig_params_t p = params_or_default(params);
  check_params(h, p);
  std::string err;
  const int rc = cplane_step(h->stream, n, dA, lda, w_re, w_im, t, s, p, stream, attempt, dQ, ldq,
                             dAhat, ldah, info, &err);
  if (rc < 0) h->err = err;
  return rc;
  API_END
}

int eig_schur_complex(eig_handle_t h, int n, const double* dA, int lda, double* dT, int ldt,
                      double* dU, int ldu, double* dw, const eig_params_t* params, int enclose,
                      eig_enclosure_t* enc, int enc_cap, int* n_enc, eig_solve_info_t* info) {
  API_BEGIN
  REQUIRE(n >= 1, "n must be >= 1");
  REQUIRE(dA && lda >= n, "dA / lda invalid");
  REQUIRE(dT && ldt >= n && dU && ldu >= n && dw, "dT / dU / dw invalid");
  REQUIRE(enc_cap >= 0 && (enc_cap == 0 || enc), "enc / enc_cap invalid");
  const eig_params_t p = params_or_default(params);
  check_params(h, p);
  REQUIRE(p.leaf_size <= 64, "leaf_size must be <= 64");
  std::vector<CplaneCluster> cl;
  std::string err;
  const int rc = cplane_schur(h->stream, n, dA, lda, dT, ldt, dU, ldu, dw, p, enclose != 0, &cl,
                              info, &err);
  if (rc < 0) {
    h->err = err;
    return rc;
  }
  if (n_enc) *n_enc = (int)cl.size();
  for (int i = 0; i < (int)cl.size() && i < enc_cap; ++i) {
    eig_enclosure_t& e = enc[i];
    std::memset(&e, 0, sizeof(e));
    e.offset = cl[i].off;
    e.size = cl[i].m;
    e.c_re = cl[i].cr;
    e.c_im = cl[i].ci;
    e.R = cl[i].R;
    const int nh = (int)cl[i].hp.size();
    const int first = std::max(0, nh - EIG_MAX_HALFPLANES);
    e.nhp = nh - first;
    for (int j = first; j < nh; ++j) {
      e.w_re[j - first] = cl[i].hp[j].wr;
      e.w_im[j - first] = cl[i].hp[j].wi;
      e.t[j - first] = cl[i].hp[j].t;
    }
  }
  return rc;
  API_END
}

int eig_svd(eig_handle_t h, int m, int n, const double* dA, int lda, double* dS, double* dU,
            int ldu, double* dV, int ldv, const eig_params_t* params, eig_solve_info_t* info) {
  API_BEGIN
  REQUIRE(m >= 1 && n >= 1, "m and n must be >= 1");
  REQUIRE(dA && lda >= m, "dA / lda invalid");
  REQUIRE(dS && dU && ldu >= m && dV && ldv >= n, "dS / dU / dV invalid");
  const eig_params_t p = params_or_default(params);
  check_params(h, p);
  const int N = m + n;
  const size_t nn = (size_t)N * N;
  const size_t bytes = sizeof(double) * (2 * nn + N + 32);
  if (bytes > h->aux_bytes) {
    CK(cudaStreamSynchronize(h->stream));
    if (h->aux) cudaFree(h->aux);
    h->aux = nullptr;
    h->aux_bytes = 0;
    if (cudaMalloc(&h->aux, bytes) != cudaSuccess) {
      cudaGetLastError();
      h->err = "SVD buffer allocation failed";
      return EIG_ERR_NOMEM;
    }
    h->aux_bytes = bytes;
  }
  double* H = reinterpret_cast<double*>(h->aux);
  double* W = H + nn;
  double* w = W + nn;
  CK(svd_embed(h->stream, m, n, dA, lda, H, N));
  const int st = solve_impl(h, EIG_KIND_SYM, N, H, N, w, nullptr, W, N, p, info);
  if (st != EIG_OK) return st;
  CK(svd_extract(h->stream, m, n, W, N, w, dS, dU, ldu, dV, ldv));
  CK(cudaStreamSynchronize(h->stream));
  return EIG_OK;
  API_END
}

int eig_solve_batched(eig_handle_t h, int kind, int count, const int* n, double* const* dA,
                      const int* lda, double* const* dwr, double* const* dwi, double* const* dU,
                      const int* ldu, const eig_params_t* params, int* status,
                      eig_solve_info_t* infos) {
  API_BEGIN
  REQUIRE(kind == EIG_KIND_SYM || kind == EIG_KIND_NONSYM, "unknown kind");
  REQUIRE(count >= 0, "count < 0");
  REQUIRE(count == 0 || (n && dA && lda && dwr && dU && ldu && status), "NULL array");
  REQUIRE(kind == EIG_KIND_SYM || count == 0 || dwi, "dwi is NULL");
  for (int i = 0; i < count; ++i) {
    REQUIRE(n[i] >= 1 && dA[i] && lda[i] >= n[i] && dwr[i] && dU[i] && ldu[i] >= n[i],
            "invalid problem " + std::to_string(i));
    REQUIRE(kind == EIG_KIND_SYM || dwi[i], "dwi[" + std::to_string(i) + "] is NULL");
  }
  eig_params_t p = params_or_default(params);
  check_params(h, p);
  const int nworkers = std::max(1, std::min(p.workers, 32));
  p.workers = 1;   // each problem runs sequentially inside its worker
  CK(cudaStreamSynchronize(h->stream));   // inputs written on the caller's stream
  ensure_workers(h, nworkers);
  // largest problems first
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return n[a] > n[b]; });
  std::atomic<int> next{0};
  auto work = [&](eig_handle_t hw) {
    cudaSetDevice(hw->device);
    while (true) {
      const int t = next.fetch_add(1);
      if (t >= count) return;
      const int i = order[t];
      eig_solve_info_t inf;
      std::memset(&inf, 0, sizeof(inf));
      int rc;
      try {
        hw->err.clear();
        rc = solve_impl(hw, kind, n[i], dA[i], lda[i], dwr[i], dwi ? dwi[i] : nullptr, dU[i],
                        ldu[i], p, &inf);
      } catch (Fail f) {
        rc = f.code;
      }
      status[i] = rc;
      if (infos) infos[i] = inf;
    }
  };
  std::vector<std::thread> threads;
  for (int i = 0; i < nworkers; ++i) threads.emplace_back(work, h->workers[i]);
  for (auto& t : threads) t.join();
  CK(cudaSetDevice(h->device));
  for (int i = 0; i < nworkers; ++i) CK(cudaStreamSynchronize(h->workers[i]->stream));
  for (int i = 0; i < count; ++i)
    if (status[i] != EIG_OK) {
      h->err = "problem " + std::to_string(i) + " returned " + std::to_string(status[i]);
      return status[i] < 0 ? status[i] : EIG_OK;
    }
  return EIG_OK;
  API_END
}

}  // extern "C"

namespace {

// Launch shape of the fused batched solver on h's device: CTAs for `count`
// problems (cps CTAs per SM, 0: automatic) and the workspace bytes fused_run
// takes from the front of h's workspace for problems of at most mx rows.
size_t fused_run_bytes(eig_handle_t h, int count, int mx, int cps, int* ctas_out) {
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
  const int maxc = fused_max_ctas_per_sm();
  const int c = cps > 0 ? std::min(cps, maxc) : std::min(2, maxc);
  const int ctas = std::max(1, std::min(count, sms * c));
  if (ctas_out) *ctas_out = ctas;
  const size_t pb = round_up(sizeof(FusedProblem) * count);
  const size_t ob = round_up(sizeof(int) * count);
  const size_t rb = round_up(sizeof(FusedResult) * count);
  return pb + ob + rb + 256 + fused_workspace_bytes(std::max(mx, 1), ctas);
}

// One persistent launch of the fused batched solver over the problems
// (largest first); fills status / infos; *ms (if non-null) gets the kernel's
// CUDA-event time on the handle's stream.  nodes (optional): per problem the
// node id, interval and depth of the recursion it continues (id, lo, hi,
// depth, has_interval of FusedProblem; the other fields are ignored).
void fused_run(eig_handle_t h, int count, const int* n, double* const* dA, const int* lda,
               double* const* dw, double* const* dU, const int* ldu, const eig_params_t& p,
               int nb, int cps, int* status, eig_solve_info_t* infos, float* ms,
               const FusedProblem* nodes) {
  cudaStream_t s = h->stream;
  int mx = 1;
  for (int i = 0; i < count; ++i) mx = std::max(mx, n[i]);
  int ctas = 1;
  const size_t total = fused_run_bytes(h, count, mx, cps, &ctas);
  const size_t pb = round_up(sizeof(FusedProblem) * count);
  const size_t ob = round_up(sizeof(int) * count);
  const size_t rb = round_up(sizeof(FusedResult) * count);
  ensure_ws(h, total);
  char* base = h->ws;
  FusedProblem* dprobs = reinterpret_cast<FusedProblem*>(base);
  int* dorder = reinterpret_cast<int*>(base + pb);
  FusedResult* dres = reinterpret_cast<FusedResult*>(base + pb + ob);
  int* dcounter = reinterpret_cast<int*>(base + pb + ob + rb);
  void* dws = base + pb + ob + rb + 256;
  char* pin = static_cast<char*>(pinned(h, std::max(pb + ob, rb) + 64));
  FusedProblem* hp = reinterpret_cast<FusedProblem*>(pin);
  int* ho = reinterpret_cast<int*>(pin + pb);
  for (int i = 0; i < count; ++i) {
    hp[i] = FusedProblem{n[i], lda[i], ldu[i], 0, dA[i], dw[i], dU[i], 1, 0.0, 0.0, 0, 0};
    if (nodes) {
      hp[i].id = nodes[i].id;
      hp[i].lo = nodes[i].lo;
      hp[i].hi = nodes[i].hi;
      hp[i].depth = nodes[i].depth;
      hp[i].has_interval = nodes[i].has_interval;
    }
  }
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return n[a] > n[b]; });
  std::memcpy(ho, order.data(), sizeof(int) * count);
  CK(cudaMemcpyAsync(dprobs, hp, pb + ob, cudaMemcpyHostToDevice, s));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (ms) {
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, s));
  }
  CK(fused_batched(s, count, dprobs, dorder, dres, dcounter, p, nb, ctas, mx, dws));
  if (ms) CK(cudaEventRecord(e1, s));
  // the staging area is reused for the results once the inputs are copied
  CK(cudaStreamSynchronize(s));
  FusedResult* hr = reinterpret_cast<FusedResult*>(pin);
  CK(cudaMemcpyAsync(hr, dres, sizeof(FusedResult) * count, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (ms) {
    CK(cudaEventElapsedTime(ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  for (int i = 0; i < count; ++i) {
    const FusedResult& r = hr[i];
    status[i] = r.status;
    if (infos) {
      eig_solve_info_t inf;
      inf.status = r.status;
      inf.nodes = r.nodes;
      inf.splits = r.splits;
      inf.max_depth = r.max_depth;
      inf.total_iters = r.total_iters;
      inf.failed_attempts = r.failed_attempts;
      inf.leaves = r.leaves;
      inf.flops = r.flops;
      infos[i] = inf;
    }
  }
}

// splitmix64-based uniform in [0, 1) (host-side draws of the tuner's sizes)
double tune_uniform(uint64_t& st) {
  st += 0x9E3779B97F4A7C15ull;
  uint64_t z = st;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * 0x1p-53;
}

}  // namespace

extern "C" {

int eig_solve_batched_fused(eig_handle_t h, int count, const int* n, double* const* dA,
                            const int* lda, double* const* dw, double* const* dU, const int* ldu,
                            const eig_params_t* params, int* status, eig_solve_info_t* infos) {
  API_BEGIN
  REQUIRE(count >= 0, "count < 0");
  REQUIRE(count == 0 || (n && dA && lda && dw && dU && ldu && status), "NULL array");
  for (int i = 0; i < count; ++i) {
    REQUIRE(n[i] >= 1 && n[i] <= fused_max_n(),
            "problem " + std::to_string(i) + ": n must be in [1, " +
                std::to_string(fused_max_n()) + "]");
    REQUIRE(dA[i] && lda[i] >= n[i] && dw[i] && dU[i] && ldu[i] >= n[i],
            "invalid problem " + std::to_string(i));
  }
  if (count == 0) return EIG_OK;
  eig_params_t p = params_or_default(params);
  check_params(h, p);
  fused_run(h, count, n, dA, lda, dw, dU, ldu, p, h->fused_nb, h->fused_cps, status, infos,
            nullptr);
  for (int i = 0; i < count; ++i)
    if (status[i] != EIG_OK) {
      h->err = "problem " + std::to_string(i) + " returned " + std::to_string(status[i]);
      break;
    }
  return EIG_OK;
  API_END
}

int eig_fused_autotune(eig_handle_t h, int samples, int nmin, int nmax, uint64_t seed,
                       eig_fused_config_t* table, int table_cap, int* n_table,
                       eig_fused_config_t* best) {
  API_BEGIN
  REQUIRE(samples >= 1 && samples <= 100000, "samples must be in [1, 100000]");
  REQUIRE(nmin >= 1 && nmax >= nmin && nmax <= fused_max_n(), "need 1 <= nmin <= nmax <= 512");
  REQUIRE(table_cap >= 0 && (table_cap == 0 || table), "table / table_cap invalid");
  cudaStream_t s = h->stream;
  // sizes log-uniform in [nmin, nmax]; A = (G + G^T) / 2 from Philox Gaussians
  std::vector<int> ns(samples), lds(samples);
  uint64_t st = seed;
  size_t elems = 0;
  for (int i = 0; i < samples; ++i) {
    const double u = tune_uniform(st);
    ns[i] = std::max(nmin, std::min(nmax, (int)std::lround(std::exp(std::log((double)nmin) +
                                                                     u * (std::log((double)nmax) -
                                                                          std::log((double)nmin))))));
    lds[i] = ns[i];
    elems += 3 * (size_t)ns[i] * ns[i] + ns[i];
  }
  double* buf = nullptr;
  if (cudaMalloc(&buf, sizeof(double) * elems) != cudaSuccess) {
    cudaGetLastError();
    h->err = "autotune sample allocation failed";
    return EIG_ERR_NOMEM;
  }
  std::vector<double*> A0(samples), A(samples), w(samples), U(samples);
  size_t off = 0;
  for (int i = 0; i < samples; ++i) {
    const size_t nn = (size_t)ns[i] * ns[i];
    A0[i] = buf + off; off += nn;
    A[i] = buf + off; off += nn;
    U[i] = buf + off; off += nn;
    w[i] = buf + off; off += ns[i];
  }
  int rc = EIG_OK;
  try {
    for (int i = 0; i < samples; ++i) {
      CK(gaussian(s, ns[i], ns[i], seed, 9, (uint64_t)i, 0, A0[i], ns[i]));
      CK(symmetrize(s, ns[i], A0[i], ns[i]));
    }
    eig_params_t p;
    eig_default_params(&p);
    p.seed = seed;
    std::vector<int> stv(samples);
    const int maxc = fused_max_ctas_per_sm();
    std::vector<eig_fused_config_t> tab;
    eig_fused_config_t win{32, std::min(2, maxc), INFINITY};
    for (int nb : {16, 32}) {
      for (int cps = 1; cps <= std::min(3, maxc); ++cps) {
        for (int i = 0; i < samples; ++i)
          CK(cudaMemcpyAsync(A[i], A0[i], sizeof(double) * ns[i] * ns[i], cudaMemcpyDeviceToDevice, s));
        float ms = 0.0f;
        fused_run(h, samples, ns.data(), A.data(), lds.data(), w.data(), U.data(), lds.data(), p,
                  nb, cps, stv.data(), nullptr, &ms);
        const eig_fused_config_t c{nb, cps, (double)ms};
        tab.push_back(c);
        if (c.ms < win.ms) win = c;
      }
    }
    h->fused_nb = win.nb;
    h->fused_cps = win.ctas_per_sm;
    if (best) *best = win;
    if (n_table) *n_table = (int)tab.size();
    for (int i = 0; i < (int)tab.size() && i < table_cap; ++i) table[i] = tab[i];
  } catch (Fail f) {
    rc = f.code;
  }
  cudaStreamSynchronize(s);
  cudaFree(buf);
  return rc;
  API_END
}

int eig_qr(eig_handle_t h, int m, int n, const double* dX, int ldx, double* dQ, int ldq,
           double* dR, int ldr) {
  API_BEGIN
  REQUIRE(m >= n && n >= 1, "need m >= n >= 1");
  REQUIRE(dX && ldx >= m, "dX / ldx invalid");
  REQUIRE(!dQ || ldq >= m, "ldq invalid");
  REQUIRE(!dR || ldr >= n, "ldr invalid");
  Arena meas(nullptr);
  QRWork w;
  ensure_ws(h, carve_qr(meas, m, n, w));
  Arena a(h->ws);
  carve_qr(a, m, n, w);
  qr_explicit(h, w, m, n, dX, ldx, dQ, ldq, dR, ldr);
  CK(cudaStreamSynchronize(h->stream));
  return EIG_OK;
  API_END
}

int eig_gaussian(eig_handle_t h, int rows, int cols, uint64_t seed, int purpose, uint64_t stream,
                 int attempt, double* dG, int ldg) {
  API_BEGIN
  REQUIRE(rows >= 0 && cols >= 0 && dG && ldg >= std::max(rows, 1), "invalid arguments");
  CK(gaussian(h->stream, rows, cols, seed, purpose, stream, attempt, dG, ldg));
  CK(cudaStreamSynchronize(h->stream));
  return EIG_OK;
  API_END
}

int eig_haar(eig_handle_t h, int n, uint64_t seed, int purpose, uint64_t stream, int attempt,
             double* dV, int ldv) {
  API_BEGIN
  REQUIRE(n >= 1 && dV && ldv >= n, "invalid arguments");
  Arena meas(nullptr);
  QRWork w;
  size_t need = carve_qr(meas, n, n, w) + round_up(sizeof(double) * (size_t)n * n);
  ensure_ws(h, need);
  Arena a(h->ws);
  double* G = a.take<double>((size_t)n * n);
  carve_qr(a, n, n, w);
  CK(gaussian(h->stream, n, n, seed, purpose, stream, attempt, G, n));
  qr_explicit(h, w, n, n, G, n, dV, ldv, nullptr, 0);
  CK(cudaStreamSynchronize(h->stream));
  return EIG_OK;
  API_END
}

int eig_split_test(eig_handle_t h, int n, const double* dA, int lda, double normA, const double* dB,
                   int ldb, double normB, int* k, double* e, double* hscores) {
  API_BEGIN
  REQUIRE(n >= 2 && dA && lda >= n && k && e, "invalid arguments");
  REQUIRE(!dB || ldb >= n, "ldb invalid");
  REQUIRE(normA > 0 && (!dB || normB > 0), "norms must be > 0");
  Arena meas(nullptr);
  const size_t nrb = (size_t)(n + 31) / 32;
  meas.take<double>(n);
  meas.take<double>(nrb * n + n + 8);
  ensure_ws(h, meas.used);
  Arena a(h->ws);
  double* sc = a.take<double>(n);
  double* colpart = a.take<double>(nrb * n + n + 8);
  cudaStream_t s = h->stream;
  CK(split_scores(s, n, dA, lda, 1.0 / normA, colpart, sc, false));
  if (dB) CK(split_scores(s, n, dB, ldb, 1.0 / normB, colpart, sc, true));
  std::vector<double> hv(n - 1);
  CK(cudaMemcpyAsync(hv.data(), sc, sizeof(double) * (n - 1), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  *k = choose_k(hv.data(), n);
  *e = hv[*k - 1];
  if (hscores) std::memcpy(hscores, hv.data(), sizeof(double) * (n - 1));
  return EIG_OK;
  API_END
}

int eig_gemm(eig_handle_t h, int ta, int tb, int m, int n, int k, double alpha, const double* dA,
             int lda, const double* dB, int ldb, double beta, double* dC, int ldc) {
  API_BEGIN
  REQUIRE(m >= 0 && n >= 0 && k >= 0 && dC && ldc >= std::max(m, 1), "invalid arguments");
  const int sp = gemm_choose_splits(m, n, k);
  size_t need = sp > 1 ? sizeof(double) * (size_t)sp * m * n : 256;
  ensure_ws(h, need);
  CK(gemm(h->stream, ta != 0, tb != 0, m, n, k, alpha, dA, lda, dB, ldb, beta, dC, ldc, sp,
          reinterpret_cast<double*>(h->ws)));
  CK(cudaStreamSynchronize(h->stream));
  return EIG_OK;
  API_END
}

int eig_gemm_fp64tc(eig_handle_t h, int ta, int tb, int m, int n, int k, double alpha,
                    const double* dA, int lda, const double* dB, int ldb, double beta, double* dC,
                    int ldc) {
  API_BEGIN
  REQUIRE(m >= 0 && n >= 0 && k >= 0 && dC && ldc >= std::max(m, 1), "invalid arguments");
  REQUIRE(lda >= std::max(1, ta ? k : m) && ldb >= std::max(1, tb ? n : k), "invalid ld");
  const size_t need = tcx_gemm_workspace_bytes(m, n, k) + 256;
  ensure_ws(h, need);
  int* derr = reinterpret_cast<int*>(h->ws + need - 256);
  CK(cudaMemsetAsync(derr, 0, sizeof(int), h->stream));
  CK(tcx_gemm(h->stream, ta != 0, tb != 0, m, n, k, alpha, dA, lda, dB, ldb, beta, dC, ldc, h->ws,
              derr));
  int* hf = static_cast<int*>(pinned(h, 64));
  CK(cudaMemcpyAsync(hf, derr, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (*hf) {
    h->err = "tensor-core GEMM: a bounded wait timed out (flag " + std::to_string(*hf) + ")";
    return EIG_ERR_CUDA;
  }
  return EIG_OK;
  API_END
}

int eig_gemm_split(eig_handle_t h, int ta, int tb, int m, int n, int k, double alpha,
                   const double* dA, int lda, const double* dB, int ldb, double beta, double* dC,
                   int ldc) {
  API_BEGIN
  REQUIRE(m >= 0 && n >= 0 && k >= 0 && dC && ldc >= std::max(m, 1), "invalid arguments");
  REQUIRE(lda >= std::max(1, ta ? k : m) && ldb >= std::max(1, tb ? n : k), "invalid ld");
  const size_t need = tc_gemm_workspace_bytes(m, n, k) + 256;
  ensure_ws(h, need);
  int* derr = reinterpret_cast<int*>(h->ws + need - 256);
  CK(cudaMemsetAsync(derr, 0, sizeof(int), h->stream));
  CK(tc_gemm(h->stream, ta != 0, tb != 0, m, n, k, alpha, dA, lda, dB, ldb, beta, dC, ldc, h->ws,
             derr));
  int* hf = static_cast<int*>(pinned(h, 64));
  CK(cudaMemcpyAsync(hf, derr, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (*hf) {
    h->err = "tensor-core GEMM: a bounded wait timed out (flag " + std::to_string(*hf) + ")";
    return EIG_ERR_CUDA;
  }
  return EIG_OK;
  API_END
}

int eig_gemm_fp32tc(eig_handle_t h, int ta, int tb, int m, int n, int k, double alpha,
                    const double* dA, int lda, const double* dB, int ldb, double beta, double* dC,
                    int ldc) {
  API_BEGIN
  REQUIRE(m >= 0 && n >= 0 && k >= 0 && dC && ldc >= std::max(m, 1), "invalid arguments");
  REQUIRE(lda >= std::max(1, ta ? k : m) && ldb >= std::max(1, tb ? n : k), "invalid ld");
  const size_t need = tcx32_gemm_workspace_bytes(m, n, k) + 256;
  ensure_ws(h, need);
  int* derr = reinterpret_cast<int*>(h->ws + need - 256);
  CK(cudaMemsetAsync(derr, 0, sizeof(int), h->stream));
  CK(tcx32_gemm(h->stream, ta != 0, tb != 0, m, n, k, alpha, dA, lda, dB, ldb, beta, dC, ldc,
                h->ws, derr));
  int* hf = static_cast<int*>(pinned(h, 64));
  CK(cudaMemcpyAsync(hf, derr, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (*hf) {
    h->err = "tensor-core GEMM: a bounded wait timed out (flag " + std::to_string(*hf) + ")";
    return EIG_ERR_CUDA;
  }
  return EIG_OK;
  API_END
}

}  // extern "C"

// =================================================================== serving
// A request server over the same solver: worker threads, each with its own
// CUDA stream and workspace, take requests in arrival order as soon as a
// worker is free and the request's device footprint fits the HBM budget
// (continuous batching: requests that arrive while others run are admitted
// as slots and memory free up, and their work overlaps on the device).
namespace {

struct Request {
  uint64_t ticket;
  int kind, n, lda, ldu;
  double *dA, *dwr, *dwi, *dU;
  int ldb = 0, ldqr = 0;                                      // pencils
  double *dB = nullptr, *dQR = nullptr, *dbeta = nullptr;     // pencils
  int enclose = 0;                                            // complex plane: dQR holds T
  eig_params_t p;
  size_t footprint;
  double t_submit = 0, t_start = 0, t_end = 0;
  int status = EIG_OK;
  bool done = false;
  eig_solve_info_t info;
};

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

size_t solve_footprint(int n, int kind, int prec, int fused_tail = 0, int leaf = 64) {
  if (kind == EIG_KIND_CPLANE) return cplane_footprint(n, prec);
  Arena a(nullptr);
  SolveMain w;
  NodeWork nw;
  const bool pencil = kind == EIG_KIND_PENCIL;
  carve_main(a, n, kind == EIG_KIND_SYM && split_mode(prec), w, pencil);
  carve_node(a, n, n, prec, nw, pencil);
  size_t bytes = a.used;
  // fused tail (symmetric): at most n / (leaf + 1) nodes of at most T rows,
  // one CTA each (at most 2 per SM of 152), their eigenvector blocks and the
  // n x T product buffer
  const int t = std::min(std::min(fused_tail, fused_max_n()), n);
  if (kind == EIG_KIND_SYM && t > leaf) {
    const int cnt = std::max(1, n / (std::max(leaf, 1) + 1));
    bytes += fused_workspace_bytes(t, std::min(cnt, 2 * 152)) +
             sizeof(double) * (2 * (size_t)n * t) + (size_t)cnt * 512 + 4096;
  }
  return bytes;
}

}  // namespace

struct eig_server_s {
  int device = 0;
  size_t budget = 0;
  size_t reserved = 0, peak_reserved = 0;
  uint64_t next_ticket = 1;
  uint64_t completed = 0;
  bool stop = false;
  std::vector<eig_handle_s*> workers;
  std::vector<std::thread> threads;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::vector<Request*> all;
};

static void server_worker(eig_server_s* S, eig_handle_s* hw) {
  cudaSetDevice(hw->device);
  while (true) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lock(S->mu);
      S->cv_work.wait(lock, [&] {
        if (S->stop) return true;
        if (S->queue.empty()) return false;
        Request* h = S->queue.front();
        return S->reserved == 0 || S->reserved + h->footprint <= S->budget;
      });
      if (S->stop) return;
      r = S->queue.front();
      S->queue.pop_front();
      S->reserved += r->footprint;
      S->peak_reserved = std::max(S->peak_reserved, S->reserved);
      r->t_start = now_s();
    }
    int rc;
    eig_solve_info_t inf;
    std::memset(&inf, 0, sizeof(inf));
    try {
      NvtxRange nvtx_("eig.request");
      hw->err.clear();
      if (r->kind == EIG_KIND_PENCIL) {
        rc = pencil_impl(hw, r->n, r->dA, r->lda, r->dB, r->ldb, r->dU, r->ldu, r->dQR, r->ldqr,
                         r->dwr, r->dwi, r->dbeta, r->p, &inf);
      } else if (r->kind == EIG_KIND_CPLANE) {
        std::string err;
        rc = cplane_schur(hw->stream, r->n, r->dA, r->lda, r->dQR, r->ldqr, r->dU, r->ldu, r->dwr,
                          r->p, r->enclose != 0, nullptr, &inf, &err);
        if (rc < 0) hw->err = err;
      } else
        rc = solve_impl(hw, r->kind, r->n, r->dA, r->lda, r->dwr, r->dwi, r->dU, r->ldu, r->p,
                        &inf);
    } catch (Fail f) {
      rc = f.code;
    }
    // nothing of this request may still run once it is reported done (a
    // failed solve can stop with launches in flight)
    cudaStreamSynchronize(hw->stream);
    // keep a worker's scratch only while it is small: the budget counts
    // running requests, so large idle workspaces are returned
    if (hw->ws_bytes > ((size_t)1 << 30)) {
      cudaStreamSynchronize(hw->stream);
      cudaFree(hw->ws);
      hw->ws = nullptr;
      hw->ws_bytes = 0;
    }
    {
      std::lock_guard<std::mutex> lock(S->mu);
      r->status = rc;
      r->info = inf;
      r->t_end = now_s();
      r->done = true;
      S->reserved -= r->footprint;
      S->completed++;
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
}

extern "C" {

int eig_server_create(eig_server_t* out, int device, int workers, double hbm_budget_gb) {
  if (!out || workers < 1 || workers > 64 || !(hbm_budget_gb > 0)) return EIG_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return EIG_ERR_CUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return EIG_ERR_CUDA;
  panel_init();
  eig_server_s* S = new eig_server_s();
  S->device = device;
  S->budget = (size_t)(hbm_budget_gb * 1e9);
  for (int i = 0; i < workers; ++i) {
    eig_handle_s* w = new eig_handle_s();
    w->device = device;
    if (cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete w;
      break;
    }
    S->workers.push_back(w);
  }
  if (S->workers.empty()) {
    delete S;
    return EIG_ERR_CUDA;
  }
  for (eig_handle_s* w : S->workers) S->threads.emplace_back(server_worker, S, w);
  *out = S;
  return EIG_OK;
}

static void enqueue(eig_server_s* S, Request* r, uint64_t* ticket) {
  r->footprint = solve_footprint(r->n, r->kind, r->p.prec, r->p.fused_tail, r->p.leaf_size);
  std::memset(&r->info, 0, sizeof(r->info));
  {
    std::lock_guard<std::mutex> lock(S->mu);
    r->ticket = S->next_ticket++;
    r->t_submit = now_s();
    S->queue.push_back(r);
    S->all.push_back(r);
    *ticket = r->ticket;
  }
  S->cv_work.notify_all();
}

int eig_server_submit(eig_server_t S, int kind, int n, double* dA, int lda, double* dwr,
                      double* dwi, double* dU, int ldu, const eig_params_t* params,
                      uint64_t* ticket) {
  if (!S || !ticket) return EIG_ERR_ARG;
  if ((kind != EIG_KIND_SYM && kind != EIG_KIND_NONSYM) || n < 1 || !dA || lda < n || !dwr ||
      !dU || ldu < n || (kind == EIG_KIND_NONSYM && !dwi))
    return EIG_ERR_ARG;
  Request* r = new Request();
  r->kind = kind;
  r->n = n;
  r->dA = dA;
  r->lda = lda;
  r->dwr = dwr;
  r->dwi = dwi;
  r->dU = dU;
  r->ldu = ldu;
  eig_default_params(&r->p);
  if (params) r->p = *params;
  r->p.workers = 1;
  r->p.graphs = 0;   // the caller keeps running CUDA work while requests are served
  if (r->p.maxit < 0 || r->p.leaf_size < 1 || r->p.v_draws < 1 ||
      !valid_prec(r->p.prec)) {
    delete r;
    return EIG_ERR_ARG;
  }
  enqueue(S, r, ticket);
  return EIG_OK;
}

int eig_server_submit_pencil(eig_server_t S, int n, double* dA, int lda, double* dB, int ldb,
                             double* dQL, int ldql, double* dQR, int ldqr, double* dalphar,
                             double* dalphai, double* dbeta, const eig_params_t* params,
                             uint64_t* ticket) {
  if (!S || !ticket) return EIG_ERR_ARG;
  if (n < 1 || !dA || lda < n || !dB || ldb < n || !dQL || ldql < n || !dQR || ldqr < n ||
      !dalphar || !dalphai || !dbeta)
    return EIG_ERR_ARG;
  Request* r = new Request();
  r->kind = EIG_KIND_PENCIL;
  r->n = n;
  r->dA = dA;
  r->lda = lda;
  r->dB = dB;
  r->ldb = ldb;
  r->dU = dQL;
  r->ldu = ldql;
  r->dQR = dQR;
  r->ldqr = ldqr;
  r->dwr = dalphar;
  r->dwi = dalphai;
  r->dbeta = dbeta;
  eig_default_params(&r->p);
  if (params) r->p = *params;
  r->p.workers = 1;
  r->p.graphs = 0;
  if (r->p.maxit < 0 || r->p.leaf_size < 1 || r->p.v_draws < 1 ||
      (r->p.prec != EIG_FP64 && r->p.prec != EIG_FP64_TC)) {
    delete r;
    return EIG_ERR_ARG;
  }
  enqueue(S, r, ticket);
  return EIG_OK;
}

int eig_server_submit_complex(eig_server_t S, int n, const double* dA, int lda, double* dT,
                              int ldt, double* dU, int ldu, double* dw, const eig_params_t* params,
                              int enclose, uint64_t* ticket) {
  if (!S || !ticket) return EIG_ERR_ARG;
  if (n < 1 || !dA || lda < n || !dT || ldt < n || !dU || ldu < n || !dw) return EIG_ERR_ARG;
  Request* r = new Request();
  r->kind = EIG_KIND_CPLANE;
  r->n = n;
  r->dA = const_cast<double*>(dA);   // read only
  r->lda = lda;
  r->dQR = dT;
  r->ldqr = ldt;
  r->dU = dU;
  r->ldu = ldu;
  r->dwr = dw;
  r->enclose = enclose;
  eig_default_params(&r->p);
  if (params) r->p = *params;
  r->p.workers = 1;
  r->p.graphs = 0;
  if (r->p.maxit < 0 || r->p.leaf_size < 1 || r->p.leaf_size > 64 || r->p.v_draws < 1 ||
      r->p.max_fail < 0 || r->p.split_tol < 0 ||
      !valid_prec(r->p.prec)) {
    delete r;
    return EIG_ERR_ARG;
  }
  enqueue(S, r, ticket);
  return EIG_OK;
}

static Request* find_request(eig_server_s* S, uint64_t ticket) {
  if (ticket == 0 || ticket > S->all.size()) return nullptr;
  return S->all[ticket - 1];
}

int eig_server_poll(eig_server_t S, uint64_t ticket, int* done, int* status, double* times,
                    eig_solve_info_t* info) {
  if (!S || !done) return EIG_ERR_ARG;
  std::lock_guard<std::mutex> lock(S->mu);
  Request* r = find_request(S, ticket);
  if (!r) return EIG_ERR_ARG;
  *done = r->done ? 1 : 0;
  if (r->done) {
    if (status) *status = r->status;
    if (times) {
      times[0] = r->t_start - r->t_submit;   // queue wait
      times[1] = r->t_end - r->t_start;      // service
      times[2] = r->t_end - r->t_submit;     // latency
    }
    if (info) *info = r->info;
  }
  return EIG_OK;
}

int eig_server_cancel(eig_server_t S, uint64_t ticket) {
  if (!S) return EIG_ERR_ARG;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    Request* r = find_request(S, ticket);
    if (!r) return EIG_ERR_ARG;
    auto it = std::find(S->queue.begin(), S->queue.end(), r);
    if (it == S->queue.end()) return 0;   // started or finished: left to run
    S->queue.erase(it);
    r->status = EIG_CANCELLED;
    r->t_start = r->t_end = now_s();
    r->done = true;
  }
  S->cv_done.notify_all();
  S->cv_work.notify_all();   // the new head of the queue may fit the budget
  return 1;
}

int eig_server_wait(eig_server_t S, uint64_t ticket, double timeout_s, int* status) {
  if (!S) return EIG_ERR_ARG;
  std::unique_lock<std::mutex> lock(S->mu);
  Request* r = find_request(S, ticket);
  if (!r) return EIG_ERR_ARG;
  const bool ok = S->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s),
                                      [&] { return r->done; });
  if (!ok) return EIG_TIMEOUT;
  if (status) *status = r->status;
  return EIG_OK;
}

int eig_server_stats(eig_server_t S, unsigned long long* completed, unsigned long long* pending,
                     double* reserved_gb, double* peak_reserved_gb) {
  if (!S) return EIG_ERR_ARG;
  std::lock_guard<std::mutex> lock(S->mu);
  if (completed) *completed = S->completed;
  if (pending) *pending = S->queue.size();
  if (reserved_gb) *reserved_gb = S->reserved / 1e9;
  if (peak_reserved_gb) *peak_reserved_gb = S->peak_reserved / 1e9;
  return EIG_OK;
}

int eig_server_destroy(eig_server_t S) {
  if (!S) return EIG_ERR_ARG;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->threads) t.join();
  cudaSetDevice(S->device);
  for (eig_handle_s* w : S->workers) {
    cudaStreamSynchronize(w->stream);
    if (w->ws) cudaFree(w->ws);
    if (w->pinned) cudaFreeHost(w->pinned);
    clear_graphs(w);
    cudaStreamDestroy(w->stream);
    delete w;
  }
  for (Request* r : S->all) delete r;
  delete S;
  return EIG_OK;
}

}  // extern "C"
