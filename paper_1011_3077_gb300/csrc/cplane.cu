// Complex-plane strategy for the nonsymmetric problem (Sec. 3.3) on sm_103a.
//
// Splitting lines at random angles separate eigenvalues that real lines
// cannot (a conjugate pair, a spectrum along the imaginary axis), so this
// path runs in complex arithmetic.  Complex matrices are interleaved
// (re, im) FP64 pairs, column-major, leading dimensions in complex elements.
//
// One step on the line {z : Re(conj(w) z) = t}, |w| = 1, scale s:
//   (A_0, B_0) = (A - w (t - s) I, A - w (t + s) I)   rotated Moebius map;
//   IRS over C (Algorithm 3): QR of [B_j; -A_j], A_{j+1} = Q12^H A_j,
//   B_{j+1} = Q22^H B_j, until ||R_j - R_{j-1}||_1 <= tau ||R_{j-1}||_1;
//   splitter Q = GRURV(2, A_p + B_p, A_p, -1, +1) with a Haar unitary V
//   (Algorithm 2): A_p V^H = U R2, then the RQ of U^H (A_p + B_p) through
//   the QR of (A_p + B_p)^H U J (J reverses columns): Q = Z~ J;
//   A^ = Q^H A Q and the 1-norm split test (Algorithm 5).
// The leading k columns of Q span the invariant subspace of the eigenvalues
// with Re(conj(w) z) > t.
//
// QR convention: reflector v = x + e^{i phi} ||x|| e1 (x0 = |x0| e^{i phi}),
// normalised to u = v / v0 with tau = 1 + |x0| / ||x||, then a diagonal
// unitary makes diag(R) real and non-negative; that QR is unique, so R_j and
// the splitter agree with any other implementation of the same definition.
//
// Recursion (Sec. 3.3): the disk |z - c| <= R of a node (root: Gershgorin
// about c = tr(A)/n; after a split the smaller of ||A_ii - cI||_F about the
// block's mean eigenvalue and the enclosing circle of its side), a random angle theta = 2 pi u2 and offset
// a = R (u1 - 1/2) from Philox purpose 8; a step that finds one side empty
// chops it off; the region (disk cut by the chopped half-planes) moves to its
// enclosing circle at once when that shrinks the radius to sin(5 pi/12) R or
// less, else the next line is perpendicular and the second chop recenters
// (the 2-step rule).  A node that fails max_fail times is a cluster: with
// `enclose` it is reported with its region (Sec. 3.3 remarks on convex
// enclosures of pseudospectra) and solved by the leaf solver, otherwise the
// solve stops with EIG_NO_SPLIT.  Leaves: complex Hessenberg reduction and
// single-shift QR with Wilkinson shifts, one CTA per leaf.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/eigdc.h"
#include "cplane_strategy.h"
#include "internal.h"

namespace eigdc {
namespace {

typedef double2 zt;

constexpr int PURPOSE_HAAR_RE = 4;
constexpr int PURPOSE_HAAR_IM = 7;
constexpr int PURPOSE_LINE = 8;
constexpr int ZNB = 32;           // panel width of the complex QR (T leading dimension)
constexpr int ZLEAF_MAX = 64;     // largest leaf of the complex Schur kernel
// Largest cluster put in Schur form by the global-memory leaf solver (one CTA,
// O(m^3) serial-ish work: m = 512 is about 0.2 s).  A larger cluster is still
// reported with its enclosure, and the solve returns EIG_NO_SPLIT.
constexpr int ZLEAF_GLOBAL_MAX = 512;

__host__ __device__ __forceinline__ zt zmk(double r, double i) { return make_double2(r, i); }
__device__ __forceinline__ zt zadd(zt a, zt b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ zt zsub(zt a, zt b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ zt zconj(zt a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ zt zmul(zt a, zt b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// c + a b
__device__ __forceinline__ zt zfma(zt a, zt b, zt c) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
// c + conj(a) b
__device__ __forceinline__ zt zcfma(zt a, zt b, zt c) {
  return make_double2(fma(a.x, b.x, fma(a.y, b.y, c.x)), fma(a.x, b.y, fma(-a.y, b.x, c.y)));
}
__device__ __forceinline__ zt zscale(double s, zt a) { return make_double2(s * a.x, s * a.y); }
__device__ __forceinline__ double zabs(zt a) { return hypot(a.x, a.y); }

int nblocks(long long count, int per) { return (int)((count + per - 1) / per); }

// ------------------------------------------------------------------ ZGEMM
// C = alpha op(A) op(B) + beta C, op(X) = X or X^H.  64 x 64 tile per CTA,
// 256 threads, 4 x 4 complex outputs per thread, K slabs of 8 in shared memory.
constexpr int ZBM = 64, ZBN = 64, ZBK = 8;

// With gridDim.z > 1 (split-K), CTA z takes K in [z kchunk, (z+1) kchunk) and
// writes its partial alpha op(A) op(B) to C + z pstride (beta is then 0).
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) zgemm_kernel(int m, int n, int k, zt alpha,
                                                    const zt* __restrict__ A, int lda,
                                                    const zt* __restrict__ B, int ldb, zt beta,
                                                    zt* __restrict__ C, int ldc, int kchunk,
                                                    size_t pstride) {
  __shared__ zt As[ZBK][ZBM + 1];
  __shared__ zt Bs[ZBK][ZBN + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int row0 = blockIdx.x * ZBM, col0 = blockIdx.y * ZBN;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(k, kbeg + kchunk);
  C += blockIdx.z * pstride;
  zt acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = zmk(0.0, 0.0);
  for (int k0 = kbeg; k0 < kend; k0 += ZBK) {
    for (int e = tid; e < ZBK * ZBM; e += 256) {
      int r, kk;
      if (!TA) { r = e % ZBM; kk = e / ZBM; } else { kk = e % ZBK; r = e / ZBK; }
      const int gr = row0 + r, gk = k0 + kk;
      zt v = zmk(0.0, 0.0);
      if (gr < m && gk < kend) v = TA ? zconj(A[gk + (size_t)gr * lda]) : A[gr + (size_t)gk * lda];
      As[kk][r] = v;
    }
    for (int e = tid; e < ZBK * ZBN; e += 256) {
      int c, kk;
      if (!TB) { kk = e % ZBK; c = e / ZBK; } else { c = e % ZBN; kk = e / ZBN; }
      const int gc = col0 + c, gk = k0 + kk;
      zt v = zmk(0.0, 0.0);
      if (gc < n && gk < kend) v = TB ? zconj(B[gc + (size_t)gk * ldb]) : B[gk + (size_t)gc * ldb];
      Bs[kk][c] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < ZBK; ++kk) {
      zt a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = zfma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  const bool use_c = beta.x != 0.0 || beta.y != 0.0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = row0 + ty + 16 * i;
    if (r >= m) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = col0 + tx + 16 * j;
      if (c >= n) continue;
      zt v = zmul(alpha, acc[i][j]);
      if (use_c) v = zfma(beta, C[r + (size_t)c * ldc], v);
      C[r + (size_t)c * ldc] = v;
    }
  }
}

// C = sum_z P[z] (in z order) + beta C; P[z] is m x n with leading dimension m
__global__ void zreduce_kernel(int m, int n, int splits, const zt* __restrict__ P, size_t pstride,
                               zt beta, zt* __restrict__ C, int ldc) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)m * n) return;
  const int i = (int)(e % m), j = (int)(e / m);
  zt v = P[e];
  for (int z = 1; z < splits; ++z) v = zadd(v, P[e + z * pstride]);
  if (beta.x != 0.0 || beta.y != 0.0) v = zfma(beta, C[i + (size_t)j * ldc], v);
  C[i + (size_t)j * ldc] = v;
}

void zgemm_launch(cudaStream_t s, bool ta, bool tb, dim3 g, int m, int n, int k, zt alpha,
                  const zt* A, int lda, const zt* B, int ldb, zt beta, zt* C, int ldc, int kchunk,
                  size_t pstride) {
  note_launches(1);
  if (!ta && !tb)
    zgemm_kernel<false, false><<<g, 256, 0, s>>>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, kchunk, pstride);
  else if (ta && !tb)
    zgemm_kernel<true, false><<<g, 256, 0, s>>>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, kchunk, pstride);
  else if (!ta && tb)
    zgemm_kernel<false, true><<<g, 256, 0, s>>>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, kchunk, pstride);
  else
    zgemm_kernel<true, true><<<g, 256, 0, s>>>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, kchunk, pstride);
}

}  // namespace

cudaError_t zgemm(cudaStream_t s, bool ta, bool tb, int m, int n, int k, double2 alpha,
                  const double2* A, int lda, const double2* B, int ldb, double2 beta, double2* C,
                  int ldc) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  dim3 g(nblocks(m, ZBM), nblocks(n, ZBN), 1);
  zgemm_launch(s, ta, tb, g, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, std::max(k, 1), 0);
  return cudaGetLastError();
}

namespace {

// Splits of K for a product whose tile grid is small: about two CTAs per SM
// (152 SMs) without chunks shorter than 256.
int zsplits(int m, int n, int k) {
  const long long tiles = (long long)nblocks(m, ZBM) * nblocks(n, ZBN);
  int sp = (int)std::min<long long>(16, std::max<long long>(1, 304 / std::max<long long>(tiles, 1)));
  sp = std::min(sp, std::max(1, k / 256));
  return sp;
}

// zgemm with split-K partials in `partial` (capacity `cap` complex entries);
// falls back to one pass when the partials do not fit.
cudaError_t zgemm_sk(cudaStream_t s, bool ta, bool tb, int m, int n, int k, zt alpha, const zt* A,
                     int lda, const zt* B, int ldb, zt beta, zt* C, int ldc, zt* partial, size_t cap) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  int sp = zsplits(m, n, k);
  const size_t pstride = (size_t)m * n;
  if (!partial || (size_t)sp * pstride > cap) sp = 1;
  if (sp == 1) return zgemm(s, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
  const int kchunk = ((k + sp - 1) / sp + ZBK - 1) / ZBK * ZBK;
  sp = (k + kchunk - 1) / kchunk;
  dim3 g(nblocks(m, ZBM), nblocks(n, ZBN), sp);
  zgemm_launch(s, ta, tb, g, m, n, k, alpha, A, lda, B, ldb, zmk(0.0, 0.0), partial, m, kchunk, pstride);
  note_launches(1);
  zreduce_kernel<<<nblocks((long long)m * n, 256), 256, 0, s>>>(m, n, sp, partial, pstride, beta, C, ldc);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ elementwise
// B = A (rows x cols)
__global__ void zcopy_kernel(int rows, int cols, const zt* __restrict__ A, int lda,
                             zt* __restrict__ B, int ldb) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)rows * cols) return;
  const int i = (int)(e % rows), j = (int)(e / rows);
  B[i + (size_t)j * ldb] = A[i + (size_t)j * lda];
}

cudaError_t zcopy(cudaStream_t s, int rows, int cols, const zt* A, int lda, zt* B, int ldb) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  note_launches(1);
  zcopy_kernel<<<nblocks((long long)rows * cols, 256), 256, 0, s>>>(rows, cols, A, lda, B, ldb);
  return cudaGetLastError();
}

// A0 = A - w (t - s) I, B0 = A - w (t + s) I
__global__ void zline_map_kernel(int n, const zt* __restrict__ A, int lda, zt s0, zt s1,
                                 zt* __restrict__ A0, zt* __restrict__ B0) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  const int i = (int)(e % n), j = (int)(e / n);
  zt a = A[i + (size_t)j * lda];
  zt b = a;
  if (i == j) {
    a = zsub(a, s0);
    b = zsub(b, s1);
  }
  A0[e] = a;
  B0[e] = b;
}

// W (2n x n) = [B; -A]
__global__ void zstack_kernel(int n, const zt* __restrict__ A, const zt* __restrict__ B,
                              zt* __restrict__ W) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  const int i = (int)(e % n), j = (int)(e / n);
  const zt a = A[e];
  W[i + (size_t)j * 2 * n] = B[e];
  W[n + i + (size_t)j * 2 * n] = zmk(-a.x, -a.y);
}

// E (rows x cols) = identity block at row offset r0: E_ij = [i - r0 == j]
__global__ void zident_kernel(int rows, int cols, int r0, zt* __restrict__ E) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)rows * cols) return;
  const int i = (int)(e % rows), j = (int)(e / rows);
  E[e] = zmk(i - r0 == j ? 1.0 : 0.0, 0.0);
}

cudaError_t zident(cudaStream_t s, int rows, int cols, int r0, zt* E) {
  note_launches(1);
  zident_kernel<<<nblocks((long long)rows * cols, 256), 256, 0, s>>>(rows, cols, r0, E);
  return cudaGetLastError();
}

// C = A + B (n x n, packed)
__global__ void zadd_kernel(long long count, const zt* __restrict__ A, const zt* __restrict__ B,
                            zt* __restrict__ C) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count) C[e] = zadd(A[e], B[e]);
}

// B = A J (columns reversed), rows x n packed
__global__ void zrevcols_kernel(int rows, int n, const zt* __restrict__ A, zt* __restrict__ B) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)rows * n) return;
  const int i = (int)(e % rows), j = (int)(e / rows);
  B[i + (size_t)(n - 1 - j) * rows] = A[e];
}

// G = Gre + i Gim
__global__ void zinterleave_kernel(long long count, const double* __restrict__ re,
                                   const double* __restrict__ im, zt* __restrict__ G) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count) G[e] = zmk(re[e], im[e]);
}

// M = |A| (n x n packed, real)
__global__ void zabs_kernel(long long count, const zt* __restrict__ A, double* __restrict__ M) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count) M[e] = zabs(A[e]);
}

// T = upper triangle of A (n x n), zero below; w = diag(A)
__global__ void ztriu_kernel(int n, const zt* __restrict__ A, int lda, zt* __restrict__ T, int ldt,
                             zt* __restrict__ w) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  const int i = (int)(e % n), j = (int)(e / n);
  const zt v = A[i + (size_t)j * lda];
  T[i + (size_t)j * ldt] = i <= j ? v : zmk(0.0, 0.0);
  if (i == j && w) w[i] = v;
}

// colsum[j] = sum_i |A_ij - [i == j] c| for j < cols; one CTA per column, fixed order.
__global__ void zcolabs_kernel(int rows, int cols, const zt* __restrict__ A, int lda, zt c,
                               double* __restrict__ colsum) {
  __shared__ double red[8];
  const int j = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < rows; i += 256) {
    zt v = A[i + (size_t)j * lda];
    if (i == j) v = zsub(v, c);
    acc += zabs(v);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    colsum[j] = t;
  }
}

// colsum[j] = sum_i |A_ij - [i == j] c|^2; one CTA per column, fixed order.
__global__ void zcolsq_kernel(int rows, const zt* __restrict__ A, int lda, zt c,
                              double* __restrict__ colsum) {
  __shared__ double red[8];
  const int j = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < rows; i += 256) {
    zt v = A[i + (size_t)j * lda];
    if (i == j) v = zsub(v, c);
    acc += v.x * v.x + v.y * v.y;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    colsum[j] = t;
  }
}

// rowsum[i] = sum_j |A_ij - [i == j] c|
__global__ void zrowabs_kernel(int n, const zt* __restrict__ A, int lda, zt c,
                               double* __restrict__ rowsum) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = 0.0;
  for (int j = 0; j < n; ++j) {
    zt v = A[i + (size_t)j * lda];
    if (i == j) v = zsub(v, c);
    acc += zabs(v);
  }
  rowsum[i] = acc;
}

// colsum[j] = sum_i |A_ij - B_ij| (upper triangles of two n x n R factors)
__global__ void zcoldiff_kernel(int n, const zt* __restrict__ A, const zt* __restrict__ B,
                                double* __restrict__ colsum) {
  __shared__ double red[8];
  const int j = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) acc += zabs(zsub(A[i + (size_t)j * n], B[i + (size_t)j * n]));
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    colsum[j] = t;
  }
}

// ------------------------------------------------------------------ complex QR
// Panel factorisation of the m x jb panel P in place (one CTA, 512 threads):
// R on and above the diagonal (before the phase fix), u below it (u_j = 1
// implicit), tau[j] real.
constexpr int ZP_THREADS = 256;
constexpr int ZP_WARPS = ZP_THREADS / 32;

__device__ double zp_block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < ZP_WARPS; ++w) t += red[w];
  return t;
}

__global__ void __launch_bounds__(ZP_THREADS) zpanel_kernel(int m, int jb, zt* __restrict__ P,
                                                            int ldp, double* __restrict__ tau) {
  __shared__ double red[ZP_WARPS];
  __shared__ zt part[ZP_WARPS][ZNB + 1];
  __shared__ zt dots[ZNB];
  __shared__ zt s_inv_v0;
  __shared__ double s_tau;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int j = 0; j < jb; ++j) {
    zt* x = P + (size_t)j * ldp;
    double ss = 0.0;
    for (int r = j + tid; r < m; r += ZP_THREADS) ss += x[r].x * x[r].x + x[r].y * x[r].y;
    ss = zp_block_sum(ss, red);
    if (tid == 0) {
      const double nrm = sqrt(ss);
      const zt x0 = x[j];
      const double a0 = zabs(x0);
      if (nrm == 0.0) {
        s_tau = 0.0;
        s_inv_v0 = zmk(0.0, 0.0);
      } else {
        const zt ph = a0 > 0.0 ? zmk(x0.x / a0, x0.y / a0) : zmk(1.0, 0.0);
        const double mag = a0 + nrm;                 // v0 = ph (|x0| + ||x||)
        s_inv_v0 = zmk(ph.x / mag, -ph.y / mag);     // 1 / v0 = conj(ph) / mag
        s_tau = mag / nrm;                           // 1 + |x0| / ||x||
        x[j] = zmk(-ph.x * nrm, -ph.y * nrm);        // beta = -ph ||x||
      }
      tau[j] = s_tau;
    }
    __syncthreads();
    const double tj = s_tau;
    if (tj == 0.0) continue;                         // uniform across the block
    const zt iv = s_inv_v0;
    for (int r = j + 1 + tid; r < m; r += ZP_THREADS) x[r] = zmul(x[r], iv);
    __syncthreads();
    const int nc = jb - j - 1;
    if (nc <= 0) continue;
    // dots_c = sum_r conj(u_r) P[r, j+1+c]
    zt acc[ZNB];
#pragma unroll
    for (int c = 0; c < ZNB; ++c) acc[c] = zmk(0.0, 0.0);
    for (int r = j + tid; r < m; r += ZP_THREADS) {
      const zt u = r == j ? zmk(1.0, 0.0) : x[r];
#pragma unroll
      for (int c = 0; c < ZNB; ++c)
        if (c < nc) acc[c] = zcfma(u, P[r + (size_t)(j + 1 + c) * ldp], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < ZNB; ++c) {
      if (c < nc) {
        double re = acc[c].x, im = acc[c].y;
        for (int o = 16; o > 0; o >>= 1) {
          re += __shfl_down_sync(0xffffffffu, re, o);
          im += __shfl_down_sync(0xffffffffu, im, o);
        }
        if (lane == 0) part[warp][c] = zmk(re, im);
      }
    }
    __syncthreads();
    if (tid < nc) {
      zt t = zmk(0.0, 0.0);
      for (int w = 0; w < ZP_WARPS; ++w) t = zadd(t, part[w][tid]);
      dots[tid] = zscale(tj, t);
    }
    __syncthreads();
    for (int r = j + tid; r < m; r += ZP_THREADS) {
      const zt u = r == j ? zmk(1.0, 0.0) : x[r];
      for (int c = 0; c < nc; ++c) {
        zt* pc = P + r + (size_t)(j + 1 + c) * ldp;
        *pc = zsub(*pc, zmul(u, dots[c]));
      }
    }
    __syncthreads();
  }
}

// V (m x jb) explicit: 1 on the diagonal, 0 above, u below (from the panel).
__global__ void zextract_v_kernel(int m, int jb, const zt* __restrict__ P, int ldp,
                                  zt* __restrict__ V, int ldv) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)m * jb) return;
  const int r = (int)(e % m), c = (int)(e / m);
  V[r + (size_t)c * ldv] = r < c ? zmk(0.0, 0.0) : (r == c ? zmk(1.0, 0.0) : P[r + (size_t)c * ldp]);
}

// Partial Gram matrices of V over chunks of 64 rows: part[chunk][i + 32 j] = sum conj(V_ri) V_rj.
__global__ void __launch_bounds__(1024) zgram_kernel(int m, int jb, const zt* __restrict__ V,
                                                     int ldv, zt* __restrict__ part) {
  __shared__ zt Vs[64][ZNB + 1];
  const int r0 = blockIdx.x * 64;
  for (int e = threadIdx.x; e < 64 * ZNB; e += 1024) {
    const int r = e % 64, c = e / 64;
    Vs[r][c] = (r0 + r < m && c < jb) ? V[r0 + r + (size_t)c * ldv] : zmk(0.0, 0.0);
  }
  __syncthreads();
  const int i = threadIdx.x % 32, j = threadIdx.x / 32;
  zt s = zmk(0.0, 0.0);
  for (int r = 0; r < 64; ++r) s = zcfma(Vs[r][i], Vs[r][j], s);
  part[(size_t)blockIdx.x * 1024 + i + 32 * j] = s;
}

// T (jb x jb upper, ld ZNB) of H_0 .. H_{jb-1} = I - V T V^H from the Gram partials:
// T_cc = tau_c, T(0:c, c) = -tau_c T(0:c, 0:c) G(0:c, c).
__global__ void __launch_bounds__(1024) zlarft_kernel(int nchunks, int jb, const zt* __restrict__ part,
                                                      const double* __restrict__ tau,
                                                      zt* __restrict__ T) {
  __shared__ zt G[ZNB][ZNB + 1];
  __shared__ zt Ts[ZNB][ZNB + 1];
  const int i = threadIdx.x % 32, j = threadIdx.x / 32;
  zt s = zmk(0.0, 0.0);
  for (int ch = 0; ch < nchunks; ++ch) s = zadd(s, part[(size_t)ch * 1024 + i + 32 * j]);
  G[i][j] = s;
  Ts[i][j] = zmk(0.0, 0.0);
  __syncthreads();
  for (int c = 0; c < jb; ++c) {
    if (threadIdx.x < c) {
      const int r = threadIdx.x;
      zt acc = zmk(0.0, 0.0);
      for (int q = r; q < c; ++q) acc = zfma(Ts[r][q], G[q][c], acc);
      Ts[r][c] = zscale(-tau[c], acc);
    } else if (threadIdx.x == c) {
      Ts[c][c] = zmk(tau[c], 0.0);
    }
    __syncthreads();
  }
  // only the jb columns of this panel exist in the caller's T (ZNB x n)
  if (j < jb) T[i + ZNB * j] = i < jb ? Ts[i][j] : zmk(0.0, 0.0);
}

// R (n x n, ld ldr) = D^H triu(P(0:n, 0:n)) with D = diag(phase of P_jj); phases[j] = D_jj.
__global__ void zr_extract_kernel(int n, const zt* __restrict__ P, int ldp, zt* __restrict__ R,
                                  int ldr, zt* __restrict__ phases) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  const int i = (int)(e % n), j = (int)(e / n);
  const zt d = P[i + (size_t)i * ldp];
  const double ad = zabs(d);
  const zt ph = ad > 0.0 ? zmk(d.x / ad, d.y / ad) : zmk(1.0, 0.0);
  zt v = zmk(0.0, 0.0);
  if (i < j) v = zmul(zconj(ph), P[i + (size_t)j * ldp]);
  else if (i == j) v = zmk(ad, 0.0);
  if (R) R[i + (size_t)j * ldr] = v;
  if (j == 0 && phases) phases[i] = ph;
}

// rows 0..n-1 of E (rows x cols, packed) scaled by phases
__global__ void zscale_rows_kernel(int rows, int cols, int n, const zt* __restrict__ ph,
                                   zt* __restrict__ E) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)rows * cols) return;
  const int i = (int)(e % rows);
  if (i < n) E[e] = zmul(ph[i], E[e]);
}

// Workspace of one complex QR of an m x n matrix (m >= n).
struct ZQR {
  zt* V;        // m x n explicit reflectors (column block p holds rows p*ZNB.. meaningful)
  zt* T;        // ZNB x n: T of each panel
  double* tau;  // n
  zt* phases;   // n
  zt* W1;       // ZNB x n
  zt* W2;       // ZNB x n
  zt* gram;     // ceil(m / 64) x 1024
  zt* part = nullptr;   // split-K partials of the V^H C products
  size_t part_cap = 0;  // complex entries
  int m, n;
};

// Householder QR of P (m x n, ld ldp) in place; R (phase-fixed) to R if given.
cudaError_t zgeqrf(cudaStream_t s, int m, int n, zt* P, int ldp, const ZQR& q, zt* R, int ldr) {
  const zt one = zmk(1.0, 0.0), zero = zmk(0.0, 0.0), mone = zmk(-1.0, 0.0);
  for (int j0 = 0; j0 < n; j0 += ZNB) {
    const int jb = std::min(ZNB, n - j0);
    const int mm = m - j0;
    zt* Pp = P + j0 + (size_t)j0 * ldp;
    note_launches(1);
    zpanel_kernel<<<1, ZP_THREADS, 0, s>>>(mm, jb, Pp, ldp, q.tau + j0);
    zt* Vp = q.V + j0 + (size_t)j0 * m;
    note_launches(1);
    zextract_v_kernel<<<nblocks((long long)mm * jb, 256), 256, 0, s>>>(mm, jb, Pp, ldp, Vp, m);
    const int nch = nblocks(mm, 64);
    note_launches(1);
    zgram_kernel<<<nch, 1024, 0, s>>>(mm, jb, Vp, m, q.gram);
    zt* Tp = q.T + (size_t)j0 * ZNB;
    note_launches(1);
    zlarft_kernel<<<1, 1024, 0, s>>>(nch, jb, q.gram, q.tau + j0, Tp);
    const int nc = n - j0 - jb;
    if (nc > 0) {
      zt* C = P + j0 + (size_t)(j0 + jb) * ldp;
      cudaError_t e;
      if ((e = zgemm_sk(s, true, false, jb, nc, mm, one, Vp, m, C, ldp, zero, q.W1, ZNB, q.part,
                        q.part_cap)) != cudaSuccess) return e;
      if ((e = zgemm(s, true, false, jb, nc, jb, one, Tp, ZNB, q.W1, ZNB, zero, q.W2, ZNB)) != cudaSuccess) return e;
      if ((e = zgemm(s, false, false, mm, nc, jb, mone, Vp, m, q.W2, ZNB, one, C, ldp)) != cudaSuccess) return e;
    }
  }
  note_launches(1);
  zr_extract_kernel<<<nblocks((long long)n * n, 256), 256, 0, s>>>(n, P, ldp, R, ldr, q.phases);
  return cudaGetLastError();
}

// E <- Q E for the Q of the last zgeqrf (E is m x c, packed); phase_fix
// applies the diagonal unitary first (needed when E touches the first n rows).
cudaError_t zapply_q(cudaStream_t s, const ZQR& q, zt* E, int c, bool phase_fix) {
  const int m = q.m, n = q.n;
  const zt one = zmk(1.0, 0.0), zero = zmk(0.0, 0.0), mone = zmk(-1.0, 0.0);
  if (phase_fix) {
    note_launches(1);
    zscale_rows_kernel<<<nblocks((long long)m * c, 256), 256, 0, s>>>(m, c, n, q.phases, E);
  }
  const int np = nblocks(n, ZNB);
  for (int p = np - 1; p >= 0; --p) {
    const int j0 = p * ZNB, jb = std::min(ZNB, n - j0), mm = m - j0;
    const zt* Vp = q.V + j0 + (size_t)j0 * m;
    const zt* Tp = q.T + (size_t)j0 * ZNB;
    zt* Ep = E + j0;
    cudaError_t e;
    if ((e = zgemm_sk(s, true, false, jb, c, mm, one, Vp, m, Ep, m, zero, q.W1, ZNB, q.part,
                      q.part_cap)) != cudaSuccess) return e;
    if ((e = zgemm(s, false, false, jb, c, jb, one, Tp, ZNB, q.W1, ZNB, zero, q.W2, ZNB)) != cudaSuccess) return e;
    if ((e = zgemm(s, false, false, mm, c, jb, mone, Vp, m, q.W2, ZNB, one, Ep, m)) != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------ complex Schur leaves
struct ZLeafDesc {
  int m;
  const zt* A;   // m x m, ld lda
  int lda;
  zt* T;         // m x m, ld m
  zt* Z;         // m x m, ld m
  int* status;   // 0 ok, 1 iteration budget spent
  zt* work;      // zschur_leaf_global_kernel only: 2 m^2 + 2 m complex
};

__device__ void zleaf_givens(zt a, zt b, zt* G) {
  const double rho = sqrt(a.x * a.x + a.y * a.y + b.x * b.x + b.y * b.y);
  if (rho == 0.0) {
    G[0] = zmk(1.0, 0.0); G[1] = zmk(0.0, 0.0); G[2] = zmk(0.0, 0.0); G[3] = zmk(1.0, 0.0);
    return;
  }
  // G = [[conj a, conj b], [-b, a]] / rho, row-major G[0] G[1] / G[2] G[3]
  G[0] = zmk(a.x / rho, -a.y / rho);
  G[1] = zmk(b.x / rho, -b.y / rho);
  G[2] = zmk(-b.x / rho, -b.y / rho);
  G[3] = zmk(a.x / rho, a.y / rho);
}

// H <- G_k H G_k^H on indices (k, k+1), Z <- Z G_k^H (all threads take part).
// Storage of a leaf's H and Z: shared memory (m <= ZLEAF_MAX) or global scratch.
struct SharedMat {
  zt (*p)[ZLEAF_MAX + 1];
  __device__ zt& operator()(int i, int j) const { return p[i][j]; }
};
struct GlobalMat {
  zt* p;
  int ld;
  __device__ zt& operator()(int i, int j) const { return p[i + (size_t)j * ld]; }
};

// block-wide scalars of the leaf solver (shared memory)
struct LeafShared {
  zt G[4];
  double tau;
  int lo, hi, act;
};

template <class Mat>
__device__ void zleaf_rotate(int m, Mat H, Mat Z, int k, const zt* G) {
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    const zt h0 = H(k, c), h1 = H(k + 1, c);
    H(k, c) = zfma(G[0], h0, zmul(G[1], h1));
    H(k + 1, c) = zfma(G[2], h0, zmul(G[3], h1));
  }
  __syncthreads();
  // right multiplication by G^H: [x0, x1] G^H = [x0 conj(G0) + x1 conj(G1), x0 conj(G2) + x1 conj(G3)]
  for (int r = threadIdx.x; r < m; r += blockDim.x) {
    const zt h0 = H(r, k), h1 = H(r, k + 1);
    H(r, k) = zadd(zmul(h0, zconj(G[0])), zmul(h1, zconj(G[1])));
    H(r, k + 1) = zadd(zmul(h0, zconj(G[2])), zmul(h1, zconj(G[3])));
    const zt z0 = Z(r, k), z1 = Z(r, k + 1);
    Z(r, k) = zadd(zmul(z0, zconj(G[0])), zmul(z1, zconj(G[1])));
    Z(r, k + 1) = zadd(zmul(z0, zconj(G[2])), zmul(z1, zconj(G[3])));
  }
  __syncthreads();
}

// The leaf solver on H, Z (m x m) with the work vectors u, dots (m each).
template <class Mat>
__device__ void zleaf_solve(const ZLeafDesc& d, int m, Mat H, Mat Z, zt* u, zt* dots,
                            LeafShared& sh) {
  zt* G = sh.G;
  double& s_tau = sh.tau;
  int& s_lo = sh.lo;
  int& s_hi = sh.hi;
  int& s_act = sh.act;
  const int tid = threadIdx.x;
  for (int e = tid; e < m * m; e += blockDim.x) {
    const int i = e % m, j = e / m;
    H(i, j) = d.A[i + (size_t)j * d.lda];
    Z(i, j) = zmk(i == j ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  // Householder reduction to Hessenberg form (the reflector convention of the QR)
  for (int k = 0; k + 2 < m; ++k) {
    if (tid == 0) {
      double ss = 0.0;
      for (int r = k + 1; r < m; ++r) ss += H(r, k).x * H(r, k).x + H(r, k).y * H(r, k).y;
      const double nrm = sqrt(ss);
      const zt x0 = H(k + 1, k);
      const double a0 = zabs(x0);
      if (nrm == 0.0) {
        s_tau = 0.0;
      } else {
        const zt ph = a0 > 0.0 ? zmk(x0.x / a0, x0.y / a0) : zmk(1.0, 0.0);
        const double mag = a0 + nrm;
        const zt iv = zmk(ph.x / mag, -ph.y / mag);
        s_tau = mag / nrm;
        u[k + 1] = zmk(1.0, 0.0);
        for (int r = k + 2; r < m; ++r) u[r] = zmul(H(r, k), iv);
      }
    }
    __syncthreads();
    const double tk = s_tau;
    if (tk == 0.0) continue;
    // left: H(k+1:, :) -= tau u (u^H H(k+1:, :))
    for (int c = tid; c < m; c += blockDim.x) {
      zt acc = zmk(0.0, 0.0);
      for (int r = k + 1; r < m; ++r) acc = zcfma(u[r], H(r, c), acc);
      dots[c] = zscale(tk, acc);
    }
    __syncthreads();
    for (int e = tid; e < (m - k - 1) * m; e += blockDim.x) {
      const int r = k + 1 + e % (m - k - 1), c = e / (m - k - 1);
      H(r, c) = zsub(H(r, c), zmul(u[r], dots[c]));
    }
    __syncthreads();
    // right: H(:, k+1:) -= tau (H(:, k+1:) u) u^H, same for Z
    for (int r = tid; r < m; r += blockDim.x) {
      zt ah = zmk(0.0, 0.0), az = zmk(0.0, 0.0);
      for (int c = k + 1; c < m; ++c) {
        ah = zfma(H(r, c), u[c], ah);
        az = zfma(Z(r, c), u[c], az);
      }
      ah = zscale(tk, ah);
      az = zscale(tk, az);
      for (int c = k + 1; c < m; ++c) {
        H(r, c) = zsub(H(r, c), zmul(ah, zconj(u[c])));
        Z(r, c) = zsub(Z(r, c), zmul(az, zconj(u[c])));
      }
    }
    __syncthreads();
    for (int r = k + 2 + tid; r < m; r += blockDim.x) H(r, k) = zmk(0.0, 0.0);
    __syncthreads();
  }
  // single-shift QR with deflation, Wilkinson and exceptional shifts
  int hi = m - 1, its = 0, budget = 40 * max(m, 1);
  int ok = 1;
  while (hi > 0) {
    if (tid == 0) {
      int lo = hi;
      while (lo > 0) {
        double scale = zabs(H(lo - 1, lo - 1)) + zabs(H(lo, lo));
        if (scale == 0.0) {
          scale = 0.0;
          for (int a = lo - 1; a <= hi; ++a)
            for (int b = lo - 1; b <= hi; ++b) scale += zabs(H(a, b));
        }
        if (zabs(H(lo, lo - 1)) <= 0x1p-53 * scale) {
          H(lo, lo - 1) = zmk(0.0, 0.0);
          break;
        }
        --lo;
      }
      s_lo = lo;
      s_act = 0;
      if (lo == hi) {
        s_hi = hi - 1;
      } else {
        s_hi = hi;
        s_act = 1;
        ++its;
        --budget;
        zt mu;
        if (its % 10 == 0) {
          mu = zadd(H(hi, hi), zmk(0.75 * zabs(H(hi, hi - 1)), 0.0));
        } else {
          const zt a = H(hi - 1, hi - 1), b = H(hi - 1, hi), c = H(hi, hi - 1), dd = H(hi, hi);
          const zt tr2 = zscale(0.5, zadd(a, dd));
          const zt hd = zscale(0.5, zsub(a, dd));
          const zt disc2 = zadd(zmul(hd, hd), zmul(b, c));
          // principal complex square root
          const double r = zabs(disc2);
          // hypot may round r a little below |disc2.x| when disc2 is nearly a
          // negative real (a conjugate pair of a real block): clamp both radicands
          double sr = sqrt(0.5 * fmax(r + disc2.x, 0.0));
          double si = sqrt(0.5 * fmax(r - disc2.x, 0.0));
          if (disc2.y < 0.0) si = -si;
          const zt disc = zmk(sr, si);
          const zt l1 = zadd(tr2, disc), l2 = zsub(tr2, disc);
          mu = zabs(zsub(l1, dd)) <= zabs(zsub(l2, dd)) ? l1 : l2;
        }
        zleaf_givens(zsub(H(lo, lo), mu), H(lo + 1, lo), G);
      }
      if (budget < 0) s_act = 2;
    }
    __syncthreads();
    const int act = s_act, lo = s_lo;
    if (act == 2) {
      ok = 0;
      break;
    }
    if (act == 0) {
      hi = s_hi;
      if (tid == 0) its = 0;
      __syncthreads();
      continue;
    }
    zleaf_rotate(m, H, Z, lo, G);
    for (int k = lo + 1; k < hi; ++k) {
      if (tid == 0) zleaf_givens(H(k, k - 1), H(k + 1, k - 1), G);
      __syncthreads();
      zleaf_rotate(m, H, Z, k, G);
      if (tid == 0) H(k + 1, k - 1) = zmk(0.0, 0.0);
      __syncthreads();
    }
  }
  for (int e = tid; e < m * m; e += blockDim.x) {
    const int i = e % m, j = e / m;
    d.T[i + (size_t)j * m] = i <= j ? H(i, j) : zmk(0.0, 0.0);
    d.Z[i + (size_t)j * m] = Z(i, j);
  }
  if (tid == 0) *d.status = ok ? 0 : 1;
}

// Leaves of at most ZLEAF_MAX rows: H and Z in shared memory, one CTA each.
__global__ void __launch_bounds__(256) zschur_leaf_kernel(const ZLeafDesc* __restrict__ desc) {
  extern __shared__ zt zsm[];
  __shared__ zt u[ZLEAF_MAX];
  __shared__ zt dots[ZLEAF_MAX];
  __shared__ LeafShared sh;
  const ZLeafDesc d = desc[blockIdx.x];
  const int m = d.m;
  if (m < 1 || m > ZLEAF_MAX) {   // the shared arrays hold at most ZLEAF_MAX rows
    if (threadIdx.x == 0) *d.status = 1;
    return;
  }
  SharedMat H{reinterpret_cast<zt (*)[ZLEAF_MAX + 1]>(zsm)};
  SharedMat Z{reinterpret_cast<zt (*)[ZLEAF_MAX + 1]>(zsm + ZLEAF_MAX * (ZLEAF_MAX + 1))};
  zleaf_solve(d, m, H, Z, u, dots, sh);
}

// Larger leaves (clusters reported with an enclosure): the same solver with H,
// Z, u and dots in the global scratch d.work (2 m^2 + 2 m complex), one CTA each.
__global__ void __launch_bounds__(256) zschur_leaf_global_kernel(const ZLeafDesc* __restrict__ desc) {
  __shared__ LeafShared sh;
  const ZLeafDesc d = desc[blockIdx.x];
  const int m = d.m;
  if (m < 1 || m > ZLEAF_GLOBAL_MAX || d.work == nullptr) {
    if (threadIdx.x == 0) *d.status = 1;
    return;
  }
  const size_t mm = (size_t)m * m;
  zleaf_solve(d, m, GlobalMat{d.work, m}, GlobalMat{d.work + mm, m}, d.work + 2 * mm,
              d.work + 2 * mm + m, sh);
}

// trace of A (n x n): one CTA, fixed summation order
__global__ void ztrace_kernel(int n, const zt* __restrict__ A, int lda, zt* __restrict__ out) {
  __shared__ zt red[256];
  zt acc = zmk(0.0, 0.0);
  for (int i = threadIdx.x; i < n; i += 256) acc = zadd(acc, A[i + (size_t)i * lda]);
  red[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    zt t = zmk(0.0, 0.0);
    for (int i = 0; i < 256; ++i) t = zadd(t, red[i]);
    *out = t;
  }
}

// U (rows x cols, ld ldu) = identity
__global__ void zident_ld_kernel(int rows, int cols, zt* __restrict__ U, int ldu) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)rows * cols) return;
  const int i = (int)(e % rows), j = (int)(e / rows);
  U[i + (size_t)j * ldu] = zmk(i == j ? 1.0 : 0.0, 0.0);
}

// ------------------------------------------------------------------ geometry (host)
// Region, enclosing circle, lines and the per-node plan: cplane_strategy.h.

// The attempt's line from the Philox pair of purpose PURPOSE_LINE.
HalfPlane draw_line(const Region& g, uint64_t seed, uint64_t node, int attempt, bool has_perp,
                    double pr, double pi_) {
  double u1, u2;
  philox_pair_host(seed, PURPOSE_LINE, node, attempt, &u1, &u2);
  return make_line(g, u1, u2, has_perp, pr, pi_);
}

// ------------------------------------------------------------------ tensor-core route
// EIG_FP64_TC: a large complex product as four FP64-accurate tensor-core
// products of the real and imaginary planes (tcx_gemm, the error-free
// nine-digit split), op(A) = op(Ar) + i sa op(Ai) with sa = -1 for A^H:
//   op(A) op(B) = op(Ar)op(Br) - sa sb op(Ai)op(Bi) + i (sb op(Ar)op(Bi) + sa op(Ai)op(Br)).
struct ZTc {
  bool on = false;
  double* planes = nullptr;   // Ar Ai Br Bi P1 P2 P3 P4, `plane` doubles each
  size_t plane = 0;
  void* ws = nullptr;
  int* err = nullptr;         // bounded-wait error word of the tensor-core kernel
};

__global__ void zsplit_kernel(int rows, int cols, const zt* __restrict__ A, int lda,
                              double* __restrict__ re, double* __restrict__ im) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)rows * cols) return;
  const int i = (int)(e % rows), j = (int)(e / rows);
  const zt v = A[i + (size_t)j * lda];
  re[e] = v.x;
  im[e] = v.y;
}

// C = alpha (P1 - ss P2 + i (sb P3 + sa P4)) + beta C, alpha and beta real
__global__ void zcombine_kernel(int m, int n, double ss, double sa, double sb, double alpha,
                                double beta, const double* __restrict__ P1,
                                const double* __restrict__ P2, const double* __restrict__ P3,
                                const double* __restrict__ P4, zt* __restrict__ C, int ldc) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)m * n) return;
  const int i = (int)(e % m), j = (int)(e / m);
  zt v = zmk(alpha * (P1[e] - ss * P2[e]), alpha * (sb * P3[e] + sa * P4[e]));
  if (beta != 0.0) v = zadd(v, zscale(beta, C[i + (size_t)j * ldc]));
  C[i + (size_t)j * ldc] = v;
}

bool ztc_worth(const ZTc& tc, int m, int n, int k, zt alpha, zt beta) {
  return tc.on && m >= 128 && n >= 128 && k >= 128 && (double)m * n * k >= 33554432.0 &&
         alpha.y == 0.0 && beta.y == 0.0 && (size_t)m * k <= tc.plane &&
         (size_t)k * n <= tc.plane && (size_t)m * n <= tc.plane;
}

// zgemm, or the tensor-core route for large products when it is on
cudaError_t zmm(cudaStream_t s, const ZTc& tc, bool ta, bool tb, int m, int n, int k, zt alpha,
                const zt* A, int lda, const zt* B, int ldb, zt beta, zt* C, int ldc) {
  if (!ztc_worth(tc, m, n, k, alpha, beta))
    return zgemm(s, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
  const int ra = ta ? k : m, ca = ta ? m : k, rb = tb ? n : k, cb = tb ? k : n;
  double* Ar = tc.planes;
  double* Ai = Ar + tc.plane;
  double* Br = Ai + tc.plane;
  double* Bi = Br + tc.plane;
  double* P1 = Bi + tc.plane;
  double* P2 = P1 + tc.plane;
  double* P3 = P2 + tc.plane;
  double* P4 = P3 + tc.plane;
  note_launches(2);
  zsplit_kernel<<<nblocks((long long)ra * ca, 256), 256, 0, s>>>(ra, ca, A, lda, Ar, Ai);
  zsplit_kernel<<<nblocks((long long)rb * cb, 256), 256, 0, s>>>(rb, cb, B, ldb, Br, Bi);
  cudaError_t e;
  if ((e = tcx_gemm(s, ta, tb, m, n, k, 1.0, Ar, ra, Br, rb, 0.0, P1, m, tc.ws, tc.err)) != cudaSuccess) return e;
  if ((e = tcx_gemm(s, ta, tb, m, n, k, 1.0, Ai, ra, Bi, rb, 0.0, P2, m, tc.ws, tc.err)) != cudaSuccess) return e;
  if ((e = tcx_gemm(s, ta, tb, m, n, k, 1.0, Ar, ra, Bi, rb, 0.0, P3, m, tc.ws, tc.err)) != cudaSuccess) return e;
  if ((e = tcx_gemm(s, ta, tb, m, n, k, 1.0, Ai, ra, Br, rb, 0.0, P4, m, tc.ws, tc.err)) != cudaSuccess) return e;
  const double sa = ta ? -1.0 : 1.0, sb = tb ? -1.0 : 1.0;
  note_launches(1);
  zcombine_kernel<<<nblocks((long long)m * n, 256), 256, 0, s>>>(m, n, sa * sb, sa, sb, alpha.x, beta.x,
                                                               P1, P2, P3, P4, C, ldc);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ driver (host)
struct ZFail {
  int code;
};

struct CDriver {
  cudaStream_t s;
  std::string* err;
  std::vector<void*> owned;    // stream-ordered allocations freed at the end

  void check(cudaError_t e, const char* what) {
    if (e != cudaSuccess) {
      *err = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
      throw ZFail{EIG_ERR_CUDA};
    }
  }
  template <class T>
  T* alloc(size_t count) {
    void* p = nullptr;
    if (cudaMallocAsync(&p, std::max<size_t>(count * sizeof(T), 256), s) != cudaSuccess) {
      cudaGetLastError();
      *err = "complex-plane workspace allocation failed";
      throw ZFail{EIG_ERR_NOMEM};
    }
    owned.push_back(p);
    return static_cast<T*>(p);
  }
  ~CDriver() {
    cudaStreamSynchronize(s);
    for (void* p : owned) cudaFreeAsync(p, s);
    cudaStreamSynchronize(s);
  }
  void sync() { check(cudaStreamSynchronize(s), "stream synchronize"); }
};

// Buffers of one divide step, sized for nodes of up to `cap` rows.
struct StepBufs {
  int cap = 0;
  zt *A0, *B0, *A1, *B1, *W, *E, *Ra, *Rb;
  zt *Vh, *X, *U, *Ur, *S, *Z, *Q, *AQ, *Ahat, *R1, *R2, *tmp;
  double *Gre, *Gim, *absA, *colpart, *scores, *col1, *col2;
  ZQR q;   // V (2 cap x cap), T, tau, phases, W1, W2, gram
  ZTc tc;  // tensor-core route of the large products (EIG_FP64_TC)
};

void make_bufs(CDriver& D, StepBufs& b, int cap, bool tensor_cores) {
  const size_t c2 = (size_t)cap * cap;
  b.cap = cap;
  b.A0 = D.alloc<zt>(c2); b.B0 = D.alloc<zt>(c2); b.A1 = D.alloc<zt>(c2); b.B1 = D.alloc<zt>(c2);
  b.W = D.alloc<zt>(2 * c2); b.E = D.alloc<zt>(2 * c2);
  b.Ra = D.alloc<zt>(c2); b.Rb = D.alloc<zt>(c2);
  b.Vh = D.alloc<zt>(c2); b.X = D.alloc<zt>(c2); b.U = D.alloc<zt>(c2); b.Ur = D.alloc<zt>(c2);
  b.S = D.alloc<zt>(c2); b.Z = D.alloc<zt>(c2); b.Q = D.alloc<zt>(c2); b.AQ = D.alloc<zt>(c2);
  b.Ahat = D.alloc<zt>(c2); b.R1 = D.alloc<zt>(c2); b.R2 = D.alloc<zt>(c2);
  b.tmp = D.alloc<zt>(c2);
  b.Gre = D.alloc<double>(c2); b.Gim = D.alloc<double>(c2); b.absA = D.alloc<double>(c2);
  const int nrb = (cap + 31) / 32;
  b.colpart = D.alloc<double>((size_t)(nrb + 1) * cap + 8);
  b.scores = D.alloc<double>(cap + 1);
  b.col1 = D.alloc<double>(cap + 1);
  b.col2 = D.alloc<double>(cap + 1);
  b.q.V = D.alloc<zt>(2 * c2);
  b.q.T = D.alloc<zt>((size_t)ZNB * (nblocks(cap, ZNB) * ZNB));
  b.q.tau = D.alloc<double>(cap);
  b.q.phases = D.alloc<zt>(cap);
  b.q.W1 = D.alloc<zt>((size_t)ZNB * cap);
  b.q.W2 = D.alloc<zt>((size_t)ZNB * cap);
  b.q.gram = D.alloc<zt>((size_t)nblocks(2 * cap, 64) * 1024);
  b.q.part_cap = (size_t)16 * ZNB * cap;
  b.q.part = D.alloc<zt>(b.q.part_cap);
  if (tensor_cores && cap >= 128) {
    b.tc.on = true;
    b.tc.plane = c2;
    b.tc.planes = D.alloc<double>(8 * c2);
    b.tc.ws = D.alloc<char>(tcx_gemm_workspace_bytes(cap, cap, cap));
    b.tc.err = D.alloc<int>(1);
    D.check(cudaMemsetAsync(b.tc.err, 0, sizeof(int), D.s), "tensor-core error word");
  }
}

// The tensor-core kernel's bounded waits report through b.tc.err.
void check_tc(CDriver& D, StepBufs& b) {
  if (!b.tc.on) return;
  int e = 0;
  D.check(cudaMemcpyAsync(&e, b.tc.err, sizeof(int), cudaMemcpyDeviceToHost, D.s), "tensor-core error copy");
  D.sync();
  if (e != 0) {
    *D.err = "tensor-core GEMM: a bounded wait timed out";
    throw ZFail{EIG_ERR_CUDA};
  }
}

ZQR qr_view(const StepBufs& b, int m, int n) {
  ZQR q = b.q;
  q.m = m;
  q.n = n;
  return q;
}

// ||A||_1 of an m x m packed matrix (host max of the column sums)
double host_norm1(CDriver& D, StepBufs& b, int m, const zt* A, int lda, std::vector<double>& h) {
  note_launches(1);
  zcolabs_kernel<<<m, 256, 0, D.s>>>(m, m, A, lda, zmk(0.0, 0.0), b.col1);
  h.resize(m);
  D.check(cudaMemcpyAsync(h.data(), b.col1, sizeof(double) * m, cudaMemcpyDeviceToHost, D.s), "norm1 copy");
  D.sync();
  double mx = 0.0;
  for (double v : h) mx = std::max(mx, v);
  return mx;
}

// Gershgorin disk of A (m x m, ld lda) about c = tr(A)/m
Region gershgorin_disk(CDriver& D, StepBufs& b, int m, const zt* A, int lda) {
  note_launches(1);
  ztrace_kernel<<<1, 256, 0, D.s>>>(m, A, lda, reinterpret_cast<zt*>(b.col2));
  double tr[2];
  D.check(cudaMemcpyAsync(tr, b.col2, sizeof(double) * 2, cudaMemcpyDeviceToHost, D.s), "trace copy");
  D.sync();
  const zt c = zmk(tr[0] / m, tr[1] / m);
  note_launches(2);
  zcolabs_kernel<<<m, 256, 0, D.s>>>(m, m, A, lda, c, b.col1);
  zrowabs_kernel<<<nblocks(m, 128), 128, 0, D.s>>>(m, A, lda, c, b.col2);
  std::vector<double> h1(m), h2(m);
  D.check(cudaMemcpyAsync(h1.data(), b.col1, sizeof(double) * m, cudaMemcpyDeviceToHost, D.s), "gersh copy");
  D.check(cudaMemcpyAsync(h2.data(), b.col2, sizeof(double) * m, cudaMemcpyDeviceToHost, D.s), "gersh copy");
  D.sync();
  double cm = 0.0, rm = 0.0;
  for (int i = 0; i < m; ++i) {
    cm = std::max(cm, h1[i]);
    rm = std::max(rm, h2[i]);
  }
  Region g;
  g.cr = c.x;
  g.ci = c.y;
  g.R = std::min(rm, cm);
  return g;
}

// Disk |z - c| <= ||A - c I||_F about c = tr(A)/m: unlike a Gershgorin radius it
// does not change with the basis of the block's invariant subspace, which for
// the trailing block of a split is fixed by rounding.
Region frobenius_disk(CDriver& D, StepBufs& b, int m, const zt* A, int lda) {
  note_launches(1);
  ztrace_kernel<<<1, 256, 0, D.s>>>(m, A, lda, reinterpret_cast<zt*>(b.col2));
  double tr[2];
  D.check(cudaMemcpyAsync(tr, b.col2, sizeof(double) * 2, cudaMemcpyDeviceToHost, D.s), "trace copy");
  D.sync();
  const zt c = zmk(tr[0] / m, tr[1] / m);
  note_launches(1);
  zcolsq_kernel<<<m, 256, 0, D.s>>>(m, A, lda, c, b.col1);
  std::vector<double> h(m);
  D.check(cudaMemcpyAsync(h.data(), b.col1, sizeof(double) * m, cudaMemcpyDeviceToHost, D.s), "norm copy");
  D.sync();
  double ss = 0.0;
  for (int i = 0; i < m; ++i) ss += h[i];
  Region g;
  g.cr = c.x;
  g.ci = c.y;
  g.R = std::sqrt(ss);
  return g;
}

struct CIrs {
  int iters;
  bool converged;
  const zt* Ap;
  const zt* Bp;
};

// Algorithm 3 over C on (A_0, B_0) already in b.A0, b.B0 (m x m packed).
CIrs cirs(CDriver& D, StepBufs& b, int m, double tau, int maxit) {
  const zt one = zmk(1.0, 0.0), zero = zmk(0.0, 0.0);
  zt *Aj = b.A0, *Bj = b.B0, *An = b.A1, *Bn = b.B1;
  zt *Rc = b.Ra, *Rp = b.Rb;
  const ZQR q = qr_view(b, 2 * m, m);
  bool have_prev = false;
  std::vector<double> h1(m), h2(m);
  int j = 0;
  while (true) {
    note_launches(1);
    zstack_kernel<<<nblocks((long long)m * m, 256), 256, 0, D.s>>>(m, Aj, Bj, b.W);
    D.check(zgeqrf(D.s, 2 * m, m, b.W, 2 * m, q, Rc, m), "IRS QR");
    D.check(zident(D.s, 2 * m, m, m, b.E), "IRS complement");
    D.check(zapply_q(D.s, q, b.E, m, false), "IRS complement");
    D.check(zmm(D.s, b.tc, true, false, m, m, m, one, b.E, 2 * m, Aj, m, zero, An, m), "IRS A");
    D.check(zmm(D.s, b.tc, true, false, m, m, m, one, b.E + m, 2 * m, Bj, m, zero, Bn, m), "IRS B");
    if (have_prev) {
      note_launches(2);
      zcoldiff_kernel<<<m, 256, 0, D.s>>>(m, Rc, Rp, b.col1);
      zcolabs_kernel<<<m, 256, 0, D.s>>>(m, m, Rp, m, zmk(0.0, 0.0), b.col2);
      D.check(cudaMemcpyAsync(h1.data(), b.col1, sizeof(double) * m, cudaMemcpyDeviceToHost, D.s), "ratio copy");
      D.check(cudaMemcpyAsync(h2.data(), b.col2, sizeof(double) * m, cudaMemcpyDeviceToHost, D.s), "ratio copy");
      D.sync();
      double num = 0.0, den = 0.0;
      for (int i = 0; i < m; ++i) {
        num = std::max(num, h1[i]);
        den = std::max(den, h2[i]);
      }
      const double ratio = den > 0.0 ? num / den : (num == 0.0 ? 0.0 : INFINITY);
      if (ratio <= tau) return {j + 1, true, An, Bn};
    }
    std::swap(Rc, Rp);
    have_prev = true;
    std::swap(Aj, An);
    std::swap(Bj, Bn);
    ++j;
    if (j > maxit) return {j, false, Aj, Bj};
  }
}

// Explicit unitary factor of the last zgeqrf (m x m) into Qout.
void explicit_q(CDriver& D, const ZQR& q, zt* Qout) {
  D.check(zident(D.s, q.m, q.n, 0, Qout), "explicit Q");
  D.check(zapply_q(D.s, q, Qout, q.n, true), "explicit Q");
}

struct CStepOut {
  bool accepted = false;
  bool converged = false;
  int k = 0, rank = 0, iters = 0, draw = 0;
  double e = INFINITY;
};

// One step on the line (w, t) with scale sc for the node matrix A (m x m
// packed).  The splitter lands in b.Q and A^ in b.Ahat.
CStepOut line_step(CDriver& D, StepBufs& b, int m, const zt* A, const HalfPlane& L, double sc,
                   uint64_t seed, uint64_t node, int attempt, double tau, int maxit,
                   double split_tol, int v_draws) {
  NvtxRange nvtx_("eig.cplane.step");
  const zt one = zmk(1.0, 0.0), zero = zmk(0.0, 0.0);
  const size_t mm = (size_t)m * m;
  CStepOut out;
  const zt s0 = zmk(L.wr * (L.t - sc), L.wi * (L.t - sc));
  const zt s1 = zmk(L.wr * (L.t + sc), L.wi * (L.t + sc));
  note_launches(1);
  zline_map_kernel<<<nblocks((long long)mm, 256), 256, 0, D.s>>>(m, A, m, s0, s1, b.A0, b.B0);
  const CIrs irs = cirs(D, b, m, tau, maxit);
  out.iters = irs.iters;
  out.converged = irs.converged;
  std::vector<double> hv;
  const double normA = host_norm1(D, b, m, A, m, hv);
  const ZQR q = qr_view(b, m, m);
  std::vector<double> hs(std::max(m - 1, 1)), d1(2 * (size_t)m), d2(2 * (size_t)m);
  const int draws = std::max(1, v_draws);
  for (int draw = 0; draw < draws; ++draw) {
    const int code = ((attempt & 0x3F) << 2) | (draw & 3);
    // Haar unitary V from the complex Ginibre draw
    D.check(gaussian(D.s, m, m, seed, PURPOSE_HAAR_RE, node, code, b.Gre, m), "Haar draw");
    D.check(gaussian(D.s, m, m, seed, PURPOSE_HAAR_IM, node, code, b.Gim, m), "Haar draw");
    note_launches(1);
    zinterleave_kernel<<<nblocks((long long)mm, 256), 256, 0, D.s>>>((long long)mm, b.Gre, b.Gim, b.X);
    D.check(zgeqrf(D.s, m, m, b.X, m, q, nullptr, m), "Haar QR");
    explicit_q(D, q, b.Vh);
    // RURV(A_p): A_p V^H = U R2
    D.check(zmm(D.s, b.tc, false, true, m, m, m, one, irs.Ap, m, b.Vh, m, zero, b.X, m), "A_p V^H");
    D.check(zgeqrf(D.s, m, m, b.X, m, q, b.R2, m), "RURV QR");
    explicit_q(D, q, b.U);
    // RQ of U^H (A_p + B_p) through the QR of (A_p + B_p)^H U J
    note_launches(2);
    zadd_kernel<<<nblocks((long long)mm, 256), 256, 0, D.s>>>((long long)mm, irs.Ap, irs.Bp, b.S);
    zrevcols_kernel<<<nblocks((long long)mm, 256), 256, 0, D.s>>>(m, m, b.U, b.Ur);
    D.check(zmm(D.s, b.tc, true, false, m, m, m, one, b.S, m, b.Ur, m, zero, b.Z, m), "(A_p+B_p)^H U J");
    D.check(zgeqrf(D.s, m, m, b.Z, m, q, b.R1, m), "RQ via QR");
    explicit_q(D, q, b.Ur);
    note_launches(1);
    zrevcols_kernel<<<nblocks((long long)mm, 256), 256, 0, D.s>>>(m, m, b.Ur, b.Q);
    // similarity and split test
    D.check(zmm(D.s, b.tc, false, false, m, m, m, one, A, m, b.Q, m, zero, b.AQ, m), "A Q");
    D.check(zmm(D.s, b.tc, true, false, m, m, m, one, b.Q, m, b.AQ, m, zero, b.Ahat, m), "Q^H A Q");
    note_launches(1);
    zabs_kernel<<<nblocks((long long)mm, 256), 256, 0, D.s>>>((long long)mm, b.Ahat, b.absA);
    if (m >= 2)
      D.check(split_scores(D.s, m, b.absA, m, normA > 0.0 ? 1.0 / normA : 1.0, b.colpart, b.scores,
                           false), "split scores");
    D.check(cudaMemcpy2DAsync(d1.data(), 2 * sizeof(double), b.R1, (m + 1) * sizeof(zt),
                              2 * sizeof(double), m, cudaMemcpyDeviceToHost, D.s), "diag copy");
    D.check(cudaMemcpy2DAsync(d2.data(), 2 * sizeof(double), b.R2, (m + 1) * sizeof(zt),
                              2 * sizeof(double), m, cudaMemcpyDeviceToHost, D.s), "diag copy");
    if (m >= 2)
      D.check(cudaMemcpyAsync(hs.data(), b.scores, sizeof(double) * (m - 1), cudaMemcpyDeviceToHost, D.s),
              "scores copy");
    D.sync();
    double scale = 0.0;
    for (int i = 0; i < m; ++i) scale = std::max(scale, std::hypot(d1[2 * i], d1[2 * i + 1]));
    int rank = 0;
    if (scale > 0.0)
      for (int i = 0; i < m; ++i)
        if (std::hypot(d2[2 * i], d2[2 * i + 1]) > 1e-8 * scale) ++rank;
    out.rank = rank;
    out.draw = draw;
    if (m >= 2) {
      out.k = choose_k_host(hs.data(), m);
      out.e = hs[out.k - 1];
    } else {
      out.k = 0;
      out.e = 0.0;
    }
    out.accepted = irs.converged && out.k > 0 && out.k < m && out.e <= split_tol;
    if (out.accepted || !irs.converged || rank == 0 || rank == m) break;
  }
  return out;
}

struct CNode {
  int off, m;
  zt* A;   // m x m packed, owned
  Region reg;
  uint64_t id;
  int depth;
};

struct CLeaf {
  int off, m;
  zt* A;
};

// State shared by the node workers of one solve.
struct CShared {
  int n = 0, ldu = 0, leaf = 64, device = 0;
  zt* dU = nullptr;
  const eig_params_t* p = nullptr;
  bool enclose = false;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<CNode> queue;
  int outstanding = 0;
  std::vector<CLeaf> leaves;
  std::vector<CplaneCluster>* clusters = nullptr;
  eig_solve_info_t inf;
  int status = EIG_OK;
  std::string err;
  std::vector<void*> node_mem;   // node matrices, freed after the leaves

  // a node matrix (m x m) that outlives the worker that made it
  zt* alloc_node(cudaStream_t s, size_t count, std::string* e) {
    void* q = nullptr;
    if (cudaMallocAsync(&q, std::max<size_t>(count * sizeof(zt), 256), s) != cudaSuccess) {
      cudaGetLastError();
      *e = "complex-plane node allocation failed";
      throw ZFail{EIG_ERR_NOMEM};
    }
    std::lock_guard<std::mutex> lock(mu);
    node_mem.push_back(q);
    return static_cast<zt*>(q);
  }
};

// One node of the recursion on stream s: steps until a split (children pushed
// on the shared queue), a cluster (enclose) or NO_SPLIT.  Scratch is per node.
void process_cnode(CShared& S, cudaStream_t s, CNode nd) {
  NvtxRange nvtx_("eig.cplane.node");
  const eig_params_t& p = *S.p;
  const int n = S.n, m = nd.m, leaf = S.leaf;
  const zt one = zmk(1.0, 0.0), zero = zmk(0.0, 0.0);
  std::string err;
  try {
    CDriver D{s, &err, {}};
    StepBufs b;
    make_bufs(D, b, m, p.prec == EIG_FP64_TC);
    zt* tmpU = D.alloc<zt>((size_t)n * m);
    const double tau = p.tau > 0.0 ? p.tau : std::max(1e-14, 4.0 * std::sqrt((double)m) * 0x1p-53);
    const double stol = p.split_tol > 0.0 ? p.split_tol : std::max(1e-12, 16.0 * m * 0x1p-53);
    NodePlan plan;
    plan.reg = nd.reg;
    plan.max_fail = p.max_fail;
    int iters = 0, fails = 0;
    while (true) {
      if (!(plan.reg.R > 0.0)) break;   // A = cI: already triangular
      const HalfPlane L = draw_line(plan.reg, p.seed, nd.id, plan.attempt, plan.has_perp, plan.pr,
                                    plan.pi_);
      const CStepOut st = line_step(D, b, m, nd.A, L, plan.reg.R, p.seed, nd.id, plan.attempt, tau,
                                    p.maxit, stol, p.v_draws);
      check_tc(D, b);
      iters += st.iters;
      if (st.accepted) {
        const int k = st.k;
        // this node's columns of U only: disjoint from every other node's
        D.check(zmm(s, b.tc, false, false, n, m, m, one, S.dU + (size_t)nd.off * S.ldu, S.ldu, b.Q,
                    m, zero, tmpU, n), "U update");
        D.check(zcopy(s, n, m, tmpU, n, S.dU + (size_t)nd.off * S.ldu, S.ldu), "U update");
        zt* A11 = S.alloc_node(s, (size_t)k * k, &err);
        zt* A22 = S.alloc_node(s, (size_t)(m - k) * (m - k), &err);
        D.check(zcopy(s, k, k, b.Ahat, m, A11, k), "block copy");
        D.check(zcopy(s, m - k, m - k, b.Ahat + k + (size_t)k * m, m, A22, m - k), "block copy");
        Region g0, g1, kid0, kid1;
        if (k > leaf) g0 = frobenius_disk(D, b, k, A11, k);
        if (m - k > leaf) g1 = frobenius_disk(D, b, m - k, A22, m - k);
        child_regions(plan.reg, L, k > leaf ? &g0 : nullptr, m - k > leaf ? &g1 : nullptr, &kid0,
                      &kid1);
        D.sync();   // the children's matrices and U are complete before another stream reads them
        std::lock_guard<std::mutex> lock(S.mu);
        S.inf.splits += 1;
        S.inf.total_iters += iters;
        S.inf.failed_attempts += fails;
        S.queue.push_back({nd.off + k, m - k, A22, kid1, child_node_id(nd.id, 1), nd.depth + 1});
        S.queue.push_back({nd.off, k, A11, kid0, child_node_id(nd.id, 0), nd.depth + 1});
        S.outstanding += 2;
        S.cv.notify_all();
        return;
      }
      fails += 1;
      if (plan.after_nonsplit(L, st.converged, st.rank, m)) {
        std::lock_guard<std::mutex> lock(S.mu);
        S.inf.total_iters += iters;
        S.inf.failed_attempts += fails;
        if (S.enclose) {
          if (S.clusters) {
            S.clusters->push_back({nd.off, m, plan.reg.cr, plan.reg.ci, plan.reg.R, {}});
            for (const HalfPlane& h : plan.reg.hp) S.clusters->back().hp.push_back({h.wr, h.wi, h.t});
          }
          if (m > ZLEAF_GLOBAL_MAX) {   // too large for the one-CTA leaf solver
            if (S.status == EIG_OK) {
              S.status = EIG_NO_SPLIT;
              S.err = "cluster of " + std::to_string(m) + " rows (enclosure reported) exceeds the " +
                      std::to_string(ZLEAF_GLOBAL_MAX) + "-row leaf solver";
            }
            return;
          }
          // the leaf phase picks shared-memory or global-memory storage by m
          S.leaves.push_back({nd.off, m, nd.A});
          return;
        }
        if (S.status == EIG_OK) {
          S.status = EIG_NO_SPLIT;
          S.err = "no split found for a node of size " + std::to_string(m);
        }
        return;
      }
    }
    std::lock_guard<std::mutex> lock(S.mu);
    S.inf.total_iters += iters;
    S.inf.failed_attempts += fails;
  } catch (ZFail f) {
    std::lock_guard<std::mutex> lock(S.mu);
    if (S.status == EIG_OK) {
      S.status = f.code;
      S.err = err;
    }
  }
}

void cnode_worker(CShared& S) {
  cudaStream_t s = nullptr;
  if (cudaSetDevice(S.device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    std::lock_guard<std::mutex> lock(S.mu);
    if (S.status == EIG_OK) {
      S.status = EIG_ERR_CUDA;
      S.err = "worker stream creation failed";
    }
    S.cv.notify_all();
    return;
  }
  while (true) {
    CNode nd;
    {
      std::unique_lock<std::mutex> lock(S.mu);
      S.cv.wait(lock, [&] { return !S.queue.empty() || S.outstanding == 0 || S.status != EIG_OK; });
      if (S.status != EIG_OK || S.queue.empty()) break;
      nd = S.queue.back();   // depth first, like the sequential order
      S.queue.pop_back();
      S.inf.nodes += 1;
      S.inf.max_depth = std::max(S.inf.max_depth, nd.depth);
      if (nd.m <= S.leaf) {
        S.leaves.push_back({nd.off, nd.m, nd.A});
        S.outstanding--;
        S.cv.notify_all();
        continue;
      }
    }
    process_cnode(S, s, nd);
    std::lock_guard<std::mutex> lock(S.mu);
    S.outstanding--;
    S.cv.notify_all();
  }
  cudaStreamSynchronize(s);
  cudaStreamDestroy(s);
}

}  // namespace

// Complex Schur form A = U T U^H by the complex-plane recursion (Sec. 3.3);
// independent nodes run on p.workers host workers with their own streams.
int cplane_schur(cudaStream_t s, int n, const double* dA_, int lda, double* dT_, int ldt,
                 double* dU_, int ldu, double* dw_, const eig_params_t& p, bool enclose,
                 std::vector<CplaneCluster>* clusters, eig_solve_info_t* info, std::string* err) {
  NvtxRange nvtx_("eig.cplane.solve");
  const zt* dA = reinterpret_cast<const zt*>(dA_);
  zt* dT = reinterpret_cast<zt*>(dT_);
  zt* dU = reinterpret_cast<zt*>(dU_);
  zt* dw = reinterpret_cast<zt*>(dw_);
  const zt one = zmk(1.0, 0.0), zero = zmk(0.0, 0.0);
  CShared S;
  std::memset(&S.inf, 0, sizeof(S.inf));
  S.n = n;
  S.ldu = ldu;
  S.leaf = std::max(1, std::min(p.leaf_size > 0 ? p.leaf_size : 64, ZLEAF_MAX));
  S.dU = dU;
  S.p = &p;
  S.enclose = enclose;
  S.clusters = clusters;
  cudaGetDevice(&S.device);
  int status = EIG_OK;
  try {
    CDriver D{s, err, {}};
    note_launches(1);
    zident_ld_kernel<<<nblocks((long long)n * n, 256), 256, 0, s>>>(n, n, dU, ldu);
    zt* root = S.alloc_node(s, (size_t)n * n, err);
    D.check(zcopy(s, n, n, dA, lda, root, n), "input copy");
    Region r0;
    if (n > S.leaf) {
      StepBufs g;
      g.col1 = D.alloc<double>(n + 1);
      g.col2 = D.alloc<double>(n + 1);
      r0 = gershgorin_disk(D, g, n, root, n);
    }
    D.sync();   // the workers' streams read the root and U
    S.queue.push_back({0, n, root, r0, 1ull, 0});
    S.outstanding = 1;
    const int nw = n > S.leaf ? std::max(1, std::min(p.workers, 32)) : 1;
    std::vector<std::thread> th;
    for (int i = 0; i < nw; ++i) th.emplace_back(cnode_worker, std::ref(S));
    for (auto& t : th) t.join();
    if (clusters)   // offset order, whatever order the workers finished in
      std::sort(clusters->begin(), clusters->end(),
                [](const CplaneCluster& a, const CplaneCluster& b) { return a.off < b.off; });
    status = S.status;
    if (status < 0) *err = S.err;
    if (status == EIG_OK) {
      NvtxRange nvtx_leaves("eig.cplane.leaves");
      // leaves in offset order (the schedule does not change the result)
      std::vector<CLeaf>& leaves = S.leaves;
      std::sort(leaves.begin(), leaves.end(), [](const CLeaf& a, const CLeaf& b) { return a.off < b.off; });
      const int nl = (int)leaves.size();
      S.inf.leaves = nl;
      // small leaves in shared memory, clusters above ZLEAF_MAX rows in global scratch
      std::vector<ZLeafDesc> hsmall, hbig;
      std::vector<zt*> Zs(nl);
      int* dstat = D.alloc<int>(std::max(nl, 1));
      for (int i = 0; i < nl; ++i) {
        const int m = leaves[i].m;
        zt* TZ = D.alloc<zt>(2 * (size_t)m * m);
        Zs[i] = TZ + (size_t)m * m;
        ZLeafDesc dsc{m, leaves[i].A, m, TZ, Zs[i], dstat + i, nullptr};
        if (m <= ZLEAF_MAX) {
          hsmall.push_back(dsc);
        } else {
          dsc.work = D.alloc<zt>(2 * (size_t)m * m + 2 * (size_t)m);
          hbig.push_back(dsc);
        }
      }
      const int ns = (int)hsmall.size(), nbig = (int)hbig.size();
      ZLeafDesc* dd = D.alloc<ZLeafDesc>(std::max(nl, 1));
      if (ns > 0)
        D.check(cudaMemcpyAsync(dd, hsmall.data(), sizeof(ZLeafDesc) * ns, cudaMemcpyHostToDevice, s),
                "leaf descriptors");
      if (nbig > 0)
        D.check(cudaMemcpyAsync(dd + ns, hbig.data(), sizeof(ZLeafDesc) * nbig, cudaMemcpyHostToDevice, s),
                "leaf descriptors");
      const int smem = 2 * ZLEAF_MAX * (ZLEAF_MAX + 1) * (int)sizeof(zt);
      D.check(cudaFuncSetAttribute(zschur_leaf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
              "leaf attribute");
      if (ns > 0) {
        note_launches(1);
        zschur_leaf_kernel<<<ns, 256, smem, s>>>(dd);
        D.check(cudaGetLastError(), "leaf launch");
      }
      if (nbig > 0) {
        note_launches(1);
        zschur_leaf_global_kernel<<<nbig, 256, 0, s>>>(dd + ns);
        D.check(cudaGetLastError(), "large leaf launch");
      }
      zt* tmpU = D.alloc<zt>((size_t)n * n);
      for (int i = 0; i < nl; ++i) {
        const int off = leaves[i].off, m = leaves[i].m;
        D.check(zgemm(s, false, false, n, m, m, one, dU + (size_t)off * ldu, ldu, Zs[i], m, zero, tmpU, n),
                "leaf U update");
        D.check(zcopy(s, n, m, tmpU, n, dU + (size_t)off * ldu, ldu), "leaf U update");
      }
      std::vector<int> hst(std::max(nl, 1));
      if (nl > 0)
        D.check(cudaMemcpyAsync(hst.data(), dstat, sizeof(int) * nl, cudaMemcpyDeviceToHost, s), "leaf status");
      // T = triu(U^H A U), w = diag(T)
      StepBufs fb;
      if (p.prec == EIG_FP64_TC && n >= 128) {
        fb.tc.on = true;
        fb.tc.plane = (size_t)n * n;
        fb.tc.planes = D.alloc<double>(8 * fb.tc.plane);
        fb.tc.ws = D.alloc<char>(tcx_gemm_workspace_bytes(n, n, n));
        fb.tc.err = D.alloc<int>(1);
        D.check(cudaMemsetAsync(fb.tc.err, 0, sizeof(int), s), "tensor-core error word");
      }
      zt* AU = D.alloc<zt>((size_t)n * n);
      D.check(zmm(s, fb.tc, false, false, n, n, n, one, dA, lda, dU, ldu, zero, AU, n), "A U");
      D.check(zmm(s, fb.tc, true, false, n, n, n, one, dU, ldu, AU, n, zero, tmpU, n), "U^H A U");
      note_launches(1);
      ztriu_kernel<<<nblocks((long long)n * n, 256), 256, 0, s>>>(n, tmpU, n, dT, ldt, dw);
      D.check(cudaGetLastError(), "triangle");
      D.sync();
      check_tc(D, fb);
      for (int i = 0; i < nl; ++i)
        if (hst[i] != 0) status = EIG_NO_CONVERGENCE;
    }
    D.sync();
  } catch (ZFail f) {
    status = f.code;
  }
  cudaStreamSynchronize(s);
  for (void* q : S.node_mem) cudaFreeAsync(q, s);
  cudaStreamSynchronize(s);
  S.inf.status = status;
  if (info) *info = S.inf;
  return status;
}

size_t cplane_footprint(int n, int prec) {
  const size_t c2 = (size_t)n * n, z = sizeof(zt);
  // make_bufs at the root: 24 n^2 complex (IRS, splitter, similarity, QR
  // reflectors) + 3 n^2 doubles + panel / Gram / score vectors; the node's
  // U update scratch n^2 complex; node matrices up to 2 n^2 complex; the
  // final A U and U^H A U 2 n^2 complex
  size_t bytes = 24 * c2 * z + 3 * c2 * sizeof(double) + c2 * z + 2 * c2 * z + 2 * c2 * z;
  bytes += (size_t)(20 * ZNB + 8) * n * z + (size_t)(nblocks(2 * n, 64) * 1024) * z +
           (size_t)((n + 31) / 32 + 8) * n * sizeof(double);
  if (prec == EIG_FP64_TC && n >= 128) bytes += 8 * c2 * sizeof(double) + tcx_gemm_workspace_bytes(n, n, n);
  // leaf buffers, held beside the root's: T and Z (2 m^2 complex) per leaf and
  // the global solver's scratch (2 m^2 + 2 m) per cluster; with every leaf or
  // cluster at most ZLEAF_GLOBAL_MAX rows, sum m_i^2 <= ZLEAF_GLOBAL_MAX n
  const size_t lm = (size_t)std::min(n, ZLEAF_GLOBAL_MAX);
  bytes += (4 * lm + 2) * (size_t)n * z;
  return bytes + ((size_t)64 << 20);   // allocator granularity
}

// ------------------------------------------------------------------ building blocks
// The single steps of the complex path, for tests and callers that compose
// their own recursion (the complex counterparts of eig_qr, eig_haar and
// eig_divide_step + eig_split).

int cplane_qr(cudaStream_t s, int m, int n, const double* dX_, int ldx, double* dQ_, int ldq,
              double* dR_, int ldr, std::string* err) {
  int status = EIG_OK;
  try {
    CDriver D{s, err, {}};
    StepBufs b;
    const int cap = std::max(m, n);
    // the QR buffers of a node of size cap hold an m x n factorisation with m <= 2 cap
    b.q.V = D.alloc<zt>((size_t)m * n);
    b.q.T = D.alloc<zt>((size_t)ZNB * (nblocks(n, ZNB) * ZNB));
    b.q.tau = D.alloc<double>(n);
    b.q.phases = D.alloc<zt>(n);
    b.q.W1 = D.alloc<zt>((size_t)ZNB * cap);
    b.q.W2 = D.alloc<zt>((size_t)ZNB * cap);
    b.q.gram = D.alloc<zt>((size_t)nblocks(m, 64) * 1024);
    zt* P = D.alloc<zt>((size_t)m * n);
    D.check(zcopy(s, m, n, reinterpret_cast<const zt*>(dX_), ldx, P, m), "input copy");
    ZQR q = b.q;
    q.m = m;
    q.n = n;
    zt* R = D.alloc<zt>((size_t)n * n);
    D.check(zgeqrf(s, m, n, P, m, q, R, n), "QR");
    zt* Qp = D.alloc<zt>((size_t)m * n);
    D.check(zident(s, m, n, 0, Qp), "explicit Q");
    D.check(zapply_q(s, q, Qp, n, true), "explicit Q");
    D.check(zcopy(s, m, n, Qp, m, reinterpret_cast<zt*>(dQ_), ldq), "Q copy");
    if (dR_) D.check(zcopy(s, n, n, R, n, reinterpret_cast<zt*>(dR_), ldr), "R copy");
    D.sync();
  } catch (ZFail f) {
    status = f.code;
  }
  return status;
}

int cplane_haar(cudaStream_t s, int n, uint64_t seed, uint64_t node, int attempt, double* dV_,
                int ldv, std::string* err) {
  int status = EIG_OK;
  try {
    CDriver D{s, err, {}};
    double* Gre = D.alloc<double>((size_t)n * n);
    double* Gim = D.alloc<double>((size_t)n * n);
    zt* G = D.alloc<zt>((size_t)n * n);
    D.check(gaussian(s, n, n, seed, PURPOSE_HAAR_RE, node, attempt, Gre, n), "Haar draw");
    D.check(gaussian(s, n, n, seed, PURPOSE_HAAR_IM, node, attempt, Gim, n), "Haar draw");
    note_launches(1);
    zinterleave_kernel<<<nblocks((long long)n * n, 256), 256, 0, s>>>((long long)n * n, Gre, Gim, G);
    D.check(cudaGetLastError(), "Haar interleave");
    // the Haar unitary is the Q factor of G with a non-negative real diagonal of R
    const int rc = cplane_qr(s, n, n, reinterpret_cast<const double*>(G), n, dV_, ldv, nullptr, 0, err);
    if (rc != EIG_OK) throw ZFail{rc};
  } catch (ZFail f) {
    status = f.code;
  }
  return status;
}

int cplane_step(cudaStream_t s, int n, const double* dA_, int lda, double w_re, double w_im,
                double t, double sc, const eig_params_t& p, uint64_t node, int attempt,
                double* dQ_, int ldq, double* dAhat_, int ldah, eig_step_info_t* info,
                std::string* err) {
  int status = EIG_OK;
  try {
    CDriver D{s, err, {}};
    StepBufs b;
    make_bufs(D, b, n, p.prec == EIG_FP64_TC);
    zt* A = D.alloc<zt>((size_t)n * n);
    D.check(zcopy(s, n, n, reinterpret_cast<const zt*>(dA_), lda, A, n), "input copy");
    const double tau = p.tau > 0.0 ? p.tau : std::max(1e-14, 4.0 * std::sqrt((double)n) * 0x1p-53);
    const double stol = p.split_tol > 0.0 ? p.split_tol : std::max(1e-12, 16.0 * n * 0x1p-53);
    HalfPlane L;
    L.wr = w_re;
    L.wi = w_im;
    L.t = t;
    const CStepOut st = line_step(D, b, n, A, L, sc, p.seed, node, attempt, tau, p.maxit, stol,
                                  p.v_draws);
    check_tc(D, b);
    if (dQ_) D.check(zcopy(s, n, n, b.Q, n, reinterpret_cast<zt*>(dQ_), ldq), "Q copy");
    if (dAhat_) D.check(zcopy(s, n, n, b.Ahat, n, reinterpret_cast<zt*>(dAhat_), ldah), "A^ copy");
    D.sync();
    if (info) {
      std::memset(info, 0, sizeof(*info));
      info->iters = st.iters;
      info->converged = st.converged ? 1 : 0;
      info->k = st.k;
      info->split_residual = st.e;
      info->rank = st.rank;
      info->draw = st.draw;
    }
    status = st.accepted ? EIG_OK : (st.converged ? EIG_NO_SPLIT : EIG_NO_CONVERGENCE);
  } catch (ZFail f) {
    status = f.code;
  }
  return status;
}

cudaError_t cplane_zgemm(cudaStream_t s, bool ta, bool tb, int m, int n, int k, double ar,
                         double ai, const double* A, int lda, const double* B, int ldb, double br,
                         double bi, double* C, int ldc) {
  return zgemm(s, ta, tb, m, n, k, zmk(ar, ai), reinterpret_cast<const zt*>(A), lda,
               reinterpret_cast<const zt*>(B), ldb, zmk(br, bi), reinterpret_cast<zt*>(C), ldc);
}
}  // namespace eigdc

// ------------------------------------------------------------------ host-only C-ABI helpers
extern "C" int eig_cplane_enclosing_circle(double c_re, double c_im, double R, int nhp,
                                           const double* w_re, const double* w_im,
                                           const double* t, double* m_re, double* m_im,
                                           double* r) {
  if (nhp < 0 || (nhp > 0 && (!w_re || !w_im || !t)) || !m_re || !m_im || !r || !(R >= 0.0))
    return EIG_ERR_ARG;
  eigdc::Region g;
  g.cr = c_re;
  g.ci = c_im;
  g.R = R;
  for (int i = 0; i < nhp; ++i) g.hp.push_back({w_re[i], w_im[i], t[i]});
  eigdc::enclosing_circle(g, m_re, m_im, r);
  return EIG_OK;
}

extern "C" int eig_cplane_draw_line(uint64_t seed, uint64_t node, int attempt, double c_re,
                                    double c_im, double R, int perpendicular, double pw_re,
                                    double pw_im, double* w_re, double* w_im, double* t) {
  if (!w_re || !w_im || !t || !(R >= 0.0)) return EIG_ERR_ARG;
  eigdc::Region g;
  g.cr = c_re;
  g.ci = c_im;
  g.R = R;
  const eigdc::HalfPlane h = eigdc::draw_line(g, seed, node, attempt, perpendicular != 0, pw_re, pw_im);
  *w_re = h.wr;
  *w_im = h.wi;
  *t = h.t;
  return EIG_OK;
}
