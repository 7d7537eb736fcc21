// Element-wise and reduction kernels of the divide-and-conquer path:
// region map + stacking (Sec. 3.3 Moebius map, Algorithm 3 stacking), the
// R-difference convergence norms (Algorithm 3), the Philox Gaussian draw
// (Algorithm 1, line 1), the split-test prefix-sum / max reduction
// (Sec. 4.2.1), Gershgorin data for the strategies of Sec. 3.3-3.4, small
// reshaping kernels (index reversal for RQ / QL, transposes), the kernels of
// the FP64 refinement of the BF16 x 3 form, the SVD embedding (Sec. 3.2) and
// the generalized Schur assembly of pencils (2 x 2 pair splitting, alpha /
// beta).
#include <cuda_runtime.h>

#include <algorithm>
#include <math.h>
#include <stdint.h>

#include "internal.h"

namespace eigdc {

static inline unsigned blocks_for(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

// ---------------------------------------------------------------- shaping
__global__ void fill_identity_block_kernel(int rows, int cols, double* Y, int ldy, int off) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)rows * cols) return;
  const int i = (int)(idx % rows), j = (int)(idx / rows);
  Y[i + (size_t)j * ldy] = (i == j + off) ? 1.0 : 0.0;
}

cudaError_t fill_identity_block(cudaStream_t s, int rows, int cols, double* Y, int ldy,
                                int diag_row_offset) {
  const size_t n = (size_t)rows * cols;
  if (n == 0) return cudaSuccess;
  note_launches(1);
  fill_identity_block_kernel<<<blocks_for(n, 256), 256, 0, s>>>(rows, cols, Y, ldy, diag_row_offset);
  return cudaGetLastError();
}

// Pencil (A', B') of the region (unit circle: (A, B); circle |z-c| = r:
// (A - cB, rB); line Re z = sigma with scale s: (A - (sigma-s)B, A - (sigma+s)B)),
// written to Aj, Bj (ld n) and stacked as W = [B'; -A'] (ld 2n).
__global__ void region_stack_kernel(int n, const double* __restrict__ A, int lda,
                                    const double* __restrict__ B, int ldb, int kind, double c,
                                    double r, double* __restrict__ Aj, double* __restrict__ Bj,
                                    double* __restrict__ W) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * n) return;
  const int i = (int)(idx % n), j = (int)(idx / n);
  const double a = A[i + (size_t)j * lda];
  const double b = B ? B[i + (size_t)j * ldb] : (i == j ? 1.0 : 0.0);
  double am, bm;
  if (kind == 1) {
    am = a - c * b;
    bm = r * b;
  } else if (kind == 2) {
    am = a - (c - r) * b;
    bm = a - (c + r) * b;
  } else {
    am = a;
    bm = b;
  }
  Aj[i + (size_t)j * n] = am;
  Bj[i + (size_t)j * n] = bm;
  W[i + (size_t)j * 2 * n] = bm;
  W[n + i + (size_t)j * 2 * n] = -am;
}

cudaError_t region_stack(cudaStream_t s, int n, const double* A, int lda, const double* B, int ldb,
                         int kind, double c_or_sigma, double r_or_s, double* Aj, double* Bj,
                         double* W) {
  const size_t t = (size_t)n * n;
  if (t == 0) return cudaSuccess;
  note_launches(1);
  region_stack_kernel<<<blocks_for(t, 256), 256, 0, s>>>(n, A, lda, B, ldb, kind, c_or_sigma,
                                                         r_or_s, Aj, Bj, W);
  return cudaGetLastError();
}

__global__ void stack_pencil_kernel(int n, const double* __restrict__ Aj,
                                    const double* __restrict__ Bj, double* __restrict__ W) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * n) return;
  const int i = (int)(idx % n), j = (int)(idx / n);
  W[i + (size_t)j * 2 * n] = Bj[idx];
  W[n + i + (size_t)j * 2 * n] = -Aj[idx];
}

cudaError_t stack_pencil(cudaStream_t s, int n, const double* Aj, const double* Bj, double* W) {
  const size_t t = (size_t)n * n;
  if (t == 0) return cudaSuccess;
  note_launches(1);
  stack_pencil_kernel<<<blocks_for(t, 256), 256, 0, s>>>(n, Aj, Bj, W);
  return cudaGetLastError();
}

// Non-negative doubles order like their bit patterns, so an integer atomic max
// on the bits is an exact (and order-independent) max.
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* p, double v) {
  atomicMax(p, (unsigned long long)__double_as_longlong(v));
}

// One warp per column j of R (rows 0..j): sum |Rcur - Rprev| and |Rprev|.
__global__ void r_extract_diff_kernel(int n, const double* __restrict__ W, int ldw,
                                      double* __restrict__ Rcur, const double* __restrict__ Rprev,
                                      unsigned long long* sums) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n) return;
  const int j = warp;
  double sd = 0.0, sp = 0.0;
  for (int i = lane; i < n; i += 32) {
    const double r = (i <= j) ? W[i + (size_t)j * ldw] : 0.0;
    Rcur[i + (size_t)j * n] = r;
    if (Rprev) {
      const double p = Rprev[i + (size_t)j * n];
      sd += fabs(r - p);
      sp += fabs(p);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sd += __shfl_xor_sync(0xffffffffu, sd, o);
    sp += __shfl_xor_sync(0xffffffffu, sp, o);
  }
  if (lane == 0 && Rprev) {
    atomic_max_nonneg(&sums[0], sd);
    atomic_max_nonneg(&sums[1], sp);
  }
}

cudaError_t r_extract_diff(cudaStream_t s, int n, const double* W, int ldw, double* Rcur,
                           const double* Rprev, unsigned long long* sums) {
  if (n == 0) return cudaSuccess;
  note_launches(1);
  r_extract_diff_kernel<<<blocks_for((size_t)n * 32, 256), 256, 0, s>>>(n, W, ldw, Rcur, Rprev, sums);
  return cudaGetLastError();
}

__global__ void copy_matrix_kernel(int rows, int cols, const double* __restrict__ A, int lda,
                                   double* __restrict__ B, int ldb) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)rows * cols) return;
  const int i = (int)(idx % rows), j = (int)(idx / rows);
  B[i + (size_t)j * ldb] = A[i + (size_t)j * lda];
}

cudaError_t copy_matrix(cudaStream_t s, int rows, int cols, const double* A, int lda, double* B,
                        int ldb) {
  const size_t t = (size_t)rows * cols;
  if (t == 0) return cudaSuccess;
  note_launches(1);
  copy_matrix_kernel<<<blocks_for(t, 256), 256, 0, s>>>(rows, cols, A, lda, B, ldb);
  return cudaGetLastError();
}

__global__ void add_matrices_kernel(int rows, int cols, const double* __restrict__ A, int lda,
                                    const double* __restrict__ B, int ldb, double* __restrict__ C,
                                    int ldc) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)rows * cols) return;
  const int i = (int)(idx % rows), j = (int)(idx / rows);
  C[i + (size_t)j * ldc] = A[i + (size_t)j * lda] + B[i + (size_t)j * ldb];
}

cudaError_t add_matrices(cudaStream_t s, int rows, int cols, const double* A, int lda,
                         const double* B, int ldb, double* C, int ldc) {
  const size_t t = (size_t)rows * cols;
  if (t == 0) return cudaSuccess;
  note_launches(1);
  add_matrices_kernel<<<blocks_for(t, 256), 256, 0, s>>>(rows, cols, A, lda, B, ldb, C, ldc);
  return cudaGetLastError();
}

// Z[i][k] = Y[n-1-k][i] through a 32x32 shared tile.
__global__ void reverse_transpose_kernel(int n, const double* __restrict__ Y, int ldy,
                                         double* __restrict__ Z, int ldz) {
  __shared__ double tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;   // bx: Y column block, by: Y row block
  const int tx = threadIdx.x, ty = threadIdx.y;           // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int yr = by + tx, yc = bx + r;
    if (yr < n && yc < n) tile[r][tx] = Y[yr + (size_t)yc * ldy];
  }
  __syncthreads();
  // Z(i, k) with i = Y column, k = n-1-(Y row)
  for (int r = ty; r < 32; r += 8) {
    const int yr = by + r;     // Y row -> k
    const int yc = bx + tx;    // Y col -> i
    if (yr < n && yc < n) Z[yc + (size_t)(n - 1 - yr) * ldz] = tile[tx][r];
  }
}

cudaError_t reverse_transpose(cudaStream_t s, int n, const double* Y, int ldy, double* Z, int ldz) {
  if (n == 0) return cudaSuccess;
  dim3 grid((n + 31) / 32, (n + 31) / 32);
  note_launches(1);
  reverse_transpose_kernel<<<grid, dim3(32, 8), 0, s>>>(n, Y, ldy, Z, ldz);
  return cudaGetLastError();
}

// B (cols x rows) = A^T for A rows x cols, 32 x 32 shared tiles.
__global__ void transpose_kernel(int rows, int cols, const double* __restrict__ A, int lda,
                                 double* __restrict__ B, int ldb) {
  __shared__ double tile[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int q = ty; q < 32; q += 8) {
    const int r = r0 + tx, c = c0 + q;
    if (r < rows && c < cols) tile[q][tx] = A[r + (size_t)c * lda];
  }
  __syncthreads();
  for (int q = ty; q < 32; q += 8) {
    const int r = r0 + q, c = c0 + tx;     // B(c, r) = A(r, c)
    if (r < rows && c < cols) B[c + (size_t)r * ldb] = tile[tx][q];
  }
}

cudaError_t transpose(cudaStream_t s, int rows, int cols, const double* A, int lda, double* B,
                      int ldb) {
  if (rows == 0 || cols == 0) return cudaSuccess;
  dim3 grid((cols + 31) / 32, (rows + 31) / 32);
  note_launches(1);
  transpose_kernel<<<grid, dim3(32, 8), 0, s>>>(rows, cols, A, lda, B, ldb);
  return cudaGetLastError();
}

__global__ void reverse_columns_kernel(int rows, int n, const double* __restrict__ A, int lda,
                                       double* __restrict__ B, int ldb) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)rows * n) return;
  const int i = (int)(idx % rows), j = (int)(idx / rows);
  B[i + (size_t)j * ldb] = A[i + (size_t)(n - 1 - j) * lda];
}

cudaError_t reverse_columns(cudaStream_t s, int rows, int n, const double* A, int lda, double* B,
                            int ldb) {
  const size_t t = (size_t)rows * n;
  if (t == 0) return cudaSuccess;
  note_launches(1);
  reverse_columns_kernel<<<blocks_for(t, 256), 256, 0, s>>>(rows, n, A, lda, B, ldb);
  return cudaGetLastError();
}

// A <- (A + A^T) / 2, each pair (i, j), i > j, handled once.
__global__ void symmetrize_kernel(int n, double* A, int lda) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * n) return;
  const int i = (int)(idx % n), j = (int)(idx / n);
  if (i <= j) return;
  const double a = A[i + (size_t)j * lda], b = A[j + (size_t)i * lda];
  const double m = 0.5 * (a + b);
  A[i + (size_t)j * lda] = m;
  A[j + (size_t)i * lda] = m;
}

cudaError_t symmetrize(cudaStream_t s, int n, double* A, int lda) {
  const size_t t = (size_t)n * n;
  if (t == 0) return cudaSuccess;
  note_launches(1);
  symmetrize_kernel<<<blocks_for(t, 256), 256, 0, s>>>(n, A, lda);
  return cudaGetLastError();
}

__global__ void upper_triangle_kernel(int n, const double* __restrict__ W, int ldw,
                                      double* __restrict__ R, int ldr) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * n) return;
  const int i = (int)(idx % n), j = (int)(idx / n);
  R[i + (size_t)j * ldr] = (i <= j) ? W[i + (size_t)j * ldw] : 0.0;
}

cudaError_t upper_triangle(cudaStream_t s, int n, const double* W, int ldw, double* R, int ldr) {
  const size_t t = (size_t)n * n;
  if (t == 0) return cudaSuccess;
  note_launches(1);
  upper_triangle_kernel<<<blocks_for(t, 256), 256, 0, s>>>(n, W, ldw, R, ldr);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): multipliers and Weyl
// key increments of the published generator.
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(M0, c[0]), lo0 = M0 * c[0];
    const uint32_t hi1 = __umulhi(M1, c[2]), lo1 = M1 * c[2];
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n1 = lo1, n2 = hi0 ^ c[3] ^ k1, n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    k0 += W0;
    k1 += W1;
  }
}

// Counter layout: c0 = pair index (low 32), c1 = pair bits 32..39 | attempt << 8
// | purpose << 16, (c2, c3) = stream; key = seed.  Box-Muller on two 52-bit
// uniforms u1 = (m1 + 1/2) 2^-52, u2 = m2 2^-52.
__global__ void gaussian_kernel(int rows, int cols, uint64_t seed, int purpose, uint64_t stream,
                                int attempt, double* __restrict__ G, int ldg) {
  const uint64_t pair = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t count = (uint64_t)rows * cols;
  if (2 * pair >= count) return;
  uint32_t c[4];
  c[0] = (uint32_t)(pair & 0xFFFFFFFFull);
  c[1] = (uint32_t)((pair >> 32) & 0xFFull) | ((uint32_t)(attempt & 0xFF) << 8) |
         ((uint32_t)(purpose & 0xFFFF) << 16);
  c[2] = (uint32_t)(stream & 0xFFFFFFFFull);
  c[3] = (uint32_t)(stream >> 32);
  philox4x32_10(c, (uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32));
  const uint64_t m1 = ((uint64_t)c[0] << 20) | (c[1] >> 12);
  const uint64_t m2 = ((uint64_t)c[2] << 20) | (c[3] >> 12);
  const double u1 = ((double)m1 + 0.5) * 0x1p-52;
  const double u2 = (double)m2 * 0x1p-52;
  const double r = sqrt(-2.0 * log(u1));
  double sn, cs;
  sincospi(2.0 * u2, &sn, &cs);
  const uint64_t e0 = 2 * pair, e1 = 2 * pair + 1;
  G[(e0 % rows) + (e0 / rows) * (uint64_t)ldg] = r * cs;
  if (e1 < count) G[(e1 % rows) + (e1 / rows) * (uint64_t)ldg] = r * sn;
}

cudaError_t gaussian(cudaStream_t s, int rows, int cols, uint64_t seed, int purpose,
                     uint64_t stream, int attempt, double* G, int ldg) {
  const uint64_t count = (uint64_t)rows * cols;
  if (count == 0) return cudaSuccess;
  const uint64_t pairs = (count + 1) / 2;
  note_launches(1);
  gaussian_kernel<<<blocks_for(pairs, 256), 256, 0, s>>>(rows, cols, seed, purpose, stream,
                                                         attempt, G, ldg);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- norms
__global__ void norm1_bits_kernel(int rows, int cols, const double* __restrict__ A, int lda,
                                  unsigned long long* out) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= cols) return;
  double s = 0.0;
  for (int i = lane; i < rows; i += 32) s += fabs(A[i + (size_t)warp * lda]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) atomic_max_nonneg(out, s);
}

cudaError_t norm1_bits(cudaStream_t s, int rows, int cols, const double* A, int lda,
                       unsigned long long* out) {
  if (cols == 0) return cudaSuccess;
  note_launches(1);
  norm1_bits_kernel<<<blocks_for((size_t)cols * 32, 256), 256, 0, s>>>(rows, cols, A, lda, out);
  return cudaGetLastError();
}

__global__ void nonfinite_kernel(int rows, int cols, const double* __restrict__ A, int lda,
                                 int* flag) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)rows * cols) return;
  const int i = (int)(idx % rows), j = (int)(idx / rows);
  if (!isfinite(A[i + (size_t)j * lda])) atomicOr(flag, 1);
}

cudaError_t nonfinite_check(cudaStream_t s, int rows, int cols, const double* A, int lda,
                            int* flag) {
  const size_t t = (size_t)rows * cols;
  if (t == 0) return cudaSuccess;
  note_launches(1);
  nonfinite_kernel<<<blocks_for(t, 256), 256, 0, s>>>(rows, cols, A, lda, flag);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- power iteration
// One CTA: v = y - c x (x may be null: v = y), est = ||v||_2 (fixed-order
// reduction), xout = v / est (zero when est = 0).  xout may alias x.
__global__ void __launch_bounds__(1024)
power_norm_kernel(int n, double c, const double* x, const double* __restrict__ y, double* xout,
                  double* __restrict__ est) {
  __shared__ double red[32];
  __shared__ double tot;
  double ss = 0.0;
  for (int i = threadIdx.x; i < n; i += 1024) {
    const double v = x ? y[i] - c * x[i] : y[i];
    ss = fma(v, v, ss);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < 32; ++q) t += red[q];
    tot = sqrt(t);
    *est = tot;
  }
  __syncthreads();
  const double nrm = tot;
  for (int i = threadIdx.x; i < n; i += 1024) {
    const double v = x ? y[i] - c * x[i] : y[i];
    xout[i] = nrm > 0.0 ? v / nrm : 0.0;
  }
}

cudaError_t power_norm(cudaStream_t s, int n, double c, const double* x, const double* y,
                       double* xout, double* est) {
  if (n <= 0) return cudaSuccess;
  note_launches(1);
  power_norm_kernel<<<1, 1024, 0, s>>>(n, c, x, y, xout, est);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- split test
// S[k][j] = sum_{i>=k} |A_ij|, f(k) = max_{j<k} S[k][j] (Sec. 4.2.1), with 32-row
// blocks: (1) per-block column sums, (2) exclusive suffix over blocks, (3) a
// warp per (row block, column) forms the in-block suffix by shuffles and keeps
// a per-row running max; rows combine by an exact integer max on the bits.
__global__ void split_blocksum_kernel(int n, const double* __restrict__ A, int lda, int nrb,
                                      double* __restrict__ colpart) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int b = blockIdx.x;
  const int j = blockIdx.y * 8 + w;
  if (j >= n) return;
  const int i = b * 32 + lane;
  double x = (i < n) ? fabs(A[i + (size_t)j * lda]) : 0.0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  if (lane == 0) colpart[b + (size_t)j * nrb] = x;
}

__global__ void split_suffix_kernel(int n, int nrb, double* __restrict__ colpart) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double run = 0.0;
  for (int b = nrb - 1; b >= 0; --b) {
    const double t = colpart[b + (size_t)j * nrb];
    colpart[b + (size_t)j * nrb] = run;
    run += t;
  }
}

__global__ void split_rowmax_kernel(int n, const double* __restrict__ A, int lda, int nrb,
                                    const double* __restrict__ colpart, int cols_per_block,
                                    unsigned long long* __restrict__ fbits) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int b = blockIdx.x;
  const int k = b * 32 + lane;
  const int jlimit = min(n, (b + 1) * 32);     // only j < k matters
  const int jbeg = blockIdx.y * cols_per_block;
  const int jend = min(jlimit, jbeg + cols_per_block);
  double runmax = 0.0;
  for (int j = jbeg + w; j < jend; j += 8) {
    double x = (k < n) ? fabs(A[k + (size_t)j * lda]) : 0.0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double y = __shfl_down_sync(0xffffffffu, x, o);
      if (lane + o < 32) x += y;
    }
    const double S = x + colpart[b + (size_t)j * nrb];
    if (j < k && S > runmax) runmax = S;
  }
  if (k < n && jbeg < jend) atomic_max_nonneg(&fbits[k], runmax);
}

__global__ void split_finish_kernel(int n, const unsigned long long* __restrict__ fbits,
                                    double inv_norm, double* __restrict__ scores, int accumulate) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x + 1;
  if (k >= n) return;
  const double f = __longlong_as_double((long long)fbits[k]) * inv_norm;
  scores[k - 1] = accumulate ? scores[k - 1] + f : f;
}

cudaError_t split_scores(cudaStream_t s, int n, const double* A, int lda, double inv_norm,
                         double* colpart, double* scores, bool accumulate) {
  if (n < 2) return cudaSuccess;
  const int nrb = (n + 31) / 32;
  // colpart holds nrb*n doubles followed by n unsigned long long for f(k)
  unsigned long long* fbits = reinterpret_cast<unsigned long long*>(colpart + (size_t)nrb * n);
  cudaMemsetAsync(fbits, 0, sizeof(unsigned long long) * n, s);
  dim3 g1(nrb, (n + 7) / 8);
  note_launches(1);
  split_blocksum_kernel<<<g1, 256, 0, s>>>(n, A, lda, nrb, colpart);
  note_launches(1);
  split_suffix_kernel<<<blocks_for(n, 128), 128, 0, s>>>(n, nrb, colpart);
  const int cpb = 256;
  dim3 g3(nrb, (n + cpb - 1) / cpb);
  note_launches(1);
  split_rowmax_kernel<<<g3, 256, 0, s>>>(n, A, lda, nrb, colpart, cpb, fbits);
  note_launches(1);
  split_finish_kernel<<<blocks_for(n, 256), 256, 0, s>>>(n, fbits, inv_norm, scores, accumulate ? 1 : 0);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- strategy data
// diag[i] = A_ii, rad[i] = sum_{j != i} |A_ij| (Gershgorin row discs).
__global__ void gershgorin_kernel(int n, const double* __restrict__ A, int lda,
                                  double* __restrict__ diag, double* __restrict__ rad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double r = 0.0;
  for (int j = 0; j < n; ++j)
    if (j != i) r += fabs(A[i + (size_t)j * lda]);
  diag[i] = A[i + (size_t)i * lda];
  rad[i] = r;
}

cudaError_t diag_gershgorin(cudaStream_t s, int n, const double* A, int lda, double* diag,
                            double* rad) {
  if (n == 0) return cudaSuccess;
  note_launches(1);
  gershgorin_kernel<<<blocks_for(n, 128), 128, 0, s>>>(n, A, lda, diag, rad);
  return cudaGetLastError();
}

// RURV rank decision (one CTA): #{i : |R_ii| > rel_tol * max_i |S_ii|}, with
// R the factor of RURV(A_p) and S that of the RQ step on A_p + B_p, so A_p is
// measured against the size of A_p + B_p (the splitter's matrix is
// (A_p + B_p)^{-1} A_p).
__global__ void count_rank_kernel(int n, const double* __restrict__ R, int ldr,
                                  const double* __restrict__ Sc, int lds, double rel_tol,
                                  int* rank) {
  __shared__ double smax[256];
  __shared__ int scnt[256];
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) m = fmax(m, fabs(Sc[i + (size_t)i * lds]));
  smax[threadIdx.x] = m;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + o]);
    __syncthreads();
  }
  const double thr = rel_tol * smax[0];
  int c = 0;
  if (smax[0] > 0.0)
    for (int i = threadIdx.x; i < n; i += 256) c += (fabs(R[i + (size_t)i * ldr]) > thr) ? 1 : 0;
  scnt[threadIdx.x] = c;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) scnt[threadIdx.x] += scnt[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *rank = scnt[0];
}

cudaError_t count_rank(cudaStream_t s, int n, const double* R, int ldr, const double* Sc, int lds,
                       double rel_tol, int* rank) {
  note_launches(1);
  count_rank_kernel<<<1, 256, 0, s>>>(n, R, ldr, Sc, lds, rel_tol, rank);
  return cudaGetLastError();
}

// Keep the upper triangle and the sub-diagonal entry of each complex 2x2
// block (a pair starts at j when wi[j] > 0 and wi[j+1] = -wi[j]).
__global__ void zero_lower_quasi_kernel(int n, double* T, int ldt, const double* __restrict__ wi) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * n) return;
  const int i = (int)(idx % n), j = (int)(idx / n);
  if (i <= j) return;
  const bool keep = (i == j + 1) && wi[j] > 0.0 && wi[j + 1] == -wi[j];
  if (!keep) T[i + (size_t)j * ldt] = 0.0;
}

cudaError_t zero_lower_quasi(cudaStream_t s, int n, double* T, int ldt, const double* wi) {
  const size_t t = (size_t)n * n;
  if (t == 0) return cudaSuccess;
  note_launches(1);
  zero_lower_quasi_kernel<<<blocks_for(t, 256), 256, 0, s>>>(n, T, ldt, wi);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- SVD embedding
// H (N x N, N = m + n) = [[0, A], [A^T, 0]] for A (m x n).
__global__ void svd_embed_kernel(int m, int n, const double* __restrict__ A, int lda,
                                 double* __restrict__ H, int ldh) {
  const int N = m + n;
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)N * N) return;
  const int i = (int)(idx % N), j = (int)(idx / N);
  double v = 0.0;
  if (i < m && j >= m) v = A[i + (size_t)(j - m) * lda];
  else if (i >= m && j < m) v = A[j + (size_t)(i - m) * lda];
  H[i + (size_t)j * ldh] = v;
}

cudaError_t svd_embed(cudaStream_t s, int m, int n, const double* A, int lda, double* H, int ldh) {
  const size_t t = (size_t)(m + n) * (m + n);
  if (t == 0) return cudaSuccess;
  note_launches(1);
  svd_embed_kernel<<<blocks_for(t, 256), 256, 0, s>>>(m, n, A, lda, H, ldh);
  return cudaGetLastError();
}

// From the eigenpairs of H (eigenvalues ascending in w, vectors in W): the
// r = min(m, n) largest, descending, as singular values S[j] = w[N-1-j] with
// U[:, j] = sqrt(2) W[0:m, N-1-j] and V[:, j] = sqrt(2) W[m:N, N-1-j].
__global__ void svd_extract_kernel(int m, int n, int r, const double* __restrict__ W, int ldw,
                                   const double* __restrict__ w, double* __restrict__ S,
                                   double* __restrict__ U, int ldu, double* __restrict__ V,
                                   int ldv) {
  const int N = m + n;
  const int j = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = N - 1 - j;
  const double s2 = 1.4142135623730951;   // sqrt(2), correctly rounded
  if (i == 0) S[j] = w[c];
  if (i < m) U[i + (size_t)j * ldu] = s2 * W[i + (size_t)c * ldw];
  if (i < n) V[i + (size_t)j * ldv] = s2 * W[m + i + (size_t)c * ldw];
}

cudaError_t svd_extract(cudaStream_t s, int m, int n, const double* W, int ldw, const double* w,
                        double* S, double* U, int ldu, double* V, int ldv) {
  const int r = std::min(m, n);
  if (r == 0) return cudaSuccess;
  dim3 grid((std::max(m, n) + 127) / 128, r);
  note_launches(1);
  svd_extract_kernel<<<grid, 128, 0, s>>>(m, n, r, W, ldw, w, S, U, ldu, V, ldv);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- pencil eigenvalues
// det(S2 - z T2) = a z^2 + b z + c for the 2 x 2 block at (j, j) (T2 upper).
__device__ __forceinline__ void pair_quadratic(const double* S, int lds, const double* T, int ldt,
                                               int j, double& a, double& b, double& c,
                                               double s2[4], double t2[3]) {
  s2[0] = S[j + (size_t)j * lds];
  s2[1] = S[j + (size_t)(j + 1) * lds];
  s2[2] = S[j + 1 + (size_t)j * lds];
  s2[3] = S[j + 1 + (size_t)(j + 1) * lds];
  t2[0] = T[j + (size_t)j * ldt];
  t2[1] = T[j + (size_t)(j + 1) * ldt];
  t2[2] = T[j + 1 + (size_t)(j + 1) * ldt];
  a = t2[0] * t2[2];
  b = -(s2[0] * t2[2] + s2[3] * t2[0] - s2[2] * t2[1]);
  c = s2[0] * s2[3] - s2[1] * s2[2];
}

// Rotation plan for 2 x 2 blocks marked as complex pairs (wi[j] > 0,
// wi[j+1] = -wi[j]) whose generalized eigenvalues are real: for a real
// eigenvalue alpha/beta (in the orientation with the larger leading
// coefficient), x spans the null space of beta S2 - alpha T2 (orthogonal to
// its larger row) and y is the direction of S2 x (or T2 x); the right
// rotation Z = [x, x_perp] and the left one Q = [y, y_perp] make both blocks
// upper triangular.  Writes rot[4j..4j+3] = (x0, x1, y0, y1), act[j] = 1,
// clears the pair in wi_out and sets *flag.
__global__ void pencil_pair_plan_kernel(int n, const double* __restrict__ S, int lds,
                                        const double* __restrict__ T, int ldt,
                                        const double* __restrict__ wi, double* __restrict__ wi_out,
                                        double* __restrict__ rot, int* __restrict__ act,
                                        int* flag) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  act[j] = 0;
  if (!(j + 1 < n && wi[j] > 0.0 && wi[j + 1] == -wi[j])) return;
  double a, b, c, s2[4], t2[3];
  pair_quadratic(S, lds, T, ldt, j, a, b, c, s2, t2);
  const double disc = b * b - 4.0 * a * c;
  if (disc < 0.0 || (a == 0.0 && c == 0.0)) return;
  const double r = sqrt(disc);
  const double q = -0.5 * (b + (b >= 0.0 ? r : -r));
  double alpha, beta;
  if (fabs(a) >= fabs(c)) { alpha = q != 0.0 ? q / a : 0.0; beta = 1.0; }
  else { alpha = 1.0; beta = q != 0.0 ? q / c : 0.0; }
  // N = beta S2 - alpha T2 (T2 lower-left is zero)
  const double n00 = beta * s2[0] - alpha * t2[0], n01 = beta * s2[1] - alpha * t2[1];
  const double n10 = beta * s2[2], n11 = beta * s2[3] - alpha * t2[2];
  double x0, x1;
  if (hypot(n00, n01) >= hypot(n10, n11)) { x0 = -n01; x1 = n00; }
  else { x0 = -n11; x1 = n10; }
  double h = hypot(x0, x1);
  if (h == 0.0) { x0 = 1.0; x1 = 0.0; } else { x0 /= h; x1 /= h; }
  const double u0 = s2[0] * x0 + s2[1] * x1, u1 = s2[2] * x0 + s2[3] * x1;
  const double v0 = t2[0] * x0 + t2[1] * x1, v1 = t2[2] * x1;
  double y0, y1;
  if (hypot(u0, u1) >= hypot(v0, v1)) { y0 = u0; y1 = u1; } else { y0 = v0; y1 = v1; }
  h = hypot(y0, y1);
  if (h == 0.0) { y0 = 1.0; y1 = 0.0; } else { y0 /= h; y1 /= h; }
  rot[4 * (size_t)j] = x0;
  rot[4 * (size_t)j + 1] = x1;
  rot[4 * (size_t)j + 2] = y0;
  rot[4 * (size_t)j + 3] = y1;
  act[j] = 1;
  wi_out[j] = 0.0;
  wi_out[j + 1] = 0.0;
  atomicOr(flag, 1);
}

// Columns j, j+1 of S, T, QR times Z and of QL times Q, for every active pair
// (blockIdx.y = pair start j; column pairs of different pairs are disjoint).
__global__ void pencil_pair_cols_kernel(int n, const double* __restrict__ rot,
                                        const int* __restrict__ act, double* S, int lds,
                                        double* T, int ldt, double* QL, int ldql, double* QR,
                                        int ldqr) {
  const int j = blockIdx.y;
  if (!act[j]) return;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const double x0 = rot[4 * (size_t)j], x1 = rot[4 * (size_t)j + 1];
  const double y0 = rot[4 * (size_t)j + 2], y1 = rot[4 * (size_t)j + 3];
  auto rz = [&](double* M, int ld, double c0, double c1) {
    double* p = M + r + (size_t)j * ld;
    double* q = M + r + (size_t)(j + 1) * ld;
    const double a = *p, b = *q;
    *p = a * c0 + b * c1;      // [a b] [[c0 -c1] [c1 c0]]
    *q = -a * c1 + b * c0;
  };
  rz(S, lds, x0, x1);
  rz(T, ldt, x0, x1);
  rz(QR, ldqr, x0, x1);
  rz(QL, ldql, y0, y1);
}

// Rows j, j+1 of S and T times Q^T for every active pair (row pairs disjoint);
// the block's lower-left entries are set to zero.
__global__ void pencil_pair_rows_kernel(int n, const double* __restrict__ rot,
                                        const int* __restrict__ act, double* S, int lds,
                                        double* T, int ldt) {
  const int j = blockIdx.y;
  if (!act[j]) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const double y0 = rot[4 * (size_t)j + 2], y1 = rot[4 * (size_t)j + 3];
  auto rq = [&](double* M, int ld) {
    double* p = M + j + (size_t)c * ld;
    double* q = p + 1;
    const double a = *p, b = *q;
    *p = y0 * a + y1 * b;      // [[y0 y1] [-y1 y0]] [a; b]
    *q = -y1 * a + y0 * b;
    if (c == j) *q = 0.0;
  };
  rq(S, lds);
  rq(T, ldt);
}

cudaError_t pencil_split_real_pairs(cudaStream_t s, int n, double* S, int lds, double* T, int ldt,
                                    double* QL, int ldql, double* QR, int ldqr, double* wi,
                                    double* scratch, int* act, int* flag, int* hflag) {
  if (n < 2) {
    *hflag = 0;
    return cudaSuccess;
  }
  double* wi_out = scratch;               // n
  double* rot = scratch + n;              // 4n
  cudaError_t e = cudaMemcpyAsync(wi_out, wi, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(flag, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  note_launches(1);
  pencil_pair_plan_kernel<<<blocks_for(n, 128), 128, 0, s>>>(n, S, lds, T, ldt, wi, wi_out, rot,
                                                             act, flag);
  e = cudaMemcpyAsync(hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess || !*hflag) return e;
  dim3 grid((n + 255) / 256, n - 1);
  note_launches(2);
  pencil_pair_cols_kernel<<<grid, 256, 0, s>>>(n, rot, act, S, lds, T, ldt, QL, ldql, QR, ldqr);
  pencil_pair_rows_kernel<<<grid, 256, 0, s>>>(n, rot, act, S, lds, T, ldt);
  return cudaMemcpyAsync(wi, wi_out, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
}

// (alpha_re, alpha_im, beta) of a pencil in generalized real Schur form: S
// quasi-upper-triangular, T upper triangular.  A 1 x 1 block gives
// (s_ii, 0, t_ii); a 2 x 2 block (wi[i] > 0, wi[i+1] = -wi[i]) its roots of
// det(S2 - z T2) = a z^2 + b z + c, solved in the orientation with the larger
// leading coefficient: z = alpha, beta = 1 if |a| >= |c|, else the roots
// w = p +- i q of c w^2 + b w + a give alpha = p -+ i q, beta = p^2 + q^2.
// The first index of a pair carries the positive imaginary part.  One thread
// per index; both threads of a block evaluate the same quadratic.
__global__ void pencil_alpha_beta_kernel(int n, const double* __restrict__ S, int lds,
                                         const double* __restrict__ T, int ldt,
                                         const double* __restrict__ wi, double* __restrict__ ar,
                                         double* __restrict__ ai, double* __restrict__ be) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const bool first = i + 1 < n && wi[i] > 0.0 && wi[i + 1] == -wi[i];
  const bool second = i > 0 && wi[i - 1] > 0.0 && wi[i] == -wi[i - 1];
  if (!first && !second) {
    ar[i] = S[i + (size_t)i * lds];
    ai[i] = 0.0;
    be[i] = T[i + (size_t)i * ldt];
    return;
  }
  const int j = first ? i : i - 1;
  double a, b, c, s2[4], t2[3];
  pair_quadratic(S, lds, T, ldt, j, a, b, c, s2, t2);
  const bool direct = fabs(a) >= fabs(c);
  const double lead = direct ? a : c;
  const double disc = b * b - 4.0 * a * c;
  if (disc < 0.0) {
    const double re = -b / (2.0 * lead);
    const double im = sqrt(-disc) / (2.0 * fabs(lead));
    ar[i] = re;
    ai[i] = first ? im : -im;
    be[i] = direct ? 1.0 : re * re + im * im;
  } else {
    const double r = sqrt(disc);
    const double w = (first ? (-b + r) : (-b - r)) / (2.0 * lead);
    ar[i] = direct ? w : 1.0;
    ai[i] = 0.0;
    be[i] = direct ? 1.0 : w;
  }
}

cudaError_t pencil_alpha_beta(cudaStream_t s, int n, const double* S, int lds, const double* T,
                              int ldt, const double* wi, double* ar, double* ai, double* be) {
  if (n == 0) return cudaSuccess;
  note_launches(1);
  pencil_alpha_beta_kernel<<<blocks_for(n, 128), 128, 0, s>>>(n, S, lds, T, ldt, wi, ar, ai, be);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- refinement
// One FP64 refinement step for a symmetric eigendecomposition from approximate
// eigenvectors X (Ogita and Aishima, "Iterative refinement for symmetric
// eigenvalue decomposition", 2018): with G = X^T X and S = X^T A X,
//   lam_i = s_ii / g_ii,  R = I - G,
//   E_ij = (s_ij + lam_j r_ij) / (lam_j - lam_i) if |lam_i - lam_j| > delta,
//   E_ij = r_ij / 2 otherwise (and on the diagonal),
// and X <- X + X E.
__global__ void oa_diag_kernel(int n, const double* __restrict__ G, const double* __restrict__ S,
                               double* __restrict__ lam, unsigned long long* maxabs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double l = S[i + (size_t)i * n] / G[i + (size_t)i * n];
  lam[i] = l;
  atomic_max_nonneg(maxabs, fabs(l));
}

// max_{i != j} |s_ij| -> bits[0], max_{i,j} |r_ij| -> bits[1]
__global__ void oa_offmax_kernel(int n, const double* __restrict__ G, const double* __restrict__ S,
                                 unsigned long long* bits) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double so = 0.0, ro = 0.0;
  if (idx < (size_t)n * n) {
    const int i = (int)(idx % n), j = (int)(idx / n);
    const double r = ((i == j) ? 1.0 : 0.0) - G[idx];
    ro = fabs(r);
    if (i != j) so = fabs(S[idx]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    so = fmax(so, __shfl_xor_sync(0xffffffffu, so, o));
    ro = fmax(ro, __shfl_xor_sync(0xffffffffu, ro, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomic_max_nonneg(&bits[0], so);
    atomic_max_nonneg(&bits[1], ro);
  }
}

// Pair (i, j) counts as separated when |lam_i - lam_j| > delta and the
// first-order correction stays below 1/64 (reading: a per-pair form of the
// paper's global delta, so one close pair does not stop the others).
__global__ void oa_correction_kernel(int n, const double* __restrict__ G,
                                     const double* __restrict__ S, const double* __restrict__ lam,
                                     double delta, double* __restrict__ E) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * n) return;
  const int i = (int)(idx % n), j = (int)(idx / n);
  const double r = ((i == j) ? 1.0 : 0.0) - G[idx];
  double e = 0.5 * r;
  if (i != j) {
    const double num = S[idx] + lam[j] * r;
    const double gap = lam[j] - lam[i];
    if (fabs(gap) > delta && fabs(gap) > 64.0 * fabs(num)) e = num / gap;
  }
  E[idx] = e;
}

// lam_i = (x_i . (A x_i)) / (x_i . x_i), one warp per column
__global__ void add_inplace_kernel(size_t count, double* __restrict__ X, const double* __restrict__ D) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < count) X[idx] += D[idx];
}

cudaError_t add_inplace(cudaStream_t s, size_t count, double* X, const double* D) {
  if (count == 0) return cudaSuccess;
  note_launches(1);
  add_inplace_kernel<<<blocks_for(count, 256), 256, 0, s>>>(count, X, D);
  return cudaGetLastError();
}

cudaError_t oa_diag(cudaStream_t s, int n, const double* G, const double* S, double* lam,
                    unsigned long long* maxabs) {
  note_launches(1);
  oa_diag_kernel<<<blocks_for(n, 256), 256, 0, s>>>(n, G, S, lam, maxabs);
  return cudaGetLastError();
}

cudaError_t oa_offmax(cudaStream_t s, int n, const double* G, const double* S,
                      unsigned long long* bits) {
  note_launches(1);
  oa_offmax_kernel<<<blocks_for((size_t)n * n, 256), 256, 0, s>>>(n, G, S, bits);
  return cudaGetLastError();
}

cudaError_t oa_correction(cudaStream_t s, int n, const double* G, const double* S,
                          const double* lam, double delta, double* E) {
  note_launches(1);
  oa_correction_kernel<<<blocks_for((size_t)n * n, 256), 256, 0, s>>>(n, G, S, lam, delta, E);
  return cudaGetLastError();
}

}  // namespace eigdc
