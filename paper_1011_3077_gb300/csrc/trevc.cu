// Eigenvectors from the Schur form (the eigenvector section, blocked as in
// its blocked TREVC algorithm) on sm_103a.
//
// Input: the real Schur form A = Q T Q^T with T quasi-upper-triangular in
// standard form (2 x 2 blocks for complex pairs) and wi the imaginary parts,
// or a complex Schur form A = U T U^H (T upper triangular; step 1 is skipped).
//   1. Each 2 x 2 block is made triangular in complex arithmetic by the
//      unitary G whose first column is the block's eigenvector
//      (mu - d, c) / ||.|| for the eigenvalue mu with positive imaginary part:
//      Tc = G^H T G, Qc = Q G (all blocks at once: disjoint index pairs).
//   2. The eigenvector matrix X of Tc (upper triangular, X_jj = 1) solves
//      Tc X = X diag(Tc).  Diagonal blocks of 32 follow the recurrence
//      X_ij = (T_ij X_jj + sum_{k=i+1}^{j-1} T_ik X_kj) / (T_jj - T_ii)
//      inside one CTA each; then, block row by block row from the bottom,
//      the right-hand sides -T(I, I+1:) X(I+1:, I+1:) come from one complex
//      GEMM and (T_II - lambda_j I) X(I, j) = rhs_j is a back substitution
//      per column.  The GEMMs carry the O(n^3) work (the blocked form's point).
//   3. V = Qc X with unit 2-norm columns.
// A pivot T_jj - T_ii below u max |T_ii| is replaced by that value (equal
// eigenvalues give large, finite vectors instead of a division by zero).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/eigdc.h"
#include "internal.h"

namespace eigdc {
namespace {

typedef double2 zt;
constexpr int TB = 32;   // block size of the blocked recurrence

__device__ __forceinline__ zt tz(double r, double i) { return make_double2(r, i); }
__device__ __forceinline__ zt tadd(zt a, zt b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ zt tsub(zt a, zt b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ zt tconj(zt a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ zt tmul(zt a, zt b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ zt tdiv(zt a, zt b) {
  // a / b by scaling with the larger component of b (Smith's method)
  if (fabs(b.x) >= fabs(b.y)) {
    const double r = b.y / b.x, d = b.x + b.y * r;
    return make_double2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
  }
  const double r = b.x / b.y, d = b.y + b.x * r;
  return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
}

int tblocks(long long count, int per) { return (int)((count + per - 1) / per); }

// B (rows x cols complex, ld ldb) = A (real, ld lda)
__global__ void r2c_kernel(int rows, int cols, const double* __restrict__ A, int lda,
                           zt* __restrict__ B, int ldb) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)rows * cols) return;
  const int i = (int)(e % rows), j = (int)(e / rows);
  B[i + (size_t)j * ldb] = tz(A[i + (size_t)j * lda], 0.0);
}

// B (rows x cols complex, ld ldb) = A (complex, ld lda)
__global__ void c2c_kernel(int rows, int cols, const zt* __restrict__ A, int lda,
                           zt* __restrict__ B, int ldb) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)rows * cols) return;
  const int i = (int)(e % rows), j = (int)(e / rows);
  B[i + (size_t)j * ldb] = A[i + (size_t)j * lda];
}

// G of each 2 x 2 block at rows/cols (i, i+1): [[v0, -conj v1], [v1, conj v0]],
// v = (mu - d, c) / ||.||, mu the eigenvalue with positive imaginary part.
__global__ void block_rot_kernel(int nblk, const int* __restrict__ idx, const double* __restrict__ T,
                                 int ldt, zt* __restrict__ G) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nblk) return;
  const int i = idx[b];
  const double a = T[i + (size_t)i * ldt], bb = T[i + (size_t)(i + 1) * ldt];
  const double c = T[i + 1 + (size_t)i * ldt], d = T[i + 1 + (size_t)(i + 1) * ldt];
  const double tr = a + d, det = a * d - bb * c;
  const double q = 0.25 * tr * tr - det;
  zt mu;
  if (q < 0.0) mu = tz(0.5 * tr, sqrt(-q));
  else mu = tz(0.5 * tr + sqrt(q), 0.0);   // not a complex pair: real, no rotation needed
  zt v0 = tz(mu.x - d, mu.y), v1 = tz(c, 0.0);
  const double nv = sqrt(v0.x * v0.x + v0.y * v0.y + v1.x * v1.x + v1.y * v1.y);
  if (nv > 0.0) {
    v0 = tz(v0.x / nv, v0.y / nv);
    v1 = tz(v1.x / nv, v1.y / nv);
  } else {
    v0 = tz(1.0, 0.0);
    v1 = tz(0.0, 0.0);
  }
  G[4 * b + 0] = v0;
  G[4 * b + 1] = tz(-v1.x, v1.y);   // -conj(v1)
  G[4 * b + 2] = v1;
  G[4 * b + 3] = tconj(v0);
}

// columns (i, i+1) of T and Q times G, for every block
__global__ void rot_cols_kernel(int n, int nblk, const int* __restrict__ idx, const zt* __restrict__ G,
                                zt* __restrict__ T, int ldt, zt* __restrict__ Q, int ldq) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * nblk) return;
  const int r = (int)(e % n), b = (int)(e / n);
  const int i = idx[b];
  const zt g00 = G[4 * b], g01 = G[4 * b + 1], g10 = G[4 * b + 2], g11 = G[4 * b + 3];
  zt x0 = T[r + (size_t)i * ldt], x1 = T[r + (size_t)(i + 1) * ldt];
  T[r + (size_t)i * ldt] = tadd(tmul(x0, g00), tmul(x1, g10));
  T[r + (size_t)(i + 1) * ldt] = tadd(tmul(x0, g01), tmul(x1, g11));
  x0 = Q[r + (size_t)i * ldq];
  x1 = Q[r + (size_t)(i + 1) * ldq];
  Q[r + (size_t)i * ldq] = tadd(tmul(x0, g00), tmul(x1, g10));
  Q[r + (size_t)(i + 1) * ldq] = tadd(tmul(x0, g01), tmul(x1, g11));
}

// rows (i, i+1) of T times G^H from the left, for every block; T(i+1, i) = 0
__global__ void rot_rows_kernel(int n, int nblk, const int* __restrict__ idx, const zt* __restrict__ G,
                                zt* __restrict__ T, int ldt) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * nblk) return;
  const int c = (int)(e % n), b = (int)(e / n);
  const int i = idx[b];
  const zt g00 = G[4 * b], g01 = G[4 * b + 1], g10 = G[4 * b + 2], g11 = G[4 * b + 3];
  const zt y0 = T[i + (size_t)c * ldt], y1 = T[i + 1 + (size_t)c * ldt];
  T[i + (size_t)c * ldt] = tadd(tmul(tconj(g00), y0), tmul(tconj(g10), y1));
  T[i + 1 + (size_t)c * ldt] = c == i ? tz(0.0, 0.0) : tadd(tmul(tconj(g01), y0), tmul(tconj(g11), y1));
}

// T(i+1, i) = 0 below each complex pair's diagonal (separately zeroed where the
// row pass left rounding); also zero every other entry below the diagonal.
__global__ void lower_zero_kernel(int n, zt* __restrict__ T, int ldt) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  const int i = (int)(e % n), j = (int)(e / n);
  if (i > j) T[i + (size_t)j * ldt] = tz(0.0, 0.0);
}

// Diagonal blocks of X (one CTA per block of TB): X_jj = 1 and the recurrence
// X_ij = (T_ij + sum_{k=i+1}^{j-1} T_ik X_kj) / (T_jj - T_ii); one thread per column.
// A denominator of modulus below smin (u max |T_ii|) is replaced by smin, so
// an exact double eigenvalue gives a large, finite vector.
__device__ __forceinline__ zt guard_pivot(zt d, double smin) {
  return (d.x * d.x + d.y * d.y < smin * smin) ? tz(smin, 0.0) : d;
}

__global__ void __launch_bounds__(TB) trevc_diag_kernel(int n, const zt* __restrict__ T, int ldt,
                                                        zt* __restrict__ X, int ldx, double smin) {
  __shared__ zt Ts[TB][TB + 1];
  __shared__ zt Xs[TB][TB + 1];
  const int J0 = blockIdx.x * TB;
  const int bj = min(TB, n - J0);
  for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
    const int i = e % TB, j = e / TB;
    Ts[i][j] = (i < bj && j < bj) ? T[J0 + i + (size_t)(J0 + j) * ldt] : tz(0.0, 0.0);
    Xs[i][j] = tz(0.0, 0.0);
  }
  __syncthreads();
  const int j = threadIdx.x;
  if (j < bj) {
    Xs[j][j] = tz(1.0, 0.0);
    const zt lam = Ts[j][j];
    for (int i = j - 1; i >= 0; --i) {
      zt s = Ts[i][j];
      for (int k = i + 1; k < j; ++k) s = tadd(s, tmul(Ts[i][k], Xs[k][j]));
      Xs[i][j] = tdiv(s, guard_pivot(tsub(lam, Ts[i][i]), smin));
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < bj * bj; e += blockDim.x) {
    const int i = e % bj, jj = e / bj;
    X[J0 + i + (size_t)(J0 + jj) * ldx] = Xs[i][jj];
  }
}

// Block row I (rows I0 .. I0+bi-1) of X for the columns c0 .. n-1:
// (T_II - lambda_j I) x = rhs(:, j - c0), back substitution, one thread per column.
__global__ void __launch_bounds__(128) trevc_row_kernel(int n, int I0, int bi, int c0,
                                                        const zt* __restrict__ T, int ldt,
                                                        const zt* __restrict__ rhs, int ldr,
                                                        zt* __restrict__ X, int ldx, double smin) {
  __shared__ zt Ts[TB][TB + 1];
  for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
    const int i = e % TB, j = e / TB;
    Ts[i][j] = (i < bi && j < bi) ? T[I0 + i + (size_t)(I0 + j) * ldt] : tz(0.0, 0.0);
  }
  __syncthreads();
  const int j = c0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const zt lam = T[j + (size_t)j * ldt];
  zt x[TB];
#pragma unroll
  for (int r = 0; r < TB; ++r) x[r] = tz(0.0, 0.0);
#pragma unroll
  for (int r = TB - 1; r >= 0; --r) {
    if (r < bi) {
      zt s = rhs[r + (size_t)(j - c0) * ldr];
#pragma unroll
      for (int q = r + 1; q < TB; ++q)
        if (q < bi) s = tsub(s, tmul(Ts[r][q], x[q]));
      // (T_rr - lambda_j) x_r = s: the guarded pivot is -(lambda_j - T_rr)
      const zt g = guard_pivot(tsub(lam, Ts[r][r]), smin);
      x[r] = tdiv(s, tz(-g.x, -g.y));
    }
  }
#pragma unroll
  for (int r = 0; r < TB; ++r)
    if (r < bi) X[I0 + r + (size_t)j * ldx] = x[r];
}

// unit 2-norm columns (one CTA per column, fixed summation order)
__global__ void colnorm_kernel(int n, zt* __restrict__ V, int ldv) {
  __shared__ double red[8];
  __shared__ double s_inv;
  const int j = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) {
    const zt v = V[i + (size_t)j * ldv];
    acc += v.x * v.x + v.y * v.y;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    s_inv = t > 0.0 ? 1.0 / sqrt(t) : 1.0;
  }
  __syncthreads();
  const double inv = s_inv;
  for (int i = threadIdx.x; i < n; i += 256) {
    const zt v = V[i + (size_t)j * ldv];
    V[i + (size_t)j * ldv] = tz(v.x * inv, v.y * inv);
  }
}

__global__ void diag_kernel(int n, const zt* __restrict__ T, int ldt, zt* __restrict__ lam) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) lam[i] = T[i + (size_t)i * ldt];
}

}  // namespace

int trevc(cudaStream_t s, int n, const double* dT, int ldt, const double* dQ, int ldq,
          const double* dwi, double* dV_, int ldv, double* dlam_, std::string* err,
          bool complex_in) {
  NvtxRange nvtx_("eig.trevc");
  zt* dV = reinterpret_cast<zt*>(dV_);
  zt* dlam = reinterpret_cast<zt*>(dlam_);
  std::vector<void*> owned;
  auto cleanup = [&]() {
    cudaStreamSynchronize(s);
    for (void* p : owned) cudaFreeAsync(p, s);
    cudaStreamSynchronize(s);
  };
  auto fail = [&](cudaError_t e, const char* what) {
    *err = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
    cleanup();
    return EIG_ERR_CUDA;
  };
  auto alloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMallocAsync(&p, std::max<size_t>(bytes, 256), s) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    owned.push_back(p);
    return p;
  };
  const size_t nn = (size_t)n * n;
  zt* Tc = static_cast<zt*>(alloc(nn * sizeof(zt)));
  zt* Qc = static_cast<zt*>(alloc(nn * sizeof(zt)));
  zt* X = static_cast<zt*>(alloc(nn * sizeof(zt)));
  zt* rhs = static_cast<zt*>(alloc((size_t)TB * n * sizeof(zt)));
  if (!Tc || !Qc || !X || !rhs) {
    *err = "eigenvector workspace allocation failed";
    cleanup();
    return EIG_ERR_NOMEM;
  }
  cudaError_t e = cudaSuccess;
  std::vector<int> hidx;
  if (!complex_in) {
    // complex pairs from wi (host): a pair starts where wi > 0 and wi[i+1] = -wi[i]
    std::vector<double> hwi(n);
    e = cudaMemcpyAsync(hwi.data(), dwi, sizeof(double) * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(e, "wi copy");
    for (int i = 0; i + 1 < n; ++i)
      if (hwi[i] > 0.0 && hwi[i + 1] == -hwi[i]) {
        hidx.push_back(i);
        ++i;
      }
  }
  const int nblk = (int)hidx.size();
  note_launches(2);
  if (complex_in) {
    // a complex Schur form: already triangular
    c2c_kernel<<<tblocks((long long)nn, 256), 256, 0, s>>>(n, n, reinterpret_cast<const zt*>(dT), ldt, Tc, n);
    c2c_kernel<<<tblocks((long long)nn, 256), 256, 0, s>>>(n, n, reinterpret_cast<const zt*>(dQ), ldq, Qc, n);
  } else {
    r2c_kernel<<<tblocks((long long)nn, 256), 256, 0, s>>>(n, n, dT, ldt, Tc, n);
    r2c_kernel<<<tblocks((long long)nn, 256), 256, 0, s>>>(n, n, dQ, ldq, Qc, n);
  }
  cudaMemsetAsync(X, 0, nn * sizeof(zt), s);
  if (nblk > 0) {
    int* didx = static_cast<int*>(alloc(sizeof(int) * nblk));
    zt* G = static_cast<zt*>(alloc(sizeof(zt) * 4 * nblk));
    if (!didx || !G) {
      *err = "eigenvector workspace allocation failed";
      cleanup();
      return EIG_ERR_NOMEM;
    }
    e = cudaMemcpyAsync(didx, hidx.data(), sizeof(int) * nblk, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail(e, "block index copy");
    note_launches(3);
    block_rot_kernel<<<tblocks(nblk, 128), 128, 0, s>>>(nblk, didx, dT, ldt, G);
    rot_cols_kernel<<<tblocks((long long)n * nblk, 256), 256, 0, s>>>(n, nblk, didx, G, Tc, n, Qc, n);
    rot_rows_kernel<<<tblocks((long long)n * nblk, 256), 256, 0, s>>>(n, nblk, didx, G, Tc, n);
  }
  note_launches(1);
  lower_zero_kernel<<<tblocks((long long)nn, 256), 256, 0, s>>>(n, Tc, n);
  // smin = u max |T_ii| from the diagonal of Tc
  std::vector<double> hd(2 * (size_t)n);
  e = cudaMemcpy2DAsync(hd.data(), 2 * sizeof(double), Tc, (n + 1) * sizeof(zt), 2 * sizeof(double), n,
                        cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(e, "diagonal copy");
  double top = 0.0;
  for (int i = 0; i < n; ++i) top = std::max(top, std::hypot(hd[2 * i], hd[2 * i + 1]));
  const double smin = std::max(0x1p-53 * top, 0x1p-1022);
  const int nb = (n + TB - 1) / TB;
  note_launches(1);
  trevc_diag_kernel<<<nb, TB, 0, s>>>(n, Tc, n, X, n, smin);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "diagonal blocks");
  const zt one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0), mone = make_double2(-1.0, 0.0);
  for (int I = nb - 2; I >= 0; --I) {
    const int I0 = I * TB, bi = std::min(TB, n - I0), c0 = I0 + bi, nc = n - c0;
    // rhs = -T(I, c0:n) X(c0:n, c0:n)
    if ((e = zgemm(s, false, false, bi, nc, nc, mone, Tc + I0 + (size_t)c0 * n, n, X + c0 + (size_t)c0 * n,
                   n, zero, rhs, TB)) != cudaSuccess)
      return fail(e, "block row GEMM");
    note_launches(1);
    trevc_row_kernel<<<tblocks(nc, 128), 128, 0, s>>>(n, I0, bi, c0, Tc, n, rhs, TB, X, n, smin);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "block row solve");
  }
  if ((e = zgemm(s, false, false, n, n, n, one, Qc, n, X, n, zero, dV, ldv)) != cudaSuccess)
    return fail(e, "Q X");
  note_launches(2);
  colnorm_kernel<<<n, 256, 0, s>>>(n, dV, ldv);
  diag_kernel<<<tblocks(n, 256), 256, 0, s>>>(n, Tc, n, dlam);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "normalise");
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(e, "synchronize");
  cleanup();
  return EIG_OK;
}

}  // namespace eigdc
