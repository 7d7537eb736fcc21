// Symmetric leaf solver of the recursion ("the standard algorithm" for small
// subproblems, Sec. 3.6) as a CTA-level device function: cyclic Jacobi with
// the parallel (round-robin) ordering on an m x m block (m <= JL_MAX) held in
// shared memory; the m/2 rotations of a round act on disjoint index pairs and
// are applied together; sweeps (at most 40) until off(A) <= m u ||A||_F.
// Used by the one-CTA-per-leaf kernel and by the fused batched solver, so
// both produce the same leaf eigenvalues and vectors from the same block.
// Needs blockDim.x == JL_THREADS.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace eigdc {

constexpr int JL_MAX = 64;
constexpr int JL_THREADS = 256;

struct JacobiShared {
  double S[JL_MAX][JL_MAX + 1];
  double Vs[JL_MAX][JL_MAX + 1];
  int pr[JL_MAX / 2][2];
  double rot[JL_MAX / 2][2];
  double red[JL_THREADS / 32];
  double tol, off;
};

__device__ __forceinline__ void jl_schur2(double app, double aqq, double apq, double& c,
                                          double& s) {
  if (apq == 0.0) {
    c = 1.0;
    s = 0.0;
    return;
  }
  const double tau = (aqq - app) / (2.0 * apq);
  double t;
  if (tau >= 0.0) t = 1.0 / (tau + sqrt(1.0 + tau * tau));
  else t = -1.0 / (-tau + sqrt(1.0 + tau * tau));
  c = 1.0 / sqrt(1.0 + t * t);
  s = t * c;
}

// Eigenvalues of the block A (ld lda) into w[0..m-1], vectors into Z (ld ldz,
// Z[i + j ldz] = component i of vector j).  Returns true when the sweeps
// converged.  Every thread of the CTA must call it.
__device__ inline bool jacobi_leaf(int m, const double* __restrict__ A, int lda,
                                   double* __restrict__ w, double* __restrict__ Z, int ldz,
                                   JacobiShared& J) {
  const int tid = threadIdx.x;
  for (int idx = tid; idx < m * m; idx += JL_THREADS) {
    const int i = idx % m, j = idx / m;
    J.S[i][j] = A[(size_t)i + (size_t)j * lda];
    J.Vs[i][j] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  // ||A||_F
  double f = 0.0;
  for (int idx = tid; idx < m * m; idx += JL_THREADS) {
    const double x = J.S[idx % m][idx / m];
    f = fma(x, x, f);
  }
  for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
  if ((tid & 31) == 0) J.red[tid >> 5] = f;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int q = 0; q < JL_THREADS / 32; ++q) t += J.red[q];
    J.tol = m * 1.1102230246251565e-16 * sqrt(t);
  }
  __syncthreads();
  const int mm = m + (m & 1);
  const int npairs = mm / 2;
  bool converged = (m <= 1);
  for (int sweep = 0; sweep < 40 && !converged; ++sweep) {
    double o2 = 0.0;
    for (int idx = tid; idx < m * m; idx += JL_THREADS) {
      const int i = idx % m, j = idx / m;
      if (i != j) o2 = fma(J.S[i][j], J.S[i][j], o2);
    }
    for (int o = 16; o > 0; o >>= 1) o2 += __shfl_xor_sync(0xffffffffu, o2, o);
    __syncthreads();   // J.red is free again
    if ((tid & 31) == 0) J.red[tid >> 5] = o2;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int q = 0; q < JL_THREADS / 32; ++q) t += J.red[q];
      J.off = sqrt(t);
    }
    __syncthreads();
    if (J.off <= J.tol) {
      converged = true;
      break;
    }
    for (int r = 0; r < mm - 1; ++r) {
      if (tid < npairs) {
        auto pos = [&](int q) { return q == 0 ? 0 : ((q - 1 + r) % (mm - 1)) + 1; };
        int a = pos(tid), b = pos(mm - 1 - tid);
        const int p = min(a, b), q = max(a, b);
        double c = 1.0, s = 0.0;
        if (q < m) jl_schur2(J.S[p][p], J.S[q][q], J.S[p][q], c, s);
        J.pr[tid][0] = p;
        J.pr[tid][1] = q;
        J.rot[tid][0] = c;
        J.rot[tid][1] = s;
      }
      __syncthreads();
      for (int idx = tid; idx < npairs * m; idx += JL_THREADS) {
        const int t = idx / m, j = idx % m;
        const double s = J.rot[t][1];
        if (s == 0.0) continue;
        const double c = J.rot[t][0];
        const int p = J.pr[t][0], q = J.pr[t][1];
        const double a = J.S[p][j], b = J.S[q][j];
        J.S[p][j] = c * a - s * b;
        J.S[q][j] = s * a + c * b;
      }
      __syncthreads();
      for (int idx = tid; idx < npairs * m; idx += JL_THREADS) {
        const int t = idx / m, i = idx % m;
        const double s = J.rot[t][1];
        if (s == 0.0) continue;
        const double c = J.rot[t][0];
        const int p = J.pr[t][0], q = J.pr[t][1];
        const double a = J.S[i][p], b = J.S[i][q];
        J.S[i][p] = c * a - s * b;
        J.S[i][q] = s * a + c * b;
        const double va = J.Vs[i][p], vb = J.Vs[i][q];
        J.Vs[i][p] = c * va - s * vb;
        J.Vs[i][q] = s * va + c * vb;
      }
      __syncthreads();
    }
  }
  for (int i = tid; i < m; i += JL_THREADS) w[i] = J.S[i][i];
  for (int idx = tid; idx < m * m; idx += JL_THREADS) {
    const int i = idx % m, j = idx / m;
    Z[(size_t)i + (size_t)j * ldz] = J.Vs[i][j];
  }
  __syncthreads();
  return converged;
}

}  // namespace eigdc
