// Leaf solvers of the recursion ("the standard algorithm" for small
// subproblems, Sec. 3.6): one CTA per leaf of size <= 64, the whole leaf and
// its vectors resident in shared memory.
//   * symmetric leaves: Jacobi with the parallel (round-robin) ordering, the
//     m/2 rotations of a round act on disjoint index pairs and are applied
//     together; sweeps until off(A) <= m u ||A||_F (u = 2^-53);
//   * nonsymmetric leaves: Householder Hessenberg reduction, then Francis
//     implicit double-shift QR steps with deflation on
//     |h_{i+1,i}| <= u (|h_ii| + |h_{i+1,i+1}|) and standardised 2x2 blocks
//     (Golub and Van Loan, Matrix Computations, Ch. 7-8).
// The control decisions (deflation, shifts) are taken by thread 0 and
// broadcast through shared memory; the row / column updates are spread over
// the threads.  Every loop has a fixed iteration budget.
#include <cuda_runtime.h>
#include <math.h>

#include "internal.h"
#include "jacobi_leaf.cuh"

namespace eigdc {

constexpr int LMAX = 64;
constexpr double U_ROUND = 1.1102230246251565e-16;   // 2^-53

// ---------------------------------------------------------------- Jacobi
// One CTA per leaf; the solver body (jacobi_leaf.cuh) is shared with the
// fused batched solver.
__global__ void __launch_bounds__(JL_THREADS)
jacobi_kernel(const LeafDesc* __restrict__ desc, const double* __restrict__ A, int lda,
              double* __restrict__ w, double* __restrict__ Z, int* status) {
  __shared__ JacobiShared J;
  const LeafDesc d = desc[blockIdx.x];
  const bool ok = jacobi_leaf(d.m, A + (size_t)d.off + (size_t)d.off * lda, lda, w + d.off,
                              Z + d.zoff, LMAX, J);
  if (threadIdx.x == 0 && !ok) atomicOr(status, 1);
}

cudaError_t jacobi_leaves(cudaStream_t s, int count, const LeafDesc* d_desc, const double* A,
                          int lda, double* w, double* Z, int* status) {
  if (count == 0) return cudaSuccess;
  note_launches(1);
  jacobi_kernel<<<count, JL_THREADS, 0, s>>>(d_desc, A, lda, w, Z, status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- Francis
// Reflector of a short vector (one thread): (I - beta v v^T) x = ||x|| e1, v[0] = 1.
__device__ void house_small(const double* x, int len, double* v, double& beta) {
  double sigma = 0.0;
  for (int i = 1; i < len; ++i) sigma += x[i] * x[i];
  const double x0 = x[0];
  v[0] = 1.0;
  if (sigma == 0.0) {
    for (int i = 1; i < len; ++i) v[i] = 0.0;
    beta = (x0 >= 0.0) ? 0.0 : 2.0;
    return;
  }
  const double mu = sqrt(x0 * x0 + sigma);
  const double v0 = (x0 <= 0.0) ? (x0 - mu) : (-sigma / (x0 + mu));
  beta = 2.0 * v0 * v0 / (sigma + v0 * v0);
  for (int i = 1; i < len; ++i) v[i] = x[i] / v0;
}

struct FrancisShared {
  double H[LMAX][LMAX + 1];
  double Z[LMAX][LMAX + 1];
  double v[LMAX];
  double xv[LMAX];
  double beta;
  double rc, rs;       // rotation for 2x2 standardisation
  int action, kind, lo, hi, k, q, r, len;
};

// left: H[k0 + i][j] -= beta v_i (v . H[k0:k0+len, j]) for j in [c0, c1)
__device__ __forceinline__ void apply_left(FrancisShared& F, int k0, int len, int c0, int c1) {
  for (int j = c0 + threadIdx.x; j < c1; j += blockDim.x) {
    double dsum = 0.0;
    for (int i = 0; i < len; ++i) dsum += F.v[i] * F.H[k0 + i][j];
    for (int i = 0; i < len; ++i) F.H[k0 + i][j] -= F.beta * (F.v[i] * dsum);
  }
}

// right: M[i][k0 + l] -= beta (M[i, k0:k0+len] . v) v_l for i in [0, r1)
__device__ __forceinline__ void apply_right(double (*M)[LMAX + 1], const double* v, double beta,
                                            int k0, int len, int r1) {
  for (int i = threadIdx.x; i < r1; i += blockDim.x) {
    double e = 0.0;
    for (int l = 0; l < len; ++l) e += M[i][k0 + l] * v[l];
    for (int l = 0; l < len; ++l) M[i][k0 + l] -= beta * (e * v[l]);
  }
}

// rotation G = [[c, -s], [s, c]] on (k, k+1): H <- G^T H G, Z <- Z G
__device__ void apply_rot(FrancisShared& F, int m, int k, double c, double s) {
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    const double r0 = F.H[k][j], r1 = F.H[k + 1][j];
    F.H[k][j] = c * r0 + s * r1;
    F.H[k + 1][j] = -s * r0 + c * r1;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double c0 = F.H[i][k], c1 = F.H[i][k + 1];
    F.H[i][k] = c * c0 + s * c1;
    F.H[i][k + 1] = -s * c0 + c * c1;
    const double z0 = F.Z[i][k], z1 = F.Z[i][k + 1];
    F.Z[i][k] = c * z0 + s * z1;
    F.Z[i][k + 1] = -s * z0 + c * z1;
  }
  __syncthreads();
}

enum { ACT_DONE = 0, ACT_ONE = 1, ACT_TWO = 2, ACT_STEP = 3, ACT_FAIL = 4 };

__global__ void __launch_bounds__(128)
francis_kernel(const LeafDesc* __restrict__ desc, const double* __restrict__ A, int lda,
               double* __restrict__ wr, double* __restrict__ wi, double* __restrict__ Zout,
               int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FrancisShared& F = *reinterpret_cast<FrancisShared*>(smem_raw);
  const LeafDesc d = desc[blockIdx.x];
  const int m = d.m, off = d.off;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < m * m; idx += blockDim.x) {
    const int i = idx % m, j = idx / m;
    F.H[i][j] = A[(size_t)(off + i) + (size_t)(off + j) * lda];
    F.Z[i][j] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  // ---- Hessenberg reduction
  for (int k = 0; k < m - 2; ++k) {
    if (tid == 0) {
      const int len = m - k - 1;
      for (int i = 0; i < len; ++i) F.xv[i] = F.H[k + 1 + i][k];
      house_small(F.xv, len, F.v, F.beta);
      F.len = len;
    }
    __syncthreads();
    if (F.beta != 0.0) {
      apply_left(F, k + 1, F.len, k, m);
      __syncthreads();
      apply_right(F.H, F.v, F.beta, k + 1, F.len, m);
      apply_right(F.Z, F.v, F.beta, k + 1, F.len, m);
      __syncthreads();
      for (int i = k + 2 + tid; i < m; i += blockDim.x) F.H[i][k] = 0.0;
      __syncthreads();
    }
  }
  // ---- Francis double-shift QR with deflation
  int hi = m - 1, its = 0, budget = 40 * (m > 0 ? m : 1);
  bool ok = true;
  while (true) {
    if (tid == 0) {
      int act;
      if (hi < 0) {
        act = ACT_DONE;
      } else if (hi == 0) {
        wr[off] = F.H[0][0];
        wi[off] = 0.0;
        act = ACT_ONE;
      } else {
        int lo = hi;
        while (lo > 0) {
          double scale = fabs(F.H[lo - 1][lo - 1]) + fabs(F.H[lo][lo]);
          if (scale == 0.0) {
            scale = 0.0;
            const int a0 = lo - 1 > 0 ? lo - 1 : 0;
            for (int i = a0; i <= hi; ++i)
              for (int j = a0; j <= hi; ++j) scale += fabs(F.H[i][j]);
          }
          if (fabs(F.H[lo][lo - 1]) <= U_ROUND * scale) {
            F.H[lo][lo - 1] = 0.0;
            break;
          }
          --lo;
        }
        F.lo = lo;
        if (lo == hi) {
          wr[off + hi] = F.H[hi][hi];
          wi[off + hi] = 0.0;
          act = ACT_ONE;
        } else if (lo == hi - 1) {
          act = ACT_TWO;
        } else {
          ++its;
          --budget;
          act = (budget < 0) ? ACT_FAIL : ACT_STEP;
        }
      }
      F.action = act;
      F.hi = hi;
    }
    __syncthreads();
    const int act = F.action;
    if (act == ACT_DONE) break;
    if (act == ACT_FAIL) {
      ok = false;
      break;
    }
    if (act == ACT_ONE) {
      hi -= 1;
      its = 0;
      __syncthreads();
      continue;
    }
    if (act == ACT_TWO) {
      const int k = hi - 1;
      // standardise the 2x2 block at (k, k+1)
      int kind = 0;   // 0: already triangular, 1: real pair, 2: complex pair
      if (tid == 0) {
        const double a = F.H[k][k], b = F.H[k][k + 1], c = F.H[k + 1][k], dd = F.H[k + 1][k + 1];
        if (c == 0.0) {
          F.kind = 0;
        } else {
          const double p = 0.5 * (a - dd);
          const double disc = p * p + b * c;
          if (disc >= 0.0) {
            const double z = p + copysign(sqrt(disc), p);
            const double nrm = hypot(z, c);
            F.rc = z / nrm;
            F.rs = c / nrm;
            F.kind = 1;
          } else {
            const double th = 0.5 * atan2(-(a - dd), b + c);
            F.rc = cos(th);
            F.rs = sin(th);
            F.kind = 2;
          }
        }
      }
      __syncthreads();
      kind = F.kind;
      if (kind != 0) apply_rot(F, m, k, F.rc, F.rs);
      if (tid == 0) {
        if (kind == 0) {
          wr[off + k] = F.H[k][k];
          wi[off + k] = 0.0;
          wr[off + k + 1] = F.H[k + 1][k + 1];
          wi[off + k + 1] = 0.0;
        } else if (kind == 1) {
          F.H[k + 1][k] = 0.0;
          wr[off + k] = F.H[k][k];
          wi[off + k] = 0.0;
          wr[off + k + 1] = F.H[k + 1][k + 1];
          wi[off + k + 1] = 0.0;
        } else {
          const double mid = 0.5 * (F.H[k][k] + F.H[k + 1][k + 1]);
          F.H[k][k] = mid;
          F.H[k + 1][k + 1] = mid;
          const double im = sqrt(fabs(F.H[k][k + 1] * F.H[k + 1][k]));
          wr[off + k] = mid;
          wi[off + k] = im;
          wr[off + k + 1] = mid;
          wi[off + k + 1] = -im;
        }
      }
      hi -= 2;
      its = 0;
      __syncthreads();
      continue;
    }
    // ---- one implicit double-shift step on lo..hi (size >= 3)
    const int lo = F.lo;
    if (tid == 0) {
      const int mh = hi;
      double s, t;
      if (its % 11 == 10) {
        const double wv = fabs(F.H[mh][mh - 1]) + fabs(F.H[mh - 1][mh - 2]);
        s = 1.5 * wv + F.H[mh][mh];
        t = wv * wv;
      } else {
        s = F.H[mh - 1][mh - 1] + F.H[mh][mh];
        t = F.H[mh - 1][mh - 1] * F.H[mh][mh] - F.H[mh - 1][mh] * F.H[mh][mh - 1];
      }
      F.xv[0] = F.H[lo][lo] * F.H[lo][lo] + F.H[lo][lo + 1] * F.H[lo + 1][lo] - s * F.H[lo][lo] + t;
      F.xv[1] = F.H[lo + 1][lo] * (F.H[lo][lo] + F.H[lo + 1][lo + 1] - s);
      F.xv[2] = F.H[lo + 1][lo] * F.H[lo + 2][lo + 1];
    }
    __syncthreads();
    for (int k = lo; k < hi - 1; ++k) {
      if (tid == 0) {
        house_small(F.xv, 3, F.v, F.beta);
        F.q = max(lo, k - 1);
        F.r = min(k + 3, hi);
      }
      __syncthreads();
      apply_left(F, k, 3, F.q, m);
      __syncthreads();
      apply_right(F.H, F.v, F.beta, k, 3, F.r + 1);
      apply_right(F.Z, F.v, F.beta, k, 3, m);
      __syncthreads();
      if (tid == 0) {
        if (k > lo) {
          F.H[k + 1][k - 1] = 0.0;
          F.H[k + 2][k - 1] = 0.0;
        }
        F.xv[0] = F.H[k + 1][k];
        F.xv[1] = F.H[k + 2][k];
        if (k < hi - 2) F.xv[2] = F.H[k + 3][k];
      }
      __syncthreads();
    }
    if (tid == 0) house_small(F.xv, 2, F.v, F.beta);
    __syncthreads();
    apply_left(F, hi - 1, 2, hi - 2, m);
    __syncthreads();
    apply_right(F.H, F.v, F.beta, hi - 1, 2, hi + 1);
    apply_right(F.Z, F.v, F.beta, hi - 1, 2, m);
    __syncthreads();
    if (tid == 0) F.H[hi][hi - 2] = 0.0;
    __syncthreads();
  }
  for (int idx = tid; idx < m * m; idx += blockDim.x) {
    const int i = idx % m, j = idx / m;
    Zout[(size_t)d.zoff + i + (size_t)j * LMAX] = F.Z[i][j];
  }
  if (tid == 0 && !ok) atomicOr(status, 1);
}

cudaError_t francis_leaves(cudaStream_t s, int count, const LeafDesc* d_desc, const double* A,
                           int lda, double* wr, double* wi, double* Z, int* status) {
  if (count == 0) return cudaSuccess;
  static const bool attr = [] {   // once per process (thread-safe static init)
    cudaFuncSetAttribute(francis_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(FrancisShared));
    return true;
  }();
  (void)attr;
  note_launches(1);
  francis_kernel<<<count, 128, sizeof(FrancisShared), s>>>(d_desc, A, lda, wr, wi, Z, status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- pencil leaves
// Generalized real Schur form of a small regular pencil (A, B) (reading for
// the leaves of the pencil recursion): with B = QB RB well conditioned,
// M = A B^{-1} = (A RB^{-1}) QB^T; Francis on M gives M = QL TM QL^T; the RQ
// factorisation QL^T B = R Z gives QR = Z^T, obtained as the column-reversed Q
// of QR(B^T QL J) (J the index reversal).  Phase 1 writes M, phase 2 QR.
constexpr int PL_THREADS = 256;

struct PencilShared {
  double X[LMAX][LMAX + 1];    // matrix being factorised (R on exit)
  double V[LMAX][LMAX + 1];    // Householder vectors, V[j][i] = v_j[i] for i >= j
  double Q[LMAX][LMAX + 1];    // explicit orthogonal factor
  double W[LMAX][LMAX + 1];    // second operand
  double beta[LMAX];
  double red[PL_THREADS / 32];
};

// Householder QR of S.X (m x m) with explicit Q in S.Q (diag R >= 0).
__device__ void smem_qr_explicit(PencilShared& S, int m) {
  const int tid = threadIdx.x;
  for (int j = 0; j < m; ++j) {
    if (tid == 0) {
      double sigma = 0.0;
      for (int i = j + 1; i < m; ++i) sigma += S.X[i][j] * S.X[i][j];
      const double x0 = S.X[j][j];
      double beta, mu, v0;
      if (sigma == 0.0) {
        v0 = 0.0;
        if (x0 >= 0.0) { beta = 0.0; mu = x0; }
        else { beta = 2.0; mu = -x0; }
      } else {
        mu = sqrt(x0 * x0 + sigma);
        v0 = (x0 <= 0.0) ? (x0 - mu) : (-sigma / (x0 + mu));
        beta = 2.0 * v0 * v0 / (sigma + v0 * v0);
      }
      S.V[j][j] = 1.0;
      for (int i = j + 1; i < m; ++i) S.V[j][i] = (v0 != 0.0) ? S.X[i][j] / v0 : 0.0;
      S.beta[j] = beta;
      S.X[j][j] = mu;
      for (int i = j + 1; i < m; ++i) S.X[i][j] = 0.0;
    }
    __syncthreads();
    const double beta = S.beta[j];
    if (beta != 0.0) {
      for (int c = j + 1 + tid; c < m; c += blockDim.x) {
        double d = 0.0;
        for (int i = j; i < m; ++i) d += S.V[j][i] * S.X[i][c];
        for (int i = j; i < m; ++i) S.X[i][c] -= beta * (S.V[j][i] * d);
      }
    }
    __syncthreads();
  }
  // Q = H_0 ... H_{m-1} I, applied last reflector first
  for (int idx = tid; idx < m * m; idx += blockDim.x) {
    const int i = idx % m, c = idx / m;
    S.Q[i][c] = (i == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int j = m - 1; j >= 0; --j) {
    const double beta = S.beta[j];
    if (beta != 0.0) {
      for (int c = tid; c < m; c += blockDim.x) {
        double d = 0.0;
        for (int i = j; i < m; ++i) d += S.V[j][i] * S.Q[i][c];
        for (int i = j; i < m; ++i) S.Q[i][c] -= beta * (S.V[j][i] * d);
      }
    }
    __syncthreads();
  }
}

// Phase 1: M = P Q^{-1} into the diagonal blocks of Mout (ld ldm), (P, Q) =
// (A, B), or (B, A) for a swapped leaf; status bit 2 when Q's triangular
// factor has max|r_ii| / min|r_ii| > 1e8.
__global__ void __launch_bounds__(PL_THREADS)
pencil_leaf_phase1_kernel(const LeafDesc* __restrict__ desc, const double* __restrict__ A,
                          const double* __restrict__ B, int ld, double* __restrict__ Mout,
                          int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PencilShared& S = *reinterpret_cast<PencilShared*>(smem_raw);
  const LeafDesc d = desc[blockIdx.x];
  const int m = d.m, off = d.off, tid = threadIdx.x;
  const double* P = d.swapped ? B : A;
  const double* Qm = d.swapped ? A : B;
  for (int idx = tid; idx < m * m; idx += blockDim.x) {
    const int i = idx % m, j = idx / m;
    S.X[i][j] = Qm[(size_t)(off + i) + (size_t)(off + j) * ld];
    S.W[i][j] = P[(size_t)(off + i) + (size_t)(off + j) * ld];
  }
  __syncthreads();
  smem_qr_explicit(S, m);
  __shared__ int bad;
  if (tid == 0) {
    double mx = 0.0, mn = INFINITY;
    for (int i = 0; i < m; ++i) {
      mx = fmax(mx, fabs(S.X[i][i]));
      mn = fmin(mn, fabs(S.X[i][i]));
    }
    bad = (m > 0 && (mn == 0.0 || mx / mn > 1e8)) ? 1 : 0;
    if (bad) atomicOr(status, 2);
  }
  __syncthreads();
  if (bad) {
    for (int idx = tid; idx < m * m; idx += blockDim.x) {
      const int i = idx % m, j = idx / m;
      Mout[(size_t)(off + i) + (size_t)(off + j) * ld] = 0.0;
    }
    return;
  }
  // rows of X = A R^{-1} (X R = A), each row independent
  for (int i = tid; i < m; i += blockDim.x) {
    for (int j = 0; j < m; ++j) {
      double t = S.W[i][j];
      for (int l = 0; l < j; ++l) t -= S.W[i][l] * S.X[l][j];
      S.W[i][j] = t / S.X[j][j];
    }
  }
  __syncthreads();
  // M = X Q^T
  for (int idx = tid; idx < m * m; idx += blockDim.x) {
    const int i = idx % m, c = idx / m;
    double t = 0.0;
    for (int l = 0; l < m; ++l) t = fma(S.W[i][l], S.Q[c][l], t);
    Mout[(size_t)(off + i) + (size_t)(off + c) * ld] = t;
  }
}

// Phase 2: QR = column-reversed Q of QR(Q^T QL J), Q = B (A when swapped),
// QL = the leaf's Schur vectors (slot in ZL), written to the slot in ZR.  For
// a swapped leaf each complex block (wi[j] > 0, wi[j+1] = -wi[j]) of
// QL^T B QR is 2 x 2; the rotation Z with [b10, b11] Z = [0, r] applied to
// columns j, j+1 of QR makes it upper triangular.
__global__ void __launch_bounds__(PL_THREADS)
pencil_leaf_phase2_kernel(const LeafDesc* __restrict__ desc, const double* __restrict__ A,
                          const double* __restrict__ B, int ld, const double* __restrict__ wi,
                          const double* __restrict__ ZL, double* __restrict__ ZR) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PencilShared& S = *reinterpret_cast<PencilShared*>(smem_raw);
  const LeafDesc d = desc[blockIdx.x];
  const int m = d.m, off = d.off, tid = threadIdx.x;
  const double* Qm = d.swapped ? A : B;
  for (int idx = tid; idx < m * m; idx += blockDim.x) {
    const int i = idx % m, j = idx / m;
    S.W[i][j] = Qm[(size_t)(off + i) + (size_t)(off + j) * ld];
    S.Q[i][j] = ZL[(size_t)d.zoff + i + (size_t)j * LMAX];
  }
  __syncthreads();
  // X = B^T QL J : X[r][j] = sum_i B[i][r] QL[i][m-1-j]
  for (int idx = tid; idx < m * m; idx += blockDim.x) {
    const int r = idx % m, j = idx / m;
    double t = 0.0;
    for (int i = 0; i < m; ++i) t = fma(S.W[i][r], S.Q[i][m - 1 - j], t);
    S.X[r][j] = t;
  }
  __syncthreads();
  smem_qr_explicit(S, m);
  if (d.swapped) {
    // X <- QR (column-reversed Q); W <- B block; V <- QL
    for (int idx = tid; idx < m * m; idx += blockDim.x) {
      const int i = idx % m, j = idx / m;
      S.X[i][j] = S.Q[i][m - 1 - j];
    }
    __syncthreads();
    for (int idx = tid; idx < m * m; idx += blockDim.x) {
      const int i = idx % m, j = idx / m;
      S.W[i][j] = B[(size_t)(off + i) + (size_t)(off + j) * ld];
      S.V[i][j] = ZL[(size_t)d.zoff + i + (size_t)j * LMAX];
    }
    __syncthreads();
    // one thread per complex block; blocks touch disjoint column pairs
    for (int j = tid; j + 1 < m; j += blockDim.x) {
      const double wj = wi[off + j], wj1 = wi[off + j + 1];
      if (!(wj > 0.0 && wj1 == -wj)) continue;
      // row j+1 of QL^T B times columns j, j+1 of QR
      double b10 = 0.0, b11 = 0.0;
      for (int c = 0; c < m; ++c) {
        double t = 0.0;
        for (int i = 0; i < m; ++i) t = fma(S.V[i][j + 1], S.W[i][c], t);
        b10 = fma(t, S.X[c][j], b10);
        b11 = fma(t, S.X[c][j + 1], b11);
      }
      const double r = hypot(b10, b11);
      if (r == 0.0) continue;
      const double z00 = b11 / r, z01 = b10 / r, z10 = -b10 / r, z11 = b11 / r;
      for (int i = 0; i < m; ++i) {
        const double x0 = S.X[i][j], x1 = S.X[i][j + 1];
        S.X[i][j] = x0 * z00 + x1 * z10;
        S.X[i][j + 1] = x0 * z01 + x1 * z11;
      }
    }
    __syncthreads();
    for (int idx = tid; idx < m * m; idx += blockDim.x) {
      const int i = idx % m, j = idx / m;
      ZR[(size_t)d.zoff + i + (size_t)j * LMAX] = S.X[i][j];
    }
    return;
  }
  for (int idx = tid; idx < m * m; idx += blockDim.x) {
    const int i = idx % m, j = idx / m;
    ZR[(size_t)d.zoff + i + (size_t)j * LMAX] = S.Q[i][m - 1 - j];
  }
}

cudaError_t pencil_leaves_phase1(cudaStream_t s, int count, const LeafDesc* d_desc, const double* A,
                                 const double* B, int ld, double* Mout, int* status) {
  if (count == 0) return cudaSuccess;
  static const bool attr = [] {   // once per process (thread-safe static init)
    cudaFuncSetAttribute(pencil_leaf_phase1_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(PencilShared));
    cudaFuncSetAttribute(pencil_leaf_phase2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(PencilShared));
    return true;
  }();
  (void)attr;
  note_launches(1);
  pencil_leaf_phase1_kernel<<<count, PL_THREADS, sizeof(PencilShared), s>>>(d_desc, A, B, ld, Mout,
                                                                              status);
  return cudaGetLastError();
}

cudaError_t pencil_leaves_phase2(cudaStream_t s, int count, const LeafDesc* d_desc, const double* A,
                                 const double* B, int ld, const double* wi, const double* ZL,
                                 double* ZR) {
  if (count == 0) return cudaSuccess;
  note_launches(1);
  pencil_leaf_phase2_kernel<<<count, PL_THREADS, sizeof(PencilShared), s>>>(d_desc, A, B, ld, wi,
                                                                              ZL, ZR);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- U * Z
// For leaf t and a 64-row slab of U: U[rows, off:off+m] <- U[rows, off:off+m] Z_t.
// Each CTA reads its rows of the leaf's columns into shared memory before
// writing them, so in-place use (Uin == Uout) is safe.
__global__ void __launch_bounds__(256)
apply_leaf_vectors_kernel(const LeafDesc* __restrict__ desc, int n, const double* Uin,
                          int ldu_in, double* Uout, int ldu_out, const double* __restrict__ Z) {
  __shared__ double Us[64][LMAX + 1];
  __shared__ double Zs[LMAX][LMAX + 1];
  const LeafDesc d = desc[blockIdx.x];
  const int m = d.m, off = d.off;
  const int r0 = blockIdx.y * 64;
  const int rows = min(64, n - r0);
  if (rows <= 0) return;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < rows * m; idx += 256) {
    const int i = idx % rows, j = idx / rows;
    Us[i][j] = Uin[(size_t)(r0 + i) + (size_t)(off + j) * ldu_in];
  }
  for (int idx = tid; idx < m * m; idx += 256) {
    const int i = idx % m, j = idx / m;
    Zs[i][j] = Z[(size_t)d.zoff + i + (size_t)j * LMAX];
  }
  __syncthreads();
  for (int idx = tid; idx < rows * m; idx += 256) {
    const int i = idx % rows, j = idx / rows;
    double t = 0.0;
    for (int l = 0; l < m; ++l) t = fma(Us[i][l], Zs[l][j], t);
    Uout[(size_t)(r0 + i) + (size_t)(off + j) * ldu_out] = t;
  }
}

cudaError_t apply_leaf_vectors(cudaStream_t s, int count, const LeafDesc* d_desc, int n,
                               const double* Uin, int ldu_in, double* Uout, int ldu_out,
                               const double* Z) {
  if (count == 0 || n == 0) return cudaSuccess;
  dim3 grid(count, (n + 63) / 64);
  note_launches(1);
  apply_leaf_vectors_kernel<<<grid, 256, 0, s>>>(d_desc, n, Uin, ldu_in, Uout, ldu_out, Z);
  return cudaGetLastError();
}

}  // namespace eigdc
