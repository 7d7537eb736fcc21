// Fused batched symmetric eigensolver: the whole randomized spectral
// divide-and-conquer of one problem inside one CTA, and one persistent launch
// for a batch of independent problems (Sec. 4.3: the subproblems of the
// recursion, and a fortiori separate problems, are independent).
//
// Per problem, one CTA runs every row of the path in order:
//   * shift and scale of each node (median of the diagonal plus a Philox
//     jitter, then uniform draws in the middle half of the node's interval,
//     Sec. 3.4) and the Moebius map of the line Re z = sigma;
//   * the inverse-free iteration (Algorithm 3): blocked Householder QR of the
//     stacked [B; -A] (unblocked 32-column panels with one CTA reduction per
//     column, compact-WY trailing updates), the complement Q [0; I], the
//     products Q12^T A and Q22^T B, and the R-test;
//   * the splitter GRURV(2, A_p + B_p, A_p, -1, +1) (Algorithms 1-2) with a
//     Haar V from Philox4x32-10 Gaussians, the RURV rank, the similarity
//     U^T A U with symmetrisation and the 1-norm split test (Algorithm 6);
//   * the recursion with a node stack in global memory, Jacobi leaves
//     (jacobi_leaf.cuh, the same solver as the one-CTA-per-leaf kernel), the
//     eigenvector updates and the final ascending sort.
// The arithmetic, the Philox counters, node ids and every decision (tau,
// split tolerance, tie rule, redraws, empty-side interval shrink, max_fail)
// are those of the host-driven path, so the recursion takes the oracle's tree.
//
// Why one CTA per problem on GB300: the FP64 pipe retires about two DFMA per
// clock per SM, so a CTA of 256 threads running a register-tiled GEMM out of
// 16 KB of shared memory keeps its SM's FP64 units busy, while the host-driven
// path spends roughly two thousand launches and a host round trip per IRS
// squaring on each small problem.  CTAs take problems from an atomic counter,
// largest first; all matrices live in a per-CTA global workspace (L2-resident
// for the small problems this form is for, n <= 512).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "internal.h"
#include "jacobi_leaf.cuh"

namespace eigdc {
namespace {

constexpr int FT = JL_THREADS;   // threads per CTA (the Jacobi body needs 256)
constexpr int FMAX = 512;        // largest problem of the fused form
constexpr int GT = 64, GK = 16;  // CTA GEMM tile (64 x 64 outputs, 4 x 4 per thread)
constexpr int NBMAX = 32;        // widest panel
constexpr int PURPOSE_HAAR = 4;
constexpr int PURPOSE_SHIFT = 5;
constexpr int PURPOSE_POWER = 9;   // start vector of the root's power iteration
constexpr int POWER_STEPS = 16;
constexpr uint64_t ROOT = 1;
constexpr double UR = 1.1102230246251565e-16;   // 2^-53

struct FNode {
  int off, m, depth, pad;
  double lo, hi;
  unsigned long long id;
};

struct FLeaf {
  int off, m;
};

struct GemmSmem {
  double As[GK][GT + 1];
  double Bs[GK][GT + 1];
};

struct PanelSmem {
  double grp[FT / 32][NBMAX + 1];
  double comb0[NBMAX], comb1[NBMAX], dk[NBMAX];
  double bc[4];
  double Tsm[NBMAX][NBMAX + 1];
};

struct CtlSmem {
  double red[FT / 32];
  double dscal[8];
  int iscal[8];
  double sortv[FMAX];
  int sorti[FMAX];
};

// Shared memory of the fused kernel: the phases reuse one area.
struct FusedSmem {
  union {
    struct {
      GemmSmem g;
      PanelSmem p;
    } la;
    JacobiShared jac;
  } u;
  CtlSmem c;
};

// ------------------------------------------------------------------ CTA primitives
__device__ __forceinline__ double fwarp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double fwarp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Sum / max over the CTA, in a fixed order (the same value in every thread).
__device__ double cta_sum(double v, CtlSmem& c) {
  v = fwarp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) c.red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int q = 0; q < FT / 32; ++q) t += c.red[q];
  __syncthreads();
  return t;
}

__device__ double cta_max(double v, CtlSmem& c) {
  v = fwarp_max(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) c.red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int q = 0; q < FT / 32; ++q) t = fmax(t, c.red[q]);
  __syncthreads();
  return t;
}

// C = alpha op(A) op(B) + beta C (column-major; C must not alias A or B; beta
// = 0 does not read C).  64 x 64 output tiles in turn, 16-deep K slabs
// staged in shared memory, thread (tx, ty) owns rows tx + 16 i, columns
// ty + 16 j (i, j < 4): coalesced stores, conflict-free shared reads.
__device__ void cta_gemm(bool ta, bool tb, int m, int n, int k, double alpha,
                         const double* __restrict__ A, int lda, const double* __restrict__ B,
                         int ldb, double beta, double* __restrict__ C, int ldc, GemmSmem& g) {
  if (m <= 0 || n <= 0) return;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int mt = (m + GT - 1) / GT, nt = (n + GT - 1) / GT;
  for (int t = 0; t < mt * nt; ++t) {
    const int r0 = (t % mt) * GT, c0 = (t / mt) * GT;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int k0 = 0; k0 < k; k0 += GK) {
#pragma unroll
      for (int q = 0; q < (GT * GK) / FT; ++q) {
        const int idx = tid + q * FT;
        int r, kk;
        if (!ta) { r = idx % GT; kk = idx / GT; }
        else { kk = idx % GK; r = idx / GK; }
        const int gr = r0 + r, gk = k0 + kk;
        double v = 0.0;
        if (gr < m && gk < k) v = ta ? A[gk + (size_t)gr * lda] : A[gr + (size_t)gk * lda];
        g.As[kk][r] = v;
      }
#pragma unroll
      for (int q = 0; q < (GT * GK) / FT; ++q) {
        const int idx = tid + q * FT;
        int c, kk;
        if (!tb) { kk = idx % GK; c = idx / GK; }
        else { c = idx % GT; kk = idx / GT; }
        const int gc = c0 + c, gk = k0 + kk;
        double v = 0.0;
        if (gc < n && gk < k) v = tb ? B[gc + (size_t)gk * ldb] : B[gk + (size_t)gc * ldb];
        g.Bs[kk][c] = v;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < GK; ++kk) {
        double a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = g.As[kk][tx + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = g.Bs[kk][ty + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + ty + 16 * j;
      if (c >= n) continue;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = r0 + tx + 16 * i;
        if (r >= m) continue;
        double* p = C + r + (size_t)c * ldc;
        double v = alpha * acc[i][j];
        if (beta != 0.0) v = fma(beta, *p, v);
        *p = v;
      }
    }
  }
  __syncthreads();
}

// B = A (rows x cols), element loops over the CTA.
__device__ void cta_copy(int rows, int cols, const double* __restrict__ A, int lda,
                         double* __restrict__ B, int ldb) {
  for (int idx = threadIdx.x; idx < rows * cols; idx += FT) {
    const int i = idx % rows, j = idx / rows;
    B[i + (size_t)j * ldb] = A[i + (size_t)j * lda];
  }
  __syncthreads();
}

// Y (rows x cols) = I in rows r0.. (Y[r0 + j][j] = 1), zero elsewhere.
__device__ void cta_identity(int rows, int cols, int r0, double* Y, int ldy) {
  for (int idx = threadIdx.x; idx < rows * cols; idx += FT) {
    const int i = idx % rows, j = idx / rows;
    Y[i + (size_t)j * ldy] = (i == r0 + j) ? 1.0 : 0.0;
  }
  __syncthreads();
}

// Householder factorisation of the mp x jb panel P (ldp), pivot of column c
// at row c: the reflector of x = P[c:, c] maps it to +||x|| e1 (v_c = 1,
// v_r = x_r / v0; Golub and Van Loan Sec. 5.1).  One CTA reduction per column
// gives sigma = sum_{r>c} x_r^2 together with P'_k = sum_{r>c} x_r P[r, k]
// for every k; then v^T P[:, k] = P[c, k] + P'_k / v0 updates the columns
// k > c and, for k < c, extends the compact-WY T (ps.Tsm, jb x jb upper).
// On exit: R on and above the diagonal, v below it.
__device__ void cta_panel(int mp, int jb, double* __restrict__ P, int ldp, PanelSmem& ps) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int idx = tid; idx < NBMAX * (NBMAX + 1); idx += FT) (&ps.Tsm[0][0])[idx] = 0.0;
  __syncthreads();
  for (int c = 0; c < jb; ++c) {
    double part[NBMAX];
#pragma unroll
    for (int k = 0; k < NBMAX; ++k) part[k] = 0.0;
    for (int r = c + 1 + tid; r < mp; r += FT) {
      const double x = P[r + (size_t)c * ldp];
#pragma unroll
      for (int k = 0; k < NBMAX; ++k)
        if (k < jb) part[k] = fma(x, P[r + (size_t)k * ldp], part[k]);
    }
#pragma unroll
    for (int k = 0; k < NBMAX; ++k) {
      if (k < jb) {
        const double v = fwarp_sum(part[k]);
        if (lane == 0) ps.grp[warp][k] = v;
      }
    }
    __syncthreads();
    if (tid < jb) {
      double t = 0.0;
#pragma unroll
      for (int g = 0; g < FT / 32; ++g) t += ps.grp[g][tid];
      ps.comb0[tid] = t;
      ps.comb1[tid] = (c < mp) ? P[c + (size_t)tid * ldp] : 0.0;
    }
    __syncthreads();
    if (tid == 0) {
      const double sigma = ps.comb0[c];
      const double x0 = ps.comb1[c];
      double beta, mu, v0;
      if (sigma == 0.0) {
        v0 = 0.0;   // v = e1
        if (x0 >= 0.0) { beta = 0.0; mu = x0; }
        else { beta = 2.0; mu = -x0; }
      } else {
        mu = sqrt(x0 * x0 + sigma);
        v0 = (x0 <= 0.0) ? (x0 - mu) : (-sigma / (x0 + mu));
        beta = 2.0 * v0 * v0 / (sigma + v0 * v0);
      }
      ps.bc[0] = beta;
      ps.bc[1] = mu;
      ps.bc[2] = v0;
    }
    __syncthreads();
    const double beta = ps.bc[0], mu = ps.bc[1], v0 = ps.bc[2];
    if (tid < jb) ps.dk[tid] = ps.comb1[tid] + ((v0 != 0.0) ? ps.comb0[tid] / v0 : 0.0);
    for (int r = c + 1 + tid; r < mp; r += FT) {
      double* p = P + r + (size_t)c * ldp;
      *p = (v0 != 0.0) ? *p / v0 : 0.0;
    }
    __syncthreads();
    if (beta != 0.0) {
      for (int r = c + tid; r < mp; r += FT) {
        const double w = (r == c) ? 1.0 : P[r + (size_t)c * ldp];
        for (int k = c + 1; k < jb; ++k) P[r + (size_t)k * ldp] -= beta * ps.dk[k] * w;
      }
    }
    if (tid < c) {
      double t = 0.0;
      for (int l = tid; l < c; ++l) t = fma(ps.Tsm[tid][l], ps.dk[l], t);
      ps.Tsm[tid][c] = -beta * t;
    }
    if (tid == 0) ps.Tsm[c][c] = beta;
    __syncthreads();
    if (tid == 0 && c < mp) P[c + (size_t)c * ldp] = mu;
    __syncthreads();
  }
}

// Blocked Householder QR of W (M x N, M >= N, ldw) in place: R on and above
// the diagonal; the explicit unit-lower-trapezoidal reflectors into V (ldv)
// and the nb x nb T of block b at T + b nb^2 (ld nb): Q = prod_b (I - V_b T_b V_b^T).
// Wk, Wk2: nb x N scratch each.
__device__ void cta_geqrf(int M, int N, int nb, double* W, int ldw, double* V, int ldv, double* T,
                          double* Wk, double* Wk2, FusedSmem& S) {
  const int tid = threadIdx.x;
  for (int j0 = 0; j0 < N; j0 += nb) {
    const int jb = min(nb, N - j0);
    const int mp = M - j0;
    double* P = W + j0 + (size_t)j0 * ldw;
    cta_panel(mp, jb, P, ldw, S.u.la.p);
    double* Vb = V + j0 + (size_t)j0 * ldv;
    for (int idx = tid; idx < mp * jb; idx += FT) {
      const int r = idx % mp, c = idx / mp;
      Vb[r + (size_t)c * ldv] = (r < c) ? 0.0 : ((r == c) ? 1.0 : P[r + (size_t)c * ldw]);
    }
    double* Tb = T + (size_t)(j0 / nb) * nb * nb;
    for (int idx = tid; idx < nb * nb; idx += FT) {
      const int r = idx % nb, c = idx / nb;
      Tb[idx] = (r < jb && c < jb) ? S.u.la.p.Tsm[r][c] : 0.0;
    }
    __syncthreads();
    if (j0 + jb < N) {
      const int nc = N - j0 - jb;
      double* C = W + j0 + (size_t)(j0 + jb) * ldw;
      cta_gemm(true, false, jb, nc, mp, 1.0, Vb, ldv, C, ldw, 0.0, Wk, nb, S.u.la.g);
      cta_gemm(true, false, jb, nc, jb, 1.0, Tb, nb, Wk, nb, 0.0, Wk2, nb, S.u.la.g);
      cta_gemm(false, false, mp, nc, jb, -1.0, Vb, ldv, Wk2, nb, 1.0, C, ldw, S.u.la.g);
    }
  }
}

// Y (M x ncols, ldy) <- Q Y (trans = false: the last block first) or Q^T Y.
__device__ void cta_apply_q(int M, int N, int nb, const double* V, int ldv, const double* T,
                            bool trans, double* Y, int ldy, int ncols, double* Wk, double* Wk2,
                            FusedSmem& S) {
  const int nblk = (N + nb - 1) / nb;
  for (int q = 0; q < nblk; ++q) {
    const int b = trans ? q : nblk - 1 - q;
    const int j0 = b * nb, jb = min(nb, N - j0), mp = M - j0;
    const double* Vb = V + j0 + (size_t)j0 * ldv;
    const double* Tb = T + (size_t)b * nb * nb;
    double* Yb = Y + j0;
    cta_gemm(true, false, jb, ncols, mp, 1.0, Vb, ldv, Yb, ldy, 0.0, Wk, nb, S.u.la.g);
    cta_gemm(trans, false, jb, ncols, jb, 1.0, Tb, nb, Wk, nb, 0.0, Wk2, nb, S.u.la.g);
    cta_gemm(false, false, mp, ncols, jb, -1.0, Vb, ldv, Wk2, nb, 1.0, Yb, ldy, S.u.la.g);
  }
}

// Explicit Q (m x n, orthonormal columns) and R (n x n, diag >= 0) of X = QR;
// X is overwritten.  R may be null.
__device__ void cta_qr_explicit(int m, int n, int nb, double* X, int ldx, double* Q, int ldq,
                                double* R, int ldr, double* V, double* T, double* Wk,
                                double* Wk2, FusedSmem& S) {
  cta_geqrf(m, n, nb, X, ldx, V, m, T, Wk, Wk2, S);
  if (R) {
    for (int idx = threadIdx.x; idx < n * n; idx += FT) {
      const int i = idx % n, j = idx / n;
      R[i + (size_t)j * ldr] = (i <= j) ? X[i + (size_t)j * ldx] : 0.0;
    }
  }
  cta_identity(m, n, 0, Q, ldq);
  cta_apply_q(m, n, nb, V, m, T, false, Q, ldq, n, Wk, Wk2, S);
}

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with the counter layout of
// the library's Gaussian kernel: c0 = pair index, c1 = attempt << 8 | purpose
// << 16, (c2, c3) = stream; key = seed.
__device__ __forceinline__ void fphilox(uint32_t c[4], uint32_t k0, uint32_t k1) {
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

__device__ __forceinline__ void fphilox_counter(uint32_t c[4], uint64_t pair, int purpose,
                                                uint64_t stream, int attempt) {
  c[0] = (uint32_t)(pair & 0xFFFFFFFFull);
  c[1] = (uint32_t)((pair >> 32) & 0xFFull) | ((uint32_t)(attempt & 0xFF) << 8) |
         ((uint32_t)(purpose & 0xFFFF) << 16);
  c[2] = (uint32_t)(stream & 0xFFFFFFFFull);
  c[3] = (uint32_t)(stream >> 32);
}

// G (rows x cols, ldg) ~ N(0, 1): Box-Muller on the two 52-bit uniforms of each pair.
__device__ void cta_gaussian(int rows, int cols, uint64_t seed, int purpose, uint64_t stream,
                             int attempt, double* G, int ldg) {
  const uint64_t count = (uint64_t)rows * cols;
  const uint64_t pairs = (count + 1) / 2;
  for (uint64_t pair = threadIdx.x; pair < pairs; pair += FT) {
    uint32_t c[4];
    fphilox_counter(c, pair, purpose, stream, attempt);
    fphilox(c, (uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32));
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
  __syncthreads();
}

// u2 of pair 0 of (purpose, stream, attempt): a uniform in [0, 1).
__device__ double fphilox_uniform(uint64_t seed, int purpose, uint64_t stream, int attempt) {
  uint32_t c[4];
  fphilox_counter(c, 0, purpose, stream, attempt);
  fphilox(c, (uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32));
  const uint64_t m2 = ((uint64_t)c[2] << 20) | (c[3] >> 12);
  return (double)m2 * 0x1p-52;
}

// splitmix64 finaliser (Steele, Lea, Flood 2014): child ids of the tree.
__device__ __forceinline__ unsigned long long fchild(unsigned long long parent, int side) {
  unsigned long long z = 2ull * parent + (unsigned long long)side + 1ull + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// ------------------------------------------------------------------ sorting
// Ascending bitonic sort of c.sortv[0..cnt) (cnt <= FMAX) carrying c.sorti;
// equal values order by index (a stable order).
__device__ void cta_sort(int cnt, CtlSmem& c) {
  int P = 1;
  while (P < cnt) P <<= 1;
  for (int i = cnt + threadIdx.x; i < P; i += FT) {
    c.sortv[i] = INFINITY;
    c.sorti[i] = 0x7FFFFFFF;
  }
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += FT) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const double a = c.sortv[i], b = c.sortv[ixj];
          const int ia = c.sorti[i], ib = c.sorti[ixj];
          const bool greater = (a > b) || (a == b && ia > ib);
          const bool up = (i & k) == 0;
          if (greater == up) {
            c.sortv[i] = b;
            c.sortv[ixj] = a;
            c.sorti[i] = ib;
            c.sorti[ixj] = ia;
          }
        }
      }
      __syncthreads();
    }
  }
}

// ------------------------------------------------------------------ workspace
struct Ws {
  double *W, *V, *T, *Y, *Aj, *Bj, *An, *Bn, *Rc, *Rp, *Wk, *Wk2;
  double *G, *Vh, *X, *Uq, *R2, *Ss, *Ys, *Z, *Qt, *Ucur, *tmp, *Ahat, *Ssuf;
  double *Unode, *wv, *scores, *zleaf;
  FNode* stack;
  FLeaf* leaves;
};

// Carves the per-CTA workspace for problems up to mx from base (which may be
// null: only the size is wanted); returns the number of doubles used.
__host__ __device__ inline size_t carve(double* base, int mx, Ws* w) {
  const size_t m1 = (size_t)mx * mx, m2 = 2 * m1;
  const size_t nbw = (size_t)NBMAX * (size_t)(mx > 1 ? mx : 1);
  const size_t nbt = (size_t)NBMAX * ((size_t)(mx > 1 ? mx : 1) + NBMAX);   // ceil(m/nb) nb^2
  size_t used = 0;
  auto take = [&](size_t cnt) {
    double* q = base ? base + used : nullptr;
    used += cnt;
    return q;
  };
  Ws t;
  t.W = take(m2); t.V = take(m2); t.Y = take(m2);
  t.Aj = take(m1); t.Bj = take(m1); t.An = take(m1); t.Bn = take(m1); t.Rc = take(m1); t.Rp = take(m1);
  t.G = take(m1); t.Vh = take(m1); t.X = take(m1); t.Uq = take(m1); t.R2 = take(m1); t.Ss = take(m1);
  t.Ys = take(m1); t.Z = take(m1); t.Qt = take(m1); t.Ucur = take(m1); t.tmp = take(m1);
  t.Ahat = take(m1); t.Ssuf = take(m1);
  t.T = take(nbt); t.Wk = take(nbw); t.Wk2 = take(nbw);
  t.Unode = take(m1);
  t.wv = take(mx); t.scores = take(mx + 64); t.zleaf = take(64 * 64);
  t.stack = reinterpret_cast<FNode*>(take((sizeof(FNode) * (size_t)(mx + 2)) / sizeof(double) + 1));
  t.leaves = reinterpret_cast<FLeaf*>(take((sizeof(FLeaf) * (size_t)(mx + 2)) / sizeof(double) + 1));
  if (w) *w = t;
  return (used + 31) & ~(size_t)31;   // 256-byte stride between CTAs
}

// ------------------------------------------------------------------ one problem
struct FParams {
  double tau, split_tol;
  unsigned long long seed;
  int maxit, leaf, max_fail, v_draws, nb;
};

struct IrsRes {
  int iters;
  bool converged;
  bool a_in_j;   // the iterates are in (Aj, Bj) (else in (An, Bn))
};

// Inverse-free iteration (Algorithm 3) on the line Re z = sigma with scale s
// for the m x m symmetric node block An (ld lda): pencil (A - (sigma - s) I,
// A - (sigma + s) I), stacked [B; -A]; stops when ||R_j - R_{j-1}||_1 <= tau
// ||R_{j-1}||_1 or after maxit + 1 squarings.
__device__ IrsRes cta_irs(int m, const double* Anode, int lda, double sigma, double s, double tau,
                          int maxit, int nb, Ws& w, FusedSmem& S) {
  const int tid = threadIdx.x;
  const int m2 = 2 * m;
  double *Aj = w.Aj, *Bj = w.Bj, *An = w.An, *Bn = w.Bn, *Rc = w.Rc, *Rp = w.Rp;
  for (int idx = tid; idx < m * m; idx += FT) {
    const int i = idx % m, j = idx / m;
    const double a = Anode[i + (size_t)j * lda];
    const double b = (i == j) ? 1.0 : 0.0;
    const double am = a - (sigma - s) * b, bm = a - (sigma + s) * b;
    Aj[idx] = am;
    Bj[idx] = bm;
    w.W[i + (size_t)j * m2] = bm;
    w.W[m + i + (size_t)j * m2] = -am;
  }
  __syncthreads();
  IrsRes out{0, false, true};
  bool have_prev = false;
  for (int j = 0;; ++j) {
    cta_geqrf(m2, m, nb, w.W, m2, w.V, m2, w.T, w.Wk, w.Wk2, S);
    // R_j and the R-test sums: max column sums of |R_j - R_{j-1}| and |R_{j-1}|
    double sd = 0.0, sp = 0.0;
    for (int col = tid; col < m; col += FT) {
      double cd = 0.0, cp = 0.0;
      for (int i = 0; i < m; ++i) {
        const double r = (i <= col) ? w.W[i + (size_t)col * m2] : 0.0;
        Rc[i + (size_t)col * m] = r;
        if (have_prev) {
          const double pv = Rp[i + (size_t)col * m];
          cd += fabs(r - pv);
          cp += fabs(pv);
        }
      }
      sd = fmax(sd, cd);
      sp = fmax(sp, cp);
    }
    const double num = cta_max(sd, S.c), den = cta_max(sp, S.c);
    // complement [Q12; Q22] = Q [0; I] and the next iterates
    cta_identity(m2, m, m, w.Y, m2);
    cta_apply_q(m2, m, nb, w.V, m2, w.T, false, w.Y, m2, m, w.Wk, w.Wk2, S);
    cta_gemm(true, false, m, m, m, 1.0, w.Y, m2, Aj, m, 0.0, An, m, S.u.la.g);
    cta_gemm(true, false, m, m, m, 1.0, w.Y + m, m2, Bj, m, 0.0, Bn, m, S.u.la.g);
    for (int idx = tid; idx < m * m; idx += FT) {
      const int i = idx % m, c = idx / m;
      w.W[i + (size_t)c * m2] = Bn[idx];
      w.W[m + i + (size_t)c * m2] = -An[idx];
    }
    __syncthreads();
    double* t0 = Aj; Aj = An; An = t0;
    double* t1 = Bj; Bj = Bn; Bn = t1;
    if (have_prev) {
      const double ratio = den > 0.0 ? num / den : (num == 0.0 ? 0.0 : INFINITY);
      if (ratio <= tau) {
        out.iters = j + 1;
        out.converged = true;
        break;
      }
    }
    double* t2 = Rc; Rc = Rp; Rp = t2;
    have_prev = true;
    if (j + 1 > maxit) {
      out.iters = j + 1;
      out.converged = false;
      break;
    }
  }
  out.a_in_j = (Aj == w.Aj);
  return out;
}

struct SplitRes {
  int k, rank, draw;
  double e;
  bool accepted;
};

// Splitter GRURV(2, A_p + B_p, A_p, -1, +1) for Haar draw `code` into w.Ucur
// and the RURV rank of A_p (Algorithms 1-2, 6), then A^ = U^T A U
// (symmetrised) into w.Ahat and the split scores e(k) into w.scores.
__device__ SplitRes cta_split(int m, const double* Ap, const double* Bp, const double* Anode,
                              int lda, unsigned long long id, int attempt, const FParams& p,
                              Ws& w, FusedSmem& S) {
  const int tid = threadIdx.x;
  const int nb = p.nb;
  // ||A_node||_1
  double cmax = 0.0;
  for (int col = tid; col < m; col += FT) {
    double t = 0.0;
    for (int i = 0; i < m; ++i) t += fabs(Anode[i + (size_t)col * lda]);
    cmax = fmax(cmax, t);
  }
  const double normA = cta_max(cmax, S.c);
  const double inv_norm = normA > 0.0 ? 1.0 / normA : 1.0;
  const double stol = p.split_tol > 0.0 ? p.split_tol : fmax(1e-12, 16.0 * m * UR);
  SplitRes out{0, 0, 0, INFINITY, false};
  const int draws = max(1, p.v_draws);
  for (int draw = 0; draw < draws; ++draw) {
    const int code = ((attempt & 0x3F) << 2) | (draw & 3);
    // Haar V: Q of the QR of a Gaussian (diag R >= 0)
    cta_gaussian(m, m, p.seed, PURPOSE_HAAR, id, code, w.G, m);
    cta_qr_explicit(m, m, nb, w.G, m, w.Vh, m, nullptr, 0, w.V, w.T, w.Wk, w.Wk2, S);
    // RURV(A_p): [U, R2] = QR(A_p V^T)
    cta_gemm(false, true, m, m, m, 1.0, Ap, m, w.Vh, m, 0.0, w.X, m, S.u.la.g);
    cta_qr_explicit(m, m, nb, w.X, m, w.Uq, m, w.R2, m, w.V, w.T, w.Wk, w.Wk2, S);
    // RQ of U^T (A_p + B_p) by reversal: Z = (J Y)^T = Q~ R~, U_cur = Q~ J
    for (int idx = tid; idx < m * m; idx += FT) w.Ss[idx] = Ap[idx] + Bp[idx];
    __syncthreads();
    cta_gemm(true, false, m, m, m, 1.0, w.Uq, m, w.Ss, m, 0.0, w.Ys, m, S.u.la.g);
    for (int idx = tid; idx < m * m; idx += FT) {
      const int i = idx % m, k = idx / m;
      w.Z[i + (size_t)k * m] = w.Ys[(m - 1 - k) + (size_t)i * m];
    }
    __syncthreads();
    cta_qr_explicit(m, m, nb, w.Z, m, w.Qt, m, w.G, m, w.V, w.T, w.Wk, w.Wk2, S);
    // rank: #{|R2_ii| > 1e-8 max_i |R~_ii|}
    double dm = 0.0;
    for (int i = tid; i < m; i += FT) dm = fmax(dm, fabs(w.G[i + (size_t)i * m]));
    const double gmax = cta_max(dm, S.c);
    double cnt = 0.0;
    if (gmax > 0.0)
      for (int i = tid; i < m; i += FT) cnt += (fabs(w.R2[i + (size_t)i * m]) > 1e-8 * gmax) ? 1.0 : 0.0;
    const int rank = (int)cta_sum(cnt, S.c);
    for (int idx = tid; idx < m * m; idx += FT) {
      const int i = idx % m, j = idx / m;
      w.Ucur[i + (size_t)j * m] = w.Qt[i + (size_t)(m - 1 - j) * m];
    }
    __syncthreads();
    // similarity and symmetrisation
    cta_gemm(false, false, m, m, m, 1.0, Anode, lda, w.Ucur, m, 0.0, w.tmp, m, S.u.la.g);
    cta_gemm(true, false, m, m, m, 1.0, w.Ucur, m, w.tmp, m, 0.0, w.Ahat, m, S.u.la.g);
    for (int idx = tid; idx < m * m; idx += FT) {
      const int i = idx % m, j = idx / m;
      if (i < j) {
        const double a = w.Ahat[i + (size_t)j * m], b = w.Ahat[j + (size_t)i * m];
        const double h = 0.5 * (a + b);
        w.Ahat[i + (size_t)j * m] = h;
        w.Ahat[j + (size_t)i * m] = h;
      }
    }
    __syncthreads();
    // split test: S[i][j] = sum_{i' >= i} |A^_i'j|, e(k) = max_{j < k} S[k][j] / ||A||_1
    for (int col = tid; col < m; col += FT) {
      double run = 0.0;
      for (int i = m - 1; i >= 0; --i) {
        run += fabs(w.Ahat[i + (size_t)col * m]);
        w.Ssuf[i + (size_t)col * m] = run;
      }
    }
    __syncthreads();
    for (int k = 1 + tid; k < m; k += FT) {
      double f = 0.0;
      for (int j = 0; j < k; ++j) f = fmax(f, w.Ssuf[k + (size_t)j * m]);
      w.scores[k - 1] = f * inv_norm;
    }
    __syncthreads();
    if (tid == 0) {
      // smallest e(k); exact ties: closest to m/2, then the smaller k
      int best = -1;
      for (int k = 1; k < m; ++k) {
        if (best < 0) { best = k; continue; }
        const double v = w.scores[k - 1], bv = w.scores[best - 1];
        const int d = abs(2 * k - m), bd = abs(2 * best - m);
        if (v < bv || (v == bv && (d < bd || (d == bd && k < best)))) best = k;
      }
      S.c.iscal[0] = best;
      S.c.dscal[0] = best > 0 ? w.scores[best - 1] : 0.0;
    }
    __syncthreads();
    out.k = S.c.iscal[0];
    out.e = S.c.dscal[0];
    out.rank = rank;
    out.draw = draw;
    out.accepted = out.k > 0 && out.k < m && out.e <= stol;
    __syncthreads();
    if (out.accepted || rank == 0 || rank == m) break;
  }
  return out;
}

__device__ void solve_problem(const FusedProblem& pr, const FParams& p, Ws& w, FusedSmem& S,
                              FusedResult& res) {
  const int n = pr.n, lda = pr.lda, ldu = pr.ldu;
  double* A = pr.A;
  double* wout = pr.w;
  double* U = pr.U;
  const int tid = threadIdx.x;
  const int nb = p.nb;
  res = FusedResult{};
  if (n <= 0) return;
  // non-finite input
  double bad = 0.0;
  for (int idx = tid; idx < n * n; idx += FT) {
    const double x = A[(idx % n) + (size_t)(idx / n) * lda];
    if (!isfinite(x)) bad = 1.0;
  }
  if (cta_max(bad, S.c) > 0.0) {
    res.status = EIG_NONFINITE;
    return;
  }
  cta_identity(n, n, 0, U, ldu);
  const int leaf = max(1, min(JL_MAX, p.leaf));
  double lo0 = pr.lo, hi0 = pr.hi;
  if (!pr.has_interval) {
    // root interval: Gershgorin
    double glo = INFINITY, ghi = -INFINITY;
    for (int i = tid; i < n; i += FT) {
      double r = 0.0;
      for (int j = 0; j < n; ++j)
        if (j != i) r += fabs(A[i + (size_t)j * lda]);
      const double a = A[i + (size_t)i * lda];
      glo = fmin(glo, a - r);
      ghi = fmax(ghi, a + r);
    }
    lo0 = -cta_max(-glo, S.c);
    hi0 = cta_max(ghi, S.c);
    if (n > leaf) {
      // tighter root interval: [c - rho, c + rho] cut to Gershgorin, c = tr(A)/n,
      // rho = 1.1 x the power-iteration estimate of ||A - cI||_2 (as eig_solve)
      double tr = 0.0;
      for (int i = tid; i < n; i += FT) tr += A[i + (size_t)i * lda];
      const double c = cta_sum(tr, S.c) / n;
      double* x = w.wv;
      double* y = w.scores;
      cta_gaussian(n, 1, p.seed, PURPOSE_POWER, ROOT, 0, y, n);
      double ss = 0.0;
      for (int i = tid; i < n; i += FT) ss = fma(y[i], y[i], ss);
      double est = sqrt(cta_sum(ss, S.c));
      for (int i = tid; i < n; i += FT) x[i] = est > 0.0 ? y[i] / est : 0.0;
      __syncthreads();
      for (int it = 0; it < POWER_STEPS; ++it) {
        cta_gemm(false, false, n, 1, n, 1.0, A, lda, x, n, 0.0, y, n, S.u.la.g);
        ss = 0.0;
        for (int i = tid; i < n; i += FT) {
          const double v = y[i] - c * x[i];
          ss = fma(v, v, ss);
        }
        est = sqrt(cta_sum(ss, S.c));
        for (int i = tid; i < n; i += FT) {
          const double v = y[i] - c * x[i];
          x[i] = est > 0.0 ? v / est : 0.0;
        }
        __syncthreads();
      }
      const double rho = 1.1 * est;
      const double lo1 = fmax(lo0, c - rho), hi1 = fmin(hi0, c + rho);
      if (lo1 < hi1) {
        lo0 = lo1;
        hi0 = hi1;
      }
    }
  }
  int nstack = 0, nleaves = 0;
  if (tid == 0)
    w.stack[0] = pr.has_interval ? FNode{0, n, pr.depth, 0, lo0, hi0, pr.id}
                                 : FNode{0, n, 0, 0, lo0, hi0, ROOT};
  nstack = 1;
  __syncthreads();
  while (nstack > 0) {
    FNode nd = w.stack[nstack - 1];
    __syncthreads();
    --nstack;
    const int m = nd.m;
    double* An = A + nd.off + (size_t)nd.off * lda;
    res.nodes++;
    res.max_depth = max(res.max_depth, nd.depth);
    if (m <= leaf) {
      if (tid == 0) w.leaves[nleaves] = FLeaf{nd.off, m};
      ++nleaves;
      __syncthreads();
      continue;
    }
    int attempt = 0, fails = 0;
    bool split = false;
    const double tau = p.tau > 0.0 ? p.tau : fmax(1e-14, 4.0 * sqrt((double)m) * UR);
    while (true) {
      // shift: median of the diagonal + 1% jitter, later uniform in the middle half
      for (int i = tid; i < m; i += FT) {
        S.c.sortv[i] = An[i + (size_t)i * lda];
        S.c.sorti[i] = i;
      }
      __syncthreads();
      cta_sort(m, S.c);
      const double med = (m & 1) ? S.c.sortv[m / 2] : (S.c.sortv[m / 2 - 1] + S.c.sortv[m / 2]) / 2.0;
      const double c = 0.5 * (nd.lo + nd.hi);
      double R = 0.5 * (nd.hi - nd.lo);
      if (R <= 0.0) R = fmax(fabs(c), 1.0) * 1e-3;
      const double xi = fphilox_uniform(p.seed, PURPOSE_SHIFT, nd.id, attempt);
      double sigma = (attempt == 0) ? med + 0.01 * R * (2.0 * xi - 1.0) : c + R * (xi - 0.5);
      sigma = fmin(fmax(sigma, nd.lo + 1e-3 * R), nd.hi - 1e-3 * R);
      __syncthreads();
      const IrsRes ir = cta_irs(m, An, lda, sigma, R, tau, p.maxit, nb, w, S);
      res.total_iters += ir.iters;
      res.flops += ir.iters * (22.0 / 3.0) * (double)m * m * m;
      const double* Ap = ir.a_in_j ? w.Aj : w.An;
      const double* Bp = ir.a_in_j ? w.Bj : w.Bn;
      SplitRes so{0, 0, 0, INFINITY, false};
      if (ir.converged) {
        so = cta_split(m, Ap, Bp, An, lda, nd.id, attempt, p, w, S);
        res.flops += (so.draw + 1) * 16.0 * (double)m * m * m;
      }
      if (so.accepted) {
        const int k = so.k;
        // U[:, off:off+m] <- U[:, off:off+m] Q ; node block <- A^
        cta_gemm(false, false, n, m, m, 1.0, U + (size_t)nd.off * ldu, ldu, w.Ucur, m, 0.0,
                 w.Unode, n, S.u.la.g);
        cta_copy(n, m, w.Unode, n, U + (size_t)nd.off * ldu, ldu);
        res.flops += 2.0 * n * (double)m * m;
        cta_copy(m, m, w.Ahat, m, An, lda);
        if (tid == 0) {
          w.stack[nstack] = FNode{nd.off + k, m - k, nd.depth + 1, 0, nd.lo, sigma, fchild(nd.id, 1)};
          w.stack[nstack + 1] = FNode{nd.off, k, nd.depth + 1, 0, sigma, nd.hi, fchild(nd.id, 0)};
        }
        nstack += 2;
        res.splits++;
        __syncthreads();
        split = true;
        break;
      }
      res.failed_attempts++;
      if (ir.converged) {
        if (so.rank == 0) nd.hi = sigma;
        else if (so.rank == m) nd.lo = sigma;
        else fails++;
      } else {
        fails++;
      }
      attempt++;
      if (fails > p.max_fail || attempt > 250) break;
    }
    if (!split) {
      res.status = EIG_NO_SPLIT;
      return;
    }
  }
  // leaves: Jacobi, eigenvector update
  res.leaves = nleaves;
  for (int l = 0; l < nleaves; ++l) {
    const FLeaf lf = w.leaves[l];
    __syncthreads();
    const bool ok = jacobi_leaf(lf.m, A + lf.off + (size_t)lf.off * lda, lda, w.wv + lf.off,
                                w.zleaf, JL_MAX, S.u.jac);
    if (!ok) res.status = EIG_NO_CONVERGENCE;
    cta_gemm(false, false, n, lf.m, lf.m, 1.0, U + (size_t)lf.off * ldu, ldu, w.zleaf, JL_MAX,
             0.0, w.Unode, n, S.u.la.g);
    cta_copy(n, lf.m, w.Unode, n, U + (size_t)lf.off * ldu, ldu);
  }
  // eigenvalues ascending with their vectors
  for (int i = tid; i < n; i += FT) {
    S.c.sortv[i] = w.wv[i];
    S.c.sorti[i] = i;
  }
  __syncthreads();
  cta_sort(n, S.c);
  for (int i = tid; i < n; i += FT) wout[i] = S.c.sortv[i];
  for (int idx = tid; idx < n * n; idx += FT) {
    const int i = idx % n, j = idx / n;
    w.Unode[idx] = U[i + (size_t)S.c.sorti[j] * ldu];
  }
  __syncthreads();
  cta_copy(n, n, w.Unode, n, U, ldu);
}

__global__ void __launch_bounds__(FT, 2)
fused_batched_kernel(int count, const FusedProblem* __restrict__ probs,
                     const int* __restrict__ order, FusedResult* __restrict__ results,
                     int* __restrict__ counter, FParams p, double* ws, size_t ws_stride, int mx) {
  extern __shared__ __align__(16) unsigned char fsm_raw[];
  FusedSmem& S = *reinterpret_cast<FusedSmem*>(fsm_raw);
  Ws w;
  carve(ws + (size_t)blockIdx.x * ws_stride, mx, &w);
  while (true) {
    if (threadIdx.x == 0) S.c.iscal[7] = atomicAdd(counter, 1);
    __syncthreads();
    const int q = S.c.iscal[7];
    __syncthreads();
    if (q >= count) break;
    const int i = order[q];
    const FusedProblem pr = probs[i];
    FusedResult r;
    solve_problem(pr, p, w, S, r);
    if (threadIdx.x == 0) results[i] = r;
    __syncthreads();
  }
}

}  // namespace

size_t fused_workspace_bytes(int mx, int ctas) {
  return carve(nullptr, std::max(mx, 1), nullptr) * sizeof(double) * (size_t)std::max(ctas, 1) + 256;
}

size_t fused_smem_bytes() { return sizeof(FusedSmem); }

int fused_max_ctas_per_sm() {
  static const int v = [] {
    cudaFuncSetAttribute(fused_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(FusedSmem));
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fused_batched_kernel, FT,
                                                      sizeof(FusedSmem)) != cudaSuccess) {
      cudaGetLastError();
      b = 1;
    }
    return std::max(b, 1);
  }();
  return v;
}

int fused_max_n() { return FMAX; }

// Launch of the fused batched solver: probs / results / order / counter are
// device arrays (count entries; counter zeroed here), ws holds
// fused_workspace_bytes(max n, ctas).
cudaError_t fused_batched(cudaStream_t s, int count, const FusedProblem* probs, const int* order,
                          FusedResult* results, int* counter, const eig_params_t& p, int nb,
                          int ctas, int mx, void* ws) {
  if (count <= 0) return cudaSuccess;
  FParams fp;
  fp.tau = p.tau;
  fp.split_tol = p.split_tol;
  fp.seed = p.seed;
  fp.maxit = p.maxit;
  fp.leaf = p.leaf_size;
  fp.max_fail = p.max_fail;
  fp.v_draws = p.v_draws;
  fp.nb = (nb == 16) ? 16 : 32;
  const size_t smem = sizeof(FusedSmem);
  static const cudaError_t attr = cudaFuncSetAttribute(
      fused_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (attr != cudaSuccess) return attr;
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  const size_t stride = carve(nullptr, std::max(mx, 1), nullptr);
  note_launches(1);
  const TimingToken tt = timing_begin(s, TIMING_FUSED, 0.0);
  fused_batched_kernel<<<std::max(1, std::min(ctas, count)), FT, smem, s>>>(
      count, probs, order, results, counter, fp, static_cast<double*>(ws), stride, mx);
  timing_end(s, tt);
  return cudaGetLastError();
}

}  // namespace eigdc
