// FP64 dense building blocks of the inverse-free iteration on sm_103a:
//   * a register-tiled FP64 GEMM with deterministic split-K,
//   * the Householder panel factorisation held in the distributed shared
//     memory of a thread-block cluster (column reductions through DSMEM and
//     hardware cluster barriers; the panel never leaves on-chip memory while
//     it is factorised),
//   * the small "sum split-K partials, multiply by T / T^T" step of the
//     compact-WY block reflector I - V T V^T.
// The reflector convention maps x to +||x|| e1 (R with non-negative diagonal,
// Golub-Van Loan Sec. 5.1), so R_j of the stacked matrix is unique (it is the
// Cholesky factor of A_j^T A_j + B_j^T B_j) and can be compared elementwise.
#include <algorithm>
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <vector>
#include <stdint.h>

#include "internal.h"

namespace cg = cooperative_groups;

namespace eigdc {

// ------------------------------------------------------------------ GEMM
// BM x BN output tile (64 x 64, or 32 x 128 for the M <= 32 products V^T C of
// the compact-WY updates), K step 16, 256 threads, 4x4 outputs per thread.
// FP64 on GB300 is issue-bound on the DFMA pipe (the data moved per tile is a
// few GB/s per SM), so the tile only has to keep that pipe fed and waste no
// FMAs on padding; double-buffered shared memory with a register prefetch of
// the next K step does that.
constexpr int GBK = 16, GTHREADS = 256;

template <bool TA, bool TB, int BM, int BN>
__global__ void __launch_bounds__(GTHREADS)
dgemm_kernel(int M, int N, int K, double alpha, const double* __restrict__ A, int lda,
             const double* __restrict__ B, int ldb, double beta, double* __restrict__ C,
             int ldc, int kchunk, double* __restrict__ partial) {
  constexpr int TXD = BM / 4;              // threads along M
  constexpr int TYD = GTHREADS / TXD;      // threads along N
  static_assert(TYD * 4 == BN, "tile shape");
  constexpr int NA = BM * GBK / GTHREADS;  // A elements per thread per K step
  constexpr int NB = BN * GBK / GTHREADS;
  __shared__ double As[2][GBK][BM + 1];
  __shared__ double Bs[2][GBK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % TXD, ty = tid / TXD;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  double ra[NA], rb[NB];

  auto a_index = [&](int r, int& m, int& k) {
    const int idx = tid + GTHREADS * r;
    if (!TA) { m = idx % BM; k = idx / BM; }
    else { k = idx % GBK; m = idx / GBK; }
  };
  auto b_index = [&](int r, int& n, int& k) {
    const int idx = tid + GTHREADS * r;
    if (!TB) { k = idx % GBK; n = idx / GBK; }
    else { n = idx % BN; k = idx / BN; }
  };
  auto loadA = [&](int k0) {
#pragma unroll
    for (int r = 0; r < NA; ++r) {
      int m, k;
      a_index(r, m, k);
      const int gm = m0 + m, gk = k0 + k;
      double v = 0.0;
      if (gm < M && gk < kend) v = TA ? A[gk + (size_t)gm * lda] : A[gm + (size_t)gk * lda];
      ra[r] = v;
    }
  };
  auto storeA = [&](int buf) {
#pragma unroll
    for (int r = 0; r < NA; ++r) {
      int m, k;
      a_index(r, m, k);
      As[buf][k][m] = ra[r];
    }
  };
  auto loadB = [&](int k0) {
#pragma unroll
    for (int r = 0; r < NB; ++r) {
      int n, k;
      b_index(r, n, k);
      const int gn = n0 + n, gk = k0 + k;
      double v = 0.0;
      if (gn < N && gk < kend) v = TB ? B[gn + (size_t)gk * ldb] : B[gk + (size_t)gn * ldb];
      rb[r] = v;
    }
  };
  auto storeB = [&](int buf) {
#pragma unroll
    for (int r = 0; r < NB; ++r) {
      int n, k;
      b_index(r, n, k);
      Bs[buf][k][n] = rb[r];
    }
  };

  int buf = 0;
  if (kbeg < kend) {
    loadA(kbeg);
    loadB(kbeg);
    storeA(0);
    storeB(0);
  }
  __syncthreads();
  for (int k0 = kbeg; k0 < kend; k0 += GBK) {
    const bool has_next = k0 + GBK < kend;
    if (has_next) {
      loadA(k0 + GBK);
      loadB(k0 + GBK);
    }
#pragma unroll
    for (int kk = 0; kk < GBK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[buf][kk][tx + TXD * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[buf][kk][ty + TYD * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    if (has_next) {
      storeA(buf ^ 1);
      storeB(buf ^ 1);
    }
    __syncthreads();
    buf ^= 1;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + tx + TXD * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + ty + TYD * j;
      if (gn >= N) continue;
      if (partial) {
        partial[(size_t)blockIdx.z * M * N + gm + (size_t)gn * M] = alpha * acc[i][j];
      } else {
        double v = alpha * acc[i][j];
        if (beta != 0.0) v = fma(beta, C[gm + (size_t)gn * ldc], v);
        C[gm + (size_t)gn * ldc] = v;
      }
    }
  }
}

__global__ void splitk_reduce_kernel(int M, int N, int splits, const double* __restrict__ partial,
                                     double beta, double* __restrict__ C, int ldc) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t total = (size_t)M * N;
  if (idx >= total) return;
  const int i = (int)(idx % M), j = (int)(idx / M);
  double s = 0.0;
  for (int z = 0; z < splits; ++z) s += partial[(size_t)z * total + idx];
  if (beta != 0.0) s = fma(beta, C[i + (size_t)j * ldc], s);
  C[i + (size_t)j * ldc] = s;
}

static inline bool narrow_tile(int m) { return m <= 32; }

// K-chunk count: aim at whole waves of 2 CTAs per SM on the 152 SMs (the 4x4
// register tile allows two resident CTAs), each chunk at least 128 of K.
int gemm_choose_splits(int m, int n, int k) {
  const int bm = narrow_tile(m) ? 32 : 64, bn = narrow_tile(m) ? 128 : 64;
  const int tiles = ((m + bm - 1) / bm) * ((n + bn - 1) / bn);
  const int wave = 2 * 152;
  if (tiles >= wave) return 1;
  const int maxk = std::max(1, std::min(32, k / 128));
  int best = 1;
  double best_eff = 0.0;
  for (int s = 1; s <= maxk; ++s) {
    const long ctas = (long)tiles * s;
    const long waves = (ctas + wave - 1) / wave;
    // useful fraction of the issued waves, lightly favouring fewer chunks
    const double eff = (double)ctas / (double)(waves * wave) - 0.002 * s;
    if (eff > best_eff) {
      best_eff = eff;
      best = s;
    }
  }
  return best;
}

// ------------------------------------------------------------ launch timing
// Opt-in CUDA-event timing of every launch of the timed kernel families
// (dgemm_kernel, the two tensor-core splits, the fused batched solver), for
// the roofline of the dominant kernel measured inside a timed region.  Off by
// default; when on, each launch records one event before and one after it on
// its stream.  Launches being captured into a CUDA graph are not timed (their
// events would become graph nodes): the timed set is the eager launches.
namespace {
struct TimedLaunch {
  cudaEvent_t a, b;
  double work;
  int family;
};
std::mutex g_tmu;
std::atomic<bool> g_timing{false};
std::vector<TimedLaunch> g_timed;
std::vector<cudaEvent_t> g_event_pool;
double g_fam_ms[TIMING_FAMILIES], g_fam_work[TIMING_FAMILIES];
unsigned long long g_fam_count[TIMING_FAMILIES];

cudaEvent_t take_event() {   // g_tmu held
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}
}  // namespace

TimingToken timing_begin(cudaStream_t s, int family, double work) {
  TimingToken t{nullptr, nullptr, work, family};
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (g_timing.load(std::memory_order_relaxed) &&
      cudaStreamIsCapturing(s, &cap) == cudaSuccess && cap == cudaStreamCaptureStatusNone) {
    std::lock_guard<std::mutex> lock(g_tmu);
    t.a = take_event();
    t.b = take_event();
    if (t.a) cudaEventRecord(t.a, s);
  }
  return t;
}

void timing_end(cudaStream_t s, const TimingToken& t) {
  if (!t.a || !t.b) return;
  cudaEventRecord(t.b, s);
  std::lock_guard<std::mutex> lock(g_tmu);
  g_timed.push_back(TimedLaunch{t.a, t.b, t.work, t.family});
}

void gemm_timing_start() {
  std::lock_guard<std::mutex> lock(g_tmu);
  for (TimedLaunch& t : g_timed) {
    g_event_pool.push_back(t.a);
    g_event_pool.push_back(t.b);
  }
  g_timed.clear();
  g_timing.store(true);
}

cudaError_t gemm_timing_stop(double* total_ms, unsigned long long* launches, double* flops) {
  g_timing.store(false);
  std::lock_guard<std::mutex> lock(g_tmu);
  for (int f = 0; f < TIMING_FAMILIES; ++f) {
    g_fam_ms[f] = 0.0;
    g_fam_work[f] = 0.0;
    g_fam_count[f] = 0;
  }
  for (TimedLaunch& t : g_timed) {
    cudaError_t e = cudaEventSynchronize(t.b);
    if (e != cudaSuccess) return e;
    float x = 0.0f;
    e = cudaEventElapsedTime(&x, t.a, t.b);
    if (e != cudaSuccess) return e;
    g_fam_ms[t.family] += x;
    g_fam_work[t.family] += t.work;
    g_fam_count[t.family] += 1;
  }
  if (total_ms) *total_ms = g_fam_ms[0];
  if (launches) *launches = g_fam_count[0];
  if (flops) *flops = g_fam_work[0];
  return cudaSuccess;
}

void timing_family(int family, double* total_ms, unsigned long long* launches, double* work) {
  std::lock_guard<std::mutex> lock(g_tmu);
  const bool ok = family >= 0 && family < TIMING_FAMILIES;
  if (total_ms) *total_ms = ok ? g_fam_ms[family] : 0.0;
  if (launches) *launches = ok ? g_fam_count[family] : 0;
  if (work) *work = ok ? g_fam_work[family] : 0.0;
}

template <bool TA, bool TB>
static void launch_dgemm(cudaStream_t s, int m, int n, int k, int splits, int kchunk, double alpha,
                         const double* A, int lda, const double* B, int ldb, double beta,
                         double* C, int ldc, double* part) {
  note_launches(1);
  const TimingToken tl = timing_begin(s, TIMING_DGEMM, 2.0 * m * (double)n * k);
  if (narrow_tile(m)) {
    dim3 grid((m + 31) / 32, (n + 127) / 128, splits);
    dgemm_kernel<TA, TB, 32, 128><<<grid, GTHREADS, 0, s>>>(m, n, k, alpha, A, lda, B, ldb, beta,
                                                             C, ldc, kchunk, part);
  } else {
    dim3 grid((m + 63) / 64, (n + 63) / 64, splits);
    dgemm_kernel<TA, TB, 64, 64><<<grid, GTHREADS, 0, s>>>(m, n, k, alpha, A, lda, B, ldb, beta,
                                                           C, ldc, kchunk, part);
  }
  timing_end(s, tl);
}

static int effective_splits(int k, int splits, int& kchunk) {
  if (splits < 1) splits = 1;
  kchunk = (k + splits - 1) / splits;
  kchunk = ((kchunk + GBK - 1) / GBK) * GBK;
  if (kchunk < GBK) kchunk = GBK;
  return k > 0 ? (k + kchunk - 1) / kchunk : 1;
}

cudaError_t gemm(cudaStream_t s, bool ta, bool tb, int m, int n, int k, double alpha,
                 const double* A, int lda, const double* B, int ldb, double beta, double* C,
                 int ldc, int splits, double* partial) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  if (splits < 1 || partial == nullptr) splits = 1;
  int kchunk;
  splits = effective_splits(k, splits, kchunk);
  double* part = splits > 1 ? partial : nullptr;
  if (!ta && !tb) launch_dgemm<false, false>(s, m, n, k, splits, kchunk, alpha, A, lda, B, ldb, beta, C, ldc, part);
  else if (ta && !tb) launch_dgemm<true, false>(s, m, n, k, splits, kchunk, alpha, A, lda, B, ldb, beta, C, ldc, part);
  else if (!ta && tb) launch_dgemm<false, true>(s, m, n, k, splits, kchunk, alpha, A, lda, B, ldb, beta, C, ldc, part);
  else launch_dgemm<true, true>(s, m, n, k, splits, kchunk, alpha, A, lda, B, ldb, beta, C, ldc, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || splits == 1) return e;
  const size_t total = (size_t)m * n;
  note_launches(1);
  splitk_reduce_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(m, n, splits, partial, beta, C, ldc);
  return cudaGetLastError();
}

int gemm_partials(cudaStream_t s, bool ta, int m, int n, int k, const double* A, int lda,
                  const double* B, int ldb, int splits, double* partial) {
  if (m <= 0 || n <= 0) return 0;
  int kchunk;
  splits = effective_splits(k, splits, kchunk);
  if (ta) launch_dgemm<true, false>(s, m, n, k, splits, kchunk, 1.0, A, lda, B, ldb, 0.0, nullptr, m, partial);
  else launch_dgemm<false, false>(s, m, n, k, splits, kchunk, 1.0, A, lda, B, ldb, 0.0, nullptr, m, partial);
  if (cudaGetLastError() != cudaSuccess) return -1;
  return splits;
}

// ------------------------------------------------------------ panel QR
// One cluster of CS CTAs factorises an m x jb panel.  CTA q holds rows
// [q*rs, q*rs + rs) of the panel in shared memory (column-major slab with a
// padded leading dimension).  For every column c:
//   A: each CTA forms its partial sum of squares below the pivot and, if it
//      owns row c, the pivot value; cluster barrier;
//   B: every CTA reads the CS partials through DSMEM in rank order (so all
//      CTAs hold bit-identical scalars), forms the reflector (v_c = 1,
//      P x = +||x|| e1), scales its part of v, and computes its partial dot
//      products d_k = sum_r w_r P[r,k] for all k != c (k > c: the columns to
//      update; k < c: the entries V^T v that extend T); cluster barrier;
//   C: every CTA sums the CS partial dot vectors in rank order and updates
//      its rows; rank 0 extends T.
// Two cluster barriers per column; the partial buffers alternate by column
// parity so a fast CTA never overwrites values a slow one still reads.
constexpr int PQ_THREADS = 256;
constexpr int PQ_MAXJB = 32;
constexpr int PQ_GROUPS = PQ_THREADS / 32;
constexpr size_t PQ_SMEM_LIMIT = 220 * 1024;

struct PanelScratch {
  double red[2][2][PQ_MAXJB];   // [parity][0: partial dots P'_k, 1: pivot row a_k(c)][k]
  double comb[2][PQ_MAXJB];     // cluster sums of red[par]
  double grp[PQ_GROUPS][PQ_MAXJB + 1];
  double dk[PQ_MAXJB];
  double bc[4];
  double taus[PQ_MAXJB];
  double Tsm[PQ_MAXJB][PQ_MAXJB + 1];
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(PQ_THREADS)
panel_qr_kernel(int m, int jb, double* __restrict__ P, int ldp, double* __restrict__ V, int ldv,
                double* __restrict__ tau, double* __restrict__ T, int ldt, int rs, int rs_pad) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PanelScratch* sc = reinterpret_cast<PanelScratch*>(smem_raw);
  double* slab = reinterpret_cast<double*>(smem_raw + sizeof(PanelScratch));

  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int CS = (int)cluster.num_blocks();
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int r0 = rank * rs;
  const int rcount = max(0, min(rs, m - r0));

  for (int idx = tid; idx < rcount * jb; idx += PQ_THREADS) {
    const int r = idx % rcount, c = idx / rcount;
    slab[c * rs_pad + r] = P[(size_t)(r0 + r) + (size_t)c * ldp];
  }
  if (rank == 0) {
    for (int idx = tid; idx < PQ_MAXJB * (PQ_MAXJB + 1); idx += PQ_THREADS)
      (&sc->Tsm[0][0])[idx] = 0.0;
  }
  __syncthreads();
  cluster.sync();   // every CTA of the cluster is resident before any DSMEM access

  // One cluster reduction per column.  With x the column below and at the
  // pivot, v_c = 1 and v_r = x_r / v0 (r > c), every needed product follows
  // from the unnormalised partials P'_k = sum_{r > c} x_r a_k(r) (k = c gives
  // sigma = sum_{r > c} x_r^2) and the pivot row a_k(c):
  //   v^T a_k = a_k(c) + P'_k / v0   (update of column k > c; for k < c the
  //   same expression with the stored reflector v_k gives v^T v_k for T).
  for (int c = 0; c < jb; ++c) {
    const int par = c & 1;
    double* colc = slab + c * rs_pad;
    // ---- partials of this CTA's rows: thread (k = lane, g = warp)
    {
      const int k = lane, g = warp;
      double d = 0.0;
      if (k < jb) {
        const double* colk = slab + k * rs_pad;
        for (int r = g; r < rcount; r += PQ_GROUPS) {
          if (r0 + r > c) d = fma(colc[r], colk[r], d);
        }
      }
      sc->grp[g][k] = d;
    }
    __syncthreads();
    if (tid < PQ_MAXJB) {
      double t = 0.0;
      for (int g = 0; g < PQ_GROUPS; ++g) t += sc->grp[g][tid];
      sc->red[par][0][tid] = t;
      const bool own = (c >= r0 && c < r0 + rcount);
      sc->red[par][1][tid] = (own && tid < jb) ? slab[tid * rs_pad + (c - r0)] : 0.0;
    }
    cluster.sync();
    // ---- cluster sums in rank order (bit-identical in every CTA)
    if (tid < 2 * PQ_MAXJB) {
      const int w = tid / PQ_MAXJB, k = tid % PQ_MAXJB;
      double t = 0.0;
      for (int q = 0; q < CS; ++q) {
        const double* rq = cluster.map_shared_rank(&sc->red[0][0][0], q);
        t += rq[(par * 2 + w) * PQ_MAXJB + k];
      }
      sc->comb[w][k] = t;
    }
    __syncthreads();
    if (tid == 0) {
      const double sigma = sc->comb[0][c];
      const double x0 = sc->comb[1][c];
      double beta, mu, v0;
      if (sigma == 0.0) {
        v0 = 0.0;                          // v = e1 (nothing below the pivot)
        if (x0 >= 0.0) { beta = 0.0; mu = x0; }
        else { beta = 2.0; mu = -x0; }
      } else {
        mu = sqrt(x0 * x0 + sigma);
        v0 = (x0 <= 0.0) ? (x0 - mu) : (-sigma / (x0 + mu));
        beta = 2.0 * v0 * v0 / (sigma + v0 * v0);
      }
      sc->bc[0] = beta;
      sc->bc[1] = mu;
      sc->bc[2] = v0;
      sc->taus[c] = beta;
    }
    __syncthreads();
    const double beta = sc->bc[0];
    const double mu = sc->bc[1];
    const double v0 = sc->bc[2];
    if (tid < jb) {
      const double pk = sc->comb[0][tid];
      sc->dk[tid] = sc->comb[1][tid] + ((v0 != 0.0) ? pk / v0 : 0.0);
    }
    for (int r = tid; r < rcount; r += PQ_THREADS) {
      if (r0 + r > c) colc[r] = (v0 != 0.0) ? colc[r] / v0 : 0.0;
    }
    __syncthreads();
    if (beta != 0.0) {
      for (int kk = c + 1; kk < jb; ++kk) {
        const double bd = beta * sc->dk[kk];
        double* colk = slab + kk * rs_pad;
        for (int r = tid; r < rcount; r += PQ_THREADS) {
          const int gr = r0 + r;
          if (gr >= c) {
            const double w = (gr == c) ? 1.0 : colc[r];
            colk[r] -= bd * w;
          }
        }
      }
    }
    if (rank == 0) {
      if (tid < c) {
        double t = 0.0;
        for (int l = tid; l < c; ++l) t = fma(sc->Tsm[tid][l], sc->dk[l], t);
        sc->Tsm[tid][c] = -beta * t;
      }
      if (tid == 0) sc->Tsm[c][c] = beta;
    }
    if (c >= r0 && c < r0 + rcount && tid == 0) colc[c - r0] = mu;
    __syncthreads();
  }
  cluster.sync();   // no CTA leaves while another may still read its partials

  for (int idx = tid; idx < rcount * jb; idx += PQ_THREADS) {
    const int r = idx % rcount, c = idx / rcount;
    const int gr = r0 + r;
    const double x = slab[c * rs_pad + r];
    P[(size_t)gr + (size_t)c * ldp] = x;
    V[(size_t)gr + (size_t)c * ldv] = (gr < c) ? 0.0 : ((gr == c) ? 1.0 : x);
  }
  if (rank == 0) {
    if (tid < jb) tau[tid] = sc->taus[tid];
    for (int idx = tid; idx < jb * jb; idx += PQ_THREADS) {
      const int i = idx % jb, j = idx / jb;
      T[i + (size_t)j * ldt] = (i <= j) ? sc->Tsm[i][j] : 0.0;
    }
  }
}

static int g_max_cluster = 8;

// Largest cluster the panel kernel can use on this device: 16 CTAs (a
// non-portable size, opted in) when the occupancy query confirms it, else 8.
void panel_init() {
  cudaFuncSetAttribute(panel_qr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)PQ_SMEM_LIMIT + 1024);
  cudaFuncSetAttribute(panel_qr_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(16, 1, 1);
  cfg.blockDim = dim3(PQ_THREADS, 1, 1);
  cfg.dynamicSmemBytes = PQ_SMEM_LIMIT;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 16;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  cudaError_t e = cudaOccupancyMaxActiveClusters(&nclusters, panel_qr_kernel, &cfg);
  g_max_cluster = (e == cudaSuccess && nclusters > 0) ? 16 : 8;
  cudaGetLastError();
}

static void panel_geometry(int m, int& cs, int& rs, int& rs_pad) {
  cs = (m + 127) / 128;
  if (cs > g_max_cluster) cs = g_max_cluster;
  if (cs < 1) cs = 1;
  rs = (m + cs - 1) / cs;
  rs = ((rs + 7) / 8) * 8;
  rs_pad = rs + 1;
}

int panel_max_width(int m) {
  int cs, rs, rs_pad;
  panel_geometry(m, cs, rs, rs_pad);
  const size_t avail = PQ_SMEM_LIMIT - sizeof(PanelScratch);
  int jb = PQ_MAXJB;
  while (jb > 8 && (size_t)jb * rs_pad * sizeof(double) > avail) jb /= 2;
  if ((size_t)jb * rs_pad * sizeof(double) > avail) return 0;
  return jb;
}

cudaError_t panel_qr(cudaStream_t s, int m, int jb, double* P, int ldp, double* V, int ldv,
                     double* tau, double* T, int ldt) {
  int cs, rs, rs_pad;
  panel_geometry(m, cs, rs, rs_pad);
  const size_t smem = sizeof(PanelScratch) + (size_t)jb * rs_pad * sizeof(double);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs, 1, 1);
  cfg.blockDim = dim3(PQ_THREADS, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  note_launches(1);
  return cudaLaunchKernelEx(&cfg, panel_qr_kernel, m, jb, P, ldp, V, ldv, tau, T, ldt, rs, rs_pad);
}

// ------------------------------------------------------- reduce + T multiply
// out(i, col) = sum_l op(T)(i, l) * (sum_z partial[z](l, col)); op(T) = T^T
// (lower) for Q^T C, T (upper) for Q C.  Eight columns per CTA.
__global__ void __launch_bounds__(256)
reduce_trmm_kernel(int jb, int n, const double* __restrict__ partial, int splits,
                   const double* __restrict__ T, int ldt, int trans, int in_trans,
                   double* __restrict__ out) {
  __shared__ double Ts[PQ_MAXJB][PQ_MAXJB + 1];
  __shared__ double Ws[PQ_MAXJB][9];
  const int tid = threadIdx.x;
  for (int idx = tid; idx < jb * jb; idx += 256) {
    const int i = idx % jb, j = idx / jb;
    Ts[i][j] = T[i + (size_t)j * ldt];
  }
  const int i = tid & 31, cc = tid >> 5;
  const int col = blockIdx.x * 8 + cc;
  if (i < jb && col < n) {
    double s = 0.0;
    if (in_trans) {
      s = partial[col + (size_t)i * n];       // input stored n x jb (the transpose)
    } else {
      const size_t stride = (size_t)jb * n;
      for (int z = 0; z < splits; ++z) s += partial[(size_t)z * stride + i + (size_t)col * jb];
    }
    Ws[i][cc] = s;
  }
  __syncthreads();
  if (i < jb && col < n) {
    double t = 0.0;
    if (trans) {
      for (int l = 0; l <= i; ++l) t = fma(Ts[l][i], Ws[l][cc], t);
    } else {
      for (int l = i; l < jb; ++l) t = fma(Ts[i][l], Ws[l][cc], t);
    }
    out[i + (size_t)col * jb] = t;
  }
}

cudaError_t reduce_trmm(cudaStream_t s, int jb, int n, const double* partial, int splits,
                        const double* T, int ldt, bool trans, double* out, bool in_trans) {
  if (n <= 0) return cudaSuccess;
  note_launches(1);
  reduce_trmm_kernel<<<(n + 7) / 8, 256, 0, s>>>(jb, n, partial, splits, T, ldt, trans ? 1 : 0,
                                                 in_trans ? 1 : 0, out);
  return cudaGetLastError();
}

}  // namespace eigdc
