// FP64-accurate GEMM on the fifth-generation tensor cores by error-free
// splitting (the scheme of Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012):
//
//   * every row r of op(A) (and every column c of op(B)) is scaled by a power
//     of two 2^e with max |x| < 2^e, and |x| 2^-e is cut into nine signed
//     digits in balanced form: x = sign * 2^(e-5) * sum_p d_p 2^(-6p) with
//     d_0 in [0, 32] and d_p in [-32, 31] below it (53 bits of 2^e, the last
//     digit rounded; a digit of 32 or more borrows one from the digit above).
//     Each digit is an integer, stored exactly as BF16 (one plane per digit);
//   * the product of two rows is 2^(e_r + e_c - 10) sum_l L_l 2^(-6 l) with
//     the level sums L_l = sum_{i+j=l} sum_k d_i(r,k) d_j(c,k).  Levels
//     0..9 are kept (53 digit pairs); the first dropped level weighs about
//     2^-60 K relative to 2^(e_r + e_c), below FP64 rounding of the product;
//   * each level is accumulated by tcgen05.mma (kind::f16, BF16 inputs, FP32
//     accumulator) in its own TMEM columns.  Every partial sum is an integer
//     below 9 * 1792 * 32^2 < 2^24 as long as a chunk spans at most 1792 of K,
//     so the FP32 accumulation is exact; after each chunk four drain warps
//     read the ten accumulators (tcgen05.ld), combine levels 0..4 and 5..9
//     exactly in int64 and add each group, scaled by its power of two, to
//     FP64 registers.  (The balanced digits halve the digit
//     bound, so a chunk is four times longer than with digits in [0, 64]:
//     the drain's FP64 work, on a pipe about 1/1800 of the tensor rate,
//     shrinks fourfold.)
//
// Kernel (one CTA per 128 x 48 tile of C, 192 threads):
//   warp 0: TMA producer -- per 64-wide K tile the nine B digit planes
//           (48 x 64 each, one stage of a 2-stage ring) and, one by one, the
//           nine A digit planes (128 x 64, a 7-slot ring);
//   warp 1: TMEM allocation (512 columns) and the single MMA-issuing thread;
//   warps 2-5: drain and epilogue (warp w reads TMEM lanes 32 (w % 4) + 0..31,
//           i.e. rows of the tile).
// Every mbarrier wait is bounded; on a timeout the CTA records an error flag,
// skips its remaining work and still frees its TMEM.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "internal.h"
#include "tc_ptx.cuh"

namespace eigdc {

bool make_plane_map(CUtensorMap* map, void* base, int rows, int kp, int box_rows, int planes);

constexpr int TX_BM = 128, TX_BN = 48, TX_BK = 64;
constexpr int TX_BSTAGES = 2;
constexpr int TX_THREADS = 192;
constexpr int TX_TILE_A = TX_BM * TX_BK * 2;   // bytes of one digit plane slab of A
constexpr int TX_TILE_B = TX_BN * TX_BK * 2;
static_assert(TX_TILE_A % 1024 == 0 && TX_TILE_B % 1024 == 0, "1024-byte swizzle atoms");

// Digit count DIG and the levels kept:
//   DIG = 9: levels 0..9 (53 digit pairs), FP64 accuracy;
//   DIG = 5: levels 0..4 (15 digit pairs), 30 bits of each row / column
//            maximum (the split-precision form's second tier);
//   DIG = 4: levels 0..3 (10 digit pairs), FP32-level accuracy (24 bits of
//            each row / column maximum), the split-precision form.
// DIG = 9 uses balanced digits (|d| <= 32); the FP32-level tiers keep digits
// in [0, 64] (24 / 30 bits of the maximum rather than 23 / 29).
// CHUNK_TILES: 64-wide K tiles per exact FP32 chunk, so that a level's
// partial sums (pairs per level x chunk x DMAX^2) stay integers below 2^24.
// TOP / SHIFT0: F = floor(|x| 2^(TOP - e)) < 2^TOP and digit p is bits
// SHIFT0 - 6p .. SHIFT0 - 6p + 5 of F; the product of two rows carries
// 2^(e_r + e_c - SCALE).  ASLOTS: slots of the A digit-plane ring.
template <int DIG>
struct TxCfg {
  static constexpr int DIGITS = DIG;
  static constexpr bool BALANCED = (DIG == 9);
  static constexpr int LEVELS = (DIG == 9) ? 10 : DIG;
  static constexpr int MAXPAIRS = (DIG == 9) ? 9 : DIG;   // digit pairs of the fullest level
  static constexpr int DMAX = BALANCED ? 32 : 64;
  static constexpr int TOP = BALANCED ? 60 : 62;
  static constexpr int SHIFT0 = BALANCED ? 55 : 56;
  static constexpr int SCALE = BALANCED ? 10 : 12;
  static constexpr int CHUNK_TILES = (DIG == 9) ? 28 : (DIG == 5 ? 12 : 15);
  static constexpr int ASLOTS = (DIG == 9) ? 7 : 4;
  static constexpr uint32_t TMEM_COLS = (DIG == 9) ? 512 : 256;   // >= LEVELS * TX_BN, power of two
  static_assert(LEVELS * TX_BN <= (int)TMEM_COLS, "levels fit in TMEM");
  static_assert((long long)MAXPAIRS * CHUNK_TILES * TX_BK * DMAX * DMAX < (1LL << 24),
                "exact FP32 chunk");
  static_assert(SHIFT0 - 6 * (DIG - 1) - 1 >= 0 && SHIFT0 + 6 == TOP + (BALANCED ? 1 : 0),
                "digit layout");
};

template <int DIG>
struct TxSmem {
  uint8_t b[TX_BSTAGES][DIG][TX_TILE_B];
  uint8_t a[TxCfg<DIG>::ASLOTS][TX_TILE_A];
  uint64_t bfull[TX_BSTAGES], bempty[TX_BSTAGES];
  uint64_t afull[TxCfg<DIG>::ASLOTS], aempty[TxCfg<DIG>::ASLOTS];
  uint64_t accfull, accempty;
  uint32_t tmem_base;
  int abort_flag;
};

// ------------------------------------------------------------------ slicing
// mx[r] = bits of max_k |X'(r, k)| for the K-major operand X' (rows x K),
// element (r, k) = X[k + r*ldx] (kcontig) or X[r + k*ldx].  mx must be zeroed.
__global__ void __launch_bounds__(256)
rowmax_kernel(int rows, int K, const double* __restrict__ X, int ldx, int kcontig,
              unsigned long long* __restrict__ mx) {
  __shared__ unsigned long long smax[32];
  const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 64;
  const int tid = threadIdx.x;
  if (tid < 32) smax[tid] = 0ull;
  __syncthreads();
  for (int idx = tid; idx < 32 * 64; idx += 256) {
    int rr, kk;
    if (kcontig) { kk = idx % 64; rr = idx / 64; }
    else { rr = idx % 32; kk = idx / 32; }
    const int r = r0 + rr, k = k0 + kk;
    if (r < rows && k < K) {
      const double v = kcontig ? X[k + (size_t)r * ldx] : X[r + (size_t)k * ldx];
      atomicMax(&smax[rr], (unsigned long long)__double_as_longlong(fabs(v)));
    }
  }
  __syncthreads();
  if (tid < 32 && r0 + tid < rows && smax[tid] != 0ull) atomicMax(&mx[r0 + tid], smax[tid]);
}

// Exponent e with every |x| of the row below 2^e (e = E_max - 1022 for the
// biased exponent E_max of the row maximum; -1022 for zero / subnormal rows).
__device__ __forceinline__ int row_exponent(unsigned long long maxbits) {
  const int E = (int)((maxbits >> 52) & 0x7FF);
  return E == 0 ? -1022 : E - 1022;
}

// Digit planes P[p][r*kp + k] (p = 0..DIG-1) and row exponents expo[r].
template <int DIG>
__global__ void __launch_bounds__(256)
slice_kernel(int rows, int K, int kp, const double* __restrict__ X, int ldx, int kcontig,
             const unsigned long long* __restrict__ mx, __nv_bfloat16* __restrict__ P,
             size_t pstride, int* __restrict__ expo) {
  using Cfg = TxCfg<DIG>;
  __shared__ double tile[32][65];
  const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 64;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < 32 * 64; idx += 256) {
    int rr, kk;
    if (kcontig) { kk = idx % 64; rr = idx / 64; }
    else { rr = idx % 32; kk = idx / 32; }
    const int r = r0 + rr, k = k0 + kk;
    double v = 0.0;
    if (r < rows && k < K) v = kcontig ? X[k + (size_t)r * ldx] : X[r + (size_t)k * ldx];
    tile[rr][kk] = v;
  }
  __syncthreads();
  for (int idx = tid; idx < 32 * 64; idx += 256) {
    const int kk = idx % 64, rr = idx / 64;
    const int r = r0 + rr, k = k0 + kk;
    if (r >= rows || k >= kp) continue;
    const int e = row_exponent(mx[r]);
    if (k == 0) expo[r] = e;
    const unsigned long long b = (unsigned long long)__double_as_longlong(tile[rr][kk]);
    const int E = (int)((b >> 52) & 0x7FF);
    const unsigned long long mant = b & ((1ull << 52) - 1);
    const unsigned long long M = E ? (mant | (1ull << 52)) : mant;
    // F = floor(|x| 2^(TOP - e)) = M 2^(Ee - 1075 + TOP - e) < 2^TOP
    const int sh = (E ? E : 1) - 1075 + Cfg::TOP - e;
    unsigned long long F;
    if (sh >= 0) F = M << sh;
    else F = (-sh >= 64) ? 0ull : (M >> (-sh));
    const bool neg = (b >> 63) != 0;
    const size_t o = (size_t)r * kp + k;
    // the bit below the last digit rounds it; in balanced form a digit of 32
    // or more becomes d - 64 and carries one into the digit above
    int carry = (int)((F >> (Cfg::SHIFT0 - 6 * (DIG - 1) - 1)) & 1ull);
#pragma unroll
    for (int p = DIG - 1; p >= 0; --p) {
      int d = (int)((F >> (Cfg::SHIFT0 - 6 * p)) & 63ull) + carry;
      carry = 0;
      if (Cfg::BALANCED && p > 0 && d >= 32) {
        d -= 64;
        carry = 1;
      }
      P[p * pstride + o] = __int2bfloat16_rn(neg ? -d : d);
    }
  }
}

// ------------------------------------------------------------------ GEMM
template <int DIG>
__global__ void __launch_bounds__(TX_THREADS, 1)
tcx_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                int M, int N, int kp, double alpha, double beta, double* __restrict__ C, int ldc,
                const int* __restrict__ expA, const int* __restrict__ expB, int* err) {
  extern __shared__ uint8_t smem_raw[];
  using Cfg = TxCfg<DIG>;
  constexpr int TX_DIGITS = Cfg::DIGITS, TX_LEVELS = Cfg::LEVELS, TX_CHUNK_TILES = Cfg::CHUNK_TILES;
  constexpr int TX_ASLOTS = Cfg::ASLOTS;
  constexpr uint32_t TX_TMEM_COLS = Cfg::TMEM_COLS;
  TxSmem<DIG>& S = *reinterpret_cast<TxSmem<DIG>*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                   ~static_cast<uintptr_t>(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * TX_BM, n0 = blockIdx.y * TX_BN;
  const int nk = kp / TX_BK;
  const int nchunks = (nk + TX_CHUNK_TILES - 1) / TX_CHUNK_TILES;

  if (threadIdx.x == 0) {
    for (int s = 0; s < TX_BSTAGES; ++s) {
      mbar_init(&S.bfull[s], 1);
      mbar_init(&S.bempty[s], 1);
    }
    for (int s = 0; s < TX_ASLOTS; ++s) {
      mbar_init(&S.afull[s], 1);
      mbar_init(&S.aempty[s], 1);
    }
    mbar_init(&S.accfull, 1);
    mbar_init(&S.accempty, 4);
    S.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
  }
  if (warp == 1) tmem_alloc(&S.tmem_base, TX_TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem_base;

  if (warp == 0) {
    if (lane == 0) {
      // ---- TMA producer
      uint32_t u = 0;   // A slab counter over (k tile, digit)
      for (int kt = 0; kt < nk && !S.abort_flag; ++kt) {
        const int sb = kt % TX_BSTAGES;
        if (!mbar_wait(&S.bempty[sb], ((kt / TX_BSTAGES) & 1) ^ 1)) {
          S.abort_flag = 1;
          atomicOr(err, 1);
          break;
        }
        mbar_arrive_expect_tx(&S.bfull[sb], TX_DIGITS * TX_TILE_B);
        for (int p = 0; p < TX_DIGITS; ++p)
          tma_load_3d(S.b[sb][p], &tmB, &S.bfull[sb], kt * TX_BK, n0, p);
        for (int i = 0; i < TX_DIGITS; ++i, ++u) {
          const int sa = u % TX_ASLOTS;
          if (!mbar_wait(&S.aempty[sa], ((u / TX_ASLOTS) & 1) ^ 1)) {
            S.abort_flag = 1;
            atomicOr(err, 1);
            break;
          }
          mbar_arrive_expect_tx(&S.afull[sa], TX_TILE_A);
          tma_load_3d(S.a[sa], &tmA, &S.afull[sa], kt * TX_BK, m0, i);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer: level l = i + j into TMEM columns l * TX_BN
      uint32_t u = 0;
      bool ok = true;
      for (int kt = 0; kt < nk && ok; ++kt) {
        const int chunk = kt / TX_CHUNK_TILES;
        const int first = chunk * TX_CHUNK_TILES;
        const int last = std::min(nk, first + TX_CHUNK_TILES) - 1;
        if (kt == first && chunk > 0) {
          // the drain warps must have read the previous chunk
          if (!mbar_wait(&S.accempty, (chunk - 1) & 1)) {
            S.abort_flag = 1;
            atomicOr(err, 2);
            ok = false;
            break;
          }
          tc_fence_after();
        }
        const int sb = kt % TX_BSTAGES;
        if (!mbar_wait(&S.bfull[sb], (kt / TX_BSTAGES) & 1)) {
          S.abort_flag = 1;
          atomicOr(err, 2);
          ok = false;
          break;
        }
        for (int i = 0; i < TX_DIGITS; ++i, ++u) {
          const int sa = u % TX_ASLOTS;
          if (!mbar_wait(&S.afull[sa], (u / TX_ASLOTS) & 1)) {
            S.abort_flag = 1;
            atomicOr(err, 2);
            ok = false;
            break;
          }
          tc_fence_after();
          // A digit i against B digits j = j0..j1 in one MMA: the B planes
          // lie back to back in shared memory (48 rows each, 1024-byte
          // aligned), so rows 48 (j - j0) .. of an N = 48 (j1 - j0 + 1) operand
          // are digit j, and with the accumulator at TMEM column 48 (i + j0)
          // each digit's product lands in its level's columns 48 (i + j).
          // Runs are cut where the first-write flag changes (the first write
          // of level l in a chunk is the pair i = max(0, l - (DIG - 1))) and
          // at 5 digits (N <= 256).
          const int jmax = std::min(TX_DIGITS - 1, TX_LEVELS - 1 - i);
          for (int j0 = 0; j0 <= jmax;) {
            const bool f0 = (i == 0) || (j0 == TX_DIGITS - 1);
            int j1 = j0;
            while (j1 + 1 <= jmax && j1 + 1 - j0 < 5 &&
                   ((i == 0) || (j1 + 1 == TX_DIGITS - 1)) == f0)
              ++j1;
            const int cnt = j1 - j0 + 1;
            const uint32_t idesc = idesc_bf16_f32(TX_BM, TX_BN * cnt);
#pragma unroll
            for (int kk = 0; kk < TX_BK / 16; ++kk) {
              const uint64_t ad = sw128_desc(smem_u32(S.a[sa]) + kk * 32);
              const uint64_t bd = sw128_desc(smem_u32(S.b[sb][j0]) + kk * 32);
              const uint32_t acc = (f0 && kt == first && kk == 0) ? 0u : 1u;
              mma_bf16(tmem + (uint32_t)((i + j0) * TX_BN), ad, bd, idesc, acc);
            }
            j0 = j1 + 1;
          }
          mma_commit(&S.aempty[sa]);
        }
        if (!ok) break;
        mma_commit(&S.bempty[sb]);
        if (kt == last) mma_commit(&S.accfull);
      }
    }
  } else {
    // ---- drain warps 2..5: rows m0 + 32 (warp % 4) + lane
    const int q = warp & 3;
    const int row = m0 + q * 32 + lane;
    const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16);
    double acc[TX_BN];
#pragma unroll
    for (int j = 0; j < TX_BN; ++j) acc[j] = 0.0;
    bool good = true;
    for (int c = 0; c < nchunks; ++c) {
      if (!mbar_wait(&S.accfull, c & 1)) {
        atomicOr(err, 4);
        good = false;
        break;
      }
      tc_fence_after();
      // Each level's chunk sum is an integer below 2^24 in magnitude.  Levels
      // g0..g1-1 (at most five) are combined exactly in int64 as
      // sum_l L_l 2^(6 (g1 - 1 - l)) (< 2^49), so a group costs one
      // int64 -> FP64 conversion and one FMA per element on the FP64 pipe
      // instead of two per level.
#pragma unroll
      for (int t = 0; t < TX_BN / 16; ++t) {
#pragma unroll
        for (int g0 = 0; g0 < TX_LEVELS; g0 += 5) {
          const int g1 = g0 + 5 < TX_LEVELS ? g0 + 5 : TX_LEVELS;
          long long sum[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) sum[j] = 0;
#pragma unroll 1
          for (int l = g0; l < g1; ++l) {
            // 16-column loads: every start column (l * 48 + 16 t) is 16-aligned
            float v[16];
            tmem_ld16(tl + (uint32_t)(l * TX_BN + 16 * t), v);
            const long long wgt = 1LL << (6 * (g1 - 1 - l));
#pragma unroll
            for (int j = 0; j < 16; ++j) sum[j] += (long long)__float2int_rn(v[j]) * wgt;
          }
          const double sc = ldexp(1.0, -6 * (g1 - 1));   // 2^(-6 (g1 - 1)), exact
#pragma unroll
          for (int j = 0; j < 16; ++j) acc[16 * t + j] = fma((double)sum[j], sc, acc[16 * t + j]);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&S.accempty);
    }
    if (good && !S.abort_flag && row < M) {
      const int er = expA[row] - Cfg::SCALE;
#pragma unroll
      for (int j = 0; j < TX_BN; ++j) {
        const int col = n0 + j;
        if (col < N) {
          double* p = C + (size_t)row + (size_t)col * ldc;
          double r = alpha * ldexp(acc[j], er + expB[col]);
          if (beta != 0.0) r = fma(beta, *p, r);
          *p = r;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, TX_TMEM_COLS);
  }
}

// ------------------------------------------------------------------ host side
static size_t align1k(size_t b) { return (b + 1023) & ~(size_t)1023; }

template <int DIG>
static size_t tcx_ws_bytes(int m, int n, int k) {
  const size_t kp = ((size_t)std::max(k, 1) + TX_BK - 1) / TX_BK * TX_BK;
  auto planes = [&](int rows) { return align1k((size_t)DIG * rows * kp * 2); };
  return planes(m) + planes(n) + align1k((size_t)(m + n) * 8) + align1k((size_t)(m + n) * 4) + 256;
}

size_t tcx_gemm_workspace_bytes(int m, int n, int k) { return tcx_ws_bytes<9>(m, n, k); }
size_t tcx32_gemm_workspace_bytes(int m, int n, int k) { return tcx_ws_bytes<4>(m, n, k); }
size_t tcx30_gemm_workspace_bytes(int m, int n, int k) { return tcx_ws_bytes<5>(m, n, k); }

template <int DIG>
static cudaError_t slice_operand(cudaStream_t s, int rows, int K, int kp, const double* X, int ldx,
                                 bool kcontig, unsigned long long* mx, void* planes, int* expo) {
  if (rows <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(mx, 0, sizeof(unsigned long long) * rows, s);
  if (e != cudaSuccess) return e;
  dim3 g1((std::max(K, 1) + 63) / 64, (rows + 31) / 32);
  note_launches(1);
  rowmax_kernel<<<g1, 256, 0, s>>>(rows, K, X, ldx, kcontig ? 1 : 0, mx);
  dim3 g2((kp + 63) / 64, (rows + 31) / 32);
  note_launches(1);
  slice_kernel<DIG><<<g2, 256, 0, s>>>(rows, K, kp, X, ldx, kcontig ? 1 : 0, mx,
                                       static_cast<__nv_bfloat16*>(planes), (size_t)rows * kp,
                                       expo);
  return cudaGetLastError();
}

template <int DIG>
static cudaError_t tcx_run(cudaStream_t s, bool ta, bool tb, int m, int n, int k, double alpha,
                           const double* A, int lda, const double* B, int ldb, double beta,
                           double* C, int ldc, void* ws, int* err) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  if (k <= 0) return gemm(s, false, false, m, n, 0, alpha, A, lda, B, ldb, beta, C, ldc, 1, nullptr);
  const int kp = ((k + TX_BK - 1) / TX_BK) * TX_BK;
  char* base = static_cast<char*>(ws);
  const size_t abytes = align1k((size_t)DIG * m * kp * 2);
  const size_t bbytes = align1k((size_t)DIG * n * kp * 2);
  void* pa = base;
  void* pb = base + abytes;
  unsigned long long* mx = reinterpret_cast<unsigned long long*>(base + abytes + bbytes);
  int* ex = reinterpret_cast<int*>(base + abytes + bbytes + align1k((size_t)(m + n) * 8));
  // op(A) is m x k: its K-major rows are contiguous when A is stored k x m (ta)
  cudaError_t e = slice_operand<DIG>(s, m, k, kp, A, lda, ta, mx, pa, ex);
  if (e != cudaSuccess) return e;
  // the MMA's B operand is op(B)^T (n x k): contiguous in k when B is k x n (!tb)
  e = slice_operand<DIG>(s, n, k, kp, B, ldb, !tb, mx + m, pb, ex + m);
  if (e != cudaSuccess) return e;
  CUtensorMap ta_map, tb_map;
  if (!make_plane_map(&ta_map, pa, m, kp, TX_BM, DIG) ||
      !make_plane_map(&tb_map, pb, n, kp, TX_BN, DIG))
    return cudaErrorInvalidValue;
  static_assert(sizeof(TxSmem<DIG>) + 1024 <= 232448, "227 KB of dynamic shared memory");
  const size_t smem = sizeof(TxSmem<DIG>) + 1024;
  static const bool attr = [smem] {
    cudaFuncSetAttribute(tcx_gemm_kernel<DIG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    return true;
  }();
  (void)attr;
  dim3 grid((m + TX_BM - 1) / TX_BM, (n + TX_BN - 1) / TX_BN);
  note_launches(1);
  constexpr int pairs = (DIG == 9) ? 53 : (DIG == 5 ? 15 : 10);   // digit pairs of the kept levels
  const TimingToken tt = timing_begin(s, DIG == 9 ? TIMING_TCX64 : TIMING_TCX32,
                                      2.0 * pairs * m * (double)n * k);
  tcx_gemm_kernel<DIG><<<grid, TX_THREADS, smem, s>>>(ta_map, tb_map, m, n, kp, alpha, beta, C,
                                                      ldc, ex, ex + m, err);
  timing_end(s, tt);
  return cudaGetLastError();
}

cudaError_t tcx_gemm(cudaStream_t s, bool ta, bool tb, int m, int n, int k, double alpha,
                     const double* A, int lda, const double* B, int ldb, double beta, double* C,
                     int ldc, void* ws, int* err) {
  return tcx_run<9>(s, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, ws, err);
}

cudaError_t tcx30_gemm(cudaStream_t s, bool ta, bool tb, int m, int n, int k, double alpha,
                       const double* A, int lda, const double* B, int ldb, double beta, double* C,
                       int ldc, void* ws, int* err) {
  return tcx_run<5>(s, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, ws, err);
}

cudaError_t tcx32_gemm(cudaStream_t s, bool ta, bool tb, int m, int n, int k, double alpha,
                       const double* A, int lda, const double* B, int ldb, double beta, double* C,
                       int ldc, void* ws, int* err) {
  return tcx_run<4>(s, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, ws, err);
}

}  // namespace eigdc
