// Split-BF16 (three-term) GEMM on the fifth-generation tensor cores.
//
// C = alpha op(A) op(B) + beta C with FP64 storage and FP32-level accuracy:
// each FP64 operand is split into three BF16 planes x = hi + mid + lo
// (8 + 8 + 8 significant bits), and the product keeps the six terms of
// weight >= 2^-16 relative to hi*hi:
//     hi*hi + hi*mid + mid*hi + hi*lo + mid*mid + lo*hi,
// accumulated in FP32 in tensor memory.  This is the split-precision form of
// the contractions of the inverse-free iteration (trailing compact-WY updates,
// complement products); panels, norms and split tests stay FP64.
//
// Kernel structure (one CTA per 128 x 128 output tile, 128 threads):
//   * operands arrive as K-major BF16 planes (split3_kernel), loaded by TMA
//     (cp.async.bulk.tensor, 128-byte swizzle) into a 2-stage ring of shared
//     memory, each stage holding the three planes of a 128 x 64 slab of A and B;
//   * one thread issues tcgen05.mma (kind::f16, BF16 inputs, FP32 accumulate)
//     into a 128 x 128 FP32 accumulator in TMEM, 6 plane pairs x 4 K-steps per
//     stage, and frees a stage with tcgen05.commit on its "empty" mbarrier;
//   * all four warps read the accumulator with tcgen05.ld (warp w owns TMEM
//     lanes 32w..32w+31, i.e. the tile's rows) and write alpha*acc + beta*C.
// Every mbarrier wait is bounded; on a timeout the CTA records an error flag,
// skips its remaining work and still frees its TMEM.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <algorithm>

#include "internal.h"
#include "tc_ptx.cuh"

namespace eigdc {

constexpr int TC_BM = 128, TC_BN = 128, TC_BK = 64, TC_STAGES = 2, TC_THREADS = 128;
constexpr int TC_PLANES = 3;
constexpr int TC_TILE_A = TC_BM * TC_BK * 2;   // bytes of one plane slab of A
constexpr int TC_TILE_B = TC_BN * TC_BK * 2;

struct TcSmem {
  uint8_t a[TC_STAGES][TC_PLANES][TC_TILE_A];
  uint8_t b[TC_STAGES][TC_PLANES][TC_TILE_B];
  uint64_t full[TC_STAGES];
  uint64_t empty[TC_STAGES];
  uint64_t done;
  uint32_t tmem_base;
  int abort_flag;
};
static_assert(TC_TILE_A % 1024 == 0 && TC_TILE_B % 1024 == 0, "1024-byte swizzle atoms");

// ------------------------------------------------------------------ kernels
// Planes of the K-major operand X' (rows x K): element (r, k) is
// X[k + r*ldx] (kcontig) or X[r + k*ldx]; planes[p][r*kp + k], zero for k >= K.
__global__ void __launch_bounds__(256)
split3_kernel(int rows, int K, int kp, const double* __restrict__ X, int ldx, int kcontig,
              __nv_bfloat16* __restrict__ P, size_t pstride) {
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
    const double x = tile[rr][kk];
    const __nv_bfloat16 hi = __double2bfloat16(x);
    const double r1 = x - (double)__bfloat162float(hi);
    const __nv_bfloat16 mid = __double2bfloat16(r1);
    const double r2 = r1 - (double)__bfloat162float(mid);
    const __nv_bfloat16 lo = __double2bfloat16(r2);
    const size_t o = (size_t)r * kp + k;
    P[o] = hi;
    P[pstride + o] = mid;
    P[2 * pstride + o] = lo;
  }
}

__global__ void __launch_bounds__(TC_THREADS, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               int M, int N, int K, double alpha, double beta, double* __restrict__ C, int ldc,
               int* err) {
  extern __shared__ uint8_t smem_raw[];
  TcSmem& S = *reinterpret_cast<TcSmem*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                         ~static_cast<uintptr_t>(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * TC_BM, n0 = blockIdx.y * TC_BN;
  const int nk = (K + TC_BK - 1) / TC_BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&S.full[s], 1);
      mbar_init(&S.empty[s], 1);
    }
    mbar_init(&S.done, 1);
    S.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
  }
  if (warp == 2) tmem_alloc(&S.tmem_base, TC_BN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem_base;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % TC_STAGES;
      const uint32_t ph = (kt / TC_STAGES) & 1;
      if (!mbar_wait(&S.empty[s], ph ^ 1)) {
        S.abort_flag = 1;
        atomicOr(err, 1);
        break;
      }
      mbar_arrive_expect_tx(&S.full[s], TC_PLANES * (TC_TILE_A + TC_TILE_B));
      for (int p = 0; p < TC_PLANES; ++p) {
        tma_load_3d(S.a[s][p], &tmA, &S.full[s], kt * TC_BK, m0, p);
        tma_load_3d(S.b[s][p], &tmB, &S.full[s], kt * TC_BK, n0, p);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    constexpr uint32_t idesc = idesc_bf16_f32(TC_BM, TC_BN);
    // plane pairs (a, b) of weight >= 2^-16
    const int pa[6] = {0, 0, 1, 0, 1, 2};
    const int pb[6] = {0, 1, 0, 2, 1, 0};
    bool ok = true;
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % TC_STAGES;
      const uint32_t ph = (kt / TC_STAGES) & 1;
      if (!mbar_wait(&S.full[s], ph)) {
        S.abort_flag = 1;
        atomicOr(err, 2);
        ok = false;
        break;
      }
      tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < TC_BK / 16; ++kk) {
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          const uint64_t ad = sw128_desc(smem_u32(S.a[s][pa[q]]) + kk * 32);
          const uint64_t bd = sw128_desc(smem_u32(S.b[s][pb[q]]) + kk * 32);
          mma_bf16(tmem, ad, bd, idesc, (kt > 0 || kk > 0 || q > 0) ? 1u : 0u);
        }
      }
      mma_commit(&S.empty[s]);
    }
    if (ok) mma_commit(&S.done);
  }
  __syncwarp();
  // ---- epilogue: warp w owns rows m0 + 32w .. m0 + 32w + 31
  const bool done = (nk > 0) ? mbar_wait(&S.done, 0) : true;
  tc_fence_after();
  if (!done) atomicOr(err, 4);
  const bool good = done && S.abort_flag == 0;
  const int row = m0 + warp * 32 + lane;
#pragma unroll 1
  for (int c0 = 0; c0 < TC_BN; c0 += 32) {
    float v[32];
    if (nk > 0) {
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] = 0.0f;
    }
    if (good && row < M) {
#pragma unroll 4
      for (int j = 0; j < 32; ++j) {
        const int col = n0 + c0 + j;
        if (col < N) {
          double* p = C + (size_t)row + (size_t)col * ldc;
          double r = alpha * (double)v[j];
          if (beta != 0.0) r = fma(beta, *p, r);
          *p = r;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    tmem_dealloc(tmem, TC_BN);
  }
}

// ------------------------------------------------------------------ host side
// The driver's tensor-map encoder, looked up once (thread-safe static init);
// nullptr when the driver does not provide it.
static PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fnp = [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                         cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || fn == nullptr) {
      cudaGetLastError();
      return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }();
  return fnp;
}

static bool encode_fn() { return encoder() != nullptr; }

// 3-D tensor map over K-major BF16 planes: (k, row, plane), box 64 x box_rows x 1,
// 128-byte swizzle.
bool make_plane_map(CUtensorMap* map, void* base, int rows, int kp, int box_rows, int planes) {
  if (!encode_fn()) return false;
  cuuint64_t dims[3] = {(cuuint64_t)kp, (cuuint64_t)rows, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)kp * 2, (cuuint64_t)kp * 2 * (cuuint64_t)rows};
  cuuint32_t box[3] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = encoder()(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box,
                              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

size_t tc_gemm_workspace_bytes(int m, int n, int k) {
  const size_t kp = ((size_t)std::max(k, 1) + TC_BK - 1) / TC_BK * TC_BK;
  auto planes = [&](int rows) { return ((size_t)TC_PLANES * rows * kp * 2 + 1023) & ~(size_t)1023; };
  return planes(m) + planes(n) + 256;
}

cudaError_t split3(cudaStream_t s, int rows, int K, int kp, const double* X, int ldx, bool kcontig,
                   void* planes) {
  if (rows <= 0) return cudaSuccess;
  dim3 grid((kp + 63) / 64, (rows + 31) / 32);
  note_launches(1);
  split3_kernel<<<grid, 256, 0, s>>>(rows, K, kp, X, ldx, kcontig ? 1 : 0,
                                     static_cast<__nv_bfloat16*>(planes), (size_t)rows * kp);
  return cudaGetLastError();
}

cudaError_t tc_gemm(cudaStream_t s, bool ta, bool tb, int m, int n, int k, double alpha,
                    const double* A, int lda, const double* B, int ldb, double beta, double* C,
                    int ldc, void* ws, int* err) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  if (!encode_fn()) return cudaErrorNotSupported;
  const int kp = ((std::max(k, 1) + TC_BK - 1) / TC_BK) * TC_BK;
  char* base = static_cast<char*>(ws);
  const size_t abytes = ((size_t)TC_PLANES * m * kp * 2 + 1023) & ~(size_t)1023;
  void* pa = base;
  void* pb = base + abytes;
  // op(A) is m x k: K-major rows are contiguous when A is stored k x m (ta)
  cudaError_t e = split3(s, m, k, kp, A, lda, ta, pa);
  if (e != cudaSuccess) return e;
  // the MMA's B operand is op(B)^T (n x k): contiguous in k when B is k x n (!tb)
  e = split3(s, n, k, kp, B, ldb, !tb, pb);
  if (e != cudaSuccess) return e;
  CUtensorMap ta_map, tb_map;
  if (!make_plane_map(&ta_map, pa, m, kp, TC_BM, TC_PLANES) ||
      !make_plane_map(&tb_map, pb, n, kp, TC_BN, TC_PLANES))
    return cudaErrorInvalidValue;
  const size_t smem = sizeof(TcSmem) + 1024;
  static const bool attr = [smem] {   // once per process (thread-safe static init)
    cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return true;
  }();
  (void)attr;
  dim3 grid((m + TC_BM - 1) / TC_BM, (n + TC_BN - 1) / TC_BN);
  note_launches(1);
  tc_gemm_kernel<<<grid, TC_THREADS, smem, s>>>(ta_map, tb_map, m, n, k, alpha, beta, C, ldc, err);
  return cudaGetLastError();
}

}  // namespace eigdc
