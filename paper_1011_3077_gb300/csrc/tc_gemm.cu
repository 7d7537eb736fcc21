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

namespace eigdc {

constexpr int TC_BM = 128, TC_BN = 128, TC_BK = 64, TC_STAGES = 2, TC_THREADS = 128;
constexpr int TC_PLANES = 3;
constexpr int TC_TILE_A = TC_BM * TC_BK * 2;   // bytes of one plane slab of A
constexpr int TC_TILE_B = TC_BN * TC_BK * 2;
constexpr uint32_t TC_WAIT_LIMIT = 1u << 26;

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

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase of the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t i = 0; i < TC_WAIT_LIMIT; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes (64 BF16) in 1024-byte groups of 8 rows.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);           // start address (16-byte units)
  d |= (uint64_t)1u << 16;                             // leading byte offset (unused here)
  d |= (uint64_t)((1024u >> 4) & 0x3FFFu) << 32;       // stride byte offset: 8 rows
  d |= (uint64_t)1u << 46;                             // descriptor version
  d |= (uint64_t)2u << 61;                             // 128-byte swizzle
  return d;
}

// Instruction descriptor of kind::f16: BF16 A and B (K-major), FP32 D, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// 32 consecutive FP32 columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

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
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

static bool encode_fn() {
  if (g_encode) return true;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                       &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || fn == nullptr) {
    cudaGetLastError();
    return false;
  }
  g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return true;
}

// 3-D tensor map over the planes: (k, row, plane), box 64 x box_rows x 1.
static bool make_plane_map(CUtensorMap* map, void* base, int rows, int kp, int box_rows) {
  cuuint64_t dims[3] = {(cuuint64_t)kp, (cuuint64_t)rows, (cuuint64_t)TC_PLANES};
  cuuint64_t strides[2] = {(cuuint64_t)kp * 2, (cuuint64_t)kp * 2 * (cuuint64_t)rows};
  cuuint32_t box[3] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box,
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
  if (!make_plane_map(&ta_map, pa, m, kp, TC_BM) || !make_plane_map(&tb_map, pb, n, kp, TC_BN))
    return cudaErrorInvalidValue;
  static bool attr = false;
  const size_t smem = sizeof(TcSmem) + 1024;
  if (!attr) {
    cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  dim3 grid((m + TC_BM - 1) / TC_BM, (n + TC_BN - 1) / TC_BN);
  note_launches(1);
  tc_gemm_kernel<<<grid, TC_THREADS, smem, s>>>(ta_map, tb_map, m, n, k, alpha, beta, C, ldc, err);
  return cudaGetLastError();
}

}  // namespace eigdc
