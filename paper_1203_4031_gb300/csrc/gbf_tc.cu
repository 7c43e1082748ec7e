// Tensor-core GEMM building block for sm_103a (tcgen05 + TMA + TMEM):
//   C[b] (M x N, FP32, column-major, ldc) = A[b] (M x K) * B[b]^T (N x K)
// with A and B bf16, both K-major (row r holds its K values contiguously,
// row pitch K, K a multiple of 8), batches b strided by M*K / N*K.
//
// One CTA computes one BM x BN tile (BM = 128 TMEM lanes, BN = 128 FP32
// TMEM columns) with warp roles:
//   warp 0  TMA producer: 3-D tiled loads (box 64 x 128 x 1, 128-byte
//           swizzle) of the A and B k-tiles into a STAGES-deep ring, each
//           stage guarded by a "full" mbarrier (expect_tx bytes);
//   warp 1  allocates the TMEM accumulator; one elected thread issues
//           tcgen05.mma (kind::f16, BF16 x BF16 -> FP32, M=128, N=BN, K=16,
//           four per 64-wide k-tile) and tcgen05.commit to the stage's
//           "empty" mbarrier, then to the accumulator barrier;
//   warps 2-5 epilogue: tcgen05.ld 32x32b.x16 of their 32-lane quarter of
//           the accumulator, FP32 stores (or FP64 accumulation with a scale).
// Every mbarrier wait is bounded: on time-out the thread raises the CTA's
// abort flag and a global error word, the other roles stop at their next
// wait, and the CTA still frees its TMEM before returning.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "gbf_common.cuh"

namespace gbf {
namespace tc {

constexpr int BM = 128, BN = 128, BK = 64, STAGES = 4;
constexpr int A_TILE = BM * BK * 2;  // bytes
constexpr int B_TILE = BN * BK * 2;
constexpr int STAGE = A_TILE + B_TILE;
constexpr int SMEM_BYTES = STAGES * STAGE + 1024 /* align */ + 256 /* barriers */;
constexpr int THREADS = 192;
constexpr long WAIT_LIMIT = 1L << 26;

__device__ __forceinline__ uint32_t sm_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sm_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sm_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(sm_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait; false when the CTA aborted (time-out here or elsewhere).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag, int *gerr,
                                          int code) {
  for (long it = 0; it < WAIT_LIMIT; ++it) {
    if (mbar_try(bar, parity)) return true;
    if (*abort_flag) return false;
  }
  *abort_flag = 1;
  atomicCAS(gerr, 0, code);
  return false;
}

// Bounded wait that ignores the abort flag: used to let this thread's own
// asynchronous work (copies, MMAs) finish before the CTA frees resources.
__device__ __forceinline__ void mbar_drain(uint64_t *bar, uint32_t parity, int *gerr, int code) {
  for (long it = 0; it < WAIT_LIMIT; ++it)
    if (mbar_try(bar, parity)) return;
  atomicCAS(gerr, 0, code);
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1,
                                            int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
      "[%2];" ::"r"(sm_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(sm_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle
// (8-row x 128-byte atoms, stride between 8-row groups 1024 bytes).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);  // start address
  d |= (uint64_t)1 << 16;                   // leading byte offset (16 B, unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;         // stride byte offset
  d |= (uint64_t)1 << 46;                   // descriptor version
  d |= (uint64_t)2 << 61;                   // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: FP32 accumulate, BF16 A and B, both
// K-major, N = BN, M = BM.
__host__ __device__ constexpr uint32_t idesc_bf16() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(sm_u32(bar))
               : "memory");
}

// Epilogue mode 0: C = acc (FP32).  Mode 1: C64 += scale * acc (FP64).
template <int MODE>
__global__ void __launch_bounds__(THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, int M, int N,
                   int K, float *C, double *C64, long ldc, long sc, double scale, int *gerr) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned stage ring, then the barriers
  unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t *full = reinterpret_cast<uint64_t *>(base + STAGES * STAGE);
  uint64_t *empty = full + STAGES;
  uint64_t *accb = empty + STAGES;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(accb + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN, b = blockIdx.z;
  const int num_k = (K + BK - 1) / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accb, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sm_u32(tmem_slot)),
                 "r"((uint32_t)BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // producer
    int issued = 0;
    for (int kt = 0; kt < num_k; ++kt) {
      const int s = kt % STAGES;
      const uint32_t round = kt / STAGES;
      if (kt >= STAGES && !mbar_wait(&empty[s], (round - 1) & 1, abort_flag, gerr, 1)) break;
      unsigned char *sa = base + s * STAGE;
      mbar_expect_tx(&full[s], STAGE);
      tma_load_3d(sa, &ta, &full[s], kt * BK, m0, b);
      tma_load_3d(sa + A_TILE, &tb, &full[s], kt * BK, n0, b);
      issued = kt + 1;
    }
    // drain: every copy this thread issued has landed before it moves on
    for (int kt = (issued > STAGES ? issued - STAGES : 0); kt < issued; ++kt)
      mbar_drain(&full[kt % STAGES], (kt / STAGES) & 1, gerr, 2);
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    constexpr uint32_t idesc = idesc_bf16();
    bool ok = true;
    for (int kt = 0; kt < num_k && ok; ++kt) {
      const int s = kt % STAGES;
      if (!mbar_wait(&full[s], (kt / STAGES) & 1, abort_flag, gerr, 3)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = sm_u32(base + s * STAGE);
      const uint64_t ad = sdesc_sw128(sa), bd = sdesc_sw128(sa + A_TILE);
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk)
        mma_bf16(tmem, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), idesc, (kt > 0 || kk > 0) ? 1u : 0u);
      mma_commit(&empty[s]);
    }
    mma_commit(accb);
    // every MMA this thread issued has completed before TMEM can be freed
    mbar_drain(accb, 0, gerr, 5);
  } else if (warp >= 2) {
    // epilogue: warp w reads TMEM lanes 32*(w % 4) .. +31; the decision to
    // read is warp-uniform (tcgen05.ld is .sync.aligned)
    const int q = warp & 3;
    int okw = 0;
    if (lane == 0) okw = mbar_wait(accb, 0, abort_flag, gerr, 4) ? 1 : 0;
    const bool ok = __shfl_sync(0xffffffffu, okw, 0) != 0;
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
      const int row = m0 + q * 32 + lane;
      for (int c0 = 0; c0 < BN; c0 += 16) {
        uint32_t r[16];
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
            "[%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (row < M) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int col = n0 + c0 + j;
            if (col < N) {
              const float v = __uint_as_float(r[j]);
              const long off = (long)b * sc + row + (long)col * ldc;
              if (MODE == 0)
                C[off] = v;
              else
                C64[off] += scale * (double)v;
            }
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)BN) : "memory");
}

// ------------------------------------------------------------- host side --
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 3-D map over a bf16 [batch][rows][K] array, box 64 (K) x 128 (rows) x 1.
static int make_map(CUtensorMap *map, const void *ptr, long rows, long K, int batch) {
  auto fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled unavailable");
    return -4;
  }
  if ((K % 8) != 0 || ((uintptr_t)ptr & 15) != 0) {
    set_error("tensor-core GEMM: K must be a multiple of 8 and the base 16-byte aligned");
    return -4;
  }
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)batch};
  cuuint64_t strides[2] = {(cuuint64_t)K * 2, (cuuint64_t)rows * K * 2};
  cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)BM, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(ptr), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
    return -4;
  }
  return 0;
}

template <int MODE>
static int launch(cudaStream_t st, int M, int N, int K, int batch, const void *A, const void *B, float *C,
                  double *C64, long ldc, long sc, double scale, int *gerr) {
  CUtensorMap ta, tb;
  if (int rc = make_map(&ta, A, M, K, batch)) return rc;
  if (int rc = make_map(&tb, B, N, K, batch)) return rc;
  static bool attr = false;
  if (!attr) {
    GBF_CUDA(cudaFuncSetAttribute(tc_gemm_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    attr = true;
  }
  dim3 grid(ceil_div(M, BM), ceil_div(N, BN), batch);
  tc_gemm_kernel<MODE><<<grid, THREADS, SMEM_BYTES, st>>>(ta, tb, M, N, K, C, C64, ldc, sc, scale, gerr);
  GBF_LAUNCHED();
  GBF_CUDA(cudaGetLastError());
  return 0;
}

}  // namespace tc

int tc_gemm_bf16_f32(cudaStream_t st, int M, int N, int K, int batch, const void *A, const void *B, float *C,
                     long ldc, long sc, int *gerr) {
  return tc::launch<0>(st, M, N, K, batch, A, B, C, nullptr, ldc, sc, 0.0, gerr);
}
int tc_gemm_bf16_acc64(cudaStream_t st, int M, int N, int K, int batch, const void *A, const void *B, double *C64,
                       long ldc, long sc, double scale, int *gerr) {
  return tc::launch<1>(st, M, N, K, batch, A, B, nullptr, C64, ldc, sc, scale, gerr);
}

}  // namespace gbf

// Verification entry (C ABI): C (FP32, column-major, ldc, batch stride
// sc) = A B^T with A [batch][M][K], B [batch][N][K] bf16 (K-major).
// Returns 0, -4 on a CUDA error, or -5 when a bounded wait timed out in
// the kernel (error word non-zero).
extern "C" int gbf_tc_gemm_bf16(void *stream, int M, int N, int K, int batch, const void *dA, const void *dB,
                                float *dC, long ldc, long sc, int *dErr) {
  if (M < 1 || N < 1 || K < 1 || batch < 1) return -102;
  cudaStream_t st = (cudaStream_t)stream;
  GBF_CUDA(cudaMemsetAsync(dErr, 0, sizeof(int), st));
  int rc = gbf::tc_gemm_bf16_f32(st, M, N, K, batch, dA, dB, dC, ldc, sc, dErr);
  if (rc) return rc;
  int herr = 0;
  GBF_CUDA(cudaMemcpyAsync(&herr, dErr, sizeof(int), cudaMemcpyDeviceToHost, st));
  GBF_CUDA(cudaStreamSynchronize(st));
  if (herr) {
    gbf::set_error("tensor-core GEMM: bounded wait timed out (code %d)", herr);
    return -5;
  }
  return 0;
}
