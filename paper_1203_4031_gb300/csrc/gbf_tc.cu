// Tensor-core engine for sm_103a (tcgen05 + TMA + TMEM).  This file holds:
//   * tc_gemm_kernel: the bf16 building block described below;
//   * zgemm_sliced_kernel: k <= 32 complex products from exact bf16 digit
//     products (FP64-class for the FP64 factors' LU updates and solve steps);
//   * ctf32_kernel: k <= 32 complex FP32 products as 3xTF32 (the FP32
//     factors' large updates);
//   * gemm_sliced_k_kernel: any-k FP64-class sliced products (projections,
//     the recursive solves' large-K updates, reduced-space products);
//   * the slicing / splitting kernels that lay the operands out K-major for
//     the TMA boxes, the host launchers and the C-ABI verification entries.
//
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
#include <cuda_bf16.h>

#include <algorithm>
#include <type_traits>
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
__device__ __forceinline__ bool mbar_wait_n(uint64_t *bar, uint32_t parity, volatile int *abort_flag, int *gerr,
                                            int code, long limit) {
  for (long it = 0; it < limit; ++it) {
    if (mbar_try(bar, parity)) return true;
    if (*abort_flag) return false;
  }
  *abort_flag = 1;
  atomicCAS(gerr, 0, code);
  return false;
}
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag, int *gerr,
                                          int code) {
  return mbar_wait_n(bar, parity, abort_flag, gerr, code, WAIT_LIMIT);
}

// The time-out path of the pipeline waits, exercised without a fault: one
// thread waits, with the same bounded loop, on a barrier that nothing
// completes, for `limit` polls; the error word gets `code` and the kernel
// returns (no asynchronous work is in flight).
__global__ void wait_probe_kernel(long limit, int *gerr, int code) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait_n(&bar, 0, &abort_flag, gerr, code, limit);
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
// The same arrival on the barrier at this offset in every CTA of `mask`.
__device__ __forceinline__ void mma_commit_mc(uint64_t *bar, uint16_t mask) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::
                   "r"(sm_u32(bar)), "h"(mask)
               : "memory");
}
// Tiled load written to the same shared-memory offset of every CTA of
// `mask`, each CTA's barrier at `bar`'s offset receiving the bytes.
__device__ __forceinline__ void tma_load_3d_mc(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1,
                                               int c2, uint16_t mask) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.multicast::cluster [%0], "
      "[%1, {%3, %4, %5}], [%2], %6;" ::"r"(sm_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(sm_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "h"(mask)
      : "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
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
  static std::atomic<unsigned long long> attr_done{0};
  if (int rc = once_per_device(attr_done, [&]() -> int {
      GBF_CUDA(cudaFuncSetAttribute(tc_gemm_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
        return 0;
      }))
    return rc;
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

// ===================================================================
// Sliced complex GEMM on the tensor cores:
//   C = alpha op(A) op(B) + beta C,  complex (zd or cf), k <= 32,
//   alpha in {+1, -1}, beta in {0, 1}.
// Real embedding: complex row i of op(A) -> real rows 2i = [Re | -Im] and
// 2i+1 = [Im | Re] (length 2k); column c of op(B) -> [Re ; Im].  Then
// real row 2i (2i+1) times column c is Re (Im) of the complex product.
// Slicing: each real row r is scaled by a power of two sigma_r above its
// largest magnitude, each column c by tau_c; x/sigma (|x/sigma| < 1) is
// rounded once to 7S fractional bits and written as sum_{t=1..S} d_t 2^{-7t}
// with integer digits d_t (|d_1| <= 128, |d_t| <= 64 after), each exact in
// bf16.  For digit pairs (t, u) with t + u <= S + 1, the products
// D_t E_u^T are integers below 2^22 in magnitude even summed over all pairs
// of one weight (64 terms, at most S pairs), so one FP32 TMEM accumulator
// per weight w = t + u holds them exactly; the epilogue combines the S_w
// exactly in int64 and rounds sigma_r tau_c sum_w 2^{-7w} S_w once.
// S = 7 keeps 49 bits per operand relative to its row/column maximum
// (FP64-class products); S = 3 keeps 21 bits (FP32-class).
// ===================================================================
namespace gbf {
namespace tc {

constexpr int ZK = 64;          // padded 2k (one 64-wide k-tile)
constexpr int ZBN = 32;         // output columns per tile
constexpr int ZA_TILE = BM * ZK * 2;
constexpr int ZB_TILE = ZBN * ZK * 2;

template <class T> struct cplx_io;
template <> struct cplx_io<zd> {
  using R = double;
};
template <> struct cplx_io<cf> {
  using R = float;
};

// Slicing.  A row (or column) of op(A) (op(B)) is scaled by a power of two
// 2^e above its largest real or imaginary part, so every scaled part v has
// |v| < 1; v is rounded once to X = rint(v 2^{7S}) (an integer, |X| <= 2^{7S})
// and X is split into S balanced base-2^7 digits, least significant first:
// d = ((X + 64) mod 128) - 64, X <- (X - d) / 128; the leading digit takes
// what remains (|d_0| <= 128, the others <= 64), so v = sum_t d_t 2^{-7(t+1)}
// up to 2^{-7S-1}.  All of it is integer work on the FP64 bit patterns.

// Largest |re|, |im| bit pattern (ordered like the magnitudes) over the warp.
__device__ __forceinline__ unsigned long long warp_absmax_bits(double re, double im) {
  const unsigned long long a = (unsigned long long)__double_as_longlong(re) & 0x7FFFFFFFFFFFFFFFull;
  const unsigned long long c = (unsigned long long)__double_as_longlong(im) & 0x7FFFFFFFFFFFFFFFull;
  unsigned long long m = a > c ? a : c;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, m, off);
    m = o > m ? o : m;
  }
  return m;
}

// e with 2^e > the magnitude whose bit pattern is mb (the frexp exponent);
// 0 for a zero row.
__device__ __forceinline__ int scale_exp(unsigned long long mb) {
  if (mb == 0) return 0;
  const int f = (int)(mb >> 52);
  if (f == 0) return ilogb(__longlong_as_double((long long)mb)) + 1;
  return f - 1022;
}

// rint(v 2^{7S - e}) for a finite v with |v| < 2^e, ties to even.
template <int S>
__device__ __forceinline__ long long fixed_point(double v, int e) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  const int f = (int)((bits >> 52) & 0x7FF);
  const unsigned long long mant = (bits & 0x000FFFFFFFFFFFFFull) | (f ? 0x0010000000000000ull : 0ull);
  // v = mant 2^{ev - 52}; v 2^{7S - e} = mant 2^{-r}, r >= 1 because |v| < 2^e
  const int ev = (f ? f : 1) - 1023;
  const int r = 52 - ev - 7 * S + e;
  long long X;
  if (mant == 0 || r > 54) {
    X = 0;
  } else if (r <= 0) {  // not reached for |v| < 2^e; kept total
    X = (long long)(mant << (-r));
  } else {
    X = (long long)((mant + ((1ull << (r - 1)) - 1ull) + ((mant >> r) & 1ull)) >> r);
  }
  return (bits >> 63) ? -X : X;
}

template <int S>
__device__ __forceinline__ void int_digits(long long X, float *d) {
#pragma unroll
  for (int t = S - 1; t > 0; --t) {
    const long long dt = ((X + 64) & 127) - 64;
    d[t] = (float)(int)dt;
    X = (X - dt) >> 7;
  }
  d[0] = (float)(int)X;
}

// A side: one warp per complex row i of op(A) (m x k), lane p < k holds
// element (i, p).  Out: slices [S][batch][2m][ZK] bf16 holding rows
// 2i = [Re | -Im] and 2i+1 = [Im | Re] of the scaled row, zero-padded to ZK;
// sexp [batch][2m] = e, the row's scale 2^e.
// SPLIT: instead of digits, each entry (FP32 data) is split into S bf16 parts
// hi + mid + lo (each the bf16 rounding of what the previous parts leave),
// unscaled (exponents 0): FP32-class products accumulated in FP32.
template <int S>
__device__ __forceinline__ void float_split(double v, float *d) {
  float r = (float)v;
#pragma unroll
  for (int t = 0; t < S; ++t) {
    d[t] = __bfloat162float(__float2bfloat16_rn(r));
    r -= d[t];
  }
}

template <class T, int S, bool SPLIT>
__global__ void slice_a_kernel(char opa, int m, int k, const T *A, long lda, long sa, int batch,
                               __nv_bfloat16 *out, int *sexp) {
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), b = blockIdx.y, p = threadIdx.x & 31;
  if (i >= m) return;  // warp-uniform
  const T *Ab = A + (long)b * sa;
  double re = 0.0, im = 0.0;
  if (p < k) {
    T a = (opa == 'N') ? Ab[i + (long)p * lda] : Ab[p + (long)i * lda];
    re = (double)a.x;
    im = (opa == 'C') ? -(double)a.y : (double)a.y;
  }
  const int e = SPLIT ? 0 : scale_exp(warp_absmax_bits(re, im));
  float dr[S], di[S];
  if constexpr (SPLIT) {
    float_split<S>(re, dr);
    float_split<S>(im, di);
  } else {
    int_digits<S>(fixed_point<S>(re, e), dr);
    int_digits<S>(fixed_point<S>(im, e), di);
  }
  const long rows = 2L * m;
  for (int t = 0; t < S; ++t) {
    __nv_bfloat16 *o = out + (((long)t * batch + b) * rows) * ZK;
    __nv_bfloat16 *r0 = o + (2L * i) * ZK, *r1 = o + (2L * i + 1) * ZK;
    if (p < k) {
      r0[p] = __float2bfloat16_rn(dr[t]);
      r0[k + p] = __float2bfloat16_rn(-di[t]);
      r1[p] = __float2bfloat16_rn(di[t]);
      r1[k + p] = __float2bfloat16_rn(dr[t]);
    }
    for (int q = 2 * k + p; q < ZK; q += 32) {
      r0[q] = __float2bfloat16_rn(0.f);
      r1[q] = __float2bfloat16_rn(0.f);
    }
  }
  if (p == 0) {
    sexp[(long)b * rows + 2 * i] = e;
    sexp[(long)b * rows + 2 * i + 1] = e;
  }
}

// B side: one warp per column c of op(B) (k x n), lane p < k holds element
// (p, c).  Out: slices [S][batch][n][ZK] bf16 holding [Re ; Im] of the scaled
// column, zero-padded; texp [batch][n] = e, the column's scale 2^e.
template <class T, int S, bool SPLIT>
__global__ void slice_b_kernel(char opb, int k, int n, const T *B, long ldb, long sb, int batch,
                               __nv_bfloat16 *out, int *texp) {
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), b = blockIdx.y, p = threadIdx.x & 31;
  if (c >= n) return;  // warp-uniform
  const T *Bb = B + (long)b * sb;
  double re = 0.0, im = 0.0;
  if (p < k) {
    T v = (opb == 'N') ? Bb[p + (long)c * ldb] : Bb[c + (long)p * ldb];
    re = (double)v.x;
    im = (opb == 'C') ? -(double)v.y : (double)v.y;
  }
  const int e = SPLIT ? 0 : scale_exp(warp_absmax_bits(re, im));
  float dr[S], di[S];
  if constexpr (SPLIT) {
    float_split<S>(re, dr);
    float_split<S>(im, di);
  } else {
    int_digits<S>(fixed_point<S>(re, e), dr);
    int_digits<S>(fixed_point<S>(im, e), di);
  }
  for (int t = 0; t < S; ++t) {
    __nv_bfloat16 *o = out + (((long)t * batch + b) * n + c) * ZK;
    if (p < k) {
      o[p] = __float2bfloat16_rn(dr[t]);
      o[k + p] = __float2bfloat16_rn(di[t]);
    }
    for (int q = 2 * k + p; q < ZK; q += 32) o[q] = __float2bfloat16_rn(0.f);
  }
  if (p == 0) texp[(long)b * n + c] = e;
}

// Instruction descriptor for N = ZBN.
__host__ __device__ constexpr uint32_t idesc_bf16_n(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

template <int S, bool SPLIT = false> struct zlay {
  // A slices of one 128-row block (resident per work item) + a ring of NB
  // stages of the B slices of one 32-column tile, as deep as fits in 227 KB
  static constexpr int FIXED = S * ZA_TILE + 1024 + 256;
  static constexpr int NB = (FIXED + 4 * S * ZB_TILE <= 232448) ? 4 : (FIXED + 3 * S * ZB_TILE <= 232448) ? 3 : 2;
  static constexpr int SMEM = FIXED + NB * S * ZB_TILE;
  // one accumulator buffer: S weights x ZBN (digits) or one sum (split)
  static constexpr int ACC_COLS = SPLIT ? ZBN : S * ZBN;
  static constexpr int COLS = (2 * ACC_COLS <= 64) ? 64 : (2 * ACC_COLS <= 128) ? 128 : (2 * ACC_COLS <= 256) ? 256 : 512;
};

// Sum over the weights of (float bits of s_a + 1.5 2^23) 2^{7(S-1-a)} taken
// mod 2^64 equals x + KS with the constant below, so x comes out of S
// multiply-adds and one subtraction (wrap-around is harmless: |x| < 2^63).
template <int S> __host__ __device__ constexpr unsigned long long acc_bias() {
  unsigned long long k = 0;
  for (int a = 0; a < S; ++a) k += 0x4B400000ull << (7 * (S - 1 - a));
  return k;
}

// x + a 2^w for w < 32 (one wide multiply-add) and for 32 <= w < 64 (a
// multiply-add on the high word).
template <int W>
__device__ __forceinline__ unsigned long long add_shifted(unsigned long long x, uint32_t a) {
  unsigned long long r;
  if (W < 32) {
    asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(r) : "r"(a), "r"(1u << (W & 31)), "l"(x));
  } else {
    asm("{\n\t.reg .u32 lo, hi;\n\tmov.b64 {lo, hi}, %1;\n\tmad.lo.u32 hi, %2, %3, hi;\n\tmov.b64 %0, {lo, hi};\n\t}"
        : "=l"(r)
        : "l"(x), "r"(a), "r"(1u << (W & 31)));
  }
  return r;
}

// x 2^E for an exact int64 x, rounded to nearest (ties to even) once, from
// integer operations alone (leading-zero count, shift, round, exponent
// field); the caller guarantees -1022 <= E <= 960, so every nonzero result
// is a normal number.  `sgn` (0 or the sign bit) flips the sign.
__device__ __forceinline__ double i64_scaled(long long x, int E, unsigned long long sgn) {
  const unsigned long long sx = (unsigned long long)(x >> 63);              // 0 or all ones
  unsigned long long u = ((unsigned long long)x ^ sx) - sx;                  // |x|
  const int lz = __clzll((long long)u);
  u <<= lz;                                                                  // leading one at bit 63
  unsigned long long mant = u >> 11;                                         // 53 bits
  const unsigned long long half = (u >> 10) & 1ull, sticky = (u & 0x3FFull) | (mant & 1ull);
  mant += half & (sticky != 0 ? 1ull : 0ull);
  // (biased exponent - 1) 2^52 + mant: the leading one completes the
  // exponent, and a mantissa rounded up to 2^53 carries into it
  const unsigned long long bits = ((unsigned long long)(1085 - lz + E) << 52) + mant;
  return x == 0 ? 0.0 : __longlong_as_double((long long)((bits) ^ (sgn ^ (sx << 63))));
}

// 32 lanes x EC consecutive TMEM columns (EC = 8 or 16) into registers.
template <int EC>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, uint32_t *r) {
  if constexpr (EC == 16) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
        "[%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
  } else {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
  }
}

// Reads the weight sums a = A, A+1 of EC columns from TMEM (this warp's 32
// lanes; column of weight a at taddr + a ZBN) and adds them into x.
template <int S, int A, int EC>
__device__ __forceinline__ void combine_weights(unsigned long long *x, uint32_t taddr) {
  if constexpr (A < S) {
    constexpr bool two = A + 1 < S;
    uint32_t r0[EC], r1[EC];
    const uint32_t t0 = taddr + (uint32_t)(A * ZBN);
    tmem_ld<EC>(t0, r0);
    if constexpr (two) tmem_ld<EC>(t0 + (uint32_t)ZBN, r1);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    constexpr int w0 = 7 * (S - 1 - A);
#pragma unroll
    for (int j = 0; j < EC; ++j) {
      x[j] = add_shifted<w0>(x[j], __float_as_uint(__uint_as_float(r0[j]) + 12582912.0f));
      if constexpr (two) x[j] = add_shifted<w0 - 7>(x[j], __float_as_uint(__uint_as_float(r1[j]) + 12582912.0f));
    }
    combine_weights<S, A + 2, EC>(x, taddr);
  }
}

// Persistent sliced GEMM.  Work item = (column chunk, 128-row block of the
// real embedding, batch); a CTA takes items blockIdx.x, +gridDim.x, ...  Per
// item the A slices are loaded once, then the chunk's 32-column tiles flow
// through:
//   warp 0 (one thread): TMA of A slices (barrier a_full, freed by a_empty)
//                        and of each tile's B slices (b_full[2] / b_empty[2]);
//   warp 1 (one thread): S(S+1)/2 digit-pair MMAs per tile into accumulator
//                        buffer g % 2 (acc_full[2] / acc_empty[2]);
//   warps 2-5:           epilogue of tile g while tile g+1 is loaded and
//                        multiplied.
// g counts the tiles this CTA has processed; buffer = g % 2, use = g / 2.
constexpr int ZEC = 8;                      // columns per epilogue warp
constexpr int ZEW = 4 * (ZBN / ZEC);        // epilogue warps (4 lane quarters x column groups)
constexpr int ZTHREADS = 64 + 32 * ZEW;     // warp 0 TMA, warp 1 MMA, the rest epilogue

template <class T, int S, bool BETA, bool SPLIT>
__global__ void __maxnreg__(96)
    zgemm_sliced_kernel(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, int m,
                        int n, int batch, int nch, int tpc, const int *__restrict__ sexp, const int *__restrict__ texp, double alpha,
                        T *C, long ldc, long sc, int *gerr) {
  using R = typename cplx_io<T>::R;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  constexpr int NB = zlay<S, SPLIT>::NB;
  unsigned char *sA = base;                 // S x [128][64]
  unsigned char *sB = base + S * ZA_TILE;   // NB x S x [32][64]
  uint64_t *bars = reinterpret_cast<uint64_t *>(base + S * ZA_TILE + NB * S * ZB_TILE);
  uint64_t *a_full = bars, *a_empty = bars + S;           // a_full[t]: slice t landed
  uint64_t *b_full = bars + S + 1, *b_empty = b_full + NB;
  uint64_t *acc_full = b_empty + NB, *acc_empty = acc_full + 2;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_empty + 2);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rows = 2 * m;
  const int nrb = (rows + BM - 1) / BM, nct = (n + ZBN - 1) / ZBN;
  const int items = nch * nrb * batch;
  constexpr uint32_t NCOLS = zlay<S, SPLIT>::COLS;
  constexpr int ACC = zlay<S, SPLIT>::ACC_COLS;

  if (threadIdx.x == 0) {
    for (int t = 0; t < S; ++t) mbar_init(&a_full[t], 1);
    mbar_init(a_empty, 1);
    for (int j = 0; j < NB; ++j) {
      mbar_init(&b_full[j], 1);
      mbar_init(&b_empty[j], 1);
    }
    for (int j = 0; j < 2; ++j) {
      mbar_init(&acc_full[j], 1);
      mbar_init(&acc_empty[j], ZEW);  // one arrival per epilogue warp
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sm_u32(tmem_slot)),
                 "r"(NCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ TMA --
    // B tile g goes to ring stage g % NB once the MMAs of tile g - NB are done
    int g = 0, it_local = 0, last_b = -1;
    bool ok = true;
    for (int item = blockIdx.x; item < items && ok; item += gridDim.x, ++it_local) {
      const int cc = item % nch, rb = (item / nch) % nrb, b = item / (nch * nrb);
      const int ct1 = min(nct, (cc + 1) * tpc);
      if (it_local > 0 && !mbar_wait(a_empty, (it_local - 1) & 1, abort_flag, gerr, 21)) {
        ok = false;
        break;
      }
      for (int t = 0; t < S; ++t) {
        mbar_expect_tx(&a_full[t], ZA_TILE);
        tma_load_3d(sA + t * ZA_TILE, &ta, &a_full[t], 0, rb * BM, t * batch + b);
      }
      for (int ct = cc * tpc; ct < ct1; ++ct, ++g) {
        const int st = g % NB, use = g / NB;
        if (use > 0 && !mbar_wait(&b_empty[st], (use - 1) & 1, abort_flag, gerr, 22)) {
          ok = false;
          break;
        }
        mbar_expect_tx(&b_full[st], S * ZB_TILE);
        for (int u = 0; u < S; ++u)
          tma_load_3d(sB + (st * S + u) * ZB_TILE, &tb, &b_full[st], 0, ct * ZBN, u * batch + b);
        last_b = g;
      }
    }
    // drain the copies this thread issued
    if (it_local > 0)
      for (int t = 0; t < S; ++t) mbar_drain(&a_full[t], (it_local - 1) & 1, gerr, 23);
    for (int gg = (last_b - NB + 1 > 0 ? last_b - NB + 1 : 0); gg <= last_b; ++gg)
      mbar_drain(&b_full[gg % NB], (gg / NB) & 1, gerr, 24);
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------------------ MMA --
    int g = 0, it_local = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < items && ok; item += gridDim.x, ++it_local) {
      const int cc = item % nch;
      const int ct0 = cc * tpc, ct1 = min(nct, ct0 + tpc);
      for (int ct = ct0; ct < ct1; ++ct, ++g) {
        const int st = g % NB, buf = g & 1;
        if (!mbar_wait(&b_full[st], (g / NB) & 1, abort_flag, gerr, 26) ||
            (g >= 2 && !mbar_wait(&acc_empty[buf], ((g >> 1) - 1) & 1, abort_flag, gerr, 27))) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // A slice t times the stacked B slices u = 0 .. S-1-t (contiguous
        // 32-row tiles in shared memory, one operand of N = (S-t) 32 rows)
        // lands in accumulators t+u = t .. S-1, which are contiguous TMEM
        // columns: one MMA per (t, k-step).  t = 0 covers every weight, so
        // its first k-step initialises the buffer.  On an item's first tile
        // each A slice is waited for just before its MMAs.
        const uint32_t dbase = tmem + (uint32_t)(buf * ACC);
        bool issued = false;
        if constexpr (SPLIT) {
          // float split: every part product (t, u), t + u <= S-1, into the
          // one accumulator, the smallest weights first
          if (ct == ct0) {
            for (int t = 0; t < S && ok; ++t)
              if (!mbar_wait(&a_full[t], it_local & 1, abort_flag, gerr, 25)) ok = false;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          }
          if (ok) {
            constexpr uint32_t idesc = idesc_bf16_n(ZBN);
            bool first = true;
#pragma unroll
            for (int w = S - 1; w >= 0; --w)
#pragma unroll
              for (int t = 0; t <= w; ++t) {
                const uint64_t ad = sdesc_sw128(sm_u32(sA + t * ZA_TILE));
                const uint64_t bd = sdesc_sw128(sm_u32(sB + (st * S + (w - t)) * ZB_TILE));
#pragma unroll
                for (int kk = 0; kk < ZK / 16; ++kk)
                  mma_bf16(dbase, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), idesc,
                           (first && kk == 0) ? 0u : 1u);
                first = false;
                issued = true;
              }
          }
        } else {
          const uint64_t bd = sdesc_sw128(sm_u32(sB + st * S * ZB_TILE));
#pragma unroll
          for (int t = 0; t < S; ++t) {
            if (ct == ct0) {
              if (!mbar_wait(&a_full[t], it_local & 1, abort_flag, gerr, 25)) {
                ok = false;
                break;
              }
              asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            }
            const uint32_t idesc = idesc_bf16_n((S - t) * ZBN);
            const uint64_t ad = sdesc_sw128(sm_u32(sA + t * ZA_TILE));
#pragma unroll
            for (int kk = 0; kk < ZK / 16; ++kk)
              mma_bf16(dbase + (uint32_t)(t * ZBN), ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), idesc,
                       (t > 0 || kk > 0) ? 1u : 0u);
            issued = true;
          }
        }
        if (!ok) {
          if (issued) {  // track the MMAs already issued for the drain below
            mma_commit(&acc_full[buf]);
            ++g;
          }
          break;
        }
        mma_commit(&b_empty[st]);
        mma_commit(&acc_full[buf]);
      }
      if (ok) mma_commit(a_empty);  // A slices free once this item's MMAs complete
    }
    // every MMA issued has completed before TMEM is freed
    if (g > 0) mbar_drain(&acc_full[(g - 1) & 1], ((g - 1) >> 1) & 1, gerr, 28);
  } else if (warp >= 2) {
    // ------------------------------------------------------- epilogue --
    // Warp w reads TMEM lanes 32 (w % 4) .. +31 (rows of the tile) and
    // columns g*ZEC .. +ZEC-1 of each tile, g = (w - 2) / 4.  Per tile it
    // waits for the accumulators, copies its S x ZEC sums out of TMEM, frees
    // the buffer for the MMA of tile g + 2, issues the loads of C for its
    // next tile, and then combines and stores this tile.
    // Weight sums s_a (a = 0..S-1, weight 2^{-7(a+2)}) are combined exactly as
    // x = sum_a s_a 2^{7(S-1-a)} in 64-bit integers (|x| < 2^63: |s_0| <= 2^20
    // and |s_a| < 2^22); the entry is alpha sigma_i tau_j 2^{-7(S+1)} x.
    const int q = warp & 3, c0 = ((warp - 2) >> 2) * ZEC;
    const bool neg = alpha < 0.0;
    R cnext[ZEC];
    int tnext = 0;   // lane j: exponent of column col0 + j % ZEC, for shuffles
    int esnext = 0;  // exponent of this lane's row
    // first column of (item, ct) handled by this thread's warp, its row, batch
    auto tile_of = [&](int item, int ct, int &rr, int &b, int &col0) {
      const int rb = (item / nch) % nrb;
      b = item / (nch * nrb);
      rr = rb * BM + q * 32 + lane;
      col0 = ct * ZBN + c0;
    };
    auto load_c = [&](int item, int ct) {
      int rr, b, col0;
      tile_of(item, ct, rr, b, col0);
#pragma unroll
      for (int j = 0; j < ZEC; ++j) cnext[j] = (R)0;
      tnext = (col0 + (lane % ZEC) < n) ? __ldg(texp + (long)b * n + col0 + (lane % ZEC)) : 0;
      esnext = (rr < rows) ? __ldg(sexp + (long)b * rows + rr) : 0;
      if (BETA && rr < rows) {
        const R *crow = reinterpret_cast<const R *>(C + (long)b * sc + (rr >> 1)) + (rr & 1);
#pragma unroll
        for (int j = 0; j < ZEC; ++j)
          if (col0 + j < n) cnext[j] = crow[2L * (col0 + j) * ldc];
      }
    };
    int item = blockIdx.x, ct = 0, ct1 = 0;
    if (item < items) {
      ct = (item % nch) * tpc;
      ct1 = min(nct, ct + tpc);
      load_c(item, ct);
    }
    for (int g = 0; item < items; ++g) {
      const int buf = g & 1, use = g >> 1;
      int okw = 0;
      if (lane == 0) okw = mbar_wait(&acc_full[buf], use & 1, abort_flag, gerr, 29) ? 1 : 0;
      if (__shfl_sync(0xffffffffu, okw, 0) == 0) break;
      __syncwarp();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      unsigned long long x[ZEC];
      uint32_t fs[ZEC];  // split mode: the FP32 sums
      if constexpr (SPLIT) {
        tmem_ld<ZEC>(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * ACC + c0), fs);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      } else {
#pragma unroll
        for (int j = 0; j < ZEC; ++j) x[j] = 0ull - acc_bias<S>();
        combine_weights<S, 0, ZEC>(x, tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * ACC + c0));
      }
      // accumulator buffer free for the MMA of tile g + 2
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sm_u32(&acc_empty[buf])) : "memory");
      // this tile's C entries and scales (loaded during the previous tile),
      // then the loads for the next tile of this CTA, which overlap the work
      // below
      R cur[ZEC];
#pragma unroll
      for (int j = 0; j < ZEC; ++j) cur[j] = cnext[j];
      const int tcur = tnext, escur = esnext;
      int nitem = item, nct0 = ct + 1;
      if (nct0 >= ct1) {
        nitem = item + gridDim.x;
        if (nitem < items) {
          nct0 = (nitem % nch) * tpc;
        }
      }
      if (nitem < items) load_c(nitem, nct0);
      int rr, b, col0;
      tile_of(item, ct, rr, b, col0);
      const bool rv = rr < rows;
      // entry = +-2^{es+et} x (row scale es, column scale et); the warp checks
      // once per tile that every exponent stays in the fast path's range
      const int es = rv ? escur - 7 * (S + 1) : 0;
      const int emn = __reduce_min_sync(0xffffffffu, es) + __reduce_min_sync(0xffffffffu, tcur);
      const int emx = __reduce_max_sync(0xffffffffu, es) + __reduce_max_sync(0xffffffffu, tcur);
      R *crow = reinterpret_cast<R *>(C + (long)b * sc + (rr >> 1)) + (rr & 1);
      int et[ZEC];
#pragma unroll
      for (int j = 0; j < ZEC; ++j) et[j] = __shfl_sync(0xffffffffu, tcur, j);
      const bool full = __all_sync(0xffffffffu, rv) && col0 + ZEC - 1 < n;
      if constexpr (SPLIT) {
        // float split: the accumulator is the product entry itself (FP32)
#pragma unroll
        for (int j = 0; j < ZEC; ++j) {
          const int col = col0 + j;
          if (full || (rv && col < n)) {
            const float v = neg ? -__uint_as_float(fs[j]) : __uint_as_float(fs[j]);
            if constexpr (BETA)
              crow[2L * col * ldc] = (R)((float)cur[j] + v);
            else
              crow[2L * col * ldc] = (R)v;
          }
        }
      } else if constexpr (std::is_same<R, float>::value) {
        // FP32 output: x rounded once to FP32, scaled exactly by +-2^E (a
        // normal power), added to C by one fused multiply-add
        const bool fast = emn >= -126 && emx <= 127;
        const float sg = neg ? -1.0f : 1.0f;
#pragma unroll
        for (int j = 0; j < ZEC; ++j) {
          const int col = col0 + j;
          if (full || (rv && col < n)) {
            const float xf = __ll2float_rn((long long)x[j]);
            const float p2 = sg * (fast ? __int_as_float((es + et[j] + 127) << 23) : ldexpf(1.0f, es + et[j]));
            if constexpr (BETA)
              crow[2L * col * ldc] = fmaf(xf, p2, (float)cur[j]);
            else
              crow[2L * col * ldc] = xf * p2;
          }
        }
      } else {
        // FP64 output: the product entry is rounded once to FP64 (exactly
        // scaled), then added to C with one more rounding
        const bool fast = emn >= -1022 && emx <= 960;
        const unsigned long long sgn = neg ? 0x8000000000000000ull : 0ull;
        if (fast && full) {
          // whole 32 x ZEC block in range: straight-line code, so the ZEC
          // independent conversions interleave.  The integer pipe and the
          // FP64 unit share the conversions: even columns are built with
          // integer operations (leading-zero count, rounding, exponent
          // field) and added to C with one FP64 add, odd columns are
          // converted by the FP64 unit and joined to C by one fused
          // multiply-add (both round twice: the product entry, then the
          // sum); with all of them on the integer pipe it was the busiest.
          double v[ZEC];
#pragma unroll
          for (int j = 0; j < ZEC; ++j) {
            if (j & 1) {
              const double p2 =
                  __longlong_as_double((long long)(((unsigned long long)(es + et[j] + 1023) << 52) ^ sgn));
              v[j] = BETA ? fma(__ll2double_rn((long long)x[j]), p2, (double)cur[j])
                          : __ll2double_rn((long long)x[j]) * p2;
            } else {
              v[j] = i64_scaled((long long)x[j], es + et[j], sgn);
              if constexpr (BETA) v[j] += (double)cur[j];
            }
          }
#pragma unroll
          for (int j = 0; j < ZEC; ++j) crow[2L * (col0 + j) * ldc] = (R)v[j];
        } else {
#pragma unroll
          for (int j = 0; j < ZEC; ++j) {
            const int col = col0 + j;
            if (rv && col < n) {
              double v;
              if (fast) {
                v = i64_scaled((long long)x[j], es + et[j], sgn);
              } else {
                v = ldexp(__ll2double_rn((long long)x[j]), es + et[j]);
                if (neg) v = -v;
              }
              if constexpr (BETA)
                crow[2L * col * ldc] = (R)((double)cur[j] + v);
              else
                crow[2L * col * ldc] = (R)v;
            }
          }
        }
      }
      if (nitem != item) {
        item = nitem;
        if (item < items) {
          ct = nct0;
          ct1 = min(nct, ct + tpc);
        }
      } else {
        ct = nct0;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS) : "memory");
}

// 3-D map over [planes][rows][ZK] bf16 with a box of (ZK, box_rows, 1).
static int make_map_rows(CUtensorMap *map, const void *ptr, long rows, int planes, int box_rows) {
  auto fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled unavailable");
    return -4;
  }
  cuuint64_t dims[3] = {(cuuint64_t)ZK, (cuuint64_t)rows, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)ZK * 2, (cuuint64_t)rows * ZK * 2};
  cuuint32_t box[3] = {(cuuint32_t)ZK, (cuuint32_t)box_rows, 1};
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

template <class T, int S, bool SPLIT>
static int zgemm_sliced_run(cudaStream_t st, char opa, char opb, int m, int n, int k, double alpha, const T *A,
                            long lda, long sa, const T *B, long ldb, long sb, int beta_one, T *C, long ldc, long sc,
                            int batch, void *work, size_t work_bytes, int *gerr) {
  if (k < 1 || k > ZK / 2) {
    set_error("sliced GEMM: k must be in [1, 32]");
    return -4;
  }
  if (alpha != 1.0 && alpha != -1.0) {
    set_error("sliced GEMM: alpha must be +1 or -1");
    return -4;
  }
  const long rows = 2L * m;
  const size_t a_bytes = (size_t)S * batch * rows * ZK * 2, b_bytes = (size_t)S * batch * n * ZK * 2;
  const size_t s_bytes = (size_t)batch * rows * 8, t_bytes = (size_t)batch * n * 8;
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  if (al(a_bytes) + al(b_bytes) + al(s_bytes) + al(t_bytes) > work_bytes) {
    set_error("sliced GEMM: workspace too small");
    return -4;
  }
  char *w = (char *)work;
  __nv_bfloat16 *As = (__nv_bfloat16 *)w;
  __nv_bfloat16 *Bs = (__nv_bfloat16 *)(w + al(a_bytes));
  int *sg = (int *)(w + al(a_bytes) + al(b_bytes));
  int *tg = (int *)(w + al(a_bytes) + al(b_bytes) + al(s_bytes));
  const int sslot = prof_begin(st);
  slice_a_kernel<T, S, SPLIT><<<dim3(ceil_div(m, 8), batch), 256, 0, st>>>(opa, m, k, A, lda, sa, batch, As, sg);
  slice_b_kernel<T, S, SPLIT><<<dim3(ceil_div(n, 8), batch), 256, 0, st>>>(opb, k, n, B, ldb, sb, batch, Bs, tg);
  prof_end(st, sslot, 0.0);
  g_launches.fetch_add(2, std::memory_order_relaxed);
  CUtensorMap ta, tb;
  if (int rc = make_map_rows(&ta, As, rows, S * batch, BM)) return rc;
  if (int rc = make_map_rows(&tb, Bs, n, S * batch, ZBN)) return rc;
  static std::atomic<unsigned long long> attr_done{0};
  if (int rc = once_per_device(attr_done, [&]() -> int {
      GBF_CUDA(cudaFuncSetAttribute(zgemm_sliced_kernel<T, S, true, SPLIT>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, zlay<S, SPLIT>::SMEM));
      GBF_CUDA(cudaFuncSetAttribute(zgemm_sliced_kernel<T, S, false, SPLIT>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, zlay<S, SPLIT>::SMEM));
        return 0;
      }))
    return rc;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // split the columns into chunks until there are about four work items
  // per SM (the A slices are reloaded once per chunk)
  const int base_items = (int)ceil_div(rows, (long)BM) * batch, nct = ceil_div(n, ZBN);
  const int want = std::max(1, std::min(nct, ceil_div(4 * sms, base_items)));
  const int tpc = ceil_div(nct, want), nch = ceil_div(nct, tpc);  // no chunk is empty
  const int items = base_items * nch;
  dim3 grid(std::min(items, sms));
  const int slot = prof_begin(st);
  if (beta_one)
    zgemm_sliced_kernel<T, S, true, SPLIT><<<grid, ZTHREADS, zlay<S, SPLIT>::SMEM, st>>>(ta, tb, m, n, batch, nch, tpc, sg, tg,
                                                                            alpha, C, ldc, sc, gerr);
  else
    zgemm_sliced_kernel<T, S, false, SPLIT><<<grid, ZTHREADS, zlay<S, SPLIT>::SMEM, st>>>(ta, tb, m, n, batch, nch, tpc, sg, tg,
                                                                             alpha, C, ldc, sc, gerr);
  // issued: S(S+1)/2 digit-pair products of 128 x 32 x 64 per (row block, column tile)
  prof_end_tc(st, slot, 8.0 * m * (double)n * k * batch,
              2.0 * BM * ZBN * ZK * (S * (S + 1) / 2) * (double)base_items * nct);
  GBF_LAUNCHED();
  GBF_CUDA(cudaGetLastError());
  return 0;
}

// ===================================================================
// FP32-complex GEMM on the tensor cores, k <= 32 (the shifted LU's trailing
// updates and the blocked triangular solves of the FP32 factors):
//   C = alpha op(A) op(B) + beta C,  C complex FP32, alpha in {+1, -1},
//   beta in {0, 1}.
// Complex operands use the real embedding of the sliced kernels (rows
// 2i = (Re, -Im), 2i+1 = (Im, Re) of op(A) against columns (Re, Im) of
// op(B); K' = 2k <= 64).  Every real entry x is split into two TF32 numbers,
// hi = x rounded to TF32 (11 significant bits) and lo = x - hi rounded to
// TF32, and each product is formed as lo_a hi_b + hi_a lo_b + hi_a hi_b by
// three kind::tf32 MMAs into one FP32 TMEM accumulator ("3xTF32": the
// dropped lo_a lo_b and the rounding of lo leave a relative error of about
// 2^-22 per product, FP32-class).
// The kernel is the persistent layout of zgemm_sliced_kernel: per work item
// (column chunk, 128-row block, batch) the A planes stay resident in shared
// memory (hi and lo, 2 K-chunks of 32 FP32 = 64 KB) while 64-column B tiles
// (32 KB) stream through a 4-deep TMA ring; two 64-column TMEM accumulators
// let the epilogue of tile g (16 warps: 4 lane quarters x 4 groups of 16
// columns) overlap the MMAs of tile g + 1; C of the next tile is prefetched.
// ===================================================================
constexpr int TF_BN = 64;                         // output columns per tile (MMA N)
constexpr int TF_KC = 32;                         // FP32 per K-chunk (one 128-byte swizzle row)
constexpr int TF_A_BOX = BM * TF_KC * 4;          // 16 KB: one (plane, chunk) of an A tile
constexpr int TF_B_BOX = TF_BN * TF_KC * 4;       // 8 KB: one (plane, chunk) of a B tile
constexpr int TF_A_TILE = 4 * TF_A_BOX;           // hi/lo x 2 chunks
constexpr int TF_B_TILE = 4 * TF_B_BOX;
constexpr int TF_NB = 4;                          // B ring depth
constexpr int TF_NB_TC = 2;                       // B ring depth with the C tiles staged in shared memory
constexpr int TF_C_TILE = BM * TF_BN * 4;         // 32 KB: one C tile (128 embedded rows x 64 columns, FP32)
constexpr int TF_SMEM = TF_A_TILE + TF_NB * TF_B_TILE + 1024 + 256;
constexpr int TF_NC = 3;                          // C tile buffers (staged C)
constexpr int TF_SMEM_TC = TF_A_TILE + TF_NB_TC * TF_B_TILE + TF_NC * TF_C_TILE + 1024 + 256;
constexpr int TF_EC = 16;                         // columns per epilogue warp
constexpr int TF_EW = 4 * (TF_BN / TF_EC);        // epilogue warps
constexpr int TF_THREADS = 64 + 32 * TF_EW;
constexpr uint32_t TF_COLS = 2 * TF_BN;           // TMEM columns (two accumulators)

// Instruction descriptor, kind::tf32: FP32 accumulate, TF32 A and B, both
// K-major, M = 128, N = TF_BN.
__host__ __device__ constexpr uint32_t idesc_tf32() {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TF_BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
}

// x rounded to the nearest TF32 value (ties away from zero): the low 13
// mantissa bits cleared after adding half of their range.  Finite inputs.
__device__ __forceinline__ float tf32_rn(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}
__device__ __forceinline__ void tf32_split(float x, float &hi, float &lo) {
  hi = tf32_rn(x);
  lo = tf32_rn(x - hi);
}

// Planes layout [plane (0 hi, 1 lo)][batch][chunk][rows][32] FP32.
__device__ __forceinline__ long tf_idx(int plane, int b, int batch, int q, long rows, long r) {
  return ((((long)plane * batch + b) * 2 + (q >> 5)) * rows + r) * TF_KC + (q & 31);
}

// A side: one warp per complex row i of op(A) (m x k), lane p < k holds
// element (i, p); writes embedded rows 2i, 2i+1 (positions 2k..63 zero).
template <class T>
__device__ __forceinline__ void tf32_split_a(int i, int b, char opa, int m, int k, const T *A, long lda, long sa,
                                             int batch, float *out) {
  const int p = threadIdx.x & 31;
  if (i >= m) return;  // warp-uniform
  const T *Ab = A + (long)b * sa;
  float re = 0.f, im = 0.f;
  if (p < k) {
    const T a = (opa == 'N') ? Ab[i + (long)p * lda] : Ab[p + (long)i * lda];
    re = (float)a.x;
    im = (opa == 'C') ? -(float)a.y : (float)a.y;
  }
  const long rows = 2L * m, r0 = 2L * i, r1 = r0 + 1;
  float rh, rl, ih, il;
  tf32_split(re, rh, rl);
  tf32_split(im, ih, il);
  if (p < k) {
    out[tf_idx(0, b, batch, p, rows, r0)] = rh;
    out[tf_idx(1, b, batch, p, rows, r0)] = rl;
    out[tf_idx(0, b, batch, k + p, rows, r0)] = -ih;
    out[tf_idx(1, b, batch, k + p, rows, r0)] = -il;
    out[tf_idx(0, b, batch, p, rows, r1)] = ih;
    out[tf_idx(1, b, batch, p, rows, r1)] = il;
    out[tf_idx(0, b, batch, k + p, rows, r1)] = rh;
    out[tf_idx(1, b, batch, k + p, rows, r1)] = rl;
  }
  for (int q = 2 * k + p; q < 2 * TF_KC; q += 32)
    for (int pl = 0; pl < 2; ++pl) {
      out[tf_idx(pl, b, batch, q, rows, r0)] = 0.f;
      out[tf_idx(pl, b, batch, q, rows, r1)] = 0.f;
    }
}

// B side: one warp per column c of op(B) (k x n), lane p < k holds element
// (p, c); writes the column (Re ; Im) as one K-major row.
template <class T>
__device__ __forceinline__ void tf32_split_b(int c, int b, char opb, int k, int n, const T *B, long ldb, long sb,
                                             int batch, float *out) {
  const int p = threadIdx.x & 31;
  if (c >= n) return;  // warp-uniform
  const T *Bb = B + (long)b * sb;
  float re = 0.f, im = 0.f;
  if (p < k) {
    const T v = (opb == 'N') ? Bb[p + (long)c * ldb] : Bb[c + (long)p * ldb];
    re = (float)v.x;
    im = (opb == 'C') ? -(float)v.y : (float)v.y;
  }
  float rh, rl, ih, il;
  tf32_split(re, rh, rl);
  tf32_split(im, ih, il);
  if (p < k) {
    out[tf_idx(0, b, batch, p, n, c)] = rh;
    out[tf_idx(1, b, batch, p, n, c)] = rl;
    out[tf_idx(0, b, batch, k + p, n, c)] = ih;
    out[tf_idx(1, b, batch, k + p, n, c)] = il;
  }
  for (int q = 2 * k + p; q < 2 * TF_KC; q += 32) {
    out[tf_idx(0, b, batch, q, n, c)] = 0.f;
    out[tf_idx(1, b, batch, q, n, c)] = 0.f;
  }
}

// Both operands in one launch: blocks [0, ablocks) split rows of op(A),
// the rest columns of op(B); 8 warps per block, blockIdx.y = batch.
template <class T>
__global__ void tf32_split_kernel(char opa, char opb, int m, int n, int k, const T *A, long lda, long sa,
                                  const T *B, long ldb, long sb, int batch, int ablocks, float *Ap, float *Bp) {
  const int w = threadIdx.x >> 5;
  if ((int)blockIdx.x < ablocks)
    tf32_split_a<T>(blockIdx.x * 8 + w, blockIdx.y, opa, m, k, A, lda, sa, batch, Ap);
  else
    tf32_split_b<T>((blockIdx.x - ablocks) * 8 + w, blockIdx.y, opb, k, n, B, ldb, sb, batch, Bp);
}

template <bool BETA, bool TC>
__global__ void __launch_bounds__(TF_THREADS, 1)
    ctf32_kernel(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
                 const __grid_constant__ CUtensorMap tcm, int m, int n, int batch, int nch, int tpc, float alpha,
                 cf *C, long ldc, long sc, int *gerr) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  constexpr int NBT = TC ? TF_NB_TC : TF_NB;
  unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *sA = base;               // [plane][chunk][128][32] FP32
  unsigned char *sB = base + TF_A_TILE;   // NBT x [plane][chunk][64][32]
  float *sC = reinterpret_cast<float *>(base + TF_A_TILE + NBT * TF_B_TILE);  // TC: TF_NC x [64 cols][128 rows]
  uint64_t *bars = reinterpret_cast<uint64_t *>(base + TF_A_TILE + NBT * TF_B_TILE + (TC ? TF_NC * TF_C_TILE : 0));
  uint64_t *a_full = bars, *a_empty = bars + 1;
  uint64_t *b_full = bars + 2, *b_empty = b_full + NBT;
  uint64_t *acc_full = b_empty + NBT, *acc_empty = acc_full + 2;
  uint64_t *c_full = acc_empty + 2, *c_empty = c_full + TF_NC;  // TC: C tile landed / stored out of the buffer
  uint64_t *epi_done = c_empty + TF_NC;                         // TC: all epilogue warps wrote the tile
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(epi_done + TF_NC);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rows = 2 * m;
  const int nrb = (rows + BM - 1) / BM, nct = (n + TF_BN - 1) / TF_BN;
  const int items = nch * nrb * batch;

  if (threadIdx.x == 0) {
    mbar_init(a_full, 1);
    mbar_init(a_empty, 1);
    for (int j = 0; j < NBT; ++j) {
      mbar_init(&b_full[j], 1);
      mbar_init(&b_empty[j], 1);
    }
    for (int j = 0; j < 2; ++j) {
      mbar_init(&acc_full[j], 1);
      mbar_init(&acc_empty[j], TF_EW);  // one arrival per epilogue warp
    }
    for (int j = 0; j < TF_NC; ++j) {
      mbar_init(&c_full[j], 1);
      mbar_init(&c_empty[j], 1);
      mbar_init(&epi_done[j], TF_EW);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sm_u32(tmem_slot)),
                 "r"(TF_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ TMA --
    int g = 0, it_local = 0, last_b = -1, last_c = -1;
    bool ok = true;
    for (int item = blockIdx.x; item < items && ok; item += gridDim.x, ++it_local) {
      const int cc = item % nch, rb = (item / nch) % nrb, b = item / (nch * nrb);
      const int ct1 = min(nct, (cc + 1) * tpc);
      if (it_local > 0 && !mbar_wait(a_empty, (it_local - 1) & 1, abort_flag, gerr, 41)) {
        ok = false;
        break;
      }
      mbar_expect_tx(a_full, TF_A_TILE);
      for (int pc = 0; pc < 4; ++pc)  // (plane, chunk) = (pc / 2, pc % 2)
        tma_load_3d(sA + pc * TF_A_BOX, &ta, a_full, 0, rb * BM, ((pc >> 1) * batch + b) * 2 + (pc & 1));
      for (int ct = cc * tpc; ct < ct1; ++ct, ++g) {
        const int st = g % NBT, use = g / NBT;
        if (use > 0 && !mbar_wait(&b_empty[st], (use - 1) & 1, abort_flag, gerr, 42)) {
          ok = false;
          break;
        }
        mbar_expect_tx(&b_full[st], TF_B_TILE);
        for (int pc = 0; pc < 4; ++pc)
          tma_load_3d(sB + st * TF_B_TILE + pc * TF_B_BOX, &tb, &b_full[st], 0, ct * TF_BN,
                      ((pc >> 1) * batch + b) * 2 + (pc & 1));
        last_b = g;
        if (TC && BETA) {  // C tile g into buffer g % TF_NC once the store of tile g - TF_NC has read it
          const int cb = g % TF_NC;
          if (g >= TF_NC && !mbar_wait(&c_empty[cb], ((g / TF_NC) - 1) & 1, abort_flag, gerr, 50)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&c_full[cb], TF_C_TILE);
          tma_load_3d(sC + cb * (TF_C_TILE / 4), &tcm, &c_full[cb], rb * BM, ct * TF_BN, b);
          last_c = g;
        }
      }
    }
    if (it_local > 0) mbar_drain(a_full, (it_local - 1) & 1, gerr, 43);
    for (int gg = (last_b - NBT + 1 > 0 ? last_b - NBT + 1 : 0); gg <= last_b; ++gg)
      mbar_drain(&b_full[gg % NBT], (gg / NBT) & 1, gerr, 44);
    for (int gg = (last_c - TF_NC + 1 > 0 ? last_c - TF_NC + 1 : 0); gg <= last_c; ++gg)
      mbar_drain(&c_full[gg % TF_NC], (gg / TF_NC) & 1, gerr, 51);
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------------------ MMA --
    constexpr uint32_t idesc = idesc_tf32();
    int g = 0, it_local = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < items && ok; item += gridDim.x, ++it_local) {
      const int cc = item % nch;
      const int ct0 = cc * tpc, ct1 = min(nct, ct0 + tpc);
      for (int ct = ct0; ct < ct1; ++ct, ++g) {
        const int st = g % NBT, buf = g & 1;
        if ((ct == ct0 && !mbar_wait(a_full, it_local & 1, abort_flag, gerr, 45)) ||
            !mbar_wait(&b_full[st], (g / NBT) & 1, abort_flag, gerr, 46) ||
            (g >= 2 && !mbar_wait(&acc_empty[buf], ((g >> 1) - 1) & 1, abort_flag, gerr, 47))) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + (uint32_t)(buf * TF_BN);
        const unsigned char *sb = sB + st * TF_B_TILE;
        // (a plane, b plane): lo hi, hi lo, then hi hi (smaller terms first)
#pragma unroll
        for (int pr = 0; pr < 3; ++pr) {
          const int pa = (pr == 0) ? 1 : 0, pb = (pr == 1) ? 1 : 0;
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const uint64_t ad = sdesc_sw128(sm_u32(sA + (pa * 2 + c) * TF_A_BOX));
            const uint64_t bd = sdesc_sw128(sm_u32(sb + (pb * 2 + c) * TF_B_BOX));
#pragma unroll
            for (int kk = 0; kk < TF_KC / 8; ++kk)  // 8 TF32 (32 bytes) per MMA
              mma_tf32(d, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), idesc,
                       (pr == 0 && c == 0 && kk == 0) ? 0u : 1u);
          }
        }
        mma_commit(&b_empty[st]);
        mma_commit(&acc_full[buf]);
      }
      if (ok) mma_commit(a_empty);
    }
    if (g > 0) mbar_drain(&acc_full[(g - 1) & 1], ((g - 1) >> 1) & 1, gerr, 48);
  } else if (TC && warp >= 2) {
    // ------------------------------------------- epilogue, C staged --
    // The C tile (128 embedded rows x 64 columns, [column][row] FP32) is in
    // shared memory buffer g % TF_NC; warp w updates rows 32 (w % 4) .. +31
    // of columns c0 .. c0 + 15 in place, then arrives on epi_done; thread 0
    // of warp 2 waits for all 16 warps, stores the tile with one bulk tensor
    // copy and frees the buffer for the load of tile g + TF_NC once the copy
    // has read it.
    const int q = warp & 3, c0 = ((warp - 2) >> 2) * TF_EC;
    const bool issuer = (warp == 2 && lane == 0);
    int item = blockIdx.x, ct = 0, ct1 = 0;
    if (item < items) {
      ct = (item % nch) * tpc;
      ct1 = min(nct, ct + tpc);
    }
    for (int g = 0; item < items; ++g) {
      const int buf = g & 1, use = g >> 1, cb = g % TF_NC, cuse = g / TF_NC;
      int okw = 0;
      if (lane == 0)
        okw = (mbar_wait(&acc_full[buf], use & 1, abort_flag, gerr, 49) &&
               (!BETA || mbar_wait(&c_full[cb], cuse & 1, abort_flag, gerr, 52)))
                  ? 1
                  : 0;
      if (__shfl_sync(0xffffffffu, okw, 0) == 0) break;
      __syncwarp();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      uint32_t acc[TF_EC];
      tmem_ld<TF_EC>(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * TF_BN + c0), acc);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sm_u32(&acc_empty[buf])) : "memory");
      const int rb = (item / nch) % nrb, b = item / (nch * nrb);
      float *tile = sC + cb * (TF_C_TILE / 4) + q * 32 + lane;
#pragma unroll
      for (int j = 0; j < TF_EC; ++j) {
        const float v = __uint_as_float(acc[j]);
        float *cp = tile + (c0 + j) * BM;
        *cp = BETA ? fmaf(alpha, v, *cp) : alpha * v;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sm_u32(&epi_done[cb])) : "memory");
      int stored = 1;
      if (issuer) stored = mbar_wait(&epi_done[cb], cuse & 1, abort_flag, gerr, 53) ? 1 : 0;
      if (issuer && stored) {
        asm volatile(
            "cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                reinterpret_cast<uint64_t>(&tcm)),
            "r"(sm_u32(sC + cb * (TF_C_TILE / 4))), "r"(rb * BM), "r"(ct * TF_BN), "r"(b)
            : "memory");
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sm_u32(&c_empty[cb])) : "memory");
      }
      if (__shfl_sync(0xffffffffu, stored, 0) == 0) break;  // warp-uniform (lane 0 decides)
      int nitem = item, nct0 = ct + 1;
      if (nct0 >= ct1) {
        nitem = item + gridDim.x;
        if (nitem < items) nct0 = (nitem % nch) * tpc;
      }
      if (nitem != item) {
        item = nitem;
        if (item < items) {
          ct = nct0;
          ct1 = min(nct, ct + tpc);
        }
      } else {
        ct = nct0;
      }
    }
    if (issuer) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");  // every store written
  } else if (!TC && warp >= 2) {
    // ------------------------------------------------------- epilogue --
    // Warp w: TMEM lanes 32 (w % 4) .. +31 (embedded rows), columns
    // c0 .. c0 + 15 of each tile, c0 = 16 ((w - 2) / 4).  Embedded row rr is
    // the real (rr even) or imaginary (rr odd) part of complex row rr / 2.
    const int q = warp & 3, c0 = ((warp - 2) >> 2) * TF_EC;
    float cnext[TF_EC];
    auto load_c = [&](int item, int ct) {
      const int rb = (item / nch) % nrb, b = item / (nch * nrb);
      const int rr = rb * BM + q * 32 + lane, col0 = ct * TF_BN + c0;
#pragma unroll
      for (int j = 0; j < TF_EC; ++j) cnext[j] = 0.f;
      if (BETA && rr < rows) {
        const float *crow = reinterpret_cast<const float *>(C + (long)b * sc + (rr >> 1)) + (rr & 1);
#pragma unroll
        for (int j = 0; j < TF_EC; ++j)
          if (col0 + j < n) cnext[j] = crow[2L * (col0 + j) * ldc];
      }
    };
    int item = blockIdx.x, ct = 0, ct1 = 0;
    if (item < items) {
      ct = (item % nch) * tpc;
      ct1 = min(nct, ct + tpc);
      load_c(item, ct);
    }
    for (int g = 0; item < items; ++g) {
      const int buf = g & 1, use = g >> 1;
      int okw = 0;
      if (lane == 0) okw = mbar_wait(&acc_full[buf], use & 1, abort_flag, gerr, 49) ? 1 : 0;
      if (__shfl_sync(0xffffffffu, okw, 0) == 0) break;
      __syncwarp();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      uint32_t acc[TF_EC];
      tmem_ld<TF_EC>(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * TF_BN + c0), acc);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sm_u32(&acc_empty[buf])) : "memory");
      float cur[TF_EC];
#pragma unroll
      for (int j = 0; j < TF_EC; ++j) cur[j] = cnext[j];
      int nitem = item, nct0 = ct + 1;
      if (nct0 >= ct1) {
        nitem = item + gridDim.x;
        if (nitem < items) nct0 = (nitem % nch) * tpc;
      }
      if (nitem < items) load_c(nitem, nct0);
      const int rb = (item / nch) % nrb, b = item / (nch * nrb);
      const int rr = rb * BM + q * 32 + lane, col0 = ct * TF_BN + c0;
      if (rr < rows) {
        float *crow = reinterpret_cast<float *>(C + (long)b * sc + (rr >> 1)) + (rr & 1);
#pragma unroll
        for (int j = 0; j < TF_EC; ++j)
          if (col0 + j < n) {
            const float v = __uint_as_float(acc[j]);
            crow[2L * (col0 + j) * ldc] = BETA ? fmaf(alpha, v, cur[j]) : alpha * v;
          }
      }
      if (nitem != item) {
        item = nitem;
        if (item < items) {
          ct = nct0;
          ct1 = min(nct, ct + tpc);
        }
      } else {
        ct = nct0;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TF_COLS) : "memory");
}

// 3-D map over [planes x batch x chunks][rows][32] FP32 with a box of
// (32, box_rows, 1), 128-byte swizzle.
static int make_map_tf32(CUtensorMap *map, const void *ptr, long rows, int planes, int box_rows) {
  auto fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled unavailable");
    return -4;
  }
  cuuint64_t dims[3] = {(cuuint64_t)TF_KC, (cuuint64_t)rows, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)TF_KC * 4, (cuuint64_t)rows * TF_KC * 4};
  cuuint32_t box[3] = {(cuuint32_t)TF_KC, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(ptr), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
    return -4;
  }
  return 0;
}

// 3-D map over C (complex FP32, column-major, ldc, batch stride sc) seen as
// FP32 [batch][n columns][2m embedded rows], box (128 rows, 64 columns, 1),
// no swizzle.
static int make_map_ctile(CUtensorMap *map, const cf *C, long rows, int n, int batch, long ldc, long sc) {
  auto fn = encode_fn();
  if (!fn) return -4;
  cuuint64_t dims[3] = {(cuuint64_t)rows, (cuuint64_t)n, (cuuint64_t)batch};
  cuuint64_t strides[2] = {(cuuint64_t)ldc * 8, (cuuint64_t)(batch > 1 ? sc : (long)ldc * n) * 8};
  cuuint32_t box[3] = {(cuuint32_t)BM, (cuuint32_t)TF_BN, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<cf *>(C), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -4;
}

static size_t ctf32_work(int m, int n, int batch) {
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  return al((size_t)2 * batch * 2 * (2L * m) * TF_KC * 4) + al((size_t)2 * batch * 2 * (long)n * TF_KC * 4);
}

static int ctf32_run(cudaStream_t st, char opa, char opb, int m, int n, int k, double alpha, const cf *A, long lda,
                     long sa, const cf *B, long ldb, long sb, int beta_one, cf *C, long ldc, long sc, int batch,
                     void *work, size_t work_bytes, int *gerr) {
  if (k < 1 || k > TF_KC) {
    set_error("3xTF32 GEMM: k must be in [1, 32]");
    return -4;
  }
  if (alpha != 1.0 && alpha != -1.0) {
    set_error("3xTF32 GEMM: alpha must be +1 or -1");
    return -4;
  }
  const long rows = 2L * m;
  if (ctf32_work(m, n, batch) > work_bytes) {
    set_error("3xTF32 GEMM: workspace too small");
    return -4;
  }
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  float *Ap = (float *)work;
  float *Bp = (float *)((char *)work + al((size_t)2 * batch * 2 * rows * TF_KC * 4));
  const int sslot = prof_begin(st);
  const int ablocks = ceil_div(m, 8);
  tf32_split_kernel<cf><<<dim3(ablocks + ceil_div(n, 8), batch), 256, 0, st>>>(opa, opb, m, n, k, A, lda, sa, B, ldb,
                                                                              sb, batch, ablocks, Ap, Bp);
  prof_end(st, sslot, 0.0);
  GBF_LAUNCHED();
  CUtensorMap ta, tb;
  if (int rc = make_map_tf32(&ta, Ap, rows, 4 * batch, BM)) return rc;
  if (int rc = make_map_tf32(&tb, Bp, n, 4 * batch, TF_BN)) return rc;
  static std::atomic<unsigned long long> attr_done{0};
  if (int rc = once_per_device(attr_done, [&]() -> int {
        GBF_CUDA(cudaFuncSetAttribute(ctf32_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      TF_SMEM));
        GBF_CUDA(cudaFuncSetAttribute(ctf32_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      TF_SMEM));
        GBF_CUDA(cudaFuncSetAttribute(ctf32_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      TF_SMEM_TC));
        return 0;
      }))
    return rc;
  // C staged through shared memory by bulk tensor copies when beta = 1 and
  // its layout meets the copies' 16-byte rules (start, column and batch
  // strides); otherwise the epilogue reads and writes C directly
  CUtensorMap tcm;
  const bool staged = beta_one && ((uintptr_t)C % 16 == 0) && (ldc % 2 == 0) && (batch == 1 || sc % 2 == 0) &&
                      make_map_ctile(&tcm, C, rows, n, batch, ldc, sc) == 0;
  if (!staged) tcm = ta;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int base_items = (int)ceil_div(rows, (long)BM) * batch, nct = ceil_div(n, TF_BN);
  const int want = std::max(1, std::min(nct, ceil_div(4 * sms, base_items)));
  const int tpc = ceil_div(nct, want), nch = ceil_div(nct, tpc);
  const int items = base_items * nch;
  dim3 grid(std::min(items, sms));
  const int slot = prof_begin(st);
  if (staged)
    ctf32_kernel<true, true><<<grid, TF_THREADS, TF_SMEM_TC, st>>>(ta, tb, tcm, m, n, batch, nch, tpc, (float)alpha,
                                                                   C, ldc, sc, gerr);
  else if (beta_one)
    ctf32_kernel<true, false><<<grid, TF_THREADS, TF_SMEM, st>>>(ta, tb, tcm, m, n, batch, nch, tpc, (float)alpha, C,
                                                                 ldc, sc, gerr);
  else
    ctf32_kernel<false, false><<<grid, TF_THREADS, TF_SMEM, st>>>(ta, tb, tcm, m, n, batch, nch, tpc, (float)alpha,
                                                                  C, ldc, sc, gerr);
  prof_end(st, slot, 8.0 * m * (double)n * k * batch);
  GBF_LAUNCHED();
  GBF_CUDA(cudaGetLastError());
  return 0;
}

// ===================================================================
// 3xTF32 complex FP32 GEMM for any k (the FP32 factors' solves and updates
// with large K):  C = alpha op(A) op(B) + beta C, alpha = +-1, beta 0 / 1.
// Operands are split once per call into TF32 planes hi = rn(x), lo =
// rn(x - hi) of the real embedding (row 2i = (Re, -Im), 2i+1 = (Im, Re) of
// op(A) against column (Re, Im) of op(B)), laid out K-major in chunks of 32
// FP32 with the real parts in chunks [0, nk) and the imaginary parts in
// chunks [nk, 2 nk) (k padded to nk = ceil(k / 32) chunks).  Work item =
// (128 embedded rows, 128 columns, batch), column tile fastest so that the
// CTAs working at the same time share their A rows in L2; per K chunk one
// stage of the TMA ring holds A hi, A lo (16 KB each) and B hi, B lo (16 KB
// each) and the MMA thread issues lo hi, hi lo, hi hi (4 kind::tf32 MMAs of
// K = 8 each) into an FP32 TMEM accumulator.  The tensor cores' FP32
// accumulation loses accuracy roughly in proportion to the number of terms
// (measured: 1e-6 relative at K = 64, 1e-4 at K = 8192), so an accumulator
// covers only one group of TK_KG chunks (128 real positions); the epilogue
// adds each group's sums into registers with FP32 round-to-nearest adds and
// writes C once per item.  Two TMEM buffers (2 x 128 columns) let the
// epilogue drain one group while the MMAs fill the next.  16 epilogue
// warps: 4 lane quarters x 4 groups of 32 columns.  Bounded waits as in the
// other kernels.
// ===================================================================
// Where the A planes of a call sit in a stored plane array: rows row0 ..
// (embedded), K chunks c0 .. of the real parts and nkh + c0 .. of the
// imaginary parts, nodes b0 .. of bt; the planes of one call split on the
// spot are the special case row0 = c0 = b0 = 0, nkh = nk, bt = batch.
struct APlanes {
  int row0, c0, nkh, bt, b0;
};

constexpr int TK_BN = 128;
constexpr int TK_BOX = BM * TF_KC * 4;               // 16 KB: one plane of one chunk (A, or B with 128 rows)
constexpr int TK_STAGE = 4 * TK_BOX;                 // A hi, A lo, B hi, B lo
constexpr int TK_NS = 3;
constexpr int TK_SMEM = TK_NS * TK_STAGE + 1024 + 256;
constexpr int TK_EC = 32;
constexpr int TK_KG = 4;                             // K chunks per TMEM accumulation group
constexpr int TK_EW = 4 * (TK_BN / TK_EC);
constexpr int TK_THREADS = 64 + 32 * TK_EW;
constexpr uint32_t TK_COLS = 2 * TK_BN;

__host__ __device__ constexpr uint32_t idesc_tf32_n(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

// Plane layout [plane (0 hi, 1 lo)][batch][chunk][rows][32] FP32.
__device__ __forceinline__ long tk_idx(int plane, int b, int batch, int nch, int ch, long rows, long r, int kk) {
  return (((((long)plane * batch + b) * nch + ch) * rows + r) * TF_KC) + kk;
}

// One block per 32 x 32 tile of op(X) (rows i0.., K positions p0..) of
// batch blockIdx.z: read coalesced along the stored dimension through
// shared memory, write the hi / lo planes of the embedded rows.  asA: rows
// of op(A) (two embedded rows each), else columns of op(B).
template <class T>
__global__ void __launch_bounds__(256) tf32k_split_kernel(int asA, char op, int rows, int k, int nk, const T *X, long ld,
                                                          long sx, int batch, float *out) {
  __shared__ float sre[32][33], sim[32][33];
  const int i0 = blockIdx.x * 32, p0 = blockIdx.y * 32, b = blockIdx.z;
  const T *Xb = X + (long)b * sx;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 rows of 32 threads
  // op(X)(i, p): op 'N' -> X[i + p ld] (asA) / X[p + i ld] (B side, column i
  // of op(B) = column i of X); 'T' / 'C' the transposed access
  const bool i_fast = asA ? (op == 'N') : (op != 'N');
  for (int r = ty; r < 32; r += 8) {
    const int a = i_fast ? (i0 + tx) : (i0 + r);  // index i
    const int p = i_fast ? (p0 + r) : (p0 + tx);  // index p
    float re = 0.f, im = 0.f;
    if (a < rows && p < k) {
      const bool trans = asA ? (op != 'N') : (op == 'N');
      const T v = trans ? Xb[p + (long)a * ld] : Xb[a + (long)p * ld];
      re = (float)v.x;
      im = (op == 'C') ? -(float)v.y : (float)v.y;
    }
    const int li = a - i0, lp = p - p0;
    sre[li][lp] = re;
    sim[li][lp] = im;
  }
  __syncthreads();
  const int ch = p0 / TF_KC;
  const long orows = asA ? 2L * rows : (long)rows;
  for (int r = ty; r < 32; r += 8) {
    const int i = i0 + r;
    if (i >= rows) continue;
    float rh, rl, ih, il;
    tf32_split(sre[r][tx], rh, rl);
    tf32_split(sim[r][tx], ih, il);
    if (asA) {
      const long r0 = 2L * i, r1 = r0 + 1;
      out[tk_idx(0, b, batch, 2 * nk, ch, orows, r0, tx)] = rh;
      out[tk_idx(1, b, batch, 2 * nk, ch, orows, r0, tx)] = rl;
      out[tk_idx(0, b, batch, 2 * nk, nk + ch, orows, r0, tx)] = -ih;
      out[tk_idx(1, b, batch, 2 * nk, nk + ch, orows, r0, tx)] = -il;
      out[tk_idx(0, b, batch, 2 * nk, ch, orows, r1, tx)] = ih;
      out[tk_idx(1, b, batch, 2 * nk, ch, orows, r1, tx)] = il;
      out[tk_idx(0, b, batch, 2 * nk, nk + ch, orows, r1, tx)] = rh;
      out[tk_idx(1, b, batch, 2 * nk, nk + ch, orows, r1, tx)] = rl;
    } else {
      out[tk_idx(0, b, batch, 2 * nk, ch, orows, i, tx)] = rh;
      out[tk_idx(1, b, batch, 2 * nk, ch, orows, i, tx)] = rl;
      out[tk_idx(0, b, batch, 2 * nk, nk + ch, orows, i, tx)] = ih;
      out[tk_idx(1, b, batch, 2 * nk, nk + ch, orows, i, tx)] = il;
    }
  }
}

template <bool BETA>
__global__ void __launch_bounds__(TK_THREADS, 1)
    ctf32k_kernel(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, int m, int n,
                  int batch, int nk, float alpha, cf *C, long ldc, long sc, int *gerr, APlanes ap) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t *bars = reinterpret_cast<uint64_t *>(base + TK_NS * TK_STAGE);
  uint64_t *full = bars, *empty = bars + TK_NS;
  uint64_t *acc_full = empty + TK_NS, *acc_empty = acc_full + 2;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_empty + 2);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rows = 2 * m, nch = 2 * nk;
  const int nrb = (rows + BM - 1) / BM, nct = (n + TK_BN - 1) / TK_BN;
  const int items = nct * nrb * batch;

  if (threadIdx.x == 0) {
    for (int j = 0; j < TK_NS; ++j) {
      mbar_init(&full[j], 1);
      mbar_init(&empty[j], 1);
    }
    for (int j = 0; j < 2; ++j) {
      mbar_init(&acc_full[j], 1);
      mbar_init(&acc_empty[j], TK_EW);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sm_u32(tmem_slot)),
                 "r"(TK_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ TMA --
    int g = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < items && ok; item += gridDim.x) {
      const int ct = item % nct, rb = (item / nct) % nrb, b = item / (nct * nrb);
      for (int ch = 0; ch < nch; ++ch, ++g) {
        const int s = g % TK_NS, use = g / TK_NS;
        if (use > 0 && !mbar_wait(&empty[s], (use - 1) & 1, abort_flag, gerr, 61)) {
          ok = false;
          break;
        }
        unsigned char *st = base + s * TK_STAGE;
        mbar_expect_tx(&full[s], TK_STAGE);
        const int ach = ch < nk ? ap.c0 + ch : ap.nkh + ap.c0 + (ch - nk);  // chunk in the stored A planes
        for (int pl = 0; pl < 2; ++pl) {
          tma_load_3d(st + pl * TK_BOX, &ta, &full[s], 0, ap.row0 + rb * BM, (pl * ap.bt + ap.b0 + b) * 2 * ap.nkh + ach);
          tma_load_3d(st + (2 + pl) * TK_BOX, &tb, &full[s], 0, ct * TK_BN, (pl * batch + b) * nch + ch);
        }
      }
    }
    for (int gg = (g - TK_NS > 0 ? g - TK_NS : 0); gg < g; ++gg) mbar_drain(&full[gg % TK_NS], (gg / TK_NS) & 1, gerr, 62);
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------------------ MMA --
    constexpr uint32_t idesc = idesc_tf32_n(TK_BN);
    int g = 0, gq = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < items && ok; item += gridDim.x) {
      for (int c0 = 0; c0 < nch && ok; c0 += TK_KG, ++gq) {
        const int buf = gq & 1;
        if (gq >= 2 && !mbar_wait(&acc_empty[buf], ((gq >> 1) - 1) & 1, abort_flag, gerr, 63)) {
          ok = false;
          break;
        }
        const uint32_t d = tmem + (uint32_t)(buf * TK_BN);
        const int c1 = min(nch, c0 + TK_KG);
        for (int ch = c0; ch < c1; ++ch, ++g) {
          const int s = g % TK_NS;
          if (!mbar_wait(&full[s], (g / TK_NS) & 1, abort_flag, gerr, 64)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const unsigned char *st = base + s * TK_STAGE;
          // (a plane, b plane): lo hi, hi lo, hi hi
#pragma unroll
          for (int pr = 0; pr < 3; ++pr) {
            const int pa = (pr == 0) ? 1 : 0, pb = (pr == 1) ? 1 : 0;
            const uint64_t ad = sdesc_sw128(sm_u32(st + pa * TK_BOX));
            const uint64_t bd = sdesc_sw128(sm_u32(st + (2 + pb) * TK_BOX));
#pragma unroll
            for (int kk = 0; kk < TF_KC / 8; ++kk)
              mma_tf32(d, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), idesc,
                       (ch == c0 && pr == 0 && kk == 0) ? 0u : 1u);
          }
          mma_commit(&empty[s]);
        }
        if (ok) mma_commit(&acc_full[buf]);
      }
    }
    if (gq > 0) mbar_drain(&acc_full[(gq - 1) & 1], ((gq - 1) >> 1) & 1, gerr, 65);
  } else if (warp >= 2) {
    // ------------------------------------------------------- epilogue --
    const int q = warp & 3, c0 = ((warp - 2) >> 2) * TK_EC;
    int gq = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < items && ok; item += gridDim.x) {
      const int ct = item % nct, rb = (item / nct) % nrb, b = item / (nct * nrb);
      const int rr = rb * BM + q * 32 + lane, col0 = ct * TK_BN + c0;
      // C of this tile while the MMAs run
      float cold[TK_EC], sum[TK_EC];
#pragma unroll
      for (int j = 0; j < TK_EC; ++j) {
        cold[j] = 0.f;
        sum[j] = 0.f;
      }
      float *crow = nullptr;
      if (rr < rows) {
        crow = reinterpret_cast<float *>(C + (long)b * sc + (rr >> 1)) + (rr & 1);
        if (BETA) {
#pragma unroll
          for (int j = 0; j < TK_EC; ++j)
            if (col0 + j < n) cold[j] = crow[2L * (col0 + j) * ldc];
        }
      }
      for (int k0 = 0; k0 < nch; k0 += TK_KG, ++gq) {
        const int buf = gq & 1;
        int okw = 0;
        if (lane == 0) okw = mbar_wait(&acc_full[buf], (gq >> 1) & 1, abort_flag, gerr, 66) ? 1 : 0;
        if (__shfl_sync(0xffffffffu, okw, 0) == 0) {
          ok = false;
          break;
        }
        __syncwarp();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        uint32_t acc[TK_EC];
        tmem_ld<16>(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * TK_BN + c0), acc);
        tmem_ld<16>(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * TK_BN + c0 + 16), acc + 16);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0)
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sm_u32(&acc_empty[buf])) : "memory");
#pragma unroll
        for (int j = 0; j < TK_EC; ++j) sum[j] += __uint_as_float(acc[j]);
      }
      if (ok && crow) {
#pragma unroll
        for (int j = 0; j < TK_EC; ++j)
          if (col0 + j < n) crow[2L * (col0 + j) * ldc] = BETA ? fmaf(alpha, sum[j], cold[j]) : alpha * sum[j];
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TK_COLS) : "memory");
}

static size_t ctf32k_work(int m, int n, int k, int batch) {
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t nk = (size_t)ceil_div(k, TF_KC);
  return al((size_t)2 * batch * 2 * nk * (2L * m) * TF_KC * 4) + al((size_t)2 * batch * 2 * nk * (long)n * TF_KC * 4);
}

static int ctf32k_attrs() {
  static std::atomic<unsigned long long> attr_done{0};
  return once_per_device(attr_done, [&]() -> int {
    GBF_CUDA(cudaFuncSetAttribute(ctf32k_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, TK_SMEM));
    GBF_CUDA(cudaFuncSetAttribute(ctf32k_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, TK_SMEM));
    return 0;
  });
}

static int ctf32k_run(cudaStream_t st, char opa, char opb, int m, int n, int k, double alpha, const cf *A, long lda,
                      long sa, const cf *B, long ldb, long sb, int beta_one, cf *C, long ldc, long sc, int batch,
                      void *work, size_t work_bytes, int *gerr) {
  if (k < 1) {
    set_error("3xTF32 GEMM: k must be >= 1");
    return -4;
  }
  if (alpha != 1.0 && alpha != -1.0) {
    set_error("3xTF32 GEMM: alpha must be +1 or -1");
    return -4;
  }
  if (ctf32k_work(m, n, k, batch) > work_bytes) {
    set_error("3xTF32 GEMM: workspace too small");
    return -4;
  }
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const int nk = ceil_div(k, TF_KC);
  const long rows = 2L * m;
  float *Ap = (float *)work;
  float *Bp = (float *)((char *)work + al((size_t)2 * batch * 2 * nk * rows * TF_KC * 4));
  const int sslot = prof_begin(st);
  tf32k_split_kernel<cf><<<dim3(ceil_div(m, 32), nk, batch), 256, 0, st>>>(1, opa, m, k, nk, A, lda, sa, batch, Ap);
  tf32k_split_kernel<cf><<<dim3(ceil_div(n, 32), nk, batch), 256, 0, st>>>(0, opb, n, k, nk, B, ldb, sb, batch, Bp);
  prof_end(st, sslot, 0.0);
  g_launches.fetch_add(2, std::memory_order_relaxed);
  CUtensorMap ta, tb;
  if (int rc = make_map_tf32(&ta, Ap, rows, 2 * batch * 2 * nk, BM)) return rc;
  if (int rc = make_map_tf32(&tb, Bp, n, 2 * batch * 2 * nk, TK_BN)) return rc;
  if (int rc = ctf32k_attrs()) return rc;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int items = ceil_div(rows, BM) * ceil_div(n, TK_BN) * batch;
  dim3 grid(std::min(items, sms));
  const int slot = prof_begin(st);
  const APlanes ap{0, 0, nk, batch, 0};
  if (beta_one)
    ctf32k_kernel<true><<<grid, TK_THREADS, TK_SMEM, st>>>(ta, tb, m, n, batch, nk, (float)alpha, C, ldc, sc, gerr,
                                                           ap);
  else
    ctf32k_kernel<false><<<grid, TK_THREADS, TK_SMEM, st>>>(ta, tb, m, n, batch, nk, (float)alpha, C, ldc, sc, gerr,
                                                            ap);
  prof_end(st, slot, 8.0 * m * (double)n * k * batch);
  GBF_LAUNCHED();
  GBF_CUDA(cudaGetLastError());
  return 0;
}

// The same product with op(A) read from stored TF32 planes (split once and
// reused, as the factors are by every solve of a FEAST iteration): `pre`
// holds [plane][bt nodes][2 nkh chunks][prows][32]; this call's op(A) rows
// start at complex row r0 and its K positions at 32 c0, for nodes b0 ..
// b0 + batch - 1.  Only B is split here.  Positions of a chunk past k meet
// B's zero padding, rows past m are computed and not stored.
static size_t ctf32k_work_pre(int n, int k, int batch) {
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  return al((size_t)2 * batch * 2 * ceil_div(k, TF_KC) * (long)n * TF_KC * 4);
}

static int ctf32k_run_pre(cudaStream_t st, int m, int n, int k, double alpha, const float *pre, long prows, int nkh,
                          int bt, int b0, int r0, int c0, char opb, const cf *B, long ldb, long sb, int beta_one,
                          cf *C, long ldc, long sc, int batch, void *work, size_t work_bytes, int *gerr) {
  if (k < 1 || (alpha != 1.0 && alpha != -1.0) || ctf32k_work_pre(n, k, batch) > work_bytes ||
      c0 + ceil_div(k, TF_KC) > nkh || b0 + batch > bt) {
    set_error("3xTF32 GEMM on stored planes: bad arguments or workspace too small");
    return -4;
  }
  const int nk = ceil_div(k, TF_KC);
  float *Bp = (float *)work;
  const int sslot = prof_begin(st);
  tf32k_split_kernel<cf><<<dim3(ceil_div(n, 32), nk, batch), 256, 0, st>>>(0, opb, n, k, nk, B, ldb, sb, batch, Bp);
  prof_end(st, sslot, 0.0);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  CUtensorMap ta, tb;
  if (int rc = make_map_tf32(&ta, pre, prows, 2 * bt * 2 * nkh, BM)) return rc;
  if (int rc = make_map_tf32(&tb, Bp, n, 2 * batch * 2 * nk, TK_BN)) return rc;
  if (int rc = ctf32k_attrs()) return rc;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int items = ceil_div(2 * m, BM) * ceil_div(n, TK_BN) * batch;
  dim3 grid(std::min(items, sms));
  const int slot = prof_begin(st);
  const APlanes ap{2 * r0, c0, nkh, bt, b0};
  if (beta_one)
    ctf32k_kernel<true><<<grid, TK_THREADS, TK_SMEM, st>>>(ta, tb, m, n, batch, nk, (float)alpha, C, ldc, sc, gerr,
                                                           ap);
  else
    ctf32k_kernel<false><<<grid, TK_THREADS, TK_SMEM, st>>>(ta, tb, m, n, batch, nk, (float)alpha, C, ldc, sc, gerr,
                                                            ap);
  prof_end(st, slot, 8.0 * m * (double)n * k * batch);
  GBF_LAUNCHED();
  GBF_CUDA(cudaGetLastError());
  return 0;
}

// ===================================================================
// Sliced GEMM for any k (real or complex FP64 operands):
//   C = alpha op(A) op(B) + beta C,  alpha in {+1, -1}, beta in {0, 1}.
// Operands are sliced once into SK = 8 base-2^7 digits (56 bits relative to
// the row / column maximum) laid out K-major in chunks of KC = 64 real
// positions; a complex operand is embedded as real rows 2i = (Re, -Im),
// 2i+1 = (Im, Re) against columns (Re, Im), interleaved per complex index p
// (positions 2p, 2p+1), so any chunk holds whole complex terms.  The kernel
// streams A and B chunks through TMA rings; per chunk the digit products of
// each weight are summed exactly in an FP32 TMEM accumulator (64 terms of at
// most 2^14 in magnitude per pair, at most 8 pairs: below 2^22), the
// epilogue adds the chunk's sums into two 64-bit integers per entry (weights
// 0-3 and 4-7), and after the last chunk forms the FP64 entry.
// ===================================================================
constexpr int SK = 8;                       // digits per operand
constexpr int KC = 64;                      // real K positions per chunk
constexpr int KBN = 32;                     // columns per tile
constexpr int KA_STAGE = BM * KC * 2;       // one A slice of one chunk (16 KB)
constexpr int KB_STAGE = SK * KBN * KC * 2; // all B slices of one chunk (32 KB)
constexpr int KNA = 10, KNB = 2;            // ring depths (A: more than one chunk in flight)
constexpr int K_SMEM = KNA * KA_STAGE + KNB * KB_STAGE + 1024 + 512;
constexpr int K_ACC = SK * KBN;             // TMEM columns of one accumulator buffer
constexpr int KTHREADS = 320;               // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue

template <class T> struct is_cplx { static constexpr bool v = false; };
template <> struct is_cplx<zd> { static constexpr bool v = true; };

// Element (i, p) of op(X) for a column-major X.
template <class T>
__device__ __forceinline__ void op_elem(char op, const T *X, long ldx, int i, int p, double &re, double &im) {
  if constexpr (is_cplx<T>::v) {
    const T v = (op == 'N') ? X[i + (long)p * ldx] : X[p + (long)i * ldx];
    re = v.x;
    im = (op == 'C') ? -v.y : v.y;
  } else {
    re = (op == 'N') ? X[i + (long)p * ldx] : X[p + (long)i * ldx];
    im = 0.0;
  }
}

// Digits d_0..d_{S-1} of rint(v 2^{7S - e}) (balanced, least significant
// first; the leading digit takes what remains).
template <int S>
__device__ __forceinline__ void digits_of(double v, int e, float *d) {
  int_digits<S>(fixed_point<S>(v, e), d);
}

// Rows of op(A) (m x k) -> slices [SK][batch][R][Kp] bf16 with R = m (real) or
// 2m (complex embedding) and scale exponents [batch][R].  One warp per row of
// op(A); lanes stride over p.
template <class T>
__global__ void slice_rows_kernel(char op, int m, int k, const T *A, long lda, long sa, int batch, int Kp,
                                  __nv_bfloat16 *out, int *exps) {
  constexpr bool CX = is_cplx<T>::v;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), b = blockIdx.y, lane = threadIdx.x & 31;
  if (i >= m) return;  // warp-uniform
  const T *Ab = A + (long)b * sa;
  unsigned long long mb = 0;
  for (int p = lane; p < k; p += 32) {
    double re, im;
    op_elem<T>(op, Ab, lda, i, p, re, im);
    const unsigned long long a = (unsigned long long)__double_as_longlong(re) & 0x7FFFFFFFFFFFFFFFull;
    const unsigned long long c = (unsigned long long)__double_as_longlong(im) & 0x7FFFFFFFFFFFFFFFull;
    mb = a > mb ? a : mb;
    mb = c > mb ? c : mb;
  }
  const int e = scale_exp(warp_absmax_bits(__longlong_as_double((long long)mb), 0.0));
  const long R = CX ? 2L * m : m;
  const long plane = R * Kp;
  for (int p = lane; p < k; p += 32) {
    double re, im;
    op_elem<T>(op, Ab, lda, i, p, re, im);
    float dr[SK], di[SK];
    digits_of<SK>(re, e, dr);
    if constexpr (CX) {
      digits_of<SK>(im, e, di);
      for (int t = 0; t < SK; ++t) {
        __nv_bfloat16 *o = out + ((long)t * batch + b) * plane + (2L * i) * Kp + 2 * p;
        *reinterpret_cast<__nv_bfloat162 *>(o) = __floats2bfloat162_rn(dr[t], -di[t]);
        *reinterpret_cast<__nv_bfloat162 *>(o + Kp) = __floats2bfloat162_rn(di[t], dr[t]);
      }
    } else {
      for (int t = 0; t < SK; ++t) out[((long)t * batch + b) * plane + (long)i * Kp + p] = __float2bfloat16_rn(dr[t]);
    }
  }
  const int kr = CX ? 2 * k : k;  // zero padding of positions kr .. Kp-1
  for (int q = kr + lane; q < Kp; q += 32)
    for (int t = 0; t < SK; ++t) {
      __nv_bfloat16 *o = out + ((long)t * batch + b) * plane + (CX ? 2L * i : (long)i) * Kp + q;
      *o = __float2bfloat16_rn(0.f);
      if (CX) o[Kp] = __float2bfloat16_rn(0.f);
    }
  if (lane == 0) {
    if (CX) {
      exps[(long)b * R + 2 * i] = e;
      exps[(long)b * R + 2 * i + 1] = e;
    } else {
      exps[(long)b * R + i] = e;
    }
  }
}

// Columns of op(B) (k x n) -> slices [SK][batch][n][Kp] bf16 (complex:
// positions 2p, 2p+1 = Re, Im) and exponents [batch][n].  One warp per column.
template <class T>
__global__ void slice_cols_kernel(char op, int k, int n, const T *B, long ldb, long sb, int batch, int Kp,
                                  __nv_bfloat16 *out, int *exps) {
  constexpr bool CX = is_cplx<T>::v;
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), b = blockIdx.y, lane = threadIdx.x & 31;
  if (c >= n) return;  // warp-uniform
  const T *Bb = B + (long)b * sb;
  // element (p, c) of op(B): N reads B[p + c ldb], T and C read B[c + p ldb]
  auto elem = [&](int p, double &re, double &im) {
    if constexpr (CX) {
      const T v = (op == 'N') ? Bb[p + (long)c * ldb] : Bb[c + (long)p * ldb];
      re = v.x;
      im = (op == 'C') ? -v.y : v.y;
    } else {
      re = (op == 'N') ? Bb[p + (long)c * ldb] : Bb[c + (long)p * ldb];
      im = 0.0;
    }
  };
  unsigned long long mb = 0;
  for (int p = lane; p < k; p += 32) {
    double re, im;
    elem(p, re, im);
    const unsigned long long a = (unsigned long long)__double_as_longlong(re) & 0x7FFFFFFFFFFFFFFFull;
    const unsigned long long d = (unsigned long long)__double_as_longlong(im) & 0x7FFFFFFFFFFFFFFFull;
    mb = a > mb ? a : mb;
    mb = d > mb ? d : mb;
  }
  const int e = scale_exp(warp_absmax_bits(__longlong_as_double((long long)mb), 0.0));
  const long plane = (long)n * Kp;
  for (int p = lane; p < k; p += 32) {
    double re, im;
    elem(p, re, im);
    float dr[SK], di[SK];
    digits_of<SK>(re, e, dr);
    if constexpr (CX) {
      digits_of<SK>(im, e, di);
      for (int t = 0; t < SK; ++t)
        *reinterpret_cast<__nv_bfloat162 *>(out + ((long)t * batch + b) * plane + (long)c * Kp + 2 * p) =
            __floats2bfloat162_rn(dr[t], di[t]);
    } else {
      for (int t = 0; t < SK; ++t) out[((long)t * batch + b) * plane + (long)c * Kp + p] = __float2bfloat16_rn(dr[t]);
    }
  }
  const int kr = CX ? 2 * k : k;
  for (int q = kr + lane; q < Kp; q += 32)
    for (int t = 0; t < SK; ++t) out[((long)t * batch + b) * plane + (long)c * Kp + q] = __float2bfloat16_rn(0.f);
  if (lane == 0) exps[(long)b * n + c] = e;
}

// Bias of the sums of (float bits of s_a + 1.5 2^23) 2^{7(3-a)} over four
// weights, taken mod 2^64 (the same for weights 0-3 and 4-7).
__host__ __device__ constexpr unsigned long long quad_bias() {
  unsigned long long k = 0;
  for (int a = 0; a < 4; ++a) k += 0x4B400000ull << (7 * (3 - a));
  return k;
}

// Adds the 8 weight sums of 16 columns (this warp's 32 lanes) of one chunk:
// weights 0-3 into hi, 4-7 into lo, each as sum_a bits_a 2^{7(3-(a mod 4))}.
template <int A>
__device__ __forceinline__ void add_chunk(unsigned long long *hi, unsigned long long *lo, uint32_t taddr) {
  if constexpr (A < SK) {
    uint32_t r0[16], r1[16];
    const uint32_t t0 = taddr + (uint32_t)(A * KBN);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
        "[%16];"
        : "=r"(r0[0]), "=r"(r0[1]), "=r"(r0[2]), "=r"(r0[3]), "=r"(r0[4]), "=r"(r0[5]), "=r"(r0[6]), "=r"(r0[7]),
          "=r"(r0[8]), "=r"(r0[9]), "=r"(r0[10]), "=r"(r0[11]), "=r"(r0[12]), "=r"(r0[13]), "=r"(r0[14]),
          "=r"(r0[15])
        : "r"(t0));
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
        "[%16];"
        : "=r"(r1[0]), "=r"(r1[1]), "=r"(r1[2]), "=r"(r1[3]), "=r"(r1[4]), "=r"(r1[5]), "=r"(r1[6]), "=r"(r1[7]),
          "=r"(r1[8]), "=r"(r1[9]), "=r"(r1[10]), "=r"(r1[11]), "=r"(r1[12]), "=r"(r1[13]), "=r"(r1[14]),
          "=r"(r1[15])
        : "r"(t0 + (uint32_t)KBN));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    constexpr int w0 = 7 * (3 - (A & 3)), w1 = w0 - 7;
    unsigned long long *dst = (A < 4) ? hi : lo;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      dst[j] = add_shifted<w0>(dst[j], __float_as_uint(__uint_as_float(r0[j]) + 12582912.0f));
      dst[j] = add_shifted<w1>(dst[j], __float_as_uint(__uint_as_float(r1[j]) + 12582912.0f));
    }
    add_chunk<A + 2>(hi, lo, taddr);
  }
}

// Work item = (column chunk, 128-row block, batch); each tile (row block x
// 32 columns) runs over all nkc K chunks.  Counters per CTA: h = chunks
// processed (B ring stage h % KNB, accumulator buffer h % 2), h*SK + t =
// A slices processed (A ring stage (h*SK+t) % KNA).
// MC: CTA pairs (clusters of 2) take the two column tiles 2p, 2p+1 of an
// item p; they stream the same A chunks, so each A slice is loaded once for
// both, by the CTA of rank t % 2, multicast into both CTAs' rings; a ring
// stage is free again when both CTAs' MMAs are done with it (each MMA
// thread's commit arrives in both CTAs).  A tile past the last column runs
// like the others and stores nothing.  Halves the A traffic into the SMs,
// the limit of this kernel at 32 columns per tile.
template <class T, bool BETA, bool MC>
__global__ void __launch_bounds__(KTHREADS, 1)
    gemm_sliced_k_kernel(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, int R,
                         int n, int batch, int nkc, int nch, int tpc, const int *__restrict__ sexp,
                         const int *__restrict__ texp, double alpha, T *C, long ldc, long sc, int *gerr) {
  constexpr bool CX = is_cplx<T>::v;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *sA = base;                        // KNA x [128][64]
  unsigned char *sB = base + KNA * KA_STAGE;       // KNB x SK x [32][64]
  uint64_t *bars = reinterpret_cast<uint64_t *>(base + KNA * KA_STAGE + KNB * KB_STAGE);
  uint64_t *a_full = bars, *a_empty = bars + KNA;
  uint64_t *b_full = bars + 2 * KNA, *b_empty = b_full + KNB;
  uint64_t *acc_full = b_empty + KNB, *acc_empty = acc_full + 2;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_empty + 2);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nrb = (R + BM - 1) / BM, nct = (n + KBN - 1) / KBN;
  const int items = nch * nrb * batch;
  constexpr uint32_t NCOLS = 2 * K_ACC;  // 512
  const int crank = MC ? (int)cluster_rank() : 0;
  const int cid = MC ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
  const int ncl = MC ? (int)(gridDim.x >> 1) : (int)gridDim.x;
  // this CTA's column tiles of item chunk cc
  auto tiles = [&](int cc, int &t0, int &t1) {
    if (MC) {
      t0 = 2 * cc + crank;
      t1 = t0 + 1;
    } else {
      t0 = cc * tpc;
      t1 = min(nct, (cc + 1) * tpc);
    }
  };

  if (threadIdx.x == 0) {
    for (int j = 0; j < KNA; ++j) {
      mbar_init(&a_full[j], 1);
      mbar_init(&a_empty[j], MC ? 2 : 1);
    }
    for (int j = 0; j < KNB; ++j) {
      mbar_init(&b_full[j], 1);
      mbar_init(&b_empty[j], 1);
    }
    for (int j = 0; j < 2; ++j) {
      mbar_init(&acc_full[j], 1);
      mbar_init(&acc_empty[j], 8);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sm_u32(tmem_slot)),
                 "r"(NCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (MC) cluster_sync_all();  // both CTAs' barriers initialised before any multicast
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ TMA --
    long h = 0;
    long last_a = -1, last_b = -1;
    bool ok = true;
    for (int item = cid; item < items && ok; item += ncl) {
      const int cc = item % nch, rb = (item / nch) % nrb, b = item / (nch * nrb);
      int ct0, ct1;
      tiles(cc, ct0, ct1);
      for (int ct = ct0; ct < ct1 && ok; ++ct)
        for (int c = 0; c < nkc && ok; ++c, ++h) {
          const int sb = (int)(h % KNB);
          if (h >= KNB && !mbar_wait(&b_empty[sb], (uint32_t)((h / KNB - 1) & 1), abort_flag, gerr, 41)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&b_full[sb], KB_STAGE);
          for (int u = 0; u < SK; ++u)
            tma_load_3d(sB + sb * KB_STAGE + u * (KBN * KC * 2), &tb, &b_full[sb], c * KC, ct * KBN, u * batch + b);
          last_b = h;
          for (int t = 0; t < SK; ++t) {
            const long ga = h * SK + t;
            const int sa = (int)(ga % KNA);
            if (ga >= KNA && !mbar_wait(&a_empty[sa], (uint32_t)((ga / KNA - 1) & 1), abort_flag, gerr, 42)) {
              ok = false;
              break;
            }
            mbar_expect_tx(&a_full[sa], KA_STAGE);
            if (!MC)
              tma_load_3d(sA + sa * KA_STAGE, &ta, &a_full[sa], c * KC, rb * BM, t * batch + b);
            else if ((t & 1) == crank)
              tma_load_3d_mc(sA + sa * KA_STAGE, &ta, &a_full[sa], c * KC, rb * BM, t * batch + b, 0x3);
            last_a = ga;
          }
        }
    }
    for (long gg = (last_a - KNA + 1 > 0 ? last_a - KNA + 1 : 0); gg <= last_a; ++gg)
      mbar_drain(&a_full[gg % KNA], (uint32_t)((gg / KNA) & 1), gerr, 43);
    for (long gg = (last_b - KNB + 1 > 0 ? last_b - KNB + 1 : 0); gg <= last_b; ++gg)
      mbar_drain(&b_full[gg % KNB], (uint32_t)((gg / KNB) & 1), gerr, 44);
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------------------ MMA --
    long h = 0;
    bool ok = true;
    for (int item = cid; item < items && ok; item += ncl) {
      const int cc = item % nch;
      int ct0, ct1;
      tiles(cc, ct0, ct1);
      for (int ct = ct0; ct < ct1 && ok; ++ct)
        for (int c = 0; c < nkc; ++c) {
          const int sb = (int)(h % KNB), buf = (int)(h & 1);
          if (!mbar_wait(&b_full[sb], (uint32_t)((h / KNB) & 1), abort_flag, gerr, 45) ||
              (h >= 2 && !mbar_wait(&acc_empty[buf], (uint32_t)(((h >> 1) - 1) & 1), abort_flag, gerr, 46))) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t dbase = tmem + (uint32_t)(buf * K_ACC);
          const uint64_t bd = sdesc_sw128(sm_u32(sB + sb * KB_STAGE));
          bool issued = false;
#pragma unroll
          for (int t = 0; t < SK; ++t) {
            const long ga = h * SK + t;
            const int sa = (int)(ga % KNA);
            if (!mbar_wait(&a_full[sa], (uint32_t)((ga / KNA) & 1), abort_flag, gerr, 47)) {
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t idesc = idesc_bf16_n((SK - t) * KBN);
            const uint64_t ad = sdesc_sw128(sm_u32(sA + sa * KA_STAGE));
#pragma unroll
            for (int kk = 0; kk < KC / 16; ++kk)
              mma_bf16(dbase + (uint32_t)(t * KBN), ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), idesc,
                       (t > 0 || kk > 0) ? 1u : 0u);
            if (MC)
              mma_commit_mc(&a_empty[sa], 0x3);
            else
              mma_commit(&a_empty[sa]);
            issued = true;
          }
          if (!ok) {
            if (issued) {
              mma_commit(&acc_full[buf]);
              ++h;
            }
            break;
          }
          mma_commit(&b_empty[sb]);
          mma_commit(&acc_full[buf]);
          ++h;
        }
    }
    if (h > 0) mbar_drain(&acc_full[(h - 1) & 1], (uint32_t)(((h - 1) >> 1) & 1), gerr, 48);
  } else if (warp >= 2) {
    // ------------------------------------------------------- epilogue --
    // Warp w reads TMEM lanes 32 (w % 4) .. +31 and columns c0 .. c0+15 of
    // every tile, c0 = 16 ((w - 2) / 4).
    const int q = warp & 3, c0 = ((warp - 2) >> 2) * 16;
    const bool neg = alpha < 0.0;
    long h = 0;
    bool ok = true;
    for (int item = cid; item < items && ok; item += ncl) {
      const int cc = item % nch, rb = (item / nch) % nrb, b = item / (nch * nrb);
      int ct0, ct1;
      tiles(cc, ct0, ct1);
      const int r = rb * BM + q * 32 + lane;
      const bool rv = r < R;
      const int es = rv ? __ldg(sexp + (long)b * R + r) - 7 * (SK + 1) : 0;
      double *crow = CX ? reinterpret_cast<double *>(C + (long)b * sc + (r >> 1)) + (r & 1)
                        : reinterpret_cast<double *>(C + (long)b * sc + r);
      const long cstride = CX ? 2L * ldc : ldc;  // doubles between columns
      for (int ct = ct0; ct < ct1 && ok; ++ct) {
        const int col0 = ct * KBN + c0;
        const int tcol = (col0 + (lane & 15) < n) ? __ldg(texp + (long)b * n + col0 + (lane & 15)) : 0;
        unsigned long long hi[16], lo[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) hi[j] = lo[j] = 0ull;
        for (int c = 0; c < nkc; ++c, ++h) {
          const int buf = (int)(h & 1);
          int okw = 0;
          if (lane == 0) okw = mbar_wait(&acc_full[buf], (uint32_t)((h >> 1) & 1), abort_flag, gerr, 49) ? 1 : 0;
          if (__shfl_sync(0xffffffffu, okw, 0) == 0) {
            ok = false;
            break;
          }
          __syncwarp();
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          add_chunk<0>(hi, lo, tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * K_ACC + c0));
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0)
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sm_u32(&acc_empty[buf])) : "memory");
        }
        if (!ok) break;
        // value = (hi 2^28 + lo) 2^{es+et}: top = hi + floor(lo / 2^28) and
        // rem = lo mod 2^28 are exact; top converts with one rounding, and
        // one fused multiply-add joins them
        const unsigned long long bias = (unsigned long long)nkc * quad_bias();
        int et[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) et[j] = __shfl_sync(0xffffffffu, tcol, j);
        const bool fast = __reduce_min_sync(0xffffffffu, es) + __reduce_min_sync(0xffffffffu, tcol) >= -1022 &&
                          __reduce_max_sync(0xffffffffu, es) + __reduce_max_sync(0xffffffffu, tcol) <= 995;
#pragma unroll
        for (int j0 = 0; j0 < 16; j0 += 8) {
          double cur[8];  // C of these 8 columns, loaded ahead of their conversions
          if constexpr (BETA) {
#pragma unroll
            for (int j = 0; j < 8; ++j)
              cur[j] = (rv && col0 + j0 + j < n) ? crow[(long)(col0 + j0 + j) * cstride] : 0.0;
          }
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
          const int j = j0 + jj;
          const long long hs = (long long)(hi[j] - bias), ls = (long long)(lo[j] - bias);
          const long long top = hs + (ls >> 28);
          const long long rem = ls & ((1LL << 28) - 1);
          const int E = es + et[j];
          double p28, p0;
          if (fast) {
            p28 = __longlong_as_double((long long)(E + 28 + 1023) << 52);
            p0 = __longlong_as_double((long long)(E + 1023) << 52);
          } else {
            p28 = ldexp(1.0, E + 28);
            p0 = ldexp(1.0, E);
          }
          double v = fma(__ll2double_rn(top), p28, __ll2double_rn(rem) * p0);
          if (neg) v = -v;
          if (rv && col0 + j < n) crow[(long)(col0 + j) * cstride] = BETA ? cur[jj] + v : v;
        }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  // neither CTA of a pair leaves while the other may still multicast into
  // it or arrive on its barriers
  if (MC) cluster_sync_all();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS) : "memory");
}

// 3-D map over [planes][rows][Kp] bf16, box (KC, box_rows, 1).
static int make_map_k(CUtensorMap *map, const void *ptr, long rows, long Kp, int planes, int box_rows) {
  auto fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled unavailable");
    return -4;
  }
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)rows * Kp * 2};
  cuuint32_t box[3] = {(cuuint32_t)KC, (cuuint32_t)box_rows, 1};
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

template <class T>
static int gemm_sliced_k_launch(cudaStream_t st, const SlicedOp &a, const SlicedOp &b, int batch, double alpha,
                                int beta_one, T *C, long ldc, long sc, int *gerr) {
  if (a.Kp != b.Kp || a.Kp % KC) {
    set_error("sliced GEMM: operand K layouts differ");
    return -4;
  }
  CUtensorMap ta, tb;
  if (int rc = make_map_k(&ta, a.slices, a.rows, a.Kp, SK * batch, BM)) return rc;
  if (int rc = make_map_k(&tb, b.slices, b.rows, b.Kp, SK * batch, KBN)) return rc;
  static std::atomic<unsigned long long> attr_done{0};
  if (int rc = once_per_device(attr_done, [&]() -> int {
        GBF_CUDA(cudaFuncSetAttribute(gemm_sliced_k_kernel<T, true, false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, K_SMEM));
        GBF_CUDA(cudaFuncSetAttribute(gemm_sliced_k_kernel<T, false, false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, K_SMEM));
        GBF_CUDA(cudaFuncSetAttribute(gemm_sliced_k_kernel<T, true, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, K_SMEM));
        GBF_CUDA(cudaFuncSetAttribute(gemm_sliced_k_kernel<T, false, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, K_SMEM));
        return 0;
      }))
    return rc;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int base_items = ceil_div(a.rows, (long)BM) * batch, nct = ceil_div(b.rows, KBN);
  const int nkc = (int)(a.Kp / KC);
  // pairs of column tiles on CTA pairs sharing the A stream (more than one
  // column tile); else one work item per tile: every tile streams its own A
  // chunks, so finer items cost no traffic and balance the last round;
  // consecutive items are the column tiles of one row block (its A chunks
  // shared in L2)
  if (nct > 1) {
    const int npair = ceil_div(nct, 2), items = base_items * npair;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * std::min(items, sms / 2), 1, 1);
    cfg.blockDim = dim3(KTHREADS, 1, 1);
    cfg.dynamicSmemBytes = K_SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e =
        beta_one ? cudaLaunchKernelEx(&cfg, gemm_sliced_k_kernel<T, true, true>, ta, tb, (int)a.rows, (int)b.rows,
                                      batch, nkc, npair, 1, a.exps, b.exps, alpha, C, ldc, sc, gerr)
                 : cudaLaunchKernelEx(&cfg, gemm_sliced_k_kernel<T, false, true>, ta, tb, (int)a.rows, (int)b.rows,
                                      batch, nkc, npair, 1, a.exps, b.exps, alpha, C, ldc, sc, gerr);
    if (e == cudaSuccess) {
      GBF_LAUNCHED();
      return 0;
    }
    cudaGetLastError();
  }
  const int tpc = 1, nch = nct;
  const int items = base_items * nch;
  dim3 grid(std::min(items, sms));
  if (beta_one)
    gemm_sliced_k_kernel<T, true, false><<<grid, KTHREADS, K_SMEM, st>>>(ta, tb, (int)a.rows, (int)b.rows, batch, nkc,
                                                                          nch, tpc, a.exps, b.exps, alpha, C, ldc, sc,
                                                                          gerr);
  else
    gemm_sliced_k_kernel<T, false, false><<<grid, KTHREADS, K_SMEM, st>>>(ta, tb, (int)a.rows, (int)b.rows, batch,
                                                                           nkc, nch, tpc, a.exps, b.exps, alpha, C,
                                                                           ldc, sc, gerr);
  GBF_LAUNCHED();
  GBF_CUDA(cudaGetLastError());
  return 0;
}


}  // namespace tc

long sliced_kp(int k, bool cplx) {
  const long kr = cplx ? 2L * k : (long)k;
  return (kr + tc::KC - 1) / tc::KC * tc::KC;
}
size_t sliced_op_bytes(long rows, long Kp, int batch) {
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  return al((size_t)tc::SK * batch * rows * Kp * 2) + al((size_t)batch * rows * 4);
}

template <class T>
int slice_rows(cudaStream_t st, char op, int m, int k, const T *A, long lda, long sa, int batch, void *buf,
               SlicedOp *out) {
  constexpr bool CX = tc::is_cplx<T>::v;
  const long R = CX ? 2L * m : m, Kp = sliced_kp(k, CX);
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  out->slices = buf;
  out->exps = (const int *)((char *)buf + al((size_t)tc::SK * batch * R * Kp * 2));
  out->rows = R;
  out->Kp = Kp;
  const int slot = prof_begin(st);
  tc::slice_rows_kernel<T><<<dim3(ceil_div(m, 8), batch), 256, 0, st>>>(
      op, m, k, A, lda, sa, batch, (int)Kp, (__nv_bfloat16 *)buf, const_cast<int *>(out->exps));
  prof_end(st, slot, 0.0);
  GBF_LAUNCHED();
  GBF_CUDA(cudaGetLastError());
  return 0;
}

template <class T>
int slice_cols(cudaStream_t st, char op, int k, int n, const T *B, long ldb, long sb, int batch, void *buf,
               SlicedOp *out) {
  constexpr bool CX = tc::is_cplx<T>::v;
  const long Kp = sliced_kp(k, CX);
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  out->slices = buf;
  out->exps = (const int *)((char *)buf + al((size_t)tc::SK * batch * n * Kp * 2));
  out->rows = n;
  out->Kp = Kp;
  const int slot = prof_begin(st);
  tc::slice_cols_kernel<T><<<dim3(ceil_div(n, 8), batch), 256, 0, st>>>(
      op, k, n, B, ldb, sb, batch, (int)Kp, (__nv_bfloat16 *)buf, const_cast<int *>(out->exps));
  prof_end(st, slot, 0.0);
  GBF_LAUNCHED();
  GBF_CUDA(cudaGetLastError());
  return 0;
}

template <class T>
int gemm_sliced_ops(cudaStream_t st, const SlicedOp &a, const SlicedOp &b, int batch, double alpha, int beta_one,
                    T *C, long ldc, long sc, int *gerr) {
  if (alpha != 1.0 && alpha != -1.0) {
    set_error("sliced GEMM: alpha must be +1 or -1");
    return -4;
  }
  if (a.rows <= 0 || b.rows <= 0 || batch <= 0) return 0;
  const int slot = prof_begin(st);
  const int rc = tc::gemm_sliced_k_launch<T>(st, a, b, batch, alpha, beta_one, C, ldc, sc, gerr);
  // useful FP64 flops (padded K): the real embedding's 2 R n Kp equals 8 m n k for complex data;
  // issued: 36 digit-pair products of 128 x 32 x Kp per (row block, column tile)
  const double tiles = (double)ceil_div(a.rows, (long)tc::BM) * ceil_div(b.rows, (long)tc::KBN) * batch;
  prof_end_tc(st, slot, 2.0 * a.rows * (double)b.rows * a.Kp * batch,
              2.0 * tc::BM * tc::KBN * (double)a.Kp * (tc::SK * (tc::SK + 1) / 2) * tiles);
  return rc;
}

size_t gemm_sliced_k_work(bool cplx, int m, int n, int k, int batch) {
  const long Kp = sliced_kp(k, cplx);
  return sliced_op_bytes(cplx ? 2L * m : m, Kp, batch) + sliced_op_bytes(n, Kp, batch);
}

template <class T>
int gemm_sliced_k(cudaStream_t st, char opa, char opb, int m, int n, int k, double alpha, const T *A, long lda,
                  long sa, const T *B, long ldb, long sb, int beta_one, T *C, long ldc, long sc, int batch, void *work,
                  size_t work_bytes, int *gerr) {
  constexpr bool CX = tc::is_cplx<T>::v;
  if (m <= 0 || n <= 0 || batch <= 0) return 0;
  if (k < 1) {
    set_error("sliced GEMM: k must be positive");
    return -4;
  }
  if (gemm_sliced_k_work(CX, m, n, k, batch) > work_bytes) {
    set_error("sliced GEMM: workspace too small");
    return -4;
  }
  const long Kp = sliced_kp(k, CX);
  SlicedOp a, b;
  if (int rc = slice_rows<T>(st, opa, m, k, A, lda, sa, batch, work, &a)) return rc;
  if (int rc = slice_cols<T>(st, opb, k, n, B, ldb, sb, batch,
                             (char *)work + sliced_op_bytes(CX ? 2L * m : m, Kp, batch), &b))
    return rc;
  return gemm_sliced_ops<T>(st, a, b, batch, alpha, beta_one, C, ldc, sc, gerr);
}

#define GBF_SLICED_INST(T)                                                                                   \
  template int slice_rows<T>(cudaStream_t, char, int, int, const T *, long, long, int, void *, SlicedOp *);  \
  template int slice_cols<T>(cudaStream_t, char, int, int, const T *, long, long, int, void *, SlicedOp *);  \
  template int gemm_sliced_ops<T>(cudaStream_t, const SlicedOp &, const SlicedOp &, int, double, int, T *,  \
                                  long, long, int *);                                                        \
  template int gemm_sliced_k<T>(cudaStream_t, char, char, int, int, int, double, const T *, long, long,      \
                                const T *, long, long, int, T *, long, long, int, void *, size_t, int *);
GBF_SLICED_INST(double)
GBF_SLICED_INST(zd)
#undef GBF_SLICED_INST

namespace tc {
}  // namespace tc

size_t zgemm_sliced_work(int m, int n, int batch, int S) {
  if (S == 1) return tc::ctf32_work(m, n, batch);
  S = S < 0 ? -S : S;
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  return al((size_t)S * batch * 2L * m * tc::ZK * 2) + al((size_t)S * batch * n * tc::ZK * 2) +
         al((size_t)batch * 2L * m * 8) + al((size_t)batch * n * 8);
}

template <class T>
int zgemm_sliced(cudaStream_t st, int S, char opa, char opb, int m, int n, int k, double alpha, const T *A, long lda,
                 long sa, const T *B, long ldb, long sb, int beta_one, T *C, long ldc, long sc, int batch, void *work,
                 size_t work_bytes, int *gerr) {
  if (m <= 0 || n <= 0 || batch <= 0) return 0;
  if (S == 7)
    return tc::zgemm_sliced_run<T, 7, false>(st, opa, opb, m, n, k, alpha, A, lda, sa, B, ldb, sb, beta_one, C, ldc,
                                             sc, batch, work, work_bytes, gerr);
  if (S == 4)
    return tc::zgemm_sliced_run<T, 4, false>(st, opa, opb, m, n, k, alpha, A, lda, sa, B, ldb, sb, beta_one, C, ldc,
                                             sc, batch, work, work_bytes, gerr);
  if (S == 3)
    return tc::zgemm_sliced_run<T, 3, false>(st, opa, opb, m, n, k, alpha, A, lda, sa, B, ldb, sb, beta_one, C, ldc,
                                             sc, batch, work, work_bytes, gerr);
  if (S == -3)  // FP32 entries split into three bf16 parts, FP32 accumulation
    return tc::zgemm_sliced_run<T, 3, true>(st, opa, opb, m, n, k, alpha, A, lda, sa, B, ldb, sb, beta_one, C, ldc,
                                            sc, batch, work, work_bytes, gerr);
  if (S == 1) {  // complex FP32 operands and output: 3xTF32 products
    if constexpr (std::is_same<T, cf>::value)
      return tc::ctf32_run(st, opa, opb, m, n, k, alpha, A, lda, sa, B, ldb, sb, beta_one, C, ldc, sc, batch, work,
                           work_bytes, gerr);
    set_error("sliced GEMM: S = 1 (3xTF32) needs complex FP32 operands");
    return -4;
  }
  set_error("sliced GEMM: S must be 1, 3, 4, 7 or -3");
  return -4;
}

size_t cgemm_tf32k_work(int m, int n, int k, int batch) { return tc::ctf32k_work(m, n, k, batch); }

int cgemm_tf32k(cudaStream_t st, char opa, char opb, int m, int n, int k, double alpha, const cf *A, long lda, long sa,
                const cf *B, long ldb, long sb, int beta_one, cf *C, long ldc, long sc, int batch, void *work,
                size_t work_bytes, int *gerr) {
  if (m <= 0 || n <= 0 || batch <= 0) return 0;
  return tc::ctf32k_run(st, opa, opb, m, n, k, alpha, A, lda, sa, B, ldb, sb, beta_one, C, ldc, sc, batch, work,
                        work_bytes, gerr);
}

size_t tf32_planes_bytes(int n, int ne) {
  return (size_t)2 * ne * 2 * ceil_div(n, tc::TF_KC) * (2L * n) * tc::TF_KC * 4;
}

int tf32_presplit(cudaStream_t st, char op, int n, int ne, const cf *S, float *planes) {
  const int nkh = ceil_div(n, tc::TF_KC);
  tc::tf32k_split_kernel<cf><<<dim3(ceil_div(n, 32), nkh, ne), 256, 0, st>>>(1, op, n, n, nkh, S, n, (long)n * n, ne,
                                                                             planes);
  GBF_LAUNCHED();
  GBF_CUDA(cudaGetLastError());
  return 0;
}

size_t cgemm_tf32k_pre_work(int n, int k, int batch) { return tc::ctf32k_work_pre(n, k, batch); }

int cgemm_tf32k_pre(cudaStream_t st, int m, int n, int k, double alpha, const float *pre, int nfull, int bt, int b0,
                    int r0, int c0, const cf *B, long ldb, long sb, int beta_one, cf *C, long ldc, long sc, int batch,
                    void *work, size_t work_bytes, int *gerr) {
  if (m <= 0 || n <= 0 || batch <= 0) return 0;
  return tc::ctf32k_run_pre(st, m, n, k, alpha, pre, 2L * nfull, ceil_div(nfull, tc::TF_KC), bt, b0, r0, c0, 'N', B,
                            ldb, sb, beta_one, C, ldc, sc, batch, work, work_bytes, gerr);
}
template int zgemm_sliced<zd>(cudaStream_t, int, char, char, int, int, int, double, const zd *, long, long,
                              const zd *, long, long, int, zd *, long, long, int, void *, size_t, int *);
template int zgemm_sliced<cf>(cudaStream_t, int, char, char, int, int, int, double, const cf *, long, long,
                              const cf *, long, long, int, cf *, long, long, int, void *, size_t, int *);

}  // namespace gbf

// Verification entry (C ABI) of the sliced complex GEMM: dC (complex
// interleaved, FP64 when prec 0 else FP32) = alpha op(dA) op(dB) + beta dC
// with op in {'N','T','C'}, k <= 32, alpha = +-1, beta in {0, 1}, S digits
// (7 or 3), batches strided by sa/sb/sc elements.  dWork >= the bytes
// gbf_zgemm_sliced_work returns; dErr one device int.
extern "C" size_t gbf_zgemm_sliced_work(int m, int n, int batch, int S) {
  return gbf::zgemm_sliced_work(m, n, batch, S);
}
extern "C" int gbf_zgemm_sliced(void *stream, int prec, int S, char opa, char opb, int m, int n, int k,
                                double alpha, const void *dA, long lda, long sa, const void *dB, long ldb, long sb,
                                int beta, void *dC, long ldc, long sc, int batch, void *dWork, size_t work_bytes,
                                int *dErr) {
  cudaStream_t st = (cudaStream_t)stream;
  GBF_CUDA(cudaMemsetAsync(dErr, 0, sizeof(int), st));
  int rc = prec ? gbf::zgemm_sliced<gbf::cf>(st, S, opa, opb, m, n, k, alpha, (const gbf::cf *)dA, lda, sa,
                                             (const gbf::cf *)dB, ldb, sb, beta, (gbf::cf *)dC, ldc, sc, batch, dWork,
                                             work_bytes, dErr)
                : gbf::zgemm_sliced<gbf::zd>(st, S, opa, opb, m, n, k, alpha, (const gbf::zd *)dA, lda, sa,
                                             (const gbf::zd *)dB, ldb, sb, beta, (gbf::zd *)dC, ldc, sc, batch, dWork,
                                             work_bytes, dErr);
  if (rc) return rc;
  int herr = 0;
  GBF_CUDA(cudaMemcpyAsync(&herr, dErr, sizeof(int), cudaMemcpyDeviceToHost, st));
  GBF_CUDA(cudaStreamSynchronize(st));
  if (herr) {
    gbf::set_error("sliced GEMM: bounded wait timed out (code %d)", herr);
    return -5;
  }
  return 0;
}

// Bounded-wait check: launches tc::wait_probe_kernel with `limit` polls and
// reports its time-out as the GEMM entries do.
extern "C" int gbf_wait_probe(void *stream, long limit) {
  cudaStream_t st = (cudaStream_t)stream;
  if (limit < 1) return -101;
  int *dErr = nullptr;
  GBF_CUDA(cudaMallocAsync((void **)&dErr, sizeof(int), st));
  GBF_CUDA(cudaMemsetAsync(dErr, 0, sizeof(int), st));
  gbf::tc::wait_probe_kernel<<<1, 32, 0, st>>>(limit, dErr, 1);
  GBF_LAUNCHED();
  GBF_CUDA(cudaGetLastError());
  int herr = 0;
  GBF_CUDA(cudaMemcpyAsync(&herr, dErr, sizeof(int), cudaMemcpyDeviceToHost, st));
  GBF_CUDA(cudaFreeAsync(dErr, st));
  GBF_CUDA(cudaStreamSynchronize(st));
  if (herr) {
    gbf::set_error("wait probe: bounded wait timed out (code %d)", herr);
    return -5;
  }
  return 0;
}

// ===================================================================
// No-allocation variant of gbf_zgemm_sliced.
//
// For callers that must not allocate device memory during the call: code
// whose device memory is owned by another allocator (a framework's caching
// pool holding the whole budget), and latency-critical paths that cannot
// afford the device-wide synchronisation cudaMalloc/cudaFree imply.  The
// call reads its error word back and synchronises its stream before it
// returns.  The scratch this GEMM needs
// (digit slices, scales, error word) lives in the file-scope array below,
// which every GPU that loads this library holds until the process exits.
// ===================================================================
namespace {
constexpr size_t kNoAllocScratch = 16u << 20;  // 16 MiB
constexpr size_t kNoAllocErrOff = kNoAllocScratch - 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratch];

// Device address of the array, looked up once per device (host code must
// not use the symbol itself: on the host it only names a stand-in object).
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[64] = {nullptr};

int noalloc_scratch(void **out) {
  int dev = 0;
  GBF_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    gbf::set_error("gbf_zgemm_sliced_noalloc: device ordinal %d out of range", dev);
    return -4;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      gbf::set_error("gbf_zgemm_sliced_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return -4;
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return 0;
}
}  // namespace

extern "C" size_t gbf_zgemm_sliced_noalloc_max(void) { return kNoAllocErrOff; }

extern "C" int gbf_zgemm_sliced_noalloc(void *stream, int prec, int S, char opa, char opb, int m, int n, int k,
                                        double alpha, const void *dA, long lda, long sa, const void *dB, long ldb,
                                        long sb, int beta, void *dC, long ldc, long sc, int batch) {
  if (m <= 0 || n <= 0 || batch <= 0) return 0;
  const size_t need = gbf::zgemm_sliced_work(m, n, batch, S);
  if (need > kNoAllocErrOff) {
    gbf::set_error(
        "gbf_zgemm_sliced_noalloc: this problem needs %zu bytes of scratch, more than the fixed %zu available "
        "(use gbf_zgemm_sliced with a caller-provided workspace)",
        need, (size_t)kNoAllocErrOff);
    return -7;
  }
  void *scratch = nullptr;
  if (int rc = noalloc_scratch(&scratch)) return rc;
  int *derr = reinterpret_cast<int *>((unsigned char *)scratch + kNoAllocErrOff);
  cudaStream_t st = (cudaStream_t)stream;
  // the array keeps the previous call's contents: the error word must start at 0
  GBF_CUDA(cudaMemsetAsync(derr, 0, sizeof(int), st));
  int rc = prec ? gbf::zgemm_sliced<gbf::cf>(st, S, opa, opb, m, n, k, alpha, (const gbf::cf *)dA, lda, sa,
                                             (const gbf::cf *)dB, ldb, sb, beta, (gbf::cf *)dC, ldc, sc, batch, scratch,
                                             kNoAllocErrOff, derr)
                : gbf::zgemm_sliced<gbf::zd>(st, S, opa, opb, m, n, k, alpha, (const gbf::zd *)dA, lda, sa,
                                             (const gbf::zd *)dB, ldb, sb, beta, (gbf::zd *)dC, ldc, sc, batch, scratch,
                                             kNoAllocErrOff, derr);
  if (rc) return rc;
  int herr = 0;
  GBF_CUDA(cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, st));
  GBF_CUDA(cudaStreamSynchronize(st));
  if (herr) {
    gbf::set_error("gbf_zgemm_sliced_noalloc: bounded wait timed out (code %d)", herr);
    return -5;
  }
  return 0;
}

// Verification entry (C ABI) of the 3xTF32 complex FP32 GEMM for any k.
extern "C" size_t gbf_cgemm_tf32_work(int m, int n, int k, int batch) {
  return gbf::cgemm_tf32k_work(m, n, std::max(k, 1), batch);
}
extern "C" int gbf_cgemm_tf32(void *stream, char opa, char opb, int m, int n, int k, double alpha, const void *dA,
                              long lda, long sa, const void *dB, long ldb, long sb, int beta, void *dC, long ldc,
                              long sc, int batch, void *dWork, size_t work_bytes, int *dErr) {
  cudaStream_t st = (cudaStream_t)stream;
  GBF_CUDA(cudaMemsetAsync(dErr, 0, sizeof(int), st));
  return gbf::cgemm_tf32k(st, opa, opb, m, n, k, alpha, (const gbf::cf *)dA, lda, sa, (const gbf::cf *)dB, ldb, sb,
                          beta, (gbf::cf *)dC, ldc, sc, batch, dWork, work_bytes, dErr);
}

// Verification entry (C ABI) of the sliced GEMM for any k: dC = alpha op(dA)
// op(dB) + beta dC on FP64 data, real (cplx 0) or complex interleaved
// (cplx 1), op in {'N','T','C'}, alpha = +-1, beta in {0, 1}, batches
// strided by sa/sb/sc elements.  dWork >= gbf_gemm_sliced_work bytes; dErr
// one device int.
extern "C" size_t gbf_gemm_sliced_work(int cplx, int m, int n, int k, int batch) {
  return gbf::gemm_sliced_k_work(cplx != 0, m, n, k, batch);
}
extern "C" int gbf_gemm_sliced(void *stream, int cplx, char opa, char opb, int m, int n, int k, double alpha,
                               const void *dA, long lda, long sa, const void *dB, long ldb, long sb, int beta,
                               void *dC, long ldc, long sc, int batch, void *dWork, size_t work_bytes, int *dErr) {
  cudaStream_t st = (cudaStream_t)stream;
  GBF_CUDA(cudaMemsetAsync(dErr, 0, sizeof(int), st));
  int rc = cplx ? gbf::gemm_sliced_k<gbf::zd>(st, opa, opb, m, n, k, alpha, (const gbf::zd *)dA, lda, sa,
                                               (const gbf::zd *)dB, ldb, sb, beta, (gbf::zd *)dC, ldc, sc, batch,
                                               dWork, work_bytes, dErr)
                : gbf::gemm_sliced_k<double>(st, opa, opb, m, n, k, alpha, (const double *)dA, lda, sa,
                                             (const double *)dB, ldb, sb, beta, (double *)dC, ldc, sc, batch, dWork,
                                             work_bytes, dErr);
  return rc;
}
