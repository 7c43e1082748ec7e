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

// ===================================================================
// Sliced complex GEMM on the tensor cores:
//   C = alpha op(A) op(B) + beta C,  complex (zd or cf), k <= 32,
//   alpha in {+1, -1}, beta in {0, 1}.
// Real embedding: complex row i of op(A) -> real rows 2i = [Re | -Im] and
// 2i+1 = [Im | Re] (length 2k); column c of op(B) -> [Re ; Im].  Then
// real row 2i (2i+1) times column c is Re (Im) of the complex product.
// Slicing (exact error-free split): each real row r is scaled by a power of
// two sigma_r >= its largest magnitude, each column c by tau_c; x/sigma in
// [-1, 1] is written as sum_{t=1..S} d_t 2^{-7t} with integer digits d_t
// (|d_1| <= 128, |d_t| <= 64 after), each exact in bf16.  For digit pairs
// (t, u) with t + u <= S + 1, the products D_t E_u^T are integers below
// 2^24 in magnitude even summed over all pairs of one weight (64 terms of
// at most 2^14, at most S pairs), so one FP32 TMEM accumulator per weight
// w = t + u holds them exactly; the epilogue forms
//   sigma_r tau_c sum_w 2^{-7w} S_w  in FP64.
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

__device__ __forceinline__ double pow2_ceil(double mx) {
  if (!(mx > 0.0)) return 1.0;
  int e;
  const double f = frexp(mx, &e);  // mx = f 2^e, f in [0.5, 1)
  (void)f;
  return ldexp(1.0, e);            // 2^e >= mx
}

// digits of v in [-1, 1]: v = sum_t d_t 2^{-7t} + rest (exact recursion)
template <int S>
__device__ __forceinline__ void digits(double v, float *d) {
#pragma unroll
  for (int t = 0; t < S; ++t) {
    v *= 128.0;
    const double r = rint(v);
    d[t] = (float)r;
    v -= r;
  }
}

// A side: one block per complex row i of op(A) (m x k), thread p < k.
// Out: slices [S][batch][2m][ZK] bf16, sigma [batch][2m].
template <class T, int S>
__global__ void slice_a_kernel(char opa, int m, int k, const T *A, long lda, long sa, int batch,
                               __nv_bfloat16 *out, double *sigma) {
  const int i = blockIdx.x, b = blockIdx.y, p = threadIdx.x;
  const T *Ab = A + (long)b * sa;
  double re = 0.0, im = 0.0;
  if (p < k) {
    T a = (opa == 'N') ? Ab[i + (long)p * lda] : Ab[p + (long)i * lda];
    re = (double)a.x;
    im = (opa == 'C') ? -(double)a.y : (double)a.y;
  }
  double mx = fmax(fabs(re), fabs(im));
  for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  __shared__ double wm[2];
  if ((p & 31) == 0) wm[p >> 5] = mx;
  __syncthreads();
  mx = (blockDim.x > 32) ? fmax(wm[0], wm[1]) : wm[0];
  const double sg = pow2_ceil(mx);
  float dr[S], di[S];
  digits<S>(re / sg, dr);
  digits<S>(im / sg, di);
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
    for (int q = 2 * k + p; q < ZK; q += blockDim.x) {
      r0[q] = __float2bfloat16_rn(0.f);
      r1[q] = __float2bfloat16_rn(0.f);
    }
  }
  if (p == 0) {
    sigma[(long)b * rows + 2 * i] = sg;
    sigma[(long)b * rows + 2 * i + 1] = sg;
  }
}

// B side: one block per column c of op(B) (k x n), thread p < k.
// Out: slices [S][batch][n][ZK] bf16, tau [batch][n].
template <class T, int S>
__global__ void slice_b_kernel(char opb, int k, int n, const T *B, long ldb, long sb, int batch,
                               __nv_bfloat16 *out, double *tau) {
  const int c = blockIdx.x, b = blockIdx.y, p = threadIdx.x;
  const T *Bb = B + (long)b * sb;
  double re = 0.0, im = 0.0;
  if (p < k) {
    T v = (opb == 'N') ? Bb[p + (long)c * ldb] : Bb[c + (long)p * ldb];
    re = (double)v.x;
    im = (opb == 'C') ? -(double)v.y : (double)v.y;
  }
  double mx = fmax(fabs(re), fabs(im));
  for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  __shared__ double wm[2];
  if ((p & 31) == 0) wm[p >> 5] = mx;
  __syncthreads();
  mx = (blockDim.x > 32) ? fmax(wm[0], wm[1]) : wm[0];
  const double tg = pow2_ceil(mx);
  float dr[S], di[S];
  digits<S>(re / tg, dr);
  digits<S>(im / tg, di);
  for (int t = 0; t < S; ++t) {
    __nv_bfloat16 *o = out + (((long)t * batch + b) * n + c) * ZK;
    if (p < k) {
      o[p] = __float2bfloat16_rn(dr[t]);
      o[k + p] = __float2bfloat16_rn(di[t]);
    }
    for (int q = 2 * k + p; q < ZK; q += blockDim.x) o[q] = __float2bfloat16_rn(0.f);
  }
  if (p == 0) tau[(long)b * n + c] = tg;
}

// Instruction descriptor for N = ZBN.
__host__ __device__ constexpr uint32_t idesc_bf16_n(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

template <int S> struct zlay {
  static constexpr int SMEM = S * (ZA_TILE + ZB_TILE) + 1024 + 256;
  static constexpr int ACC = S;  // weights 2 .. S+1
  static constexpr int COLS = (S * ZBN <= 32) ? 32 : (S * ZBN <= 64) ? 64 : (S * ZBN <= 128) ? 128 : 256;
};

template <class T, int S>
__global__ void __launch_bounds__(THREADS, 1)
    zgemm_sliced_kernel(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, int m,
                        int n, int batch, const double *sigma, const double *tau, double alpha, int beta_one,
                        T *C, long ldc, long sc, int *gerr) {
  using R = typename cplx_io<T>::R;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *sA = base;                        // S x [128][64] bf16
  unsigned char *sB = base + S * ZA_TILE;          // S x [ZBN][64] bf16
  uint64_t *full = reinterpret_cast<uint64_t *>(base + S * (ZA_TILE + ZB_TILE));
  uint64_t *accb = full + 1;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(accb + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rows = 2 * m;
  const int r0 = blockIdx.x * BM, n0 = blockIdx.y * ZBN, b = blockIdx.z;
  constexpr uint32_t NCOLS = zlay<S>::COLS;

  if (threadIdx.x == 0) {
    mbar_init(full, 1);
    mbar_init(accb, 1);
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
    mbar_expect_tx(full, S * (ZA_TILE + ZB_TILE));
    for (int t = 0; t < S; ++t) {
      tma_load_3d(sA + t * ZA_TILE, &ta, full, 0, r0, t * batch + b);
      tma_load_3d(sB + t * ZB_TILE, &tb, full, 0, n0, t * batch + b);
    }
    mbar_drain(full, 0, gerr, 12);
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = idesc_bf16_n(ZBN);
    if (mbar_wait(full, 0, abort_flag, gerr, 13)) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      uint32_t used = 0;  // accumulator a (weight a + 2) already written
#pragma unroll
      for (int t = 0; t < S; ++t)
#pragma unroll
        for (int u = 0; u < S; ++u) {
          if (t + u > S - 1) continue;  // digits 1-based: (t+1)+(u+1) <= S+1
          const int a = t + u;
          const uint64_t ad = sdesc_sw128(sm_u32(sA + t * ZA_TILE));
          const uint64_t bd = sdesc_sw128(sm_u32(sB + u * ZB_TILE));
#pragma unroll
          for (int kk = 0; kk < ZK / 16; ++kk) {
            const uint32_t acc = ((used >> a) & 1u) || kk > 0 ? 1u : 0u;
            mma_bf16(tmem + (uint32_t)(a * ZBN), ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), idesc, acc);
          }
          used |= 1u << a;
        }
    }
    mma_commit(accb);
    mbar_drain(accb, 0, gerr, 14);
  } else if (warp >= 2) {
    const int q = warp & 3;
    int okw = 0;
    if (lane == 0) okw = mbar_wait(accb, 0, abort_flag, gerr, 15) ? 1 : 0;
    const bool ok = __shfl_sync(0xffffffffu, okw, 0) != 0;
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
      const int rr = r0 + q * 32 + lane;  // real row
      const double sg = (rr < rows) ? sigma[(long)b * rows + rr] : 0.0;
      // The weight sums S_a (exact integers below 2^24, weight 2^{-7(a+2)})
      // are recombined in 64-bit integers (Horner in base 2^7, two words so
      // nothing overflows), leaving a handful of FP64 operations per entry:
      //   x = hi 2^{7(S-H)} + lo,  value = sigma tau 2^{-7(S+1)} x.
      constexpr int H = (S + 1) / 2 < 3 ? (S + 1) / 2 : 3;
      const double base_scale = alpha * sg * ldexp(1.0, -7 * (S + 1));
      const double hi_w = ldexp(1.0, 7 * (S - H));
      for (int c0 = 0; c0 < ZBN; c0 += 16) {
        long long hi[16], lo[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) hi[j] = lo[j] = 0;
#pragma unroll
        for (int a = 0; a < S; ++a) {
          uint32_t r[16];
          const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * ZBN + c0);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
              "[%16];"
              : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                "=r"(r[15])
              : "r"(taddr));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const long long v = (long long)__float2int_rn(__uint_as_float(r[j]));
            if (a < H)
              hi[j] = hi[j] * 128 + v;
            else
              lo[j] = lo[j] * 128 + v;
          }
        }
        if (rr < rows) {
          const int i = rr >> 1, part = rr & 1;
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int col = n0 + c0 + j;
            if (col < n) {
              const double x = fma((double)hi[j], hi_w, (double)lo[j]);
              const double val = base_scale * tau[(long)b * n + col] * x;
              R *cp = reinterpret_cast<R *>(C + (long)b * sc + i + (long)col * ldc) + part;
              *cp = (R)(beta_one ? (double)*cp + val : val);
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

template <class T, int S>
static int zgemm_sliced_run(cudaStream_t st, char opa, char opb, int m, int n, int k, double alpha, const T *A,
                            long lda, long sa, const T *B, long ldb, long sb, int beta_one, T *C, long ldc, long sc,
                            int batch, void *work, size_t work_bytes, int *gerr) {
  if (k < 1 || k > ZK / 2) {
    set_error("sliced GEMM: k must be in [1, 32]");
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
  double *sg = (double *)(w + al(a_bytes) + al(b_bytes));
  double *tg = (double *)(w + al(a_bytes) + al(b_bytes) + al(s_bytes));
  slice_a_kernel<T, S><<<dim3(m, batch), 64, 0, st>>>(opa, m, k, A, lda, sa, batch, As, sg);
  slice_b_kernel<T, S><<<dim3(n, batch), 64, 0, st>>>(opb, k, n, B, ldb, sb, batch, Bs, tg);
  g_launches.fetch_add(2, std::memory_order_relaxed);
  CUtensorMap ta, tb;
  if (int rc = make_map_rows(&ta, As, rows, S * batch, BM)) return rc;
  if (int rc = make_map_rows(&tb, Bs, n, S * batch, ZBN)) return rc;
  static bool attr = false;
  if (!attr) {
    GBF_CUDA(cudaFuncSetAttribute(zgemm_sliced_kernel<T, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  zlay<S>::SMEM));
    attr = true;
  }
  dim3 grid(ceil_div(rows, BM), ceil_div(n, ZBN), batch);
  zgemm_sliced_kernel<T, S><<<grid, THREADS, zlay<S>::SMEM, st>>>(ta, tb, m, n, batch, sg, tg, alpha, beta_one, C,
                                                                   ldc, sc, gerr);
  GBF_LAUNCHED();
  GBF_CUDA(cudaGetLastError());
  return 0;
}

}  // namespace tc

size_t zgemm_sliced_work(int m, int n, int batch, int S) {
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
    return tc::zgemm_sliced_run<T, 7>(st, opa, opb, m, n, k, alpha, A, lda, sa, B, ldb, sb, beta_one, C, ldc, sc,
                                      batch, work, work_bytes, gerr);
  if (S == 3)
    return tc::zgemm_sliced_run<T, 3>(st, opa, opb, m, n, k, alpha, A, lda, sa, B, ldb, sb, beta_one, C, ldc, sc,
                                      batch, work, work_bytes, gerr);
  set_error("sliced GEMM: S must be 3 or 7");
  return -4;
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

// ===================================================================
// No-allocation variant of gbf_zgemm_sliced.
//
// For callers that must not allocate device memory during the call: code
// whose device memory is owned by another allocator (a framework's caching
// pool holding the whole budget), latency-critical paths that cannot afford
// the device-wide synchronisation cudaMalloc/cudaFree imply, and sequences
// that will later be recorded into a CUDA graph.  The scratch this GEMM needs
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
