// Register-tiled SIMT GEMM for the FP64 path (real and complex double) and
// the FP32-complex factor/solve path: C = alpha op(A) op(B) + beta C,
// column-major, strided batches over contour nodes, optional split-K for the
// tall-skinny reductions of the Rayleigh-Ritz projection (Q^H (A Q)).
//
// Tiles: BM x BN per CTA, BK deep, staged in shared memory; each thread owns
// a TM x TN register block whose rows/columns are interleaved with stride
// BM/TM and BN/TN so that global stores and shared-memory reads are unit
// stride across a warp.
#include <type_traits>

#include "gbf_common.cuh"

namespace gbf {

thread_local TcCtx *g_tc = nullptr;
thread_local AuxStreams *g_aux = nullptr;

template <class T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
    gemm_kernel(int m, int n, int k, T alpha, const T *__restrict__ A, long lda, long sa,
                const T *B, long ldb, long sb, T beta, int beta_zero, T *C, long ldc,
                long sc, char opa, char opb, int kchunk, int batch, T *work) {
  using X = tr<T>;
  constexpr int NT = (BM / TM) * (BN / TN);
  constexpr int RX = BM / TM;  // threads along rows
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int zb = blockIdx.z;
  const int bi = zb % batch, kc = zb / batch;
  const int k0 = kc * kchunk;
  const int k1 = min(k, k0 + kchunk);
  A += (long)bi * sa;
  B += (long)bi * sb;
  const int i0 = blockIdx.x * BM, j0 = blockIdx.y * BN;
  const int tid = threadIdx.x;
  const int tx = tid % RX, ty = tid / RX;
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = X::zero();

  for (int kk = k0; kk < k1; kk += BK) {
    for (int e = tid; e < BM * BK; e += NT) {
      int ii, pp;
      if (opa == 'N') {
        ii = e % BM;
        pp = e / BM;
      } else {
        pp = e % BK;
        ii = e / BK;
      }
      const int gi = i0 + ii, gp = kk + pp;
      T v = X::zero();
      if (gi < m && gp < k1) {
        if (opa == 'N')
          v = A[gi + (long)gp * lda];
        else if (opa == 'T')
          v = A[gp + (long)gi * lda];
        else
          v = X::conj(A[gp + (long)gi * lda]);
      }
      As[pp][ii] = v;
    }
    for (int e = tid; e < BN * BK; e += NT) {
      int jj, pp;
      if (opb == 'N') {
        pp = e % BK;
        jj = e / BK;
      } else {
        jj = e % BN;
        pp = e / BN;
      }
      const int gj = j0 + jj, gp = kk + pp;
      T v = X::zero();
      if (gj < n && gp < k1) {
        if (opb == 'N')
          v = B[gp + (long)gj * ldb];
        else if (opb == 'T')
          v = B[gj + (long)gp * ldb];
        else
          v = X::conj(B[gj + (long)gp * ldb]);
      }
      Bs[pp][jj] = v;
    }
    __syncthreads();
#pragma unroll
    for (int pp = 0; pp < BK; ++pp) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[pp][tx + i * RX];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[pp][ty + j * (BN / TN)];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = X::fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }

#pragma unroll
  for (int j = 0; j < TN; ++j) {
    const int gj = j0 + ty + j * (BN / TN);
    if (gj >= n) continue;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int gi = i0 + tx + i * RX;
      if (gi >= m) continue;
      T v = X::mul(alpha, acc[i][j]);
      if (work) {
        work[((long)kc * batch + bi) * (long)m * n + gi + (long)gj * m] = v;
      } else {
        T *cp = C + (long)bi * sc + gi + (long)gj * ldc;
        if (!beta_zero) v = X::fma(beta, *cp, v);
        *cp = v;
      }
    }
  }
}

template <class T>
__global__ void splitk_reduce(int m, int n, int ksplit, int batch, const T *__restrict__ work, T beta,
                              int beta_zero, T *C, long ldc, long sc) {
  using X = tr<T>;
  const long mn = (long)m * n;
  const long total = mn * batch;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const int bi = (int)(t / mn);
    const long r = t - (long)bi * mn;
    const int i = (int)(r % m), j = (int)(r / m);
    T s = X::zero();
    for (int kc = 0; kc < ksplit; ++kc) s = X::add(s, work[((long)kc * batch + bi) * mn + r]);
    T *cp = C + (long)bi * sc + i + (long)j * ldc;
    if (!beta_zero) s = X::fma(beta, *cp, s);
    *cp = s;
  }
}

template <class T> struct gemm_cfg;
template <> struct gemm_cfg<double> { static constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4; };
template <> struct gemm_cfg<zd> { static constexpr int BM = 64, BN = 64, BK = 8, TM = 4, TN = 4; };
template <> struct gemm_cfg<cf> { static constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4; };

template <class T> static bool is_zero(T v);
template <> bool is_zero<double>(double v) { return v == 0.0; }
template <> bool is_zero<zd>(zd v) { return v.x == 0.0 && v.y == 0.0; }
template <> bool is_zero<cf>(cf v) { return v.x == 0.f && v.y == 0.f; }

// real scalar +-1 / 0-1 tests for the sliced tensor-core path
template <class T> static bool sliced_ok(T alpha, T beta, double &a, int &b);
template <> bool sliced_ok<zd>(zd alpha, zd beta, double &a, int &b) {
  if (alpha.y != 0.0 || (alpha.x != 1.0 && alpha.x != -1.0) || beta.y != 0.0 || (beta.x != 0.0 && beta.x != 1.0))
    return false;
  a = alpha.x;
  b = beta.x != 0.0;
  return true;
}
template <> bool sliced_ok<cf>(cf alpha, cf beta, double &a, int &b) {
  if (alpha.y != 0.f || (alpha.x != 1.f && alpha.x != -1.f) || beta.y != 0.f || (beta.x != 0.f && beta.x != 1.f))
    return false;
  a = alpha.x;
  b = beta.x != 0.f;
  return true;
}

constexpr long TF32_MIN_ENTRIES = 8L << 20;

template <class T>
int gemm(cudaStream_t st, char opa, char opb, int m, int n, int k, T alpha, const T *A, long lda, long sa,
         const T *B, long ldb, long sb, T beta, T *C, long ldc, long sc, int batch, int ksplit, T *work) {
  if (m <= 0 || n <= 0 || batch <= 0) return 0;
  if constexpr (tr<T>::cplx) {
    double a = 0.0;
    int b1 = 0;
    TcCtx *tcx = g_tc;
    // S = 1 (3xTF32) serves the FP32 factors, the digit counts the FP64 ones.
    // 3xTF32 adds a splitting launch and writes C at the memory rate, while
    // the FP32 CUDA-core kernel at k = 32 is bound by its FMA rate: the
    // tensor cores pay off once C holds a few million entries (the large
    // trailing updates and the solves of large problems).
    const bool tf32 = tcx && tcx->S == 1;
    const bool kind_ok = tcx && (tf32 == std::is_same<T, cf>::value) &&
                         (!tf32 || (long)m * n * batch >= TF32_MIN_ENTRIES);
    if (kind_ok && tcx->S != 0 && k >= 1 && k <= 32 && m >= 16 && n >= 16 && sliced_ok<T>(alpha, beta, a, b1) &&
        zgemm_sliced_work(m, n, batch, tcx->S) <= tcx->bytes) {
      return zgemm_sliced<T>(st, tcx->S, opa, opb, m, n, k, a, A, lda, sa, B, ldb, sb, b1, C, ldc, sc, batch,
                             tcx->work, tcx->bytes, tcx->gerr);
    }
  }
  using G = gemm_cfg<T>;
  if (ksplit < 1 || !work) ksplit = 1;
  int kchunk = k;
  if (ksplit > 1) {
    kchunk = ceil_div(ceil_div(k, ksplit), G::BK) * G::BK;
    ksplit = ceil_div(k, kchunk);
    if (ksplit <= 1) {
      ksplit = 1;
      kchunk = k;
    }
  }
  if (kchunk < 1) kchunk = 1;
  dim3 grid(ceil_div(m, G::BM), ceil_div(n, G::BN), batch * ksplit);
  const int nt = (G::BM / G::TM) * (G::BN / G::TN);
  const int slot = prof_begin(st);
  gemm_kernel<T, G::BM, G::BN, G::BK, G::TM, G::TN><<<grid, nt, 0, st>>>(
      m, n, k, alpha, A, lda, sa, B, ldb, sb, beta, is_zero(beta) ? 1 : 0, C, ldc, sc, opa, opb, kchunk,
      batch, ksplit > 1 ? work : nullptr);
  GBF_LAUNCHED();
  if (ksplit > 1) {
    long total = (long)m * n * batch;
    int blocks = (int)std::min<long>((total + 255) / 256, 152L * 8);
    splitk_reduce<T><<<blocks, 256, 0, st>>>(m, n, ksplit, batch, work, beta, is_zero(beta) ? 1 : 0, C, ldc, sc);
    GBF_LAUNCHED();
  }
  prof_end(st, slot, (tr<T>::cplx ? 8.0 : 2.0) * m * (double)n * k * batch);
  GBF_CUDA(cudaGetLastError());
  return 0;
}

template int gemm<double>(cudaStream_t, char, char, int, int, int, double, const double *, long, long,
                          const double *, long, long, double, double *, long, long, int, int, double *);
template int gemm<zd>(cudaStream_t, char, char, int, int, int, zd, const zd *, long, long, const zd *, long,
                      long, zd, zd *, long, long, int, int, zd *);
template int gemm<cf>(cudaStream_t, char, char, int, int, int, cf, const cf *, long, long, const cf *, long,
                      long, cf, cf *, long, long, int, int, cf *);

}  // namespace gbf
