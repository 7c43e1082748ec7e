// Shared device/host helpers of the CUDA path (complex types, launch
// bookkeeping, kernel entry points used across translation units).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <atomic>
#include <mutex>
#include <unordered_map>

namespace gbf {

// ---------------------------------------------------------------- complex --
struct __align__(16) zd {
  double x, y;
};
struct __align__(8) cf {
  float x, y;
};

__host__ __device__ inline zd mkz(double a, double b) { return zd{a, b}; }
__host__ __device__ inline cf mkc(float a, float b) { return cf{a, b}; }

// Scalar traits: real double, complex double (zd), complex float (cf).
template <class T> struct tr;
template <> struct tr<double> {
  using R = double;
  static constexpr bool cplx = false;
  __host__ __device__ static double zero() { return 0.0; }
  __host__ __device__ static double one() { return 1.0; }
  __host__ __device__ static double conj(double a) { return a; }
  __host__ __device__ static double mul(double a, double b) { return a * b; }
  __host__ __device__ static double fma(double a, double b, double c) { return ::fma(a, b, c); }
  __host__ __device__ static double add(double a, double b) { return a + b; }
  __host__ __device__ static double sub(double a, double b) { return a - b; }
  __host__ __device__ static double re(double a) { return a; }
  __host__ __device__ static double abs1(double a) { return fabs(a); }
  __host__ __device__ static double neg(double a) { return -a; }
};
template <> struct tr<zd> {
  using R = double;
  static constexpr bool cplx = true;
  __host__ __device__ static zd zero() { return zd{0.0, 0.0}; }
  __host__ __device__ static zd one() { return zd{1.0, 0.0}; }
  __host__ __device__ static zd conj(zd a) { return zd{a.x, -a.y}; }
  __host__ __device__ static zd mul(zd a, zd b) { return zd{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
  // a*b + c
  __host__ __device__ static zd fma(zd a, zd b, zd c) {
    c.x = ::fma(a.x, b.x, c.x);
    c.x = ::fma(-a.y, b.y, c.x);
    c.y = ::fma(a.x, b.y, c.y);
    c.y = ::fma(a.y, b.x, c.y);
    return c;
  }
  __host__ __device__ static zd add(zd a, zd b) { return zd{a.x + b.x, a.y + b.y}; }
  __host__ __device__ static zd sub(zd a, zd b) { return zd{a.x - b.x, a.y - b.y}; }
  __host__ __device__ static double re(zd a) { return a.x; }
  __host__ __device__ static double abs1(zd a) { return fabs(a.x) + fabs(a.y); }
  __host__ __device__ static zd neg(zd a) { return zd{-a.x, -a.y}; }
};
template <> struct tr<cf> {
  using R = float;
  static constexpr bool cplx = true;
  __host__ __device__ static cf zero() { return cf{0.f, 0.f}; }
  __host__ __device__ static cf one() { return cf{1.f, 0.f}; }
  __host__ __device__ static cf conj(cf a) { return cf{a.x, -a.y}; }
  __host__ __device__ static cf mul(cf a, cf b) { return cf{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
  __host__ __device__ static cf fma(cf a, cf b, cf c) {
    c.x = fmaf(a.x, b.x, c.x);
    c.x = fmaf(-a.y, b.y, c.x);
    c.y = fmaf(a.x, b.y, c.y);
    c.y = fmaf(a.y, b.x, c.y);
    return c;
  }
  __host__ __device__ static cf add(cf a, cf b) { return cf{a.x + b.x, a.y + b.y}; }
  __host__ __device__ static cf sub(cf a, cf b) { return cf{a.x - b.x, a.y - b.y}; }
  __host__ __device__ static float re(cf a) { return a.x; }
  __host__ __device__ static float abs1(cf a) { return fabsf(a.x) + fabsf(a.y); }
  __host__ __device__ static cf neg(cf a) { return cf{-a.x, -a.y}; }
};

// Complex double arithmetic used by host and device helpers.
__host__ __device__ inline zd zmul(zd a, zd b) { return tr<zd>::mul(a, b); }
// 1/d and 1/sqrt(x) for the serial scalar steps of the reduced-space
// kernels (a pivot's reciprocal, a reflector's norm), where one thread's
// chain of dependent FP64 instructions is the critical path: the hardware's
// approximate value (about 20 correct bits) refined by two steps of
// Newton's iteration, r <- r + r (1 - d r) for the reciprocal and
// y <- y (3/2 - (x/2) y^2) for the reciprocal square root: a few ulp, in
// fewer dependent instructions than a division or a square root.  Outside
// [2^-1000, 2^1000] in magnitude (and for zero, non-finite or, for the
// square root, non-positive input) the exact operations are used.
__device__ __forceinline__ bool fast_range(double v) {
  const int eb = (int)((__double_as_longlong(v) >> 52) & 0x7FF);
  return eb > 23 && eb < 2023;
}
__device__ __forceinline__ double fast_rcp(double d) {
  if (!fast_range(d)) return 1.0 / d;
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
  r = fma(r, fma(-d, r, 1.0), r);
  return fma(r, fma(-d, r, 1.0), r);
}
__device__ __forceinline__ double fast_rsqrt(double x) {
  if (!(x > 0.0) || !fast_range(x)) return 1.0 / sqrt(x);
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double h = 0.5 * x;
  y = y * fma(-h * y, y, 1.5);
  return y * fma(-h * y, y, 1.5);
}

__host__ __device__ inline zd zdiv(zd a, zd b) {
  // Smith's algorithm (scaled division)
  if (fabs(b.x) >= fabs(b.y)) {
    double r = b.y / b.x, d = b.x + b.y * r;
    return zd{(a.x + a.y * r) / d, (a.y - a.x * r) / d};
  } else {
    double r = b.x / b.y, d = b.x * r + b.y;
    return zd{(a.x * r + a.y) / d, (a.y * r - a.x) / d};
  }
}
__host__ __device__ inline double zabs(zd a) { return hypot(a.x, a.y); }

// Conversions between the arithmetic types.
template <class D, class S> __host__ __device__ inline D cvt(S s);
template <> __host__ __device__ inline zd cvt<zd, zd>(zd s) { return s; }
template <> __host__ __device__ inline cf cvt<cf, zd>(zd s) { return cf{(float)s.x, (float)s.y}; }
template <> __host__ __device__ inline zd cvt<zd, cf>(cf s) { return zd{(double)s.x, (double)s.y}; }
template <> __host__ __device__ inline cf cvt<cf, cf>(cf s) { return s; }
template <> __host__ __device__ inline zd cvt<zd, double>(double s) { return zd{s, 0.0}; }
template <> __host__ __device__ inline cf cvt<cf, double>(double s) { return cf{(float)s, 0.f}; }
template <> __host__ __device__ inline double cvt<double, double>(double s) { return s; }

// ------------------------------------------------------------ bookkeeping --
// Number of kernels launched through this library (all launches go through
// the GBF_LAUNCHED macro after a <<<>>> launch).
extern std::atomic<long long> g_launches;
#define GBF_LAUNCHED() (::gbf::g_launches.fetch_add(1, std::memory_order_relaxed))

// Last error text for gbf_last_error(); set by the host driver.
void set_error(const char *fmt, ...);

#define GBF_CUDA(call)                                                               \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      ::gbf::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
      return -4;                                                                     \
    }                                                                                \
  } while (0)

inline int ceil_div(long a, long b) { return (int)((a + b - 1) / b); }

// Runs f() (which returns 0 or an error code) once per device for the
// device current on the calling thread: kernel attributes such as the
// dynamic shared-memory limit are per device, so a process-wide flag would
// leave a second device without them.  Thread-safe; ordinals >= 64 run f()
// on every call.
template <class F>
int once_per_device(std::atomic<unsigned long long> &mask, F f) {
  int dev = 0;
  GBF_CUDA(cudaGetDevice(&dev));
  const unsigned long long bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
  if (bit && (mask.load(std::memory_order_acquire) & bit)) return 0;
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  if (bit && (mask.load(std::memory_order_acquire) & bit)) return 0;
  if (int rc = f()) return rc;
  mask.fetch_or(bit, std::memory_order_acq_rel);
  return 0;
}

// -------------------------------------------------------------- profiling --
// Optional per-category timing of launches (gbf_profile): a CUDA event pair
// on the launching stream around each instrumented launch, with the
// algorithmic flop count of that launch; summed by gbf_profile_read.
enum Cat {
  CAT_LU_UPDATE = 0,  // trailing update GEMM of the blocked LU
  CAT_LU_PANEL,       // panel factorisation
  CAT_LU_SWAP,        // row swaps outside the panel + U12 solve
  CAT_SOLVE,          // GEMM steps of the triangular solves
  CAT_PROJECT,        // n-sized FP64 GEMMs of the Rayleigh-Ritz step
  CAT_REDUCED,        // M0-sized GEMMs + Jacobi rounds
  CAT_OTHER,          // everything else (shift, gather, accumulate, ...)
  CAT_COUNT
};
extern thread_local int g_cat;
struct CatScope {
  int prev;
  explicit CatScope(int c) : prev(g_cat) { g_cat = c; }
  ~CatScope() { g_cat = prev; }
};
bool prof_on();
int prof_begin(cudaStream_t st);                      // slot or -1
void prof_end(cudaStream_t st, int slot, double flops);
// same for a sliced tensor-core GEMM kernel: useful flops and issued bf16 tensor flops
void prof_end_tc(cudaStream_t st, int slot, double flops, double tensor_flops);
void prof_set_flops(int slot, double flops);  // flops known only after the launch

// ------------------------------------------------------------------ GEMM --
// Tensor-core engine for complex GEMMs with k <= 32 (LU trailing updates and
// solve steps): while a TcScope is active on this thread, gemm<zd> / gemm<cf>
// calls that fit (k <= 32, alpha = +-1, beta in {0, 1}, m and n large
// enough) run on the tensor cores using the scope's workspace and error
// word: S = 7 sliced digits (FP64-class) for zd, S = 1 3xTF32 products
// (FP32-class) for cf.
struct SliceCache;
struct TcCtx {
  void *work = nullptr;
  size_t bytes = 0;
  int *gerr = nullptr;
  int S = 0;
  void *kwork = nullptr;  // workspace of the any-k sliced GEMMs of the recursive solves
  size_t kbytes = 0;
  void *dinv_l = nullptr;  // inverses of the 128 x 128 diagonal blocks of L and U (FP64
  void *dinv_u = nullptr;  // factors, n a multiple of 128): the recursive solves' leaves
  const float *fpre_n = nullptr;  // FP32 factors split once into TF32 planes, op 'N' and op 'C'
  const float *fpre_c = nullptr;  // (tf32_presplit; nullptr: every update splits its operand)
  int fpre_ne = 0;                // nodes in the planes
  SliceCache *acache = nullptr;   // FP64 factors: digit slices of the solves' factor blocks, kept
                                  // from the first solve of a factorisation for the later ones
};
// Workspace bytes of the recursive solves' any-k sliced updates for n x n
// factors, nrhs right-hand sides, block size bs (node groups of up to 8).
size_t solve_kwork_bytes(int n, int nrhs, int bs, int ne);
// The same for FP32 factors (3xTF32 any-k updates of the recursive solves).
size_t solve_kwork_bytes_cf(int n, int nrhs, int bs, int ne);
// Bytes of the factor-block slices of nkinds recursive FP64 sweeps (the
// SliceCache of TcCtx; leaves128: the 128-row leaf inverses are used).
size_t solve_slice_cache_bytes(int n, int nrhs, int bs, int ne, int nkinds, bool leaves128);
extern thread_local TcCtx *g_tc;
// Side stream (high priority) and two events of the calling context, for
// the factorisation's look-ahead: panel k+1 runs there while the rest of
// panel k's trailing update runs on the main stream.
struct AuxStreams {
  cudaStream_t s = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
};
extern thread_local AuxStreams *g_aux;
struct AuxScope {
  AuxStreams *prev;
  explicit AuxScope(AuxStreams *x) : prev(g_aux) { g_aux = x; }
  ~AuxScope() { g_aux = prev; }
};
struct TcScope {
  TcCtx *prev;
  explicit TcScope(TcCtx *c) : prev(g_tc) { g_tc = c; }
  ~TcScope() { g_tc = prev; }
};
// Operand sliced for the any-k sliced GEMM: digit planes (bf16) of the rows
// of op(A) (or columns of op(B)), per-row exponents, rows, padded K.
struct SlicedOp {
  const void *slices;
  const int *exps;
  long rows;
  long Kp;
};
// Slices of operands that stay fixed across calls (the factor blocks of the
// recursive solves: the same blocks in every FEAST iteration), in a region
// of the caller's workspace, looked up by (address, op, shape, batch).
// Cleared when the factors change.  A block that no longer fits is sliced
// per call as before.
struct SliceKey {
  const void *A;
  long lda, sa;
  int m, k, batch;
  char op;
  bool operator==(const SliceKey &o) const {
    return A == o.A && lda == o.lda && sa == o.sa && m == o.m && k == o.k && batch == o.batch && op == o.op;
  }
};
struct SliceKeyHash {
  size_t operator()(const SliceKey &s) const {
    uint64_t h = (uint64_t)(uintptr_t)s.A;
    h = h * 0x9E3779B97F4A7C15ULL ^ (uint64_t)s.lda;
    h = h * 0x9E3779B97F4A7C15ULL ^ (uint64_t)s.sa;
    h = h * 0x9E3779B97F4A7C15ULL ^ ((uint64_t)(unsigned)s.m << 32 | (uint64_t)(unsigned)s.k);
    h = h * 0x9E3779B97F4A7C15ULL ^ ((uint64_t)(unsigned)s.batch << 8 | (uint64_t)(unsigned char)s.op);
    return (size_t)(h ^ (h >> 29));
  }
};
struct SliceCache {
  char *base = nullptr;
  size_t cap = 0, used = 0;
  std::unordered_map<SliceKey, SlicedOp, SliceKeyHash> ops;  // exact keys: no collisions
  void reset() {
    used = 0;
    ops.clear();
  }
};
long sliced_kp(int k, bool cplx);
size_t sliced_op_bytes(long rows, long Kp, int batch);
template <class T>
int slice_rows(cudaStream_t st, char op, int m, int k, const T *A, long lda, long sa, int batch, void *buf,
               SlicedOp *out);
template <class T>
int slice_cols(cudaStream_t st, char op, int k, int n, const T *B, long ldb, long sb, int batch, void *buf,
               SlicedOp *out);
template <class T>
int gemm_sliced_ops(cudaStream_t st, const SlicedOp &a, const SlicedOp &b, int batch, double alpha, int beta_one,
                    T *C, long ldc, long sc, int *gerr);
size_t gemm_sliced_k_work(bool cplx, int m, int n, int k, int batch);
template <class T>
int gemm_sliced_k(cudaStream_t st, char opa, char opb, int m, int n, int k, double alpha, const T *A, long lda,
                  long sa, const T *B, long ldb, long sb, int beta_one, T *C, long ldc, long sc, int batch, void *work,
                  size_t work_bytes, int *gerr);
size_t zgemm_sliced_work(int m, int n, int batch, int S);
// 3xTF32 complex FP32 GEMM for any k on the tensor cores (the FP32 factors'
// large-K solve updates): C = alpha op(A) op(B) + beta C, alpha = +-1, beta
// in {0, 1}; work: cgemm_tf32k_work bytes (the split TF32 planes).
size_t cgemm_tf32k_work(int m, int n, int k, int batch);
// TF32 hi/lo planes of op(S) (op 'N' or 'C') for ne complex FP32 n x n
// matrices (node stride n^2), in the any-k 3xTF32 GEMM's A layout, and the
// product C -= op(S)[r0 .. r0+m, 32 c0 .. 32 c0 + k] Y read from them (nodes
// b0 .. b0 + batch - 1 of bt; only Y is split per call).
size_t tf32_planes_bytes(int n, int ne);
int tf32_presplit(cudaStream_t st, char op, int n, int ne, const cf *S, float *planes);
size_t cgemm_tf32k_pre_work(int n, int k, int batch);
int cgemm_tf32k_pre(cudaStream_t st, int m, int n, int k, double alpha, const float *pre, int nfull, int bt, int b0,
                    int r0, int c0, const cf *B, long ldb, long sb, int beta_one, cf *C, long ldc, long sc, int batch,
                    void *work, size_t work_bytes, int *gerr);
int cgemm_tf32k(cudaStream_t st, char opa, char opb, int m, int n, int k, double alpha, const cf *A, long lda, long sa,
                const cf *B, long ldb, long sb, int beta_one, cf *C, long ldc, long sc, int batch, void *work,
                size_t work_bytes, int *gerr);
template <class T>
int zgemm_sliced(cudaStream_t st, int S, char opa, char opb, int m, int n, int k, double alpha, const T *A, long lda,
                 long sa, const T *B, long ldb, long sb, int beta_one, T *C, long ldc, long sc, int batch, void *work,
                 size_t work_bytes, int *gerr);

// C = alpha * op(A) * op(B) + beta * C, column-major, strided batches.
// op: 'N' (as stored), 'T' (transpose), 'C' (conjugate transpose).
// A is m x k after op, B is k x n after op.  When ksplit > 1 the k range is
// split into ksplit chunks whose partial products go to `work` (ksplit *
// batch * m * n elements) and are summed in chunk order by a second kernel.
template <class T>
int gemm(cudaStream_t st, char opa, char opb, int m, int n, int k, T alpha, const T *A, long lda,
         long sa, const T *B, long ldb, long sb, T beta, T *C, long ldc, long sc, int batch,
         int ksplit = 1, T *work = nullptr);

// ------------------------------------------------------ LU / solve (lu.cu) --
// Form S_e = z_e B - A for all nodes (B == nullptr: B = I) in type T.
// kindA: 0 real input (double), 1 complex input (zd). uplo: 'F','L','U'
// (Hermitian: the referenced triangle, a real diagonal) or 'G' (a general
// matrix, every entry as stored).
// bad (may be null): set to 1 when a referenced entry of A or B is not finite.
template <class T>
int form_shift(cudaStream_t st, int n, int ne, const zd *z, int kindA, char uplo, const void *A,
               long lda, const void *B, long ldb, T *S, int *bad = nullptr);

// Blocked right-looking LU with partial pivoting of ne matrices (stride n*n,
// ld n).  ipiv 0-based absolute rows (ne x n).  perm receives the final row
// permutation (P b)[i] = b[perm[i]].  Linv/Uinv receive inverted diagonal
// blocks (bs x bs each, n/bs rounded up per node).  sing: per-node first
// zero pivot (0 = none).
template <class T>
int getrf_batched(cudaStream_t st, int n, int ne, T *S, int *ipiv, int *perm, T *Linv, T *Uinv,
                  int bs, int *sing, T *gemm_work);

// Solve S_e Y_e = P-gathered RHS for all nodes (trans 0) or S_e^H Y_e = RHS
// (trans 1).  Y: ne x (n x nrhs), ld n.  The RHS gather is done by the caller
// (gather kernels below); this applies the triangular solves in place.
template <class T>
int getrs_inplace(cudaStream_t st, int trans, int n, int ne, int nrhs, const T *S, const T *Linv,
                  const T *Uinv, int bs, T *Y, T *tmp);

// Y_e[i, j] = RHS[perm_e[i], j] * scale_e[j]  (scale may be null => 1).
// RHS kind: 0 real double, 1 complex double.  Output type T.
template <class T>
int gather_rhs(cudaStream_t st, int n, int ne, int nrhs, const int *perm, int kindR, const void *RHS,
               long ldr, const zd *scale, T *Y);

// Inverse permutation for adjoint solves: out[perm_e[i], j] = Y_e[i, j] (in place via tmp).
template <class T>
int scatter_perm(cudaStream_t st, int n, int ne, int nrhs, const int *perm, const T *Yin, T *Yout);

// ------------------------------------------------------------ eig (eig.cu) --
// Hermitian (T = zd) or real symmetric (T = double) Jacobi eigensolver of an
// m x m matrix A (ld m, overwritten); w ascending (device), V eigenvectors.
// work: 2 m^2 + 2m T; dwork: >= 4m + 8 doubles; iwork: >= 5m + 96 ints (device);
// hflag: pinned host int used to read the per-sweep convergence flag.
template <class T>
int heev_jacobi(cudaStream_t st, int m, T *A, double *w, T *V, T *work, double *dwork, int *iwork, int *hflag,
                int *sweeps_out);

// Reduced Hermitian eigensolver (tridiag.cu): Householder tridiagonalisation
// in one thread-block cluster, bisection, inverse iteration, back-transform.
// A (m x m, ld m, full storage) is not modified; w ascending, V (m x m, ld m)
// eigenvectors.  work: heev_tridiag_work bytes.  Returns 0, 1 when it
// declines (m outside 2..1024 or no cluster shape fits; nothing launched),
// or -4.
size_t heev_tridiag_work(int m, bool cplx);
template <class T> int heev_tridiag(cudaStream_t st, int m, const T *A, double *w, T *V, void *work, size_t work_bytes);
// Cholesky A = L L^H of an m x m Hermitian matrix (full storage, ld m, not
// modified) in one thread-block cluster; fail = first non-positive pivot + 1.
// Returns 0, or 1 when the cluster kernel cannot take m (nothing launched).
template <class T> int chol_cluster(cudaStream_t st, int m, const T *A, T *L, int *fail);

// Small dense FP64 kernels (small.cu): cooperative Cholesky (A = L L^H, A
// overwritten as workspace, fail = first non-positive pivot + 1), inverse of
// a lower triangular matrix, and the Jacobi eigensolver core.
template <class T> int chol_lower(cudaStream_t st, int m, T *A, T *L, int *fail);
template <class T> int trinv_lower(cudaStream_t st, int m, const T *L, T *Linv, double *rd /* m scratch */);
template <class T> int jacobi_coop(cudaStream_t st, int m, int maxsw, T *A, T *V, T *work, double *dw, int *iw);

// Rayleigh-Ritz glue (eig.cu).
template <class T>
int rr_prepare(cudaStream_t st, int m, const T *Aq, const T *Bq, double *s, int *flag, T *As, T *Bs);
template <class T>
int make_t(cudaStream_t st, int m, int mk, int first, const T *V, const double *d, T *Tm);
template <class T> int hermitize(cudaStream_t st, int m, const T *Cin, T *Cout);
template <class T> int scale_rows(cudaStream_t st, int m, int mk, const double *s, T *W);
template <class T>
int ritz_residual(cudaStream_t st, int n, int mk, const T *AX, const T *BX, const double *lam, double alpha,
                  double *res);
int order_and_stats(cudaStream_t st, int mk, const double *lam, const double *res, const int *spur, double emin,
                    double emax, int *pos, int *nin, double *E, double *R, double *stats);
template <class T>
int spurious_flags(cudaStream_t st, int m, int mk, const T *W, const double *lam, double emin, double emax,
                   const double *f, int check, int *spur);
template <class T> int permute_cols(cudaStream_t st, int n, int m, const int *pos, const T *in, T *out);
int filter_values(cudaStream_t st, int mk, int ne, const zd *z, const zd *w, const double *lam, double *f, zd *D,
                  zd *Dc);
template <class T>
int eig_residual(cudaStream_t st, int n, int mk, const T *AX, const T *BX, const double *lam, T *R);
template <class TY, class TQ>
int accumulate(cudaStream_t st, int n, int m, int ne, const zd *w, const TY *Y, const TY *Yadj, const TQ *X0,
               const double *f, TQ *Q);
template <class TQ> int random_subspace(cudaStream_t st, long count, uint64_t seed, TQ *Y);
// Stochastic eigenvalue count (fpm(14)=2): +-1 probes from the same counter
// generator, and res(j) = mean over probes 1..j of Re(y^H q) (device res).
template <class TQ> int rademacher_probes(cudaStream_t st, long count, uint64_t seed, TQ *Y);
template <class TQ> int probe_running_mean(cudaStream_t st, int n, int m, const TQ *Y, const TQ *Q, double *res);
template <class T> int ns_prep(cudaStream_t st, int m, const T *P, T *Tn, double *norm);

// ----------------------------------------- non-Hermitian FEAST (gen.cu) --
// Elementwise glue of the dual-subspace iteration (n x m column-major, ld n).
int gen_widen(cudaStream_t st, int n, const double *A, long lda, zd *Af);
int gen_conj_pair(cudaStream_t st, int n, int m, const zd *src, zd *dst);
// Q = X0 diag(g) + the sum over the nf factored nodes of c_e Y_e (+ the
// mirror node's term conj(c_e Y_e[:, m..2m)) when `half`), c_e = w_e and
// g = f, or conj(w_e) and conj(f) when `left` (X0 null: no first term).
template <class TY>
int gen_accumulate(cudaStream_t st, int n, int m, int nf, const zd *w, const TY *Y, int mw, int half, int left,
                   const zd *X0, const zd *f, zd *Q);
// Residual-correction form: per-node column scales of the right and left
// right-hand sides and the filter values f(lam) of the Ritz values.
int gen_scales(cudaStream_t st, int m, int nf, int ne, const zd *z, const zd *w, const zd *lam, int half, zd *SCr,
               zd *SCl, zd *f);
// R = MX - NX diag(lam or conj(lam)), columns divided by sc (sc null: 1).
int gen_eig_residual(cudaStream_t st, int n, int m, const zd *MX, const zd *NX, const zd *lam, int conjl,
                     const double *sc, zd *R);
int gen_col_norms(cudaStream_t st, int n, int m, const zd *X, double *nrm);
int gen_col_scale(cudaStream_t st, int n, int m, const zd *src, zd *dst, const double *s, int divide);
int gen_residual(cudaStream_t st, int n, int m, const zd *MX, const zd *NX, const zd *lam, int conjl, double alpha,
                 double *res);
int gen_order(cudaStream_t st, int m, const zd *lam, const double *rr, const double *rl, zd emid, double r,
              double rho, double angle_deg, int *pos, int *src, zd *Eo, double *Rr, double *Rl, double *stats);
int gen_biorth(cudaStream_t st, int m, int nin, const zd *P, const double *nr, const int *src, double *out);
int gen_identity(cudaStream_t st, int m, zd *I);
// Reduced non-Hermitian eigensolver steps (m x m, ld m): Hessenberg form
// with Z accumulated; complex Schur form by shifted QR (err = 1: no
// convergence); eigenvectors of the triangular factor.
int gen_hessenberg(cudaStream_t st, int m, zd *G, zd *Z);
int gen_hqr(cudaStream_t st, int m, zd *H, zd *Z, zd *lam, int *err);
int gen_trevc(cudaStream_t st, int m, const zd *T, zd *Y);

}  // namespace gbf
