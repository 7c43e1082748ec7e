// Host driver and C ABI of the FEAST hot path (see include/gbfeast.h).
//
// One call runs, on the caller's stream (FEAST v3.0 guide: "The FEAST
// Algorithm" summary, RCI loop of Fig. "fig_rci", outputs of Table
// "tab_common", info codes of Table "tab_info"):
//   nodes/weights (host) -> S_e = z_e B - A and LU for all nodes (kept) ->
//   loop k: RHS = B Y -> Y_e = S_e^{-1} RHS (+ adjoint solves for complex
//   Hermitian) -> Q = sum_e w_e Y_e (fused quadrature sum) -> AQ, BQ,
//   Aq = Q^H A Q, Bq = Q^H B Q -> B-orthonormalise + reduced eigenproblem ->
//   X = Q W, AX, BX -> residuals, ordering, trace -> convergence.
// Every n-sized step runs in this library's kernels; the host reads back a
// few scalars per iteration (Jacobi sweep flags, the M0 eigenvalues of the
// scaled Q^H B Q, and M / trace / max residual) to steer the loop.
//
// Mixed precision (fpm(42)=1): factors and solves in complex FP32.  The first
// contour solves S_e Y_e = B Y in FP32.  Later contours use the identity
//   S_e^{-1} B X = X (z_e - Lambda)^{-1} + S_e^{-1} R (z_e - Lambda)^{-1},
//   R = A X - B X Lambda  (FP64, from the previous Rayleigh-Ritz step),
// so Q = X f(Lambda) + sum_e Re[w_e S_e^{-1} R D_e] (Hermitian: the adjoint
// pair), and the FP32 solve error is proportional to ||R||, which the
// subspace iteration drives to FP64 rounding level.
#include <math.h>
#include <stdarg.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "gbf_common.cuh"
#include "gbfeast.h"

namespace gbf {
std::atomic<long long> g_launches{0};
static std::mutex g_err_mu;
static char g_err[1024] = "";
void set_error(const char *fmt, ...) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}
}  // namespace gbf

using namespace gbf;

static const uint64_t SUBSPACE_SEED = 0x3C6EF372FE94F82BULL;
static const double PI_ = 3.14159265358979323846264338327950288;

struct gbf_context {
  int device = 0;
  char *arena = nullptr;
  size_t cap = 0;
  int *hflag = nullptr;       // pinned
  double *hbuf = nullptr;     // pinned scratch
  size_t hbuf_cap = 0;
  cudaStream_t own = nullptr;  // stream of the host-pointer entries
  AuxStreams aux;              // look-ahead side stream and events (created on first use)
  // factors kept by gbf_factor_dev
  int f_n = 0, f_ne = 0, f_prec = -1, f_bs = 32;
  size_t f_bytes = 0;
  double gen_biorth = 0.0;  // bi-orthonormality defect of the last converged non-Hermitian solve
};

// ------------------------------------------------------------ quadrature --
// Legendre roots by Newton iteration from cos(pi (i + 3/4) / (ne + 1/2)),
// with P_ne from the three-term recurrence and P'_ne from
// (x^2 - 1) P'_n = n (x P_n - P_{n-1}); weights 2 / ((1 - x^2) P'_n^2).
static void gl_nodes(int ne, double *x, double *om) {
  for (int i = 0; i < ne; ++i) {
    double t = cos(PI_ * (i + 0.75) / (ne + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;
      for (int k = 2; k <= ne; ++k) {
        const double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (ne == 1) p0 = 1.0;
      dp = ne * (t * p1 - p0) / (t * t - 1.0);
      const double dt = p1 / dp;
      t -= dt;
      if (fabs(dt) < 1e-16) break;
    }
    double p0 = 1.0, p1 = t;
    for (int k = 2; k <= ne; ++k) {
      const double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = ne * (t * p1 - p0) / (t * t - 1.0);
    x[ne - 1 - i] = t;
    om[ne - 1 - i] = 2.0 / ((1.0 - t * t) * dp * dp);
  }
}

static int make_contour(double emin, double emax, int ne, int qtype, int ratio, zd *z, zd *w) {
  if (!(emin < emax)) return 200;
  if (ne < 1) return 102;
  if (qtype != 0 && qtype != 1) return 116;
  if (ratio <= 0) return 118;
  std::vector<double> x(ne), om(ne);
  if (qtype == 0) {
    gl_nodes(ne, x.data(), om.data());
  } else {
    for (int e = 0; e < ne; ++e) {
      x[e] = 1.0 - 2.0 * (ne - e - 0.5) / ne;
      om[e] = 2.0 / ne;
    }
  }
  const double r0 = 0.5 * (emin + emax), R = 0.5 * (emax - emin), rho = ratio / 100.0;
  for (int e = 0; e < ne; ++e) {
    const double t = 0.5 * PI_ * (1.0 - x[e]);
    z[e] = zd{r0 + R * cos(t), rho * R * sin(t)};
    w[e] = zd{0.5 * om[e] * R * rho * cos(t), 0.5 * om[e] * R * sin(t)};
  }
  return 0;
}

static int check_fpm(const int *fpm) {
  const int ne = fpm[1], qtype = fpm[15];
  if (qtype != 0 && qtype != 1) return 116;
  if (qtype == 0) {
    const bool ok = (ne >= 1 && ne <= 20) || ne == 24 || ne == 32 || ne == 40 || ne == 48 || ne == 56;
    if (!ok) return 102;
  } else if (ne < 1) {
    return 102;
  }
  if (fpm[2] < 0 || fpm[2] > 16) return 103;
  if (fpm[3] < 0) return 104;
  if (fpm[4] != 0 && fpm[4] != 1) return 105;
  if (fpm[5] != 0 && fpm[5] != 1) return 106;
  if (fpm[13] != 0 && fpm[13] != 1 && fpm[13] != 2) return 114;
  if (fpm[17] <= 0) return 118;
  if (fpm[41] != 0 && fpm[41] != 1) return 142;
  if (fpm[42] != 0 && (fpm[42] < 8 || fpm[42] > 64 || fpm[42] % 8)) return 143;
  if (fpm[43] != 0 && fpm[43] != 1) return 144;
  return 0;
}

// ----------------------------------------------------------------- arena --
struct Bump {
  char *base;
  size_t off = 0;
  explicit Bump(char *b) : base(b) {}
  template <class T> T *take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    T *p = reinterpret_cast<T *>(base + off);
    off += count * sizeof(T) + 16;
    return p;
  }
};

static int ensure_arena(gbf_context *h, size_t need) {
  if (h->cap >= need) return 0;
  if (h->arena) {
    cudaDeviceSynchronize();
    cudaFree(h->arena);
    h->arena = nullptr;
    h->cap = 0;
  }
  cudaError_t e = cudaMalloc((void **)&h->arena, need);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc of %zu bytes failed: %s", need, cudaGetErrorString(e));
    h->arena = nullptr;
    return -1;
  }
  h->cap = need;
  h->f_prec = -1;  // any stored factors are gone
  return 0;
}

static int ensure_hbuf(gbf_context *h, size_t count) {
  if (h->hbuf_cap >= count) return 0;
  if (h->hbuf) cudaFreeHost(h->hbuf);
  h->hbuf = nullptr;
  if (cudaMallocHost((void **)&h->hbuf, count * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMallocHost failed");
    h->hbuf_cap = 0;
    return -1;
  }
  h->hbuf_cap = count;
  return 0;
}

// --------------------------------------------------------- small kernels --
template <class TQ>
__global__ void expand_uplo_kernel(int n, char uplo, const TQ *A, long lda, TQ *F) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= n) return;
  const bool mirror = (uplo == 'L' && i < j) || (uplo == 'U' && i > j);
  TQ v = mirror ? tr<TQ>::conj(A[j + (long)i * lda]) : A[i + (long)j * lda];
  if (i == j) v = cvt<TQ, double>(tr<TQ>::re(v));
  F[i + (long)j * n] = v;
}

template <class TQ>
__global__ void copy_cols_kernel(int n, int m, const TQ *src, long lds, TQ *dst, long ldd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i < n && j < m) dst[i + (long)j * ldd] = src[i + (long)j * lds];
}

// out = in^H (m x m)
template <class TQ>
__global__ void copy_t_kernel(int m, const TQ *in, TQ *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i < m) out[i + (long)j * m] = tr<TQ>::conj(in[j + (long)i * m]);
}

template <class TL>
__global__ void widen_kernel(long count, const TL *src, zd *dst) {
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t < count) dst[t] = cvt<zd, TL>(src[t]);
}

// ---------------------------------------------------------------- driver --
template <class TQ> struct kind_of;
template <> struct kind_of<double> { static constexpr int v = 0; };
template <> struct kind_of<zd> { static constexpr int v = 1; };

struct Req {
  char uplo;
  int n;
  const void *A;
  long lda;
  const void *B;
  long ldb;
  const int *fpm;
  double emin, emax;
  int m0;
  const double *Zne, *Wne;
  double *E;
  void *X;
  double *res;
  const gbf_shard *sh;  // node sharding across processes, or null
};
struct Res {
  double epsout = 1.0;
  int loop = 0, M = 0, m0 = 0, info = 0;
};

// The context's look-ahead stream and events, created once; null (no
// look-ahead) if they cannot be made.
static AuxStreams *ensure_aux(gbf_context *h) {
  if (!h->aux.s) {
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (cudaStreamCreateWithPriority(&h->aux.s, cudaStreamNonBlocking, hi) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->aux.a, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->aux.b, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
  }
  return &h->aux;
}

template <class TQ, class TL> struct WS {
  TL *S, *Linv, *Uinv, *Ysol, *Yadj, *Ytmp;
  int *ipiv, *perm, *sing, *pos, *nin, *iwork, *flag, *spur;
  TQ *Af, *Bf, *Q, *AQ, *BQ, *Xc, *AXc, *BXc, *Xu, *AXu, *BXu, *R, *RHS;
  TQ *Aq, *Bq, *As, *Bs, *V, *Tm, *Ctmp, *Cm, *Cs, *U, *W, *jwork, *kwork;
  double *d, *lam, *s, *resu, *Es, *Rs, *f, *dwork, *stats;
  zd *z, *w, *D, *Dc;
  void *tcw;
  size_t tcw_bytes;
  int *tc_err;
  void *pja, *pjb, *pjq;  // sliced operands of the projections: A, B (rows), Q / Y (columns)
  void *pjh, *pjx, *pjw;  // Q^H (rows), Q / AQ / BQ (rows, for X = Q W), W (columns)
  void *rrw;              // both operands of the M0 x M0 x M0 reduced-space products
  size_t rrw_bytes;
  void *trw;              // reduced eigensolver (tridiagonal route)
  size_t trw_bytes;
  void *kw;               // any-k sliced updates of the recursive solves
  size_t kw_bytes;
  TL *dinv_l, *dinv_u;    // 128 x 128 diagonal-block inverses (recursive solves' leaves)
  float *fpre_n, *fpre_c; // TF32 planes of the FP32 factors (op N, op C), split once
  char *acache_base;      // FP64 factors: digit slices of the solves' factor blocks
  size_t acache_bytes;
  SliceCache acache;

  // ne: quadrature nodes; nf: nodes factored and solved here (all of them,
  // or this shard's share); slots: node solution blocks (ne, or nranks x the
  // share size so the blocks can be exchanged in equal chunks)
  void layout(Bump &b, int n, int m0, int ne, int nf, int slots, int bs, bool herm, bool hasB, bool needAf,
              bool needBf, int ksplit, int tcS, bool proj) {
    const size_t nn = (size_t)n * n, nm = (size_t)n * m0, mm = (size_t)m0 * m0;
    const int nblk = ceil_div(n, bs);
    const int nfa = std::max(nf, 1);
    S = b.take<TL>((size_t)nfa * nn);
    Linv = b.take<TL>((size_t)nfa * nblk * bs * bs);
    Uinv = b.take<TL>((size_t)nfa * nblk * bs * bs);
    Ysol = b.take<TL>((size_t)slots * nm);
    Yadj = herm ? b.take<TL>((size_t)slots * nm) : nullptr;
    Ytmp = herm ? b.take<TL>((size_t)nfa * nm) : nullptr;
    ipiv = b.take<int>((size_t)nfa * n);
    perm = b.take<int>((size_t)nfa * n);
    sing = b.take<int>(nfa + 1);  // + the non-finite-input flag
    pos = b.take<int>(m0);
    spur = b.take<int>(m0);
    nin = b.take<int>(4);
    iwork = b.take<int>(5 * m0 + 96);
    flag = b.take<int>(4);
    Af = needAf ? b.take<TQ>(nn) : nullptr;
    Bf = needBf ? b.take<TQ>(nn) : nullptr;
    Q = b.take<TQ>(nm);
    AQ = b.take<TQ>(nm);
    BQ = hasB ? b.take<TQ>(nm) : nullptr;
    Xc = b.take<TQ>(nm);
    AXc = b.take<TQ>(nm);
    BXc = hasB ? b.take<TQ>(nm) : nullptr;
    Xu = b.take<TQ>(nm);
    AXu = b.take<TQ>(nm);
    BXu = hasB ? b.take<TQ>(nm) : nullptr;
    R = b.take<TQ>(nm);
    RHS = hasB ? b.take<TQ>(nm) : nullptr;
    Aq = b.take<TQ>(mm);
    Bq = b.take<TQ>(mm);
    As = b.take<TQ>(mm);
    Bs = b.take<TQ>(mm);
    V = b.take<TQ>(mm);
    Tm = b.take<TQ>(mm);
    Ctmp = b.take<TQ>(mm);
    Cm = b.take<TQ>(mm);
    Cs = b.take<TQ>(mm);
    U = b.take<TQ>(mm);
    W = b.take<TQ>(mm);
    jwork = b.take<TQ>(2 * mm + 2 * m0);
    kwork = b.take<TQ>((size_t)std::max(ksplit, 1) * mm);
    d = b.take<double>(m0);
    lam = b.take<double>(m0);
    s = b.take<double>(m0);
    resu = b.take<double>(m0);
    Es = b.take<double>(m0);
    Rs = b.take<double>(m0);
    f = b.take<double>(m0);
    dwork = b.take<double>(8 + 4 * m0);
    stats = b.take<double>(8);
    z = b.take<zd>(ne);
    w = b.take<zd>(ne);
    D = b.take<zd>((size_t)ne * m0);
    Dc = b.take<zd>((size_t)ne * m0);
    tcw_bytes = tcS ? std::max(zgemm_sliced_work(n, n, nfa, tcS), zgemm_sliced_work(n, m0, nfa, tcS)) : 0;
    tcw = tcS ? (void *)b.take<char>(tcw_bytes) : nullptr;
    tc_err = b.take<int>(4);
    kw_bytes = !tcS ? 0 : (sizeof(TL) == sizeof(zd) ? solve_kwork_bytes(n, m0, bs, nfa)
                                                     : solve_kwork_bytes_cf(n, m0, bs, nfa));
    kw = kw_bytes ? (void *)b.take<char>(kw_bytes) : nullptr;
    const bool big = kw_bytes && sizeof(TL) == sizeof(zd) && bs == 32 && n % 128 == 0;
    dinv_l = big ? b.take<TL>((size_t)nfa * n * 128) : nullptr;
    dinv_u = big ? b.take<TL>((size_t)nfa * n * 128) : nullptr;
    // FP32 factors of large problems: TF32 planes split once per
    // factorisation for the solves' large-K updates (op N; op C for the
    // adjoint solves of Hermitian problems)
    const bool pre = kw_bytes && sizeof(TL) == sizeof(cf) && n >= 1024;
    fpre_n = pre ? b.take<float>(tf32_planes_bytes(n, nfa) / 4) : nullptr;
    fpre_c = pre && herm ? b.take<float>(tf32_planes_bytes(n, nfa) / 4) : nullptr;
    // FP64 factors: the factor blocks' slices, kept across the FEAST
    // iterations (sweeps L, U, and for adjoint solves U^H, L^H), at most 24 GB
    acache_bytes = (kw_bytes && sizeof(TL) == sizeof(zd))
                       ? std::min(solve_slice_cache_bytes(n, m0, bs, nfa, herm ? 4 : 2, big), (size_t)24 << 30)
                       : 0;
    acache_base = acache_bytes ? b.take<char>(acache_bytes) : nullptr;
    pja = pjb = pjq = pjh = pjx = pjw = rrw = nullptr;
    rrw_bytes = 0;
    if (proj) {
      const bool cx = sizeof(TQ) == sizeof(zd);
      const long Kp = sliced_kp(n, cx), R = cx ? 2L * n : n;
      const long Km = sliced_kp(m0, cx), Rm = cx ? 2L * m0 : m0;
      pja = b.take<char>(sliced_op_bytes(R, Kp, 1));
      pjb = hasB ? (void *)b.take<char>(sliced_op_bytes(R, Kp, 1)) : nullptr;
      pjq = b.take<char>(sliced_op_bytes(m0, Kp, 1));
      pjh = b.take<char>(sliced_op_bytes(Rm, Kp, 1));
      pjx = b.take<char>(sliced_op_bytes(R, Km, 1));
      pjw = b.take<char>(sliced_op_bytes(m0, Km, 1));
    }
    rrw_bytes = proj ? gemm_sliced_k_work(sizeof(TQ) == sizeof(zd), m0, m0, m0, 1) : 0;
    rrw = proj ? (void *)b.take<char>(rrw_bytes) : nullptr;
    trw_bytes = heev_tridiag_work(m0, sizeof(TQ) == sizeof(zd));
    trw = b.take<char>(trw_bytes);
  }
};

static int pick_ksplit(int m, int k) {
  const int tiles = ceil_div(m, 64) * ceil_div(m, 64);
  int ks = ceil_div(4 * 152, tiles);
  ks = std::min(ks, std::max(1, k / 128));
  return std::max(ks, 1);
}

// Share of the quadrature nodes of shard `rank` of `nranks`: the nodes are
// dealt out in contiguous blocks of chunk = ceil(ne / nranks), so shard r
// holds nodes [r chunk, min(ne, (r+1) chunk)) and every shard's node
// solutions form one equal-sized chunk of the exchanged buffer.
static void shard_share(int ne, int rank, int nranks, int *lo, int *cnt, int *chunk) {
  const int c = ceil_div(ne, nranks);
  const int a = std::min(ne, rank * c);
  *lo = a;
  *cnt = std::min(ne, a + c) - a;
  *chunk = c;
}

// Combine a status code over all shards (the agreement callback returns the
// minimum, so an error anywhere stops every shard at the same point).
static int shard_agree(const gbf_shard *sh, int code) {
  int c = code;
  if (sh->agree(sh->user, &c) != 0) {
    set_error("node sharding: the agreement callback failed");
    return -4;
  }
  if (c != code && code == 0) set_error("node sharding: another shard stopped with info %d", c);
  return c;
}

static int shard_allgather(const gbf_shard *sh, cudaStream_t st, void *buf, size_t chunk_bytes) {
  if (sh->allgather(sh->user, (void *)st, buf, chunk_bytes) != 0) {
    set_error("node sharding: the all-gather callback failed");
    return -4;
  }
  return 0;
}

#define CK(...)                            \
  do {                                     \
    int rc_ = (__VA_ARGS__);               \
    if (rc_) {                             \
      out.info = rc_ == -1 ? -1 : -4;      \
      return out.info;                     \
    }                                      \
  } while (0)

template <class TQ, class TL>
static int feast_run(gbf_context *h, cudaStream_t st, const Req &q, Res &out) {
  using XQ = tr<TQ>;
  const int n = q.n, m0 = q.m0;
  const int *fpm = q.fpm;
  const bool herm = kind_of<TQ>::v == 1;
  const bool hasB = q.B != nullptr;
  const bool mixed = fpm[41] == 1;
  const int ne = fpm[1];
  const int bs = fpm[42] ? fpm[42] : 32;
  // nodes factored and solved here: all, or this shard's [nlo, nlo + nf)
  const gbf_shard *sh = q.sh;
  int nlo = 0, nf = ne, chunk = ne, slots = ne;
  if (sh) {
    shard_share(ne, sh->rank, sh->nranks, &nlo, &nf, &chunk);
    slots = chunk * sh->nranks;
  }
  const int nfa = std::max(nf, 1);
  const double eps = pow(10.0, -fpm[2]);
  const double alpha = std::max(fabs(q.emin), fabs(q.emax));
  out = Res{};
  out.m0 = m0;

  // contour
  std::vector<zd> zh(ne), wh(ne);
  if (q.Zne && q.Wne) {
    for (int e = 0; e < ne; ++e) {
      zh[e] = zd{q.Zne[2 * e], q.Zne[2 * e + 1]};
      wh[e] = zd{q.Wne[2 * e], q.Wne[2 * e + 1]};
    }
  } else {
    const int rc = make_contour(q.emin, q.emax, ne, fpm[15], fpm[17], zh.data(), wh.data());
    if (rc) return out.info = rc;
  }

  // workspace
  const bool needAf = q.uplo != 'F';
  const bool needBf = hasB && q.uplo != 'F';
  const int ksplit = pick_ksplit(m0, n);
  // complex GEMMs of the FP64 factorisation and solves on the tensor cores
  // (7-digit sliced products, FP64-class) unless fpm(44) = 1.  FP32 factors
  // stay on CUDA cores: both FP32-class tensor-core variants (4 digits; bf16
  // three-part split with FP32 sums) were slower here, and one small complex
  // Hermitian case did not converge with them
  // tensor-core engine: 7-digit sliced products for FP64 factors, 3xTF32
  // for FP32 factors (k <= 32 needs the block size <= 32)
  const int tcS = (fpm[43] == 0 && bs <= 32) ? (sizeof(TL) == sizeof(zd) ? 7 : 1) : 0;
  // the n x n products of the projections (A Q, B Q, B Y): sliced tensor-core
  // GEMMs with A and B sliced once per call, unless fpm(44) = 1
  const bool proj = fpm[43] == 0;
  WS<TQ, TL> ws;
  {
    Bump sizing(nullptr);
    ws.layout(sizing, n, m0, ne, nf, slots, bs, herm, hasB, needAf, needBf, ksplit, tcS, proj);
    if (ensure_arena(h, sizing.off + 4096)) return out.info = -1;
    Bump real(h->arena);
    ws.layout(real, n, m0, ne, nf, slots, bs, herm, hasB, needAf, needBf, ksplit, tcS, proj);
  }
  TcCtx tcx;
  tcx.work = ws.tcw;
  tcx.bytes = ws.tcw_bytes;
  tcx.gerr = ws.tc_err;
  tcx.S = tcS;
  tcx.kwork = ws.kw;
  tcx.kbytes = ws.kw_bytes;
  tcx.dinv_l = ws.dinv_l;
  tcx.dinv_u = ws.dinv_u;
  tcx.fpre_n = ws.fpre_n;
  tcx.fpre_c = ws.fpre_c;
  tcx.fpre_ne = ws.fpre_n ? std::max(nf, 1) : 0;
  ws.acache.base = ws.acache_base;
  ws.acache.cap = ws.acache_bytes;
  ws.acache.reset();
  tcx.acache = ws.acache_bytes ? &ws.acache : nullptr;
  TcScope tc_scope(tcS ? &tcx : nullptr);
  AuxScope aux_scope(ensure_aux(h));
  if (ensure_hbuf(h, (size_t)std::max(m0, ne) + 64)) return out.info = -1;
  h->f_prec = -1;

  GBF_CUDA(cudaMemcpyAsync(ws.z, zh.data(), sizeof(zd) * ne, cudaMemcpyHostToDevice, st));
  GBF_CUDA(cudaMemcpyAsync(ws.w, wh.data(), sizeof(zd) * ne, cudaMemcpyHostToDevice, st));
  GBF_CUDA(cudaMemsetAsync(ws.sing, 0, sizeof(int) * (nfa + 1), st));
  GBF_CUDA(cudaMemsetAsync(ws.tc_err, 0, sizeof(int) * 4, st));
  GBF_CUDA(cudaMemsetAsync(ws.flag, 0, sizeof(int) * 4, st));

  const TQ *Af = (const TQ *)q.A;
  long lda = q.lda;
  const TQ *Bf = (const TQ *)q.B;
  long ldb = q.ldb;
  if (needAf) {
    expand_uplo_kernel<TQ><<<dim3(ceil_div(n, 256), n), 256, 0, st>>>(n, q.uplo, (const TQ *)q.A, q.lda, ws.Af);
    GBF_LAUNCHED();
    Af = ws.Af;
    lda = n;
  }
  if (needBf) {
    expand_uplo_kernel<TQ><<<dim3(ceil_div(n, 256), n), 256, 0, st>>>(n, q.uplo, (const TQ *)q.B, q.ldb, ws.Bf);
    GBF_LAUNCHED();
    Bf = ws.Bf;
    ldb = n;
  }

  // factor all nodes (kept for the whole iteration)
  CatScope cat_other(CAT_OTHER);
  if (nf > 0) {
    CK(form_shift<TL>(st, n, nf, ws.z + nlo, kind_of<TQ>::v, 'F', Af, lda, hasB ? (const void *)Bf : nullptr, ldb,
                      ws.S, ws.sing + nfa));
    CK(getrf_batched<TL>(st, n, nf, ws.S, ws.ipiv, ws.perm, ws.Linv, ws.Uinv, bs, ws.sing, nullptr));
    ws.acache.reset();  // slices of these factors are taken by the first solves
    if constexpr (std::is_same<TL, cf>::value) {
      if (ws.fpre_n) CK(tf32_presplit(st, 'N', n, nf, ws.S, ws.fpre_n));
      if (ws.fpre_c) CK(tf32_presplit(st, 'C', n, nf, ws.S, ws.fpre_c));
    }
  }
  {
    int *hs = (int *)h->hbuf;
    GBF_CUDA(cudaMemcpyAsync(hs, ws.sing, sizeof(int) * (nfa + 1), cudaMemcpyDeviceToHost, st));
    GBF_CUDA(cudaMemcpyAsync(hs + nfa + 1, ws.tc_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    GBF_CUDA(cudaStreamSynchronize(st));
    int code = 0;
    if (hs[nfa + 1]) {
      set_error("tensor-core GEMM: bounded wait timed out (code %d)", hs[nfa + 1]);
      code = -4;
    } else if (hs[nfa]) {
      set_error("A or B holds a non-finite entry (NaN or Inf)");
      code = -2;
    } else {
      for (int e = 0; e < nf; ++e)
        if (hs[e]) {
          set_error("zero pivot in column %d of the shifted system of node %d", hs[e], nlo + e);
          code = -2;
          break;
        }
    }
    if (sh) code = shard_agree(sh, code);
    if (code) return out.info = code;
  }

  // rows of A and B (A^T = A, A^H = A: contiguous columns) sliced once
  SlicedOp opA{}, opB{};
  const char opS = herm ? 'C' : 'T';
  if (proj) {
    CatScope cat_pj(CAT_PROJECT);
    CK(slice_rows<TQ>(st, opS, n, n, Af, lda, 0, 1, ws.pja, &opA));
    if (hasB) CK(slice_rows<TQ>(st, opS, n, n, Bf, ldb, 0, 1, ws.pjb, &opB));
  }
  // Y -> op Y for a sliced operand (columns of Y, n x mm)
  auto sliced_product = [&](const SlicedOp &opM, const TQ *Y, int mm, TQ *out_) -> int {
    SlicedOp opY;
    if (int rc = slice_cols<TQ>(st, 'N', n, mm, Y, n, 0, 1, ws.pjq, &opY)) return rc;
    return gemm_sliced_ops<TQ>(st, opM, opY, 1, 1.0, 0, out_, n, 0, ws.tc_err);
  };

  // M0-sized products of the reduced space (B-orthonormalisation, reduced
  // matrix, W): any-k sliced GEMM on the tensor-core engine
  auto rr_gemm = [&](char opa, char opb, int mm, int nn2, int kk, const TQ *A_, int lda_, const TQ *B_, int ldb_,
                     TQ *C_, int ldc_) -> int {
    if (proj)
      return gemm_sliced_k<TQ>(st, opa, opb, mm, nn2, kk, 1.0, A_, lda_, 0, B_, ldb_, 0, 0, C_, ldc_, 0, 1, ws.rrw,
                               ws.rrw_bytes, ws.tc_err);
    return gemm<TQ>(st, opa, opb, mm, nn2, kk, XQ::one(), A_, lda_, 0, B_, ldb_, 0, XQ::zero(), C_, ldc_, 0, 1);
  };

  // initial subspace into Xc (the probes of the stochastic count when fpm(14)=2)
  if (fpm[4] == 1) {
    copy_cols_kernel<TQ><<<dim3(ceil_div(n, 256), m0), 256, 0, st>>>(n, m0, (const TQ *)q.X, n, ws.Xc, n);
    GBF_LAUNCHED();
  } else if (fpm[13] == 2) {
    CK(rademacher_probes<TQ>(st, (long)n * m0, SUBSPACE_SEED, ws.Xc));
  } else {
    CK(random_subspace<TQ>(st, (long)n * m0, SUBSPACE_SEED, ws.Xc));
  }

  const TQ one = XQ::one(), zero = XQ::zero();
  const int kindR = kind_of<TQ>::v;
  int m = m0;
  double trace_prev = 0.0;
  for (int k = 0;; ++k) {
    // ---- spectral projection: Q = sum_e w_e S_e^{-1} B Y (Y = Xc) ----
    const bool rc_form = mixed && k > 0;
    const TQ *rhs;
    const zd *scale = nullptr, *scalec = nullptr;
    if (rc_form) {
      const TQ *BXp = hasB ? ws.BXc : ws.Xc;
      CK(eig_residual<TQ>(st, n, m, ws.AXc, BXp, ws.Es, ws.R));
      CK(filter_values(st, m, ne, ws.z, ws.w, ws.Es, ws.f, ws.D, ws.Dc));
      rhs = ws.R;
      scale = ws.D;
      scalec = ws.Dc;
    } else if (hasB) {
      if (k == 0) {
        if (proj)
          CK(sliced_product(opB, ws.Xc, m, ws.RHS));
        else
          CK(gemm<TQ>(st, 'N', 'N', n, m, n, one, Bf, ldb, 0, ws.Xc, n, 0, zero, ws.RHS, n, 0, 1));
      }
      rhs = (k == 0) ? ws.RHS : ws.BXc;
    } else {
      rhs = ws.Xc;
    }
    // this shard's nodes [nlo, nlo + nf) (all nodes without sharding)
    const size_t nmc = (size_t)n * m;
    if (nf > 0) {
      TL *Yown = ws.Ysol + (size_t)nlo * nmc;
      CK(gather_rhs<TL>(st, n, nf, m, ws.perm, kindR, rhs, n, scale ? scale + (size_t)nlo * m : nullptr, Yown));
      CK(getrs_inplace<TL>(st, 0, n, nf, m, ws.S, ws.Linv, ws.Uinv, bs, Yown, nullptr));
      if (herm) {
        CK(gather_rhs<TL>(st, n, nf, m, nullptr, kindR, rhs, n, scalec ? scalec + (size_t)nlo * m : nullptr,
                          ws.Ytmp));
        CK(getrs_inplace<TL>(st, 1, n, nf, m, ws.S, ws.Linv, ws.Uinv, bs, ws.Ytmp, nullptr));
        CK(scatter_perm<TL>(st, n, nf, m, ws.perm, ws.Ytmp, ws.Yadj + (size_t)nlo * nmc));
      }
    }
    if (sh) {
      // the exchange step: every shard receives every node's solution block,
      // then all of them form the same Q with the node-ordered sum below
      const size_t cb = (size_t)chunk * nmc * sizeof(TL);
      CK(shard_allgather(sh, st, ws.Ysol, cb));
      if (herm) CK(shard_allgather(sh, st, ws.Yadj, cb));
    }
    CK(accumulate<TL, TQ>(st, n, m, ne, ws.w, ws.Ysol, herm ? ws.Yadj : nullptr, rc_form ? ws.Xc : nullptr,
                          rc_form ? ws.f : nullptr, ws.Q));

    if (fpm[13] == 2) {
      // stochastic count (guide section "Stochastic estimate"): Q = f(B^-1 A) Y
      // for +-1 probes Y, so the mean of Re(y^H q) estimates trace f = the
      // count; res(j) = running mean, M = res(M0) rounded, within [0, N],
      // X = the probes, E = 0, info 5
      CK(probe_running_mean<TQ>(st, n, m0, ws.Xc, ws.Q, q.res));
      copy_cols_kernel<TQ><<<dim3(ceil_div(n, 256), m0), 256, 0, st>>>(n, m0, ws.Xc, n, (TQ *)q.X, n);
      GBF_LAUNCHED();
      GBF_CUDA(cudaMemsetAsync(q.E, 0, sizeof(double) * m0, st));
      GBF_CUDA(cudaMemcpyAsync(h->hbuf, q.res + (m0 - 1), sizeof(double), cudaMemcpyDeviceToHost, st));
      GBF_CUDA(cudaStreamSynchronize(st));
      const double mh = std::floor(h->hbuf[0] + 0.5);
      out.M = mh > 0.0 ? (int)std::min(mh, (double)n) : 0;
      out.loop = 0;
      out.m0 = m0;
      return out.info = 5;
    }
    if (fpm[13] == 1) {  // return the subspace after one contour
      GBF_CUDA(cudaMemsetAsync(q.X, 0, sizeof(TQ) * (size_t)n * m0, st));
      copy_cols_kernel<TQ><<<dim3(ceil_div(n, 256), m), 256, 0, st>>>(n, m, ws.Q, n, (TQ *)q.X, n);
      GBF_LAUNCHED();
      GBF_CUDA(cudaMemsetAsync(q.E, 0, sizeof(double) * m0, st));
      GBF_CUDA(cudaMemsetAsync(q.res, 0, sizeof(double) * m0, st));
      GBF_CUDA(cudaStreamSynchronize(st));
      out.loop = k;
      out.m0 = m;
      return out.info = 4;
    }

    // ---- Rayleigh-Ritz ----
    CatScope cat_proj(CAT_PROJECT);
    const TQ *BQ = ws.Q;
    if (proj) {
      SlicedOp opQ;
      CK(slice_cols<TQ>(st, 'N', n, m, ws.Q, n, 0, 1, ws.pjq, &opQ));
      CK(gemm_sliced_ops<TQ>(st, opA, opQ, 1, 1.0, 0, ws.AQ, n, 0, ws.tc_err));
      if (hasB) {
        CK(gemm_sliced_ops<TQ>(st, opB, opQ, 1, 1.0, 0, ws.BQ, n, 0, ws.tc_err));
        BQ = ws.BQ;
      }
    } else {
      CK(gemm<TQ>(st, 'N', 'N', n, m, n, one, Af, lda, 0, ws.Q, n, 0, zero, ws.AQ, n, 0, 1));
      if (hasB) {
        CK(gemm<TQ>(st, 'N', 'N', n, m, n, one, Bf, ldb, 0, ws.Q, n, 0, zero, ws.BQ, n, 0, 1));
        BQ = ws.BQ;
      }
    }
    // split-K chunks, capped by the workspace sized for (ksplit, m0)
    const int ks = std::max(1, std::min(pick_ksplit(m, n), (int)(((size_t)ksplit * m0 * m0) / ((size_t)m * m))));
    if (proj) {  // Q^H sliced once for both products
      SlicedOp opQh, opM;
      CK(slice_rows<TQ>(st, 'C', m, n, ws.Q, n, 0, 1, ws.pjh, &opQh));
      CK(slice_cols<TQ>(st, 'N', n, m, ws.AQ, n, 0, 1, ws.pjq, &opM));
      CK(gemm_sliced_ops<TQ>(st, opQh, opM, 1, 1.0, 0, ws.Aq, m, 0, ws.tc_err));
      CK(slice_cols<TQ>(st, 'N', n, m, BQ, n, 0, 1, ws.pjq, &opM));
      CK(gemm_sliced_ops<TQ>(st, opQh, opM, 1, 1.0, 0, ws.Bq, m, 0, ws.tc_err));
    } else {
      CK(gemm<TQ>(st, 'C', 'N', m, m, n, one, ws.Q, n, 0, ws.AQ, n, 0, zero, ws.Aq, m, 0, 1, ks, ws.kwork));
      CK(gemm<TQ>(st, 'C', 'N', m, m, n, one, ws.Q, n, 0, BQ, n, 0, zero, ws.Bq, m, 0, 1, ks, ws.kwork));
    }
    CK(rr_prepare<TQ>(st, m, ws.Aq, ws.Bq, ws.s, ws.flag, ws.As, ws.Bs));
    // B-orthonormal basis T of span(Q) (scaled): CholeskyQR passes on the
    // scaled Q^H B Q (T <- T L^{-H}, G <- T^H Bs T, until ||G - I||_F is at
    // rounding level, at most 3 passes); when a pivot is not positive or
    // the passes stall, the rank-revealing Jacobi route with truncation.
    int mk = m, first = 0;
    bool ns_done = false;  // "orthonormal basis found without Jacobi"
    int sw_b = -2, sw_c = -2, ns_it = 0;
    double *hd = h->hbuf;
    {
      CatScope cat_red(CAT_REDUCED);
      TQ *G = ws.Ctmp, *Gw = ws.Cm, *L = ws.U, *Li = ws.V, *Tn = ws.W;
      GBF_CUDA(cudaMemcpyAsync(G, ws.Bs, sizeof(TQ) * (size_t)m * m, cudaMemcpyDeviceToDevice, st));
      for (int pass = 0; pass < 3; ++pass) {
        ns_it = pass + 1;
        GBF_CUDA(cudaMemcpyAsync(Gw, G, sizeof(TQ) * (size_t)m * m, cudaMemcpyDeviceToDevice, st));
        GBF_CUDA(cudaMemsetAsync(ws.flag + 1, 0, sizeof(int), st));
        CK(chol_lower<TQ>(st, m, Gw, L, ws.flag + 1));
        CK(trinv_lower<TQ>(st, m, L, Li, ws.resu));
        if (pass == 0) {
          // T = L^{-H}
          copy_t_kernel<TQ><<<dim3(ceil_div(m, 256), m), 256, 0, st>>>(m, Li, ws.Tm);
          GBF_LAUNCHED();
        } else {
          CK(rr_gemm('N', 'C', m, m, m, ws.Tm, m, Li, m, Tn, m));
          GBF_CUDA(cudaMemcpyAsync(ws.Tm, Tn, sizeof(TQ) * (size_t)m * m, cudaMemcpyDeviceToDevice, st));
        }
        // G = T^H Bs T
        CK(rr_gemm('N', 'N', m, m, m, ws.Bs, m, ws.Tm, m, Tn, m));
        CK(rr_gemm('C', 'N', m, m, m, ws.Tm, m, Tn, m, G, m));
        CK(ns_prep<TQ>(st, m, G, (TQ *)nullptr, ws.dwork + 4));
        GBF_CUDA(cudaMemcpyAsync(hd, ws.dwork + 4, sizeof(double), cudaMemcpyDeviceToHost, st));
        GBF_CUDA(cudaMemcpyAsync(h->hflag, ws.flag, sizeof(int) * 2, cudaMemcpyDeviceToHost, st));
        GBF_CUDA(cudaStreamSynchronize(st));
        if (h->hflag[0]) {
          set_error("Q^H B Q has a non-positive diagonal (B not HPD on the subspace)");
          return out.info = -3;
        }
        if (h->hflag[1] || !(hd[0] == hd[0])) break;  // not positive definite: Jacobi route
        // at rounding level (or, after the last pass, at the rounding floor
        // u*kappa of a full-rank basis with kappa below ~1e10, where the
        // truncation route would keep every direction as well)
        if (hd[0] < 1e-13 * m || (pass == 2 && hd[0] < 1e-5)) {
          ns_done = true;
          break;
        }
      }
    }
    if (!ns_done) {
      CK(heev_jacobi<TQ>(st, m, ws.Bs, ws.d, ws.V, ws.jwork, ws.dwork, ws.iwork, h->hflag, &sw_b));
      GBF_CUDA(cudaMemcpyAsync(hd, ws.d, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
      GBF_CUDA(cudaMemcpyAsync(h->hflag, ws.flag, sizeof(int), cudaMemcpyDeviceToHost, st));
      GBF_CUDA(cudaStreamSynchronize(st));
      const double dmax = hd[m - 1];
      if (*h->hflag || !(dmax > 0.0) || !(hd[0] >= -1e-8 * dmax)) {
        set_error("Q^H B Q is not positive definite (B not HPD on the subspace)");
        return out.info = -3;
      }
      while (first < m && !(hd[first] > 1e-12 * dmax)) ++first;
      mk = m - first;
    }
    {
    CatScope cat_red(CAT_REDUCED);
    if (!ns_done) CK(make_t<TQ>(st, m, mk, first, ws.V, ws.d, ws.Tm));
    CK(rr_gemm('N', 'N', m, mk, m, ws.As, m, ws.Tm, m, ws.Ctmp, m));
    CK(rr_gemm('C', 'N', mk, mk, m, ws.Tm, m, ws.Ctmp, m, ws.Cm, mk));
    CK(hermitize<TQ>(st, mk, ws.Cm, ws.Cs));
    {
      // tridiagonal route (one cluster); cyclic Jacobi when it declines
      const int trc = heev_tridiag<TQ>(st, mk, ws.Cs, ws.lam, ws.U, ws.trw, ws.trw_bytes);
      if (trc == 1)
        CK(heev_jacobi<TQ>(st, mk, ws.Cs, ws.lam, ws.U, ws.jwork, ws.dwork, ws.iwork, h->hflag, &sw_c));
      else
        CK(trc);
    }
    CK(rr_gemm('N', 'N', m, mk, mk, ws.Tm, m, ws.U, mk, ws.W, m));
    CK(scale_rows<TQ>(st, m, mk, ws.s, ws.W));
    }
    const TQ *BXu = ws.Xu;
    if (proj) {  // X, AX, BX = (Q, AQ, BQ) W with W sliced once
      SlicedOp opW, opM;
      CK(slice_cols<TQ>(st, 'N', m, mk, ws.W, m, 0, 1, ws.pjw, &opW));
      CK(slice_rows<TQ>(st, 'N', n, m, ws.Q, n, 0, 1, ws.pjx, &opM));
      CK(gemm_sliced_ops<TQ>(st, opM, opW, 1, 1.0, 0, ws.Xu, n, 0, ws.tc_err));
      CK(slice_rows<TQ>(st, 'N', n, m, ws.AQ, n, 0, 1, ws.pjx, &opM));
      CK(gemm_sliced_ops<TQ>(st, opM, opW, 1, 1.0, 0, ws.AXu, n, 0, ws.tc_err));
      if (hasB) {
        CK(slice_rows<TQ>(st, 'N', n, m, ws.BQ, n, 0, 1, ws.pjx, &opM));
        CK(gemm_sliced_ops<TQ>(st, opM, opW, 1, 1.0, 0, ws.BXu, n, 0, ws.tc_err));
        BXu = ws.BXu;
      }
    } else {
      CK(gemm<TQ>(st, 'N', 'N', n, mk, m, one, ws.Q, n, 0, ws.W, m, 0, zero, ws.Xu, n, 0, 1));
      CK(gemm<TQ>(st, 'N', 'N', n, mk, m, one, ws.AQ, n, 0, ws.W, m, 0, zero, ws.AXu, n, 0, 1));
      if (hasB) {
        CK(gemm<TQ>(st, 'N', 'N', n, mk, m, one, ws.BQ, n, 0, ws.W, m, 0, zero, ws.BXu, n, 0, 1));
        BXu = ws.BXu;
      }
    }
    CK(ritz_residual<TQ>(st, n, mk, ws.AXu, BXu, ws.lam, alpha, ws.resu));
    // spurious pairs: from loop 1 on, Y = Xc holds the previous B-orthonormal Ritz vectors
    CK(filter_values(st, mk, ne, ws.z, ws.w, ws.lam, ws.f, ws.D, ws.Dc));
    CK(spurious_flags<TQ>(st, m, mk, ws.W, ws.lam, q.emin, q.emax, ws.f, k >= 1 ? 1 : 0, ws.spur));
    CK(order_and_stats(st, mk, ws.lam, ws.resu, ws.spur, q.emin, q.emax, ws.pos, ws.nin, ws.Es, ws.Rs,
                       ws.stats));
    CK(permute_cols<TQ>(st, n, mk, ws.pos, ws.Xu, ws.Xc));
    CK(permute_cols<TQ>(st, n, mk, ws.pos, ws.AXu, ws.AXc));
    if (hasB) CK(permute_cols<TQ>(st, n, mk, ws.pos, ws.BXu, ws.BXc));
    double *hs = h->hbuf;
    GBF_CUDA(cudaMemcpyAsync(hs, ws.stats, sizeof(double) * 4, cudaMemcpyDeviceToHost, st));
    GBF_CUDA(cudaMemcpyAsync(h->hflag + 2, ws.tc_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    GBF_CUDA(cudaStreamSynchronize(st));
    {
      int code = 0;
      if (h->hflag[2]) {
        set_error("tensor-core GEMM: bounded wait timed out (code %d)", h->hflag[2]);
        code = -4;
      }
      if (sh) code = shard_agree(sh, code);
      if (code) return out.info = code;
    }
    const int nin = (int)hs[0];
    const double trace = hs[1], maxres = hs[2];
    const bool finite = hs[3] != 0.0;
    const double eout = (k == 0) ? 1.0 : fabs(trace - trace_prev) / alpha;
    out.M = nin;
    out.loop = k;
    out.epsout = eout;
    out.m0 = mk;
    if (fpm[0] == 1)  // runtime comments (fpm(1)): one line per loop, as the guide's output
      fprintf(stderr, "%d\t%d\t%.15e\t%.15e\t%.15e\t(M0 %d; B-orth: %s %d; reduced: %s %d)\n", k, nin,
              trace, eout, maxres, mk, ns_done ? "CholeskyQR passes" : "Jacobi sweeps",
              ns_done ? ns_it : sw_b + 1, sw_c == -2 ? "tridiagonal" : "Jacobi sweeps", sw_c + 1);
    int info = -99;
    if (!finite) {
      set_error("non-finite Ritz values or residuals");
      info = -2;
    } else if (nin == 0) {
      info = 1;
    } else if (nin >= m0 && m0 < n) {
      info = 3;
    } else if ((fpm[5] == 0) ? (eout < eps) : (maxres < eps)) {
      info = 0;
    } else if (k >= fpm[3]) {
      info = 2;
    }
    if (info != -99) {
      // outputs: E, res (first mk), X (n x mk), zero past mk
      GBF_CUDA(cudaMemsetAsync(q.E, 0, sizeof(double) * m0, st));
      GBF_CUDA(cudaMemsetAsync(q.res, 0, sizeof(double) * m0, st));
      GBF_CUDA(cudaMemsetAsync(q.X, 0, sizeof(TQ) * (size_t)n * m0, st));
      GBF_CUDA(cudaMemcpyAsync(q.E, ws.Es, sizeof(double) * mk, cudaMemcpyDeviceToDevice, st));
      GBF_CUDA(cudaMemcpyAsync(q.res, ws.Rs, sizeof(double) * mk, cudaMemcpyDeviceToDevice, st));
      GBF_CUDA(cudaMemcpyAsync(q.X, ws.Xc, sizeof(TQ) * (size_t)n * mk, cudaMemcpyDeviceToDevice, st));
      GBF_CUDA(cudaStreamSynchronize(st));
      return out.info = info;
    }
    m = mk;
    trace_prev = trace;
  }
}

// ------------------------------------------------- non-Hermitian driver --
// Full-contour nodes and weights (guide: the gcontour tool).  On z(t) =
// Emid + r e^{i phi} (cos t + i rho sin t), t in [0, 2 pi), the residue
// theorem's (1 / 2 pi i) dz = (r e^{i phi} / 2 pi) (rho cos t + i sin t) dt;
// a rule in t with points t_e, weights pi omega_e (omega summing to 2) gives
// w_e = (omega_e / 2) r e^{i phi} (rho cos t_e + i sin t_e).  Gauss:
// t_e = pi (1 + x_e), x ascending; trapezoidal: t_e = 2 pi (e + 1/2) / ne.
// Node ne-1-e is the mirror image of node e (t -> 2 pi - t).
static int make_gcontour(zd emid, double r, int ne, int qtype, int ratio, int angle, zd *z, zd *w) {
  if (!(r > 0.0)) return 200;
  if (ne < 1 || ne > 1024) return 108;
  if (qtype != 0 && qtype != 1) return 117;
  if (ratio <= 0) return 118;
  if (angle < -180 || angle > 180) return 119;
  std::vector<double> x(ne), om(ne);
  if (qtype == 0) {
    gl_nodes(ne, x.data(), om.data());
  } else {
    for (int e = 0; e < ne; ++e) {
      x[e] = 2.0 * (e + 0.5) / ne - 1.0;
      om[e] = 2.0 / ne;
    }
  }
  const double rho = ratio / 100.0, ph = angle * (PI_ / 180.0);
  const double cr = r * cos(ph), sr = r * sin(ph);
  for (int e = 0; e < ne; ++e) {
    const double t = PI_ * (1.0 + x[e]), c = cos(t), s = rho * sin(t);
    const double tc = rho * cos(t), ts = sin(t);
    z[e] = zd{emid.x + cr * c - sr * s, emid.y + sr * c + cr * s};
    w[e] = zd{0.5 * om[e] * (cr * tc - sr * ts), 0.5 * om[e] * (sr * tc + cr * ts)};
  }
  return 0;
}

struct GenReq {
  int n;
  bool real;  // A, B real (double) instead of complex
  const void *A;
  long lda;
  const void *B;
  long ldb;
  const int *fpm;
  zd emid;
  double r;
  int m0;
  const double *Zne, *Wne;
  double *E;    // 2 m0 doubles: complex eigenvalues
  double *X;    // complex n x 2 m0: right vectors, then left ones
  double *res;  // 2 m0: right residuals, then left ones
};

// Non-Hermitian FEAST on the dense pencil (A, B) (guide section "From v2.1
// to v3.0": dual subspaces; Table tab_ijob, cases 10/11/21/30/31/40/41),
// FP64 factors on the tensor-core engine.  Each iteration:
//   Q  = sum_e w_e       S_e^{-1} B Y,    Q^ = sum_e conj(w_e) S_e^{-H} B^H Y^
//   Aq = Q^^H A Q, Bq = Q^^H B Q; Aq W = Bq W Lambda, V = (Bq W)^{-H}
//   X = Q W (unit columns), X^ = Q^ V (scaled so that X^^H B X = I),
//   residuals of Table tab_common, next Y = X, Y^ = X^ with unit columns.
// For real A, B, a real centre, no rotation and an even node count, node
// ne-1-e is the mirror image of node e and S_{ne-1-e} = conj(S_e): only the
// upper half is factored, each solve taking [b, conj(b)], and the mirror
// node's term is conj(c_e S_e^{-1} conj(b)).
template <class TL>
static int feast_run_gen(gbf_context *h, cudaStream_t st, const GenReq &q, Res &out) {
  constexpr bool mixed = std::is_same<TL, cf>::value;  // FP32 factors, FP64 residual correction
  const int n = q.n, m0 = q.m0;
  const int *fpm = q.fpm;
  const bool hasB = q.B != nullptr;
  const int ne = fpm[7];
  const int bs = fpm[42] ? fpm[42] : 32;
  const double eps = pow(10.0, -fpm[2]);
  const double alpha = hypot(q.emid.x, q.emid.y) + q.r;
  out = Res{};
  out.m0 = m0;
  std::vector<zd> zh(ne), wh(ne);
  if (q.Zne && q.Wne) {
    for (int e = 0; e < ne; ++e) {
      zh[e] = zd{q.Zne[2 * e], q.Zne[2 * e + 1]};
      wh[e] = zd{q.Wne[2 * e], q.Wne[2 * e + 1]};
    }
  } else {
    const int rc = make_gcontour(q.emid, q.r, ne, fpm[16], fpm[17], fpm[18], zh.data(), wh.data());
    if (rc) return out.info = rc;
  }
  const bool half = q.real && !(q.Zne && q.Wne) && q.emid.y == 0.0 && fpm[18] == 0 && ne % 2 == 0;
  const int nf = half ? ne / 2 : ne;  // factored nodes (the first nf of the rule)
  const int mw = half ? 2 * m0 : m0;  // right-hand sides per factored node
  const int nblk = ceil_div(n, bs), nbm = ceil_div(m0, bs);
  const size_t nn = (size_t)n * n, nm = (size_t)n * m0, mm = (size_t)m0 * m0;
  const int tcS = (fpm[43] == 0 && bs <= 32) ? (mixed ? 1 : 7) : 0;

  struct {
    zd *Af, *Bf, *R2, *AYr, *AYl, *YlN, *Rres, *SCr, *SCl, *fv;
    TL *S, *Linv, *Uinv, *Ysol, *Ytmp, *Yadj;
    float *fpre_n, *fpre_c;
    void *tcw_r, *kw_r;
    size_t tcw_r_bytes, kw_r_bytes;
    zd *Q, *Qh, *AQ, *BQ, *AhQh, *BhQh, *Xr, *AXr, *BXr, *Xl, *AXl, *BXl, *Yr, *Yl, *RBr, *RBl, *Tmp;
    zd *Aq, *Bq, *G, *Z, *Yv, *W, *V, *Mm, *P, *Sr, *Lr, *Ur, *Id, *Vt, *lam, *Eo, *z, *w;
    int *ipiv, *perm, *sing, *ipr, *pmr, *sgr, *pos, *src, *flag, *tc_err;
    double *rr, *rl, *nr, *nl, *Rr, *Rl, *stats;
    void *tcw, *kw, *dinv_l, *dinv_u, *pja, *pjah, *pjb, *pjbh, *pjq, *pjh, *pjx, *pjw, *rrw;
    size_t tcw_bytes, kw_bytes, rrw_bytes;
    char *acache_base;
    size_t acache_bytes;
    void *trw;  // Gram eigenproblems of the numerical-range cut
    size_t trw_bytes;
  } ws;
  SliceCache acache;
  auto layout = [&](Bump &b) {
    ws.Af = q.real ? b.take<zd>(nn) : nullptr;
    ws.Bf = (q.real && hasB) ? b.take<zd>(nn) : nullptr;
    ws.S = b.take<TL>((size_t)nf * nn);
    ws.Linv = b.take<TL>((size_t)nf * nblk * bs * bs);
    ws.Uinv = b.take<TL>((size_t)nf * nblk * bs * bs);
    ws.Ysol = b.take<TL>((size_t)nf * n * mw);
    ws.Ytmp = b.take<TL>((size_t)nf * n * mw);
    ws.Yadj = b.take<TL>((size_t)nf * n * mw);
    ws.R2 = b.take<zd>((size_t)n * mw);
    ws.AYr = b.take<zd>(nm);
    ws.AYl = b.take<zd>(nm);
    ws.YlN = b.take<zd>(nm);
    ws.Rres = b.take<zd>(nm);
    ws.SCr = b.take<zd>((size_t)nf * mw);
    ws.SCl = b.take<zd>((size_t)nf * mw);
    ws.fv = b.take<zd>(m0);
    zd **nmb[] = {&ws.Q, &ws.Qh, &ws.AQ, &ws.AhQh, &ws.Xr, &ws.AXr, &ws.Xl, &ws.AXl, &ws.Yr, &ws.Yl, &ws.RBr,
                  &ws.RBl, &ws.Tmp};
    for (zd **p : nmb) *p = b.take<zd>(nm);
    ws.BQ = hasB ? b.take<zd>(nm) : nullptr;
    ws.BhQh = hasB ? b.take<zd>(nm) : nullptr;
    ws.BXr = hasB ? b.take<zd>(nm) : nullptr;
    ws.BXl = hasB ? b.take<zd>(nm) : nullptr;
    zd **mmb[] = {&ws.Aq, &ws.Bq, &ws.G, &ws.Z, &ws.Yv, &ws.W, &ws.V, &ws.Mm, &ws.P, &ws.Sr, &ws.Id, &ws.Vt};
    for (zd **p : mmb) *p = b.take<zd>(mm);
    ws.Lr = b.take<zd>((size_t)nbm * bs * bs);
    ws.Ur = b.take<zd>((size_t)nbm * bs * bs);
    ws.lam = b.take<zd>(m0);
    ws.Eo = b.take<zd>(m0);
    ws.z = b.take<zd>(ne);
    ws.w = b.take<zd>(ne);
    ws.ipiv = b.take<int>((size_t)nf * n);
    ws.perm = b.take<int>((size_t)nf * n);
    ws.sing = b.take<int>(nf + 1);
    ws.ipr = b.take<int>(m0);
    ws.pmr = b.take<int>(m0);
    ws.sgr = b.take<int>(2);
    ws.pos = b.take<int>(m0);
    ws.src = b.take<int>(m0);
    ws.flag = b.take<int>(4);
    ws.tc_err = b.take<int>(4);
    double **db[] = {&ws.rr, &ws.rl, &ws.nr, &ws.nl, &ws.Rr, &ws.Rl};
    for (double **p : db) *p = b.take<double>(m0);
    ws.stats = b.take<double>(8);
    ws.tcw_bytes = tcS ? std::max(zgemm_sliced_work(n, n, nf, tcS), zgemm_sliced_work(n, mw, nf, tcS)) : 0;
    ws.tcw = tcS ? (void *)b.take<char>(ws.tcw_bytes) : nullptr;
    ws.kw_bytes = tcS ? (mixed ? solve_kwork_bytes_cf(n, mw, bs, nf) : solve_kwork_bytes(n, mw, bs, nf)) : 0;
    ws.kw = ws.kw_bytes ? (void *)b.take<char>(ws.kw_bytes) : nullptr;
    const bool pre = mixed && ws.kw_bytes && n >= 1024;  // FP32 factors split once into TF32 planes
    ws.fpre_n = pre ? b.take<float>(tf32_planes_bytes(n, nf) / 4) : nullptr;
    ws.fpre_c = pre ? b.take<float>(tf32_planes_bytes(n, nf) / 4) : nullptr;
    // the M0-sized LU and solves of the reduced pencil (FP64, their own
    // tensor-core workspace)
    ws.tcw_r_bytes = tcS ? zgemm_sliced_work(m0, m0, 1, 7) : 0;
    ws.tcw_r = tcS ? (void *)b.take<char>(ws.tcw_r_bytes) : nullptr;
    ws.kw_r_bytes = tcS ? solve_kwork_bytes(m0, m0, bs, 1) : 0;
    ws.kw_r = tcS ? (void *)b.take<char>(ws.kw_r_bytes) : nullptr;
    const bool big = !mixed && ws.kw_bytes && bs == 32 && n % 128 == 0;
    ws.dinv_l = big ? (void *)b.take<zd>((size_t)nf * n * 128) : nullptr;
    ws.dinv_u = big ? (void *)b.take<zd>((size_t)nf * n * 128) : nullptr;
    ws.acache_bytes = (!mixed && ws.kw_bytes)
                          ? std::min(solve_slice_cache_bytes(n, mw, bs, nf, 4, big), (size_t)24 << 30)
                          : 0;
    ws.acache_base = ws.acache_bytes ? b.take<char>(ws.acache_bytes) : nullptr;
    const long Kp = sliced_kp(n, true), R = 2L * n, Km = sliced_kp(m0, true), Rm = 2L * m0;
    ws.pja = b.take<char>(sliced_op_bytes(R, Kp, 1));
    ws.pjah = b.take<char>(sliced_op_bytes(R, Kp, 1));
    ws.pjb = hasB ? (void *)b.take<char>(sliced_op_bytes(R, Kp, 1)) : nullptr;
    ws.pjbh = hasB ? (void *)b.take<char>(sliced_op_bytes(R, Kp, 1)) : nullptr;
    ws.pjq = b.take<char>(sliced_op_bytes(m0, Kp, 1));
    ws.pjh = b.take<char>(sliced_op_bytes(Rm, Kp, 1));
    ws.pjx = b.take<char>(sliced_op_bytes(R, Km, 1));
    ws.pjw = b.take<char>(sliced_op_bytes(m0, Km, 1));
    ws.rrw_bytes = gemm_sliced_k_work(true, m0, m0, m0, 1);
    ws.rrw = b.take<char>(ws.rrw_bytes);
    ws.trw_bytes = heev_tridiag_work(m0, true);
    ws.trw = b.take<char>(ws.trw_bytes);
  };
  {
    Bump sizing(nullptr);
    layout(sizing);
    if (ensure_arena(h, sizing.off + 4096)) return out.info = -1;
    Bump real(h->arena);
    layout(real);
  }
  TcCtx tcx;
  tcx.work = ws.tcw;
  tcx.bytes = ws.tcw_bytes;
  tcx.gerr = ws.tc_err;
  tcx.S = tcS;
  tcx.kwork = ws.kw;
  tcx.kbytes = ws.kw_bytes;
  tcx.dinv_l = ws.dinv_l;
  tcx.dinv_u = ws.dinv_u;
  tcx.fpre_n = ws.fpre_n;
  tcx.fpre_c = ws.fpre_c;
  tcx.fpre_ne = ws.fpre_n ? nf : 0;
  acache.base = ws.acache_base;
  acache.cap = ws.acache_bytes;
  tcx.acache = ws.acache_bytes ? &acache : nullptr;
  // the M0-sized LU and solves of the reduced pencil: FP64 on the sliced
  // engine with their own workspace
  TcCtx tcr;
  tcr.work = ws.tcw_r;
  tcr.bytes = ws.tcw_r_bytes;
  tcr.gerr = ws.tc_err;
  tcr.S = 7;
  tcr.kwork = ws.kw_r;
  tcr.kbytes = ws.kw_r_bytes;
  TcScope tc_scope(tcS ? &tcx : nullptr);
  AuxScope aux_scope(ensure_aux(h));
  if (ensure_hbuf(h, (size_t)std::max(2 * m0, ne) + 64)) return out.info = -1;
  h->f_prec = -1;

  GBF_CUDA(cudaMemcpyAsync(ws.z, zh.data(), sizeof(zd) * ne, cudaMemcpyHostToDevice, st));
  GBF_CUDA(cudaMemcpyAsync(ws.w, wh.data(), sizeof(zd) * ne, cudaMemcpyHostToDevice, st));
  GBF_CUDA(cudaMemsetAsync(ws.sing, 0, sizeof(int) * (nf + 1), st));
  GBF_CUDA(cudaMemsetAsync(ws.tc_err, 0, sizeof(int) * 4, st));
  GBF_CUDA(cudaMemsetAsync(ws.flag, 0, sizeof(int) * 4, st));

  const zd *Af = (const zd *)q.A, *Bf = (const zd *)q.B;
  long lda = q.lda, ldb = q.ldb;
  CatScope cat_other(CAT_OTHER);
  if (q.real) {
    CK(gen_widen(st, n, (const double *)q.A, q.lda, ws.Af));
    Af = ws.Af;
    lda = n;
    if (hasB) {
      CK(gen_widen(st, n, (const double *)q.B, q.ldb, ws.Bf));
      Bf = ws.Bf;
      ldb = n;
    }
  }
  // factor the nodes (kept for the whole iteration)
  CK(form_shift<TL>(st, n, nf, ws.z, 1, 'G', Af, lda, hasB ? (const void *)Bf : nullptr, ldb, ws.S, ws.sing + nf));
  CK(getrf_batched<TL>(st, n, nf, ws.S, ws.ipiv, ws.perm, ws.Linv, ws.Uinv, bs, ws.sing, nullptr));
  acache.reset();
  if constexpr (mixed) {
    if (ws.fpre_n) CK(tf32_presplit(st, 'N', n, nf, ws.S, ws.fpre_n));
    if (ws.fpre_c) CK(tf32_presplit(st, 'C', n, nf, ws.S, ws.fpre_c));
  }
  {
    int *hs = (int *)h->hbuf;
    GBF_CUDA(cudaMemcpyAsync(hs, ws.sing, sizeof(int) * (nf + 1), cudaMemcpyDeviceToHost, st));
    GBF_CUDA(cudaMemcpyAsync(hs + nf + 1, ws.tc_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    GBF_CUDA(cudaStreamSynchronize(st));
    if (hs[nf + 1]) {
      set_error("tensor-core GEMM: bounded wait timed out (code %d)", hs[nf + 1]);
      return out.info = -4;
    }
    if (hs[nf]) {
      set_error("A or B holds a non-finite entry (NaN or Inf)");
      return out.info = -2;
    }
    for (int e = 0; e < nf; ++e)
      if (hs[e]) {
        set_error("zero pivot in column %d of the shifted system of node %d", hs[e], e);
        return out.info = -2;
      }
  }
  // rows of A, A^H, B, B^H sliced once (RCI cases 30, 31, 40, 41)
  SlicedOp opA{}, opAh{}, opB{}, opBh{};
  {
    CatScope cat_pj(CAT_PROJECT);
    CK(slice_rows<zd>(st, 'N', n, n, Af, lda, 0, 1, ws.pja, &opA));
    CK(slice_rows<zd>(st, 'C', n, n, Af, lda, 0, 1, ws.pjah, &opAh));
    if (hasB) {
      CK(slice_rows<zd>(st, 'N', n, n, Bf, ldb, 0, 1, ws.pjb, &opB));
      CK(slice_rows<zd>(st, 'C', n, n, Bf, ldb, 0, 1, ws.pjbh, &opBh));
    }
  }
  auto sliced_product = [&](const SlicedOp &opM, const zd *Y, int mm_, zd *o) -> int {
    SlicedOp opY;
    if (int rc = slice_cols<zd>(st, 'N', n, mm_, Y, n, 0, 1, ws.pjq, &opY)) return rc;
    return gemm_sliced_ops<zd>(st, opM, opY, 1, 1.0, 0, o, n, 0, ws.tc_err);
  };
  // rows(P) x cols(Mx): an n x m (or m x m) product with a sliced m x m right factor
  auto rr_gemm = [&](char opa, char opb, int mm_, int nn_, int kk, const zd *A_, int lda_, const zd *B_, int ldb_,
                     zd *C_, int ldc_) -> int {
    return gemm_sliced_k<zd>(st, opa, opb, mm_, nn_, kk, 1.0, A_, lda_, 0, B_, ldb_, 0, 0, C_, ldc_, 0, 1, ws.rrw,
                             ws.rrw_bytes, ws.tc_err);
  };

  // initial subspaces: right/left guesses from X (fpm(5)=1) or the seeded one
  int m = m0;
  if (fpm[4] == 1) {
    GBF_CUDA(cudaMemcpyAsync(ws.Yr, q.X, sizeof(zd) * nm, cudaMemcpyDeviceToDevice, st));
    GBF_CUDA(cudaMemcpyAsync(ws.Yl, (const zd *)q.X + nm, sizeof(zd) * nm, cudaMemcpyDeviceToDevice, st));
  } else {
    CK(random_subspace<zd>(st, (long)nm, SUBSPACE_SEED, ws.Yr));
    GBF_CUDA(cudaMemcpyAsync(ws.Yl, ws.Yr, sizeof(zd) * nm, cudaMemcpyDeviceToDevice, st));
  }
  if (hasB) {
    CatScope cat_pj(CAT_PROJECT);
    CK(sliced_product(opB, ws.Yr, m, ws.RBr));
    CK(sliced_product(opBh, ws.Yl, m, ws.RBl));
  } else {
    GBF_CUDA(cudaMemcpyAsync(ws.RBr, ws.Yr, sizeof(zd) * nm, cudaMemcpyDeviceToDevice, st));
    GBF_CUDA(cudaMemcpyAsync(ws.RBl, ws.Yl, sizeof(zd) * nm, cudaMemcpyDeviceToDevice, st));
  }

  zd trace_prev{0.0, 0.0};
  for (int k = 0;; ++k) {
    // ---- spectral projections (cases 11 and 21) ----
    // After the first loop, the residual-correction form
    // S_e^{-1} B X = X D_e + S_e^{-1} R D_e, R = A X - B X Lambda, D_e =
    // (z_e - Lambda)^{-1}, so Q = X f(Lambda) + sum_e w_e S_e^{-1} R D_e; on
    // the left S_e^{-H} B^H X^ = X^ conj(D_e) + S_e^{-H} R^ conj(D_e), R^ =
    // A^H X^ - B^H X^ conj(Lambda).  The same Q in exact arithmetic; the
    // solves see only the residuals, so FP32 factors reach FP64 results, and
    // a column whose filter value is far below the rounding level of the
    // solves (an eigenvalue far outside) stays accurate relative to its own
    // size instead of turning into solve noise that makes Q^^H B Q singular
    const bool rc_form = k > 0;
    const int mwk = half ? 2 * m : m;  // right-hand sides per factored node this loop
    const zd *rr_src = ws.RBr, *rl_src = ws.RBl;
    if (rc_form) {
      CK(gen_scales(st, m, nf, ne, ws.z, ws.w, ws.Eo, half ? 1 : 0, ws.SCr, ws.SCl, ws.fv));
      CK(gen_eig_residual(st, n, m, ws.AYr, hasB ? ws.RBr : ws.Yr, ws.Eo, 0, nullptr, ws.Rres));
      rr_src = ws.Rres;
    }
    if (half) {
      CK(gen_conj_pair(st, n, m, rr_src, ws.R2));
      rr_src = ws.R2;
    }
    CK(gather_rhs<TL>(st, n, nf, mwk, ws.perm, 1, rr_src, n, rc_form ? ws.SCr : nullptr, ws.Ysol));
    CK(getrs_inplace<TL>(st, 0, n, nf, mwk, ws.S, ws.Linv, ws.Uinv, bs, ws.Ysol, nullptr));
    CK(gen_accumulate<TL>(st, n, m, nf, ws.w, ws.Ysol, mwk, half ? 1 : 0, 0, rc_form ? ws.Yr : nullptr, ws.fv,
                          ws.Q));
    if (rc_form) {
      CK(gen_eig_residual(st, n, m, ws.AYl, ws.RBl, ws.Eo, 1, nullptr, ws.Rres));
      rl_src = ws.Rres;
    }
    if (half) {
      CK(gen_conj_pair(st, n, m, rl_src, ws.R2));
      rl_src = ws.R2;
    }
    CK(gather_rhs<TL>(st, n, nf, mwk, nullptr, 1, rl_src, n, rc_form ? ws.SCl : nullptr, ws.Ytmp));
    CK(getrs_inplace<TL>(st, 1, n, nf, mwk, ws.S, ws.Linv, ws.Uinv, bs, ws.Ytmp, nullptr));
    CK(scatter_perm<TL>(st, n, nf, mwk, ws.perm, ws.Ytmp, ws.Yadj));
    CK(gen_accumulate<TL>(st, n, m, nf, ws.w, ws.Yadj, mwk, half ? 1 : 0, 1, rc_form ? ws.YlN : nullptr, ws.fv,
                          ws.Qh));
    if (fpm[13] == 1) {  // the subspaces after one contour
      GBF_CUDA(cudaMemcpyAsync(q.X, ws.Q, sizeof(zd) * nm, cudaMemcpyDeviceToDevice, st));
      GBF_CUDA(cudaMemcpyAsync((zd *)q.X + nm, ws.Qh, sizeof(zd) * nm, cudaMemcpyDeviceToDevice, st));
      GBF_CUDA(cudaMemsetAsync(q.E, 0, sizeof(zd) * m0, st));
      GBF_CUDA(cudaMemsetAsync(q.res, 0, sizeof(double) * 2 * m0, st));
      GBF_CUDA(cudaStreamSynchronize(st));
      out.loop = k;
      return out.info = 4;
    }
    // ---- numerical ranges of Q and Q^: orthonormal bases of the directions
    // whose Gram eigenvalue exceeds 1e-14 of the largest (the Gram's own
    // rounding level), both cut to the smaller rank mk (the new M0).  Columns
    // of eigenvalues far outside shrink below the solves' rounding level and
    // would make the pencil singular; nearly parallel eigenvectors of a
    // nearly defective pair stay (down to angles of about 1e-7).
    {
      CatScope cat_red(CAT_REDUCED);
      zd *Gq = ws.Aq, *Gh = ws.Bq, *Vq = ws.Z, *Vh = ws.Yv, *Tq = ws.W, *Th = ws.V;
      double *wq = ws.rr, *wl = ws.rl;
      const zd *src[2] = {ws.Q, ws.Qh};
      zd *gram[2] = {Gq, Gh}, *vec[2] = {Vq, Vh};
      double *ev[2] = {wq, wl};
      for (int t = 0; t < 2; ++t) {
        SlicedOp opH, opC;
        CK(slice_rows<zd>(st, 'C', m, n, src[t], n, 0, 1, ws.pjh, &opH));
        CK(slice_cols<zd>(st, 'N', n, m, src[t], n, 0, 1, ws.pjq, &opC));
        CK(gemm_sliced_ops<zd>(st, opH, opC, 1, 1.0, 0, gram[t], m, 0, ws.tc_err));
        CK(hermitize<zd>(st, m, gram[t], ws.G));
        if (m == 1) {
          GBF_CUDA(cudaMemcpyAsync(ev[t], ws.G, sizeof(double), cudaMemcpyDeviceToDevice, st));
          CK(gen_identity(st, 1, vec[t]));
        } else {
          const int trc = heev_tridiag<zd>(st, m, ws.G, ev[t], vec[t], ws.trw, ws.trw_bytes);
          if (trc == 1) {
            set_error("subspace Gram eigenproblem: the cluster kernel cannot take m = %d", m);
            return out.info = -4;
          }
          CK(trc);
        }
      }
      double *hd = h->hbuf;
      GBF_CUDA(cudaMemcpyAsync(hd, wq, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
      GBF_CUDA(cudaMemcpyAsync(hd + m, wl, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
      GBF_CUDA(cudaStreamSynchronize(st));
      int r1 = 0, r2 = 0;
      for (int i = 0; i < m; ++i) {
        r1 += hd[i] > 1e-14 * hd[m - 1] ? 1 : 0;
        r2 += hd[m + i] > 1e-14 * hd[2 * m - 1] ? 1 : 0;
      }
      const int mk = std::min(r1, r2);
      if (mk < 1 || !(hd[m - 1] > 0.0) || !(hd[2 * m - 1] > 0.0)) {
        set_error("the filtered subspaces are empty (no direction above the rounding level)");
        return out.info = -3;
      }
      CK(make_t<zd>(st, m, mk, m - mk, Vq, wq, Tq));
      CK(make_t<zd>(st, m, mk, m - mk, Vh, wl, Th));
      SlicedOp opT, opM;
      CK(slice_cols<zd>(st, 'N', m, mk, Tq, m, 0, 1, ws.pjw, &opT));
      CK(slice_rows<zd>(st, 'N', n, m, ws.Q, n, 0, 1, ws.pjx, &opM));
      CK(gemm_sliced_ops<zd>(st, opM, opT, 1, 1.0, 0, ws.AQ, n, 0, ws.tc_err));
      CK(slice_cols<zd>(st, 'N', m, mk, Th, m, 0, 1, ws.pjw, &opT));
      CK(slice_rows<zd>(st, 'N', n, m, ws.Qh, n, 0, 1, ws.pjx, &opM));
      CK(gemm_sliced_ops<zd>(st, opM, opT, 1, 1.0, 0, ws.AhQh, n, 0, ws.tc_err));
      GBF_CUDA(cudaMemcpyAsync(ws.Q, ws.AQ, sizeof(zd) * (size_t)n * mk, cudaMemcpyDeviceToDevice, st));
      GBF_CUDA(cudaMemcpyAsync(ws.Qh, ws.AhQh, sizeof(zd) * (size_t)n * mk, cudaMemcpyDeviceToDevice, st));
      m = mk;
    }
    // ---- Rayleigh-Ritz on the dual subspaces (cases 30, 31, 40, 41) ----
    {
      CatScope cat_proj(CAT_PROJECT);
      SlicedOp opQ, opM;
      CK(slice_cols<zd>(st, 'N', n, m, ws.Q, n, 0, 1, ws.pjq, &opQ));
      CK(gemm_sliced_ops<zd>(st, opA, opQ, 1, 1.0, 0, ws.AQ, n, 0, ws.tc_err));
      if (hasB) CK(gemm_sliced_ops<zd>(st, opB, opQ, 1, 1.0, 0, ws.BQ, n, 0, ws.tc_err));
      CK(slice_cols<zd>(st, 'N', n, m, ws.Qh, n, 0, 1, ws.pjq, &opQ));
      CK(gemm_sliced_ops<zd>(st, opAh, opQ, 1, 1.0, 0, ws.AhQh, n, 0, ws.tc_err));
      if (hasB) CK(gemm_sliced_ops<zd>(st, opBh, opQ, 1, 1.0, 0, ws.BhQh, n, 0, ws.tc_err));
      SlicedOp opQhH;
      CK(slice_rows<zd>(st, 'C', m, n, ws.Qh, n, 0, 1, ws.pjh, &opQhH));
      CK(slice_cols<zd>(st, 'N', n, m, ws.AQ, n, 0, 1, ws.pjq, &opM));
      CK(gemm_sliced_ops<zd>(st, opQhH, opM, 1, 1.0, 0, ws.Aq, m, 0, ws.tc_err));
      CK(slice_cols<zd>(st, 'N', n, m, hasB ? ws.BQ : ws.Q, n, 0, 1, ws.pjq, &opM));
      CK(gemm_sliced_ops<zd>(st, opQhH, opM, 1, 1.0, 0, ws.Bq, m, 0, ws.tc_err));
    }
    // ---- reduced pencil: G = Bq^{-1} Aq = Z T Z^H, W = Z Y, V = (Bq W)^{-H} ----
    {
      CatScope cat_red(CAT_REDUCED);
      TcScope red_tc(tcS ? &tcr : nullptr);
      GBF_CUDA(cudaMemsetAsync(ws.sgr, 0, sizeof(int) * 2, st));
      GBF_CUDA(cudaMemcpyAsync(ws.Sr, ws.Bq, sizeof(zd) * mm, cudaMemcpyDeviceToDevice, st));
      CK(getrf_batched<zd>(st, m, 1, ws.Sr, ws.ipr, ws.pmr, ws.Lr, ws.Ur, bs, ws.sgr, nullptr));
      CK(gather_rhs<zd>(st, m, 1, m, ws.pmr, 1, ws.Aq, m, nullptr, ws.G));
      CK(getrs_inplace<zd>(st, 0, m, 1, m, ws.Sr, ws.Lr, ws.Ur, bs, ws.G, nullptr));
      CK(gen_hessenberg(st, m, ws.G, ws.Z));
      CK(gen_hqr(st, m, ws.G, ws.Z, ws.lam, ws.flag + 2));
      CK(gen_trevc(st, m, ws.G, ws.Yv));
      CK(rr_gemm('N', 'N', m, m, m, ws.Z, m, ws.Yv, m, ws.W, m));
      CK(gen_col_norms(st, m, m, ws.W, ws.nr));
      CK(gen_col_scale(st, m, m, ws.W, ws.W, ws.nr, 1));
      CK(rr_gemm('N', 'N', m, m, m, ws.Bq, m, ws.W, m, ws.Mm, m));
      GBF_CUDA(cudaMemcpyAsync(ws.Sr, ws.Mm, sizeof(zd) * mm, cudaMemcpyDeviceToDevice, st));
      CK(getrf_batched<zd>(st, m, 1, ws.Sr, ws.ipr, ws.pmr, ws.Lr, ws.Ur, bs, ws.sgr + 1, nullptr));
      CK(gen_identity(st, m, ws.Id));
      CK(gather_rhs<zd>(st, m, 1, m, nullptr, 1, ws.Id, m, nullptr, ws.Vt));
      CK(getrs_inplace<zd>(st, 1, m, 1, m, ws.Sr, ws.Lr, ws.Ur, bs, ws.Vt, nullptr));
      CK(scatter_perm<zd>(st, m, 1, m, ws.pmr, ws.Vt, ws.V));
    }
    // ---- Ritz vectors, residuals, order ----
    {
      CatScope cat_proj(CAT_PROJECT);
      SlicedOp opW, opM;
      CK(slice_cols<zd>(st, 'N', m, m, ws.W, m, 0, 1, ws.pjw, &opW));
      const zd *srcR[3] = {ws.Q, ws.AQ, ws.BQ};
      zd *dstR[3] = {ws.Xr, ws.AXr, ws.BXr};
      for (int t = 0; t < (hasB ? 3 : 2); ++t) {
        CK(slice_rows<zd>(st, 'N', n, m, srcR[t], n, 0, 1, ws.pjx, &opM));
        CK(gemm_sliced_ops<zd>(st, opM, opW, 1, 1.0, 0, dstR[t], n, 0, ws.tc_err));
      }
      CK(slice_cols<zd>(st, 'N', m, m, ws.V, m, 0, 1, ws.pjw, &opW));
      const zd *srcL[3] = {ws.Qh, ws.AhQh, ws.BhQh};
      zd *dstL[3] = {ws.Xl, ws.AXl, ws.BXl};
      for (int t = 0; t < (hasB ? 3 : 2); ++t) {
        CK(slice_rows<zd>(st, 'N', n, m, srcL[t], n, 0, 1, ws.pjx, &opM));
        CK(gemm_sliced_ops<zd>(st, opM, opW, 1, 1.0, 0, dstL[t], n, 0, ws.tc_err));
      }
    }
    // right vectors to unit 2-norm, left ones scaled inversely
    CK(gen_col_norms(st, n, m, ws.Xr, ws.nr));
    for (zd *p : {ws.Xr, ws.AXr, ws.BXr})
      if (p) CK(gen_col_scale(st, n, m, p, p, ws.nr, 1));
    for (zd *p : {ws.Xl, ws.AXl, ws.BXl})
      if (p) CK(gen_col_scale(st, n, m, p, p, ws.nr, 0));
    CK(gen_residual(st, n, m, ws.AXr, hasB ? ws.BXr : ws.Xr, ws.lam, 0, alpha, ws.rr));
    CK(gen_residual(st, n, m, ws.AXl, hasB ? ws.BXl : ws.Xl, ws.lam, 1, alpha, ws.rl));
    CK(gen_order(st, m, ws.lam, ws.rr, ws.rl, q.emid, q.r, fpm[17] / 100.0, (double)fpm[18], ws.pos, ws.src, ws.Eo,
                 ws.Rr, ws.Rl, ws.stats));
    // next right subspace and its B product; next left one with unit columns
    CK(permute_cols<zd>(st, n, m, ws.pos, ws.Xr, ws.Yr));
    CK(permute_cols<zd>(st, n, m, ws.pos, ws.Xl, ws.Yl));
    if (hasB) CK(permute_cols<zd>(st, n, m, ws.pos, ws.BXr, ws.RBr));
    else GBF_CUDA(cudaMemcpyAsync(ws.RBr, ws.Yr, sizeof(zd) * (size_t)n * m, cudaMemcpyDeviceToDevice, st));
    CK(gen_col_norms(st, n, m, ws.Yl, ws.nl));
    if (hasB) {
      CK(permute_cols<zd>(st, n, m, ws.pos, ws.BXl, ws.Tmp));
      CK(gen_col_scale(st, n, m, ws.Tmp, ws.RBl, ws.nl, 1));
    } else {
      CK(gen_col_scale(st, n, m, ws.Yl, ws.RBl, ws.nl, 1));
    }
    // A X and A^H X^ of the next subspaces, for the residuals
    CK(permute_cols<zd>(st, n, m, ws.pos, ws.AXr, ws.AYr));
    CK(permute_cols<zd>(st, n, m, ws.pos, ws.AXl, ws.Tmp));
    CK(gen_col_scale(st, n, m, ws.Tmp, ws.AYl, ws.nl, 1));
    CK(gen_col_scale(st, n, m, ws.Yl, ws.YlN, ws.nl, 1));
    double *hs = h->hbuf;
    GBF_CUDA(cudaMemcpyAsync(hs, ws.stats, sizeof(double) * 5, cudaMemcpyDeviceToHost, st));
    GBF_CUDA(cudaMemcpyAsync(h->hflag, ws.flag, sizeof(int) * 4, cudaMemcpyDeviceToHost, st));
    GBF_CUDA(cudaMemcpyAsync(h->hflag + 4, ws.tc_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    GBF_CUDA(cudaMemcpyAsync(h->hflag + 5, ws.sgr, sizeof(int) * 2, cudaMemcpyDeviceToHost, st));
    GBF_CUDA(cudaStreamSynchronize(st));
    if (h->hflag[4]) {
      set_error("tensor-core GEMM: bounded wait timed out (code %d)", h->hflag[4]);
      return out.info = -4;
    }
    if (h->hflag[5] || h->hflag[6]) {
      set_error("reduced pencil: %s is singular (the subspaces are not independent)",
                h->hflag[5] ? "Q^^H B Q" : "Bq W");
      return out.info = -3;
    }
    if (h->hflag[2]) {
      set_error("reduced non-Hermitian eigenproblem: the shifted QR did not converge");
      return out.info = -4;
    }
    const int nin = (int)hs[0];
    const zd trace{hs[1], hs[2]};
    const double maxres = hs[3];
    const bool finite = hs[4] != 0.0;
    const double eout = (k == 0) ? 1.0 : hypot(trace.x - trace_prev.x, trace.y - trace_prev.y) / alpha;
    out.M = nin;
    out.loop = k;
    out.epsout = eout;
    if (fpm[0] == 1)
      fprintf(stderr, "%d\t%d\t%.15e %+.15ei\t%.15e\t%.15e\t(M0 %d, non-Hermitian)\n", k, nin, trace.x, trace.y,
              eout, maxres, m);
    int info = -99;
    if (!finite) {
      set_error("non-finite Ritz values or residuals");
      info = -2;
    } else if (nin == 0) {
      info = 1;
    } else if (nin >= m && m < n) {
      info = 3;
    } else if ((fpm[5] == 0) ? (eout < eps) : (maxres < eps)) {
      info = 0;
      // bi-orthonormality of the returned pairs: X^_M^H B X_M = I
      CK(rr_gemm('C', 'N', m, m, m, ws.V, m, ws.Mm, m, ws.P, m));
      CK(gen_biorth(st, m, nin, ws.P, ws.nr, ws.src, ws.stats + 5));
      GBF_CUDA(cudaMemcpyAsync(hs + 5, ws.stats + 5, sizeof(double), cudaMemcpyDeviceToHost, st));
      GBF_CUDA(cudaStreamSynchronize(st));
      h->gen_biorth = hs[5];
      if (!(hs[5] <= 1e-8)) info = 6;
    } else if (k >= fpm[3]) {
      info = 2;
    }
    if (info != -99) {  // outputs: m pairs, zero past them; m is the new M0
      GBF_CUDA(cudaMemsetAsync(q.E, 0, sizeof(zd) * m0, st));
      GBF_CUDA(cudaMemsetAsync(q.res, 0, sizeof(double) * 2 * m0, st));
      GBF_CUDA(cudaMemsetAsync(q.X, 0, sizeof(zd) * 2 * nm, st));
      GBF_CUDA(cudaMemcpyAsync(q.E, ws.Eo, sizeof(zd) * m, cudaMemcpyDeviceToDevice, st));
      GBF_CUDA(cudaMemcpyAsync(q.res, ws.Rr, sizeof(double) * m, cudaMemcpyDeviceToDevice, st));
      GBF_CUDA(cudaMemcpyAsync(q.res + m0, ws.Rl, sizeof(double) * m, cudaMemcpyDeviceToDevice, st));
      GBF_CUDA(cudaMemcpyAsync(q.X, ws.Yr, sizeof(zd) * (size_t)n * m, cudaMemcpyDeviceToDevice, st));
      GBF_CUDA(cudaMemcpyAsync((zd *)q.X + nm, ws.Yl, sizeof(zd) * (size_t)n * m, cudaMemcpyDeviceToDevice, st));
      GBF_CUDA(cudaStreamSynchronize(st));
      out.m0 = m;
      return out.info = info;
    }
    trace_prev = trace;
  }
}

// ----------------------------------------------------------- validation --
static int validate(char uplo, int n, long lda, bool hasB, long ldb, const int *fpm, double emin, double emax,
                    int m0) {
  if (uplo != 'F' && uplo != 'L' && uplo != 'U') return -101;
  if (n < 1) return 202;
  if (lda < n) return -104;
  if (hasB && ldb < n) return -106;
  if (!fpm) return -107;
  if (m0 < 1 || m0 > n) return 201;
  if (!(emin < emax)) return 200;
  return check_fpm(fpm);
}

static gbf_context *default_ctx() {
  static std::mutex mu;
  static gbf_context *ctx[64] = {nullptr};
  std::lock_guard<std::mutex> lk(mu);
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return nullptr;
  if (!ctx[dev]) {
    gbf_handle h = nullptr;
    if (gbf_create(&h) != 0) return nullptr;
    ctx[dev] = h;
  }
  return ctx[dev];
}

template <class TQ>
static int run_dev(gbf_handle h, void *stream, char uplo, int n, const double *dA, int lda, const double *dB,
                   int ldb, int *fpm, double *epsout, int *loop, double emin, double emax, int *M0, double *dE,
                   double *dX, int *M, double *dres, int *info, const double *Zne, const double *Wne,
                   const gbf_shard *sh = nullptr) {
  int code = validate(uplo, n, lda, dB != nullptr, ldb, fpm, emin, emax, M0 ? *M0 : 0);
  Res out;
  if (code == 0 && (!dA || !dE || !dX || !dres)) code = -103;
  if (code == 0) {
    Req q{uplo, n, dA, lda, dB, ldb, fpm, emin, emax, *M0, Zne, Wne, dE, dX, dres, sh};
    cudaStream_t st = (cudaStream_t)stream;
    if (fpm[41] == 1)
      code = feast_run<TQ, cf>(h, st, q, out);
    else
      code = feast_run<TQ, zd>(h, st, q, out);
    if (epsout) *epsout = out.epsout;
    if (loop) *loop = out.loop;
    if (M) *M = out.M;
    if (M0 && code >= 0) *M0 = out.m0;
  }
  if (info) *info = code;
  return code;
}

// Checks of the non-Hermitian drivers' arguments (Table tab_info codes).
static int validate_gen(int n, long lda, bool hasB, long ldb, const int *fpm, double r, int m0) {
  if (n < 1) return 202;
  if (lda < n) return -104;
  if (hasB && ldb < n) return -106;
  if (!fpm) return -107;
  if (m0 < 1 || m0 > n || m0 > 1024) return 201;
  if (!(r > 0.0)) return 200;
  if (fpm[2] < 0 || fpm[2] > 16) return 103;
  if (fpm[3] < 0) return 104;
  if (fpm[4] != 0 && fpm[4] != 1) return 105;
  if (fpm[5] != 0 && fpm[5] != 1) return 106;
  if (fpm[7] < 1 || fpm[7] > 1024) return 108;
  if (fpm[13] != 0 && fpm[13] != 1) return 114;
  if (fpm[16] != 0 && fpm[16] != 1) return 117;
  if (fpm[17] <= 0) return 118;
  if (fpm[18] < -180 || fpm[18] > 180) return 119;
  if (fpm[41] != 0 && fpm[41] != 1) return 142;
  if (fpm[42] != 0 && (fpm[42] < 8 || fpm[42] > 64 || fpm[42] % 8)) return 143;
  if (fpm[43] != 0 && fpm[43] != 1) return 144;
  return 0;
}

static int run_gen_dev(gbf_handle h, void *stream, bool real, int n, const double *dA, int lda, const double *dB,
                       int ldb, int *fpm, double *epsout, int *loop, double emid_re, double emid_im, double r,
                       int *M0, double *dE, double *dX, int *M, double *dres, int *info, const double *Zne,
                       const double *Wne) {
  int code = validate_gen(n, lda, dB != nullptr, ldb, fpm, r, M0 ? *M0 : 0);
  Res out;
  if (code == 0 && (!dA || !dE || !dX || !dres)) code = -103;
  if (code == 0) {
    GenReq q{n, real, dA, lda, dB, ldb, fpm, zd{emid_re, emid_im}, r, *M0, Zne, Wne, dE, dX, dres};
    code = fpm[41] == 1 ? feast_run_gen<cf>(h, (cudaStream_t)stream, q, out)
                        : feast_run_gen<zd>(h, (cudaStream_t)stream, q, out);
    if (epsout) *epsout = out.epsout;
    if (loop) *loop = out.loop;
    if (M) *M = out.M;
    if (M0 && code >= 0) *M0 = out.m0;
  }
  if (info) *info = code;
  return code;
}

// Host-pointer form of the non-Hermitian drivers: the inputs copied to the
// device, the device driver on the default context's stream, the outputs
// (E: 2 M0 doubles, X: complex n x 2 M0, res: 2 M0) copied back.
static int run_gen_host(bool real, int n, const double *A, int lda, const double *B, int ldb, int *fpm,
                        double *epsout, int *loop, double emid_re, double emid_im, double r, int *M0, double *E,
                        double *X, int *M, double *res, int *info, const double *Zne, const double *Wne) {
  int code = validate_gen(n, lda, B != nullptr, ldb, fpm, r, M0 ? *M0 : 0);
  if (code != 0 || !A || !E || !X || !res) {
    if (code == 0) code = -103;
    if (info) *info = code;
    return code;
  }
  gbf_context *h = default_ctx();
  if (!h) {
    if (info) *info = -4;
    return -4;
  }
  const int m0 = *M0;
  const size_t szq = real ? sizeof(double) : sizeof(zd);
  const size_t bytes_a = szq * (size_t)lda * n, bytes_b = B ? szq * (size_t)ldb * n : 0;
  const size_t bytes_x = sizeof(zd) * (size_t)n * 2 * m0, bytes_e = sizeof(zd) * m0, bytes_r = sizeof(double) * 2 * m0;
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  char *buf = nullptr;
  const size_t total = al(bytes_a) + al(bytes_b) + al(bytes_x) + al(bytes_e) + al(bytes_r);
  if (cudaMalloc((void **)&buf, total) != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc of %zu bytes failed", total);
    if (info) *info = -1;
    return -1;
  }
  double *dA = (double *)buf;
  double *dB = B ? (double *)(buf + al(bytes_a)) : nullptr;
  double *dX = (double *)(buf + al(bytes_a) + al(bytes_b));
  double *dE = (double *)((char *)dX + al(bytes_x));
  double *dR = (double *)((char *)dE + al(bytes_e));
  cudaStream_t st = h->own;
  int rc = 0;
  if (cudaMemcpyAsync(dA, A, bytes_a, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      (B && cudaMemcpyAsync(dB, B, bytes_b, cudaMemcpyHostToDevice, st) != cudaSuccess) ||
      (fpm[4] == 1 && cudaMemcpyAsync(dX, X, bytes_x, cudaMemcpyHostToDevice, st) != cudaSuccess))
    rc = -4;
  if (rc == 0)
    rc = run_gen_dev(h, st, real, n, dA, lda, dB, ldb, fpm, epsout, loop, emid_re, emid_im, r, M0, dE, dX, M, dR,
                     info, Zne, Wne);
  if (rc >= 0 && rc != 200 && rc != 201 && rc != 202 && !(rc > 100 && rc < 200)) {
    if (cudaMemcpyAsync(E, dE, bytes_e, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(res, dR, bytes_r, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(X, dX, bytes_x, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      rc = -4;
  }
  if (rc == -4) set_error("CUDA error in host-pointer driver: %s", cudaGetErrorString(cudaGetLastError()));
  cudaStreamSynchronize(st);
  cudaFree(buf);
  if (info) *info = rc;
  return rc;
}

template <class TQ>
static int run_host(char uplo, int n, const double *A, int lda, const double *B, int ldb, int *fpm,
                    double *epsout, int *loop, double emin, double emax, int *M0, double *E, double *X, int *M,
                    double *res, int *info, const double *Zne, const double *Wne) {
  int code = validate(uplo, n, lda, B != nullptr, ldb, fpm, emin, emax, M0 ? *M0 : 0);
  if (code != 0 || !A || !E || !X || !res) {
    if (code == 0) code = -103;
    if (info) *info = code;
    return code;
  }
  gbf_context *h = default_ctx();
  if (!h) {
    if (info) *info = -4;
    return -4;
  }
  const int m0 = *M0;
  const size_t szq = sizeof(TQ);
  const size_t bytes_a = szq * (size_t)lda * n, bytes_b = B ? szq * (size_t)ldb * n : 0;
  const size_t bytes_x = szq * (size_t)n * m0, bytes_e = sizeof(double) * m0;
  char *buf = nullptr;
  const size_t total = bytes_a + bytes_b + bytes_x + 2 * bytes_e + 4 * 256;
  if (cudaMalloc((void **)&buf, total) != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc of %zu bytes failed", total);
    if (info) *info = -1;
    return -1;
  }
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  double *dA = (double *)buf;
  double *dB = B ? (double *)(buf + al(bytes_a)) : nullptr;
  double *dX = (double *)(buf + al(bytes_a) + al(bytes_b));
  double *dE = (double *)((char *)dX + al(bytes_x));
  double *dR = (double *)((char *)dE + al(bytes_e));
  cudaStream_t st = h->own;
  int rc = 0;
  if (cudaMemcpyAsync(dA, A, bytes_a, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      (B && cudaMemcpyAsync(dB, B, bytes_b, cudaMemcpyHostToDevice, st) != cudaSuccess) ||
      (fpm[4] == 1 && cudaMemcpyAsync(dX, X, bytes_x, cudaMemcpyHostToDevice, st) != cudaSuccess))
    rc = -4;
  if (rc == 0)
    rc = run_dev<TQ>(h, st, uplo, n, dA, lda, dB, ldb, fpm, epsout, loop, emin, emax, M0, dE, dX, M, dR, info, Zne,
                     Wne);
  if (rc >= 0 && rc != 200 && rc != 201 && rc != 202 && !(rc > 100 && rc < 200)) {
    if (cudaMemcpyAsync(E, dE, bytes_e, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(res, dR, bytes_e, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(X, dX, bytes_x, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      rc = -4;
  }
  if (rc == -4) set_error("CUDA error in host-pointer driver: %s", cudaGetErrorString(cudaGetLastError()));
  cudaStreamSynchronize(st);
  cudaFree(buf);
  if (info) *info = rc;
  return rc;
}

// ------------------------------------------------ batch / server glue --
namespace gbf {

int run_problem(gbf_context *h, cudaStream_t st, const gbf_problem *p, gbf_result *r) {
  int fpm[64];
  for (int i = 0; i < 64; ++i) fpm[i] = p->fpm[i];
  double eps = 1.0;
  int loop = 0, M = 0, M0 = p->m0, info = 0;
  if (p->kind == 1)
    run_dev<zd>(h, st, p->uplo, p->n, p->dA, p->lda, p->dB, p->ldb, fpm, &eps, &loop, p->emin, p->emax, &M0, p->dE,
                p->dX, &M, p->dres, &info, p->Zne, p->Wne);
  else
    run_dev<double>(h, st, p->uplo, p->n, p->dA, p->lda, p->dB, p->ldb, fpm, &eps, &loop, p->emin, p->emax, &M0,
                    p->dE, p->dX, &M, p->dres, &info, p->Zne, p->Wne);
  r->info = info;
  r->M = M;
  r->loop = loop;
  r->m0 = M0;
  r->epsout = eps;
  return info;
}

template <class TQ, class TL>
static size_t footprint_t(const gbf_problem *p) {
  const int ne = p->fpm[1] > 0 ? p->fpm[1] : 8;
  const int bs = p->fpm[42] ? p->fpm[42] : 32;
  WS<TQ, TL> ws;
  Bump b(nullptr);
  const int tcS = (p->fpm[43] == 0 && bs <= 32) ? (sizeof(TL) == sizeof(zd) ? 7 : 1) : 0;
  ws.layout(b, p->n, p->m0, ne, ne, ne, bs, p->kind == 1, p->dB != nullptr, p->uplo != 'F',
            p->dB != nullptr && p->uplo != 'F', pick_ksplit(p->m0, p->n), tcS, p->fpm[43] == 0);
  return b.off + 4096;
}

size_t problem_footprint(const gbf_problem *p) {
  const bool mixed = p->fpm[41] == 1;
  if (p->kind == 1) return mixed ? footprint_t<zd, cf>(p) : footprint_t<zd, zd>(p);
  return mixed ? footprint_t<double, cf>(p) : footprint_t<double, zd>(p);
}

}  // namespace gbf

extern "C" size_t gbf_problem_bytes(const gbf_problem *p) { return p ? problem_footprint(p) : 0; }

// ================================================================== C ABI ==
extern "C" {

int gbf_version(void) { return 100; }

const char *gbf_last_error(void) { return g_err; }

long long gbf_launch_count(void) { return g_launches.load(); }

int gbf_create(gbf_handle *hp) {
  if (!hp) return -101;
  gbf_context *h = new (std::nothrow) gbf_context();
  if (!h) return -1;
  GBF_CUDA(cudaGetDevice(&h->device));
  GBF_CUDA(cudaMallocHost((void **)&h->hflag, sizeof(int) * 16));
  GBF_CUDA(cudaStreamCreateWithFlags(&h->own, cudaStreamNonBlocking));
  *hp = h;
  return 0;
}

int gbf_destroy(gbf_handle h) {
  if (!h) return 0;
  cudaDeviceSynchronize();
  if (h->arena) cudaFree(h->arena);
  if (h->hflag) cudaFreeHost(h->hflag);
  if (h->hbuf) cudaFreeHost(h->hbuf);
  if (h->own) cudaStreamDestroy(h->own);
  if (h->aux.s) cudaStreamDestroy(h->aux.s);
  if (h->aux.a) cudaEventDestroy(h->aux.a);
  if (h->aux.b) cudaEventDestroy(h->aux.b);
  delete h;
  return 0;
}

void gbf_init(int *fpm) {
  if (!fpm) return;
  for (int i = 0; i < 64; ++i) fpm[i] = 0;
  fpm[1] = 8;
  fpm[2] = 12;
  fpm[3] = 20;
  fpm[5] = 1;
  fpm[6] = 5;
  fpm[7] = 16;
  fpm[16] = 1;
  fpm[17] = 100;
}

int gbf_contour(double emin, double emax, int ne, int fpm16, int fpm18, double *Zne, double *Wne) {
  if (ne < 1) return 102;
  std::vector<zd> z(ne), w(ne);
  const int rc = make_contour(emin, emax, ne, fpm16, fpm18, z.data(), w.data());
  if (rc) return rc;
  for (int e = 0; e < ne; ++e) {
    Zne[2 * e] = z[e].x;
    Zne[2 * e + 1] = z[e].y;
    Wne[2 * e] = w[e].x;
    Wne[2 * e + 1] = w[e].y;
  }
  return 0;
}

int gbf_rationalx(const double *Zne, const double *Wne, int ne, const double *eig, int m, double *f) {
  if (ne < 1) return 102;
  for (int i = 0; i < m; ++i) {
    double s = 0.0;
    for (int e = 0; e < ne; ++e) {
      const zd q = zdiv(zd{Wne[2 * e], Wne[2 * e + 1]}, zd{Zne[2 * e] - eig[i], Zne[2 * e + 1]});
      s += q.x;
    }
    f[i] = s;
  }
  return 0;
}

int gbf_rational(double emin, double emax, int ne, int fpm16, int fpm18, const double *eig, int m, double *f) {
  if (ne < 1) return 102;
  std::vector<double> z(2 * ne), w(2 * ne);
  const int rc = gbf_contour(emin, emax, ne, fpm16, fpm18, z.data(), w.data());
  if (rc) return rc;
  return gbf_rationalx(z.data(), w.data(), ne, eig, m, f);
}

int gbf_dsyev(char uplo, int n, const double *A, int lda, int *fpm, double *epsout, int *loop, double emin,
              double emax, int *M0, double *E, double *X, int *M, double *res, int *info) {
  return run_host<double>(uplo, n, A, lda, nullptr, n, fpm, epsout, loop, emin, emax, M0, E, X, M, res, info,
                          nullptr, nullptr);
}
int gbf_dsygv(char uplo, int n, const double *A, int lda, const double *B, int ldb, int *fpm, double *epsout,
              int *loop, double emin, double emax, int *M0, double *E, double *X, int *M, double *res, int *info) {
  return run_host<double>(uplo, n, A, lda, B, ldb, fpm, epsout, loop, emin, emax, M0, E, X, M, res, info, nullptr,
                          nullptr);
}
int gbf_zheev(char uplo, int n, const double *A, int lda, int *fpm, double *epsout, int *loop, double emin,
              double emax, int *M0, double *E, double *X, int *M, double *res, int *info) {
  return run_host<zd>(uplo, n, A, lda, nullptr, n, fpm, epsout, loop, emin, emax, M0, E, X, M, res, info, nullptr,
                      nullptr);
}
int gbf_zhegv(char uplo, int n, const double *A, int lda, const double *B, int ldb, int *fpm, double *epsout,
              int *loop, double emin, double emax, int *M0, double *E, double *X, int *M, double *res, int *info) {
  return run_host<zd>(uplo, n, A, lda, B, ldb, fpm, epsout, loop, emin, emax, M0, E, X, M, res, info, nullptr,
                      nullptr);
}
int gbf_dsygvx(char uplo, int n, const double *A, int lda, const double *B, int ldb, int *fpm, double *epsout,
               int *loop, double emin, double emax, int *M0, double *E, double *X, int *M, double *res, int *info,
               const double *Zne, const double *Wne) {
  return run_host<double>(uplo, n, A, lda, B, ldb, fpm, epsout, loop, emin, emax, M0, E, X, M, res, info, Zne,
                          Wne);
}
int gbf_zhegvx(char uplo, int n, const double *A, int lda, const double *B, int ldb, int *fpm, double *epsout,
               int *loop, double emin, double emax, int *M0, double *E, double *X, int *M, double *res, int *info,
               const double *Zne, const double *Wne) {
  return run_host<zd>(uplo, n, A, lda, B, ldb, fpm, epsout, loop, emin, emax, M0, E, X, M, res, info, Zne, Wne);
}

int gbf_dsygv_dev(gbf_handle h, void *stream, char uplo, int n, const double *dA, int lda, const double *dB,
                  int ldb, int *fpm, double *epsout, int *loop, double emin, double emax, int *M0, double *dE,
                  double *dX, int *M, double *dres, int *info, const double *Zne, const double *Wne) {
  if (!h) h = default_ctx();
  if (!h) return -4;
  return run_dev<double>(h, stream, uplo, n, dA, lda, dB, ldb, fpm, epsout, loop, emin, emax, M0, dE, dX, M, dres,
                         info, Zne, Wne);
}
int gbf_zhegv_dev(gbf_handle h, void *stream, char uplo, int n, const double *dA, int lda, const double *dB,
                  int ldb, int *fpm, double *epsout, int *loop, double emin, double emax, int *M0, double *dE,
                  double *dX, int *M, double *dres, int *info, const double *Zne, const double *Wne) {
  if (!h) h = default_ctx();
  if (!h) return -4;
  return run_dev<zd>(h, stream, uplo, n, dA, lda, dB, ldb, fpm, epsout, loop, emin, emax, M0, dE, dX, M, dres,
                     info, Zne, Wne);
}

// ---------------------------------------------------- non-Hermitian entries
int gbf_gcontour(double emid_re, double emid_im, double r, int ne, int fpm17, int fpm18, int fpm19, double *Zne,
                 double *Wne) {
  if (!Zne || !Wne) return -103;
  std::vector<zd> z(std::max(ne, 1)), w(std::max(ne, 1));
  const int rc = make_gcontour(zd{emid_re, emid_im}, r, ne, fpm17, fpm18, fpm19, z.data(), w.data());
  if (rc) return rc;
  for (int e = 0; e < ne; ++e) {
    Zne[2 * e] = z[e].x;
    Zne[2 * e + 1] = z[e].y;
    Wne[2 * e] = w[e].x;
    Wne[2 * e + 1] = w[e].y;
  }
  return 0;
}

int gbf_grationalx(const double *Zne, const double *Wne, int ne, const double *eig, int m, double *f) {
  if (!Zne || !Wne || !eig || !f || ne < 1 || m < 0) return -103;
  for (int i = 0; i < m; ++i) {
    double sx = 0.0, sy = 0.0;
    for (int e = 0; e < ne; ++e) {
      const zd q = zdiv(zd{Wne[2 * e], Wne[2 * e + 1]}, zd{Zne[2 * e] - eig[2 * i], Zne[2 * e + 1] - eig[2 * i + 1]});
      sx += q.x;
      sy += q.y;
    }
    f[2 * i] = sx;
    f[2 * i + 1] = sy;
  }
  return 0;
}

double gbf_biorth_defect(gbf_handle h) { return h ? h->gen_biorth : -1.0; }

int gbf_dgegv(int n, const double *A, int lda, const double *B, int ldb, int *fpm, double *epsout, int *loop,
              double emid_re, double emid_im, double r, int *M0, double *E, double *X, int *M, double *res, int *info,
              const double *Zne, const double *Wne) {
  return run_gen_host(true, n, A, lda, B, ldb, fpm, epsout, loop, emid_re, emid_im, r, M0, E, X, M, res, info, Zne,
                      Wne);
}
int gbf_zgegv(int n, const double *A, int lda, const double *B, int ldb, int *fpm, double *epsout, int *loop,
              double emid_re, double emid_im, double r, int *M0, double *E, double *X, int *M, double *res, int *info,
              const double *Zne, const double *Wne) {
  return run_gen_host(false, n, A, lda, B, ldb, fpm, epsout, loop, emid_re, emid_im, r, M0, E, X, M, res, info, Zne,
                      Wne);
}

int gbf_dgegv_dev(gbf_handle h, void *stream, int n, const double *dA, int lda, const double *dB, int ldb, int *fpm,
                  double *epsout, int *loop, double emid_re, double emid_im, double r, int *M0, double *dE,
                  double *dX, int *M, double *dres, int *info, const double *Zne, const double *Wne) {
  if (!h) h = default_ctx();
  if (!h) return -4;
  return run_gen_dev(h, stream, true, n, dA, lda, dB, ldb, fpm, epsout, loop, emid_re, emid_im, r, M0, dE, dX, M,
                     dres, info, Zne, Wne);
}
int gbf_zgegv_dev(gbf_handle h, void *stream, int n, const double *dA, int lda, const double *dB, int ldb, int *fpm,
                  double *epsout, int *loop, double emid_re, double emid_im, double r, int *M0, double *dE,
                  double *dX, int *M, double *dres, int *info, const double *Zne, const double *Wne) {
  if (!h) h = default_ctx();
  if (!h) return -4;
  return run_gen_dev(h, stream, false, n, dA, lda, dB, ldb, fpm, epsout, loop, emid_re, emid_im, r, M0, dE, dX, M,
                     dres, info, Zne, Wne);
}

int gbf_shard_nodes(int ne, int rank, int nranks, int *first, int *count) {
  if (ne < 1) return -101;
  if (nranks < 1) return -103;
  if (rank < 0 || rank >= nranks) return -102;
  int lo = 0, cnt = 0, chunk = 0;
  shard_share(ne, rank, nranks, &lo, &cnt, &chunk);
  if (first) *first = lo;
  if (count) *count = cnt;
  return chunk;
}

static int check_shard(const gbf_shard *sh) {
  if (!sh) return -122;
  if (sh->nranks < 1 || sh->rank < 0 || sh->rank >= sh->nranks || !sh->allgather || !sh->agree) {
    set_error("gbf_shard: need 0 <= rank < nranks and both callbacks");
    return -122;
  }
  return 0;
}

int gbf_dsygv_dev_shard(gbf_handle h, void *stream, char uplo, int n, const double *dA, int lda, const double *dB,
                        int ldb, int *fpm, double *epsout, int *loop, double emin, double emax, int *M0, double *dE,
                        double *dX, int *M, double *dres, int *info, const double *Zne, const double *Wne,
                        const gbf_shard *sh) {
  if (int rc = check_shard(sh)) {
    if (info) *info = rc;
    return rc;
  }
  if (!h) h = default_ctx();
  if (!h) return -4;
  return run_dev<double>(h, stream, uplo, n, dA, lda, dB, ldb, fpm, epsout, loop, emin, emax, M0, dE, dX, M, dres,
                         info, Zne, Wne, sh);
}
int gbf_zhegv_dev_shard(gbf_handle h, void *stream, char uplo, int n, const double *dA, int lda, const double *dB,
                        int ldb, int *fpm, double *epsout, int *loop, double emin, double emax, int *M0, double *dE,
                        double *dX, int *M, double *dres, int *info, const double *Zne, const double *Wne,
                        const gbf_shard *sh) {
  if (int rc = check_shard(sh)) {
    if (info) *info = rc;
    return rc;
  }
  if (!h) h = default_ctx();
  if (!h) return -4;
  return run_dev<zd>(h, stream, uplo, n, dA, lda, dB, ldb, fpm, epsout, loop, emin, emax, M0, dE, dX, M, dres,
                     info, Zne, Wne, sh);
}

}  // extern "C"

// ------------------------------------------------------- step entries --
template <class TL>
static int factor_impl(gbf_handle h, cudaStream_t st, int kind, char uplo, int n, const double *dA, int lda,
                       const double *dB, int ldb, int ne, const double *Zne) {
  const int bs = 32;
  const size_t nn = (size_t)n * n;
  const int nblk = ceil_div(n, bs);
  Bump sz(nullptr);
  sz.take<TL>(ne * nn);
  sz.take<TL>((size_t)ne * nblk * bs * bs);
  sz.take<TL>((size_t)ne * nblk * bs * bs);
  sz.take<int>((size_t)ne * n);
  sz.take<int>((size_t)ne * n);
  sz.take<int>(ne);
  sz.take<zd>(ne);
  const int tcS = sizeof(TL) == sizeof(zd) ? 7 : 1;  // sliced FP64 / 3xTF32 FP32
  const size_t tcb = tcS ? zgemm_sliced_work(n, n, ne, tcS) : 0;
  sz.take<char>(tcb);
  sz.take<int>(4);
  if (ensure_arena(h, sz.off + 4096)) return -1;
  if (ensure_hbuf(h, (size_t)ne + 8)) return -1;
  Bump b(h->arena);
  TL *S = b.take<TL>(ne * nn);
  TL *Li = b.take<TL>((size_t)ne * nblk * bs * bs);
  TL *Ui = b.take<TL>((size_t)ne * nblk * bs * bs);
  int *ipiv = b.take<int>((size_t)ne * n);
  int *perm = b.take<int>((size_t)ne * n);
  int *sing = b.take<int>(ne);
  zd *z = b.take<zd>(ne);
  TcCtx tcx;
  tcx.work = b.take<char>(tcb);
  tcx.bytes = tcb;
  tcx.gerr = b.take<int>(4);
  tcx.S = tcS;
  TcScope tc_scope(&tcx);
  GBF_CUDA(cudaMemsetAsync(tcx.gerr, 0, sizeof(int), st));
  std::vector<zd> zh(ne);
  for (int e = 0; e < ne; ++e) zh[e] = zd{Zne[2 * e], Zne[2 * e + 1]};
  GBF_CUDA(cudaMemcpyAsync(z, zh.data(), sizeof(zd) * ne, cudaMemcpyHostToDevice, st));
  GBF_CUDA(cudaMemsetAsync(sing, 0, sizeof(int) * ne, st));
  int rc = form_shift<TL>(st, n, ne, z, kind, uplo, dA, lda, dB, ldb, S);
  if (!rc) rc = getrf_batched<TL>(st, n, ne, S, ipiv, perm, Li, Ui, bs, sing, nullptr);
  if (rc) return rc;
  int *hs = (int *)h->hbuf;
  GBF_CUDA(cudaMemcpyAsync(hs, sing, sizeof(int) * ne, cudaMemcpyDeviceToHost, st));
  GBF_CUDA(cudaMemcpyAsync(hs + ne, tcx.gerr, sizeof(int), cudaMemcpyDeviceToHost, st));
  GBF_CUDA(cudaStreamSynchronize(st));
  if (hs[ne]) {
    h->f_prec = -1;
    set_error("tensor-core GEMM: bounded wait timed out (code %d)", hs[ne]);
    return -4;
  }
  h->f_n = n;
  h->f_ne = ne;
  h->f_bs = bs;
  h->f_bytes = b.off;
  for (int e = 0; e < ne; ++e)
    if (hs[e]) {
      h->f_prec = -1;
      set_error("zero pivot in node %d", e);
      return -2;
    }
  return 0;
}

template <class TL>
static int solve_impl(gbf_handle h, cudaStream_t st, int trans, int nrhs, const double *dRHS, double *dY) {
  const int n = h->f_n, ne = h->f_ne, bs = h->f_bs;
  const size_t nn = (size_t)n * n;
  const int nblk = ceil_div(n, bs);
  const size_t ny = (size_t)ne * n * nrhs;
  Bump b(h->arena);
  TL *S = b.take<TL>(ne * nn);
  TL *Li = b.take<TL>((size_t)ne * nblk * bs * bs);
  TL *Ui = b.take<TL>((size_t)ne * nblk * bs * bs);
  b.take<int>((size_t)ne * n);
  int *perm = b.take<int>((size_t)ne * n);
  b.take<int>(ne);
  b.take<zd>(ne);
  const int tcS = sizeof(TL) == sizeof(zd) ? 7 : 1;  // sliced FP64 / 3xTF32 FP32
  b.take<char>(tcS ? zgemm_sliced_work(n, n, ne, tcS) : 0);
  int *tc_err = b.take<int>(4);
  const size_t base = b.off;
  TL *Y = b.take<TL>(ny);
  TL *Y2 = b.take<TL>(ny);
  const size_t tcb = tcS ? zgemm_sliced_work(n, nrhs, ne, tcS) : 0;
  void *tcw = b.take<char>(tcb);
  // the recursive solves of the FEAST loop (large-K products on the tensor
  // cores: sliced for FP64 factors, 3xTF32 for FP32 ones)
  const size_t kwb = sizeof(TL) == sizeof(zd) ? solve_kwork_bytes(n, nrhs, bs, ne)
                                              : solve_kwork_bytes_cf(n, nrhs, bs, ne);
  void *kw = b.take<char>(kwb);
  if (b.off + 4096 > h->cap) {
    // grow while keeping the factors
    char *na = nullptr;
    const size_t need = b.off + 4096;
    if (cudaMalloc((void **)&na, need) != cudaSuccess) {
      cudaGetLastError();
      return -1;
    }
    GBF_CUDA(cudaMemcpyAsync(na, h->arena, base, cudaMemcpyDeviceToDevice, st));
    GBF_CUDA(cudaStreamSynchronize(st));
    cudaFree(h->arena);
    h->arena = na;
    h->cap = need;
    return solve_impl<TL>(h, st, trans, nrhs, dRHS, dY);
  }
  TcCtx tcx;
  tcx.work = tcw;
  tcx.bytes = tcb;
  tcx.gerr = tc_err;
  tcx.S = tcS;
  tcx.kwork = kw;
  tcx.kbytes = kwb;
  TcScope tc_scope(&tcx);
  int rc;
  if (!trans) {
    rc = gather_rhs<TL>(st, n, ne, nrhs, perm, 1, dRHS, n, nullptr, Y);
    if (!rc) rc = getrs_inplace<TL>(st, 0, n, ne, nrhs, S, Li, Ui, bs, Y, nullptr);
  } else {
    rc = gather_rhs<TL>(st, n, ne, nrhs, nullptr, 1, dRHS, n, nullptr, Y2);
    if (!rc) rc = getrs_inplace<TL>(st, 1, n, ne, nrhs, S, Li, Ui, bs, Y2, nullptr);
    if (!rc) rc = scatter_perm<TL>(st, n, ne, nrhs, perm, Y2, Y);
  }
  if (rc) return rc;
  widen_kernel<TL><<<ceil_div((long)ny, 256), 256, 0, st>>>((long)ny, Y, (zd *)dY);
  GBF_LAUNCHED();
  GBF_CUDA(cudaMemcpyAsync(h->hflag + 2, tc_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  GBF_CUDA(cudaStreamSynchronize(st));
  if (h->hflag[2]) {
    set_error("tensor-core GEMM: bounded wait timed out (code %d)", h->hflag[2]);
    return -4;
  }
  return 0;
}

extern "C" int gbf_factor_dev(gbf_handle h, void *stream, int kind, int prec, char uplo, int n, const double *dA, int lda,
                   const double *dB, int ldb, int ne, const double *Zne) {
  if (!h) h = default_ctx();
  if (!h) return -4;
  if (kind != 0 && kind != 1) return -103;
  if (prec != 0 && prec != 1) return -104;
  if (uplo != 'F' && uplo != 'L' && uplo != 'U') return -105;
  if (n < 1) return 202;
  if (lda < n) return -108;
  if (dB && ldb < n) return -110;
  if (ne < 1) return -111;
  if (!dA || !Zne) return -107;
  cudaStream_t st = (cudaStream_t)stream;
  const int rc = prec ? factor_impl<cf>(h, st, kind, uplo, n, dA, lda, dB, ldb, ne, Zne)
                      : factor_impl<zd>(h, st, kind, uplo, n, dA, lda, dB, ldb, ne, Zne);
  if (rc == 0) h->f_prec = prec;
  return rc;
}

extern "C" int gbf_solve_dev(gbf_handle h, void *stream, int trans, int nrhs, const double *dRHS, double *dY) {
  if (!h) h = default_ctx();
  if (!h) return -4;
  if (h->f_prec < 0) {
    set_error("gbf_solve_dev: no stored factorisation (call gbf_factor_dev first)");
    return -2;
  }
  if (trans != 0 && trans != 1) return -103;
  if (nrhs < 1) return -104;
  if (!dRHS || !dY) return -105;
  cudaStream_t st = (cudaStream_t)stream;
  return h->f_prec ? solve_impl<cf>(h, st, trans, nrhs, dRHS, dY) : solve_impl<zd>(h, st, trans, nrhs, dRHS, dY);
}

template <class T>
static int heev_impl(gbf_handle h, cudaStream_t st, int m, T *A, double *w, T *V) {
  Bump sz(nullptr);
  sz.take<T>(2 * (size_t)m * m + 2 * m);
  sz.take<double>(8 + 4 * m);
  sz.take<int>(5 * m + 96);
  const size_t tb = heev_tridiag_work(m, tr<T>::cplx);
  sz.take<char>(tb);
  if (ensure_arena(h, sz.off + 4096)) return -1;
  h->f_prec = -1;
  Bump b(h->arena);
  T *work = b.take<T>(2 * (size_t)m * m + 2 * m);
  double *dwork = b.take<double>(8 + 4 * m);
  int *iwork = b.take<int>(5 * m + 96);
  void *tw = b.take<char>(tb);
  // the solver of the FEAST loop (tridiagonal route), Jacobi when it declines
  const int trc = heev_tridiag<T>(st, m, A, w, V, tw, tb);
  if (trc != 1) {
    if (trc) return trc;
    GBF_CUDA(cudaStreamSynchronize(st));
    return 0;
  }
  int sweeps = 0;
  const int rc = heev_jacobi<T>(st, m, A, w, V, work, dwork, iwork, h->hflag, &sweeps);
  if (rc) return rc;
  GBF_CUDA(cudaStreamSynchronize(st));
  if (sweeps < 0) {
    set_error("Jacobi did not converge in 80 sweeps");
    return -3;
  }
  return 0;
}

extern "C" int gbf_heev_dev(gbf_handle h, void *stream, int kind, int m, double *dA, double *dW, double *dV) {
  if (!h) h = default_ctx();
  if (!h) return -4;
  if (kind != 0 && kind != 1) return -103;
  if (m < 1) return -104;
  if (!dA || !dW || !dV) return -105;
  cudaStream_t st = (cudaStream_t)stream;
  return kind ? heev_impl<zd>(h, st, m, (zd *)dA, dW, (zd *)dV) : heev_impl<double>(h, st, m, dA, dW, dV);
}


