// Reduced dense eigenproblem of the Rayleigh-Ritz step and the small
// kernels around it (FEAST v3.0 guide, "The FEAST Algorithm": Rayleigh-Ritz
// on the reduced system; Table "tab_common": residual definition, output
// ordering; the quadrature sum Q = sum_e w_e Q_e).
//
// heev_jacobi: parallel two-sided cyclic Jacobi (kernel in gbf_small.cu).  A
// sweep is P-1 rounds of the circle-method tournament over P = m rounded up
// to even players; in round r, index x is paired with (2r - x) mod (P-1)
// (x = r pairs with P-1), so the P/2 rotations of a round are disjoint and
// one grid-wide phase applies all of them as A <- J^H A J, V <- V J with
// every element computed from at most four old elements.  For the pair (p < q), b = A[p][q] = |b| e^{i phi}:
//   tau = (A[q][q] - A[p][p]) / (2|b|), t = sign(tau)/(|tau| + sqrt(1+tau^2)),
//   c = 1/sqrt(1+t^2), s = t c, J = [[c, s e^{i phi}], [-s e^{-i phi}, c]].
// A rotation is skipped when |b| <= eps/2 sqrt|A[p][p]| sqrt|A[q][q]| or
// |b| <= 1e-18 ||A||_F; a sweep ends the iteration once no pair violates it.
#include <algorithm>
#include <mutex>
#include <vector>

#include "gbf_common.cuh"

namespace gbf {

__host__ __device__ inline double absT(double a) { return fabs(a); }
__host__ __device__ inline double absT(zd a) { return hypot(a.x, a.y); }
__host__ __device__ inline double scaleT(double a, double s) { return a * s; }
__host__ __device__ inline zd scaleT(zd a, double s) { return zd{a.x * s, a.y * s}; }


template <class T>
__global__ void fro_kernel(int m, const T *A, double *out) {
  __shared__ double red[256];
  double s = 0.0;
  for (long t = threadIdx.x; t < (long)m * m; t += blockDim.x) {
    const double v = absT(A[t]);
    s += v * v;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sqrt(red[0]);
}

// eigenvalues ascending (stable on ties); NaN sorts last
template <class T>
__global__ void rank_kernel(int m, const T *A, double *w, int *rank) {
  using X = tr<T>;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  const double dj = X::re(A[j + (long)j * m]);
  const bool nj = isnan(dj);
  int rk = 0;
  for (int i = 0; i < m; ++i) {
    const double di = X::re(A[i + (long)i * m]);
    const bool ni = isnan(di);
    bool before;
    if (nj)
      before = ni ? (i < j) : true;
    else
      before = ni ? false : (di < dj || (di == dj && i < j));
    rk += before;
  }
  rank[j] = rk;
  w[rk] = dj;
}

template <class T>
__global__ void permute_cols_kernel(int n, int m, const int *__restrict__ pos, const T *__restrict__ in, long ldi,
                                    T *__restrict__ out, long ldo) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= n || j >= m) return;
  out[i + (long)pos[j] * ldo] = in[i + (long)j * ldi];
}

template <class T>
int heev_jacobi(cudaStream_t st, int m, T *A, double *w, T *V, T *work, double *dwork, int *iwork, int *hflag,
                int *sweeps_out) {
  if (m <= 0) return 0;
  CatScope cat_red(CAT_REDUCED);
  const int maxsw = 80;
  const int slot = prof_begin(st);
  if (int rc = jacobi_coop<T>(st, m, maxsw, A, V, work, dwork, iwork)) return rc;
  prof_end(st, slot, 0.0);
  // eigenvalues ascending with their vectors (rank by counting)
  int *rank = iwork + 2 * m + maxsw + 8;
  rank_kernel<T><<<ceil_div(m, 128), 128, 0, st>>>(m, A, w, rank);
  GBF_LAUNCHED();
  dim3 gp(ceil_div(m, 128), m);
  permute_cols_kernel<T><<<gp, 128, 0, st>>>(m, m, rank, V, m, work, m);
  GBF_LAUNCHED();
  GBF_CUDA(cudaMemcpyAsync(V, work, sizeof(T) * (size_t)m * m, cudaMemcpyDeviceToDevice, st));
  GBF_CUDA(cudaMemcpyAsync(hflag, iwork + 2 * m + maxsw, sizeof(int), cudaMemcpyDeviceToHost, st));
  GBF_CUDA(cudaStreamSynchronize(st));
  if (sweeps_out) *sweeps_out = *hflag;
  // per round every entry of A (up to 4 multiply-adds) and V (2) is rewritten
  const int P = m + (m & 1);
  prof_set_flops(slot, (double)(*hflag + 1) * (P - 1) * (double)m * m * (tr<T>::cplx ? 4.0 : 1.0) * 12.0);
  GBF_CUDA(cudaGetLastError());
  return 0;
}

// ------------------------------------------------------ Rayleigh-Ritz glue --
// s_i = 1 / sqrt(Re Bq_ii); flag when a diagonal is not positive.
template <class T>
__global__ void rr_diag_kernel(int m, const T *Bq, double *s, int *flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const double d = tr<T>::re(Bq[i + (long)i * m]);
  if (!(d > 0.0)) {
    atomicOr(flag, 1);
    s[i] = 0.0;
  } else {
    s[i] = 1.0 / sqrt(d);
  }
}

// out = s_i s_j (M + M^H)/2 for M in {Aq, Bq}
template <class T>
__global__ void rr_scale_kernel(int m, const double *s, const T *Aq, const T *Bq, T *As, T *Bs) {
  using X = tr<T>;
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t >= (long)m * m) return;
  const int i = (int)(t % m), j = (int)(t / m);
  const double f = 0.5 * s[i] * s[j];
  As[t] = scaleT(X::add(Aq[t], X::conj(Aq[j + (long)i * m])), f);
  Bs[t] = scaleT(X::add(Bq[t], X::conj(Bq[j + (long)i * m])), f);
}

// T[:, j] = V[:, first + j] / sqrt(d[first + j])
template <class T>
__global__ void make_t_kernel(int m, int mk, int first, const T *V, const double *d, T *Tm) {
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t >= (long)m * mk) return;
  const int i = (int)(t % m), j = (int)(t / m);
  Tm[t] = scaleT(V[i + (long)(first + j) * m], 1.0 / sqrt(d[first + j]));
}

template <class T>
__global__ void hermitize_kernel(int m, const T *Cin, T *Cout) {
  using X = tr<T>;
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t >= (long)m * m) return;
  const int i = (int)(t % m), j = (int)(t / m);
  Cout[t] = scaleT(X::add(Cin[t], X::conj(Cin[j + (long)i * m])), 0.5);
}

template <class T>
__global__ void scale_rows_kernel(int m, int mk, const double *s, T *W) {
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t >= (long)m * mk) return;
  W[t] = scaleT(W[t], s[t % m]);
}

// res_j = ||AX_j - lam_j BX_j||_1 / ||alpha BX_j||_1  (Table tab_common)
template <class T>
__global__ void ritz_residual_kernel(int n, const T *AX, const T *BX, const double *lam, double alpha,
                                     double *res) {
  using X = tr<T>;
  __shared__ double rn[256], rd[256];
  const int j = blockIdx.x;
  const double l = lam[j];
  double num = 0.0, den = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const T bx = BX[i + (long)j * n];
    num += absT(X::sub(AX[i + (long)j * n], scaleT(bx, l)));
    den += absT(scaleT(bx, alpha));
  }
  rn[threadIdx.x] = num;
  rd[threadIdx.x] = den;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      rn[threadIdx.x] += rn[threadIdx.x + o];
      rd[threadIdx.x] += rd[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) res[j] = rn[0] / rd[0];
}

// Spurious Ritz pairs (from loop 1 on, when the previous subspace Y is the
// B-orthonormal set of previous Ritz vectors): x_j = Q w_j is the filter
// applied to z_j = Y w_j, ||z_j||_B = ||w_j||_2, ||x_j||_B = 1, so the
// filter's gain on the pre-image is 1/||w_j||_2; genuine pairs have a gain
// ~ f(lambda_j) (>= 1/2 inside), a pair inside with gain < f(lambda_j)/4 is
// spurious (Table tab_common: spurious pairs go last with res = -1).
template <class T>
__global__ void spurious_kernel(int m, int mk, const T *W, const double *lam, double emin, double emax,
                                const double *f, int check, int *spur) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= mk) return;
  const double l = lam[j];
  int sp = 0;
  if (check && l >= emin && l <= emax) {
    double s = 0.0;
    for (int i = 0; i < m; ++i) {
      const double a = absT(W[i + (long)j * m]);
      s += a * a;
    }
    sp = (1.0 / sqrt(s) < 0.25 * fabs(f[j])) ? 1 : 0;
  }
  spur[j] = sp;
}

// Output order: genuine Ritz values inside [emin, emax] ascending, then the
// outside ones ascending, then spurious ones (lam is ascending).
// pos[j] = output slot of Ritz pair j; *nin_out = genuine inside count.
__global__ void order_kernel(int mk, const double *lam, const int *spur, double emin, double emax, int *pos,
                             int *nin_out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= mk) return;
  auto cls = [&](int i) {
    const double li = lam[i];
    const bool in = (li >= emin && li <= emax);
    return spur[i] ? 2 : (in ? 0 : 1);
  };
  const int cj = cls(j);
  int p = 0, nin = 0;
  for (int i = 0; i < mk; ++i) {
    const int ci = cls(i);
    nin += (ci == 0);
    if (ci < cj || (ci == cj && i < j)) ++p;
  }
  pos[j] = p;
  if (j == 0) *nin_out = nin;
}

__global__ void place_kernel(int mk, const int *pos, const int *spur, const double *lam, const double *res, double *E,
                             double *R) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= mk) return;
  E[pos[j]] = lam[j];
  R[pos[j]] = spur[j] ? -1.0 : res[j];
}

// trace over the first nin (ascending order) and max residual there
__global__ void stats_kernel(int mk, const int *nin_p, const double *E, const double *R, double *out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int nin = *nin_p;
  double tr_ = 0.0, mr = 0.0;
  bool finite = true;
  for (int j = 0; j < nin; ++j) {
    tr_ += E[j];
    if (R[j] > mr) mr = R[j];
  }
  for (int j = 0; j < mk; ++j)
    if (!isfinite(E[j]) || !isfinite(R[j])) finite = false;
  out[0] = nin;
  out[1] = tr_;
  out[2] = mr;
  out[3] = finite ? 1.0 : 0.0;
}

// Rational filter values f_j = sum_e Re[w_e / (z_e - lam_j)] and the diagonal
// scalings D_e[j] = 1/(z_e - lam_j), Dc_e[j] = 1/(conj(z_e) - lam_j).
__global__ void filter_kernel(int mk, int ne, const zd *z, const zd *w, const double *lam, double *f, zd *D,
                              zd *Dc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= mk) return;
  const double l = lam[j];
  double s = 0.0;
  for (int e = 0; e < ne; ++e) {
    const zd d = zdiv(zd{1.0, 0.0}, zd{z[e].x - l, z[e].y});
    const zd dc = zdiv(zd{1.0, 0.0}, zd{z[e].x - l, -z[e].y});
    D[(long)e * mk + j] = d;
    Dc[(long)e * mk + j] = dc;
    s += zmul(w[e], d).x;
  }
  f[j] = s;
}

// Newton-Schulz step helper: norm = ||I - P||_F (one block, fixed order) and,
// when T is given, T = (3I - P)/2.
template <class T>
__global__ void ns_prep_kernel(int m, const T *P, T *Tn, double *norm) {
  using X = tr<T>;
  __shared__ double red[1024];
  double s = 0.0;
  for (long t = threadIdx.x; t < (long)m * m; t += blockDim.x) {
    const int i = (int)(t % m), j = (int)(t / m);
    T e = X::neg(P[t]);
    if (i == j) e = X::add(e, X::one());
    const double a = absT(e);
    s += a * a;
    if (Tn) {
      T v = scaleT(X::neg(P[t]), 0.5);
      if (i == j) v = X::add(v, cvt<T, double>(1.5));
      Tn[t] = v;
    }
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *norm = sqrt(red[0]);
}

template <class T>
int ns_prep(cudaStream_t st, int m, const T *P, T *Tn, double *norm) {
  ns_prep_kernel<T><<<1, 1024, 0, st>>>(m, P, Tn, norm);
  GBF_LAUNCHED();
  return 0;
}

// R = AX - BX diag(lam)
template <class T>
__global__ void eig_residual_kernel(int n, int mk, const T *AX, const T *BX, const double *lam, T *R) {
  using X = tr<T>;
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t >= (long)n * mk) return;
  R[t] = X::sub(AX[t], scaleT(BX[t], lam[t / n]));
}

// Quadrature sum (fused over nodes, in node order):
//   real symmetric:    Q = X0 f + sum_e Re(w_e Y_e)
//   complex Hermitian: Q = X0 f + sum_e (w_e Y_e + conj(w_e) Yadj_e) / 2
// X0/f optional (residual-correction form of the mixed path).
template <class TQ> __device__ inline void store_q(TQ &q, zd v);
template <> __device__ inline void store_q<double>(double &q, zd v) { q = v.x; }
template <> __device__ inline void store_q<zd>(zd &q, zd v) { q = v; }
__device__ inline zd as_zd(double v) { return zd{v, 0.0}; }
__device__ inline zd as_zd(zd v) { return v; }

template <class TY, class TQ>
__global__ void accumulate_kernel(int n, int m, int ne, const zd *__restrict__ w, const TY *__restrict__ Y,
                                  const TY *__restrict__ Yadj, const TQ *__restrict__ X0,
                                  const double *__restrict__ f, TQ *__restrict__ Q) {
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  const long nm = (long)n * m;
  if (t >= nm) return;
  zd acc = zd{0.0, 0.0};
  if (X0) {
    const zd x = as_zd(X0[t]);
    const double fj = f[t / n];
    acc = zd{x.x * fj, x.y * fj};
  }
  for (int e = 0; e < ne; ++e) {
    const zd y = cvt<zd, TY>(Y[e * nm + t]);
    const zd a = zmul(w[e], y);
    if (Yadj) {
      const zd ya = cvt<zd, TY>(Yadj[e * nm + t]);
      const zd b = zmul(zd{w[e].x, -w[e].y}, ya);
      acc.x += 0.5 * (a.x + b.x);
      acc.y += 0.5 * (a.y + b.y);
    } else {
      acc.x += a.x;
    }
  }
  store_q<TQ>(Q[t], acc);
}

// SplitMix64 (Steele, Lea & Flood 2014), counter form: mix(seed + (i+1) G).
__device__ inline uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ inline double u11(uint64_t seed, uint64_t i) {
  return (double)(splitmix64_at(seed, i) >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}
template <class TQ> __device__ inline TQ rand_entry(uint64_t seed, uint64_t i);
template <> __device__ inline double rand_entry<double>(uint64_t seed, uint64_t i) { return u11(seed, i); }
template <> __device__ inline zd rand_entry<zd>(uint64_t seed, uint64_t i) {
  return zd{u11(seed, 2 * i), u11(seed, 2 * i + 1)};
}
template <class TQ>
__global__ void random_subspace_kernel(long count, uint64_t seed, TQ *Y) {
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t < count) Y[t] = rand_entry<TQ>(seed, (uint64_t)t);
}
// Rademacher probes of the stochastic count: +1 or -1 by the top bit of the
// generator at the column-major index (real part only for complex types).
template <class TQ>
__global__ void rademacher_kernel(long count, uint64_t seed, TQ *Y) {
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t < count) {
    TQ v = tr<TQ>::zero();
    reinterpret_cast<double *>(&v)[0] = (splitmix64_at(seed, (uint64_t)t) >> 63) ? -1.0 : 1.0;
    Y[t] = v;
  }
}

// Stochastic count, one block per probe column j: t_j = Re(y_j^H q_j) with a
// fixed-order FP64 tree (each thread strides the rows, then a shared-memory
// halving), so the result does not depend on scheduling.
constexpr int PROBE_THREADS = 256;
template <class TQ>
__global__ void __launch_bounds__(PROBE_THREADS) probe_form_kernel(int n, const TQ *Y, const TQ *Q, double *t) {
  __shared__ double red[PROBE_THREADS];
  const TQ *y = Y + (size_t)blockIdx.x * n, *q = Q + (size_t)blockIdx.x * n;
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += PROBE_THREADS) acc += tr<TQ>::re(tr<TQ>::mul(tr<TQ>::conj(y[i]), q[i]));
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = PROBE_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) t[blockIdx.x] = red[0];
}
// res(j) = (t_1 + ... + t_j) / j, in place; one thread (m is the probe count).
__global__ void running_mean_kernel(int m, double *res) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int j = 0; j < m; ++j) {
    s += res[j];
    res[j] = s / (j + 1);
  }
}

// ------------------------------------------------------------ launchers --
#define L1D(count) ceil_div((long)(count), 256), 256, 0, st

template <class T>
int rr_prepare(cudaStream_t st, int m, const T *Aq, const T *Bq, double *s, int *flag, T *As, T *Bs) {
  rr_diag_kernel<T><<<ceil_div(m, 128), 128, 0, st>>>(m, Bq, s, flag);
  GBF_LAUNCHED();
  rr_scale_kernel<T><<<L1D((long)m * m)>>>(m, s, Aq, Bq, As, Bs);
  GBF_LAUNCHED();
  GBF_CUDA(cudaGetLastError());
  return 0;
}
template <class T>
int make_t(cudaStream_t st, int m, int mk, int first, const T *V, const double *d, T *Tm) {
  make_t_kernel<T><<<L1D((long)m * mk)>>>(m, mk, first, V, d, Tm);
  GBF_LAUNCHED();
  return 0;
}
template <class T>
int hermitize(cudaStream_t st, int m, const T *Cin, T *Cout) {
  hermitize_kernel<T><<<L1D((long)m * m)>>>(m, Cin, Cout);
  GBF_LAUNCHED();
  return 0;
}
template <class T>
int scale_rows(cudaStream_t st, int m, int mk, const double *s, T *W) {
  scale_rows_kernel<T><<<L1D((long)m * mk)>>>(m, mk, s, W);
  GBF_LAUNCHED();
  return 0;
}
template <class T>
int ritz_residual(cudaStream_t st, int n, int mk, const T *AX, const T *BX, const double *lam, double alpha,
                  double *res) {
  ritz_residual_kernel<T><<<mk, 256, 0, st>>>(n, AX, BX, lam, alpha, res);
  GBF_LAUNCHED();
  return 0;
}
template <class T>
int spurious_flags(cudaStream_t st, int m, int mk, const T *W, const double *lam, double emin, double emax,
                   const double *f, int check, int *spur) {
  spurious_kernel<T><<<ceil_div(mk, 128), 128, 0, st>>>(m, mk, W, lam, emin, emax, f, check, spur);
  GBF_LAUNCHED();
  return 0;
}
int order_and_stats(cudaStream_t st, int mk, const double *lam, const double *res, const int *spur, double emin,
                    double emax, int *pos, int *nin, double *E, double *R, double *stats) {
  order_kernel<<<ceil_div(mk, 128), 128, 0, st>>>(mk, lam, spur, emin, emax, pos, nin);
  GBF_LAUNCHED();
  place_kernel<<<ceil_div(mk, 128), 128, 0, st>>>(mk, pos, spur, lam, res, E, R);
  GBF_LAUNCHED();
  stats_kernel<<<1, 32, 0, st>>>(mk, nin, E, R, stats);
  GBF_LAUNCHED();
  GBF_CUDA(cudaGetLastError());
  return 0;
}
template <class T>
int permute_cols(cudaStream_t st, int n, int m, const int *pos, const T *in, T *out) {
  dim3 g(ceil_div(n, 256), m);
  permute_cols_kernel<T><<<g, 256, 0, st>>>(n, m, pos, in, n, out, n);
  GBF_LAUNCHED();
  return 0;
}
int filter_values(cudaStream_t st, int mk, int ne, const zd *z, const zd *w, const double *lam, double *f, zd *D,
                  zd *Dc) {
  filter_kernel<<<ceil_div(mk, 128), 128, 0, st>>>(mk, ne, z, w, lam, f, D, Dc);
  GBF_LAUNCHED();
  return 0;
}
template <class T>
int eig_residual(cudaStream_t st, int n, int mk, const T *AX, const T *BX, const double *lam, T *R) {
  eig_residual_kernel<T><<<L1D((long)n * mk)>>>(n, mk, AX, BX, lam, R);
  GBF_LAUNCHED();
  return 0;
}
template <class TY, class TQ>
int accumulate(cudaStream_t st, int n, int m, int ne, const zd *w, const TY *Y, const TY *Yadj, const TQ *X0,
               const double *f, TQ *Q) {
  accumulate_kernel<TY, TQ><<<L1D((long)n * m)>>>(n, m, ne, w, Y, Yadj, X0, f, Q);
  GBF_LAUNCHED();
  GBF_CUDA(cudaGetLastError());
  return 0;
}
template <class TQ>
int random_subspace(cudaStream_t st, long count, uint64_t seed, TQ *Y) {
  random_subspace_kernel<TQ><<<L1D(count)>>>(count, seed, Y);
  GBF_LAUNCHED();
  return 0;
}

template <class TQ>
int rademacher_probes(cudaStream_t st, long count, uint64_t seed, TQ *Y) {
  rademacher_kernel<TQ><<<L1D(count)>>>(count, seed, Y);
  GBF_LAUNCHED();
  return 0;
}
template <class TQ>
int probe_running_mean(cudaStream_t st, int n, int m, const TQ *Y, const TQ *Q, double *res) {
  if (m < 1) return 0;
  probe_form_kernel<TQ><<<m, PROBE_THREADS, 0, st>>>(n, Y, Q, res);
  GBF_LAUNCHED();
  running_mean_kernel<<<1, 32, 0, st>>>(m, res);
  GBF_LAUNCHED();
  GBF_CUDA(cudaGetLastError());
  return 0;
}

#define EIG_INST(T)                                                                                         \
  template int heev_jacobi<T>(cudaStream_t, int, T *, double *, T *, T *, double *, int *, int *, int *);   \
  template int rr_prepare<T>(cudaStream_t, int, const T *, const T *, double *, int *, T *, T *);           \
  template int make_t<T>(cudaStream_t, int, int, int, const T *, const double *, T *);                      \
  template int hermitize<T>(cudaStream_t, int, const T *, T *);                                             \
  template int scale_rows<T>(cudaStream_t, int, int, const double *, T *);                                  \
  template int ritz_residual<T>(cudaStream_t, int, int, const T *, const T *, const double *, double,       \
                                double *);                                                                  \
  template int permute_cols<T>(cudaStream_t, int, int, const int *, const T *, T *);                        \
  template int eig_residual<T>(cudaStream_t, int, int, const T *, const T *, const double *, T *);          \
  template int random_subspace<T>(cudaStream_t, long, uint64_t, T *);                                \
  template int rademacher_probes<T>(cudaStream_t, long, uint64_t, T *);                              \
  template int probe_running_mean<T>(cudaStream_t, int, int, const T *, const T *, double *);        \
  template int spurious_flags<T>(cudaStream_t, int, int, const T *, const double *, double, double,        \
                                 const double *, int, int *);                                             \
  template int ns_prep<T>(cudaStream_t, int, const T *, T *, double *);
EIG_INST(double)
EIG_INST(zd)
template int accumulate<zd, double>(cudaStream_t, int, int, int, const zd *, const zd *, const zd *,
                                    const double *, const double *, double *);
template int accumulate<zd, zd>(cudaStream_t, int, int, int, const zd *, const zd *, const zd *, const zd *,
                                const double *, zd *);
template int accumulate<cf, double>(cudaStream_t, int, int, int, const zd *, const cf *, const cf *,
                                    const double *, const double *, double *);
template int accumulate<cf, zd>(cudaStream_t, int, int, int, const zd *, const cf *, const cf *, const zd *,
                                const double *, zd *);

}  // namespace gbf
