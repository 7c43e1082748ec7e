// Reduced dense Hermitian eigensolver of the Rayleigh-Ritz step (FEAST v3.0
// guide, "The FEAST Algorithm": the reduced eigenproblem Aq W = Bq W Lambda,
// solved after B-orthonormalisation as a standard Hermitian problem C U = U
// Lambda) and the Cholesky factor of the B-orthonormalisation, as
// thread-block-cluster kernels.
//
// The M0 x M0 problems are small (M0 <= a few hundred) but their O(M0^3)
// work is FP64, which runs at ~2 fused multiply-adds per clock per SM on this
// GPU.  A cyclic Jacobi method costs ~6 M0^3 multiply-adds per sweep and
// (in a grid-wide form) one grid barrier per round; the path here costs
// ~M0^3 multiply-adds in all and keeps its M0-step recurrences inside one
// cluster, whose barrier is a hardware barrier:
//
//   sytrd_cluster   Householder reduction C = Q T_c Q^H to a Hermitian
//                   tridiagonal T_c (one cluster of up to 16 CTAs; the
//                   matrix lives in distributed shared memory, rows dealt
//                   cyclically to the CTAs; one cluster barrier per column)
//   tridiag_prep    T_c = D T D^H with T real symmetric tridiagonal (D a
//                   diagonal of unit phases), Gershgorin bounds
//   stebz           every eigenvalue of T by bisection on its Sturm count
//                   (the sign changes of the characteristic-polynomial
//                   recurrence, rescaled against overflow), one warp each
//                   (32-point multisection)
//   stein           eigenvectors of T by inverse iteration (tridiagonal LU
//                   with partial pivoting of T - lambda I), two steps from
//                   a fixed pseudo-random start (three in a cluster);
//                   eigenvalues closer than
//                   1e-10 ||T|| form a cluster whose vectors one thread
//                   computes in turn, each orthogonalised against the
//                   previous ones
//   ormtr           U = Q D Z: the reflectors applied to D Z in reverse
//                   order, a few columns per CTA
//   chol_cluster    C = L L^H (lower), right-looking, the same cluster layout
//
// Householder reflector of step j (column j below the diagonal, x):
//   H = I - tau v v^H with v = (1, x_2..x_k) / (ph (|x_1| + ||x||)),
//   ph = x_1 / |x_1| (1 if x_1 = 0), tau = 1 + |x_1| / ||x||, so that
//   H x = -ph ||x|| e_1 (H Hermitian and unitary); the trailing block
//   becomes A - v w^H - w v^H with p = tau A v, w = p - (tau/2)(v^H p) v.
#include <cooperative_groups.h>

#include <algorithm>

#include "gbf_common.cuh"

namespace cg = cooperative_groups;

namespace gbf {

constexpr int TRD_THREADS = 640;
constexpr int TRD_SMEM_CAP = 200 * 1024;

__device__ inline double absq(double a) { return a * a; }
__device__ inline double absq(zd a) { return a.x * a.x + a.y * a.y; }
__device__ inline double scl(double a, double s) { return a * s; }
__device__ inline zd scl(zd a, double s) { return zd{a.x * s, a.y * s}; }
__device__ inline double shfl_x(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ inline zd shfl_x(zd v, int o) {
  return zd{__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o)};
}
// Sum over the warp of one double per lane, exactly in fixed point and
// rounded once: each value is shifted to the warp's largest exponent (57
// significant bits kept; the bits dropped lie below 2^-57 of the largest
// term), the 32 integers are summed by hardware warp reductions on three
// 20-bit chunks (no carry can leave a chunk), and the sum is converted once.
// Independent of the lanes' order, hence the same in every CTA.  In these
// kernels a shuffle-and-add butterfly took several times longer than its
// latency in isolation while the other CTAs' remote loads were being served.
// Zero, infinite or NaN extremes take the butterfly.
__device__ inline double warp_sum_fx(double v) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  const int ex = (int)((bits >> 52) & 0x7FF);
  const unsigned emax = __reduce_max_sync(0xffffffffu, (unsigned)ex);
  if (emax == 0 || emax == 0x7FF) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
  }
  const unsigned long long mant = (bits & 0x000FFFFFFFFFFFFFull) | (ex ? 0x0010000000000000ull : 0ull);
  const int sh = (int)emax - (ex ? ex : 1);  // >= 0
  const long long q = sh > 57 ? 0LL : (long long)((mant << 4) >> sh);  // < 2^57
  const unsigned long long u = (unsigned long long)((bits >> 63) ? -q : q) + (1ull << 57);  // in [0, 2^58)
  const unsigned c0 = __reduce_add_sync(0xffffffffu, (unsigned)(u & 0xFFFFFu));
  const unsigned c1 = __reduce_add_sync(0xffffffffu, (unsigned)((u >> 20) & 0xFFFFFu));
  const unsigned c2 = __reduce_add_sync(0xffffffffu, (unsigned)(u >> 40));
  const long long sum = (long long)((unsigned long long)c0 + ((unsigned long long)c1 << 20) +
                                    ((unsigned long long)c2 << 40) - (32ull << 57));
  // value = sum 2^(emax - 1075 - 4); emax - 1079 >= -1078 may be below the
  // normal range: scale in two exact steps
  const int e2 = (int)emax - 1079;
  const double h = __longlong_as_double((long long)(e2 / 2 + 1023) << 52);
  const double r = __longlong_as_double((long long)(e2 - e2 / 2 + 1023) << 52);
  return (__ll2double_rn(sum) * h) * r;
}
__device__ inline double warp_sum_v(double v) { return warp_sum_fx(v); }
__device__ inline zd warp_sum_v(zd v) { return zd{warp_sum_fx(v.x), warp_sum_fx(v.y)}; }
template <class T> __device__ inline T warp_sum(T v) { return warp_sum_v(v); }

// Deterministic CTA sum of one value per thread (fixed shuffle pattern, then
// the warps' partials in warp order, added by one thread: FP64 instructions
// are scarce, so the final sum is not repeated by every warp).  Every thread
// gets the result (red[32] holds it).
template <class T> __device__ T cta_sum(T v, T *red) {
  using X = tr<T>;
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    T s = X::zero();
    for (int i = 0; i < nw; ++i) s = X::add(s, red[i]);
    red[32] = s;
  }
  __syncthreads();
  return red[32];
}

// The cluster kernels deal the rows of the m x m matrix cyclically to the C
// CTAs of the cluster: row i lives in CTA i % C at local row i / C, stored
// whole (m entries) in that CTA's shared memory.

// ------------------------------------------------- tridiagonalisation --
// Step j, with the rows of the trailing block dealt to the CTAs as above and
// one cluster barrier per step:
//  (a) every CTA holds row j as updated by steps 0..j-1 (xrow) and forms
//      the reflector from it (the matrix is Hermitian, so column j below
//      the diagonal is the conjugate of row j right of it): the same inputs
//      and the same instructions give the same v and tau in every CTA, so
//      nothing is published; the owner of row j writes tau, the new
//      subdiagonal entry, column j of Vr and the diagonal entry;
//  (b) p_i = tau sum_k A[i][k] v_k for the own rows i > j (one warp per
//      row) and this CTA's part of v^H p, written into every CTA's buffers
//      of the step's parity; the owner of row j+1, who never updates it in
//      place after step j-1, writes it into every CTA as well;
//  -- cluster barrier --
//  (c) every CTA sums the parts of v^H p in CTA order (so K = tau/2
//      Re(v^H p) is the same everywhere), forms w = p - K v, updates its own
//      rows i > j+1 by A[i][k] -= v_i conj(w_k) + w_i conj(v_k), and row j+1
//      the same way in xrow.
// Everything a CTA needs after the barrier is in its own shared memory: the
// writes to other CTAs go out before the barrier, no remote load waits after
// it.  FP64 work as fused multiply-adds.
template <class T>
__global__ void __launch_bounds__(TRD_THREADS, 1)
    sytrd_cluster_kernel(int m, const T *__restrict__ A, long lda, T *__restrict__ Vr, double *__restrict__ tau,
                         T *__restrict__ betac, double *__restrict__ dd) {
  using X = tr<T>;
  constexpr int NW = TRD_THREADS / 32;
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks(), q = (int)cl.block_rank();
  const int rl = (m + C - 1) / C;
  extern __shared__ __align__(16) unsigned char smem[];
  T *L = reinterpret_cast<T *>(smem);  // [rl][m]
  T *pfull = L + (size_t)rl * m;       // [2][m] p of every row, by step parity (written by the rows' CTAs)
  T *xnext = pfull + 2 * (size_t)m;    // [2][m] row j+1 as its owner holds it, by step parity
  T *vfull = xnext + 2 * (size_t)m;    // [m] v of the current step
  T *wfull = vfull + m;                // [m] w of the current step
  T *xrow = wfull + m;                 // [m] row j as updated by the steps before j
  __shared__ T s_pvw[NW];              // each warp's part of v^H p
  __shared__ T s_parts[2][16];         // every CTA's part of v^H p, by step parity
  __shared__ double s_tau;
  __shared__ T s_sc, s_tot;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  for (long t = tid; t < (long)rl * m; t += blockDim.x) {
    const int k = (int)(t / rl), il = (int)(t % rl);
    const int i = il * C + q;
    L[(long)il * m + k] = (i < m) ? A[i + (long)k * lda] : X::zero();
  }
  cl.sync();  // every CTA's rows in place before the first remote read
  {
    const T *r0 = cl.map_shared_rank(L, 0);  // row 0: local row 0 of CTA 0
    for (int k = tid; k < m; k += blockDim.x) xrow[k] = r0[k];
  }
  __syncthreads();

  for (int j = 0; j < m - 1; ++j) {
    const int par = j & 1;
    const bool own = (j % C) == q;
    // (a) x = conj(xrow)[j+1 ..]: ||x_{2..}||^2 by warp 0 (fixed order),
    // the reflector by its lane 0, v by the whole CTA
    if (warp == 0) {
      double part = 0.0;
      for (int k = j + 2 + lane; k < m; k += 32) part += absq(xrow[k]);
      const double rest = warp_sum(part);
      if (lane == 0) {
        const T x0 = X::conj(xrow[j + 1]);
        double tj = 0.0;
        T beta = x0, sc = X::zero();
        if (rest > 0.0) {
          // |x0| and ||x|| from reciprocal square roots (independent),
          // then one reciprocal: the shortest chain on the FP64 unit
          const double q0 = absq(x0), s2 = q0 + rest;
          const double ia0 = q0 > 0.0 ? fast_rsqrt(q0) : 0.0, inx = fast_rsqrt(s2);
          const double a0 = q0 * ia0, nx = s2 * inx;
          const T ph = a0 > 0.0 ? scl(x0, ia0) : X::one();
          beta = scl(ph, -nx);
          sc = scl(X::conj(ph), fast_rcp(a0 + nx));
          tj = 1.0 + a0 * inx;
        }
        s_tau = tj;
        s_sc = sc;
        if (own) {
          tau[j] = tj;
          betac[j] = beta;
          dd[j] = X::re(xrow[j]);
        }
      }
    }
    __syncthreads();
    const double tj = s_tau;
    {
      const T sc = s_sc;
      for (int k = j + 1 + tid; k < m; k += blockDim.x) {
        const T v = (k == j + 1) ? X::one() : X::mul(X::conj(xrow[k]), sc);
        vfull[k] = v;
        if (own) Vr[k + (long)j * m] = v;
      }
    }
    __syncthreads();
    // (b) p_i for the own rows i > j, one warp per row; each warp's part of
    // v^H p to s_pvw, this CTA's part (the warps' parts in warp order) to
    // s_pcta
    T pv = X::zero();
    for (int il = warp; il < rl; il += NW) {
      const int i = il * C + q;
      if (i < j + 1 || i >= m) continue;
      const T *Li = L + (long)il * m;
      T s = X::zero();
      for (int k = j + 1 + lane; k < m; k += 32) s = X::fma(Li[k], vfull[k], s);
      s = scl(warp_sum(s), tj);
      if (lane < C) cl.map_shared_rank(pfull, lane)[(size_t)par * m + i] = s;
      pv = X::fma(X::conj(vfull[i]), s, pv);
    }
    if (lane == 0) s_pvw[warp] = pv;
    if ((j + 1) % C == q) {  // row j+1, as the step j-1 update left it, into every CTA
      const T *rn = L + (size_t)((j + 1) / C) * m;
      for (int k = j + 1 + tid; k < m; k += blockDim.x) {
        const T v = rn[k];
        for (int d = 0; d < C; ++d) cl.map_shared_rank(xnext, d)[(size_t)par * m + k] = v;
      }
    }
    __syncthreads();
    if (warp == 0) {
      const T r = warp_sum(lane < NW ? s_pvw[lane] : X::zero());
      if (lane < C) cl.map_shared_rank(&s_parts[0][0], lane)[par * 16 + q] = r;
    }
    cl.sync();  // every CTA's p, part of v^H p and row j+1 in every CTA
    // (c) v^H p: the C parts in CTA order (the same sum in every CTA)
    if (warp == 0) {
      const T tot = warp_sum(lane < C ? s_parts[par][lane] : X::zero());
      if (lane == 0) s_tot = tot;
    }
    for (int k = j + 1 + tid; k < m; k += blockDim.x) xrow[k] = xnext[(size_t)par * m + k];
    __syncthreads();
    const double kk = 0.5 * tj * X::re(s_tot);
    for (int k = j + 1 + tid; k < m; k += blockDim.x)
      wfull[k] = X::sub(pfull[(size_t)par * m + k], scl(vfull[k], kk));
    __syncthreads();
    // A[i][k] -= v_i conj(w_k) + w_i conj(v_k): own rows i > j+1 (one warp
    // per row, lanes over the columns k > j), and row j+1 in xrow
    for (int il = warp; il < rl; il += NW) {
      const int i = il * C + q;
      if (i < j + 2 || i >= m) continue;
      T *Li = L + (long)il * m;
      const T vi = X::neg(vfull[i]), wi = X::neg(wfull[i]);
      for (int k = j + 1 + lane; k < m; k += 32) {
        T a = Li[k];
        a = X::fma(vi, X::conj(wfull[k]), a);
        a = X::fma(wi, X::conj(vfull[k]), a);
        Li[k] = a;
      }
    }
    {
      const T vi = X::neg(vfull[j + 1]), wi = X::neg(wfull[j + 1]);
      for (int k = j + 1 + tid; k < m; k += blockDim.x) {
        T a = xrow[k];
        a = X::fma(vi, X::conj(wfull[k]), a);
        a = X::fma(wi, X::conj(vfull[k]), a);
        xrow[k] = a;
      }
    }
    __syncthreads();
  }
  if (tid == 0 && ((m - 1) % C) == q) dd[m - 1] = X::re(xrow[m - 1]);
  cl.sync();  // no CTA leaves while another may read its shared memory
}

// T_c (diagonal dd, subdiagonal betac) = D T D^H with T real (diagonal dd,
// subdiagonal e = |betac|), D = diag(delta): delta_0 = 1, delta_{k+1} =
// delta_k betac_k / |betac_k| (a prefix product of unit phases, formed by a
// parallel scan).  Also e^2 and the Gershgorin interval [gl, gu] with tnorm
// = max(|gl|, |gu|) in sc[0..2].  One block of PREP_THREADS >= m threads.
constexpr int PREP_THREADS = 1024;
template <class T>
__global__ void __launch_bounds__(PREP_THREADS) tridiag_prep_kernel(int m, const double *dd, const T *betac, double *e,
                                                                   double *e2, T *delta, double *sc) {
  using X = tr<T>;
  __shared__ T ph[PREP_THREADS];
  __shared__ double mn[PREP_THREADS / 32], mx[PREP_THREADS / 32];
  const int k = threadIdx.x;
  double ek = 0.0;
  T u = X::one();  // phase of betac_{k-1} (1 for k = 0)
  if (k < m - 1) {
    ek = sqrt(absq(betac[k]));
    e[k] = ek;
    e2[k] = ek * ek;
  }
  if (k >= 1 && k < m) {
    const double a = sqrt(absq(betac[k - 1]));
    if (a > 0.0) u = scl(betac[k - 1], 1.0 / a);
  }
  ph[k] = u;
  __syncthreads();
  for (int o = 1; o < PREP_THREADS; o <<= 1) {  // inclusive scan: delta_k = u_1 ... u_k
    const T v = (k >= o) ? ph[k - o] : X::one();
    __syncthreads();
    ph[k] = X::mul(v, ph[k]);
    __syncthreads();
  }
  if (k < m) delta[k] = ph[k];
  double lo = 1e300, hi = -1e300;
  if (k < m) {
    const double r = (k > 0 ? sqrt(absq(betac[k - 1])) : 0.0) + ek;
    lo = dd[k] - r;
    hi = dd[k] + r;
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if ((k & 31) == 0) {
    mn[k >> 5] = lo;
    mx[k >> 5] = hi;
  }
  __syncthreads();
  if (k == 0) {
    double gl = mn[0], gu = mx[0];
    for (int w = 1; w < PREP_THREADS / 32; ++w) {
      gl = fmin(gl, mn[w]);
      gu = fmax(gu, mx[w]);
    }
    const double tn = fmax(fabs(gl), fabs(gu));
    sc[0] = gl - 2.2e-16 * tn * 2 * m - 1e-300;
    sc[1] = gu + 2.2e-16 * tn * 2 * m + 1e-300;
    sc[2] = tn;
  }
}

// ----------------------------------------------------------- bisection --
// Number of eigenvalues of T below x: sign changes of 1, p_0, ..., p_{m-1},
// p_k = (d_k - x) p_{k-1} - e_{k-1}^2 p_{k-2}, i.e. the negative pivots of
// the LDL^T factorisation of T - x I.  A zero p_k counts as a sign change
// (as a tiny negative pivot).  The pair (p_{k-1}, p_k) is rescaled by
// powers of two whenever p_k leaves [2^-600, 2^600].  Three FP64
// operations per step; signs, zero tests and exponents are read from the
// bit patterns with integer operations (FP64 instructions are the scarce
// resource on this GPU).
__device__ inline int sgnb(double v) { return (int)((unsigned long long)__double_as_longlong(v) >> 63); }
__device__ inline int expb(double v) { return (int)(((unsigned long long)__double_as_longlong(v) >> 52) & 0x7FF); }
__device__ inline bool zerob(double v) { return ((unsigned long long)__double_as_longlong(v) << 1) == 0ull; }

__device__ inline int sturm_count(int m, const double *__restrict__ d, const double *__restrict__ e2, double x) {
  // per step: three FP64 operations and a few 32-bit integer operations on
  // the high word (sign, zero test, exponent range); the rare rescaling and
  // zero fix-up leave the main path
  double pm = 1.0, p = d[0] - x;
  if (zerob(p)) p = -0x1p-1000;
  int hp = __double2hiint(p);
  int cnt = (int)((unsigned)hp >> 31);
  for (int k = 1; k < m; ++k) {
    double pn = fma(d[k] - x, p, -(e2[k - 1] * pm));
    int hn = __double2hiint(pn);
    // biased exponent outside [1023 - 600, 1023 + 600], or zero / subnormal
    if ((unsigned)(((hn >> 20) & 0x7FF) - (1023 - 600)) > 1200u) {
      if (zerob(pn)) {
        pn = hp < 0 ? 0x1p-1000 : -0x1p-1000;
      } else if (((hn >> 20) & 0x7FF) > 1023 + 600) {
        pn *= 0x1p-600;
        p *= 0x1p-600;
      } else if (expb(p) < 1023 - 600) {
        pn *= 0x1p600;
        p *= 0x1p600;
      }
      hn = __double2hiint(pn);
    }
    cnt += (int)((unsigned)(hn ^ hp) >> 31);
    pm = p;
    p = pn;
    hp = hn;
  }
  return cnt;
}

// Eigenvalue k (ascending) lies in (lo, hi] with count(lo) <= k < count(hi).
// One warp per eigenvalue: its 32 lanes count at 32 interior points of the
// interval (multisection, 5 bits per round), until the interval is below
// 1e-3 eps ||T|| or holds no interior double; hi is returned (so an isolated
// eigenvalue that is a double, e.g. of a diagonal T, comes back exactly).
constexpr int STEBZ_WARPS = 1;
__global__ void __launch_bounds__(32 * STEBZ_WARPS) stebz_kernel(int m, const double *__restrict__ d,
                                                               const double *__restrict__ e2,
                                                               const double *__restrict__ sc, double *__restrict__ w) {
  const int k = blockIdx.x * STEBZ_WARPS + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (k >= m) return;  // warp-uniform
  double lo = sc[0], hi = sc[1];
  const double floor_w = 1e-3 * 2.220446049250313e-16 * sc[2];
  for (int round = 0; round < 40; ++round) {
    const double wd = hi - lo;
    if (wd <= floor_w) break;
    const double x = fma((double)(lane + 1), wd * (1.0 / 33.0), lo);
    int c;
    if (!(x > lo))
      c = 0;  // count(lo) <= k
    else if (!(x < hi))
      c = 1;  // count(hi) > k
    else
      c = sturm_count(m, d, e2, x) > k;
    const unsigned mask = __ballot_sync(0xffffffffu, c);
    double nlo, nhi;
    if (mask == 0u) {
      nlo = __shfl_sync(0xffffffffu, x, 31);
      nhi = hi;
    } else {
      const int f = __ffs(mask) - 1;
      nhi = __shfl_sync(0xffffffffu, x, f);
      const double xl = __shfl_sync(0xffffffffu, x, f > 0 ? f - 1 : 0);
      nlo = f > 0 ? xl : lo;
    }
    nlo = fmax(nlo, lo);
    nhi = fmin(nhi, hi);
    if (nlo == lo && nhi == hi) break;  // no interior double left
    lo = nlo;
    hi = nhi;
  }
  if (lane == 0) w[k] = hi;
}

// ---------------------------------------------------- inverse iteration --
__device__ inline double unit_rand(uint64_t k, uint64_t i) {
  uint64_t z = 0x9E3779B97F4A7C15ull * (k * 0x100000001B3ull + i + 1ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// Thread k (the first eigenvalue of its cluster) computes the eigenvectors
// of eigenvalues k, k+1, ... of its cluster (consecutive eigenvalues within
// 1e-10 tnorm of each other) into columns of Z (m x m, ld m).  Scratch: six
// m-vectors per thread, interleaved across the 32 lanes of a warp (element
// i of lane l at i * 32 + l) so that a warp's accesses are contiguous.
__global__ void __launch_bounds__(32) stein_kernel(int m, const double *__restrict__ d, const double *__restrict__ e,
                                                   const double *__restrict__ sc, const double *__restrict__ w,
                                                   double *__restrict__ Z, double *__restrict__ wk) {
  const int lane = threadIdx.x;
  const int k = blockIdx.x * 32 + lane;
  const size_t vs = (size_t)m * 32;
  double *base = wk + (size_t)blockIdx.x * 6 * vs + lane;
  double *a = base;            // U diagonal (then its reciprocals)
  double *b = base + vs;       // U first superdiagonal
  double *c2 = base + 2 * vs;  // U second superdiagonal
  double *l = base + 3 * vs;   // multipliers
  double *fl = base + 4 * vs;  // 1: rows i, i+1 swapped
  double *x = base + 5 * vs;   // the iterate
#define V(arr, i) arr[(size_t)(i) * 32]
  if (k >= m) return;
  const double tn = sc[2];
  const double ctol = 1e-10 * tn;
  if (k > 0 && w[k] - w[k - 1] <= ctol) return;  // not the first of its cluster
  int kend = k + 1;
  while (kend < m && w[kend] - w[kend - 1] <= ctol) ++kend;
  const double tiny = 2.220446049250313e-16 * tn + 1e-300;
  for (int kk = k; kk < kend; ++kk) {
    const double lam = w[kk];
    // LU with partial pivoting of T - lam I (tridiagonal; U gets a second
    // superdiagonal from the swaps), the running diagonal and superdiagonal
    // entries carried in registers; pivots below eps tnorm become eps tnorm
    // and are kept as reciprocals
    double ai = d[0] - lam, bi = m > 1 ? e[0] : 0.0;
    for (int i = 0; i < m - 1; ++i) {
      const double sub = e[i];
      const double dn = d[i + 1] - lam, en = (i + 1 < m - 1) ? e[i + 1] : 0.0;
      // one division per step: the pivot (raised to eps tnorm in modulus
      // when smaller) is inverted once and the multiplier formed from it
      const bool noswap = fabs(ai) >= fabs(sub);
      double piv = noswap ? ai : sub;
      if (fabs(piv) < tiny) piv = (piv < 0.0 ? -tiny : tiny);
      const double r = fast_rcp(piv);
      const double f = (noswap ? sub : ai) * r;
      double an, bn;
      if (noswap) {
        V(b, i) = bi;
        V(c2, i) = 0.0;
        V(fl, i) = 0.0;
        an = fma(-f, bi, dn);
        bn = en;
      } else {
        V(b, i) = dn;
        V(c2, i) = en;
        V(fl, i) = 1.0;
        an = fma(-f, dn, bi);
        bn = -f * en;
      }
      V(l, i) = f;
      V(a, i) = r;
      ai = an;
      bi = bn;
    }
    V(a, m - 1) = fast_rcp((fabs(ai) < tiny) ? (ai < 0.0 ? -tiny : tiny) : ai);
    for (int i = 0; i < m; ++i) V(x, i) = unit_rand(kk, i);
    // two solves reach the backward error for an isolated eigenvalue; a
    // cluster member, orthogonalised against the earlier ones, gets three
    const int nit = (kk == k) ? 2 : 3;
    for (int it = 0; it < nit; ++it) {
      // x <- (T - lam I)^{-1} x
      {
        double xi = V(x, 0);
        for (int i = 0; i < m - 1; ++i) {
          const double xn = V(x, i + 1), li = V(l, i);
          if (V(fl, i) != 0.0) {
            V(x, i) = xn;
            xi = fma(-li, xn, xi);
          } else {
            V(x, i) = xi;
            xi = fma(-li, xi, xn);
          }
        }
        V(x, m - 1) = xi;
      }
      double xn1 = V(x, m - 1) * V(a, m - 1), xn2 = 0.0;
      V(x, m - 1) = xn1;
      if (m > 1) {
        xn2 = (V(x, m - 2) - V(b, m - 2) * xn1) * V(a, m - 2);
        V(x, m - 2) = xn2;
      }
      for (int i = m - 3; i >= 0; --i) {
        const double xi = (V(x, i) - V(b, i) * xn2 - V(c2, i) * xn1) * V(a, i);
        V(x, i) = xi;
        xn1 = xn2;
        xn2 = xi;
      }
      // orthogonalise against the cluster's earlier vectors, normalise
      for (int jj = k; jj < kk; ++jj) {
        const double *y = Z + (size_t)jj * m;
        double s = 0.0;
        for (int i = 0; i < m; ++i) s = fma(y[i], V(x, i), s);
        for (int i = 0; i < m; ++i) V(x, i) = fma(-s, y[i], V(x, i));
      }
      // normalise: scale by a power of two near 1 / max|x| (exact), then by
      // 1 / ||x||
      int emx = 0;
      for (int i = 0; i < m; ++i) emx = max(emx, expb(V(x, i)));
      const double p2 = __longlong_as_double((long long)(2046 - min(emx, 2045)) << 52);
      double nn = 0.0;
      for (int i = 0; i < m; ++i) {
        const double xi = V(x, i) * p2;
        V(x, i) = xi;
        nn = fma(xi, xi, nn);
      }
      const double r = fast_rsqrt(nn);
      for (int i = 0; i < m; ++i) V(x, i) *= r;
    }
    for (int i = 0; i < m; ++i) Z[(size_t)kk * m + i] = V(x, i);
  }
#undef V
}

// ------------------------------------------------------ back-transform --
// U = Q D Z, Q = H_0 H_1 ... H_{m-2}: every CTA takes OCOLS columns of D Z
// into shared memory and applies H_{m-2}, ..., H_0 to them.  Few columns per
// CTA spread the FP64 work over many SMs; the next reflector is read into
// registers while the current one is applied.
constexpr int OCOLS = 2;
constexpr int OR_THREADS = 128;
constexpr int OR_PER = 8;  // reflector entries a thread prefetches (m <= OR_THREADS * OR_PER)

template <class T>
__global__ void __launch_bounds__(OR_THREADS)
    ormtr_kernel(int m, const T *__restrict__ Vr, const double *__restrict__ tau, const T *__restrict__ delta,
                 const double *__restrict__ Z, T *__restrict__ U) {
  using X = tr<T>;
  extern __shared__ __align__(16) unsigned char smem[];
  T *Y = reinterpret_cast<T *>(smem);  // [OCOLS][m]
  T *v = Y + (size_t)OCOLS * m;        // [m]
  __shared__ T dots[OCOLS];
  const int c0 = blockIdx.x * OCOLS;
  const int nc = min(OCOLS, m - c0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int t = tid; t < nc * m; t += blockDim.x) {
    const int c = t / m, i = t % m;
    Y[(long)c * m + i] = scl(delta[i], Z[i + (long)(c0 + c) * m]);
  }
  T pre[OR_PER];
  auto fetch = [&](int j) {
#pragma unroll
    for (int u = 0; u < OR_PER; ++u) {
      const int i = j + 1 + tid + u * OR_THREADS;
      pre[u] = (j >= 0 && i < m) ? Vr[i + (long)j * m] : X::zero();
    }
  };
  fetch(m - 2);
  for (int j = m - 2; j >= 0; --j) {
    const double tj = tau[j];
    __syncthreads();  // previous update done with v
#pragma unroll
    for (int u = 0; u < OR_PER; ++u) {
      const int i = j + 1 + tid + u * OR_THREADS;
      if (i < m) v[i] = pre[u];
    }
    __syncthreads();
    fetch(j - 1);  // in flight while this reflector is applied
    if (tj == 0.0) continue;  // uniform over the CTA
    if (warp < nc) {
      const T *y = Y + (long)warp * m;
      T s = X::zero();
      for (int i = j + 1 + lane; i < m; i += 32) s = X::fma(X::conj(v[i]), y[i], s);
      s = warp_sum(s);
      if (lane == 0) dots[warp] = scl(s, tj);
    }
    __syncthreads();
    const int w = m - j - 1;
    for (int t = tid; t < nc * w; t += blockDim.x) {
      const int c = t / w, i = j + 1 + t % w;
      Y[(long)c * m + i] = X::sub(Y[(long)c * m + i], X::mul(v[i], dots[c]));
    }
  }
  __syncthreads();
  for (int t = tid; t < nc * m; t += blockDim.x) {
    const int c = t / m, i = t % m;
    U[i + (long)(c0 + c) * m] = Y[(long)c * m + i];
  }
}

// ------------------------------------------------------------- Cholesky --
// A = L L^H (lower), right-looking; rows dealt cyclically to the cluster's
// CTAs as above.  Column j of L is conj(row j) / sqrt(a_jj) right of the
// diagonal, so the owner of row j forms and publishes the whole column (and
// writes it to Lout); after one cluster barrier every CTA updates its rows
// whole, A[i][k] -= l_i conj(l_k) for k > j (the row of the next pivot is
// then complete in its owner).  fail: first column whose pivot is not
// positive, + 1.  One cluster barrier per column.
template <class T>
__global__ void __launch_bounds__(TRD_THREADS, 1)
    chol_cluster_kernel(int m, const T *__restrict__ A, T *__restrict__ Lout, int *fail) {
  using X = tr<T>;
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks(), q = (int)cl.block_rank();
  const int rl = (m + C - 1) / C;
  extern __shared__ __align__(16) unsigned char smem[];
  T *L = reinterpret_cast<T *>(smem);  // [rl][m]
  T *lcol = L + (size_t)rl * m;        // [2][m] column j of L, written here by the owner of row j
  __shared__ int s_fail[2];            // the owner's pivot test, written here with the column
  __shared__ double s_r, s_ir;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (long t = tid; t < (long)rl * m; t += blockDim.x) {
    const int k = (int)(t / rl), il = (int)(t % rl);
    const int i = il * C + q;
    L[(long)il * m + k] = (i < m) ? A[i + (long)k * m] : X::zero();
  }
  __syncthreads();
  for (int j = 0; j < m; ++j) {
    const int own = j % C, par = j & 1;
    T *lc = lcol + (size_t)par * m;
    if (q == own) {
      // the owner forms column j from its row j (Hermitian: column j below
      // the diagonal is the conjugate of row j right of it) and writes it,
      // with the pivot test, into every CTA's buffer of this parity
      const T *Lj = L + (long)(j / C) * m;
      if (tid == 0) {  // the pivot's root and reciprocal, once
        const double piv = X::re(Lj[j]);
        const bool okp = piv > 0.0;
        const int f = okp ? 0 : j + 1;
        const double ir = okp ? fast_rsqrt(piv) : 0.0;  // one reciprocal square root
        s_r = piv * ir;
        s_ir = ir;
        for (int d = 0; d < C; ++d) cl.map_shared_rank(s_fail, d)[par] = f;
      }
      __syncthreads();
      const double r = s_r, ir = s_ir;
      for (int k = j + tid; k < m; k += blockDim.x) {
        const T l = (k == j) ? cvt<T, double>(r) : scl(X::conj(Lj[k]), ir);
        for (int d = 0; d < C; ++d) cl.map_shared_rank(lc, d)[k] = l;
      }
      for (int k = tid; k < m; k += blockDim.x) {
        T l = X::zero();
        if (k == j)
          l = cvt<T, double>(r);
        else if (k > j)
          l = scl(X::conj(Lj[k]), ir);
        Lout[k + (long)j * m] = l;
      }
    }
    cl.sync();  // column j of L (or the failure) in every CTA
    const int f = s_fail[par];
    if (f) {  // uniform: every CTA holds the owner's flag
      if (tid == 0 && q == 0) *fail = f;
      break;
    }
    for (int il = warp; il < rl; il += nw) {
      const int i = il * C + q;
      if (i <= j || i >= m) continue;
      T *Li = L + (long)il * m;
      const T li = X::neg(lc[i]);
      for (int k = j + 1 + lane; k < m; k += 32) Li[k] = X::fma(li, X::conj(lc[k]), Li[k]);
    }
    __syncthreads();
  }
  cl.sync();
}

// ------------------------------------------------------------ launchers --
// Cluster size and per-CTA shared memory for an m x m matrix of T with
// `extra` more vectors of T per CTA: the smallest power-of-two cluster
// (>= 2, <= 16) whose slices fit, preferring ~20 rows per CTA.
template <class T> static int cluster_shape(int m, int extra_rows, int extra_vecs, size_t *smem) {
  int C = 2;
  while (C < 16 && (m + C - 1) / C > 20) C *= 2;
  for (; C <= 16; C *= 2) {
    const int rl = (m + C - 1) / C;
    const size_t b = ((size_t)rl * m + (size_t)extra_rows * rl + (size_t)extra_vecs * m) * sizeof(T) + 64;
    if (b <= (size_t)TRD_SMEM_CAP) {
      *smem = b;
      return C;
    }
  }
  return 0;
}

// Launches kern as one cluster of C CTAs; returns 1 (nothing launched) when
// the cluster cannot be scheduled, so the caller can fall back.
template <class K, class... Args>
static int launch_cluster(K kern, int C, size_t smem, cudaStream_t st, Args... args) {
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, TRD_SMEM_CAP) != cudaSuccess ||
      cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C, 1, 1);
  cfg.blockDim = dim3(TRD_THREADS, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const cudaError_t err = cudaLaunchKernelEx(&cfg, kern, args...);
  if (err != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  GBF_LAUNCHED();
  return 0;
}

size_t heev_tridiag_work(int m, bool cplx) {
  const size_t ts = cplx ? sizeof(zd) : sizeof(double);
  const size_t mm = (size_t)m * m;
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t stein_b = (size_t)ceil_div(m, 32) * 6 * 32 * m * sizeof(double);
  return al(mm * ts) + 3 * al(m * ts) + 5 * al(m * sizeof(double)) + al(8 * sizeof(double)) +
         al(mm * sizeof(double)) + al(stein_b);
}

template <class T>
int heev_tridiag(cudaStream_t st, int m, const T *A, double *w, T *V, void *work, size_t work_bytes) {
  if (m < 2 || m > OR_THREADS * OR_PER) return 1;
  if (heev_tridiag_work(m, tr<T>::cplx) > work_bytes) return 1;
  size_t sm_t = 0;
  const int C = cluster_shape<T>(m, 0, 7, &sm_t);
  if (C == 0) return 1;
  const size_t mm = (size_t)m * m;
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  char *p = (char *)work;
  T *Vr = (T *)p;
  p += al(mm * sizeof(T));
  T *betac = (T *)p;
  p += al(m * sizeof(T));
  T *delta = (T *)p;
  p += al(m * sizeof(T));
  p += al(m * sizeof(T));
  double *tau = (double *)p;
  p += al(m * sizeof(double));
  double *dd = (double *)p;
  p += al(m * sizeof(double));
  double *e = (double *)p;
  p += al(m * sizeof(double));
  double *e2 = (double *)p;
  p += al(m * sizeof(double));
  p += al(m * sizeof(double));
  double *sc = (double *)p;
  p += al(8 * sizeof(double));
  double *Z = (double *)p;
  p += al(mm * sizeof(double));
  double *wk = (double *)p;
  const int slot = prof_begin(st);
  if (launch_cluster(sytrd_cluster_kernel<T>, C, sm_t, st, m, A, (long)m, Vr, tau, betac, dd)) return 1;
  tridiag_prep_kernel<T><<<1, PREP_THREADS, 0, st>>>(m, dd, betac, e, e2, delta, sc);
  GBF_LAUNCHED();
  stebz_kernel<<<ceil_div(m, STEBZ_WARPS), 32 * STEBZ_WARPS, 0, st>>>(m, dd, e2, sc, w);
  GBF_LAUNCHED();
  stein_kernel<<<ceil_div(m, 32), 32, 0, st>>>(m, dd, e, sc, w, Z, wk);
  GBF_LAUNCHED();
  const size_t sm_o = ((size_t)OCOLS * m + m) * sizeof(T);
  ormtr_kernel<T><<<ceil_div(m, OCOLS), OR_THREADS, sm_o, st>>>(m, Vr, tau, delta, Z, V);
  GBF_LAUNCHED();
  GBF_CUDA(cudaGetLastError());
  prof_end(st, slot, 0.0);
  return 0;
}

// Cholesky of the M0 x M0 Hermitian A (full storage, ld m, not modified):
// L (lower, ld m, strict upper part zero); *fail = first non-positive pivot
// column + 1.  Returns 1 when the cluster kernel cannot take m.
template <class T> int chol_cluster(cudaStream_t st, int m, const T *A, T *L, int *fail) {
  size_t sm = 0;
  const int C = cluster_shape<T>(m, 0, 2, &sm);
  if (C == 0) return 1;
  return launch_cluster(chol_cluster_kernel<T>, C, sm, st, m, A, L, fail);
}

#define TRD_INST(T)                                                                         \
  template int heev_tridiag<T>(cudaStream_t, int, const T *, double *, T *, void *, size_t); \
  template int chol_cluster<T>(cudaStream_t, int, const T *, T *, int *);
TRD_INST(double)
TRD_INST(zd)

}  // namespace gbf
