// Small dense FP64 kernels of the Rayleigh-Ritz step (M0 x M0 matrices),
// written as persistent cooperative kernels: one launch runs a whole
// factorisation / eigensolver over every SM, with grid-wide barriers
// (cooperative_groups grid sync, launched with cudaLaunchCooperativeKernel,
// which refuses a grid that cannot be co-resident) between dependent phases.
//
//   chol_coop    A = L L^H (lower), right-looking by columns; reports the
//                first non-positive pivot.
//   trinv_lower  Linv = L^{-1}, one warp per column (forward substitution with
//                warp-reduced dot products).
//   jacobi_coop  the parallel cyclic Jacobi of heev_jacobi (same rotations,
//                same circle-method rounds, same stopping rule) with all
//                sweeps in one launch.
#include <cooperative_groups.h>

#include <algorithm>
#include <mutex>

#include "gbf_common.cuh"

namespace cg = cooperative_groups;

namespace gbf {

__device__ inline double absS(double a) { return fabs(a); }
__device__ inline double absS(zd a) { return hypot(a.x, a.y); }
__device__ inline double scS(double a, double s) { return a * s; }
__device__ inline zd scS(zd a, double s) { return zd{a.x * s, a.y * s}; }

// At most one cooperative grid runs at a time in this process: two grids
// that each wait at a grid barrier for SMs the other holds could never
// finish.  The lock is held from launch to completion; ordinary kernels of
// other streams keep running beside it and always free their SMs.
static std::mutex g_coop_mu;

static int coop_run(const void *fn, int blocks, int threads, void **args, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_coop_mu);
  GBF_CUDA(cudaLaunchCooperativeKernel(fn, blocks, threads, args, 0, st));
  GBF_LAUNCHED();
  GBF_CUDA(cudaStreamSynchronize(st));
  return 0;
}

// Grid of a cooperative launch: sized from the problem alone (so results do
// not depend on what else runs), about 2 m^2 / 512 blocks (one block per
// SM at most), never more than can be co-resident.
static int coop_grid(const void *fn, int threads, size_t smem, int m) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, smem);
  if (per < 1) return 0;
  const long want = std::max(1L, (2L * m * m + 511) / 512);
  return (int)std::min<long>(want, sms);
}

// ------------------------------------------------------------- Cholesky --
// In: A (m x m, ld m, Hermitian, full storage).  Out: L (m x m, lower; the
// strict upper part is zeroed).  A is used as the working trailing matrix.
template <class T>
__global__ void chol_coop_kernel(int m, T *A, T *L, int *fail) {
  using X = tr<T>;
  cg::grid_group grid = cg::this_grid();
  const long nthr = (long)gridDim.x * blockDim.x;
  const long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  for (long t = tid; t < (long)m * m; t += nthr) {
    const int i = (int)(t % m), j = (int)(t / m);
    if (i < j) L[t] = X::zero();
  }
  for (int j = 0; j < m; ++j) {
    const double d = X::re(A[j + (long)j * m]);
    if (!(d > 0.0)) {
      if (tid == 0 && *fail == 0) *fail = j + 1;
      return;  // uniform: every thread reads the same d
    }
    const double ljj = sqrt(d), inv = 1.0 / ljj;
    // column j of L, and the trailing update from the unscaled column of A
    const int rest = m - j - 1;
    if (tid == 0) L[j + (long)j * m] = cvt<T, double>(ljj);
    for (long t = tid; t < (long)rest; t += nthr) {
      const int i = j + 1 + (int)t;
      L[i + (long)j * m] = scS(A[i + (long)j * m], inv);
    }
    const double inv2 = 1.0 / d;
    for (long t = tid; t < (long)rest * rest; t += nthr) {
      const int ii = (int)(t % rest), kk = (int)(t / rest);
      if (ii < kk) continue;  // lower triangle of the trailing block
      const int i = j + 1 + ii, k = j + 1 + kk;
      const T aij = A[i + (long)j * m], akj = A[k + (long)j * m];
      A[i + (long)k * m] = X::fma(scS(aij, -inv2), X::conj(akj), A[i + (long)k * m]);
    }
    grid.sync();
  }
}

// ------------------------------------------------- triangular inverse --
// Linv = L^{-1} for lower triangular L; warp w of the grid computes column j.
template <class T>
__global__ void trinv_lower_kernel(int m, const T *L, T *Linv) {
  using X = tr<T>;
  const int lane = threadIdx.x & 31;
  const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (j >= m) return;
  T *x = Linv + (long)j * m;
  for (int i = lane; i < m; i += 32) x[i] = X::zero();
  __syncwarp();
  for (int i = j; i < m; ++i) {
    // x_i = (delta_ij - sum_{k=j}^{i-1} L_ik x_k) / L_ii
    T s = X::zero();
    for (int k = j + lane; k < i; k += 32) s = X::fma(L[i + (long)k * m], x[k], s);
    for (int off = 16; off > 0; off >>= 1) {
      if constexpr (tr<T>::cplx) {
        s.x += __shfl_xor_sync(0xffffffffu, s.x, off);
        s.y += __shfl_xor_sync(0xffffffffu, s.y, off);
      } else {
        s += __shfl_xor_sync(0xffffffffu, s, off);
      }
    }
    if (lane == 0) {
      T rhs = (i == j) ? X::sub(X::one(), s) : X::neg(s);
      x[i] = X::mul(rhs, cvt<T, double>(1.0 / X::re(L[i + (long)i * m])));
    }
    __syncwarp();
  }
}

template <class T>
int chol_lower(cudaStream_t st, int m, T *A, T *L, int *fail) {
  const int threads = 512;
  const int blocks = coop_grid((const void *)chol_coop_kernel<T>, threads, 0, m);
  if (blocks < 1) {
    set_error("chol_coop: no co-resident grid");
    return -4;
  }
  void *args[] = {&m, &A, &L, &fail};
  return coop_run((const void *)chol_coop_kernel<T>, blocks, threads, args, st);
}

template <class T>
int trinv_lower(cudaStream_t st, int m, const T *L, T *Linv) {
  trinv_lower_kernel<T><<<ceil_div((long)m * 32, 256), 256, 0, st>>>(m, L, Linv);
  GBF_LAUNCHED();
  GBF_CUDA(cudaGetLastError());
  return 0;
}

// -------------------------------------------------------------- Jacobi --
constexpr double EPS_J = 2.220446049250313e-16;

__device__ inline int jpartner(int x, int P, int r) {
  if (x == P - 1) return r;
  if (x == r) return P - 1;
  int p = (2 * r - x) % (P - 1);
  return p < 0 ? p + P - 1 : p;
}

// Rotation of the pair (x, partner) from a = A[p][p], d = A[q][q],
// b = A[p][q] (p < q).  Out: c, beta (coefficient of the partner row), px
// (= x when not rotated) and the new diagonal entry of x.
template <class T>
__device__ void jrot_vals(int x, int p, int m, double a, double d, T b, double fro, double &c, T &beta, int &px,
                          double &nd) {
  using X = tr<T>;
  c = 1.0;
  beta = X::zero();
  px = x;
  const int pp = min(x, p);
  nd = (x == pp) ? a : d;
  if (p >= m || x >= m) return;
  const double ab = absS(b);
  if (ab == 0.0 || ab <= 0.5 * EPS_J * sqrt(fabs(a)) * sqrt(fabs(d)) || ab <= 1e-18 * fro) return;
  const T ph = scS(b, 1.0 / ab);
  const double tau = (d - a) / (2.0 * ab);
  const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
  c = 1.0 / sqrt(1.0 + t * t);
  const double s = t * c;
  px = p;
  if (x == pp) {
    beta = scS(ph, -s);
    nd = a - t * ab;
  } else {
    beta = scS(X::conj(ph), s);
    nd = d + t * ab;
  }
}

template <class T> struct JParams {
  double *cc, *nd;
  T *bb;
  int *pp;
};

// Entry (i, j) of J^H A J for the rotations in prm.
template <class T>
__device__ inline T jelem(int i, int j, int m, const T *A, const JParams<T> &prm) {
  using X = tr<T>;
  const double cj = prm.cc[j], ci = prm.cc[i];
  const T bj = prm.bb[j], bi = prm.bb[i];
  const int pj = prm.pp[j], pi = prm.pp[i];
  if (pi != i && pi == j) return X::zero();
  if (i == j && pi != i) return cvt<T, double>(prm.nd[i]);
  T out = scS(A[i + (long)j * m], ci * cj);
  if (pj != j) out = X::fma(scS(X::conj(bj), ci), A[i + (long)pj * m], out);
  if (pi != i) {
    out = X::fma(scS(bi, cj), A[pi + (long)j * m], out);
    if (pj != j) out = X::fma(X::mul(bi, X::conj(bj)), A[pi + (long)pj * m], out);
  }
  return out;
}

// A (in/out, the final diagonal holds the eigenvalues), V = eigenvectors.
// work: A2, V2 (m^2 each) + 2 x m (beta); dw: 2 x (c, nd) (4m) + fro;
// iw: 2 x m (partners) + per-sweep flags (maxsw) + sweeps.  Each round does
// one grid-wide phase: every thread updates its entries of A and V with the
// round's rotations, and thread s < P/2 also forms the three entries of
// pair s of the NEXT round and that pair's rotation (double-buffered
// parameters), so rounds need a single barrier.
template <class T>
__global__ void jacobi_coop_kernel(int m, int maxsw, T *A, T *V, T *work, double *dw, int *iw) {
  using X = tr<T>;
  cg::grid_group grid = cg::this_grid();
  const int P = m + (m & 1);
  const long nthr = (long)gridDim.x * blockDim.x;
  const long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long mm = (long)m * m;
  T *A2 = work, *V2 = work + mm;
  JParams<T> prm[2];
  for (int b = 0; b < 2; ++b) {
    prm[b].bb = work + 2 * mm + (long)b * m;
    prm[b].cc = dw + (long)b * 2 * m;
    prm[b].nd = dw + (long)b * 2 * m + m;
    prm[b].pp = iw + (long)b * m;
  }
  double *frop = dw + 4 * m;
  int *flags = iw + 2 * m, *sweeps_out = iw + 2 * m + maxsw;
  __shared__ double red[32];
  if (blockIdx.x == 0) {
    double s = 0.0;
    for (long t = threadIdx.x; t < mm; t += blockDim.x) {
      const double v = absS(A[t]);
      s += v * v;
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
      *frop = sqrt(tot);
    }
  }
  for (long t = tid; t < mm; t += nthr) V[t] = ((t % m) == (t / m)) ? X::one() : X::zero();
  for (long t = tid; t < maxsw; t += nthr) flags[t] = 0;
  grid.sync();
  const double fro = *frop;
  // rotations of round 0 from the input matrix
  for (long x = tid; x < m; x += nthr) {
    const int p = jpartner((int)x, P, 0);
    const int lo = min((int)x, p), hi = max((int)x, p);
    double a = 0.0, d = 0.0;
    T b = X::zero();
    if (p < m) {
      a = X::re(A[lo + (long)lo * m]);
      d = X::re(A[hi + (long)hi * m]);
      b = A[lo + (long)hi * m];
    } else {
      a = d = X::re(A[x + x * (long)m]);
    }
    double c, nd;
    T be;
    int px;
    jrot_vals<T>((int)x, p, m, a, d, b, fro, c, be, px, nd);
    prm[0].cc[x] = c;
    prm[0].bb[x] = be;
    prm[0].pp[x] = px;
    prm[0].nd[x] = nd;
  }
  grid.sync();
  T *Ac = A, *An = A2, *Vc = V, *Vn = V2;
  int cur = 0, done_sweeps = -1;
  for (int sw = 0; sw < maxsw; ++sw) {
    for (int r = 0; r < P - 1; ++r) {
      const JParams<T> &pc = prm[cur];
      // next round's rotations, from this round's result
      const int rn = (r + 1 < P - 1) ? r + 1 : 0;
      // pairs of the next round are spread over blocks first (their FP64
      // divisions and square roots then run on different SMs' FP64 units)
      // (lane 0 of warp w of block b takes pair b + gridDim.x * w)
      const int sidx = (threadIdx.x & 31) ? -1 : (int)blockIdx.x + (int)gridDim.x * (int)(threadIdx.x >> 5);
      if (sidx >= 0 && sidx < P / 2) {
        const int s = sidx;
        int x, y;
        if (s == 0) {
          x = rn;
          y = P - 1;
        } else {
          x = (rn + s) % (P - 1);
          y = (rn - s + (P - 1)) % (P - 1);
        }
        const int lo = min(x, y), hi = max(x, y);
        JParams<T> &pn = prm[cur ^ 1];
        if (hi < m) {
          const double a = X::re(jelem<T>(lo, lo, m, Ac, pc));
          const double d = X::re(jelem<T>(hi, hi, m, Ac, pc));
          const T b = jelem<T>(lo, hi, m, Ac, pc);
          double c, nd;
          T be;
          int px;
          jrot_vals<T>(lo, hi, m, a, d, b, fro, c, be, px, nd);
          pn.cc[lo] = c;
          pn.bb[lo] = be;
          pn.pp[lo] = px;
          pn.nd[lo] = nd;
          jrot_vals<T>(hi, lo, m, a, d, b, fro, c, be, px, nd);
          pn.cc[hi] = c;
          pn.bb[hi] = be;
          pn.pp[hi] = px;
          pn.nd[hi] = nd;
        } else if (lo < m) {  // partner is the padding player: no rotation
          pn.cc[lo] = 1.0;
          pn.bb[lo] = X::zero();
          pn.pp[lo] = lo;
          pn.nd[lo] = 0.0;
        }
      }
      for (long t = tid; t < 2 * mm; t += nthr) {
        if (t < mm) {
          An[t] = jelem<T>((int)(t % m), (int)(t / m), m, Ac, pc);
        } else {
          const long u = t - mm;
          const int i = (int)(u % m), j = (int)(u / m);
          const int pj = pc.pp[j];
          T out = scS(Vc[u], pc.cc[j]);
          if (pj != j) out = X::fma(X::conj(pc.bb[j]), Vc[i + (long)pj * m], out);
          Vn[u] = out;
        }
      }
      grid.sync();
      T *t1 = Ac;
      Ac = An;
      An = t1;
      t1 = Vc;
      Vc = Vn;
      Vn = t1;
      cur ^= 1;
    }
    // convergence: any pair still above the rotation threshold?
    int viol = 0;
    for (long t = tid; t < mm; t += nthr) {
      const int i = (int)(t % m), j = (int)(t / m);
      if (i >= j) continue;
      const double b = absS(Ac[t]);
      const double a = fabs(X::re(Ac[i + (long)i * m])), d = fabs(X::re(Ac[j + (long)j * m]));
      if (b > 0.0 && b > 0.5 * EPS_J * sqrt(a) * sqrt(d) && b > 1e-18 * fro) viol = 1;
    }
    viol = __syncthreads_or(viol);
    if (viol && threadIdx.x == 0) atomicOr(&flags[sw], 1);
    grid.sync();
    if (atomicOr(&flags[sw], 0) == 0) {
      done_sweeps = sw;
      break;
    }
  }
  if (Ac != A) {
    for (long t = tid; t < mm; t += nthr) {
      A[t] = Ac[t];
      V[t] = Vc[t];
    }
  }
  if (tid == 0) *sweeps_out = done_sweeps;
}

template <class T>
int jacobi_coop(cudaStream_t st, int m, int maxsw, T *A, T *V, T *work, double *dw, int *iw) {
  const int threads = 512;
  const int blocks = coop_grid((const void *)jacobi_coop_kernel<T>, threads, 0, m);
  if (blocks < 1) {
    set_error("jacobi_coop: no co-resident grid");
    return -4;
  }
  void *args[] = {&m, &maxsw, &A, &V, &work, &dw, &iw};
  return coop_run((const void *)jacobi_coop_kernel<T>, blocks, threads, args, st);
}

#define SMALL_INST(T)                                                                          \
  template int chol_lower<T>(cudaStream_t, int, T *, T *, int *);                             \
  template int trinv_lower<T>(cudaStream_t, int, const T *, T *);                             \
  template int jacobi_coop<T>(cudaStream_t, int, int, T *, T *, T *, double *, int *);
SMALL_INST(double)
SMALL_INST(zd)

}  // namespace gbf
