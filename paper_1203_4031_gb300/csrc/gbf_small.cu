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
// rd: the reciprocals of L's (real, positive) diagonal, formed once by
// recip_diag_kernel (FP64 divisions are costly; every column needs them).
template <class T>
__global__ void recip_diag_kernel(int m, const T *L, double *rd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) rd[i] = 1.0 / tr<T>::re(L[i + (long)i * m]);
}
// Column j of L^{-1} by one warp, in the column-oriented (axpy) form of the
// forward substitution: the running sums acc_i = sum_{k<i} L_ik x_k sit in
// shared memory; at step k the warp forms x_k = (delta_kj - acc_k) / L_kk
// and adds L_ik x_k into acc_i for every i > k, the lanes on consecutive
// rows (coalesced column of L).  One dependent step per row and no
// reduction across lanes.
template <class T>
__global__ void __launch_bounds__(256) trinv_lower_kernel(int m, const T *L, const double *rd, T *Linv) {
  using X = tr<T>;
  extern __shared__ __align__(16) unsigned char tsm_raw[];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int j = blockIdx.x * (blockDim.x >> 5) + wl;
  if (j >= m) return;  // warp-uniform; no block-wide barrier below
  T *acc = reinterpret_cast<T *>(tsm_raw) + (long)wl * m;
  for (int i = j + lane; i < m; i += 32) acc[i] = X::zero();
  __syncwarp();
  for (int k = j; k < m; ++k) {
    const T a = acc[k];
    const T xk = X::mul((k == j) ? X::sub(X::one(), a) : X::neg(a), cvt<T, double>(rd[k]));
    __syncwarp();
    const T *Lk = L + (long)k * m;
    for (int i = k + 1 + lane; i < m; i += 32) acc[i] = X::fma(Lk[i], xk, acc[i]);
    if (lane == 0) acc[k] = xk;
    __syncwarp();
  }
  T *x = Linv + (long)j * m;
  for (int i = lane; i < m; i += 32) x[i] = (i < j) ? X::zero() : acc[i];
}

template <class T>
int chol_lower(cudaStream_t st, int m, T *A, T *L, int *fail) {
  // one thread-block cluster (hardware barriers) when the matrix fits in its
  // shared memory; the cooperative grid-wide form otherwise
  if (chol_cluster<T>(st, m, A, L, fail) == 0) return 0;
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
int trinv_lower(cudaStream_t st, int m, const T *L, T *Linv, double *rd) {
  recip_diag_kernel<T><<<ceil_div(m, 256), 256, 0, st>>>(m, L, rd);
  GBF_LAUNCHED();
  // warps per block: as many columns' running sums as fit 48 KB of shared
  // memory (one column up to 200 KB)
  if ((size_t)m * sizeof(T) > 200 * 1024) {
    set_error("triangular inverse: m too large (%d)", m);
    return -4;
  }
  static std::atomic<unsigned long long> attr_done{0};
  if (int rc = once_per_device(attr_done, [&]() -> int {
        GBF_CUDA(cudaFuncSetAttribute(trinv_lower_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        return 0;
      }))
    return rc;
  const int wpb = (int)std::max<size_t>(1, std::min<size_t>(8, (48 * 1024) / ((size_t)m * sizeof(T))));
  trinv_lower_kernel<T><<<ceil_div(m, wpb), 32 * wpb, (size_t)wpb * m * sizeof(T), st>>>(m, L, rd, Linv);
  GBF_LAUNCHED();
  GBF_CUDA(cudaGetLastError());
  return 0;
}

// -------------------------------------------------------------- Jacobi --
constexpr double EPS_J = 2.220446049250313e-16;

template <class T> struct JParams {
  double *cc, *nd;
  T *bb;
  int *pp;
};

// Rotation of the pair lo < hi from a = A[lo][lo], d = A[hi][hi], b =
// A[lo][hi], written for both members: c (same for both), beta (coefficient
// of the partner column), partner (= self when not rotated) and the new
// diagonal entry.  Rotation angle from tau = (d - a) / (2|b|): t = sign(tau)
// / (|tau| + sqrt(1 + tau^2)), c = 1 / sqrt(1 + t^2), s = t c; no rotation
// when |b| is at rounding level of sqrt(|a d|) or of the Frobenius norm.
// The expensive operations are few: |b|^-1 by one reciprocal square root,
// the threshold tests on squares, t by one square root and one division, c
// by one reciprocal square root.
template <class T>
__device__ void jrot_pair(int lo, int hi, int m, double a, double d, T b, double fro, JParams<T> &pn) {
  using X = tr<T>;
  double c = 1.0;
  T blo = X::zero(), bhi = X::zero();
  int plo = lo, phi = hi;
  double ndlo = a, ndhi = d;
  const double b2 = X::re(X::mul(b, X::conj(b)));  // |b|^2
  if (hi < m && b2 > 0.0 && b2 > 0.25 * EPS_J * EPS_J * fabs(a) * fabs(d) && b2 > 1e-36 * fro * fro) {
    const double iab = rsqrt(b2);  // 1 / |b|
    const double ab = b2 * iab;
    const T ph = scS(b, iab);
    const double tau = 0.5 * (d - a) * iab;
    const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
    c = rsqrt(1.0 + t * t);
    const double sn = t * c;
    blo = scS(ph, -sn);
    bhi = scS(X::conj(ph), sn);
    plo = hi;
    phi = lo;
    ndlo = a - t * ab;
    ndhi = d + t * ab;
  }
  pn.cc[lo] = c;
  pn.bb[lo] = blo;
  pn.pp[lo] = plo;
  pn.nd[lo] = ndlo;
  if (hi < m) {
    pn.cc[hi] = c;
    pn.bb[hi] = bhi;
    pn.pp[hi] = phi;
    pn.nd[hi] = ndhi;
  }
}



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
__global__ void __launch_bounds__(512, 1) jacobi_coop_kernel(int m, int maxsw, T *A, T *V, T *work, double *dw, int *iw) {
  using X = tr<T>;
  cg::grid_group grid = cg::this_grid();
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
  // active indices (deflation): flag per index, sorted list, count; after
  // iw[2m + maxsw + 8 .. + m) (the caller's ranking space)
  int *act_flag = iw + 3 * m + maxsw + 8, *act = act_flag + m, *nact = act + m;
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
      *nact = m;
    }
  }
  for (long t = tid; t < mm; t += nthr) V[t] = ((t % m) == (t / m)) ? X::one() : X::zero();
  for (long t = tid; t < maxsw; t += nthr) flags[t] = 0;
  for (long t = tid; t < m; t += nthr) {
    act[t] = (int)t;
    act_flag[t] = 0;
  }
  grid.sync();
  const double fro = *frop;
  T *Ac = A, *An = A2, *Vc = V, *Vn = V2;
  int cur = 0, done_sweeps = -1;
  const int lane = threadIdx.x & 31;
  // the matrix index of player x of a round over Pa players (Pa - 1 is the
  // padding player when the active count is odd)
  auto player = [&](int x, int ma) { return x < ma ? act[x] : m; };
  for (int sw = 0; sw < maxsw; ++sw) {
    // Each sweep pairs only the active indices: those with an off-diagonal
    // entry above the rotation threshold after the previous sweep (all in
    // sweep 0).  An index outside the set keeps the identity rotation; its
    // entries with active indices are at rounding level and stay there.
    const int ma = *nact;
    const int Pa = ma + (ma & 1);
    // warps per block that form rotations (one pair each), the rest update
    const int npw = min((Pa / 2 + (int)gridDim.x - 1) / (int)gridDim.x, (int)(blockDim.x >> 5) - 1);
    const long wid = (long)blockIdx.x * (blockDim.x - 32 * npw) + (long)threadIdx.x - 32 * npw;
    const long nw = (long)gridDim.x * (blockDim.x - 32 * npw);
    // identity rotations everywhere, then the active pairs of round 0
    for (long t = tid; t < m; t += nthr)
      for (int b = 0; b < 2; ++b) {
        prm[b].cc[t] = 1.0;
        prm[b].bb[t] = X::zero();
        prm[b].pp[t] = (int)t;
        prm[b].nd[t] = 0.0;
      }
    grid.sync();
    for (long s = tid; s < Pa / 2; s += nthr) {
      const int x = (s == 0) ? 0 : (int)s;
      const int y = (s == 0) ? Pa - 1 : (int)((Pa - 1 - s) % (Pa - 1));
      const int ix = player(x, ma), iy = player(y, ma);
      const int lo = min(ix, iy), hi = max(ix, iy);
      if (hi < m)
        jrot_pair<T>(lo, hi, m, X::re(Ac[lo + (long)lo * m]), X::re(Ac[hi + (long)hi * m]), Ac[lo + (long)hi * m],
                     fro, prm[cur]);
    }
    grid.sync();
    for (int r = 0; r < Pa - 1; ++r) {
      const JParams<T> &pc = prm[cur];
      JParams<T> &pn = prm[cur ^ 1];
      // pairs of the next round (none after the last round of the sweep)
      // are spread over blocks (their FP64 square roots and divisions then
      // run on different SMs' FP64 units): warp w < npw of block b takes
      // pair b + gridDim.x * w; lanes 0, 1, 2 read the pair's entries a, d,
      // b of this round's result, lane 0 forms the rotation
      const int rn = r + 1;
      const int sidx = (int)blockIdx.x + (int)gridDim.x * (int)(threadIdx.x >> 5);
      for (int s = sidx; rn < Pa - 1 && (int)(threadIdx.x >> 5) < npw && lane < 3 && s < Pa / 2;
           s += (int)gridDim.x * npw) {
        int x, y;
        if (s == 0) {
          x = rn;
          y = Pa - 1;
        } else {
          x = (rn + s) % (Pa - 1);
          y = (rn - s + (Pa - 1)) % (Pa - 1);
        }
        const int ix = player(x, ma), iy = player(y, ma);
        const int lo = min(ix, iy), hi = max(ix, iy);
        T v = X::zero();
        if (hi < m) v = jelem<T>(lane == 1 ? hi : lo, lane == 0 ? lo : hi, m, Ac, pc);
        const unsigned msk = 0x7u;
        T vd, vb;
        if constexpr (tr<T>::cplx) {
          vd.x = __shfl_sync(msk, v.x, 1);
          vd.y = __shfl_sync(msk, v.y, 1);
          vb.x = __shfl_sync(msk, v.x, 2);
          vb.y = __shfl_sync(msk, v.y, 2);
        } else {
          vd = __shfl_sync(msk, v, 1);
          vb = __shfl_sync(msk, v, 2);
        }
        if (lane == 0 && hi < m) jrot_pair<T>(lo, hi, m, X::re(v), X::re(vd), vb, fro, pn);
        if (lane == 0 && hi >= m && lo < m) {  // the padding player's partner: identity
          pn.cc[lo] = 1.0;
          pn.bb[lo] = X::zero();
          pn.pp[lo] = lo;
        }
      }
      // entries of this round: warps npw.. of every block (warps below npw
      // form the next round's rotations meanwhile)
      for (long t = ((int)threadIdx.x >= 32 * npw) ? wid : 2 * mm; t < 2 * mm; t += nw) {
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
    // convergence: pairs still above the rotation threshold; their indices
    // form the next sweep's active set
    int viol = 0;
    for (long t = tid; t < mm; t += nthr) {
      const int i = (int)(t % m), j = (int)(t / m);
      if (i >= j) continue;
      const double b = absS(Ac[t]);
      const double a = fabs(X::re(Ac[i + (long)i * m])), d = fabs(X::re(Ac[j + (long)j * m]));
      if (b > 0.0 && b * b > 0.25 * EPS_J * EPS_J * a * d && b > 1e-18 * fro) {
        viol = 1;
        act_flag[i] = 1;
        act_flag[j] = 1;
      }
    }
    viol = __syncthreads_or(viol);
    if (viol && threadIdx.x == 0) atomicOr(&flags[sw], 1);
    grid.sync();
    if (atomicOr(&flags[sw], 0) == 0) {
      done_sweeps = sw;
      break;
    }
    // the sorted active list (one block), flags cleared for the next sweep
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      int c = 0;
      for (int i = 0; i < m; ++i)
        if (act_flag[i]) {
          act[c++] = i;
          act_flag[i] = 0;
        }
      *nact = c;
    }
    grid.sync();
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
  template int trinv_lower<T>(cudaStream_t, int, const T *, T *, double *);                   \
  template int jacobi_coop<T>(cudaStream_t, int, int, T *, T *, T *, double *, int *);
SMALL_INST(double)
SMALL_INST(zd)

}  // namespace gbf
