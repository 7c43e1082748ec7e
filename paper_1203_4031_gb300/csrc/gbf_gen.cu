// Non-Hermitian FEAST (guide section "From v2.1 to v3.0": dual subspaces Q
// and Q^ for the right and left eigenvectors, a full contour around complex
// eigenvalues; RCI cases 11/21 and 30/31/40/41 of Table tab_ijob): the node
// sums of the two subspaces, the reduced non-Hermitian eigensolver of the
// Rayleigh-Ritz step, and the residuals, ordering and bi-orthonormality
// check of Tables tab_common and tab_info.
//
// Reduced eigensolver.  After G = Bq^{-1} Aq (LU of Bq on the batched LU
// engine), G = Z T Z^H by
//   hessenberg   Householder reduction to upper Hessenberg form, reflectors
//                accumulated into Z (one CTA),
//   hqr          complex single-shift QR sweeps with the Wilkinson shift of
//                the trailing 2 x 2 block (an exceptional shift every tenth
//                sweep), small subdiagonals deflated, rotations applied to
//                the whole of T (Schur form) and accumulated into Z (one CTA;
//                all threads run the same control flow on the same values),
//   trevc        eigenvectors of the triangular T by back substitution, one
//                warp per eigenvector, column-oriented (a running sum per
//                row in registers, no reduction per row),
// then W = Z Y on the sliced tensor-core GEMM.  These M0-sized kernels are
// latency- and FP64-bound on one SM; their cost grows as M0^3.
#include "gbf_common.cuh"

#include <cfloat>

namespace gbf {
namespace {
using X = tr<zd>;

__device__ __forceinline__ double cabs1(zd a) { return fabs(a.x) + fabs(a.y); }
__device__ __forceinline__ zd zsc(zd a, double s) { return zd{a.x * s, a.y * s}; }
__device__ __forceinline__ double absq(zd a) { return a.x * a.x + a.y * a.y; }

// principal square root of a complex number
__device__ zd zsqrt(zd z) {
  const double r = hypot(z.x, z.y);
  if (r == 0.0) return zd{0.0, 0.0};
  if (z.x >= 0.0) {
    const double t = sqrt(0.5 * (r + z.x));
    return zd{t, z.y / (2.0 * t)};
  }
  const double t = sqrt(0.5 * (r - z.x));
  return zd{fabs(z.y) / (2.0 * t), copysign(t, z.y)};
}

// Deterministic block sum / max (fixed tree over blockDim.x = 256).
constexpr int RT = 256;
__device__ double block_sum(double v, double *red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int s = RT / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}
__device__ double block_max(double v, double *red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int s = RT / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

// ------------------------------------------------------------ elementwise --
__global__ void widen_ld_kernel(int n, const double *A, long lda, zd *Af) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i < n) Af[i + (long)j * n] = zd{A[i + (long)j * lda], 0.0};
}

// dst = [src, conj(src)] (n x 2m): the right-hand sides of a node and of its
// mirror image, whose system is the conjugate of this one for real A, B
__global__ void conj_pair_kernel(int n, int m, const zd *src, zd *dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= n) return;
  const zd v = src[i + (long)j * n];
  dst[i + (long)j * n] = v;
  dst[i + (long)(m + j) * n] = X::conj(v);
}

// Q[i, j] = X0[i, j] g_j + sum_e c_e Y_e[i, j] (+ conj(c_e Y_e[i, m + j])
// for the mirror node when `half`), c_e = w_e (right) or conj(w_e) (left),
// g = f or conj(f) (the residual-correction form; X0 may be null); nodes in
// order.
template <class TY>
__global__ void accum_gen_kernel(int n, int m, int nf, const zd *w, const TY *Y, int mw, int half, int left,
                                 const zd *X0, const zd *f, zd *Q) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= n) return;
  const long ny = (long)n * mw;
  zd acc{0.0, 0.0};
  if (X0) acc = X::mul(X0[i + (long)j * n], left ? X::conj(f[j]) : f[j]);
  for (int e = 0; e < nf; ++e) {
    const zd ce = left ? X::conj(w[e]) : w[e];
    const TY *Ye = Y + e * ny;
    acc = X::fma(ce, cvt<zd, TY>(Ye[i + (long)j * n]), acc);
    if (half) acc = X::add(acc, X::conj(X::mul(ce, cvt<zd, TY>(Ye[i + (long)(m + j) * n]))));
  }
  Q[i + (long)j * n] = acc;
}

// Per-node column scales of the residual-correction right-hand sides: right
// (left = 0) D_e[j] = 1/(z_e - lam_j), left conj(D_e[j]); with `half`, the
// mirror node's column m + j holds conj(D_{e'}[j]) (right) or D_e'-conj form
// (left), z_{e'} = conj(z_e): 1/(z_e - conj(lam_j)) and 1/(conj(z_e) -
// lam_j).  Also f_j = sum over all ne nodes of w_e / (z_e - lam_j).
__global__ void gen_scales_kernel(int m, int nf, int ne, const zd *z, const zd *w, const zd *lam, int half,
                                  zd *SCr, zd *SCl, zd *f) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  const zd l = lam[j], lc = X::conj(l);
  const int mw = half ? 2 * m : m;
  for (int e = 0; e < nf; ++e) {
    const zd de = zdiv(zd{1.0, 0.0}, X::sub(z[e], l));
    SCr[(long)e * mw + j] = de;
    SCl[(long)e * mw + j] = X::conj(de);
    if (half) {
      SCr[(long)e * mw + m + j] = zdiv(zd{1.0, 0.0}, X::sub(z[e], lc));
      SCl[(long)e * mw + m + j] = zdiv(zd{1.0, 0.0}, X::sub(X::conj(z[e]), l));
    }
  }
  zd s{0.0, 0.0};
  for (int e = 0; e < ne; ++e) s = X::add(s, zdiv(w[e], X::sub(z[e], l)));
  f[j] = s;
}

// R[:, j] = MX[:, j] - lt_j NX[:, j] * s_j, lt = lam or conj(lam), s_j = 1 or
// 1/sc_j (sc null: 1): the eigen-residual of the Ritz pairs, the
// right-hand side of the residual-correction form
__global__ void gen_eig_residual_kernel(int n, const zd *MX, const zd *NX, const zd *lam, int conjl, const double *sc,
                                        zd *R) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= n) return;
  const zd l = conjl ? X::conj(lam[j]) : lam[j];
  const double s = sc ? 1.0 / sc[j] : 1.0;
  const long o = i + (long)j * n;
  R[o] = zsc(X::sub(MX[o], X::mul(l, NX[o])), s);
}

__global__ void __launch_bounds__(RT) col_norms_kernel(int n, const zd *Xm, double *nrm) {
  __shared__ double red[RT];
  const int j = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += RT) s += absq(Xm[i + (long)j * n]);
  s = block_sum(s, red);
  if (threadIdx.x == 0) nrm[j] = sqrt(s);
}

// dst[:, j] = src[:, j] * s_j (or / s_j); dst may alias src
__global__ void col_scale_kernel(int n, const zd *src, zd *dst, const double *s, int divide) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= n) return;
  const double f = divide ? 1.0 / s[j] : s[j];
  dst[i + (long)j * n] = zsc(src[i + (long)j * n], f);
}

// res_j = ||MX_j - l_j NX_j||_1 / ||alpha NX_j||_1, l_j = lam_j or conj(lam_j)
__global__ void __launch_bounds__(RT) gen_residual_kernel(int n, const zd *MX, const zd *NX, const zd *lam,
                                                           int conjl, double alpha, double *res) {
  __shared__ double red[RT];
  const int j = blockIdx.x;
  const zd l = conjl ? X::conj(lam[j]) : lam[j];
  double num = 0.0, den = 0.0;
  for (int i = threadIdx.x; i < n; i += RT) {
    const zd b = NX[i + (long)j * n];
    const zd d = X::sub(MX[i + (long)j * n], X::mul(l, b));
    num += hypot(d.x, d.y);
    den += hypot(b.x, b.y);
  }
  num = block_sum(num, red);
  den = block_sum(den, red);
  if (threadIdx.x == 0) res[j] = num / (alpha * den);
}

// Order: pairs inside the contour first, each group by ascending (Re, Im)
// (then index); pos[j] = output slot of pair j, src[slot] = j; outputs in
// that order; stats = {nin, Re trace, Im trace, max over inside of
// max(right, left residual), all finite}.
__global__ void order_gen_kernel(int m, const zd *lam, const double *rr, const double *rl, double er, double ei,
                                 double r, double rho, double cph, double sph, int *pos, int *src, zd *Eo,
                                 double *Rr, double *Rl, double *stats) {
  __shared__ int s_in[1024];
  const int j = threadIdx.x;
  if (j < m) {
    const double dx = lam[j].x - er, dy = lam[j].y - ei;
    const double ux = (dx * cph + dy * sph) / r, uy = (dy * cph - dx * sph) / r;
    s_in[j] = (ux * ux + (uy / rho) * (uy / rho) <= 1.0) ? 1 : 0;
  }
  __syncthreads();
  if (j < m) {
    const int ij = s_in[j];
    const zd lj = lam[j];
    int rank = 0;
    for (int k = 0; k < m; ++k) {
      if (k == j) continue;
      const int ik = s_in[k];
      const zd lk = lam[k];
      bool before;
      if (ik != ij) before = ik > ij;
      else if (lk.x != lj.x) before = lk.x < lj.x;
      else if (lk.y != lj.y) before = lk.y < lj.y;
      else before = k < j;
      rank += before ? 1 : 0;
    }
    pos[j] = rank;
    src[rank] = j;
    Eo[rank] = lj;
    Rr[rank] = rr[j];
    Rl[rank] = rl[j];
  }
  __syncthreads();
  if (j == 0) {
    int nin = 0;
    for (int k = 0; k < m; ++k) nin += s_in[k];
    double tx = 0.0, ty = 0.0, mx = 0.0;
    for (int k = 0; k < nin; ++k) {
      tx += Eo[k].x;
      ty += Eo[k].y;
      mx = fmax(mx, fmax(Rr[k], Rl[k]));
    }
    bool fin = true;
    for (int k = 0; k < m; ++k)
      fin = fin && isfinite(lam[k].x) && isfinite(lam[k].y) && isfinite(rr[k]) && isfinite(rl[k]);
    stats[0] = nin;
    stats[1] = tx;
    stats[2] = ty;
    stats[3] = mx;
    stats[4] = fin ? 1.0 : 0.0;
  }
}

// max over slots a, b < nin of |(nr_pa / nr_pb) P[pa, pb] - delta_ab| (pa =
// src[a]): the bi-orthonormality defect of the returned pairs, X^_a^H B X_b -
// delta_ab, from P = V^H Bq W and the rescaling x = Q W / nr, x^ = Q^ V nr
__global__ void __launch_bounds__(RT) biorth_kernel(int m, int nin, const zd *P, const double *nr, const int *src,
                                                     double *out) {
  __shared__ double red[RT];
  double mx = 0.0;
  for (long t = threadIdx.x; t < (long)nin * nin; t += RT) {
    const int a = (int)(t % nin), b = (int)(t / nin);
    const int pa = src[a], pb = src[b];
    zd v = zsc(P[pa + (long)pb * m], nr[pa] / nr[pb]);
    if (a == b) v.x -= 1.0;
    mx = fmax(mx, hypot(v.x, v.y));
  }
  mx = block_max(mx, red);
  if (threadIdx.x == 0) out[0] = mx;
}

__global__ void identity_kernel(int m, zd *I) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i < m) I[i + (long)j * m] = zd{i == j ? 1.0 : 0.0, 0.0};
}

// ------------------------------------------------------------ Hessenberg --
// G <- H_j G H_j for j = 0..m-3, H_j = I - tau v v^H (Hermitian, unitary)
// annihilating G[j+2.., j]; v_{j+1} = 1, v_i = x_i conj(ph) / (|x_{j+1}| +
// ||x||) with ph the phase of x_{j+1}, tau = 1 + |x_{j+1}| / ||x||, so that
// H_j x = -ph ||x|| e_{j+1}.  Z <- Z H_j from Z = I.  G and Z are worked on
// in shared memory when they fit (`in_smem`), else in place in global memory.
__global__ void __launch_bounds__(RT) hessenberg_kernel(int m, zd *Gg, zd *Zg, int in_smem) {
  extern __shared__ __align__(16) unsigned char smem[];
  zd *sv = reinterpret_cast<zd *>(smem);  // [m]
  zd *G = in_smem ? sv + m : Gg;
  zd *Z = in_smem ? sv + m + (size_t)m * m : Zg;
  __shared__ double red[RT];
  __shared__ double s_tau;
  __shared__ zd s_sc, s_beta;
  const int tid = threadIdx.x;
  const long mm = (long)m * m;
  for (long t = tid; t < mm; t += RT) {
    if (in_smem) G[t] = Gg[t];
    Z[t] = zd{(t % m) == (t / m) ? 1.0 : 0.0, 0.0};
  }
  __syncthreads();
  for (int j = 0; j + 2 < m; ++j) {
    double part = 0.0;
    for (int i = j + 2 + tid; i < m; i += RT) part += absq(G[i + (long)j * m]);
    const double rest = block_sum(part, red);
    if (tid == 0) {
      const zd x0 = G[j + 1 + (long)j * m];
      double tau = 0.0;
      zd sc{0.0, 0.0}, beta = x0;
      if (rest > 0.0) {
        const double a0 = hypot(x0.x, x0.y), nx = sqrt(a0 * a0 + rest);
        const zd ph = a0 > 0.0 ? zd{x0.x / a0, x0.y / a0} : zd{1.0, 0.0};
        beta = zsc(ph, -nx);
        sc = zsc(X::conj(ph), 1.0 / (a0 + nx));
        tau = 1.0 + a0 / nx;
      }
      s_tau = tau;
      s_sc = sc;
      s_beta = beta;
    }
    __syncthreads();
    const double tau = s_tau;
    if (tau == 0.0) continue;  // uniform: column already in Hessenberg form
    const zd sc = s_sc;
    for (int i = j + 1 + tid; i < m; i += RT) sv[i] = (i == j + 1) ? zd{1.0, 0.0} : X::mul(G[i + (long)j * m], sc);
    __syncthreads();
    // left: columns c > j; four lanes per column, each over every fourth
    // row, partial sums combined by two shuffles (a fixed order)
    for (int c0 = j + 1; c0 < m; c0 += RT / 4) {
      const int c = c0 + (tid >> 2), q = tid & 3;
      const bool act = c < m;
      zd *Gc = G + (long)c * m;
      zd sp{0.0, 0.0};
      if (act)
        for (int r = j + 1 + q; r < m; r += 4) sp = X::fma(X::conj(sv[r]), Gc[r], sp);
      sp.x += __shfl_xor_sync(0xffffffffu, sp.x, 1);
      sp.y += __shfl_xor_sync(0xffffffffu, sp.y, 1);
      sp.x += __shfl_xor_sync(0xffffffffu, sp.x, 2);
      sp.y += __shfl_xor_sync(0xffffffffu, sp.y, 2);
      sp = zsc(sp, tau);
      if (act)
        for (int r = j + 1 + q; r < m; r += 4) Gc[r] = X::sub(Gc[r], X::mul(sv[r], sp));
    }
    for (int r = j + 1 + tid; r < m; r += RT) G[r + (long)j * m] = (r == j + 1) ? s_beta : zd{0.0, 0.0};
    __syncthreads();
    // right: every row of G and Z, four lanes per row over every fourth column
    for (int i0 = 0; i0 < m; i0 += RT / 4) {
      const int i = i0 + (tid >> 2), q = tid & 3;
      const bool act = i < m;
      zd t{0.0, 0.0}, u{0.0, 0.0};
      if (act)
        for (int c = j + 1 + q; c < m; c += 4) {
          t = X::fma(G[i + (long)c * m], sv[c], t);
          u = X::fma(Z[i + (long)c * m], sv[c], u);
        }
      t.x += __shfl_xor_sync(0xffffffffu, t.x, 1);
      t.y += __shfl_xor_sync(0xffffffffu, t.y, 1);
      u.x += __shfl_xor_sync(0xffffffffu, u.x, 1);
      u.y += __shfl_xor_sync(0xffffffffu, u.y, 1);
      t.x += __shfl_xor_sync(0xffffffffu, t.x, 2);
      t.y += __shfl_xor_sync(0xffffffffu, t.y, 2);
      u.x += __shfl_xor_sync(0xffffffffu, u.x, 2);
      u.y += __shfl_xor_sync(0xffffffffu, u.y, 2);
      t = zsc(t, tau);
      u = zsc(u, tau);
      if (act)
        for (int c = j + 1 + q; c < m; c += 4) {
          const zd vc = X::conj(sv[c]);
          G[i + (long)c * m] = X::sub(G[i + (long)c * m], X::mul(t, vc));
          Z[i + (long)c * m] = X::sub(Z[i + (long)c * m], X::mul(u, vc));
        }
    }
    __syncthreads();
  }
  if (in_smem)
    for (long t = tid; t < mm; t += RT) {
      Gg[t] = G[t];
      Zg[t] = Z[t];
    }
}

// -------------------------------------------------------------------- QR --
// Plane rotation R = (1/nu) [[conj(x), conj(y)], [-y, x]], nu = ||(x, y)||,
// as c = conj(x)/nu, s = conj(y)/nu: R [x; y] = [nu; 0], R unitary.  One
// reciprocal square root (the FP64 chain of one thread is the critical path
// of every rotation); inputs rescaled first when |x|^2 + |y|^2 would leave
// the normal range.
__device__ void make_rot(zd x, zd y, zd &c, zd &s) {
  double n2 = fma(x.x, x.x, fma(x.y, x.y, fma(y.x, y.x, y.y * y.y)));
  if (!(n2 > 1e-290 && n2 < 1e290)) {
    const double sc = fmax(fmax(fabs(x.x), fabs(x.y)), fmax(fabs(y.x), fabs(y.y)));
    if (!(sc > 0.0) || !isfinite(sc)) {
      c = zd{1.0, 0.0};
      s = zd{0.0, 0.0};
      return;
    }
    const double is = 1.0 / sc;
    x = zsc(x, is);
    y = zsc(y, is);
    n2 = fma(x.x, x.x, fma(x.y, x.y, fma(y.x, y.x, y.y * y.y)));
  }
  const double r = fast_rsqrt(n2);
  c = zd{x.x * r, -x.y * r};
  s = zd{y.x * r, -y.y * r};
}

// Complex Schur form of the upper Hessenberg H (in place) with Z <- Z R^H for
// every rotation R; lam = diag(T).  err = 1 when more than 30 m sweeps were
// needed (not converged).  H (and Z) are worked on in shared memory when they
// fit.  FP64 instructions issue slowly per warp on this GPU, so the serial
// scalar steps (deflation test, shift, rotation) run in one thread, and each
// rotation's update gives every thread one complex output: the two threads
// of a row (or column) pair read both inputs, meet at a warp barrier, then
// write.
__global__ void __launch_bounds__(RT) hqr_kernel(int m, zd *Hg, zd *Zg, zd *lam, int *err, int h_smem, int z_smem) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ zd s_x, s_y, s_c, s_s;
  // lo of step t in slot t % 3; slot (t + 2) % 3 is cleared after step t's
  // barrier, which every thread passes only after reading slot (t - 1) % 3,
  // and step t + 2 scans only after step t + 1's barrier
  __shared__ int s_lo[3];
  const int tid = threadIdx.x;
  const long mm = (long)m * m;
  zd *H = h_smem ? reinterpret_cast<zd *>(smem) : Hg;
  zd *Z = z_smem ? reinterpret_cast<zd *>(smem) + (h_smem ? mm : 0) : Zg;
  for (long t = tid; t < mm; t += RT) {
    if (h_smem) H[t] = Hg[t];
    if (z_smem) Z[t] = Zg[t];
  }
  auto h = [&](int i, int j) -> zd & { return H[i + (long)j * m]; };
  __shared__ double red[RT];
  double part = 0.0;
  for (long t = tid; t < mm; t += RT) part = fmax(part, cabs1(H[t]));
  const double hnorm = block_max(part, red);  // (ends with a barrier)
  const double small = DBL_MIN * ((double)m / DBL_EPSILON);
  const int maxsweeps = 30 * (m > 10 ? m : 10);
  int hi = m - 1, its = 0, sweeps = 0, par = 0;
  if (tid == 0) s_lo[0] = s_lo[1] = s_lo[2] = 0;
  __syncthreads();
  while (hi > 0) {
    // lo: the largest l <= hi with a negligible h(l, l-1), else 0
    for (int l = 1 + tid; l <= hi; l += RT) {
      const double sl = cabs1(h(l, l - 1));
      double tst = cabs1(h(l - 1, l - 1)) + cabs1(h(l, l));
      if (tst == 0.0) tst = hnorm;
      if (sl <= small || sl <= DBL_EPSILON * tst) atomicMax(&s_lo[par], l);
    }
    __syncthreads();
    const int lo = s_lo[par];
    if (tid == 0) s_lo[(par + 2) % 3] = 0;
    par = (par + 1) % 3;
    if (lo > 0 && tid == 0) h(lo, lo - 1) = zd{0.0, 0.0};
    if (lo == hi) {  // h(hi, hi) is an eigenvalue of the deflated block
      --hi;
      its = 0;
      continue;
    }
    if (++sweeps > maxsweeps) {
      if (tid == 0) *err = 1;
      break;
    }
    ++its;
    if (tid == 0) {
      zd mu;
      if (its % 10 == 0) {  // exceptional shift
        mu = X::add(h(hi, hi), zd{0.75 * cabs1(h(hi, hi - 1)), 0.0});
      } else {  // eigenvalue of the trailing 2 x 2 block closer to h(hi, hi)
        const zd a = h(hi - 1, hi - 1), b = h(hi - 1, hi), cc = h(hi, hi - 1), d = h(hi, hi);
        const zd t = zsc(X::sub(a, d), 0.5), bc = X::mul(b, cc);
        zd disc = zsqrt(X::fma(t, t, bc));
        if (t.x * disc.x + t.y * disc.y < 0.0) disc = X::neg(disc);
        const zd den = X::add(t, disc);
        mu = (den.x == 0.0 && den.y == 0.0) ? d : X::sub(d, zdiv(bc, den));
      }
      s_x = X::sub(h(lo, lo), mu);
      s_y = h(lo + 1, lo);
    }
    for (int k = lo; k < hi; ++k) {
      if (tid == 0) {
        zd c, sn;
        make_rot(s_x, s_y, c, sn);
        s_c = c;
        s_s = sn;
      }
      __syncthreads();
      const zd c = s_c, sn = s_s, cc = X::conj(c), cs = X::conj(sn), ms = X::neg(sn), mcs = X::neg(cs);
      // left: rows k, k+1 from column k-1 (k > lo: the bulge column) on;
      // lanes 2q, 2q+1 take column j0 + q, rows k and k+1
      const int j0 = (k == lo) ? lo : k - 1;
      for (int base = 0; base < 2 * (m - j0); base += RT) {
        const int t = base + tid, j = j0 + (t >> 1);
        const bool act = j < m;
        zd a{0.0, 0.0}, b{0.0, 0.0};
        if (act) {
          a = h(k, j);
          b = h(k + 1, j);
        }
        __syncwarp();
        if (act) {
          if ((t & 1) == 0) h(k, j) = X::fma(sn, b, X::mul(c, a));
          else h(k + 1, j) = (j == k - 1) ? zd{0.0, 0.0} : X::fma(mcs, a, X::mul(cc, b));
        }
      }
      __syncthreads();
      // right: columns k, k+1 of rows 0..i1 of H and of every row of Z;
      // lanes 2q, 2q+1 take one row, columns k and k+1
      const int i1 = (k + 2 < hi) ? k + 2 : hi;
      const int nh = 2 * (i1 + 1), items = nh + 2 * m;
      for (int base = 0; base < items; base += RT) {
        const int t = base + tid;
        const bool act = t < items, onH = t < nh;
        const int i = onH ? (t >> 1) : ((t - nh) >> 1);
        zd *P = onH ? H : Z;
        zd a{0.0, 0.0}, b{0.0, 0.0};
        if (act) {
          a = P[i + (long)k * m];
          b = P[i + (long)(k + 1) * m];
        }
        __syncwarp();
        if (act) {
          if ((t & 1) == 0) {
            const zd na = X::fma(cs, b, X::mul(cc, a));
            P[i + (long)k * m] = na;
            if (onH && i == k + 1) s_x = na;  // the next rotation's pair
            if (onH && i == k + 2) s_y = na;
          } else {
            P[i + (long)(k + 1) * m] = X::fma(ms, a, X::mul(c, b));
          }
        }
      }
      __syncthreads();
    }
  }
  __syncthreads();
  for (int i = tid; i < m; i += RT) lam[i] = h(i, i);
  for (long t = tid; t < mm; t += RT) {
    if (h_smem) Hg[t] = H[t];
    if (z_smem) Zg[t] = Z[t];
  }
}

// ------------------------------------------------------------ eigenvectors --
// Column k of Y: the eigenvector of the upper triangular T for T[k, k]:
// y_k = 1, y_i = -(sum_{l=i+1..k} T[i, l] y_l) / (T[i, i] - T[k, k]) for
// i < k (the denominator raised to smin when smaller), y_i = 0 for i > k.
// One warp per k; lane l keeps the running sums of rows l, l+32, ...
template <int MAXR>
__global__ void trevc_kernel(int m, const zd *T, zd *Y) {
  const int k = (int)((blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (k >= m) return;
  const zd tkk = T[k + (long)k * m];
  const double smin = fmax(DBL_EPSILON * cabs1(tkk), DBL_MIN * ((double)m / DBL_EPSILON));
  zd acc[MAXR];
#pragma unroll
  for (int r = 0; r < MAXR; ++r) {
    const int i = lane + 32 * r;
    acc[r] = (i < k) ? T[i + (long)k * m] : zd{0.0, 0.0};
  }
  zd *Yk = Y + (long)k * m;
  for (int i = k + lane; i < m; i += 32) Yk[i] = zd{(i == k) ? 1.0 : 0.0, 0.0};
#pragma unroll
  for (int r = MAXR - 1; r >= 0; --r) {
    if (32 * r >= k) continue;
    for (int l = 31; l >= 0; --l) {
      const int i = 32 * r + l;
      if (i >= k) continue;
      zd y{0.0, 0.0};
      if (lane == l) {
        zd den = X::sub(T[i + (long)i * m], tkk);
        if (cabs1(den) < smin) den = zd{smin, 0.0};
        y = X::neg(zdiv(acc[r], den));
        Yk[i] = y;
      }
      y.x = __shfl_sync(0xffffffffu, y.x, l);
      y.y = __shfl_sync(0xffffffffu, y.y, l);
      const zd *Ti = T + (long)i * m;
#pragma unroll
      for (int q = 0; q < MAXR; ++q) {
        if (q > r) break;
        const int row = lane + 32 * q;
        if (row < i) acc[q] = X::fma(Ti[row], y, acc[q]);
      }
    }
  }
}

}  // namespace

// ------------------------------------------------------------- launchers --
static dim3 grid2(int n, int m) { return dim3((unsigned)ceil_div(n, 256), (unsigned)m); }

int gen_widen(cudaStream_t st, int n, const double *A, long lda, zd *Af) {
  widen_ld_kernel<<<grid2(n, n), 256, 0, st>>>(n, A, lda, Af);
  GBF_LAUNCHED();
  GBF_CUDA(cudaGetLastError());
  return 0;
}
int gen_conj_pair(cudaStream_t st, int n, int m, const zd *src, zd *dst) {
  if (m < 1) return 0;
  conj_pair_kernel<<<grid2(n, m), 256, 0, st>>>(n, m, src, dst);
  GBF_LAUNCHED();
  GBF_CUDA(cudaGetLastError());
  return 0;
}
template <class TY>
int gen_accumulate(cudaStream_t st, int n, int m, int nf, const zd *w, const TY *Y, int mw, int half, int left,
                   const zd *X0, const zd *f, zd *Q) {
  if (m < 1) return 0;
  accum_gen_kernel<TY><<<grid2(n, m), 256, 0, st>>>(n, m, nf, w, Y, mw, half, left, X0, f, Q);
  GBF_LAUNCHED();
  GBF_CUDA(cudaGetLastError());
  return 0;
}
template int gen_accumulate<zd>(cudaStream_t, int, int, int, const zd *, const zd *, int, int, int, const zd *,
                                const zd *, zd *);
template int gen_accumulate<cf>(cudaStream_t, int, int, int, const zd *, const cf *, int, int, int, const zd *,
                                const zd *, zd *);
int gen_scales(cudaStream_t st, int m, int nf, int ne, const zd *z, const zd *w, const zd *lam, int half, zd *SCr,
               zd *SCl, zd *f) {
  gen_scales_kernel<<<ceil_div(m, 128), 128, 0, st>>>(m, nf, ne, z, w, lam, half, SCr, SCl, f);
  GBF_LAUNCHED();
  GBF_CUDA(cudaGetLastError());
  return 0;
}
int gen_eig_residual(cudaStream_t st, int n, int m, const zd *MX, const zd *NX, const zd *lam, int conjl,
                     const double *sc, zd *R) {
  if (m < 1) return 0;
  gen_eig_residual_kernel<<<grid2(n, m), 256, 0, st>>>(n, MX, NX, lam, conjl, sc, R);
  GBF_LAUNCHED();
  GBF_CUDA(cudaGetLastError());
  return 0;
}
int gen_col_norms(cudaStream_t st, int n, int m, const zd *Xm, double *nrm) {
  if (m < 1) return 0;
  col_norms_kernel<<<m, RT, 0, st>>>(n, Xm, nrm);
  GBF_LAUNCHED();
  GBF_CUDA(cudaGetLastError());
  return 0;
}
int gen_col_scale(cudaStream_t st, int n, int m, const zd *src, zd *dst, const double *s, int divide) {
  if (m < 1) return 0;
  col_scale_kernel<<<grid2(n, m), 256, 0, st>>>(n, src, dst, s, divide);
  GBF_LAUNCHED();
  GBF_CUDA(cudaGetLastError());
  return 0;
}
int gen_residual(cudaStream_t st, int n, int m, const zd *MX, const zd *NX, const zd *lam, int conjl, double alpha,
                 double *res) {
  if (m < 1) return 0;
  gen_residual_kernel<<<m, RT, 0, st>>>(n, MX, NX, lam, conjl, alpha, res);
  GBF_LAUNCHED();
  GBF_CUDA(cudaGetLastError());
  return 0;
}
int gen_order(cudaStream_t st, int m, const zd *lam, const double *rr, const double *rl, zd emid, double r,
              double rho, double angle_deg, int *pos, int *src, zd *Eo, double *Rr, double *Rl, double *stats) {
  if (m < 1 || m > 1024) {
    set_error("non-Hermitian ordering: subspace size %d outside 1..1024", m);
    return -4;
  }
  const double ph = angle_deg * (3.14159265358979323846 / 180.0);
  order_gen_kernel<<<1, (m + 31) / 32 * 32, 0, st>>>(m, lam, rr, rl, emid.x, emid.y, r, rho, cos(ph), sin(ph), pos,
                                                      src, Eo, Rr, Rl, stats);
  GBF_LAUNCHED();
  GBF_CUDA(cudaGetLastError());
  return 0;
}
int gen_biorth(cudaStream_t st, int m, int nin, const zd *P, const double *nr, const int *src, double *out) {
  biorth_kernel<<<1, RT, 0, st>>>(m, nin, P, nr, src, out);
  GBF_LAUNCHED();
  GBF_CUDA(cudaGetLastError());
  return 0;
}
int gen_identity(cudaStream_t st, int m, zd *I) {
  identity_kernel<<<grid2(m, m), 256, 0, st>>>(m, I);
  GBF_LAUNCHED();
  GBF_CUDA(cudaGetLastError());
  return 0;
}
static constexpr size_t GEN_SMEM = 200 * 1024;
int gen_hessenberg(cudaStream_t st, int m, zd *G, zd *Z) {
  static std::atomic<unsigned long long> attr{0};
  if (int rc = once_per_device(attr, [] {
        GBF_CUDA(cudaFuncSetAttribute(hessenberg_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GEN_SMEM));
        return 0;
      }))
    return rc;
  const size_t full = sizeof(zd) * ((size_t)m + 2 * (size_t)m * m);
  const int in_smem = full <= GEN_SMEM ? 1 : 0;
  const size_t sm = in_smem ? full : sizeof(zd) * (size_t)m;
  if (sm > GEN_SMEM) {
    set_error("Hessenberg reduction: subspace size %d too large", m);
    return -4;
  }
  const int slot = prof_begin(st);
  hessenberg_kernel<<<1, RT, sm, st>>>(m, G, Z, in_smem);
  GBF_LAUNCHED();
  GBF_CUDA(cudaGetLastError());
  prof_end(st, slot, 0.0);
  return 0;
}
int gen_hqr(cudaStream_t st, int m, zd *H, zd *Z, zd *lam, int *err) {
  static std::atomic<unsigned long long> attr{0};
  if (int rc = once_per_device(attr, [] {
        GBF_CUDA(cudaFuncSetAttribute(hqr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GEN_SMEM));
        return 0;
      }))
    return rc;
  const size_t one = sizeof(zd) * (size_t)m * m;
  const int h_smem = one <= GEN_SMEM ? 1 : 0;
  const int z_smem = (h_smem && 2 * one <= GEN_SMEM) ? 1 : 0;
  const size_t sm = one * (h_smem + z_smem);
  const int slot = prof_begin(st);
  hqr_kernel<<<1, RT, sm, st>>>(m, H, Z, lam, err, h_smem, z_smem);
  GBF_LAUNCHED();
  GBF_CUDA(cudaGetLastError());
  prof_end(st, slot, 0.0);
  return 0;
}
int gen_trevc(cudaStream_t st, int m, const zd *T, zd *Y) {
  const int blocks = ceil_div(m, 8);
  if (m > 1024) {
    set_error("triangular eigenvectors: subspace size %d above 1024", m);
    return -4;
  }
  const int slot = prof_begin(st);
  if (m <= 64)
    trevc_kernel<2><<<blocks, 256, 0, st>>>(m, T, Y);
  else if (m <= 256)
    trevc_kernel<8><<<blocks, 256, 0, st>>>(m, T, Y);
  else
    trevc_kernel<32><<<blocks, 256, 0, st>>>(m, T, Y);
  GBF_LAUNCHED();
  GBF_CUDA(cudaGetLastError());
  prof_end(st, slot, 0.0);
  return 0;
}

}  // namespace gbf
