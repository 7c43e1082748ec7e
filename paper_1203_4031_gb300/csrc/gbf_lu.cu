// Shifted-system factorisation and multi-RHS solves for all contour nodes
// (the dense driver's inner solver: RCI cases 10, 11 and 21 of the FEAST
// v3.0 guide, Fig. "fig_rci").
//
//   form_shift     S_e = z_e B - A for every node in one pass over A and B
//   getrf_batched  blocked right-looking LU with partial pivoting, all nodes
//                  in each launch (node = grid dimension):
//                    panel  : one CTA per node, warp-shuffle argmax pivot
//                             search, row swap, scale, rank-1 updates
//                    laswp+trsm : swaps outside the panel, U12 = L11^{-1} A12
//                    update : A22 -= L21 U12 (batched GEMM)
//                  then the row permutation and inverted bs x bs diagonal
//                  blocks of L and U (reused by every solve of every FEAST
//                  iteration, since the factors are kept: fpm(10)=1 style).
//   getrs_inplace  triangular solves in which every step is a GEMM: leaves
//                  Y_b <- inv(T_bb) Y_b and updates, recursive (large-K
//                  updates) on the tensor-core engine, blocked otherwise.
//                  trans=1 gives S^H Y = R from the same factors (case 21).
#include <cooperative_groups.h>

#include <algorithm>
#include <type_traits>

#include "gbf_common.cuh"

namespace cg = cooperative_groups;

namespace gbf {

template <class T> __device__ inline T cinv(T a);
template <> __device__ inline zd cinv<zd>(zd a) { return zdiv(zd{1.0, 0.0}, a); }
template <> __device__ inline cf cinv<cf>(cf a) {
  zd r = zdiv(zd{1.0, 0.0}, zd{(double)a.x, (double)a.y});
  return cf{(float)r.x, (float)r.y};
}

// ------------------------------------------------------------ form_shift --
template <class T>
__global__ void form_shift_kernel(int n, int ne, const zd *__restrict__ z, int kindA, char uplo,
                                  const void *__restrict__ Av, long lda, const void *__restrict__ Bv,
                                  long ldb, T *__restrict__ S, int *bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= n) return;
  // element (i, j) of the full Hermitian matrix from the referenced triangle
  const bool mirror = (uplo == 'L' && i < j) || (uplo == 'U' && i > j);
  const long src = mirror ? (j + (long)i * lda) : (i + (long)j * lda);
  const long srcb = mirror ? (j + (long)i * ldb) : (i + (long)j * ldb);
  zd a, b;
  if (kindA == 0) {
    a = zd{((const double *)Av)[src], 0.0};
    b = Bv ? zd{((const double *)Bv)[srcb], 0.0} : zd{i == j ? 1.0 : 0.0, 0.0};
  } else {
    a = ((const zd *)Av)[src];
    b = Bv ? ((const zd *)Bv)[srcb] : zd{i == j ? 1.0 : 0.0, 0.0};
    if (mirror) {
      a.y = -a.y;
      b.y = -b.y;
    }
    if (i == j && uplo != 'G') {  // 'G': a general (non-Hermitian) pencil, taken as stored
      a.y = 0.0;
      b.y = 0.0;
    }
  }
  if (bad && !(isfinite(a.x) && isfinite(a.y) && isfinite(b.x) && isfinite(b.y))) *bad = 1;
  const long nn = (long)n * n;
  const long off = i + (long)j * n;
  for (int e = 0; e < ne; ++e) {
    const zd ze = z[e];
    zd s = zd{ze.x * b.x - ze.y * b.y - a.x, ze.x * b.y + ze.y * b.x - a.y};
    S[e * nn + off] = cvt<T, zd>(s);
  }
}

template <class T>
int form_shift(cudaStream_t st, int n, int ne, const zd *z, int kindA, char uplo, const void *A, long lda,
               const void *B, long ldb, T *S, int *bad) {
  dim3 grid(ceil_div(n, 256), n);
  form_shift_kernel<T><<<grid, 256, 0, st>>>(n, ne, z, kindA, uplo, A, lda, B, ldb, S, bad);
  GBF_LAUNCHED();
  GBF_CUDA(cudaGetLastError());
  return 0;
}

// ---------------------------------------------------------------- panel --
// Pivot comparison key of a magnitude |re| + |im| >= 0: its bit pattern as
// an integer (ordered like the value for non-negative numbers), -1 for NaN
// (never chosen).  The argmax then runs on the integer units: FP64
// instructions are the scarce resource on this GPU.
__device__ inline long long pivkey(double v) {
  const long long b = __double_as_longlong(v);
  return b > 0x7FF0000000000000LL ? -1LL : b;
}
__device__ inline long long pivkey(float v) {
  const int b = __float_as_int(v);
  return b > 0x7F800000 ? -1LL : (long long)b;
}

// One CTA per node factors columns [k, k+w) of rows [k, n).
constexpr int PANEL_THREADS = 512;
constexpr int MAX_NB = 64;

template <class T>
__global__ void __launch_bounds__(PANEL_THREADS)
    lu_panel_kernel(int n, int k, int w, T *S, int *ipiv, int *sing) {
  using X = tr<T>;
  using R = typename X::R;
  const int e = blockIdx.x;
  const long nn = (long)n * n;
  T *a = S + e * nn;
  int *piv = ipiv + (long)e * n;
  __shared__ long long sval[32];
  __shared__ int sidx[32];
  __shared__ T urow[MAX_NB];
  __shared__ T s_inv;
  __shared__ int s_p, s_ok;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = blockDim.x >> 5;

  for (int j = 0; j < w; ++j) {
    const int c = k + j;
    const T *col = a + (long)c * n;
    long long best = -1;
    int bidx = n;
    for (int r = c + tid; r < n; r += blockDim.x) {
      const long long v = pivkey(X::abs1(col[r]));
      if (v > best) {
        best = v;
        bidx = r;
      }
    }
    for (int off = 16; off > 0; off >>= 1) {
      const long long ov = __shfl_down_sync(0xffffffffu, best, off);
      const int oi = __shfl_down_sync(0xffffffffu, bidx, off);
      if (ov > best || (ov == best && oi < bidx)) {
        best = ov;
        bidx = oi;
      }
    }
    if (lane == 0) {
      sval[warp] = best;
      sidx[warp] = bidx;
    }
    __syncthreads();
    if (warp == 0) {
      best = lane < nwarps ? sval[lane] : -1;
      bidx = lane < nwarps ? sidx[lane] : n;
      for (int off = 16; off > 0; off >>= 1) {
        const long long ov = __shfl_down_sync(0xffffffffu, best, off);
        const int oi = __shfl_down_sync(0xffffffffu, bidx, off);
        if (ov > best || (ov == best && oi < bidx)) {
          best = ov;
          bidx = oi;
        }
      }
      if (lane == 0) {
        const int ok = (best > 0) && (bidx < n);
        s_ok = ok;
        s_p = ok ? bidx : c;
        piv[c] = ok ? bidx : c;
        if (!ok && sing[e] == 0) sing[e] = c + 1;
      }
    }
    __syncthreads();
    const int p = s_p;
    if (!s_ok) continue;  // zero column: nothing to eliminate (reported via sing)
    if (p != c)
      for (int jj = tid; jj < w; jj += blockDim.x) {
        T *cj = a + (long)(k + jj) * n;
        const T t = cj[c];
        cj[c] = cj[p];
        cj[p] = t;
      }
    __syncthreads();
    for (int jj = tid; jj < w; jj += blockDim.x) urow[jj] = a[c + (long)(k + jj) * n];
    __syncthreads();
    // the pivot's reciprocal, formed once (a complex division is several FP64
    // divisions; every thread forming it cost more than the rank-1 update)
    if (tid == 0) s_inv = cinv<T>(urow[j]);
    __syncthreads();
    const T inv = s_inv;
    T *colc = a + (long)c * n;
    for (int r = c + 1 + tid; r < n; r += blockDim.x) {
      const T l = X::mul(colc[r], inv);
      colc[r] = l;
      for (int jj = j + 1; jj < w; ++jj) {
        T *cj = a + (long)(k + jj) * n;
        const T u = urow[jj];
        cj[r] = X::fma(l, X::neg(u), cj[r]);
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------- cluster panel --
// The panel of node e (rows [k, n), columns [k, k+w)) split by rows over the
// C CTAs of a thread-block cluster, R >= w rows each, so that the diagonal
// row c = k + j of every column j lies in CTA 0.  The slice sits in shared
// memory (column-major, ld R) when it fits, else the CTA works on it in
// place in the matrix (ld n; a few MB per node, L2-resident).
// One cluster barrier per column:
//   1. each CTA publishes its best pivot candidate for column j (key, row
//      index and the row's w entries) and CTA 0 also the current row c, in
//      the buffer of parity j % 2;
//   2. cluster barrier;
//   3. every CTA reads all C candidates and row c over distributed shared
//      memory (one round of remote loads), warp 0 picks the pivot (largest
//      |re| + |im|, lowest row on ties; the same choice in every CTA), writes
//      the swap into the CTA's own rows and forms the pivot's reciprocal;
//   4. the column below c is scaled, then the rank-1 update runs on all
//      warps (each thread one row and every G-th column), and the thread
//      that updates column j + 1 of a row forms that row's next candidate.
// A buffer of parity j % 2 is rewritten at column j + 2, after every CTA has
// passed barrier j + 1 and therefore finished its reads of it.
// Leading dimension of a panel slice of R rows in shared memory.
__host__ __device__ constexpr int panel_ld(int R) { return ((R + 15) & ~15) + 1; }

template <class T>
struct PanelPub {
  T row[MAX_NB];   // entries of this CTA's candidate row
  T diag[MAX_NB];  // CTA 0: the current row c
  long long key;
  int idx;
  int pad;
};

// Argmax of (key, row) pairs over a warp: the larger key wins, the lower row
// on ties; every lane ends with the result.  Keys are >= -1 and rows >= 0.
// Three hardware warp reductions (the key's high word, its low word among
// the lanes holding that high word, the lowest row holding the key): the
// five-round 64-bit shuffle butterfly took about ten times longer here.
__device__ __forceinline__ void argmax_all(long long &b, int &bi) {
  const unsigned long long u = (unsigned long long)(b + 1);
  const unsigned hi = __reduce_max_sync(0xffffffffu, (unsigned)(u >> 32));
  const unsigned lo = __reduce_max_sync(0xffffffffu, (unsigned)(u >> 32) == hi ? (unsigned)u : 0u);
  const long long mx = (long long)(((unsigned long long)hi << 32) | lo) - 1;
  bi = (int)__reduce_min_sync(0xffffffffu, b == mx ? (unsigned)bi : 0xffffffffu);
  b = mx;
}

__device__ __forceinline__ zd shfl_t(zd v, int src) {
  return zd{__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src)};
}
__device__ __forceinline__ cf shfl_t(cf v, int src) {
  return cf{__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src)};
}

// Reciprocal of a nonzero pivot: a is scaled by the power of two f that
// brings its larger part into [1, 2) (exact), then 1/a = conj(f a) f / d
// with d = |f a|^2 in [1, 8), 1/d by fast_rcp (a few ulp, a much shorter
// chain on this GPU's FP64 unit than a division).  Zero, subnormal, huge or
// non-finite pivots take Smith's division.
__device__ inline zd pivot_recip(zd a) {
  const double s = fmax(fabs(a.x), fabs(a.y));
  const long long eb = (__double_as_longlong(s) >> 52) & 0x7FF;
  if (eb == 0 || eb >= 2046) return zdiv(zd{1.0, 0.0}, a);
  const double f = __longlong_as_double((2046LL - eb) << 52);
  const double ax = a.x * f, ay = a.y * f;
  const double r = fast_rcp(fma(ax, ax, ay * ay)) * f;
  return zd{ax * r, -ay * r};
}
__device__ inline cf pivot_recip(cf a) {
  const float s = fmaxf(fabsf(a.x), fabsf(a.y));
  const int eb = (__float_as_int(s) >> 23) & 0xFF;
  if (eb == 0 || eb >= 254) return cinv<cf>(a);
  const float f = __int_as_float((254 - eb) << 23);
  const float ax = a.x * f, ay = a.y * f;
  const float r = f / fmaf(ax, ax, ay * ay);
  return cf{ax * r, -ay * r};
}

template <class T, bool SMEM>
__global__ void __launch_bounds__(PANEL_THREADS)
    lu_panel_cluster_kernel(int n, int k, int w, int R, T *S, int *ipiv, int *sing, T *linv, long lsb, int lld) {
  using X = tr<T>;
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int q = (int)cl.block_rank();
  const int e = blockIdx.y;
  const long nn = (long)n * n;
  T *a = S + e * nn;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int r0 = k + q * R;
  const int rows = max(0, min(R, n - r0));
  unsigned char *sp = smem_raw;
  T *sl;
  long ld;
  if constexpr (SMEM) {
    // leading dimension 1 mod 16: the row accesses (publishing a candidate,
    // the swap) fall into distinct banks; column accesses stay contiguous
    sl = reinterpret_cast<T *>(sp);
    ld = panel_ld(R);
    sp += (size_t)ld * w * sizeof(T);
  } else {
    sl = a + r0 + (long)k * n;
    ld = n;
  }
  PanelPub<T> *pub = reinterpret_cast<PanelPub<T> *>(sp);  // [2]
  sp += 2 * sizeof(PanelPub<T>);
  T *srow = reinterpret_cast<T *>(sp);  // [C][w] candidate rows of all CTAs
  sp += (size_t)C * w * sizeof(T);
  T *sdiag = reinterpret_cast<T *>(sp);  // [w] row c
  sp += (size_t)MAX_NB * sizeof(T);
  T *l11 = reinterpret_cast<T *>(sp);  // [32][32] copy of L11 for its inverse
  sp += (size_t)32 * 32 * sizeof(T);
  long long *skey = reinterpret_cast<long long *>(sp);  // [C]
  int *sidx = reinterpret_cast<int *>(skey + 16);       // [C]
  __shared__ long long wv[PANEL_THREADS / 32];
  __shared__ int wi[PANEL_THREADS / 32];
  __shared__ T s_inv;
  __shared__ int s_p, s_ok;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  // thread (rt, g): rows rt, rt + Rt, ...; columns j+1+g, j+1+g+G, ...
  const int Rt = min((int)blockDim.x, max(32, (rows + 31) & ~31));
  const int G = (int)blockDim.x / Rt;
  const int rt = tid % Rt, g = tid / Rt;
  if constexpr (SMEM) {
    for (int t = tid; t < rows * w; t += blockDim.x) {
      const int rl = t % rows, jj = t / rows;
      sl[(long)jj * ld + rl] = a[(r0 + rl) + (long)(k + jj) * n];
    }
    __syncthreads();
  }
  // candidates of column 0 (rows >= k: all of them)
  long long best = -1;
  int bidx = n;
  if (g == 0)
    for (int rl = rt; rl < rows; rl += Rt) {
      const long long v = pivkey(X::abs1(sl[rl]));
      if (v > best) {
        best = v;
        bidx = r0 + rl;
      }
    }
  for (int j = 0; j < w; ++j) {
    const int c = k + j, par = j & 1;
    // 1. this CTA's candidate, published with its row (and row c by CTA 0)
    argmax_all(best, bidx);
    if (lane == 0) {
      wv[warp] = best;
      wi[warp] = bidx;
    }
    __syncthreads();
    if (warp == 0) {
      long long b = lane < nwarps ? wv[lane] : -1;
      int bi = lane < nwarps ? wi[lane] : n;
      argmax_all(b, bi);
      if (lane == 0) {
        pub[par].key = b;
        pub[par].idx = bi;
      }
      const int lr = (b > 0 && bi < n) ? bi - r0 : -1;
      for (int jj = lane; jj < w; jj += 32) {
        if (lr >= 0) pub[par].row[jj] = sl[(long)jj * ld + lr];
        if (q == 0) pub[par].diag[jj] = sl[(long)jj * ld + j];
      }
    }
    cl.sync();  // every candidate of column j published; column j-1 done everywhere
    // 2. all candidates and row c, one round of remote loads
    const int nload = C * w + C + w;
    for (int t = tid; t < nload; t += blockDim.x) {
      if (t < C * w) {
        srow[t] = cl.map_shared_rank(pub + par, t / w)->row[t % w];
      } else if (t < C * w + C) {
        const PanelPub<T> *rp = cl.map_shared_rank(pub + par, t - C * w);
        skey[t - C * w] = rp->key;
        sidx[t - C * w] = rp->idx;
      } else {
        sdiag[t - C * w - C] = cl.map_shared_rank(pub + par, 0)->diag[t - C * w - C];
      }
    }
    __syncthreads();
    // 3. pivot, swap of this CTA's rows, reciprocal (warp 0)
    if (warp == 0) {
      long long b = lane < C ? skey[lane] : -1;
      int bi = lane < C ? sidx[lane] : n;
      argmax_all(b, bi);
      const int ok = (b > 0) && (bi < n);
      const int p = ok ? bi : c;
      const int qp = (p - k) / R;
      const T *urow = srow + (long)qp * w;
      if (ok && p != c)
        for (int jj = lane; jj < w; jj += 32) {
          if (q == 0) sl[(long)jj * ld + j] = urow[jj];
          if (q == qp) sl[(long)jj * ld + (p - r0)] = sdiag[jj];
        }
      if (lane == 0) {
        s_p = p;
        s_ok = ok;
        if (ok) s_inv = pivot_recip(urow[j]);
        if (q == 0) {
          ipiv[(long)e * n + c] = p;
          if (!ok && sing[e] == 0) sing[e] = c + 1;
        }
      }
    }
    __syncthreads();
    const int ok = s_ok;
    const T *urow = srow + (long)((s_p - k) / R) * w;
    // 4a. scale the column below c
    if (ok && g == 0) {
      const T inv = s_inv;
      for (int rl = rt; rl < rows; rl += Rt)
        if (r0 + rl > c) sl[(long)j * ld + rl] = X::mul(sl[(long)j * ld + rl], inv);
    }
    __syncthreads();
    // 4b. rank-1 update; column j+1's candidates from the updated entries
    best = -1;
    bidx = n;
    if (g < G && j + 1 < w) {
      for (int rl = rt; rl < rows; rl += Rt) {
        const int gr = r0 + rl;
        if (gr <= c) continue;
        int jj = j + 1 + g;
        if (ok) {
          const T l = sl[(long)j * ld + rl];
          if (g == 0) {
            const T v = X::fma(l, X::neg(urow[jj]), sl[(long)jj * ld + rl]);
            sl[(long)jj * ld + rl] = v;
            const long long kv = pivkey(X::abs1(v));
            if (kv > best) {
              best = kv;
              bidx = gr;
            }
            jj += G;
          }
          for (; jj < w; jj += G) sl[(long)jj * ld + rl] = X::fma(l, X::neg(urow[jj]), sl[(long)jj * ld + rl]);
        } else if (g == 0) {
          const long long kv = pivkey(X::abs1(sl[(long)jj * ld + rl]));
          if (kv > best) {
            best = kv;
            bidx = gr;
          }
        }
      }
    }
  }
  __syncthreads();
  if (linv) {
    // L11^{-1} (unit lower, w x w, ld lld), the columns dealt to the warps
    // of all CTAs: column j by warp j / C of CTA j % C, lane i holding entry
    // i, forward substitution with the column of L11 broadcast per step
    cl.sync();  // rows k .. k+w-1 final in CTA 0
    for (int t = tid; t < w * w; t += blockDim.x) {
      const int i = t % w, l = t / w;
      T v;
      if constexpr (SMEM)
        v = (q == 0) ? sl[(long)l * ld + i] : cl.map_shared_rank(sl, 0)[(long)l * ld + i];
      else
        v = a[(k + i) + (long)(k + l) * n];
      l11[i + l * 32] = v;
    }
    __syncthreads();
    T *li = linv + (long)e * lsb;
    for (int j = q + C * warp; j < w; j += C * nwarps) {
      T x = lane == j ? X::one() : X::zero();
      for (int l = j; l < w - 1; ++l) {
        const T xl = shfl_t(x, l);
        if (lane > l && lane < w) x = X::fma(l11[l * 32 + lane], X::neg(xl), x);
      }
      if (lane < w) li[lane + (long)j * lld] = x;
    }
  }
  if constexpr (SMEM)
    for (int t = tid; t < rows * w; t += blockDim.x) {
      const int rl = t % rows, jj = t / rows;
      a[(r0 + rl) + (long)(k + jj) * n] = sl[(long)jj * ld + rl];
    }
  cl.sync();  // no CTA leaves while another may still read its buffers
}

// Dynamic shared memory of the cluster panel for C CTAs of R rows.
template <class T>
static size_t panel_smem(int R, int w, int C, bool slice_in_smem) {
  return (slice_in_smem ? (size_t)panel_ld(R) * w * sizeof(T) : 0) + 2 * sizeof(PanelPub<T>) + (size_t)C * w * sizeof(T) +
         MAX_NB * sizeof(T) + 32 * 32 * sizeof(T) + 16 * (sizeof(long long) + sizeof(int));
}

// Clusters of C CTAs with `smem` bytes of dynamic shared memory each that
// the device runs at once (queried once per device, C and 16 KB bucket).
template <class T>
static int panel_clusters(int C, size_t smem) {
  static std::atomic<int> cache[16][5][14];
  int dev = 0;
  cudaGetDevice(&dev);
  int lc = 0;
  while ((1 << lc) < C) ++lc;
  const int sb = (int)((smem + 16383) / 16384);
  if (dev >= 16 || lc > 4 || sb > 13) return 0;
  int v = cache[dev][lc][sb].load(std::memory_order_relaxed);
  if (v != 0) return v - 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C, 1, 1);
  cfg.blockDim = dim3(PANEL_THREADS, 1, 1);
  cfg.dynamicSmemBytes = (size_t)sb * 16384;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nc = 0;
  if (cudaOccupancyMaxActiveClusters(&nc, lu_panel_cluster_kernel<T, true>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    nc = 0;
  }
  cache[dev][lc][sb].store(nc + 1, std::memory_order_relaxed);
  return nc;
}

// Launch the cluster panel.  C (a power of two <= 16, R = ceil((n-k)/C) >= w
// rows per CTA) and the slice's place minimise waves x (R + 64): the FP64
// rank-1 work of a CTA grows with R, and the per-column barrier and
// remote-load latency costs about as much as 64 rows; waves = ceil(ne /
// clusters the device runs at once).  With linv, the kernel also writes L11^{-1} of every node there
// (ld lld, node stride lsb).  Returns 1 when the caller should use the
// single-CTA panel
// instead (no cluster shape can run).
template <class T>
static int launch_cluster_panel(cudaStream_t st, int n, int ne, int k, int w, T *S, int *ipiv, int *sing, T *linv,
                                long lsb, int lld) {
  const int rowsp = n - k;
  const size_t cap = 200 * 1024;
  static std::atomic<unsigned long long> attr_done{0};
  once_per_device(attr_done, [&]() -> int {
    cudaFuncSetAttribute(lu_panel_cluster_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
    cudaFuncSetAttribute(lu_panel_cluster_kernel<T, true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(lu_panel_cluster_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    cudaFuncSetAttribute(lu_panel_cluster_kernel<T, false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaGetLastError();
    return 0;
  });
  // candidates: every C with the slice in shared memory (when it fits) and
  // in place; in place costs a quarter more per row (its row accesses go to
  // L2) but needs little shared memory, so more clusters run at once
  int bestC = 0;
  bool best_smem = true;
  double best_cost = 0.0;
  for (int C = 1; C <= 16; C *= 2) {
    const int R = ceil_div(rowsp, C);
    if (C > 1 && R < w) break;
    for (int mode = 0; mode < 2; ++mode) {
      const bool sm_mode = (mode == 0);
      const size_t sm = panel_smem<T>(R, w, C, sm_mode);
      if (sm_mode && sm > cap) continue;
      const int nc = panel_clusters<T>(C, sm);
      if (nc < 1) continue;
      const double cost = (double)ceil_div(ne, nc) * (R * (sm_mode ? 1.0 : 1.25) + 64);
      if (bestC == 0 || cost < best_cost) {
        bestC = C;
        best_smem = sm_mode;
        best_cost = cost;
      }
    }
  }
  if (bestC == 0) return 1;
  const int C = bestC, R = ceil_div(rowsp, C);
  const bool in_smem = best_smem;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C, ne, 1);
  cfg.blockDim = dim3(PANEL_THREADS, 1, 1);
  cfg.dynamicSmemBytes = panel_smem<T>(R, w, C, in_smem);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t rc =
      in_smem ? cudaLaunchKernelEx(&cfg, lu_panel_cluster_kernel<T, true>, n, k, w, R, S, ipiv, sing, linv, lsb, lld)
              : cudaLaunchKernelEx(&cfg, lu_panel_cluster_kernel<T, false>, n, k, w, R, S, ipiv, sing, linv, lsb, lld);
  if (rc != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  GBF_LAUNCHED();
  return 0;
}

// --------------------------------------------------------- laswp + trsm --
// Columns outside the panel: apply the panel's row swaps; columns right of
// the panel additionally get U12 = L11^{-1} A12 (unit lower forward solve).
// One thread per column.
constexpr int SWAP_COLS = 64;

// Panels of more than 32 columns: the swaps one after another.
template <class T>
__global__ void __launch_bounds__(SWAP_COLS)
    laswp_trsm_wide_kernel(int n, int k, int w, T *S, const int *ipiv) {
  using X = tr<T>;
  const int e = blockIdx.y;
  const long nn = (long)n * n;
  T *a = S + e * nn;
  const int *piv = ipiv + (long)e * n + k;
  // dynamic shared memory: L11 (w x w, ld w) then the w pivots
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *L = reinterpret_cast<T *>(smem_raw);
  int *sp = reinterpret_cast<int *>(L + w * w);
  for (int t = threadIdx.x; t < w; t += blockDim.x) sp[t] = piv[t];
  for (int t = threadIdx.x; t < w * w; t += blockDim.x) {
    const int ii = t % w, jj = t / w;
    L[ii + jj * w] = a[(k + ii) + (long)(k + jj) * n];
  }
  __syncthreads();
  const int idx = blockIdx.x * SWAP_COLS + threadIdx.x;
  if (idx >= n - w) return;
  const int col = idx < k ? idx : idx + w;
  T *cj = a + (long)col * n;
  for (int jj = 0; jj < w; ++jj) {
    const int p = sp[jj];
    if (p != k + jj) {
      const T t = cj[k + jj];
      cj[k + jj] = cj[p];
      cj[p] = t;
    }
  }
  if (col < k + w) return;
  T x[MAX_NB];
  for (int jj = 0; jj < w; ++jj) x[jj] = cj[k + jj];
  for (int jj = 0; jj < w; ++jj) {
    const T xj = x[jj];
    for (int ii = jj + 1; ii < w; ++ii) x[ii] = X::fma(L[ii + jj * w], X::neg(xj), x[ii]);
  }
  for (int jj = 0; jj < w; ++jj) cj[k + jj] = x[jj];
}

// Panels of at most 32 columns.  Warp 0 first turns the swap sequence (row
// k+jj with ipiv[k+jj], jj = 0..w-1) into the rows' final sources: panel row
// k+jj receives original row srcp[jj], and each row below the panel that was
// chosen as a pivot receives an original panel row.  (A row chosen at step
// jj hands its contents to panel row k+jj, which no later step touches, so
// rows below the panel only ever receive panel rows.)  Every thread then
// reads all its sources before it writes anything: independent loads instead
// of a chain of dependent swaps.  The solve (trsm != 0; otherwise U12 is
// formed afterwards by a product with L11^{-1}) keeps the 32 entries in
// registers.
template <class T>
__global__ void __launch_bounds__(SWAP_COLS)
    laswp_trsm_kernel(int n, int k, int w, T *S, const int *ipiv, int trsm) {
  using X = tr<T>;
  const int e = blockIdx.y;
  const long nn = (long)n * n;
  T *a = S + e * nn;
  const int *piv = ipiv + (long)e * n + k;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *L = reinterpret_cast<T *>(smem_raw);         // [w][w]
  int *srcp = reinterpret_cast<int *>(L + w * w);  // [32] source of panel row k + jj
  int *orow = srcp + 32;                           // [32] rows below the panel that receive ...
  int *osrc = orow + 32;                           // [32] ... this original panel row
  __shared__ int s_nout;
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid < 32) {
    const unsigned FULL = 0xffffffffu;
    const int pv = lane < w ? piv[lane] : -1;
    int cont = k + lane, bef = k + lane;  // lane jj: contents of row k+jj now / before step jj
    for (int jj = 0; jj < w; ++jj) {
      const int P = __shfl_sync(FULL, pv, jj);
      const int cj = __shfl_sync(FULL, cont, jj);
      if (lane == jj) bef = cj;
      if (P == k + jj) continue;
      if (P < k + w) {  // swap inside the panel
        const int cp = __shfl_sync(FULL, cont, P - k);
        if (lane == jj) cont = cp;
        if (lane == P - k) cont = cj;
      } else {  // row P holds what it received at its last earlier step, else itself
        const unsigned m = __ballot_sync(FULL, lane < jj && pv == P);
        const int v = __shfl_sync(FULL, bef, m ? 31 - __clz((int)m) : 0);
        if (lane == jj) cont = m ? v : P;
      }
    }
    if (lane < w) srcp[lane] = cont;
    const bool below = lane < w && pv >= k + w;
    const unsigned grp = __match_any_sync(FULL, below ? pv : -1 - lane);
    const bool last = below && 31 - __clz((int)grp) == lane;  // the row's last step
    const unsigned lm = __ballot_sync(FULL, last);
    if (last) {
      const int slot = __popc(lm & ((1u << lane) - 1u));
      orow[slot] = pv;
      osrc[slot] = bef;
    }
    if (lane == 0) s_nout = __popc(lm);
  }
  if (trsm)
    for (int t = tid; t < w * w; t += blockDim.x) {
      const int ii = t % w, jj = t / w;
      L[ii + jj * w] = a[(k + ii) + (long)(k + jj) * n];
    }
  __syncthreads();
  const int idx = blockIdx.x * SWAP_COLS + tid;
  if (idx >= n - w) return;
  const int col = idx < k ? idx : idx + w;
  T *cj = a + (long)col * n;
  const int nout = s_nout;
  T x[32];
#pragma unroll
  for (int jj = 0; jj < 32; ++jj)
    if (jj < w) x[jj] = cj[srcp[jj]];
  for (int i0 = 0; i0 < nout; i0 += 8) {
    T v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if (i0 + i < nout) v[i] = cj[osrc[i0 + i]];
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if (i0 + i < nout) cj[orow[i0 + i]] = v[i];
  }
  if (trsm && col >= k + w) {
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) {
      if (jj < w) {
        const T xj = X::neg(x[jj]);
#pragma unroll
        for (int ii = jj + 1; ii < 32; ++ii)
          if (ii < w) x[ii] = X::fma(L[ii + jj * w], xj, x[ii]);
      }
    }
  }
#pragma unroll
  for (int jj = 0; jj < 32; ++jj)
    if (jj < w) cj[k + jj] = x[jj];
}

// -------------------------------------------------------- permutation --
__global__ void perm_from_ipiv_kernel(int n, const int *ipiv, int *perm) {
  const int e = blockIdx.x;
  const int *pv = ipiv + (long)e * n;
  int *pe = perm + (long)e * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) pe[i] = i;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int i = 0; i < n; ++i) {
      const int p = pv[i];
      if (p != i) {
        const int t = pe[i];
        pe[i] = pe[p];
        pe[p] = t;
      }
    }
}

// ----------------------------------------- inverted diagonal blocks --
// Block b of node e: Linv = inverse of the unit lower triangle, Uinv of the
// upper triangle, both bs x bs (identity-padded past n).  Thread j forms
// column j by substitution against e_j.
template <class T>
__global__ void tri_inverse_kernel(int n, int bs, int nblk, const T *S, T *Linv, T *Uinv) {
  using X = tr<T>;
  const int b = blockIdx.x, e = blockIdx.y;
  const int r0 = b * bs;
  const int bsz = min(bs, n - r0);
  const long nn = (long)n * n;
  const T *a = S + e * nn + r0 + (long)r0 * n;  // top-left of the diagonal block
  T *li = Linv + ((long)e * nblk + b) * bs * bs;
  T *ui = Uinv + ((long)e * nblk + b) * bs * bs;
  const int j = threadIdx.x;
  if (j >= bs) return;
  T x[MAX_NB];
  // L: unit lower, forward substitution
  for (int i = 0; i < bs; ++i) x[i] = (i == j) ? X::one() : X::zero();
  if (j < bsz)
    for (int i = j + 1; i < bsz; ++i) {
      T s = x[i];
      for (int l = j; l < i; ++l) s = X::fma(a[i + (long)l * n], X::neg(x[l]), s);
      x[i] = s;
    }
  for (int i = 0; i < bs; ++i) li[i + (long)j * bs] = x[i];
  // U: upper, backward substitution
  for (int i = 0; i < bs; ++i) x[i] = (i == j) ? X::one() : X::zero();
  if (j < bsz)
    for (int i = j; i >= 0; --i) {
      T s = x[i];
      for (int l = i + 1; l <= j; ++l) s = X::fma(a[i + (long)l * n], X::neg(x[l]), s);
      x[i] = X::mul(s, cinv<T>(a[i + (long)i * n]));
    }
  for (int i = 0; i < bs; ++i) ui[i + (long)j * bs] = x[i];
}

// 128 x 128 diagonal blocks of L^-1 and U^-1 with their four 32 x 32
// diagonal sub-blocks copied from the 32-block inverses and zeros elsewhere
// (the off-diagonal sub-blocks are filled by block doubling below).
template <class T>
__global__ void big_diag_init_kernel(int nb32, int nb128, const T *Linv, const T *Uinv, T *L128, T *U128) {
  const int b = blockIdx.x, e = blockIdx.y;
  T *l = L128 + ((long)e * nb128 + b) * 128 * 128;
  T *u = U128 + ((long)e * nb128 + b) * 128 * 128;
  for (int t = threadIdx.x; t < 128 * 128; t += blockDim.x) {
    const int i = t % 128, j = t / 128;
    T lv = tr<T>::zero(), uv = tr<T>::zero();
    if (i / 32 == j / 32) {
      const long src = ((long)e * nb32 + b * 4 + i / 32) * 32 * 32 + (i % 32) + (long)(j % 32) * 32;
      lv = Linv[src];
      uv = Uinv[src];
    }
    l[t] = lv;
    u[t] = uv;
  }
}

// Copies, for every node e and 128-block b, the h x h sub-block of S at
// (r + ro, r + co), r = 128 b, into out[(e nb128 + b)] (h x h, ld h).
template <class T>
__global__ void gather_sub_kernel(int n, int nb128, int h, int ro, int co, const T *S, T *out) {
  const int b = blockIdx.x, e = blockIdx.y;
  const T *src = S + (long)e * n * n + (long)(b * 128 + ro) + (long)(b * 128 + co) * n;
  T *dst = out + ((long)e * nb128 + b) * h * h;
  for (int t = threadIdx.x; t < h * h; t += blockDim.x) dst[t] = src[(t % h) + (long)(t / h) * n];
}

// Inverses of the 128 x 128 diagonal blocks (n a multiple of 128, bs = 32),
// by doubling: for L = [A 0; C D], L^-1 = [A^-1 0; -D^-1 C A^-1 D^-1]; for
// U = [A C; 0 D], U^-1 = [A^-1 -A^-1 C D^-1; 0 D^-1]; 32 -> 64 -> 128.  All
// nodes and blocks in each batched product (the C blocks are gathered
// first); tmp holds 2 x ne x n/128 x 64 x 64 entries.
template <class T>
static int build_big_inverses(cudaStream_t st, int n, int ne, const T *S, const T *Linv, const T *Uinv, T *L128,
                              T *U128, T *tmp) {
  using X = tr<T>;
  const int nb32 = n / 32, nb128 = n / 128, nb = ne * nb128;
  const long blk = 128L * 128, sq = 64L * 64;
  const T one = X::one(), zero = X::zero(), m1 = X::sub(X::zero(), X::one());
  T *tc = tmp, *tp = tmp + (long)nb * sq;
  big_diag_init_kernel<T><<<dim3(nb128, ne), 256, 0, st>>>(nb32, nb128, Linv, Uinv, L128, U128);
  GBF_LAUNCHED();
  int rc;
  for (int h = 32; h <= 64; h *= 2)             // half size: 32 (-> 64 blocks), 64 (-> 128)
    for (int off = 0; off < 128; off += 2 * h) {  // the (2h)-blocks inside each 128-block
      // L: tp = C A^-1, X = -D^-1 tp  (C = S[off+h.., off..], X at (off+h, off))
      gather_sub_kernel<T><<<dim3(nb128, ne), 256, 0, st>>>(n, nb128, h, off + h, off, S, tc);
      GBF_LAUNCHED();
      if ((rc = gemm<T>(st, 'N', 'N', h, h, h, one, tc, h, (long)h * h, L128 + off + (long)off * 128, 128, blk, zero,
                        tp, h, (long)h * h, nb)))
        return rc;
      if ((rc = gemm<T>(st, 'N', 'N', h, h, h, m1, L128 + (off + h) + (long)(off + h) * 128, 128, blk, tp, h,
                        (long)h * h, zero, L128 + (off + h) + (long)off * 128, 128, blk, nb)))
        return rc;
      // U: tp = C D^-1, X = -A^-1 tp  (C = S[off.., off+h..], X at (off, off+h))
      gather_sub_kernel<T><<<dim3(nb128, ne), 256, 0, st>>>(n, nb128, h, off, off + h, S, tc);
      GBF_LAUNCHED();
      if ((rc = gemm<T>(st, 'N', 'N', h, h, h, one, tc, h, (long)h * h, U128 + (off + h) + (long)(off + h) * 128,
                        128, blk, zero, tp, h, (long)h * h, nb)))
        return rc;
      if ((rc = gemm<T>(st, 'N', 'N', h, h, h, m1, U128 + off + (long)off * 128, 128, blk, tp, h, (long)h * h, zero,
                        U128 + off + (long)(off + h) * 128, 128, blk, nb)))
        return rc;
    }
  return 0;
}

template <class T>
int getrf_batched(cudaStream_t st, int n, int ne, T *S, int *ipiv, int *perm, T *Linv, T *Uinv, int bs,
                  int *sing, T *) {
  using X = tr<T>;
  const int nb = std::min(bs, MAX_NB);
  const long nn = (long)n * n;
  T m1 = X::zero();
  m1 = X::sub(m1, X::one());
  // FP64 factors: U12 = L11^{-1} A12 as a product on the engine of the
  // trailing updates, with L11^{-1} formed by the cluster panel straight into
  // its block of Linv (the inverted diagonal blocks the solves use; rows
  // k .. k+w-1 are final once their panel is done), when the blocks are the
  // panel's width.  (FP32 factors: the substitution in the swap kernel costs
  // less than the extra launches.)
  const int nblk = ceil_div(n, bs);
  const long sblk = (long)nblk * bs * bs;
  const bool inv_trsm = std::is_same<T, zd>::value && nb == bs && bs <= 32;
  bool linv_ready = false;  // set by the panel of the step being processed
  auto panel = [&](cudaStream_t s, int k) {
    const int w = std::min(nb, n - k);
    CatScope cat_panel(CAT_LU_PANEL);
    const int slot = prof_begin(s);
    T *li = inv_trsm ? Linv + (long)(k / bs) * bs * bs : nullptr;
    linv_ready = inv_trsm;
    if (launch_cluster_panel<T>(s, n, ne, k, w, S, ipiv, sing, li, sblk, bs)) {
      lu_panel_kernel<T><<<ne, PANEL_THREADS, 0, s>>>(n, k, w, S, ipiv, sing);
      GBF_LAUNCHED();
      linv_ready = false;
    }
    prof_end(s, slot, 0.0);
  };
  // trailing update of panel k on the columns [c0, c1) (rows below the panel)
  auto update = [&](int k, int c0, int c1) -> int {
    const int w = std::min(nb, n - k);
    if (c1 <= c0 || n - k - w <= 0) return 0;
    CatScope cat_update(CAT_LU_UPDATE);
    return gemm<T>(st, 'N', 'N', n - k - w, c1 - c0, w, m1, S + (k + w) + (long)k * n, n, nn, S + k + (long)c0 * n,
                   n, nn, X::one(), S + (k + w) + (long)c0 * n, n, nn, ne);
  };
  // Look-ahead: the next panel depends only on its own columns, so once
  // they are updated it runs on the side stream while the main stream
  // updates the remaining columns; the next swap step waits for both.
  AuxStreams *ax = g_aux;
  panel(st, 0);
  for (int k = 0; k < n; k += nb) {
    const int w = std::min(nb, n - k);
    if (n - w > 0) {
      CatScope cat_swap(CAT_LU_SWAP);
      const int slot2 = prof_begin(st);
      dim3 g(ceil_div(n - w, SWAP_COLS), ne);
      static std::atomic<unsigned long long> attr_set{0};
      if (int rc = once_per_device(attr_set, [&]() -> int {
            GBF_CUDA(cudaFuncSetAttribute(laswp_trsm_wide_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)(MAX_NB * MAX_NB * sizeof(T) + MAX_NB * sizeof(int))));
            return 0;
          }))
        return rc;
      const bool by_inverse = linv_ready && w <= 32 && n - k - w > 0;
      if (w <= 32)
        laswp_trsm_kernel<T><<<g, SWAP_COLS, (size_t)w * w * sizeof(T) + 96 * sizeof(int), st>>>(
            n, k, w, S, ipiv, by_inverse ? 0 : 1);
      else
        laswp_trsm_wide_kernel<T><<<g, SWAP_COLS, (size_t)w * w * sizeof(T) + (size_t)w * sizeof(int), st>>>(
            n, k, w, S, ipiv);
      GBF_LAUNCHED();
      prof_end(st, slot2, 0.0);
      if (by_inverse) {  // the product times itself, in the same category
        T *A12 = S + k + (long)(k + w) * n;
        if (int rc = gemm<T>(st, 'N', 'N', w, n - k - w, w, X::one(), Linv + (long)(k / bs) * bs * bs, bs, sblk, A12,
                             n, nn, X::zero(), A12, n, nn, ne))
          return rc;
      }
    }
    const int kn = k + w;  // next panel
    if (kn >= n) break;
    const int wn = std::min(nb, n - kn);
    int rc;
    if (ax) {
      if ((rc = update(k, kn, kn + wn))) return rc;
      GBF_CUDA(cudaEventRecord(ax->a, st));
      GBF_CUDA(cudaStreamWaitEvent(ax->s, ax->a, 0));
      panel(ax->s, kn);
      GBF_CUDA(cudaEventRecord(ax->b, ax->s));
      if ((rc = update(k, kn + wn, n))) return rc;
      GBF_CUDA(cudaStreamWaitEvent(st, ax->b, 0));
    } else {
      if ((rc = update(k, kn, n))) return rc;
      panel(st, kn);
    }
  }
  perm_from_ipiv_kernel<<<ne, 256, 0, st>>>(n, ipiv, perm);
  GBF_LAUNCHED();
  dim3 g(nblk, ne);
  tri_inverse_kernel<T><<<g, bs, 0, st>>>(n, bs, nblk, S, Linv, Uinv);
  GBF_LAUNCHED();
  GBF_CUDA(cudaGetLastError());
  if constexpr (std::is_same<T, zd>::value) {
    if (g_tc && g_tc->dinv_l && bs == 32 && n % 128 == 0) {
      CatScope cat_inv(CAT_LU_SWAP);
      // the product buffer: the solves' workspace is free at this point
      return build_big_inverses<T>(st, n, ne, S, Linv, Uinv, (T *)g_tc->dinv_l, (T *)g_tc->dinv_u,
                                   (T *)g_tc->kwork);
    }
  }
  return 0;
}

// ---------------------------------------------------------------- solves --
size_t solve_kwork_bytes(int n, int nrhs, int bs, int ne) {
  const int nblk = ceil_div(n, bs);
  const int half = std::min(n, (nblk - nblk / 2) * bs);  // largest update: rows and K at most this
  size_t b = gemm_sliced_k_work(true, half, nrhs, half, std::min(ne, 8));
  if (bs == 32 && n % 128 == 0) {  // 128-row leaves (all nodes) and the doubling products
    b = std::max(b, gemm_sliced_k_work(true, 128, nrhs, 128, ne));
    b = std::max(b, (size_t)2 * ne * (n / 128) * 64 * 64 * sizeof(zd));
  }
  return b;
}

// Bytes of the factor-block slices the recursive FP64 solves would keep in a
// SliceCache for `nkinds` sweeps (kinds 0, 1 and, for adjoint solves, 2, 3):
// the same walk over the block ranges as trsv_rec, with the same node groups.
size_t solve_slice_cache_bytes(int n, int nrhs, int bs, int ne, int nkinds, bool leaves128) {
  const size_t kb = solve_kwork_bytes(n, nrhs, bs, ne);
  const int nblk = ceil_div(n, bs);
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  size_t total = 0;
  // kinds 0/2 and 1/3 have the same update shapes (m, k swapped by side)
  auto walk = [&](auto &&self, int kind, int b0, int b1) -> void {
    if (b1 - b0 == 1) return;
    if (leaves128 && b1 - b0 == 4 && bs == 32 && b0 % 4 == 0 && n % 128 == 0) {
      total += al(sliced_op_bytes(256, sliced_kp(128, true), ne));
      return;
    }
    const int mid = b0 + (b1 - b0) / 2;
    const int r0 = b0 * bs, rm = mid * bs, r1 = std::min(n, b1 * bs);
    self(self, kind, b0, mid);
    const bool lowerside = (kind == 0 || kind == 2);
    const int m = lowerside ? r1 - rm : rm - r0, k = lowerside ? rm - r0 : r1 - rm;
    if (k > 32) {
      const size_t per = gemm_sliced_k_work(true, m, nrhs, k, 1);
      const int g = (int)std::max<size_t>(1, std::min<size_t>(ne, kb / std::max<size_t>(per, 1)));
      for (int e0 = 0; e0 < ne; e0 += g)
        total += al(sliced_op_bytes(2L * m, sliced_kp(k, true), std::min(g, ne - e0)));
    }
    self(self, kind, mid, b1);
  };
  for (int kind = 0; kind < nkinds; ++kind) walk(walk, kind, 0, nblk);
  return total;
}

size_t solve_kwork_bytes_cf(int n, int nrhs, int bs, int ne) {
  const int nblk = ceil_div(n, bs);
  const int half = std::min(n, (nblk - nblk / 2) * bs);
  return cgemm_tf32k_work(half, nrhs, half, std::min(ne, 8));
}

// Leaf of the recursive solves with FP32 factors: up to four 32-row blocks
// [b0, b0 + nb) of one triangular sweep in one launch, with the same
// operations as the blocked sweep (multiply by the inverted diagonal block,
// then subtract its product from the blocks still to be solved), on the CUDA
// cores in FP32.  One CTA per (16-column slab of Y, node): the slab's rows
// and every factor block the leaf needs (at most 4 inverted diagonal blocks
// and 6 off-diagonal blocks, as op(block) rows, stride 33) are staged in
// shared memory once.  Thread (ry, cx) owns rows ry and ry + 16 of a block,
// column cx of the slab.  Rows past n are zero (the inverted blocks are
// identity-padded there).
constexpr int LEAF_NC = 16, LEAF_THREADS = 256, LEAF_LD = 33;
constexpr int LEAF_YLD = LEAF_NC + 1;  // slab row stride: the row-wise staging stores hit distinct banks
constexpr size_t LEAF_SMEM = (size_t)128 * LEAF_YLD * sizeof(cf) + (size_t)10 * 32 * LEAF_LD * sizeof(cf);

__global__ void __launch_bounds__(LEAF_THREADS)
    trsv_leaf_kernel(int kind, int n, int nrhs, int b0, int nb, const cf *__restrict__ S, const cf *__restrict__ Dinv,
                     long sblk, cf *Y) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cf *ys = reinterpret_cast<cf *>(smem_raw);  // [128][LEAF_YLD]
  cf *fb = ys + 128 * LEAF_YLD;              // blocks [slot][32][LEAF_LD]
  const int e = blockIdx.y, c0 = blockIdx.x * LEAF_NC;
  const long nn = (long)n * n;
  const cf *Se = S + e * nn;
  const cf *De = Dinv + e * sblk;
  cf *Ye = Y + e * (long)n * nrhs;
  const int r0 = b0 * 32, tid = threadIdx.x;
  const bool fwd = (kind == 0 || kind == 2), herm = kind >= 2;
  // slot of the block that updates block d from block s (s solved first):
  // the (s, d) pairs in solve order, at most 6
  auto pair_slot = [&](int s2, int d2) {
    // position of s in solve order, then d among the later blocks
    const int ps = fwd ? s2 : nb - 1 - s2, pd = fwd ? d2 - s2 - 1 : s2 - d2 - 1;
    int base = 0;
    for (int i = 0; i < ps; ++i) base += nb - 1 - i;
    return 4 + base + pd;
  };
  // 1. stage Y and the factor blocks
#pragma unroll
  for (int t = tid; t < 128 * LEAF_NC; t += LEAF_THREADS) {
    const int r = t % 128, c = t / 128;
    const int gr = r0 + r, gc = c0 + c;
    ys[r * LEAF_YLD + c] = (r < nb * 32 && gr < n && gc < nrhs) ? Ye[gr + (long)gc * n] : cf{0.f, 0.f};
  }
  for (int d = 0; d < nb; ++d) {
    const cf *D = De + (long)(b0 + d) * 32 * 32;
    cf *dst = fb + d * 32 * LEAF_LD;
#pragma unroll
    for (int t = tid; t < 32 * 32; t += LEAF_THREADS) {
      const int i = t % 32, j = t / 32;  // element (i, j) of the stored block
      const cf v = D[i + j * 32];
      if (herm)
        dst[j * LEAF_LD + i] = cf{v.x, -v.y};
      else
        dst[i * LEAF_LD + j] = v;
    }
  }
  for (int s2 = 0; s2 < nb; ++s2)
    for (int d2 = 0; d2 < nb; ++d2) {
      if (fwd ? d2 <= s2 : d2 >= s2) continue;
      cf *dst = fb + pair_slot(s2, d2) * 32 * LEAF_LD;
      // op(A)[r][l]: r a row of block d2, l a row of block s2
      //   kind 0/1: A = S[rows of d2, cols of s2]          (op N)
      //   kind 2/3: A = S[rows of s2, cols of d2]^H        (op C)
      const int rd = r0 + d2 * 32, rs = r0 + s2 * 32;
#pragma unroll
      for (int t = tid; t < 32 * 32; t += LEAF_THREADS) {
        const int i = t % 32, j = t / 32;  // element (i, j) of the stored block, i fastest
        if (!herm) {
          const int gr = rd + i, gc = rs + j;
          dst[i * LEAF_LD + j] = (gr < n && gc < n) ? Se[gr + (long)gc * n] : cf{0.f, 0.f};
        } else {
          const int gr = rs + i, gc = rd + j;
          const cf v = (gr < n && gc < n) ? Se[gr + (long)gc * n] : cf{0.f, 0.f};
          dst[j * LEAF_LD + i] = cf{v.x, -v.y};
        }
      }
    }
  __syncthreads();
  // 2. the sweep
  const int ry = tid / LEAF_NC, cx = tid % LEAF_NC;
  for (int step = 0; step < nb; ++step) {
    const int s2 = fwd ? step : nb - 1 - step;
    // y_s <- op(Dinv_s) y_s
    {
      const cf *A = fb + s2 * 32 * LEAF_LD;
      const cf *yb = ys + s2 * 32 * LEAF_YLD;
      float a0r = 0.f, a0i = 0.f, a1r = 0.f, a1i = 0.f;
#pragma unroll 8
      for (int l = 0; l < 32; ++l) {
        const cf y = yb[l * LEAF_YLD + cx];
        const cf p = A[ry * LEAF_LD + l], q = A[(ry + 16) * LEAF_LD + l];
        a0r = fmaf(p.x, y.x, fmaf(-p.y, y.y, a0r));
        a0i = fmaf(p.x, y.y, fmaf(p.y, y.x, a0i));
        a1r = fmaf(q.x, y.x, fmaf(-q.y, y.y, a1r));
        a1i = fmaf(q.x, y.y, fmaf(q.y, y.x, a1i));
      }
      __syncthreads();
      ys[(s2 * 32 + ry) * LEAF_YLD + cx] = cf{a0r, a0i};
      ys[(s2 * 32 + ry + 16) * LEAF_YLD + cx] = cf{a1r, a1i};
      __syncthreads();
    }
    // y_d -= op(A_ds) y_s for the blocks d solved later
    for (int d2 = 0; d2 < nb; ++d2) {
      if (fwd ? d2 <= s2 : d2 >= s2) continue;
      const cf *A = fb + pair_slot(s2, d2) * 32 * LEAF_LD;
      const cf *yb = ys + s2 * 32 * LEAF_YLD;
      float a0r = 0.f, a0i = 0.f, a1r = 0.f, a1i = 0.f;
#pragma unroll 8
      for (int l = 0; l < 32; ++l) {
        const cf y = yb[l * LEAF_YLD + cx];
        const cf p = A[ry * LEAF_LD + l], q = A[(ry + 16) * LEAF_LD + l];
        a0r = fmaf(p.x, y.x, fmaf(-p.y, y.y, a0r));
        a0i = fmaf(p.x, y.y, fmaf(p.y, y.x, a0i));
        a1r = fmaf(q.x, y.x, fmaf(-q.y, y.y, a1r));
        a1i = fmaf(q.x, y.y, fmaf(q.y, y.x, a1i));
      }
      cf *o0 = ys + (d2 * 32 + ry) * LEAF_YLD + cx, *o1 = ys + (d2 * 32 + ry + 16) * LEAF_YLD + cx;
      *o0 = cf{o0->x - a0r, o0->y - a0i};
      *o1 = cf{o1->x - a1r, o1->y - a1i};
    }
    __syncthreads();
  }
  // 3. write back
#pragma unroll
  for (int t = tid; t < 128 * LEAF_NC; t += LEAF_THREADS) {
    const int r = t % 128, c = t / 128;
    const int gr = r0 + r, gc = c0 + c;
    if (r < nb * 32 && gr < n && gc < nrhs) Ye[gr + (long)gc * n] = ys[r * LEAF_YLD + c];
  }
}

static int trsv_leaf(cudaStream_t st, int kind, int n, int ne, int nrhs, const cf *S, const cf *Dinv, cf *Y, int b0,
                     int nb) {
  static std::atomic<unsigned long long> attr_done{0};
  if (int rc = once_per_device(attr_done, [&]() -> int {
        GBF_CUDA(cudaFuncSetAttribute(trsv_leaf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LEAF_SMEM));
        return 0;
      }))
    return rc;
  const long sblk = (long)ceil_div(n, 32) * 32 * 32;
  trsv_leaf_kernel<<<dim3(ceil_div(nrhs, LEAF_NC), ne), LEAF_THREADS, LEAF_SMEM, st>>>(kind, n, nrhs, b0, nb, S,
                                                                                       Dinv, sblk, Y);
  GBF_LAUNCHED();
  GBF_CUDA(cudaGetLastError());
  return 0;
}

// C[e] -= op(A[e]) Y[e] for all nodes e with the any-k 3xTF32 GEMM (FP32
// factors), nodes grouped so that each group's TF32 planes fit the workspace.
// op(A) is the block of op(S) at complex row ar and column ac; when the
// factors were split into TF32 planes once (g_tc->fpre_*), they are read
// from there and only Y is split.
static int tf32_update(cudaStream_t st, char opa, int m, int k, int nrhs, const cf *A, long lda, long sa,
                       const cf *Y, long ldy, long sy, cf *C, long ldc, long sc, int ne, int n, int ar, int ac) {
  const float *pre = (opa == 'N') ? g_tc->fpre_n : g_tc->fpre_c;
  if (pre && g_tc->fpre_ne >= ne && ac % 32 == 0) {
    const size_t per = cgemm_tf32k_pre_work(nrhs, k, 1);
    const int g = (int)std::max<size_t>(1, std::min<size_t>(ne, g_tc->kbytes / std::max<size_t>(per, 1)));
    for (int e0 = 0; e0 < ne; e0 += g) {
      const int gb = std::min(g, ne - e0);
      const int rc = cgemm_tf32k_pre(st, m, nrhs, k, -1.0, pre, n, g_tc->fpre_ne, e0, ar, ac / 32, Y + (long)e0 * sy,
                                     ldy, sy, 1, C + (long)e0 * sc, ldc, sc, gb, g_tc->kwork, g_tc->kbytes, g_tc->gerr);
      if (rc) return rc;
    }
    return 0;
  }
  const size_t per = cgemm_tf32k_work(m, nrhs, k, 1);
  const int g = (int)std::max<size_t>(1, std::min<size_t>(ne, g_tc->kbytes / std::max<size_t>(per, 1)));
  for (int e0 = 0; e0 < ne; e0 += g) {
    const int gb = std::min(g, ne - e0);
    const int rc = cgemm_tf32k(st, opa, 'N', m, nrhs, k, -1.0, A + (long)e0 * sa, lda, sa, Y + (long)e0 * sy, ldy, sy,
                               1, C + (long)e0 * sc, ldc, sc, gb, g_tc->kwork, g_tc->kbytes, g_tc->gerr);
    if (rc) return rc;
  }
  return 0;
}

// C = alpha op(A) Y (+ C when beta_one) for a group of gb nodes with the any-k
// sliced GEMM; A's slices come from the factorisation's slice cache when
// there is one (sliced on first use, kept until the factors change), else
// A is sliced into the workspace with Y.  Same slices either way, so the
// same results.
static int sliced_gemm_cached(cudaStream_t st, char opa, int m, int nrhs, int k, double alpha, const zd *A, long lda,
                              long sa, const zd *Y, long ldy, long sy, int beta_one, zd *C, long ldc, long sc,
                              int gb) {
  SliceCache *cache = g_tc->acache;
  if (cache) {
    const SliceKey key{A, lda, sa, m, k, gb, opa};
    SlicedOp a;
    bool have = false;
    const auto it = cache->ops.find(key);
    if (it != cache->ops.end()) {
      a = it->second;
      have = true;
    } else {
      const size_t bytes = (sliced_op_bytes(2L * m, sliced_kp(k, true), gb) + 255) & ~(size_t)255;
      if (cache->used + bytes <= cache->cap) {
        if (int rc = slice_rows<zd>(st, opa, m, k, A, lda, sa, gb, cache->base + cache->used, &a)) return rc;
        cache->used += bytes;
        cache->ops.emplace(key, a);
        have = true;
      }
    }
    if (have) {
      SlicedOp b;
      if (int rc = slice_cols<zd>(st, 'N', k, nrhs, Y, ldy, sy, gb, g_tc->kwork, &b)) return rc;
      return gemm_sliced_ops<zd>(st, a, b, gb, alpha, beta_one, C, ldc, sc, g_tc->gerr);
    }
  }
  return gemm_sliced_k<zd>(st, opa, 'N', m, nrhs, k, alpha, A, lda, sa, Y, ldy, sy, beta_one, C, ldc, sc, gb,
                           g_tc->kwork, g_tc->kbytes, g_tc->gerr);
}

// C[e] -= op(A[e]) Y[e] for all nodes e with the any-k sliced GEMM, nodes
// grouped so that each group's slices fit the workspace.
template <class T>
static int sliced_update(cudaStream_t st, char opa, int m, int k, int nrhs, const T *A, long lda, long sa,
                         const T *Y, long ldy, long sy, T *C, long ldc, long sc, int ne) {
  const size_t per = gemm_sliced_k_work(true, m, nrhs, k, 1);
  const int g = (int)std::max<size_t>(1, std::min<size_t>(ne, g_tc->kbytes / std::max<size_t>(per, 1)));
  for (int e0 = 0; e0 < ne; e0 += g) {
    const int gb = std::min(g, ne - e0);
    int rc;
    if constexpr (std::is_same<T, zd>::value)
      rc = sliced_gemm_cached(st, opa, m, nrhs, k, -1.0, A + (long)e0 * sa, lda, sa, Y + (long)e0 * sy, ldy, sy, 1,
                              C + (long)e0 * sc, ldc, sc, gb);
    else
      rc = gemm_sliced_k<T>(st, opa, 'N', m, nrhs, k, -1.0, A + (long)e0 * sa, lda, sa, Y + (long)e0 * sy, ldy, sy,
                            1, C + (long)e0 * sc, ldc, sc, gb, g_tc->kwork, g_tc->kbytes, g_tc->gerr);
    if (rc) return rc;
  }
  return 0;
}

// Recursive triangular solves (FP64 factors on the tensor-core engine): the
// block range [b0, b1) splits in halves; the off-diagonal update between
// them is one any-k GEMM (K up to n/2), the leaves multiply by the inverted
// diagonal blocks.  Same operations as the blocked sweep, regrouped so that
// almost all the work sits in a few large-K products.
//   kind 0: L (unit lower), forward      kind 1: U (upper), backward
//   kind 2: U^H (lower), forward         kind 3: L^H (unit upper), backward
template <class T>
static int trsv_rec(cudaStream_t st, int kind, int n, int ne, int nrhs, const T *S, const T *Dinv, int bs, T *Y,
                    int b0, int b1) {
  using X = tr<T>;
  const long nn = (long)n * n, ny = (long)n * nrhs, sblk = (long)ceil_div(n, bs) * bs * bs;
  const T one = X::one(), zero = X::zero(), m1 = X::sub(X::zero(), X::one());
  if constexpr (std::is_same<T, cf>::value) {
    if (b1 - b0 <= 4 && bs == 32 && g_tc && g_tc->kwork) return trsv_leaf(st, kind, n, ne, nrhs, S, Dinv, Y, b0, b1 - b0);
  }
  if (b1 - b0 == 1) {
    const int r0 = b0 * bs, bsz = std::min(bs, n - r0);
    return gemm<T>(st, kind >= 2 ? 'C' : 'N', 'N', bsz, nrhs, bsz, one, Dinv + (long)b0 * bs * bs, bs, sblk,
                   Y + r0, n, ny, zero, Y + r0, n, ny, ne);
  }
  if constexpr (std::is_same<T, zd>::value) {
    if (b1 - b0 == 4 && bs == 32 && b0 % 4 == 0 && n % 128 == 0 && g_tc && g_tc->dinv_l) {
      // a 128-row leaf: one product with the inverted 128 x 128 diagonal block
      const T *D = (const T *)((kind == 0 || kind == 3) ? g_tc->dinv_l : g_tc->dinv_u);
      const long nb128 = n / 128;
      return sliced_gemm_cached(st, kind >= 2 ? 'C' : 'N', 128, nrhs, 128, 1.0, D + (long)(b0 / 4) * 128 * 128, 128,
                                nb128 * 128 * 128, Y + (long)b0 * bs, n, ny, 0, Y + (long)b0 * bs, n, ny, ne);
    }
  }
  const int mid = b0 + (b1 - b0) / 2;
  const int r0 = b0 * bs, rm = mid * bs, r1 = std::min(n, b1 * bs);
  const bool forward = (kind == 0 || kind == 2);
  int rc;
  if ((rc = trsv_rec<T>(st, kind, n, ne, nrhs, S, Dinv, bs, Y, forward ? b0 : mid, forward ? mid : b1))) return rc;
  // the update: rows of the second half from the solved first half
  const T *A;
  char op;
  int m, k, rdst, rsrc;
  switch (kind) {
    case 0: A = S + rm + (long)r0 * n; op = 'N'; m = r1 - rm; k = rm - r0; rdst = rm; rsrc = r0; break;
    case 1: A = S + r0 + (long)rm * n; op = 'N'; m = rm - r0; k = r1 - rm; rdst = r0; rsrc = rm; break;
    case 2: A = S + r0 + (long)rm * n; op = 'C'; m = r1 - rm; k = rm - r0; rdst = rm; rsrc = r0; break;
    default: A = S + rm + (long)r0 * n; op = 'C'; m = rm - r0; k = r1 - rm; rdst = r0; rsrc = rm; break;
  }
  // op(A) is the block of op(S) at complex row rdst, column rsrc
  bool done = false;
  if constexpr (std::is_same<T, zd>::value) {
    if (k > 32 && g_tc && g_tc->kwork) {  // FP64 factors on the tensor-core engine
      rc = sliced_update<T>(st, op, m, k, nrhs, A, n, nn, Y + rsrc, n, ny, Y + rdst, n, ny, ne);
      done = true;
    }
  }
  if constexpr (std::is_same<T, cf>::value) {
    if (k > 32 && g_tc && g_tc->kwork) {  // FP32 factors: 3xTF32 on the tensor cores
      rc = tf32_update(st, op, m, k, nrhs, A, n, nn, Y + rsrc, n, ny, Y + rdst, n, ny, ne, n, rdst, rsrc);
      done = true;
    }
  }
  if (!done) rc = gemm<T>(st, op, 'N', m, nrhs, k, m1, A, n, nn, Y + rsrc, n, ny, one, Y + rdst, n, ny, ne);
  if (rc) return rc;
  return trsv_rec<T>(st, kind, n, ne, nrhs, S, Dinv, bs, Y, forward ? mid : b0, forward ? b1 : mid);
}

template <class T>
int getrs_inplace(cudaStream_t st, int trans, int n, int ne, int nrhs, const T *S, const T *Linv,
                  const T *Uinv, int bs, T *Y, T *) {
  using X = tr<T>;
  CatScope cat_solve(CAT_SOLVE);
  const long nn = (long)n * n, ny = (long)n * nrhs;
  const int nblk = ceil_div(n, bs);
  const long sblk = (long)nblk * bs * bs;
  const T one = X::one();
  const T m1 = X::sub(X::zero(), X::one());
  const T zero = X::zero();
  int rc;
  // factors on the tensor-core engine (FP64: sliced; FP32: 3xTF32):
  // recursive (large-K products); otherwise the blocked chain, which suits
  // the CUDA-core GEMM better
  if constexpr (std::is_same<T, zd>::value || std::is_same<T, cf>::value) {
    if (g_tc && g_tc->kwork) {
      if (!trans) {
        if ((rc = trsv_rec<T>(st, 0, n, ne, nrhs, S, Linv, bs, Y, 0, nblk))) return rc;
        return trsv_rec<T>(st, 1, n, ne, nrhs, S, Uinv, bs, Y, 0, nblk);
      }
      if ((rc = trsv_rec<T>(st, 2, n, ne, nrhs, S, Uinv, bs, Y, 0, nblk))) return rc;
      return trsv_rec<T>(st, 3, n, ne, nrhs, S, Linv, bs, Y, 0, nblk);
    }
  }
  auto blk = [&](int b) { return std::min(bs, n - b * bs); };
  if (!trans) {
    // L (unit lower): Y_b <- Linv_b Y_b ; Y_below -= L_{below,b} Y_b
    for (int b = 0; b < nblk; ++b) {
      const int r0 = b * bs, bsz = blk(b);
      if ((rc = gemm<T>(st, 'N', 'N', bsz, nrhs, bsz, one, Linv + (long)b * bs * bs, bs, sblk, Y + r0, n, ny,
                        zero, Y + r0, n, ny, ne)))
        return rc;
      const int below = n - r0 - bsz;
      if (below > 0 &&
          (rc = gemm<T>(st, 'N', 'N', below, nrhs, bsz, m1, S + (r0 + bsz) + (long)r0 * n, n, nn, Y + r0, n, ny,
                        one, Y + r0 + bsz, n, ny, ne)))
        return rc;
    }
    // U (upper): backward
    for (int b = nblk - 1; b >= 0; --b) {
      const int r0 = b * bs, bsz = blk(b);
      if ((rc = gemm<T>(st, 'N', 'N', bsz, nrhs, bsz, one, Uinv + (long)b * bs * bs, bs, sblk, Y + r0, n, ny,
                        zero, Y + r0, n, ny, ne)))
        return rc;
      if (r0 > 0 && (rc = gemm<T>(st, 'N', 'N', r0, nrhs, bsz, m1, S + (long)r0 * n, n, nn, Y + r0, n, ny, one,
                                  Y, n, ny, ne)))
        return rc;
    }
  } else {
    // U^H (lower): forward
    for (int b = 0; b < nblk; ++b) {
      const int r0 = b * bs, bsz = blk(b);
      if ((rc = gemm<T>(st, 'C', 'N', bsz, nrhs, bsz, one, Uinv + (long)b * bs * bs, bs, sblk, Y + r0, n, ny,
                        zero, Y + r0, n, ny, ne)))
        return rc;
      const int below = n - r0 - bsz;
      if (below > 0 &&
          (rc = gemm<T>(st, 'C', 'N', below, nrhs, bsz, m1, S + r0 + (long)(r0 + bsz) * n, n, nn, Y + r0, n, ny,
                        one, Y + r0 + bsz, n, ny, ne)))
        return rc;
    }
    // L^H (unit upper): backward
    for (int b = nblk - 1; b >= 0; --b) {
      const int r0 = b * bs, bsz = blk(b);
      if ((rc = gemm<T>(st, 'C', 'N', bsz, nrhs, bsz, one, Linv + (long)b * bs * bs, bs, sblk, Y + r0, n, ny,
                        zero, Y + r0, n, ny, ne)))
        return rc;
      if (r0 > 0 && (rc = gemm<T>(st, 'C', 'N', r0, nrhs, bsz, m1, S + r0, n, nn, Y + r0, n, ny, one, Y, n, ny,
                                  ne)))
        return rc;
    }
  }
  return 0;
}

// ---------------------------------------------------------- gather/scatter --
template <class T>
__global__ void gather_rhs_kernel(int n, int nrhs, const int *__restrict__ perm, int kindR, const void *RHS,
                                  long ldr, const zd *__restrict__ scale, T *__restrict__ Y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y, e = blockIdx.z;
  if (i >= n) return;
  const int src = perm ? perm[(long)e * n + i] : i;
  zd v;
  if (kindR == 0)
    v = zd{((const double *)RHS)[src + (long)j * ldr], 0.0};
  else
    v = ((const zd *)RHS)[src + (long)j * ldr];
  if (scale) v = zmul(v, scale[(long)e * nrhs + j]);
  Y[(long)e * n * nrhs + i + (long)j * n] = cvt<T, zd>(v);
}

template <class T>
int gather_rhs(cudaStream_t st, int n, int ne, int nrhs, const int *perm, int kindR, const void *RHS, long ldr,
               const zd *scale, T *Y) {
  dim3 g(ceil_div(n, 256), nrhs, ne);
  gather_rhs_kernel<T><<<g, 256, 0, st>>>(n, nrhs, perm, kindR, RHS, ldr, scale, Y);
  GBF_LAUNCHED();
  GBF_CUDA(cudaGetLastError());
  return 0;
}

template <class T>
__global__ void scatter_perm_kernel(int n, int nrhs, const int *__restrict__ perm, const T *__restrict__ Yin,
                                    T *__restrict__ Yout) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y, e = blockIdx.z;
  if (i >= n) return;
  const long base = (long)e * n * nrhs + (long)j * n;
  Yout[base + perm[(long)e * n + i]] = Yin[base + i];
}

template <class T>
int scatter_perm(cudaStream_t st, int n, int ne, int nrhs, const int *perm, const T *Yin, T *Yout) {
  dim3 g(ceil_div(n, 256), nrhs, ne);
  scatter_perm_kernel<T><<<g, 256, 0, st>>>(n, nrhs, perm, Yin, Yout);
  GBF_LAUNCHED();
  GBF_CUDA(cudaGetLastError());
  return 0;
}

#define GBF_INST(T)                                                                                        \
  template int form_shift<T>(cudaStream_t, int, int, const zd *, int, char, const void *, long, const void *, \
                             long, T *, int *);                                                            \
  template int getrf_batched<T>(cudaStream_t, int, int, T *, int *, int *, T *, T *, int, int *, T *);       \
  template int getrs_inplace<T>(cudaStream_t, int, int, int, int, const T *, const T *, const T *, int, T *,  \
                                T *);                                                                      \
  template int gather_rhs<T>(cudaStream_t, int, int, int, const int *, int, const void *, long, const zd *,  \
                             T *);                                                                         \
  template int scatter_perm<T>(cudaStream_t, int, int, int, const int *, const T *, T *);
GBF_INST(zd)
GBF_INST(cf)

}  // namespace gbf
