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
    if (i == j) {
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
// C CTAs of a thread-block cluster, each slice held in shared memory
// (column-major, R rows).  Per column: local argmax (warp shuffles), the C
// candidates read over distributed shared memory and reduced identically by
// every CTA (largest |re|+|im|, lowest row on ties), the pivot row and the
// displaced row read remotely, a cluster barrier, the swap written locally,
// then the local scale + rank-1 update.  Two cluster barriers per column.
template <class T>
__global__ void __launch_bounds__(PANEL_THREADS)
    lu_panel_cluster_kernel(int n, int k, int w, int R, T *S, int *ipiv, int *sing) {
  using X = tr<T>;
  using Rt = typename X::R;
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int q = (int)cl.block_rank();
  const int e = blockIdx.y;
  const long nn = (long)n * n;
  T *a = S + e * nn;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sl = reinterpret_cast<T *>(smem_raw);  // [w][R]
  T *urow = sl + (long)w * R;               // pivot row (old row p)
  T *xrow = urow + MAX_NB;                  // old row c (kept by the owner of p)
  long long *cval = reinterpret_cast<long long *>(xrow + MAX_NB);
  int *cidx = reinterpret_cast<int *>(cval + 2);
  __shared__ long long wv[32];
  __shared__ int wi[32];
  __shared__ T s_inv;
  __shared__ int s_p, s_ok;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int r0 = k + q * R;
  const int rows = max(0, min(R, n - r0));
  for (int t = tid; t < rows * w; t += blockDim.x) {
    const int rl = t % rows, jj = t / rows;
    sl[(long)jj * R + rl] = a[(r0 + rl) + (long)(k + jj) * n];
  }
  __syncthreads();
  for (int j = 0; j < w; ++j) {
    const int c = k + j;
    // 1. local candidate
    long long best = -1;
    int bidx = n;
    for (int rl = tid; rl < rows; rl += blockDim.x) {
      const int gr = r0 + rl;
      if (gr < c) continue;
      const long long v = pivkey(X::abs1(sl[(long)j * R + rl]));
      if (v > best) {
        best = v;
        bidx = gr;
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
      wv[warp] = best;
      wi[warp] = bidx;
    }
    __syncthreads();
    if (tid == 0) {
      long long b = -1;
      int bi = n;
      for (int w2 = 0; w2 < nwarps; ++w2)
        if (wv[w2] > b || (wv[w2] == b && wi[w2] < bi)) {
          b = wv[w2];
          bi = wi[w2];
        }
      cval[0] = b;
      cidx[0] = bi;
    }
    cl.sync();  // (A) candidates visible; previous column's updates complete
    // 2. cluster argmax (every CTA reduces the same list in the same order)
    if (warp == 0) {
      long long b = -1;
      int bi = n;
      if (lane < C) {
        b = *cl.map_shared_rank(cval, lane);
        bi = *cl.map_shared_rank(cidx, lane);
      }
      for (int off = 16; off > 0; off >>= 1) {
        const long long ov = __shfl_down_sync(0xffffffffu, b, off);
        const int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ov > b || (ov == b && oi < bi)) {
          b = ov;
          bi = oi;
        }
      }
      if (lane == 0) {
        const int ok = (b > 0) && (bi < n);
        s_ok = ok;
        s_p = ok ? bi : c;
      }
    }
    __syncthreads();
    const int p = s_p, ok = s_ok;
    const int qc = (c - k) / R, lc = (c - k) % R;
    const int qp = (p - k) / R, lp = (p - k) % R;
    // 3. remote reads of the old rows p and c
    if (ok && tid < w) {
      urow[tid] = cl.map_shared_rank(sl, qp)[(long)tid * R + lp];
      if (q == qp && p != c) xrow[tid] = cl.map_shared_rank(sl, qc)[(long)tid * R + lc];
    }
    cl.sync();  // (B) every read done before any write
    // 4. swap (local writes)
    if (ok && p != c && tid < w) {
      if (q == qc) sl[(long)tid * R + lc] = urow[tid];
      if (q == qp) sl[(long)tid * R + lp] = xrow[tid];
    }
    if (q == 0 && tid == 0) {
      ipiv[(long)e * n + c] = ok ? p : c;
      if (!ok && sing[e] == 0) sing[e] = c + 1;
    }
    // the pivot's reciprocal, formed once per CTA (a complex division is
    // several FP64 divisions; every thread forming it cost more than the
    // rank-1 update)
    if (tid == 32 && ok) s_inv = cinv<T>(urow[j]);
    __syncthreads();
    // 5. scale and rank-1 update of the local rows below c
    if (ok) {
      const T inv = s_inv;
      for (int rl = tid; rl < rows; rl += blockDim.x) {
        if (r0 + rl <= c) continue;
        const T l = X::mul(sl[(long)j * R + rl], inv);
        sl[(long)j * R + rl] = l;
        for (int jj = j + 1; jj < w; ++jj) sl[(long)jj * R + rl] = X::fma(l, X::neg(urow[jj]), sl[(long)jj * R + rl]);
      }
    }
    __syncthreads();
  }
  for (int t = tid; t < rows * w; t += blockDim.x) {
    const int rl = t % rows, jj = t / rows;
    a[(r0 + rl) + (long)(k + jj) * n] = sl[(long)jj * R + rl];
  }
  cl.sync();  // no CTA leaves while another may still read its slice
}

// Launch the cluster panel: C CTAs (power of two <= 16) so that each slice
// fits in shared memory.  Returns 1 when the caller should use the
// single-CTA panel instead (no suitable cluster shape).
template <class T>
static int launch_cluster_panel(cudaStream_t st, int n, int ne, int k, int w, T *S, int *ipiv, int *sing) {
  const int rowsp = n - k;
  const size_t cap = 200 * 1024;
  static std::atomic<unsigned long long> attr_done{0};
  once_per_device(attr_done, [&]() -> int {
    cudaFuncSetAttribute(lu_panel_cluster_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
    cudaFuncSetAttribute(lu_panel_cluster_kernel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaGetLastError();
    return 0;
  });
  int C0 = 1;
  while (C0 < 16 && C0 * 256 < rowsp) C0 *= 2;
  // largest C first (more SMs per panel), smaller clusters when the GPU
  // cannot co-schedule it; every candidate must fit the shared memory cap
  for (int C = C0; C >= 1; C /= 2) {
    const int R = ceil_div(rowsp, C);
    const size_t smem = (size_t)R * w * sizeof(T) + 2 * MAX_NB * sizeof(T) + 64;
    if (smem > cap) break;  // smaller C only makes the slice larger
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, ne, 1);
    cfg.blockDim = dim3(PANEL_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, lu_panel_cluster_kernel<T>, &cfg) != cudaSuccess ||
        nclusters < 1) {
      cudaGetLastError();
      continue;
    }
    if (cudaLaunchKernelEx(&cfg, lu_panel_cluster_kernel<T>, n, k, w, R, S, ipiv, sing) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    GBF_LAUNCHED();
    return 0;
  }
  return 1;
}

// --------------------------------------------------------- laswp + trsm --
// Columns outside the panel: apply the panel's row swaps; columns right of
// the panel additionally get U12 = L11^{-1} A12 (unit lower forward solve).
constexpr int SWAP_COLS = 64;

template <class T>
__global__ void __launch_bounds__(SWAP_COLS)
    laswp_trsm_kernel(int n, int k, int w, T *S, const int *ipiv) {
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
  auto panel = [&](cudaStream_t s, int k) {
    const int w = std::min(nb, n - k);
    CatScope cat_panel(CAT_LU_PANEL);
    const int slot = prof_begin(s);
    if (launch_cluster_panel<T>(s, n, ne, k, w, S, ipiv, sing)) {
      lu_panel_kernel<T><<<ne, PANEL_THREADS, 0, s>>>(n, k, w, S, ipiv, sing);
      GBF_LAUNCHED();
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
      const size_t sm = (size_t)w * w * sizeof(T) + (size_t)w * sizeof(int);
      static std::atomic<unsigned long long> attr_set{0};
      if (int rc = once_per_device(attr_set, [&]() -> int {
            GBF_CUDA(cudaFuncSetAttribute(laswp_trsm_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)(MAX_NB * MAX_NB * sizeof(T) + MAX_NB * sizeof(int))));
            return 0;
          }))
        return rc;
      laswp_trsm_kernel<T><<<g, SWAP_COLS, sm, st>>>(n, k, w, S, ipiv);
      GBF_LAUNCHED();
      prof_end(st, slot2, 0.0);
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
  const int nblk = ceil_div(n, bs);
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

size_t solve_kwork_bytes_cf(int n, int nrhs, int bs, int ne) {
  const int nblk = ceil_div(n, bs);
  const int half = std::min(n, (nblk - nblk / 2) * bs);
  return cgemm_tf32k_work(half, nrhs, half, std::min(ne, 8));
}

// C[e] -= op(A[e]) Y[e] for all nodes e with the any-k 3xTF32 GEMM (FP32
// factors), nodes grouped so that each group's TF32 planes fit the workspace.
static int tf32_update(cudaStream_t st, char opa, int m, int k, int nrhs, const cf *A, long lda, long sa,
                       const cf *Y, long ldy, long sy, cf *C, long ldc, long sc, int ne) {
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

// C[e] -= op(A[e]) Y[e] for all nodes e with the any-k sliced GEMM, nodes
// grouped so that each group's slices fit the workspace.
template <class T>
static int sliced_update(cudaStream_t st, char opa, int m, int k, int nrhs, const T *A, long lda, long sa,
                         const T *Y, long ldy, long sy, T *C, long ldc, long sc, int ne) {
  const size_t per = gemm_sliced_k_work(true, m, nrhs, k, 1);
  const int g = (int)std::max<size_t>(1, std::min<size_t>(ne, g_tc->kbytes / std::max<size_t>(per, 1)));
  for (int e0 = 0; e0 < ne; e0 += g) {
    const int gb = std::min(g, ne - e0);
    const int rc = gemm_sliced_k<T>(st, opa, 'N', m, nrhs, k, -1.0, A + (long)e0 * sa, lda, sa, Y + (long)e0 * sy,
                                    ldy, sy, 1, C + (long)e0 * sc, ldc, sc, gb, g_tc->kwork, g_tc->kbytes, g_tc->gerr);
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
      return gemm_sliced_k<T>(st, kind >= 2 ? 'C' : 'N', 'N', 128, nrhs, 128, 1.0, D + (long)(b0 / 4) * 128 * 128,
                              128, nb128 * 128 * 128, Y + (long)b0 * bs, n, ny, 0, Y + (long)b0 * bs, n, ny, ne,
                              g_tc->kwork, g_tc->kbytes, g_tc->gerr);
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
  bool done = false;
  if constexpr (std::is_same<T, zd>::value) {
    if (k > 32 && g_tc && g_tc->kwork) {  // FP64 factors on the tensor-core engine
      rc = sliced_update<T>(st, op, m, k, nrhs, A, n, nn, Y + rsrc, n, ny, Y + rdst, n, ny, ne);
      done = true;
    }
  }
  if constexpr (std::is_same<T, cf>::value) {
    if (k > 32 && g_tc && g_tc->kwork) {  // FP32 factors: 3xTF32 on the tensor cores
      rc = tf32_update(st, op, m, k, nrhs, A, n, nn, Y + rsrc, n, ny, Y + rdst, n, ny, ne);
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
