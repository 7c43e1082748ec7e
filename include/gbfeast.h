/*
 * gbfeast -- FEAST's spectral projection + Rayleigh-Ritz subspace iteration
 * (Hermitian family, dense storage) on one NVIDIA GB300 GPU (sm_103a).
 *
 * Problem (FEAST v3.0 user guide, arXiv:1203.4031, "The FEAST Algorithm"):
 * find all eigenpairs of A x = lambda B x (A Hermitian / real symmetric, B
 * Hermitian positive definite, or B = I) with lambda in [Emin, Emax], using
 * a search subspace of size M0 and Ne = fpm(2) quadrature nodes on the upper
 * half of a contour through Emin and Emax.
 *
 * Conventions shared by every entry point
 *  - Matrices are column-major (the guide's dense format, "Matrix storage");
 *    lda >= n.  uplo: 'F' full, 'L' lower, 'U' upper triangle referenced.
 *  - Complex arrays are interleaved (re, im) doubles: C99 double _Complex,
 *    numpy complex128.  Pointers named d* are DEVICE pointers (cudaMalloc'ed
 *    or torch CUDA tensors); all others are host pointers.
 *  - fpm is the 64-entry parameter array of Table "tab_fpm"; C index i-1
 *    holds fpm(i).  gbf_init writes the defaults.  Extensions in the unused
 *    range fpm(40..63):
 *        fpm(42) arithmetic of the factorisation and solves:
 *                0 = complex FP64 (default),
 *                1 = complex FP32 with FP64 correction: every FEAST iteration
 *                    after the first solves only for the FP64 eigen-residual
 *                    R = A X - B X Lambda (see gbf_dsygv), so the subspace
 *                    reaches FP64 accuracy.
 *        fpm(43) LU panel width / diagonal block size (0 = default 32).
 *        fpm(44) engine of the complex GEMMs of the factorisation and the
 *                solves: 0 = tensor cores (default; FP64 factors: exact
 *                bf16 digit products, 7 digits; FP32 factors (fpm(42)=1):
 *                3xTF32 products; see gbf_zgemm_sliced S = 7 and S = 1),
 *                1 = CUDA-core FMA.
 *  - Outputs follow Table "tab_common": E[M0] eigenvalues (first M inside the
 *    interval, ascending, then the remaining Ritz values ascending), X (N x
 *    M0, ld N) B-orthonormal Ritz vectors in the same order, res[M0] relative
 *    residuals ||A x_i - lambda_i B x_i||_1 / ||alpha B x_i||_1 with alpha =
 *    max(|Emin|, |Emax|), M the count inside, loop the number of refinement
 *    loops, epsout = |trace_k - trace_{k-1}| / alpha (1 at loop 0).  On exit
 *    M0 holds the subspace size kept after B-orthonormalisation (the "new
 *    suitable M0"); entries past it are zero.
 *  - Return value == *info, codes of Table "tab_info": 202 bad N, 201 bad M0,
 *    200 Emin >= Emax, 100+i bad fpm(i), 5 stochastic count returned
 *    (fpm(14)=2), 4 subspace returned (fpm(14)=1),
 *    3 M0 too small (every Ritz value inside and M0 < N), 2 no convergence
 *    within fpm(4) loops, 1 no eigenvalue in the interval, 0 success,
 *    -1 allocation failure, -2 inner solver failure (zero pivot or
 *    non-finite values), -3 reduced eigensolver failure (B not positive
 *    definite on the subspace), -(100+i) bad argument i.  Extension: -4 CUDA
 *    error; text through gbf_last_error().
 *  - Initial subspace when fpm(5)=0: entries uniform in [-1, 1) from the
 *    counter-based SplitMix64 generator (Steele, Lea & Flood 2014) with seed
 *    0x3C6EF372FE94F82B, value i (column-major linear index; complex: real
 *    part 2i, imaginary part 2i+1).
 *  - Stochastic eigenvalue count, fpm(14)=2 (guide section "Stochastic
 *    estimate"): one contour filters M0 probe vectors Y into Q = f(B^-1 A) Y
 *    and returns res[j] = mean over probes 0..j of Re(y^H q) (an unbiased
 *    estimate of trace f, the eigenvalue count of the interval), M = res[M0-1]
 *    rounded to nearest within [0, N], E = 0, X = the probes, loop 0, info 5.
 *    Probes: X on entry when fpm(5)=1, else +1/-1 by the top bit of the same
 *    SplitMix64 value i (column-major index; complex: real probes).  A few
 *    nodes (fpm(2) ~ 3) and fpm(42)=1 suffice for the estimate.
 *  - Memory: the library owns its workspace (stored factorisations for all
 *    nodes, as fpm(10)=1 in the guide, subspace blocks, reduced matrices);
 *    it lives in the handle and is reused across calls.  Inputs are read
 *    only; nothing the caller owns is overwritten except the outputs.
 *  - Threading: one call at a time per handle.
 */
#ifndef GBFEAST_H
#define GBFEAST_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gbf_context *gbf_handle;

/* Library version (major*10000 + minor*100 + patch). */
int gbf_version(void);

/* Text of the last error (CUDA failure or argument problem); never NULL. */
const char *gbf_last_error(void);

/* Kernels launched by this library since load (monotone counter). */
long long gbf_launch_count(void);

/* Launch profiling.  gbf_profile(1) clears the records and starts timing
 * instrumented launches with CUDA events on their own stream (GEMMs, LU
 * panels, Jacobi sweeps), bucketed by category; gbf_profile(0) stops.
 * gbf_profile_read waits for the recorded events and returns, for category
 * cat (0 <= cat < gbf_profile_categories()), the number of timed launches,
 * their summed device time in ms and their algorithmic flops (complex
 * multiply-add = 8 flops, real = 2).  Names: gbf_profile_name(cat). */
int gbf_profile(int enable);
int gbf_profile_categories(void);
const char *gbf_profile_name(int cat);
int gbf_profile_read(int cat, long long *launches, double *ms, double *flops);
/* The sliced tensor-core GEMM kernels alone (all categories, slicing
 * excluded): timed launches, milliseconds, useful flops (as above) and the
 * bf16 tensor-core flops they issue (digit-pair products over the padded
 * tiles).  Returns 0 or -4. */
int gbf_profile_tc(long long *launches, double *ms, double *flops, double *tensor_flops);

/* Handle for the current CUDA device.  Returns 0, or -1 (allocation) / -4. */
int gbf_create(gbf_handle *h);
/* Releases the handle's device workspace. */
int gbf_destroy(gbf_handle h);

/* feastinit (Table tab_fpm defaults): fpm(2)=8, fpm(3)=12, fpm(4)=20,
 * fpm(6)=1, fpm(7)=5, fpm(8)=16, fpm(17)=1, fpm(18)=100, rest 0. */
void gbf_init(int *fpm);

/* Quadrature nodes and weights of the half contour (tool zfeast_contour,
 * "Defining a search contour").  Contour z(t) = r0 + R cos t + i rho R sin t,
 * t in (0, pi), r0 = (Emin+Emax)/2, R = (Emax-Emin)/2, rho = fpm18/100;
 * t_e = (pi/2)(1 - x_e) for Gauss-Legendre x_e, omega_e on [-1,1]
 * (fpm16 = 0) or the midpoint rule (fpm16 = 1, x_e equispaced, omega_e =
 * 2/ne); w_e = omega_e R (rho cos t_e + i sin t_e) / 2, so the projector is
 * (1/2) sum_e [w_e (z_e B - A)^{-1} + conj(w_e) (conj(z_e) B - A)^{-1}] B.
 * Nodes are ordered from the Emin side.  Zne, Wne: host, 2*ne doubles each.
 * Returns 0, 200 (Emin >= Emax), 102 (ne < 1), 116 (fpm16), 118 (fpm18). */
int gbf_contour(double emin, double emax, int ne, int fpm16, int fpm18, double *Zne, double *Wne);

/* Rational filter f(l) = sum_e Re[w_e / (z_e - l)] of that contour at the
 * m real points eig (tool dfeast_rational); f = 1 at the centre of a circle
 * and 1/2 at its ends.  Host arrays.  Returns as gbf_contour. */
int gbf_rational(double emin, double emax, int ne, int fpm16, int fpm18, const double *eig, int m, double *f);
/* Same with user nodes/weights (dfeast_rationalx). */
int gbf_rationalx(const double *Zne, const double *Wne, int ne, const double *eig, int m, double *f);

/* ---------------------------------------------------------------------
 * Dense drivers, HOST pointers (Tfeast_YFgv / Tfeast_YFev of the guide,
 * "FEAST predefined interfaces").  The library copies A (and B) to the
 * device, runs the device driver below and copies E, X, res back.
 *   d: real symmetric A, B (double); z: complex Hermitian (interleaved).
 *   *ev: standard problem (B = I).  X (N x M0) is read when fpm(5)=1.
 * ------------------------------------------------------------------- */
int gbf_dsyev(char uplo, int n, const double *A, int lda, int *fpm, double *epsout, int *loop, double emin,
              double emax, int *M0, double *E, double *X, int *M, double *res, int *info);
int gbf_dsygv(char uplo, int n, const double *A, int lda, const double *B, int ldb, int *fpm, double *epsout,
              int *loop, double emin, double emax, int *M0, double *E, double *X, int *M, double *res,
              int *info);
int gbf_zheev(char uplo, int n, const double *A, int lda, int *fpm, double *epsout, int *loop, double emin,
              double emax, int *M0, double *E, double *X, int *M, double *res, int *info);
int gbf_zhegv(char uplo, int n, const double *A, int lda, const double *B, int ldb, int *fpm, double *epsout,
              int *loop, double emin, double emax, int *M0, double *E, double *X, int *M, double *res,
              int *info);
/* Expert variants ("...x"): user quadrature Zne, Wne (host, 2*fpm(2)
 * doubles each) replace the contour of fpm(2)/fpm(16)/fpm(18). */
int gbf_dsygvx(char uplo, int n, const double *A, int lda, const double *B, int ldb, int *fpm, double *epsout,
               int *loop, double emin, double emax, int *M0, double *E, double *X, int *M, double *res,
               int *info, const double *Zne, const double *Wne);
int gbf_zhegvx(char uplo, int n, const double *A, int lda, const double *B, int ldb, int *fpm, double *epsout,
               int *loop, double emin, double emax, int *M0, double *E, double *X, int *M, double *res,
               int *info, const double *Zne, const double *Wne);

/* ---------------------------------------------------------------------
 * Dense drivers, DEVICE pointers, on the caller's stream (cudaStream_t
 * passed as void*, NULL = legacy default stream).  dA, dB (NULL: B = I)
 * stay device-resident; dE[M0], dX (N x M0, ld N), dres[M0] are device
 * outputs; dX is read first when fpm(5)=1.  Scalars (epsout, loop, M0, M,
 * info) are host pointers.  The call returns after the stream has
 * finished the solve (the host reads a few scalars per iteration to steer
 * the loop).  Zne/Wne: host, NULL for the contour from fpm.
 * ------------------------------------------------------------------- */
int gbf_dsygv_dev(gbf_handle h, void *stream, char uplo, int n, const double *dA, int lda, const double *dB,
                  int ldb, int *fpm, double *epsout, int *loop, double emin, double emax, int *M0, double *dE,
                  double *dX, int *M, double *dres, int *info, const double *Zne, const double *Wne);
int gbf_zhegv_dev(gbf_handle h, void *stream, char uplo, int n, const double *dA, int lda, const double *dB,
                  int ldb, int *fpm, double *epsout, int *loop, double emin, double emax, int *M0, double *dE,
                  double *dX, int *M, double *dres, int *info, const double *Zne, const double *Wne);

/* ---------------------------------------------------------------------
 * Node sharding across processes (one GPU each): the guide's second level
 * of parallelism ("Using the FEAST-MPI version"; "Single search interval
 * and FEAST-MPI": the contour nodes of one interval are spread over the
 * ranks, each factors and solves only its own shifted systems, and the
 * filtered subspace is summed over the ranks once per iteration).
 *
 * Shard `rank` of `nranks` holds the nodes [rank*c, min(Ne, (rank+1)*c)),
 * c = ceil(Ne / nranks) (gbf_shard_nodes; a shard may hold none), keeps
 * only those factorisations, and solves only those systems.  The exchange
 * step is one all-gather per FEAST iteration of the node solution blocks
 * (and of the adjoint blocks for complex Hermitian problems), after which
 * every shard forms Q with the same node-ordered sum and runs the
 * Rayleigh-Ritz step itself (replicated, deterministic), so every shard
 * returns the same E, X, res, M, loop, bit for bit, and these equal what
 * the unsharded gbf_dsygv_dev / gbf_zhegv_dev return for the same inputs.
 *
 * The collective is the caller's (e.g. NCCL through torch.distributed):
 *  - allgather(user, stream, dbuf, chunk_bytes): dbuf is a device buffer
 *    of nranks chunks of chunk_bytes; on entry chunk `rank` holds this
 *    shard's blocks (written by work queued on `stream`); on return every
 *    chunk must hold its shard's blocks for all work queued on `stream`
 *    after the call.  Return 0, or nonzero to fail the solve with -4.
 *  - agree(user, code): host-side; *code holds this shard's status (0 or a
 *    negative info); on return it must hold the minimum over all shards.
 *    Called after the factorisation and once per iteration, so an error on
 *    any shard ends the solve on every shard at the same point.
 * All shards must call with the same arguments (A, B, fpm, interval, M0,
 * nodes); dA, dB are each shard's own copies.  nranks = 1 is the unsharded
 * solve.  Errors: -122 for a missing or inconsistent shard description;
 * otherwise those of gbf_dsygv_dev.
 * ------------------------------------------------------------------- */
typedef struct {
  int rank;    /* 0 <= rank < nranks */
  int nranks;  /* number of shards */
  int (*allgather)(void *user, void *stream, void *dbuf, size_t chunk_bytes);
  int (*agree)(void *user, int *code);
  void *user;  /* passed back to both callbacks */
} gbf_shard;

/* Nodes of shard `rank` of `nranks` for Ne = ne: *first, *count; returns the
 * chunk size c (node blocks per shard in the exchanged buffer), or
 * -101 / -102 / -103 for a bad ne / rank / nranks. */
int gbf_shard_nodes(int ne, int rank, int nranks, int *first, int *count);

int gbf_dsygv_dev_shard(gbf_handle h, void *stream, char uplo, int n, const double *dA, int lda, const double *dB,
                        int ldb, int *fpm, double *epsout, int *loop, double emin, double emax, int *M0, double *dE,
                        double *dX, int *M, double *dres, int *info, const double *Zne, const double *Wne,
                        const gbf_shard *sh);
int gbf_zhegv_dev_shard(gbf_handle h, void *stream, char uplo, int n, const double *dA, int lda, const double *dB,
                        int ldb, int *fpm, double *epsout, int *loop, double emin, double emax, int *M0, double *dE,
                        double *dX, int *M, double *dres, int *info, const double *Zne, const double *Wne,
                        const gbf_shard *sh);

/* ---------------------------------------------------------------------
 * Non-Hermitian FEAST (guide section "From v2.1 to v3.0": dual subspaces Q,
 * Q^ for the right and left eigenvectors; RCI cases 10/11/21/30/31/40/41 of
 * Table "tab_ijob"; outputs of Table "tab_common" for the general types).
 * Dense A (and B) of any structure, all eigenvalues inside an ellipse of
 * centre Emid = (emid_re, emid_im), horizontal semi-axis r,
 * vertical/horizontal ratio fpm(18)/100, rotated by fpm(19) degrees.
 * ------------------------------------------------------------------- */
/* Full-contour nodes and weights (the guide's gcontour tool): fpm(8) = ne
 * points, fpm(17) = 0 Gauss, 1 trapezoidal in the angle t of z(t) = Emid +
 * r e^{i phi} (cos t + i rho sin t); f(lambda) = sum_e w_e / (z_e - lambda)
 * approximates 1 inside and 0 outside.  Gauss: t_e = pi (1 + x_e) (x the
 * ascending Legendre points, omega their weights); trapezoidal: t_e =
 * 2 pi (e + 1/2) / ne, omega_e = 2 / ne; w_e = (omega_e / 2) r e^{i phi}
 * (rho cos t_e + i sin t_e).  Zne, Wne: ne complex (host).  Returns 0, 200
 * (r <= 0), 108, 117, 118 or 119 (bad fpm(8), fpm(17), fpm(18), fpm(19)). */
int gbf_gcontour(double emid_re, double emid_im, double r, int ne, int fpm17, int fpm18, int fpm19, double *Zne,
                 double *Wne);
/* f(eig_i) = sum_e Wne_e / (Zne_e - eig_i) for m complex eig (host; f complex). */
int gbf_grationalx(const double *Zne, const double *Wne, int ne, const double *eig, int m, double *f);

/* Solve A x = lambda B x (dB NULL: the standard problem, the guide's
 * [dz]feast_geev; otherwise [dz]feast_gegv), A, B general dense: real
 * (gbf_dgegv_dev, dA/dB doubles) or complex (gbf_zgegv_dev).  Device
 * pointers; the work runs on `stream` and the call returns after it.
 *  - fpm: fpm(8) nodes (default 16), fpm(17) rule (default 1, trapezoidal),
 *    fpm(18), fpm(19) the ellipse; fpm(3), fpm(4), fpm(5), fpm(6), fpm(14) =
 *    0/1 and fpm(43), fpm(44) as above.  fpm(42) = 0: complex FP64 factors;
 *    1: complex FP32 factors, and from the second loop on the solves take
 *    only the FP64 eigen-residuals R = A X - B X Lambda (right) and A^H X^ -
 *    B^H X^ conj(Lambda) (left), as for the Hermitian drivers, so the
 *    results reach FP64 accuracy.  For real A, B, a real Emid, fpm(19) = 0 and an even
 *    fpm(8), the nodes pair up as z and conj(z) and only fpm(8)/2 systems are
 *    factored (the guide's remark on real non-symmetric problems).
 *  - *M0 (1..min(n, 1024)): subspace size; on exit the size kept (each
 *    loop replaces Q and Q^ by orthonormal bases of their numerical ranges,
 *    dropping directions whose Gram eigenvalue is at most 1e-12 of the
 *    largest; entries past it are zero).  dE: M0 complex eigenvalues,
 *    the M inside first, each group ordered by ascending (Re, Im).  dX:
 *    complex n x 2 M0 (ld n): right eigenvectors in columns 0..M0-1 (unit
 *    2-norm), left ones in columns M0..2 M0-1, scaled so that the returned
 *    pairs are bi-orthonormal (X^^H B X = I).  dres: 2 M0 residuals,
 *    right ||A x - lambda B x||_1 / ||alpha B x||_1, then left
 *    ||A^H x^ - conj(lambda) B^H x^||_1 / ||alpha B^H x^||_1, alpha =
 *    |Emid| + r.  fpm(14) = 1: dX holds Q and Q^ after one contour, info 4.
 *  - Convergence: fpm(6) = 1 on the largest right or left residual of the
 *    pairs inside, fpm(6) = 0 on |trace_k - trace_{k-1}| / alpha (complex
 *    trace of the pairs inside).
 *  - info: 0, 1 (none inside), 2 (loops > fpm(4)), 3 (M0 too small), 4,
 *    6 (converged, but the returned pairs' bi-orthonormality defect
 *    max |X^^H B X - I| exceeds 1e-8), 200/201/202/1xx (bad arguments),
 *    -1 (device memory), -2 (zero pivot or non-finite input/results), -3
 *    (the reduced pencil is singular), -4 (CUDA error, bounded wait timed
 *    out, or the reduced QR did not converge). */
int gbf_dgegv_dev(gbf_handle h, void *stream, int n, const double *dA, int lda, const double *dB, int ldb, int *fpm,
                  double *epsout, int *loop, double emid_re, double emid_im, double r, int *M0, double *dE,
                  double *dX, int *M, double *dres, int *info, const double *Zne, const double *Wne);
int gbf_zgegv_dev(gbf_handle h, void *stream, int n, const double *dA, int lda, const double *dB, int ldb, int *fpm,
                  double *epsout, int *loop, double emid_re, double emid_im, double r, int *M0, double *dE,
                  double *dX, int *M, double *dres, int *info, const double *Zne, const double *Wne);
/* max |X^^H B X - I| over the pairs inside of the last converged
 * non-Hermitian solve on this handle (the quantity info 6 tests). */
double gbf_biorth_defect(gbf_handle h);
/* The same drivers on HOST arrays (the guide's predefined [dz]feast_geev /
 * [dz]feast_gegv, B NULL for the standard problem; with non-NULL Zne, Wne
 * the expert form with the caller's fpm(8) nodes and weights): A, B copied
 * to the device, solved with the library's default context for the current
 * device, E (M0 complex), X (complex n x 2 M0; read when fpm(5)=1) and res
 * (2 M0) copied back.  Same codes as the device-pointer drivers. */
int gbf_dgegv(int n, const double *A, int lda, const double *B, int ldb, int *fpm, double *epsout, int *loop,
              double emid_re, double emid_im, double r, int *M0, double *E, double *X, int *M, double *res, int *info,
              const double *Zne, const double *Wne);
int gbf_zgegv(int n, const double *A, int lda, const double *B, int ldb, int *fpm, double *epsout, int *loop,
              double emid_re, double emid_im, double r, int *M0, double *E, double *X, int *M, double *res, int *info,
              const double *Zne, const double *Wne);

/* ---------------------------------------------------------------------
 * Step-level entry points (device pointers) exposing single rows of the
 * hot path for verification and for callers that drive the iteration
 * themselves (the RCI pattern of Fig. "fig_rci").
 * ------------------------------------------------------------------- */
/* RCI case 10 for every node: form S_e = z_e B - A (dB NULL: B = I) and
 * factor P_e S_e = L_e U_e with partial pivoting (|re|+|im| pivot), kept in
 * the handle.  kind 0: dA/dB real double; 1: complex interleaved.  prec:
 * 0 complex FP64, 1 complex FP32.  Zne: host, 2*ne doubles.  Returns 0,
 * -2 when some S_e has a zero pivot, or an error code. */
int gbf_factor_dev(gbf_handle h, void *stream, int kind, int prec, char uplo, int n, const double *dA, int lda,
                   const double *dB, int ldb, int ne, const double *Zne);
/* RCI case 11 (trans 0) / case 21 (trans 1) with the stored factors:
 * dY_e = S_e^{-1} dRHS or S_e^{-H} dRHS for every node e.  dRHS: complex
 * n x nrhs (ld n); dY: complex ne x n x nrhs (node-major, ld n), FP64
 * interleaved whatever prec the factors were made in. */
int gbf_solve_dev(gbf_handle h, void *stream, int trans, int nrhs, const double *dRHS, double *dY);
/* Reduced dense eigensolver of the Rayleigh-Ritz step, the one the FEAST
 * loop runs: Householder tridiagonalisation in one thread-block cluster,
 * bisection for the eigenvalues, inverse iteration for the eigenvectors of
 * the tridiagonal matrix, back-transformation (cyclic Jacobi for m = 1, for
 * m above 1024 or when no cluster shape fits).  dA (m x m, ld m; real if
 * kind 0, complex interleaved if kind 1; full storage) may be overwritten;
 * dW[m] ascending eigenvalues; dV (m x m) orthonormal eigenvectors. */
int gbf_heev_dev(gbf_handle h, void *stream, int kind, int m, double *dA, double *dW, double *dV);

/* Tensor-core building block (tcgen05 + TMA + TMEM, sm_103a): dC (FP32,
 * column-major, ld ldc, batch stride sc) = dA dB^T per batch, dA
 * [batch][M][K] and dB [batch][N][K] bf16 row-major (K contiguous, K a
 * multiple of 8, 16-byte aligned bases).  dErr: one device int (scratch).
 * Returns 0, -4 (CUDA error), -5 (an in-kernel bounded wait timed out).
 * The guide has no counterpart: this is the contraction engine the sliced
 * FP64 and split-FP32 products are built on. */
int gbf_tc_gemm_bf16(void *stream, int M, int N, int K, int batch, const void *dA, const void *dB, float *dC,
                     long ldc, long sc, int *dErr);

/* Sliced GEMM for any k on the tensor cores (verification entry of the
 * engine behind the Rayleigh-Ritz projections A Q and B Q of the FP64
 * path): dC = alpha op(dA) op(dB) + beta dC on FP64 data, real (cplx 0) or
 * interleaved complex (cplx 1), op in 'N','T','C', op(A) m x k, op(B) k x n,
 * k >= 1, alpha = +1 or -1, beta 0 or 1, batches strided by sa, sb, sc
 * elements.  Each row of op(A) and column of op(B) is scaled by a power of
 * two and split into 8 base-2^7 digits (56 bits) held exactly in bf16; the
 * digit products of each 64-wide K chunk are summed exactly in FP32 tensor
 * memory and accumulated exactly in 64-bit integers across chunks; the FP64
 * entry is formed once.  dWork: gbf_gemm_sliced_work bytes; dErr: one
 * device int.  Returns 0, -4 (CUDA error / bad argument), -5 (an in-kernel
 * bounded wait timed out).  No counterpart in the guide. */
size_t gbf_gemm_sliced_work(int cplx, int m, int n, int k, int batch);
int gbf_gemm_sliced(void *stream, int cplx, char opa, char opb, int m, int n, int k, double alpha, const void *dA,
                    long lda, long sa, const void *dB, long ldb, long sb, int beta, void *dC, long ldc, long sc,
                    int batch, void *dWork, size_t work_bytes, int *dErr);

/* Sliced complex GEMM on the tensor cores (verification entry of the
 * engine behind the FP64 factorisation and solves): dC = alpha op(dA)
 * op(dB) + beta dC for interleaved complex data (prec 0: FP64, 1: FP32),
 * op in 'N','T','C', op(A) m x k, op(B) k x n with k <= 32, alpha = +1 or
 * -1, beta 0 or 1, S = 7 (FP64-class), 4 (28 bits) or 3 digits, or S = -3 (FP32 data:
 * every entry split into three bf16 parts, part products summed in FP32), or
 * S = 1 (prec 1 only, the FP32-factor engine: every entry split into two
 * TF32 parts hi + lo and each product formed as lo hi + hi lo + hi hi by
 * kind::tf32 MMAs into an FP32 accumulator, about 2^-22 relative), batches
 * strided by sa, sb, sc elements.  Every operand row of op(A) / column of
 * op(B) is scaled by a power of two and split into S base-2^7 integer
 * digits held exactly in bf16; digit products are summed exactly in FP32
 * tensor memory and recombined in FP64.  dWork: gbf_zgemm_sliced_work
 * bytes; dErr: one device int.  Returns 0, -4 (CUDA error / bad shape),
 * -5 (an in-kernel bounded wait timed out).  No counterpart in the guide. */
size_t gbf_zgemm_sliced_work(int m, int n, int batch, int S);
int gbf_zgemm_sliced(void *stream, int prec, int S, char opa, char opb, int m, int n, int k, double alpha,
                     const void *dA, long lda, long sa, const void *dB, long ldb, long sb, int beta, void *dC,
                     long ldc, long sc, int batch, void *dWork, size_t work_bytes, int *dErr);

/* 3xTF32 complex FP32 GEMM for any k on the tensor cores (verification entry
 * of the engine behind the FP32 factors' recursive solves in the mixed
 * path, fpm(42)=1): dC = alpha op(dA) op(dB) + beta dC for interleaved
 * complex FP32 data (numpy complex64), op in 'N','T','C', op(A) m x k,
 * op(B) k x n, k >= 1, alpha = +1 or -1, beta 0 or 1, batches strided by
 * sa, sb, sc elements.  Every FP32 value of the real embedding is split
 * into TF32 parts hi + lo and each product is formed as lo hi + hi lo +
 * hi hi by kind::tf32 MMAs into one FP32 accumulator over the whole K
 * (about 2^-22 relative per product).  dWork: gbf_cgemm_tf32_work bytes;
 * dErr: one device int.  Returns 0, -4 (CUDA error / bad argument), -5 (an
 * in-kernel bounded wait timed out).  No counterpart in the guide. */
size_t gbf_cgemm_tf32_work(int m, int n, int k, int batch);
int gbf_cgemm_tf32(void *stream, char opa, char opb, int m, int n, int k, double alpha, const void *dA, long lda,
                   long sa, const void *dB, long ldb, long sb, int beta, void *dC, long ldc, long sc, int batch,
                   void *dWork, size_t work_bytes, int *dErr);

/* gbf_zgemm_sliced without any device allocation, for callers that cannot
 * allocate device memory during the call: their device memory belongs to
 * another allocator (a framework's caching pool that holds the whole
 * budget), or they cannot afford the device-wide synchronisation that
 * cudaMalloc/cudaFree imply.  The guide has no counterpart.  Same operation, arguments and return codes
 * as gbf_zgemm_sliced, but the scratch (digit slices, scales, error word) is
 * a fixed 16 MiB device array inside the library, which every GPU that loads
 * the library keeps until the process exits.  Limits and rules:
 *  - a problem whose scratch (gbf_zgemm_sliced_work) exceeds
 *    gbf_zgemm_sliced_noalloc_max() bytes is rejected with -7 and a message
 *    in gbf_last_error(); nothing is launched;
 *  - the first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current;
 *  - every call shares the one array and it keeps the last call's contents
 *    (the call clears what must start at zero): calls whose work overlaps on
 *    the GPU (other streams, other threads) race and must not be issued;
 *  - the call reads the error word back and synchronises `stream` before
 *    it returns, so it returns after its stream has finished the work. */
/* Bounded-wait check (no counterpart in the guide): one thread waits on a
 * shared-memory barrier that nothing completes, with the same bounded loop
 * as the tensor-core engine's pipeline waits, for `limit` (>= 1) polls.
 * Returns -5 with a message in gbf_last_error() when the wait runs out (as
 * every entry above reports an in-kernel time-out), -101 for limit < 1, -4
 * on a CUDA error.  The device stays usable afterwards: the kernel returns
 * with nothing in flight.  For tests of the failure path. */
int gbf_wait_probe(void *stream, long limit);

size_t gbf_zgemm_sliced_noalloc_max(void);
int gbf_zgemm_sliced_noalloc(void *stream, int prec, int S, char opa, char opb, int m, int n, int k, double alpha,
                             const void *dA, long lda, long sa, const void *dB, long ldb, long sb, int beta, void *dC,
                             long ldc, long sc, int batch);

/* ---------------------------------------------------------------------
 * Independent problems: batches and the serving loop (the guide's first
 * level of parallelism -- separate search intervals / problems -- inside one
 * GPU; no counterpart API in the guide).  A problem names DEVICE buffers the
 * caller owns until its result is returned.  Each problem is solved exactly
 * as by gbf_dsygv_dev / gbf_zhegv_dev (kind 0 / 1) with its own fpm; results
 * are bitwise the same whether a problem runs alone or beside others.
 * ------------------------------------------------------------------- */
typedef struct {
  int kind;                /* 0: real symmetric (double), 1: complex Hermitian (interleaved) */
  char uplo;               /* 'F', 'L', 'U' */
  int n;
  const double *dA;        /* device, n x n, ld lda */
  int lda;
  const double *dB;        /* device, NULL for B = I */
  int ldb;
  double emin, emax;
  int m0;                  /* subspace size M0 */
  int fpm[64];             /* parameters (gbf_init defaults + changes) */
  double *dE, *dX, *dres;  /* device outputs: E[m0], X (n x m0, ld n), res[m0] */
  const double *Zne, *Wne; /* host expert quadrature (2*fpm(2) doubles) or NULL */
} gbf_problem;

typedef struct {
  int info, M, loop, m0;   /* as the dense drivers (m0 = kept subspace size) */
  double epsout;
  double queue_ms;         /* server: submit -> start; batch: 0 */
  double run_ms;           /* start -> result */
} gbf_result;

/* Device workspace one problem needs (bytes), the admission unit of the
 * server (caller-owned inputs and outputs are not included). */
size_t gbf_problem_bytes(const gbf_problem *p);

/* Solve nprob independent problems with nworkers concurrent workers (each a
 * handle + stream; largest problems first).  Work starts after the prior
 * work on `stream` and `stream` waits for all of it.  Returns 0 or the first
 * negative info among the results (every result is filled). */
int gbf_batch_solve(gbf_handle h, void *stream, int nprob, const gbf_problem *probs, gbf_result *outs,
                    int nworkers);

/* Serving loop: requests are admitted in arrival order when a worker is
 * free and their workspace (gbf_problem_bytes) fits in what is left of
 * hbm_budget_bytes; while one request runs, later ones are admitted as
 * workers and memory free up, so their work overlaps on the device.  A
 * request larger than the whole budget completes with info -1. */
typedef struct gbf_server_s *gbf_server;
int gbf_server_create(size_t hbm_budget_bytes, int nworkers, gbf_server *out);
/* Queues a copy of *p; the buffers it names must stay valid until done. */
int gbf_server_submit(gbf_server s, const gbf_problem *p, unsigned long long *ticket);
/* 0: done (*out filled, ticket released), 1: queued or running, -101: unknown. */
int gbf_server_poll(gbf_server s, unsigned long long ticket, gbf_result *out);
/* Blocks until done; then as gbf_server_poll returning 0. */
int gbf_server_wait(gbf_server s, unsigned long long ticket, gbf_result *out);
/* Current and peak admitted bytes, queued and running request counts. */
int gbf_server_stats(gbf_server s, size_t *in_use, size_t *peak, int *queued, int *running);
/* Finishes every queued request, then releases the workers. */
int gbf_server_destroy(gbf_server s);

#ifdef __cplusplus
}
#endif
#endif
