/*
 * Plain FP64 CPU FEAST oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
 * reference leg may load this library.  The CUDA product path never links,
 * includes or calls anything in oracle/, and the two share no code.
 *
 * Every routine follows the FEAST v3.0 user guide (Polizzi & Kestyn,
 * arXiv:1203.4031); each definition cites the section / table it restates.
 * Storage is column-major (Fortran order) as in the guide's dense format
 * ("Matrix storage" section); complex numbers are interleaved doubles
 * (C99 double complex).
 */
#ifndef FEAST_ORACLE_H
#define FEAST_ORACLE_H

#include <complex.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Gauss-Legendre nodes x[0..ne) (ascending) and weights w on [-1,1]. */
int ora_gauss_legendre(int ne, double *x, double *w);

/* Half-contour nodes/weights for [emin,emax] ("Defining a search contour",
 * tool zfeast_contour).  type 0 = Gauss-Legendre, 1 = trapezoidal;
 * ratio = fpm(18) (100 = circle).  Returns 0 or a negative error. */
int ora_contour(double emin, double emax, int ne, int type, int ratio,
                double complex *zne, double complex *wne);

/* Rational filter f(l) = sum_e Re[w_e / (z_e - l)] (tool dfeast_rationalx). */
void ora_rationalx(const double complex *zne, const double complex *wne,
                   int ne, const double *eig, int m, double *f);

/* Unblocked LU with partial pivoting (|re|+|im| pivot, lowest index on
 * ties).  ipiv is 0-based.  Returns 0 or k+1 for the first zero pivot. */
int ora_zgetrf(int n, double complex *a, int lda, int *ipiv);

/* Solve S X = B (trans=0) or S^H X = B (trans=1) with the factors above. */
void ora_zgetrs(int trans, int n, int nrhs, const double complex *a, int lda,
                const int *ipiv, double complex *b, int ldb);

/* Cyclic two-sided Jacobi for a Hermitian matrix (overwritten).  w ascending,
 * v unitary eigenvectors (column j <-> w[j]).  Returns number of sweeps or
 * -1 if it did not converge in the sweep cap. */
int ora_zheev_jacobi(int n, double complex *a, int lda, double *w,
                     double complex *v, int ldv);

/* Number of negative eigenvalues of a Hermitian matrix (Sylvester inertia via
 * Bunch-Kaufman LDL^H).  h is overwritten.  zero_out (may be NULL) receives
 * the number of exactly-zero pivots. */
long ora_inertia_neg(int n, double complex *h, int ldh, long *zero_out);

/* SplitMix64 (Steele, Lea & Flood 2014) as a counter-based generator:
 * value(i) = mix(seed + (i+1) * 0x9E3779B97F4A7C15). */
uint64_t ora_splitmix64(uint64_t seed, uint64_t i);

/* FEAST for the Hermitian family (kind 0: real symmetric, Q = sum Re(w_e G_e);
 * kind 1: complex Hermitian, adjoint solves).  A, B full n x n (B NULL =>
 * standard problem).  zne/wne NULL => contour from fpm.  X n x m0 (input
 * subspace when fpm[4] == 1).  Outputs E[m0], res[m0], X; scalars through
 * pointers.  *m0_out = subspace size kept after B-orthonormalisation.
 * Returns info (also stored in *info). */
int ora_feast(int kind, int n, const double complex *A, int lda,
              const double complex *B, int ldb, const int *fpm,
              double emin, double emax, int m0,
              const double complex *zne, const double complex *wne,
              double complex *X, double *E, double *res, int *M, int *loop,
              double *epsout, int *m0_out, int *info, int nthreads);

#ifdef __cplusplus
}
#endif
#endif
