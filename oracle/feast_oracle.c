/*
 * Plain FP64 CPU FEAST oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
 * reference leg may load this library.  The CUDA product path never links,
 * includes or calls it, and shares no code with it.
 *
 * What it computes (FEAST v3.0 user guide, Polizzi & Kestyn, arXiv:1203.4031):
 *   - the FEAST algorithm summary in "The FEAST Algorithm" section: a
 *     quadrature Q = sum_j w_j Q_j over independent shifted solves
 *     (z_j B - A) Q_j = Y along a complex contour, then a Rayleigh-Ritz step
 *     on the reduced dense problem, repeated as a subspace iteration;
 *   - the RCI loop of Fig. "fig_rci" (cases 10/11 factor and solve, 20/21
 *     the adjoint solve for complex Hermitian, 30/40 A*X and B*X);
 *   - the outputs of Table "tab_common" (epsout, loop, M0, E, X, M, res,
 *     info) and the info codes of Table "tab_info";
 *   - the fpm parameters and defaults of Table "tab_fpm".
 * The guide does not print the quadrature formula; this file derives it from
 * the residue theorem on a circle through Emin and Emax, with Gauss-Legendre
 * (or midpoint/trapezoidal) points in the angle (see ora_contour).
 *
 * Readings where the guide is silent (each listed in the design notes):
 *   - initial subspace when fpm(5)=0: SplitMix64 uniform [-1,1) entries;
 *   - B-orthonormalisation of Q: unit-diagonal scaling, Jacobi on the scaled
 *     Q^H B Q, drop directions with eigenvalue <= 1e-12 * max (the kept
 *     count is the "new suitable M0" of Table tab_common); a negative
 *     eigenvalue below -1e-8 * max means B is not positive definite (info -3);
 *   - output order: eigenpairs inside [Emin,Emax] ascending, then the others
 *     ascending (the hello-world output lists 1 then 3);
 *   - spurious Ritz pairs (Table tab_common's remark gives no criterion):
 *     from loop 1 on, a pair inside the interval whose filter gain
 *     1/||w_j||_2 on its pre-image in the previous B-orthonormal subspace is
 *     below f(lambda_j)/4 is spurious; it leaves M, the trace and the
 *     convergence test and goes to the end of E/X with res = -1;
 *   - info 1 as soon as no Ritz value is inside; info 3 when every one of the
 *     M0 requested Ritz values is inside and M0 < N;
 *   - epsout = 1 at loop 0 (the hello-world output prints 1.0 at loop 0);
 *   - stochastic estimate (fpm(14)=2): Rademacher probes (fpm(5)=0) or the
 *     input X as probes (fpm(5)=1); res(j) = running mean over probes 1..j,
 *     M = res(M0) rounded to nearest and clamped to [0, N], X = the probes.
 *
 * Arithmetic: C99 double complex, compiled with -fcx-limited-range (textbook
 * complex multiply/divide without the Annex G inf/NaN recovery).
 */
#include "feast_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex zc;
#define IX(i, j, ld) ((size_t)(i) + (size_t)(j) * (size_t)(ld))

static const double PI = 3.14159265358979323846264338327950288;

/* ------------------------------------------------------------------------ */
/* Gauss-Legendre nodes and weights on [-1, 1].                              */
/* Roots of the Legendre polynomial P_ne by Newton's method, using the       */
/* three-term recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1} and        */
/* P'_n(x) = n (x P_n - P_{n-1}) / (x^2 - 1); weight 2 / ((1-x^2) P'_n^2).   */
/* ------------------------------------------------------------------------ */
static void legendre_eval(int ne, double x, double *pn, double *dpn)
{
    double p_prev = 1.0, p = x;
    for (int k = 1; k < ne; ++k) {
        double p_next = ((2.0 * k + 1.0) * x * p - k * p_prev) / (k + 1.0);
        p_prev = p;
        p = p_next;
    }
    *pn = p;
    *dpn = ne * (x * p - p_prev) / (x * x - 1.0);
}

int ora_gauss_legendre(int ne, double *x, double *w)
{
    if (ne < 1) return -1;
    for (int i = 0; i < ne; ++i) {
        /* i-th largest root; classical starting guess */
        double t = cos(PI * (i + 0.75) / (ne + 0.5));
        for (int it = 0; it < 100; ++it) {
            double pn, dpn;
            legendre_eval(ne, t, &pn, &dpn);
            double dt = pn / dpn;
            t -= dt;
            if (fabs(dt) < 1e-16) break;
        }
        double pn, dpn;
        legendre_eval(ne, t, &pn, &dpn);
        x[ne - 1 - i] = t;
        w[ne - 1 - i] = 2.0 / ((1.0 - t * t) * dpn * dpn);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Half-contour quadrature ("Defining a search contour"; zfeast_contour).    */
/* Contour: z(theta) = r0 + R cos(theta) + i*rho*R sin(theta), theta in      */
/* (0, pi) for the upper half, r0 = (Emin+Emax)/2, R = (Emax-Emin)/2,         */
/* rho = fpm(18)/100.  theta = (pi/2)(1 - x) maps x in [-1,1] onto it.        */
/* (1/2 pi i) * integral over the upper half of g(z) dz                       */
/*   = (1/2 pi i) (pi/2) sum_e omega_e g(z_e) z'(theta_e)                      */
/*   = 1/2 sum_e w_e g(z_e),  w_e = (1/2) omega_e R (rho cos + i sin)(theta_e) */
/* and the lower half gives the conjugate terms, so for Hermitian problems   */
/* the projector is (1/2) sum_e [w_e G(z_e) + conj(w_e) G(conj z_e)].         */
/* type 0: Gauss-Legendre x_e, omega_e; type 1: midpoint rule in theta       */
/* (x_e equispaced, omega_e = 2/ne).  Node order: x ascending (Emin side).    */
/* ------------------------------------------------------------------------ */
int ora_contour(double emin, double emax, int ne, int type, int ratio,
                zc *zne, zc *wne)
{
    if (ne < 1 || !(emin < emax) || ratio <= 0) return -1;
    double *x = (double *)malloc(sizeof(double) * ne);
    double *om = (double *)malloc(sizeof(double) * ne);
    if (type == 0) {
        ora_gauss_legendre(ne, x, om);
    } else if (type == 1) {
        for (int e = 0; e < ne; ++e) {
            double theta = PI * (ne - e - 0.5) / ne;
            x[e] = 1.0 - 2.0 * theta / PI;
            om[e] = 2.0 / ne;
        }
    } else {
        free(x);
        free(om);
        return -2;
    }
    double r0 = 0.5 * (emin + emax), R = 0.5 * (emax - emin);
    double rho = ratio / 100.0;
    for (int e = 0; e < ne; ++e) {
        double theta = 0.5 * PI * (1.0 - x[e]);
        double c = cos(theta), s = sin(theta);
        zne[e] = (r0 + R * c) + I * (rho * R * s);
        wne[e] = 0.5 * om[e] * R * ((rho * c) + I * s);
    }
    free(x);
    free(om);
    return 0;
}

/* Rational (selection) function of the quadrature (dfeast_rationalx):        */
/* f(l) = (1/2) sum_e [w_e/(z_e - l) + conj(w_e)/(conj(z_e) - l)]             */
/*      = sum_e Re[w_e / (z_e - l)] for real l.                               */
void ora_rationalx(const zc *zne, const zc *wne, int ne, const double *eig,
                   int m, double *f)
{
    for (int i = 0; i < m; ++i) {
        double s = 0.0;
        for (int e = 0; e < ne; ++e) s += creal(wne[e] / (zne[e] - eig[i]));
        f[i] = s;
    }
}

/* ------------------------------------------------------------------------ */
/* Dense LU with partial pivoting (the dense driver's inner solver, RCI     */
/* case 10).  Right-looking, unblocked.                                      */
/* ------------------------------------------------------------------------ */
static double cabs1(zc z) { return fabs(creal(z)) + fabs(cimag(z)); }

int ora_zgetrf(int n, zc *a, int lda, int *ipiv)
{
    int info = 0;
    for (int k = 0; k < n; ++k) {
        int p = k;
        double pmax = cabs1(a[IX(k, k, lda)]);
        for (int i = k + 1; i < n; ++i) {
            double v = cabs1(a[IX(i, k, lda)]);
            if (v > pmax) {
                pmax = v;
                p = i;
            }
        }
        ipiv[k] = p;
        if (pmax == 0.0) {
            if (!info) info = k + 1;
            continue;
        }
        if (p != k)
            for (int j = 0; j < n; ++j) {
                zc t = a[IX(k, j, lda)];
                a[IX(k, j, lda)] = a[IX(p, j, lda)];
                a[IX(p, j, lda)] = t;
            }
        zc inv = 1.0 / a[IX(k, k, lda)];
        for (int i = k + 1; i < n; ++i) a[IX(i, k, lda)] *= inv;
        for (int j = k + 1; j < n; ++j) {
            zc ukj = a[IX(k, j, lda)];
            zc *cj = a + IX(0, j, lda);
            const zc *ck = a + IX(0, k, lda);
            for (int i = k + 1; i < n; ++i) cj[i] -= ck[i] * ukj;
        }
    }
    return info;
}

/* Solves with P S = L U (RCI case 11) or its adjoint (case 21):              */
/*   S X = B:    X = U^{-1} L^{-1} P B                                         */
/*   S^H X = B:  S^H = U^H L^H P, so X = P^T L^{-H} U^{-H} B                    */
void ora_zgetrs(int trans, int n, int nrhs, const zc *a, int lda,
                const int *ipiv, zc *b, int ldb)
{
    for (int j = 0; j < nrhs; ++j) {
        zc *x = b + IX(0, j, ldb);
        if (!trans) {
            for (int k = 0; k < n; ++k)
                if (ipiv[k] != k) {
                    zc t = x[k];
                    x[k] = x[ipiv[k]];
                    x[ipiv[k]] = t;
                }
            for (int k = 0; k < n; ++k) {
                zc xk = x[k];
                const zc *lk = a + IX(0, k, lda);
                for (int i = k + 1; i < n; ++i) x[i] -= lk[i] * xk;
            }
            for (int k = n - 1; k >= 0; --k) {
                const zc *uk = a + IX(0, k, lda);
                x[k] /= uk[k];
                zc xk = x[k];
                for (int i = 0; i < k; ++i) x[i] -= uk[i] * xk;
            }
        } else {
            for (int k = 0; k < n; ++k) {
                const zc *uk = a + IX(0, k, lda);
                zc s = x[k];
                for (int i = 0; i < k; ++i) s -= conj(uk[i]) * x[i];
                x[k] = s / conj(uk[k]);
            }
            for (int k = n - 1; k >= 0; --k) {
                const zc *lk = a + IX(0, k, lda);
                zc s = x[k];
                for (int i = k + 1; i < n; ++i) s -= conj(lk[i]) * x[i];
                x[k] = s;
            }
            for (int k = n - 1; k >= 0; --k)
                if (ipiv[k] != k) {
                    zc t = x[k];
                    x[k] = x[ipiv[k]];
                    x[ipiv[k]] = t;
                }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Cyclic-by-row two-sided Jacobi for a Hermitian matrix (the reduced dense  */
/* eigenproblem of the Rayleigh-Ritz step).  For the pivot block            */
/* [[a, b], [conj(b), d]] with b = |b| e^{i phi}:                             */
/*   tau = (d - a) / (2|b|),  t = sign(tau) / (|tau| + sqrt(1 + tau^2)),       */
/*   c = 1 / sqrt(1 + t^2),   s = t c,                                          */
/*   J = [[c, s e^{i phi}], [-s e^{-i phi}, c]],  A <- J^H A J,  V <- V J,       */
/* which zeroes A[p][q] and moves a -> a - t|b|, d -> d + t|b|.              */
/* A rotation is skipped when |b| <= eps/2 * sqrt(|a| |d|) or |b| is below   */
/* 1e-18 ||A||_F; a sweep without rotations ends the iteration.              */
/* ------------------------------------------------------------------------ */
int ora_zheev_jacobi(int n, zc *a, int lda, double *w, zc *v, int ldv)
{
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) v[IX(i, j, ldv)] = (i == j) ? 1.0 : 0.0;
    double fro = 0.0;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) fro += creal(a[IX(i, j, lda)] * conj(a[IX(i, j, lda)]));
    fro = sqrt(fro);
    const double eps = 2.220446049250313e-16;
    int sweeps = -1;
    for (int sweep = 0; sweep < 80; ++sweep) {
        long rotations = 0;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                zc b = a[IX(p, q, lda)];
                double ab = cabs(b);
                double app = creal(a[IX(p, p, lda)]), aqq = creal(a[IX(q, q, lda)]);
                if (ab == 0.0 || ab <= 0.5 * eps * sqrt(fabs(app)) * sqrt(fabs(aqq)) ||
                    ab <= 1e-18 * fro)
                    continue;
                ++rotations;
                zc ph = b / ab; /* e^{i phi} */
                double tau = (aqq - app) / (2.0 * ab);
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                zc sp = s * ph, sm = s * conj(ph); /* s e^{i phi}, s e^{-i phi} */
                /* columns: A <- A J */
                for (int i = 0; i < n; ++i) {
                    zc xp = a[IX(i, p, lda)], xq = a[IX(i, q, lda)];
                    a[IX(i, p, lda)] = c * xp - sm * xq;
                    a[IX(i, q, lda)] = sp * xp + c * xq;
                }
                /* rows: A <- J^H A */
                for (int j = 0; j < n; ++j) {
                    zc yp = a[IX(p, j, lda)], yq = a[IX(q, j, lda)];
                    a[IX(p, j, lda)] = c * yp - sp * yq;
                    a[IX(q, j, lda)] = sm * yp + c * yq;
                }
                a[IX(p, q, lda)] = 0.0;
                a[IX(q, p, lda)] = 0.0;
                a[IX(p, p, lda)] = app - t * ab;
                a[IX(q, q, lda)] = aqq + t * ab;
                for (int i = 0; i < n; ++i) {
                    zc xp = v[IX(i, p, ldv)], xq = v[IX(i, q, ldv)];
                    v[IX(i, p, ldv)] = c * xp - sm * xq;
                    v[IX(i, q, ldv)] = sp * xp + c * xq;
                }
            }
        if (rotations == 0) {
            sweeps = sweep;
            break;
        }
    }
    /* eigenvalues ascending (stable on ties), columns of V follow */
    int *idx = (int *)malloc(sizeof(int) * (n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) idx[i] = i;
    for (int i = 1; i < n; ++i) { /* insertion sort: small n only */
        int t = idx[i];
        double key = creal(a[IX(t, t, lda)]);
        int j = i - 1;
        while (j >= 0 && creal(a[IX(idx[j], idx[j], lda)]) > key) {
            idx[j + 1] = idx[j];
            --j;
        }
        idx[j + 1] = t;
    }
    zc *vs = (zc *)malloc(sizeof(zc) * (size_t)n * (n > 0 ? n : 1));
    for (int j = 0; j < n; ++j) {
        w[j] = creal(a[IX(idx[j], idx[j], lda)]);
        for (int i = 0; i < n; ++i) vs[IX(i, j, n)] = v[IX(i, idx[j], ldv)];
    }
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) v[IX(i, j, ldv)] = vs[IX(i, j, n)];
    free(vs);
    free(idx);
    return sweeps;
}

/* ------------------------------------------------------------------------ */
/* Sylvester inertia: number of negative eigenvalues of Hermitian H through  */
/* the congruence P H P^T = L D L^H with Bunch-Kaufman diagonal pivoting      */
/* (1x1 and 2x2 blocks, alpha = (1 + sqrt 17)/8).  For a Hermitian-definite  */
/* pencil, #eig in [a,b] = neg(A - bB) - neg(A - aB).                         */
/* ------------------------------------------------------------------------ */
long ora_inertia_neg(int n, zc *h, int ldh, long *zero_out)
{
    const double alpha = (1.0 + sqrt(17.0)) / 8.0;
    long neg = 0, zero = 0;
    int k = 0;
#define HH(i, j) h[IX(i, j, ldh)]
    while (k < n) {
        double absakk = fabs(creal(HH(k, k)));
        int r = k;
        double colmax = 0.0;
        for (int i = k + 1; i < n; ++i) {
            double v = cabs(HH(i, k));
            if (v > colmax) {
                colmax = v;
                r = i;
            }
        }
        if (absakk == 0.0 && colmax == 0.0) {
            ++zero;
            ++k;
            continue;
        }
        int kstep = 1, kp = k;
        if (absakk < alpha * colmax) {
            double rowmax = 0.0;
            for (int j = k; j < n; ++j)
                if (j != r) {
                    double v = cabs(HH(r, j));
                    if (v > rowmax) rowmax = v;
                }
            if (absakk >= alpha * colmax * (colmax / rowmax)) {
                kp = k;
            } else if (fabs(creal(HH(r, r))) >= alpha * rowmax) {
                kp = r;
            } else {
                kp = r;
                kstep = 2;
            }
        }
        int kk = k + kstep - 1;
        if (kp != kk) { /* symmetric swap kk <-> kp */
            for (int j = 0; j < n; ++j) {
                zc t = HH(kk, j);
                HH(kk, j) = HH(kp, j);
                HH(kp, j) = t;
            }
            for (int i = 0; i < n; ++i) {
                zc t = HH(i, kk);
                HH(i, kk) = HH(i, kp);
                HH(i, kp) = t;
            }
        }
        if (kstep == 1) {
            double d = creal(HH(k, k));
            if (d < 0.0) ++neg;
            if (d == 0.0) {
                ++zero;
                ++k;
                continue;
            }
#pragma omp parallel for schedule(static)
            for (int j = k + 1; j < n; ++j) {
                zc f = conj(HH(j, k)) / d;
                for (int i = k + 1; i < n; ++i) HH(i, j) -= HH(i, k) * f;
            }
        } else {
            double a = creal(HH(k, k)), c = creal(HH(k + 1, k + 1));
            zc b = HH(k + 1, k);
            double det = a * c - creal(b * conj(b));
            if (det < 0.0)
                neg += 1;
            else if (det > 0.0 && a + c < 0.0)
                neg += 2;
            else if (det == 0.0)
                ++zero;
#pragma omp parallel for schedule(static)
            for (int j = k + 2; j < n; ++j) {
                zc c1 = conj(HH(j, k)), c2 = conj(HH(j, k + 1));
                zc g1 = (c * c1 - conj(b) * c2) / det;
                zc g2 = (-b * c1 + a * c2) / det;
                for (int i = k + 2; i < n; ++i) HH(i, j) -= HH(i, k) * g1 + HH(i, k + 1) * g2;
            }
        }
        k += kstep;
    }
#undef HH
    if (zero_out) *zero_out = zero;
    return neg;
}

/* ------------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), counter-based form.         */
/* ------------------------------------------------------------------------ */
uint64_t ora_splitmix64(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static double u11(uint64_t seed, uint64_t i) /* uniform [-1, 1) */
{
    return (double)(ora_splitmix64(seed, i) >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

/* ------------------------------------------------------------------------ */
/* Dense helpers (plain loops).                                              */
/* ------------------------------------------------------------------------ */
/* C(m x n) = op(A) * B, op(A) = A (m x k, opa 0) or A^H (A is k x m, opa 1) */
static void zgemm_plain(int opa, int m, int n, int k, const zc *A, int lda,
                        const zc *B, int ldb, zc *C, int ldc, int nt)
{
#pragma omp parallel for schedule(static) num_threads(nt)
    for (int j = 0; j < n; ++j) {
        zc *c = C + IX(0, j, ldc);
        if (!opa) {
            for (int i = 0; i < m; ++i) c[i] = 0.0;
            for (int p = 0; p < k; ++p) {
                zc bpj = B[IX(p, j, ldb)];
                const zc *ap = A + IX(0, p, lda);
                for (int i = 0; i < m; ++i) c[i] += ap[i] * bpj;
            }
        } else {
            const zc *bj = B + IX(0, j, ldb);
            for (int i = 0; i < m; ++i) {
                const zc *ai = A + IX(0, i, lda);
                zc s = 0.0;
                for (int p = 0; p < k; ++p) s += conj(ai[p]) * bj[p];
                c[i] = s;
            }
        }
    }
}

static void herm_sym(int m, zc *a) /* a <- (a + a^H)/2 */
{
    for (int j = 0; j < m; ++j)
        for (int i = 0; i <= j; ++i) {
            zc s = 0.5 * (a[IX(i, j, m)] + conj(a[IX(j, i, m)]));
            a[IX(i, j, m)] = s;
            a[IX(j, i, m)] = conj(s);
        }
}

/* ------------------------------------------------------------------------ */
/* FEAST, Hermitian family (real symmetric: RCI cases 10/11/30/40;           */
/* complex Hermitian: additionally case 21, the adjoint solve).              */
/* ------------------------------------------------------------------------ */
#define ORA_SEED 0x3C6EF372FE94F82BULL /* initial-subspace seed (fpm(5)=0) */

static int check_fpm(const int *fpm)
{
    int ne = fpm[1], qtype = fpm[15];
    if (qtype != 0 && qtype != 1) return 116;
    if (qtype == 0) {
        int ok = (ne >= 1 && ne <= 20) || ne == 24 || ne == 32 || ne == 40 || ne == 48 || ne == 56;
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
    return 0;
}

int ora_feast(int kind, int n, const zc *A, int lda, const zc *B, int ldb,
              const int *fpm, double emin, double emax, int m0, const zc *zne_in,
              const zc *wne_in, zc *X, double *E, double *res, int *M, int *loop,
              double *epsout, int *m0_out, int *info_out, int nthreads)
{
    int info = 0;
    *M = 0;
    *loop = 0;
    *epsout = 1.0;
    *m0_out = m0;
    if (n < 1) { info = 202; goto done_early; }
    if (m0 < 1 || m0 > n) { info = 201; goto done_early; }
    if (!(emin < emax)) { info = 200; goto done_early; }
    if ((info = check_fpm(fpm)) != 0) goto done_early;
    if (nthreads < 1) nthreads = 1;

    {
        const int ne = fpm[1];
        const double eps = pow(10.0, -fpm[2]);
        const double alpha = fmax(fabs(emin), fabs(emax));
        zc *zne = (zc *)malloc(sizeof(zc) * ne), *wne = (zc *)malloc(sizeof(zc) * ne);
        if (zne_in && wne_in) {
            memcpy(zne, zne_in, sizeof(zc) * ne);
            memcpy(wne, wne_in, sizeof(zc) * ne);
        } else {
            ora_contour(emin, emax, ne, fpm[15], fpm[17], zne, wne);
        }
        size_t nn = (size_t)n * n, nm = (size_t)n * m0, mm = (size_t)m0 * m0;
        zc *Y = (zc *)malloc(sizeof(zc) * nm), *RHS = (zc *)malloc(sizeof(zc) * nm);
        zc *Q = (zc *)malloc(sizeof(zc) * nm), *AQ = (zc *)malloc(sizeof(zc) * nm);
        zc *BQ = (zc *)malloc(sizeof(zc) * nm), *AX = (zc *)malloc(sizeof(zc) * nm);
        zc *BX = (zc *)malloc(sizeof(zc) * nm), *Xn = (zc *)malloc(sizeof(zc) * nm);
        zc *Qe = (zc *)malloc(sizeof(zc) * nm * ne);
        zc *Aq = (zc *)malloc(sizeof(zc) * mm), *Bq = (zc *)malloc(sizeof(zc) * mm);
        zc *V = (zc *)malloc(sizeof(zc) * mm), *T = (zc *)malloc(sizeof(zc) * mm);
        zc *Cm = (zc *)malloc(sizeof(zc) * mm), *U = (zc *)malloc(sizeof(zc) * mm);
        zc *Wm = (zc *)malloc(sizeof(zc) * mm), *tmp = (zc *)malloc(sizeof(zc) * mm);
        double *d = (double *)malloc(sizeof(double) * m0), *lam = (double *)malloc(sizeof(double) * m0);
        double *sc = (double *)malloc(sizeof(double) * m0), *rr = (double *)malloc(sizeof(double) * m0);
        int *ord = (int *)malloc(sizeof(int) * m0);
        int *spur = (int *)malloc(sizeof(int) * m0);
        int *singular = (int *)calloc(ne, sizeof(int));
        if (!Y || !RHS || !Q || !AQ || !BQ || !AX || !BX || !Xn || !Qe || !Aq || !Bq || !V ||
            !T || !Cm || !U || !Wm || !tmp || !d || !lam || !sc || !rr || !ord || !spur || !singular) {
            info = -1;
            goto cleanup;
        }

        /* initial subspace Y (n x m0): input X (fpm(5)=1) or SplitMix64;
         * for the stochastic estimate (fpm(14)=2) the generated columns are
         * Rademacher probes, +1 or -1 by the top bit of SplitMix64 */
        if (fpm[4] == 1) {
            memcpy(Y, X, sizeof(zc) * nm);
        } else if (fpm[13] == 2) {
            for (size_t i = 0; i < nm; ++i) Y[i] = (ora_splitmix64(ORA_SEED, i) >> 63) ? -1.0 : 1.0;
        } else {
            for (size_t i = 0; i < nm; ++i)
                Y[i] = kind ? (u11(ORA_SEED, 2 * i) + I * u11(ORA_SEED, 2 * i + 1)) : u11(ORA_SEED, i);
        }
        int m = m0; /* current subspace size */
        double trace_prev = 0.0;

        for (int k = 0;; ++k) {
            /* RHS = B Y (RCI case 40; a copy for the standard problem) */
            if (B)
                zgemm_plain(0, n, m, n, B, ldb, Y, n, RHS, n, nthreads);
            else
                memcpy(RHS, Y, sizeof(zc) * n * m);

            /* contour nodes: independent factor + solve(s) (cases 10, 11, 21) */
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
            for (int e = 0; e < ne; ++e) {
                zc *S = (zc *)malloc(sizeof(zc) * nn);
                zc *G = (zc *)malloc(sizeof(zc) * (size_t)n * m);
                zc *G2 = kind ? (zc *)malloc(sizeof(zc) * (size_t)n * m) : NULL;
                int *ipiv = (int *)malloc(sizeof(int) * n);
                zc *qe = Qe + (size_t)e * n * m;
                if (!S || !G || !ipiv || (kind && !G2)) {
                    singular[e] = -1;
                } else {
                    for (int j = 0; j < n; ++j)
                        for (int i = 0; i < n; ++i)
                            S[IX(i, j, n)] = (B ? zne[e] * B[IX(i, j, ldb)] : (i == j ? zne[e] : 0.0)) -
                                             A[IX(i, j, lda)];
                    if (ora_zgetrf(n, S, n, ipiv) != 0) singular[e] = 1;
                    memcpy(G, RHS, sizeof(zc) * (size_t)n * m);
                    ora_zgetrs(0, n, m, S, n, ipiv, G, n);
                    if (!kind) {
                        for (size_t i = 0; i < (size_t)n * m; ++i) qe[i] = creal(wne[e] * G[i]);
                    } else {
                        memcpy(G2, RHS, sizeof(zc) * (size_t)n * m);
                        ora_zgetrs(1, n, m, S, n, ipiv, G2, n);
                        for (size_t i = 0; i < (size_t)n * m; ++i)
                            qe[i] = 0.5 * (wne[e] * G[i] + conj(wne[e]) * G2[i]);
                    }
                }
                free(S);
                free(G);
                free(G2);
                free(ipiv);
            }
            for (int e = 0; e < ne; ++e) {
                if (singular[e] < 0) { info = -1; goto cleanup; }
                if (singular[e] > 0) { info = -2; goto cleanup; }
            }
            /* Q = sum_e (node contributions), summed in node order */
            for (size_t i = 0; i < (size_t)n * m; ++i) {
                zc s = 0.0;
                for (int e = 0; e < ne; ++e) s += Qe[(size_t)e * n * m + i];
                Q[i] = s;
            }
            if (fpm[13] == 2) {
                /* stochastic count ("Stochastic estimate" section, after Di
                 * Napoli, Polizzi & Saad): Q = f(B^-1 A) Y is the filtered
                 * probe block, and for a probe y with independent +-1
                 * entries E[y^H f(B^-1 A) y] = trace f(B^-1 A), which is the
                 * eigenvalue count in the interval when f is the indicator.
                 * res(j) = mean of Re(y_i^H q_i) over the first j probes;
                 * M = that mean over all M0 probes, rounded, within [0, N];
                 * X returns the probes Y. */
                double s = 0.0;
                for (int j = 0; j < m0; ++j) {
                    double t = 0.0;
                    for (int i = 0; i < n; ++i) t += creal(conj(Y[IX(i, j, n)]) * Q[IX(i, j, n)]);
                    s += t;
                    res[j] = s / (j + 1);
                    E[j] = 0.0;
                }
                double mh = floor(res[m0 - 1] + 0.5);
                *M = mh > 0.0 ? (mh < n ? (int)mh : n) : 0;
                memcpy(X, Y, sizeof(zc) * nm);
                *loop = 0;
                info = 5;
                goto cleanup;
            }
            if (fpm[13] == 1) { /* return the subspace after one contour */
                memset(X, 0, sizeof(zc) * nm);
                memcpy(X, Q, sizeof(zc) * n * m);
                *loop = k;
                info = 4;
                goto cleanup;
            }

            /* Rayleigh-Ritz: Aq = Q^H A Q, Bq = Q^H B Q (cases 30, 40) */
            zgemm_plain(0, n, m, n, A, lda, Q, n, AQ, n, nthreads);
            if (B)
                zgemm_plain(0, n, m, n, B, ldb, Q, n, BQ, n, nthreads);
            else
                memcpy(BQ, Q, sizeof(zc) * n * m);
            zgemm_plain(1, m, m, n, Q, n, AQ, n, Aq, m, nthreads);
            zgemm_plain(1, m, m, n, Q, n, BQ, n, Bq, m, nthreads);
            herm_sym(m, Aq);
            herm_sym(m, Bq);

            /* B-orthonormalisation: unit-diagonal scaling, then Jacobi on Bq */
            for (int i = 0; i < m; ++i) {
                double bii = creal(Bq[IX(i, i, m)]);
                if (!(bii > 0.0)) { info = -3; goto cleanup; }
                sc[i] = 1.0 / sqrt(bii);
            }
            for (int j = 0; j < m; ++j)
                for (int i = 0; i < m; ++i) {
                    Bq[IX(i, j, m)] *= sc[i] * sc[j];
                    Aq[IX(i, j, m)] *= sc[i] * sc[j];
                }
            ora_zheev_jacobi(m, Bq, m, d, V, m);
            double dmax = d[m - 1];
            if (!(dmax > 0.0) || d[0] < -1e-8 * dmax) { info = -3; goto cleanup; }
            int first = 0; /* d ascending: keep d_i > 1e-12 dmax */
            while (first < m && !(d[first] > 1e-12 * dmax)) ++first;
            int mk = m - first;
            /* T = V_keep D_keep^{-1/2}  (m x mk) */
            for (int j = 0; j < mk; ++j) {
                double f = 1.0 / sqrt(d[first + j]);
                for (int i = 0; i < m; ++i) T[IX(i, j, m)] = V[IX(i, first + j, m)] * f;
            }
            /* C = T^H Aq_s T (mk x mk), Jacobi -> lambda, U */
            zgemm_plain(0, m, mk, m, Aq, m, T, m, tmp, m, 1);
            zgemm_plain(1, mk, mk, m, T, m, tmp, m, Cm, mk, 1);
            herm_sym(mk, Cm);
            ora_zheev_jacobi(mk, Cm, mk, lam, U, mk);
            /* W = diag(sc) T U (m x mk) */
            zgemm_plain(0, m, mk, mk, T, m, U, mk, Wm, m, 1);
            for (int j = 0; j < mk; ++j)
                for (int i = 0; i < m; ++i) Wm[IX(i, j, m)] *= sc[i];

            /* Ritz vectors and residuals (Table tab_common: res definition) */
            zgemm_plain(0, n, mk, m, Q, n, Wm, m, Xn, n, nthreads);
            zgemm_plain(0, n, mk, m, AQ, n, Wm, m, AX, n, nthreads);
            zgemm_plain(0, n, mk, m, BQ, n, Wm, m, BX, n, nthreads);
            for (int j = 0; j < mk; ++j) {
                double num = 0.0, den = 0.0;
                for (int i = 0; i < n; ++i) {
                    num += cabs(AX[IX(i, j, n)] - lam[j] * BX[IX(i, j, n)]);
                    den += cabs(alpha * BX[IX(i, j, n)]);
                }
                rr[j] = num / den;
            }
            /* spurious pairs (loops >= 1, Y = previous B-orthonormal Ritz
             * vectors): x_j = Q w_j is the filter applied to z_j = Y w_j with
             * ||z_j||_B = ||w_j||_2 and ||x_j||_B = 1, so a_j = 1/||w_j||_2 is
             * the filter's gain on the pair's pre-image.  A genuine pair has
             * a_j ~ f(lambda_j) (>= 1/2 inside the interval); a pair inside
             * whose gain is below f(lambda_j)/4 is spurious. */
            for (int j = 0; j < mk; ++j) {
                spur[j] = 0;
                if (k == 0) continue;
                if (!(lam[j] >= emin && lam[j] <= emax)) continue;
                double nw = 0.0;
                for (int i = 0; i < m; ++i) nw += creal(Wm[IX(i, j, m)] * conj(Wm[IX(i, j, m)]));
                double fj;
                ora_rationalx(zne, wne, ne, &lam[j], 1, &fj);
                if (1.0 / sqrt(nw) < 0.25 * fabs(fj)) spur[j] = 1;
            }
            /* order: genuine pairs inside ascending, then outside ascending,
             * then spurious ones (res = -1), as Table tab_common's remark */
            int nin = 0, pos = 0;
            for (int j = 0; j < mk; ++j)
                if (lam[j] >= emin && lam[j] <= emax && !spur[j]) ord[pos++] = j, ++nin;
            for (int j = 0; j < mk; ++j)
                if (!(lam[j] >= emin && lam[j] <= emax)) ord[pos++] = j;
            for (int j = 0; j < mk; ++j)
                if (spur[j]) ord[pos++] = j;
            double trace = 0.0, maxres = 0.0;
            for (int j = 0; j < nin; ++j) {
                trace += lam[ord[j]];
                if (rr[ord[j]] > maxres) maxres = rr[ord[j]];
            }
            double eout = (k == 0) ? 1.0 : fabs(trace - trace_prev) / alpha;
            /* write outputs in that order */
            memset(X, 0, sizeof(zc) * nm);
            for (int j = 0; j < m0; ++j) {
                E[j] = 0.0;
                res[j] = 0.0;
            }
            for (int j = 0; j < mk; ++j) {
                E[j] = lam[ord[j]];
                res[j] = spur[ord[j]] ? -1.0 : rr[ord[j]];
                memcpy(X + IX(0, j, n), Xn + IX(0, ord[j], n), sizeof(zc) * n);
            }
            *M = nin;
            *loop = k;
            *epsout = eout;
            *m0_out = mk;
            if (nin == 0) { info = 1; break; }
            if (nin >= m0 && m0 < n) { info = 3; break; }
            int conv = (fpm[5] == 0) ? (eout < eps) : (maxres < eps);
            if (conv) { info = 0; break; }
            if (k >= fpm[3]) { info = 2; break; }
            /* next subspace: the Ritz vectors */
            memcpy(Y, X, sizeof(zc) * n * mk);
            m = mk;
            trace_prev = trace;
        }
    cleanup:
        free(zne); free(wne); free(Y); free(RHS); free(Q); free(AQ); free(BQ); free(AX);
        free(BX); free(Xn); free(Qe); free(Aq); free(Bq); free(V); free(T); free(Cm);
        free(U); free(Wm); free(tmp); free(d); free(lam); free(sc); free(rr); free(ord); free(spur);
        free(singular);
    }
done_early:
    *info_out = info;
    return info;
}
