/*
 * rrq_oracle.c -- CPU FP64 oracle for the recursive reduction quadrature (RRQ)
 * near-field correction rows of the Laplace S, D, S', D' operators
 * (Jiang & Zhu, "Recursive reduction quadrature for the evaluation of Laplace
 * layer potentials in three dimensions", arXiv 2411.08342).
 *
 * TEST INFRASTRUCTURE.  This file is the slow, plain reference that the CUDA
 * library is checked against.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark load it.  It shares no code, header or table
 * generator with the CUDA library.
 *
 * Every step follows the paper's algorithm in its order and notation:
 *   - regular solid harmonics R_l^m from the Legendre recurrence (Sec. 2.3,
 *     eqs. associatelegendrerecurrence, ylmdef, rlmdef), S^{(l,m)}(x,y,z) =
 *     R_l^m(y,z,x) and H^{(l,m)} = sqrt2 Im S^{(l,m)} (eqs. slmdef, hlmslmconnection);
 *   - the translation formula with T_{jk,lm} (eqs. l2ltranslation, tjklmdef),
 *     used also to differentiate S (its j=1 and j=2 terms);
 *   - the quaternion harmonic fit (eq. dlpdensitylinearsystem2), the scalar
 *     SLP fit (eq. slpdensitylinearsystem) and the S' fit
 *     (eq. sprimedensitylinearsystem), solved by LU with partial pivoting;
 *   - target-centred 1-forms (Thms. dlp1form, cslp1form), line integrals
 *     (eqs. lineintegrals, solidangle), singularity-swap quadrature (Sec. 2.4,
 *     Sec. 3.4: root t0, moments, c = U F), the D' line integrals
 *     (eq. dprimelineintegrals), and Step 8 (eq. wlmdef) with the matrix-build
 *     remark of Sec. 4.
 *
 * Readings where the paper is silent or inconsistent (each one is applied
 * identically by the CUDA path, which implements it independently):
 *   - S' sign: S'[sigma] = -int nu'.grad_r G sigma; with the fit of (0, sigma nu)
 *     the row is -[(0,nu') sum B^{lm} w^{lm}]_0 (the printed eq. sprime1formrep
 *     has the opposite overall sign).
 *   - the S^{(l,m)}(r') omega_0 term of Thm. cslp1form carries 1/(4 pi).
 *   - frame: origin = vertex mean, e_z = unit((V1-V0)x(V2-V0)), e_x along the
 *     longest edge (first of E0,E1,E2 on ties), scale 1/longest edge.
 *   - u: +e_z for a target that is a node of the patch; otherwise, if the target's
 *     footprint along e_z (the point of the node interpolant with the target's in-plane
 *     frame coordinates) lies in the patch, the +-e_z pointing from that point to the
 *     target; otherwise whichever of +e_z, -e_z maximises the minimum of
 *     u.(r'-r)/|r'-r| over the nodes and edge samples (so that the half-line from the
 *     target along u misses the patch, as Thm. dlp1form requires).
 *   - Omega_0 sign: Thm. dlp1form needs (1/4pi) d omega_0 = -grad_r G . nu da, but the
 *     printed omega_0 (eq. omega0def) integrates to +4 pi int grad_r G . nu da (checked
 *     on a disc by hand), so Omega_0 = - (line integral of the printed omega_0); its
 *     nu' derivative (eq. dprimelineintegrals) is negated the same way.
 *   - Omega_0 and its nu' derivative: composite Gauss-Legendre on panels graded
 *     geometrically toward Re t0 (the "mild adaptive" integration of Sec. 3.4).
 *   - the SSQ is used when the Bernstein radius of t0 is below rho0; otherwise
 *     the modified weights are formed by a 2*ptilde point Gauss rule applied to
 *     the Lagrange basis of the ptilde edge nodes.
 *   - on-surface (self) pairs return the principal value for D and S'
 *     (jump 1/2 applied at the coincident node), S and D' as computed.
 *   - correction = RRQ row - smooth row (K(x_t, x_i) w_i, coincident node skipped).
 */
#ifdef ORC_F128
#define __STDC_WANT_IEC_60559_TYPES_EXT__ 1
#endif
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Number type of every computed quantity.  The default build is IEEE binary64.
 * Compiled with -DORC_F128 the same source computes in IEEE binary128 (_Float128,
 * glibc's f128 functions): inputs and outputs stay binary64 at the exported
 * interface, so the binary128 build evaluates the same algorithm on the same inputs
 * with a rounding unit of 2^-113; it is the truth against which the binary64 results
 * (this oracle's and the CUDA library's) are measured. */
#ifdef ORC_F128
typedef _Float128 real;
typedef _Complex _Float128 cplx;
#define R_PI 3.14159265358979323846264338327950288f128
#define xsqrt sqrtf128
#define xfabs fabsf128
#define xcos cosf128
#define xpow powf128
#define xasinh asinhf128
#define xcabs cabsf128
#define xcsqrt csqrtf128
#define xcreal crealf128
#define xcimag cimagf128
#define xconj conjf128
#else
typedef double real;
typedef double complex cplx;
#define R_PI M_PI
#define xsqrt sqrt
#define xfabs fabs
#define xcos cos
#define xpow pow
#define xasinh asinh
#define xcabs cabs
#define xcsqrt csqrt
#define xcreal creal
#define xcimag cimag
#define xconj conj
#endif

#define ORC_PMAX 14
#define ORC_LMAX 16
#define ORC_PTMAX 32
#define ORC_NOM 16
#define HIDX(n, q) ((n) * (n) + (n) + (q))
#define NHFULL(L) (((L) + 1) * ((L) + 1))

enum { ORC_S = 1, ORC_D = 2, ORC_SP = 4, ORC_DP = 8 };
enum { FLAG_NEWTON = 1, FLAG_ONEDGE = 2, FLAG_UPOOR = 4, FLAG_SINGULAR = 8 };

typedef struct {
    int ptilde;      /* GL nodes per edge; <=0 -> 2p */
    double rho0;   /* SSQ Bernstein-radius threshold; <=0 -> 10^(5/ptilde) */
    int newton_max;  /* <=0 -> 30 */
    double eta;    /* near factor; <=0 -> 1 */
} orc_opts;

/* ------------------------------------------------------------------------- */
/* small numerics                                                             */
/* ------------------------------------------------------------------------- */

static real g_binom[2 * ORC_LMAX + 2][2 * ORC_LMAX + 2];
static int g_binom_ready = 0;

static void binom_init(void) {
    if (g_binom_ready) return;
    for (int n = 0; n < 2 * ORC_LMAX + 2; n++) {
        for (int k = 0; k < 2 * ORC_LMAX + 2; k++) g_binom[n][k] = 0.0;
        g_binom[n][0] = 1.0;
        for (int k = 1; k <= n; k++) g_binom[n][k] = g_binom[n - 1][k - 1] + (k <= n - 1 ? g_binom[n - 1][k] : 0.0);
    }
    g_binom_ready = 1;
}

static real binom(int n, int k) {
    if (n < 0 || k < 0 || k > n) return 0.0;
    return g_binom[n][k];
}

static real factd(int n) {
    real r = 1.0;
    for (int i = 2; i <= n; i++) r *= i;
    return r;
}

/* T_{jk,lm}, eq. (tjklmdef); zero when a binomial index is out of range. */
static real Tcoef(int j, int k, int l, int m) {
    return xsqrt(binom(l + m, j + k) * binom(l - m, j - k));
}

/* C_{j,l} = int_0^1 t^{j-2}(1-t)^{l-j} dt (Thm. dlp1form) */
static real Ccoef(int j, int l) { return factd(j - 2) * factd(l - j) / factd(l - 1); }
/* D_{j,l} = int_0^1 t^{j-1}(1-t)^{l-j} dt (Thm. cslp1form) */
static real Dcoef(int j, int l) { return factd(j - 1) * factd(l - j) / factd(l); }

/* Gauss-Legendre nodes and weights on [-1,1] by Newton on P_n. */
static void gauss_legendre(int n, real *x, real *w) {
    for (int i = 0; i < n; i++) {
        real t = xcos(R_PI * (i + 0.75) / (n + 0.5));
        real dp = 1.0;
        for (int it = 0; it < 100; it++) {
            real p0 = 1.0, p1 = t;
            for (int k = 2; k <= n; k++) {
                real p2 = ((2 * k - 1) * t * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = t; p0 = 1.0; }
            dp = n * (t * p1 - p0) / (t * t - 1.0);
            real dt = p1 / dp;
            t -= dt;
            if (xfabs(dt) < 1e-16) {
                /* recompute derivative at the converged point */
                p0 = 1.0; p1 = t;
                for (int k = 2; k <= n; k++) {
                    real p2 = ((2 * k - 1) * t * p1 - (k - 1) * p0) / k;
                    p0 = p1; p1 = p2;
                }
                if (n == 1) { p1 = t; p0 = 1.0; }
                dp = n * (t * p1 - p0) / (t * t - 1.0);
                break;
            }
        }
        x[n - 1 - i] = t;
        w[n - 1 - i] = 2.0 / ((1.0 - t * t) * dp * dp);
    }
}

/* In-place LU with partial pivoting of the n x n row-major matrix a; piv[n]. */
static int lu_factor(int n, real *a, int *piv) {
    for (int k = 0; k < n; k++) {
        int pr = k;
        real mx = xfabs(a[k * n + k]);
        for (int i = k + 1; i < n; i++)
            if (xfabs(a[i * n + k]) > mx) { mx = xfabs(a[i * n + k]); pr = i; }
        piv[k] = pr;
        if (mx == 0.0) return -1;
        if (pr != k)
            for (int j = 0; j < n; j++) { real t = a[k * n + j]; a[k * n + j] = a[pr * n + j]; a[pr * n + j] = t; }
        for (int i = k + 1; i < n; i++) {
            real f = a[i * n + k] / a[k * n + k];
            a[i * n + k] = f;
            for (int j = k + 1; j < n; j++) a[i * n + j] -= f * a[k * n + j];
        }
    }
    return 0;
}

/* Solve with the factors for nrhs right-hand sides stored as columns of b (n x nrhs). */
static void lu_solve(int n, const real *lu, const int *piv, int nrhs, real *b) {
    for (int k = 0; k < n; k++)
        if (piv[k] != k)
            for (int c = 0; c < nrhs; c++) { real t = b[k * nrhs + c]; b[k * nrhs + c] = b[piv[k] * nrhs + c]; b[piv[k] * nrhs + c] = t; }
    for (int i = 0; i < n; i++)
        for (int k = 0; k < i; k++) {
            real f = lu[i * n + k];
            if (f != 0.0)
                for (int c = 0; c < nrhs; c++) b[i * nrhs + c] -= f * b[k * nrhs + c];
        }
    for (int i = n - 1; i >= 0; i--) {
        for (int k = i + 1; k < n; k++) {
            real f = lu[i * n + k];
            if (f != 0.0)
                for (int c = 0; c < nrhs; c++) b[i * nrhs + c] -= f * b[k * nrhs + c];
        }
        for (int c = 0; c < nrhs; c++) b[i * nrhs + c] /= lu[i * n + i];
    }
}

/* ------------------------------------------------------------------------- */
/* Harmonic polynomials (Sec. 2.3)                                            */
/* ------------------------------------------------------------------------- */

/* R_l^m(X,Y,Z) for 0<=l<=L, -l<=m<=l, into R[HIDX(l,m)].  The recurrence of eq.
 * (associatelegendrerecurrence) is applied to W_l^m = r^l P_l^m(Z/r) e^{i m phi},
 * which removes every division by r; then R_l^m = xsqrt((l-m)!/(l+m)!) W_l^m
 * (eqs. ylmdef, rlmdef) and R_l^{-m} = (-1)^m xconj(R_l^m). */
static void solid_R(int L, real X, real Y, real Z, cplx *R) {
    cplx W[ORC_LMAX + 1][ORC_LMAX + 1];
    real r2 = X * X + Y * Y + Z * Z;
    W[0][0] = 1.0;
    for (int l = 0; l < L; l++) {
        W[l + 1][l + 1] = -(2.0 * l + 1.0) * (X + I * Y) * W[l][l];
        W[l + 1][l] = (2.0 * l + 1.0) * Z * W[l][l];
        for (int m = 0; m <= l - 1; m++)
            W[l + 1][m] = ((2.0 * l + 1.0) * Z * W[l][m] - (l + m) * r2 * W[l - 1][m]) / (l - m + 1.0);
    }
    for (int l = 0; l <= L; l++)
        for (int m = 0; m <= l; m++) {
            cplx v = xsqrt(factd(l - m) / factd(l + m)) * W[l][m];
            R[HIDX(l, m)] = v;
            if (m > 0) R[HIDX(l, -m)] = ((m & 1) ? -1.0 : 1.0) * xconj(v);
        }
}

/* S^{(l,m)}(x,y,z) = R_l^m(y,z,x), eq. (slmdef). */
static void solid_S(int L, const real y[3], cplx *S) { solid_R(L, y[1], y[2], y[0], S); }

static cplx Sget(const cplx *S, int L, int n, int q) {
    if (n < 0 || n > L || q < -n || q > n) return 0.0;
    return S[HIDX(n, q)];
}

/* Constant gradients of S^{(1,k)} and Hessians of S^{(2,k)}: S^{(1,k)} is linear and
 * S^{(2,k)} quadratic, so g_k[a] = S^{(1,k)}(e_a) and
 * H_k[a][b] = S(e_a+e_b) - S(e_a) - S(e_b). */
static cplx g1[3][3];      /* [k+1][a] */
static cplx h2[5][3][3];   /* [k+2][a][b] */
static int g_lowdeg_ready = 0;

static void lowdeg_init(void) {
    if (g_lowdeg_ready) return;
    binom_init();
    cplx S[NHFULL(2)], Sa[NHFULL(2)], Sb[NHFULL(2)];
    for (int a = 0; a < 3; a++) {
        real ea[3] = {0, 0, 0};
        ea[a] = 1.0;
        solid_S(1, ea, S);
        for (int k = -1; k <= 1; k++) g1[k + 1][a] = S[HIDX(1, k)];
    }
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            real eab[3] = {0, 0, 0}, ea[3] = {0, 0, 0}, eb[3] = {0, 0, 0};
            eab[a] += 1.0; eab[b] += 1.0; ea[a] = 1.0; eb[b] = 1.0;
            solid_S(2, eab, S);
            solid_S(2, ea, Sa);
            solid_S(2, eb, Sb);
            for (int k = -2; k <= 2; k++) h2[k + 2][a][b] = S[HIDX(2, k)] - Sa[HIDX(2, k)] - Sb[HIDX(2, k)];
        }
    g_lowdeg_ready = 1;
}

/* grad S^{(l,m)}(y) from the j=1 terms of the translation (eq. l2ltranslation):
 * grad S^{(l,m)}(y) = sum_k grad S^{(1,k)} S^{(l-1,m-k)}(y) T_{1k,lm}. */
static void grad_S(const cplx *S, int L, int l, int m, cplx g[3]) {
    g[0] = g[1] = g[2] = 0.0;
    for (int k = -1; k <= 1; k++) {
        cplx f = Sget(S, L, l - 1, m - k) * Tcoef(1, k, l, m);
        for (int a = 0; a < 3; a++) g[a] += g1[k + 1][a] * f;
    }
}

/* Hessian from the j=2 terms of the translation. */
static void hess_S(const cplx *S, int L, int l, int m, cplx H[3][3]) {
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) H[a][b] = 0.0;
    for (int k = -2; k <= 2; k++) {
        cplx f = Sget(S, L, l - 2, m - k) * Tcoef(2, k, l, m);
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) H[a][b] += h2[k + 2][a][b] * f;
    }
}

/* ------------------------------------------------------------------------- */
/* Quaternions (eq. qprule)                                                   */
/* ------------------------------------------------------------------------- */

typedef struct { cplx s, v[3]; } cquat;

static cquat cq_zero(void) { cquat q; q.s = 0; q.v[0] = q.v[1] = q.v[2] = 0; return q; }

static cquat cq_mul(cquat f, cquat g) {
    cquat r;
    r.s = f.s * g.s - (f.v[0] * g.v[0] + f.v[1] * g.v[1] + f.v[2] * g.v[2]);
    r.v[0] = f.s * g.v[0] + g.s * f.v[0] + (f.v[1] * g.v[2] - f.v[2] * g.v[1]);
    r.v[1] = f.s * g.v[1] + g.s * f.v[1] + (f.v[2] * g.v[0] - f.v[0] * g.v[2]);
    r.v[2] = f.s * g.v[2] + g.s * f.v[2] + (f.v[0] * g.v[1] - f.v[1] * g.v[0]);
    return r;
}

static cquat cq_vec(const cplx v[3]) { cquat q; q.s = 0; q.v[0] = v[0]; q.v[1] = v[1]; q.v[2] = v[2]; return q; }
static cquat cq_rvec(const real v[3]) { cquat q; q.s = 0; q.v[0] = v[0]; q.v[1] = v[1]; q.v[2] = v[2]; return q; }
static void cq_axpy(cquat *acc, cplx a, cquat x) {
    acc->s += a * x.s;
    for (int i = 0; i < 3; i++) acc->v[i] += a * x.v[i];
}

/* ------------------------------------------------------------------------- */
/* Dubiner (Koornwinder) basis on T for the node interpolant                  */
/* ------------------------------------------------------------------------- */

static void dubiner(int deg, real u, real v, real *out) {
    real x = 2.0 * u - 1.0 + v, w = 1.0 - v, eta = 2.0 * v - 1.0;
    real Lh[ORC_PMAX + 2];
    Lh[0] = 1.0;
    if (deg >= 1) Lh[1] = x;
    for (int a = 1; a < deg; a++) Lh[a + 1] = ((2 * a + 1) * x * Lh[a] - a * w * w * Lh[a - 1]) / (a + 1);
    int idx = 0;
    for (int a = 0; a <= deg; a++) {
        real al = 2 * a + 1;
        real J[ORC_PMAX + 2];
        J[0] = 1.0;
        if (deg - a >= 1) J[1] = 0.5 * ((al + 2) * eta + al);
        for (int b = 1; b < deg - a; b++) {
            real c1 = 2.0 * (b + 1) * (b + al + 1) * (2 * b + al);
            real c2 = (2 * b + al + 1) * (al * al);
            real c3 = (2 * b + al) * (2 * b + al + 1) * (2 * b + al + 2);
            real c4 = 2.0 * (b + al) * b * (2 * b + al + 2);
            J[b + 1] = ((c2 + c3 * eta) * J[b] - c4 * J[b - 1]) / c1;
        }
        for (int b = 0; b <= deg - a; b++) out[idx++] = Lh[a] * J[b];
    }
}

/* ------------------------------------------------------------------------- */
/* Per-order tables                                                           */
/* ------------------------------------------------------------------------- */

/* LU factors (with pivots) of V^T, V[q][i] = t_q^i, for the edge nodes t_q (Sec. 3.4). */
static int vt_factor(int pt, const real *tq, real *lu, int *piv) {
    for (int i = 0; i < pt; i++)
        for (int q = 0; q < pt; q++) lu[i * pt + q] = xpow(tq[q], i);
    return lu_factor(pt, lu, piv);
}

typedef struct {
    int p, np, pt, nup;
    real rho0;
    real tq[ORC_PTMAX], wq[ORC_PTMAX];          /* edge GL nodes */
    real VtLU[ORC_PTMAX * ORC_PTMAX];           /* LU factors of V^T, V[q][i] = t_q^i (Sec. 3.4) */
    int Vtpiv[ORC_PTMAX];                         /* its pivots */
    real tu[2 * ORC_PTMAX], wu[2 * ORC_PTMAX];  /* upsampled GL */
    real Lup[2 * ORC_PTMAX * ORC_PTMAX];        /* Lagrange of edge nodes at tu */
    real tom[ORC_NOM], wom[ORC_NOM];            /* GL per Omega_0 panel */
    real *Eint;                                 /* [3*pt][np] node -> edge GL samples */
    real *Vint;                                 /* [3][np] node -> vertices */
    real *VdLU;                                 /* [np][np] LU of the transposed Dubiner Vandermonde */
    int *VdPiv;                                   /* its pivots */
} orc_order;

/* edge e parametrisation (u,v)(t), t in [-1,1]: E0 v0->v1, E1 v1->v2, E2 v2->v0 */
static void edge_uv(int e, real t, real *u, real *v) {
    real s = 0.5 * (1.0 + t);
    if (e == 0) { *u = s; *v = 0.0; }
    else if (e == 1) { *u = 1.0 - s; *v = s; }
    else { *u = 0.0; *v = 1.0 - s; }
}

static int order_init(orc_order *O, int p, const double *ref_uv, const orc_opts *opt) {
    memset(O, 0, sizeof(*O));
    O->p = p;
    O->np = p * (p + 1) / 2;
    O->pt = (opt && opt->ptilde > 0) ? opt->ptilde : 2 * p;
    if (O->pt > ORC_PTMAX || p > ORC_PMAX || p < 1) return -1;
    O->nup = 2 * O->pt;
    O->rho0 = (opt && opt->rho0 > 0) ? opt->rho0 : xpow(10.0, 5.0 / O->pt);
    int pt = O->pt, np = O->np;
    gauss_legendre(pt, O->tq, O->wq);
    gauss_legendre(O->nup, O->tu, O->wu);
    gauss_legendre(ORC_NOM, O->tom, O->wom);
    /* Sec. 3.4 writes c~ = U F with U the inverse of the monomial Vandermonde V[q][i] = t_q^i;
     * then I = sum_i c~_i I_i = lambda . F with V^T lambda = (I_0 .. I_{pt-1}).  Following
     * Sec. 5.1 (the conditioning of V is harmless when the system is solved by a backward
     * stable method), lambda is obtained by solving that system with the LU factors of V^T,
     * not by multiplying with an explicitly formed inverse, whose product cancels. */
    if (vt_factor(pt, O->tq, O->VtLU, O->Vtpiv)) return -1;
    /* Lagrange basis of the pt edge nodes at the upsampled nodes */
    for (int s = 0; s < O->nup; s++)
        for (int q = 0; q < pt; q++) {
            real L = 1.0;
            for (int r = 0; r < pt; r++)
                if (r != q) L *= (O->tu[s] - O->tq[r]) / (O->tq[q] - O->tq[r]);
            O->Lup[s * pt + q] = L;
        }
    /* node interpolant: l_i(u,v) = psi(u,v)^T Vd^{-1}, Vd[i][b] = psi_b(node i) */
    real *Vd = malloc(sizeof(real) * np * np);
    int *pv = malloc(sizeof(int) * np);
    for (int i = 0; i < np; i++) dubiner(p - 1, ref_uv[2 * i], ref_uv[2 * i + 1], Vd + i * np);
    /* transpose so that we solve Vd^T X = psi(pt) -> X[i] = l_i(pt) */
    real *VdT = malloc(sizeof(real) * np * np);
    for (int i = 0; i < np; i++)
        for (int b = 0; b < np; b++) VdT[b * np + i] = Vd[i * np + b];
    if (lu_factor(np, VdT, pv)) { free(Vd); free(VdT); free(pv); return -1; }
    int nsamp = 3 * pt + 3;
    real *B = malloc(sizeof(real) * np * nsamp);
    real psi[ORC_PMAX * ORC_PMAX];
    for (int e = 0; e < 3; e++)
        for (int q = 0; q < pt; q++) {
            real u, v;
            edge_uv(e, O->tq[q], &u, &v);
            dubiner(p - 1, u, v, psi);
            for (int b = 0; b < np; b++) B[b * nsamp + e * pt + q] = psi[b];
        }
    const real vtx[3][2] = {{0, 0}, {1, 0}, {0, 1}};
    for (int k = 0; k < 3; k++) {
        dubiner(p - 1, vtx[k][0], vtx[k][1], psi);
        for (int b = 0; b < np; b++) B[b * nsamp + 3 * pt + k] = psi[b];
    }
    lu_solve(np, VdT, pv, nsamp, B);
    O->Eint = malloc(sizeof(real) * 3 * pt * np);
    O->Vint = malloc(sizeof(real) * 3 * np);
    for (int s = 0; s < 3 * pt; s++)
        for (int i = 0; i < np; i++) O->Eint[s * np + i] = B[i * nsamp + s];
    for (int k = 0; k < 3; k++)
        for (int i = 0; i < np; i++) O->Vint[k * np + i] = B[i * nsamp + 3 * pt + k];
    free(B); free(Vd);
    O->VdLU = VdT;  /* kept for the node interpolant at arbitrary (u, v) */
    O->VdPiv = pv;
    return 0;
}

static void order_free(orc_order *O) {
    free(O->Eint);
    free(O->Vint);
    free(O->VdLU);
    free(O->VdPiv);
    O->Eint = O->Vint = O->VdLU = NULL;
    O->VdPiv = NULL;
}

/* ------------------------------------------------------------------------- */
/* Patch data (source-only Steps 1-3)                                         */
/* ------------------------------------------------------------------------- */

typedef struct {
    int p, np, pt, nh;       /* nh = (p+1)^2 harmonics of degree <= p */
    real c[3], R[3][3], s; /* y = s R^T (x - c); R columns e_x, e_y, e_z */
    real V[3][3];          /* vertices, global */
    real cP[3], RP, dP;    /* near-list geometry (global) */
    real *y, *nu;          /* [np][3] local nodes and normals */
    real *ea;              /* [3][p][3] local Legendre coefficients of the edges */
    real *ey, *et;         /* [3*pt][3] local edge samples and tangents dy/dt */
    cplx *eg;                /* [3*pt][nh][3] grad S^{(j,k)} at edge samples */
    cplx *eh;                /* [3*pt][nh][3] (Hess S^{(j,k)}) tau at edge samples */
    real *XD, *XSp, *XS1, *XS2; /* fit matrices */
    real kappa1;           /* 1-norm condition number of the fit matrix A (Sec. 5.1) */
    int ok;
} orc_patch;

static void legendre_real(int n, real t, real *P, real *dP) {
    P[0] = 1.0; dP[0] = 0.0;
    if (n > 1) { P[1] = t; dP[1] = 1.0; }
    for (int k = 1; k + 1 < n; k++) {
        P[k + 1] = ((2 * k + 1) * t * P[k] - k * P[k - 1]) / (k + 1);
        dP[k + 1] = t * dP[k] + (k + 1) * P[k];
    }
}

static void legendre_cplx(int n, cplx t, cplx *P, cplx *dP) {
    P[0] = 1.0; dP[0] = 0.0;
    if (n > 1) { P[1] = t; dP[1] = 1.0; }
    for (int k = 1; k + 1 < n; k++) {
        P[k + 1] = ((2 * k + 1) * t * P[k] - k * P[k - 1]) / (k + 1);
        dP[k + 1] = t * dP[k] + (k + 1) * P[k];
    }
}

/* edge curve (local coordinates) and its derivative at real t */
static void edge_eval(const real *ea, int p, real t, real y[3], real dy[3]) {
    real P[ORC_PMAX], dP[ORC_PMAX];
    legendre_real(p, t, P, dP);
    for (int a = 0; a < 3; a++) {
        y[a] = 0; dy[a] = 0;
        for (int n = 0; n < p; n++) { y[a] += ea[n * 3 + a] * P[n]; dy[a] += ea[n * 3 + a] * dP[n]; }
    }
}

static void cross3(const real a[3], const real b[3], real c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static real dot3(const real a[3], const real b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void patch_free(orc_patch *P) {
    free(P->y); free(P->nu); free(P->ea); free(P->ey); free(P->et);
    free(P->eg); free(P->eh);
    free(P->XD); free(P->XSp); free(P->XS1); free(P->XS2);
    memset(P, 0, sizeof(*P));
}

static int patch_setup(orc_patch *P, const orc_order *O, const double *xyz, const double *nrm, int want_kappa) {
    lowdeg_init();
    memset(P, 0, sizeof(*P));
    int p = O->p, np = O->np, pt = O->pt;
    P->p = p; P->np = np; P->pt = pt; P->nh = NHFULL(p);
    int nh = P->nh;
    /* vertices and global edge samples through the node interpolant */
    for (int k = 0; k < 3; k++)
        for (int a = 0; a < 3; a++) {
            real s = 0;
            for (int i = 0; i < np; i++) s += O->Vint[k * np + i] * xyz[3 * i + a];
            P->V[k][a] = s;
        }
    real *gsamp = malloc(sizeof(real) * 3 * pt * 3);
    for (int sI = 0; sI < 3 * pt; sI++)
        for (int a = 0; a < 3; a++) {
            real s = 0;
            for (int i = 0; i < np; i++) s += O->Eint[sI * np + i] * xyz[3 * i + a];
            gsamp[sI * 3 + a] = s;
        }
    /* frame (Sec. 4 input/output; Sec. 5.1 scaling) */
    real e01[3], e12[3], e20[3], e02[3], nz[3];
    for (int a = 0; a < 3; a++) {
        P->c[a] = (P->V[0][a] + P->V[1][a] + P->V[2][a]) / 3.0;
        e01[a] = P->V[1][a] - P->V[0][a];
        e12[a] = P->V[2][a] - P->V[1][a];
        e20[a] = P->V[0][a] - P->V[2][a];
        e02[a] = P->V[2][a] - P->V[0][a];
    }
    cross3(e01, e02, nz);
    real nzl = xsqrt(dot3(nz, nz));
    if (!(nzl > 0)) { free(gsamp); return -1; }
    real L0 = xsqrt(dot3(e01, e01)), L1 = xsqrt(dot3(e12, e12)), L2 = xsqrt(dot3(e20, e20));
    const real *ex_src = e01;
    real Lm = L0;
    if (L1 > Lm) { Lm = L1; ex_src = e12; }
    if (L2 > Lm) { Lm = L2; ex_src = e20; }
    real ex[3], ey[3], ez[3];
    for (int a = 0; a < 3; a++) { ez[a] = nz[a] / nzl; ex[a] = ex_src[a] / Lm; }
    cross3(ez, ex, ey);
    for (int a = 0; a < 3; a++) { P->R[a][0] = ex[a]; P->R[a][1] = ey[a]; P->R[a][2] = ez[a]; }
    P->s = 1.0 / Lm;
    /* near-list geometry (global): c_P = vertex mean, R_P = max distance to nodes
       and vertices, d_P = longest edge */
    for (int a = 0; a < 3; a++) P->cP[a] = P->c[a];
    P->dP = Lm;
    real rp = 0;
    for (int i = 0; i < np; i++) {
        real d[3] = {xyz[3 * i] - P->cP[0], xyz[3 * i + 1] - P->cP[1], xyz[3 * i + 2] - P->cP[2]};
        real r = xsqrt(dot3(d, d));
        if (r > rp) rp = r;
    }
    for (int k = 0; k < 3; k++) {
        real d[3] = {P->V[k][0] - P->cP[0], P->V[k][1] - P->cP[1], P->V[k][2] - P->cP[2]};
        real r = xsqrt(dot3(d, d));
        if (r > rp) rp = r;
    }
    P->RP = rp;
    /* local nodes and normals */
    P->y = malloc(sizeof(real) * np * 3);
    P->nu = malloc(sizeof(real) * np * 3);
    for (int i = 0; i < np; i++)
        for (int b = 0; b < 3; b++) {
            real sy = 0, sn = 0;
            for (int a = 0; a < 3; a++) {
                sy += P->R[a][b] * (xyz[3 * i + a] - P->c[a]);
                sn += P->R[a][b] * nrm[3 * i + a];
            }
            P->y[3 * i + b] = P->s * sy;
            P->nu[3 * i + b] = sn;
        }
    /* local edge samples, Legendre coefficients a_n = (2n+1)/2 sum_q w_q y(t_q) P_n(t_q) */
    P->ey = malloc(sizeof(real) * 3 * pt * 3);
    P->et = malloc(sizeof(real) * 3 * pt * 3);
    P->ea = malloc(sizeof(real) * 3 * p * 3);
    for (int sI = 0; sI < 3 * pt; sI++)
        for (int b = 0; b < 3; b++) {
            real sy = 0;
            for (int a = 0; a < 3; a++) sy += P->R[a][b] * (gsamp[3 * sI + a] - P->c[a]);
            P->ey[3 * sI + b] = P->s * sy;
        }
    free(gsamp);
    for (int e = 0; e < 3; e++) {
        real *ea = P->ea + e * p * 3;
        for (int n = 0; n < p * 3; n++) ea[n] = 0.0;
        for (int q = 0; q < pt; q++) {
            real Pl[ORC_PMAX], dPl[ORC_PMAX];
            legendre_real(p, O->tq[q], Pl, dPl);
            for (int n = 0; n < p; n++)
                for (int b = 0; b < 3; b++)
                    ea[n * 3 + b] += 0.5 * (2 * n + 1) * O->wq[q] * P->ey[3 * (e * pt + q) + b] * Pl[n];
        }
        for (int q = 0; q < pt; q++) {
            real yy[3], dy[3];
            edge_eval(ea, p, O->tq[q], yy, dy);
            for (int b = 0; b < 3; b++) P->et[3 * (e * pt + q) + b] = dy[b];
        }
    }
    /* Step 3: harmonics at the edge samples */
    P->eg = malloc(sizeof(cplx) * 3 * pt * nh * 3);
    P->eh = malloc(sizeof(cplx) * 3 * pt * nh * 3);
    cplx *S = malloc(sizeof(cplx) * NHFULL(ORC_LMAX));
    for (int sI = 0; sI < 3 * pt; sI++) {
        solid_S(p, P->ey + 3 * sI, S);
        for (int j = 0; j <= p; j++)
            for (int k = -j; k <= j; k++) {
                cplx g[3], H[3][3];
                grad_S(S, p, j, k, g);
                hess_S(S, p, j, k, H);
                cplx *gg = P->eg + ((size_t)sI * nh + HIDX(j, k)) * 3;
                cplx *hh = P->eh + ((size_t)sI * nh + HIDX(j, k)) * 3;
                const real *tau = P->et + 3 * sI;
                for (int a = 0; a < 3; a++) {
                    gg[a] = g[a];
                    hh[a] = H[a][0] * tau[0] + H[a][1] * tau[1] + H[a][2] * tau[2];
                }
            }
    }
    /* Steps 1-2 (matrix-build variant): the system of eq. (dlpdensitylinearsystem2) */
    int n4 = 4 * np;
    real *F = malloc(sizeof(real) * 3 * np * np); /* F[a][i][lm] */
    real *Hn = malloc(sizeof(real) * np * np);
    for (int i = 0; i < np; i++) {
        solid_S(p, P->y + 3 * i, S);
        int lm = 0;
        for (int l = 1; l <= p; l++)
            for (int m = 1; m <= l; m++, lm++) {
                cplx g[3];
                grad_S(S, p, l, m, g);
                for (int a = 0; a < 3; a++) F[(a * np + i) * np + lm] = xsqrt(2.0) * xcimag(g[a]);
                Hn[i * np + lm] = xsqrt(2.0) * xcimag(S[HIDX(l, m)]);
            }
    }
    free(S);
    real *A = malloc(sizeof(real) * n4 * n4);
    memset(A, 0, sizeof(real) * n4 * n4);
#define AEL(bi, bj, i, j) A[((bi) * np + (i)) * n4 + (bj) * np + (j)]
#define FEL(a, i, j) F[((a) * np + (i)) * np + (j)]
    for (int i = 0; i < np; i++)
        for (int j = 0; j < np; j++) {
            real f1 = FEL(0, i, j), f2 = FEL(1, i, j), f3 = FEL(2, i, j);
            AEL(0, 1, i, j) = -f1; AEL(0, 2, i, j) = -f2; AEL(0, 3, i, j) = -f3;
            AEL(1, 0, i, j) = f1;  AEL(1, 2, i, j) = -f3; AEL(1, 3, i, j) = f2;
            AEL(2, 0, i, j) = f2;  AEL(2, 1, i, j) = f3;  AEL(2, 3, i, j) = -f1;
            AEL(3, 0, i, j) = f3;  AEL(3, 1, i, j) = -f2; AEL(3, 2, i, j) = f1;
        }
    /* ||A||_1 before factoring: largest column sum of |A| */
    real anorm = 0;
    for (int j = 0; j < n4; j++) {
        real cs = 0;
        for (int i = 0; i < n4; i++) cs += xfabs(A[i * n4 + j]);
        if (cs > anorm) anorm = cs;
    }
    int *piv = malloc(sizeof(int) * n4);
    int bad = lu_factor(n4, A, piv);
    /* kappa_1(A) = ||A||_1 ||A^{-1}||_1, the inverse from the LU factors */
    P->kappa1 = INFINITY;
    if (!bad && want_kappa) {
        real *Ainv = malloc(sizeof(real) * n4 * n4);
        memset(Ainv, 0, sizeof(real) * n4 * n4);
        for (int i = 0; i < n4; i++) Ainv[i * n4 + i] = 1.0;
        lu_solve(n4, A, piv, n4, Ainv);
        real inorm = 0;
        for (int j = 0; j < n4; j++) {
            real cs = 0;
            for (int i = 0; i < n4; i++) cs += xfabs(Ainv[i * n4 + j]);
            if (cs > inorm) inorm = cs;
        }
        P->kappa1 = anorm * inorm;
        free(Ainv);
    }
    P->XD = malloc(sizeof(real) * n4 * np);
    P->XSp = malloc(sizeof(real) * n4 * np);
    memset(P->XD, 0, sizeof(real) * n4 * np);
    memset(P->XSp, 0, sizeof(real) * n4 * np);
    for (int i = 0; i < np; i++) {
        P->XD[i * np + i] = 1.0;                          /* [I;0;0;0] */
        for (int a = 0; a < 3; a++) P->XSp[((a + 1) * np + i) * np + i] = P->nu[3 * i + a]; /* [0;diag nu] */
    }
    if (!bad) {
        lu_solve(n4, A, piv, np, P->XD);
        lu_solve(n4, A, piv, np, P->XSp);
    }
    /* scalar fit A_S = sum_a F_a diag(nu_a) (eq. slpdensitylinearsystem) */
    real *AS = malloc(sizeof(real) * np * np);
    for (int i = 0; i < np; i++)
        for (int j = 0; j < np; j++)
            AS[i * np + j] = FEL(0, i, j) * P->nu[3 * i] + FEL(1, i, j) * P->nu[3 * i + 1] + FEL(2, i, j) * P->nu[3 * i + 2];
    int *pivs = malloc(sizeof(int) * np);
    int bad2 = lu_factor(np, AS, pivs);
    P->XS1 = malloc(sizeof(real) * np * np);
    memset(P->XS1, 0, sizeof(real) * np * np);
    for (int i = 0; i < np; i++) P->XS1[i * np + i] = 1.0;
    if (!bad2) lu_solve(np, AS, pivs, np, P->XS1);
    /* X_S2 = X_D Hn A_S^{-1}: coefficients g of the intermediate density rho = Hn d */
    real *tmp = malloc(sizeof(real) * np * np);
    for (int i = 0; i < np; i++)
        for (int j = 0; j < np; j++) {
            real s = 0;
            for (int k = 0; k < np; k++) s += Hn[i * np + k] * P->XS1[k * np + j];
            tmp[i * np + j] = s;
        }
    P->XS2 = malloc(sizeof(real) * n4 * np);
    for (int r = 0; r < n4; r++)
        for (int j = 0; j < np; j++) {
            real s = 0;
            for (int k = 0; k < np; k++) s += P->XD[r * np + k] * tmp[k * np + j];
            P->XS2[r * np + j] = s;
        }
#undef AEL
#undef FEL
    free(tmp); free(AS); free(pivs); free(A); free(piv); free(F); free(Hn);
    P->ok = !(bad || bad2);
    return P->ok ? 0 : -2;
}

/* ------------------------------------------------------------------------- */
/* Step 5: root t0, SSQ moments, modified weights                             */
/* ------------------------------------------------------------------------- */

/* Newton on sum_a (y_a(t) - y'_a)^2 = 0 in complex t, started from the root of
 * the straight chord; Im t0 >= 0 is returned (roots come in conjugate pairs). */
static int edge_root(const real *ea, int p, const real yt[3], int maxit, cplx *t0) {
    real ym[3], yp[3], d1[3], d2[3];
    edge_eval(ea, p, -1.0, ym, d1);
    edge_eval(ea, p, 1.0, yp, d2);
    real c[3], b[3], w[3], bw[3];
    for (int a = 0; a < 3; a++) { c[a] = 0.5 * (yp[a] + ym[a]); b[a] = 0.5 * (yp[a] - ym[a]); w[a] = yt[a] - c[a]; }
    cross3(b, w, bw);
    real bb = dot3(b, b);
    cplx t = (dot3(b, w) + I * xsqrt(dot3(bw, bw))) / bb;
    int conv = 0;
    for (int it = 0; it < maxit; it++) {
        cplx P[ORC_PMAX], dP[ORC_PMAX];
        legendre_cplx(p, t, P, dP);
        cplx g = 0, gp = 0;
        for (int a = 0; a < 3; a++) {
            cplx y = 0, dy = 0;
            for (int n = 0; n < p; n++) { y += ea[n * 3 + a] * P[n]; dy += ea[n * 3 + a] * dP[n]; }
            cplx r = y - yt[a];
            g += r * r;
            gp += 2.0 * r * dy;
        }
        if (gp == 0.0) break;
        cplx dt = g / gp;
        t -= dt;
        real at = xcabs(t);
        if (xcabs(dt) <= 1e-14 * (at > 1.0 ? at : 1.0)) { conv = 1; break; }
    }
    if (xcimag(t) < 0) t = xconj(t);
    *t0 = t;
    return conv;
}

/* Bernstein-ellipse radius of z with respect to [-1,1] */
static real bernstein_rho(cplx z) {
    cplx w = z + xcsqrt(z - 1.0) * xcsqrt(z + 1.0);
    real r = xcabs(w);
    return r >= 1.0 ? r : 1.0 / r;
}

/* Moments I_i = int_{-1}^{1} t^i / ((t-t0)(t-conj t0))^{m/2} dt, m = 1 and 3,
 * by the recurrences obtained from integration by parts (Sec. 2.4). */
static void ssq_moments(int n, real a, real b, real *J, real *K) {
    real c0 = a * a + b * b;
    real sp = xsqrt((1 - a) * (1 - a) + b * b), sm = xsqrt((1 + a) * (1 + a) + b * b);
    J[0] = xasinh((1 - a) / b) + xasinh((1 + a) / b);
    if (n > 1) J[1] = (sp - sm) + a * J[0];
    for (int i = 2; i < n; i++) {
        real br = sp - ((i - 1) % 2 ? -sm : sm);
        J[i] = (br + (2 * i - 1) * a * J[i - 1] - (i - 1) * c0 * J[i - 2]) / i;
    }
    if (K) {
        K[0] = ((1 - a) / sp + (1 + a) / sm) / (b * b);
        if (n > 1) K[1] = (-1.0 / sp + 1.0 / sm) + a * K[0];
        for (int i = 0; i + 2 < n; i++) K[i + 2] = J[i] + 2 * a * K[i + 1] - c0 * K[i];
    }
}

/* Modified weights om[m-index][q] on one edge such that
 * int_{-1}^{1} f(t)/|y(t)-y'|^m dt ~ sum_q om[q] f(t_q) for smooth f. */
static void edge_weights(const orc_order *O, const real *ea, int p, const real *eyq,
                         const real yt[3], cplx t0, int use_ssq, int want3,
                         real *om1, real *om3) {
    int pt = O->pt;
    if (use_ssq) {
        real a = xcreal(t0), b = xcimag(t0);
        real J[ORC_PTMAX], K[ORC_PTMAX];
        ssq_moments(pt, a, b, J, want3 ? K : NULL);
        /* lambda = V^{-T} I for m = 1 and 3 */
        lu_solve(pt, O->VtLU, O->Vtpiv, 1, J);
        if (want3) lu_solve(pt, O->VtLU, O->Vtpiv, 1, K);
        for (int q = 0; q < pt; q++) {
            const real l1 = J[q], l3 = want3 ? K[q] : 0.0;
            real d[3] = {yt[0] - eyq[3 * q], yt[1] - eyq[3 * q + 1], yt[2] - eyq[3 * q + 2]};
            real rq = xsqrt(dot3(d, d));
            real ratio = xcabs(O->tq[q] - t0) / rq;
            om1[q] = l1 * ratio;
            if (want3) om3[q] = l3 * ratio * ratio * ratio;
        }
    } else {
        for (int q = 0; q < pt; q++) { om1[q] = 0; if (want3) om3[q] = 0; }
        for (int s = 0; s < O->nup; s++) {
            real y[3], dy[3];
            edge_eval(ea, p, O->tu[s], y, dy);
            real d[3] = {yt[0] - y[0], yt[1] - y[1], yt[2] - y[2]};
            real r = xsqrt(dot3(d, d));
            real k1 = O->wu[s] / r, k3 = k1 / (r * r);
            for (int q = 0; q < pt; q++) {
                om1[q] += k1 * O->Lup[s * pt + q];
                if (want3) om3[q] += k3 * O->Lup[s * pt + q];
            }
        }
    }
}

/* Omega_0 (eq. solidangle) and d Omega_0 / d nu' (eq. dprimelineintegrals) on one
 * edge by Gauss-Legendre panels graded geometrically toward Re t0. */
static void omega0_edge(const orc_order *O, const real *ea, int p, const real yt[3],
                        const real u[3], cplx t0, int have_root, const real *nut,
                        real *Om0, real *dOm0) {
    real c, sig;
    if (have_root) {
        c = xcreal(t0);
        if (c < -1) c = -1;
        if (c > 1) c = 1;
        sig = xcabs(t0 - c);
        if (sig < 1e-14) sig = 1e-14;
    } else { c = 0; sig = 4.0; }
    real br[256];
    int nb = 0;
    /* breakpoints: left side descending, then inner panel, right side */
    real left[128], right[128];
    int nl = 0, nr = 0;
    real lo = c - 0.5 * sig, hi = c + 0.5 * sig;
    if (lo < -1) lo = -1;
    if (hi > 1) hi = 1;
    real x = hi, len = sig;
    while (x < 1.0 && nr < 127) { real nx = x + len; if (nx > 1) nx = 1; right[nr++] = nx; x = nx; len *= 2; }
    x = lo; len = sig;
    while (x > -1.0 && nl < 127) { real nx = x - len; if (nx < -1) nx = -1; left[nl++] = nx; x = nx; len *= 2; }
    for (int i = nl - 1; i >= 0; i--) br[nb++] = left[i];
    br[nb++] = lo;
    br[nb++] = hi;
    for (int i = 0; i < nr; i++) br[nb++] = right[i];
    real s0 = 0, s1 = 0;
    for (int k = 0; k + 1 < nb; k++) {
        real a0 = br[k], a1 = br[k + 1];
        if (!(a1 > a0)) continue;
        real mid = 0.5 * (a0 + a1), half = 0.5 * (a1 - a0);
        for (int g = 0; g < ORC_NOM; g++) {
            real t = mid + half * O->tom[g];
            real y[3], tau[3];
            edge_eval(ea, p, t, y, tau);
            real d[3] = {yt[0] - y[0], yt[1] - y[1], yt[2] - y[2]};
            real r = xsqrt(dot3(d, d));
            real E = r + dot3(u, d);
            real dxu[3];
            cross3(d, u, dxu);
            real N = dot3(dxu, tau);
            real wgt = half * O->wom[g];
            s0 -= wgt * N / (r * E);
            if (dOm0) {
                real nxu[3];
                cross3(nut, u, nxu);
                real nd = dot3(nut, d), nu_u = dot3(nut, u);
                real v = dot3(nxu, tau) / (r * E) - nu_u * N / (r * E * E) - nd * N / (r * r * E * E)
                           - nd * N / (r * r * r * E);
                s1 -= wgt * v;
            }
        }
    }
    *Om0 += s0;
    if (dOm0) *dOm0 += s1;
}

/* ------------------------------------------------------------------------- */
/* Steps 4-8 for one (target, patch) pair                                     */
/* ------------------------------------------------------------------------- */

/* Node interpolant of patch P at (u, v) in the local frame: X = sum_i l_i(u,v) y_i,
 * the Lagrange functions l_i from the Dubiner basis and the nodes' Vandermonde. */
static void node_interp(const orc_order *O, const orc_patch *P, real u, real v, real X[3]) {
    real psi[ORC_PMAX * ORC_PMAX];
    dubiner(P->p - 1, u, v, psi);
    lu_solve(P->np, O->VdLU, O->VdPiv, 1, psi);
    X[0] = X[1] = X[2] = 0.0;
    for (int i = 0; i < P->np; i++)
        for (int a = 0; a < 3; a++) X[a] += psi[i] * P->y[3 * i + a];
}

/* Side of the patch on which the target lies, seen along the frame axis e_z.  The
 * point of the patch with the target's in-plane coordinates (its footprint) is found
 * by Newton on the in-plane part of the node interpolant, from the target's
 * barycentric coordinates in the projected vertex triangle (finite-difference
 * Jacobian).  Returns +1 if the footprint lies in the patch and the target is on or
 * above it, -1 if below it, 0 if the footprint is outside the patch or Newton fails. */
static int footprint_side(const orc_order *O, const orc_patch *P, const real yt[3]) {
    real vx[3][3];
    for (int k = 0; k < 3; k++)
        for (int a = 0; a < 3; a++) {
            vx[k][a] = 0.0;
            for (int i = 0; i < P->np; i++) vx[k][a] += O->Vint[k * P->np + i] * P->y[3 * i + a];
        }
    real a11 = vx[1][0] - vx[0][0], a12 = vx[2][0] - vx[0][0];
    real a21 = vx[1][1] - vx[0][1], a22 = vx[2][1] - vx[0][1];
    real det = a11 * a22 - a12 * a21;
    if (det == 0.0) return 0;
    real rx = yt[0] - vx[0][0], ry = yt[1] - vx[0][1];
    real u = (a22 * rx - a12 * ry) / det, v = (a11 * ry - a21 * rx) / det;
    int conv = 0;
    for (int it = 0; it < 30; it++) {
        const real h = 1e-6;
        real X[3], Xup[3], Xum[3], Xvp[3], Xvm[3];
        node_interp(O, P, u, v, X);
        node_interp(O, P, u + h, v, Xup);
        node_interp(O, P, u - h, v, Xum);
        node_interp(O, P, u, v + h, Xvp);
        node_interp(O, P, u, v - h, Xvm);
        real j11 = (Xup[0] - Xum[0]) / (2 * h), j12 = (Xvp[0] - Xvm[0]) / (2 * h);
        real j21 = (Xup[1] - Xum[1]) / (2 * h), j22 = (Xvp[1] - Xvm[1]) / (2 * h);
        real dj = j11 * j22 - j12 * j21;
        if (dj == 0.0) break;
        real fx = X[0] - yt[0], fy = X[1] - yt[1];
        real du = (j22 * fx - j12 * fy) / dj, dv = (j11 * fy - j21 * fx) / dj;
        u -= du;
        v -= dv;
        if (xfabs(du) + xfabs(dv) <= 1e-14 * (1.0 + xfabs(u) + xfabs(v))) { conv = 1; break; }
    }
    if (!conv) return 0;
    const real tol = 1e-12;
    if (u < -tol || v < -tol || u + v > 1.0 + tol) return 0;
    real X[3];
    node_interp(O, P, u, v, X);
    return yt[2] >= X[2] ? 1 : -1;
}

/* Quantities of Steps 4-7 for one pair: per lm (1<=m<=l<=p, lm = l(l-1)/2+m-1)
 * B[lm][4] = int over dP of beta^{(l,m)} (Thm. dlp1form, eq. dlp1formrep2),
 * Psi[lm]  = int over dP of psi^{(l,m)} (Thm. cslp1form),
 * Bd[lm][4] = d B / d nu' (Sec. 3.7), Om = (Omega_0, Omega), dOm = d Om / d nu'. */
typedef struct {
    real B[ORC_PMAX * (ORC_PMAX + 1) / 2][4];
    real Bd[ORC_PMAX * (ORC_PMAX + 1) / 2][4];
    real Psi[ORC_PMAX * (ORC_PMAX + 1) / 2];
    real Om[4], dOm[4];
    real yt[3], nut[3];
    int flags;
} orc_forms;

static int pair_forms(const orc_order *O, const orc_patch *P, const orc_opts *opt,
                      const double xt[3], const double nt[3], int self_i, int want_dp, orc_forms *F) {
    int p = P->p, np = P->np, pt = P->pt, nh = P->nh;
    int flags = 0;
    /* target in local coordinates */
    real *yt = F->yt, *nut = F->nut;
    for (int b = 0; b < 3; b++) {
        real sy = 0, sn = 0;
        for (int a = 0; a < 3; a++) { sy += P->R[a][b] * (xt[a] - P->c[a]); sn += P->R[a][b] * nt[a]; }
        yt[b] = P->s * sy;
        nut[b] = sn;
    }
    /* Step 4: harmonics at the target */
    cplx St[NHFULL(ORC_PMAX)];
    solid_S(p, yt, St);
    cplx gSt[NHFULL(ORC_PMAX)][3];
    cplx HSt[NHFULL(ORC_PMAX)][3][3];
    for (int l = 0; l <= p; l++)
        for (int m = -l; m <= l; m++) {
            grad_S(St, p, l, m, gSt[HIDX(l, m)]);
            if (want_dp) hess_S(St, p, l, m, HSt[HIDX(l, m)]);
        }
    /* choice of u (Thm. dlp1form): the half-line from the target along u must not meet
       the patch.  +e_z for a node of the patch (exterior limit); if the target's
       footprint along e_z lies in the patch, the side the target is on; otherwise the
       better of +-e_z by the smallest u.(r'-r)/|r'-r| over nodes and edge samples. */
    real u[3] = {0, 0, 1};
    const int side = self_i < 0 ? footprint_side(O, P, yt) : 0;
    if (side != 0) {
        u[2] = side;
    } else {
        real mplus = 2, mminus = 2;
        for (int s = 0; s < np + 3 * pt; s++) {
            const real *r = s < np ? P->y + 3 * s : P->ey + 3 * (s - np);
            real d[3] = {yt[0] - r[0], yt[1] - r[1], yt[2] - r[2]};
            real dl = xsqrt(dot3(d, d));
            if (dl == 0.0) continue;
            real cz = d[2] / dl;
            if (cz < mplus) mplus = cz;
            if (-cz < mminus) mminus = -cz;
        }
        if (self_i < 0 && mminus > mplus) u[2] = -1;
        real best = (u[2] > 0) ? mplus : mminus;
        if (best < -0.5) flags |= FLAG_UPOOR;
    }
    /* Steps 5-6: per-edge root, weights, line integrals (eqs. lineintegrals, solidangle,
       dprimelineintegrals) */
    static __thread cquat Q[NHFULL(ORC_PMAX)], dQ[NHFULL(ORC_PMAX)];
    cplx V[NHFULL(ORC_PMAX)];
    real Om0 = 0, dOm0 = 0, Omv[3] = {0, 0, 0}, dOmv[3] = {0, 0, 0};
    for (int h = 0; h < nh; h++) { Q[h] = cq_zero(); dQ[h] = cq_zero(); V[h] = 0; }
    for (int e = 0; e < 3; e++) {
        const real *ea = P->ea + e * p * 3;
        cplx t0;
        int conv = edge_root(ea, p, yt, (opt && opt->newton_max > 0) ? opt->newton_max : 30, &t0);
        if (!conv) flags |= FLAG_NEWTON;
        if (conv && xcimag(t0) < 1e-14 && xfabs(xcreal(t0)) <= 1.0) flags |= FLAG_ONEDGE;
        int use_ssq = conv && bernstein_rho(t0) < O->rho0 && xcimag(t0) > 0;
        real om1[ORC_PTMAX], om3[ORC_PTMAX];
        edge_weights(O, ea, p, P->ey + 3 * e * pt, yt, t0, use_ssq, want_dp, om1, om3);
        omega0_edge(O, ea, p, yt, u, t0, conv, nut, &Om0, want_dp ? &dOm0 : NULL);
        for (int q = 0; q < pt; q++) {
            int sI = e * pt + q;
            const real *yq = P->ey + 3 * sI, *tau = P->et + 3 * sI;
            real d[3] = {yt[0] - yq[0], yt[1] - yq[1], yt[2] - yq[2]};
            cquat qd = cq_rvec(d);
            cquat qn = cq_rvec(nut);
            real nd = dot3(nut, d);
            for (int a = 0; a < 3; a++) {
                Omv[a] -= om1[q] * tau[a];
                if (want_dp) dOmv[a] += om3[q] * nd * tau[a];
            }
            for (int j = 1; j <= p; j++)
                for (int k = -j; k <= j; k++) {
                    int h = HIDX(j, k);
                    const cplx *g = P->eg + ((size_t)sI * nh + h) * 3;
                    /* V^{jk}: ((r'-r) x grad S^{(j,k)}) . dr / |r'-r| */
                    cplx cx0 = d[1] * g[2] - d[2] * g[1];
                    cplx cx1 = d[2] * g[0] - d[0] * g[2];
                    cplx cx2 = d[0] * g[1] - d[1] * g[0];
                    V[h] += om1[q] * (cx0 * tau[0] + cx1 * tau[1] + cx2 * tau[2]);
                    if (j >= 2) {
                        /* Q^{jk}: (0, (r'-r)/|r'-r|)(0, d grad S^{(j,k)}), eq. (qjkdef2) */
                        const cplx *hh = P->eh + ((size_t)sI * nh + h) * 3;
                        cquat qh = cq_vec(hh);
                        cquat prod = cq_mul(qd, qh);
                        cq_axpy(&Q[h], om1[q], prod);
                        if (want_dp) {
                            cq_axpy(&dQ[h], om1[q], cq_mul(qn, qh));
                            cq_axpy(&dQ[h], -om3[q] * nd, prod);
                        }
                    }
                }
        }
    }
    F->Om[0] = Om0; F->dOm[0] = dOm0;
    for (int a = 0; a < 3; a++) { F->Om[a + 1] = Omv[a]; F->dOm[a + 1] = dOmv[a]; }
    /* Step 7: translations (eqs. cdlp1dintegral, cslp1formrep) and I[gamma] */
    const real inv4pi = 1.0 / (4.0 * R_PI), sq2 = xsqrt(2.0);
    int lm = 0;
    for (int l = 1; l <= p; l++)
        for (int m = 1; m <= l; m++, lm++) {
            cquat Ib = cq_zero(), dIb = cq_zero();
            cplx Ip = 0;
            for (int j = 1; j <= l; j++)
                for (int k = -j; k <= j; k++) {
                    real T = Tcoef(j, k, l, m);
                    if (T == 0.0) continue;
                    cplx Sv = Sget(St, p, l - j, m - k);
                    Ip += Dcoef(j, l) * V[HIDX(j, k)] * Sv * T;
                    if (j >= 2) {
                        real C = Ccoef(j, l);
                        cq_axpy(&Ib, C * Sv * T, Q[HIDX(j, k)]);
                        if (want_dp) {
                            cplx dS = 0;
                            if (abs(m - k) <= l - j) {
                                const cplx *gg = gSt[HIDX(l - j, m - k)];
                                dS = gg[0] * nut[0] + gg[1] * nut[1] + gg[2] * nut[2];
                            }
                            cq_axpy(&dIb, C * Sv * T, dQ[HIDX(j, k)]);
                            cq_axpy(&dIb, C * dS * T, Q[HIDX(j, k)]);
                        }
                    }
                }
            /* I[gamma] = (1/4pi) Omega (0, grad S(r')), eq. (gammalmdef) */
            cquat Om;
            Om.s = Om0;
            for (int a = 0; a < 3; a++) Om.v[a] = Omv[a];
            cquat Ig = cq_mul(Om, cq_vec(gSt[HIDX(l, m)]));
            F->B[lm][0] = sq2 * xcimag(inv4pi * (Ib.s + Ig.s));
            for (int a = 0; a < 3; a++) F->B[lm][a + 1] = sq2 * xcimag(inv4pi * (Ib.v[a] + Ig.v[a]));
            F->Psi[lm] = sq2 * xcimag(inv4pi * (Ip + St[HIDX(l, m)] * Om0));
            if (want_dp) {
                cquat dOm;
                dOm.s = dOm0;
                for (int a = 0; a < 3; a++) dOm.v[a] = dOmv[a];
                cplx Hn[3];
                for (int a = 0; a < 3; a++)
                    Hn[a] = HSt[HIDX(l, m)][a][0] * nut[0] + HSt[HIDX(l, m)][a][1] * nut[1] + HSt[HIDX(l, m)][a][2] * nut[2];
                cquat dIg = cq_mul(dOm, cq_vec(gSt[HIDX(l, m)]));
                cquat dIg2 = cq_mul(Om, cq_vec(Hn));
                F->Bd[lm][0] = sq2 * xcimag(inv4pi * (dIb.s + dIg.s + dIg2.s));
                for (int a = 0; a < 3; a++) F->Bd[lm][a + 1] = sq2 * xcimag(inv4pi * (dIb.v[a] + dIg.v[a] + dIg2.v[a]));
            }
        }
    F->flags = flags;
    return flags;
}

/* rows: [4][np] for S, D, S', D' (entries of kernels in mask written).
 * Returns flag bits. self_i = local node index of the target in the patch or -1. */
static int pair_rows(const orc_order *O, const orc_patch *P, const orc_opts *opt,
                     const double xt[3], const double nt[3], int self_i, unsigned mask,
                     const double *xyz, const double *nrm, const double *wts, real *rows) {
    int p = P->p, np = P->np;
    orc_forms F;
    int flags = pair_forms(O, P, opt, xt, nt, self_i, (mask & ORC_DP) != 0, &F);
    const real *nut = F.nut;
    const real inv4pi = 1.0 / (4.0 * R_PI);
    real *rS = rows, *rD = rows + np, *rSp = rows + 2 * np, *rDp = rows + 3 * np;
    real L = 1.0 / P->s;
    for (int i = 0; i < 4 * np; i++) rows[i] = 0;
    /* Step 8, matrix-build variant: row = [w^T A^{-1}]_0 */
    int lm = 0;
    for (int l = 1; l <= p; l++)
        for (int m = 1; m <= l; m++, lm++) {
            const real *B = F.B[lm], *Bd = F.Bd[lm];
            real Psi = F.Psi[lm];
            real nB = nut[0] * B[1] + nut[1] * B[2] + nut[2] * B[3];
            real nxB[3];
            cross3(nut, B + 1, nxB);
            for (int i = 0; i < np; i++) {
                real xd[4], w[4], g[4];
                for (int c = 0; c < 4; c++) {
                    xd[c] = P->XD[(size_t)(c * np + lm) * np + i];
                    w[c] = P->XSp[(size_t)(c * np + lm) * np + i];
                    g[c] = P->XS2[(size_t)(c * np + lm) * np + i];
                }
                /* D = -sum_lm [B c]_0 (eq. dlp1formrep) */
                if (mask & ORC_D) rD[i] -= B[0] * xd[0] - B[1] * xd[1] - B[2] * xd[2] - B[3] * xd[3];
                /* D' = d/d nu' of the D expression, scaled back by s (Sec. 3.7) */
                if (mask & ORC_DP) rDp[i] -= P->s * (Bd[0] * xd[0] - Bd[1] * xd[1] - Bd[2] * xd[2] - Bd[3] * xd[3]);
                /* S' = -[(0,nu') sum B w]_0 with (0, sigma nu) fitted (Sec. 3.6) */
                if (mask & ORC_SP)
                    rSp[i] += nB * w[0] + (B[0] * nut[0] + nxB[0]) * w[1] + (B[0] * nut[1] + nxB[1]) * w[2]
                              + (B[0] * nut[2] + nxB[2]) * w[3];
                /* S = sum Psi d - [B g]_0 (eq. slp1formrep), scaled back by L */
                if (mask & ORC_S)
                    rS[i] += L * (Psi * P->XS1[(size_t)lm * np + i] - (B[0] * g[0] - B[1] * g[1] - B[2] * g[2] - B[3] * g[3]));
            }
        }
    /* jump to the principal value on self pairs; smooth-rule subtraction */
    if (self_i >= 0) {
        if (mask & ORC_D) rD[self_i] -= 0.5;
        if (mask & ORC_SP) rSp[self_i] += 0.5;
    }
    const real ntr[3] = {nt[0], nt[1], nt[2]};
    for (int i = 0; i < np; i++) {
        if (i == self_i) continue;
        const real xs[3] = {xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]};
        const real ns[3] = {nrm[3 * i], nrm[3 * i + 1], nrm[3 * i + 2]};
        real d[3] = {xt[0] - xs[0], xt[1] - xs[1], xt[2] - xs[2]};
        real r2 = dot3(d, d), r = xsqrt(r2), r3 = r2 * r;
        real w = wts[i];
        if (mask & ORC_S) rS[i] -= w * inv4pi / r;
        if (mask & ORC_D) rD[i] -= w * inv4pi * dot3(d, ns) / r3;
        if (mask & ORC_SP) rSp[i] += w * inv4pi * dot3(d, ntr) / r3;
        if (mask & ORC_DP) rDp[i] -= w * inv4pi * (dot3(ntr, ns) / r3 - 3.0 * dot3(d, ns) * dot3(d, ntr) / (r3 * r2));
    }
    return flags;
}

/* ------------------------------------------------------------------------- */
/* Exported API (ctypes)                                                      */
/* ------------------------------------------------------------------------- */

typedef struct {
    int npatch;
    const int32_t *order;
    const int64_t *node_off;
    const double *xyz, *nrm, *wts;
    const double *ref_uv[ORC_PMAX + 1];
    orc_opts opt;
    orc_order ord[ORC_PMAX + 1];
    int have[ORC_PMAX + 1];
} orc_surface;

void *orc_surface_create(int npatch, const int32_t *order, const int64_t *node_off,
                         const double *xyz, const double *nrm, const double *wts,
                         const double **ref_uv /*[ORC_PMAX+1]*/, const orc_opts *opt) {
    binom_init();
    lowdeg_init();
    orc_surface *S = calloc(1, sizeof(orc_surface));
    S->npatch = npatch; S->order = order; S->node_off = node_off;
    S->xyz = xyz; S->nrm = nrm; S->wts = wts;
    if (opt) S->opt = *opt;
    for (int p = 0; p <= ORC_PMAX; p++) S->ref_uv[p] = ref_uv[p];
    for (int P = 0; P < npatch; P++) {
        int p = order[P];
        if (p < 1 || p > ORC_PMAX || !ref_uv[p]) { free(S); return NULL; }
        if (!S->have[p]) {
            if (order_init(&S->ord[p], p, ref_uv[p], &S->opt)) { free(S); return NULL; }
            S->have[p] = 1;
        }
    }
    return S;
}

void orc_surface_destroy(void *h) {
    orc_surface *S = h;
    if (!S) return;
    for (int p = 0; p <= ORC_PMAX; p++)
        if (S->have[p]) order_free(&S->ord[p]);
    free(S);
}

static int setup_patch_of(const orc_surface *S, int P, orc_patch *pd, int want_kappa) {
    int p = S->order[P];
    int64_t o = S->node_off[P];
    return patch_setup(pd, &S->ord[p], S->xyz + 3 * o, S->nrm + 3 * o, want_kappa);
}

/* Near test (global coordinates): |x_t - c_P| <= R_P + eta d_P, self always. */
static int is_near(const orc_patch *pd, const double *xt, real eta) {
    real d[3] = {xt[0] - pd->cP[0], xt[1] - pd->cP[1], xt[2] - pd->cP[2]};
    return xsqrt(dot3(d, d)) <= pd->RP + eta * pd->dP;
}

/* Geometry of every patch (c_P, R_P, d_P) -> out[npatch][5]. */
int orc_patch_bounds(void *h, double *out) {
    orc_surface *S = h;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : err)
    for (int P = 0; P < S->npatch; P++) {
        orc_patch pd;
        /* cheap: only the interpolated vertices and nodes are needed here */
        int p = S->order[P];
        const orc_order *O = &S->ord[p];
        int64_t o = S->node_off[P];
        const double *xyz = S->xyz + 3 * o;
        memset(&pd, 0, sizeof(pd));
        real V[3][3];
        for (int k = 0; k < 3; k++)
            for (int a = 0; a < 3; a++) {
                real s = 0;
                for (int i = 0; i < O->np; i++) s += O->Vint[k * O->np + i] * xyz[3 * i + a];
                V[k][a] = s;
            }
        real c[3], L = 0;
        for (int a = 0; a < 3; a++) c[a] = (V[0][a] + V[1][a] + V[2][a]) / 3.0;
        for (int k = 0; k < 3; k++) {
            real e[3] = {V[(k + 1) % 3][0] - V[k][0], V[(k + 1) % 3][1] - V[k][1], V[(k + 1) % 3][2] - V[k][2]};
            real l = xsqrt(dot3(e, e));
            if (l > L) L = l;
        }
        real rp = 0;
        for (int i = 0; i < O->np; i++) {
            real d[3] = {xyz[3 * i] - c[0], xyz[3 * i + 1] - c[1], xyz[3 * i + 2] - c[2]};
            real r = xsqrt(dot3(d, d));
            if (r > rp) rp = r;
        }
        for (int k = 0; k < 3; k++) {
            real d[3] = {V[k][0] - c[0], V[k][1] - c[1], V[k][2] - c[2]};
            real r = xsqrt(dot3(d, d));
            if (r > rp) rp = r;
        }
        out[5 * P] = c[0]; out[5 * P + 1] = c[1]; out[5 * P + 2] = c[2];
        out[5 * P + 3] = rp; out[5 * P + 4] = L;
        (void)pd;
    }
    return err;
}

/* Near lists for the targets in tsel[nsel] by brute force over all patches.
 * Pass 1 (pairs == NULL): counts[nsel].  Pass 2: pairs filled row by row with
 * ascending patch ids (offsets = exclusive scan of counts). */
int orc_near(void *h, int64_t nsel, const int64_t *tsel, const double *txyz, const int64_t *tself,
             int64_t *counts, const int64_t *offs, int32_t *pairs) {
    orc_surface *S = h;
    real eta = S->opt.eta > 0 ? S->opt.eta : 1.0;
    double *bd = malloc(sizeof(double) * 5 * S->npatch);
    orc_patch_bounds(h, bd);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < nsel; r++) {
        int64_t t = tsel[r];
        const double *xt = txyz + 3 * t;
        int64_t cnt = 0;
        int64_t sn = tself ? tself[t] : -1;
        for (int P = 0; P < S->npatch; P++) {
            real d[3] = {xt[0] - bd[5 * P], xt[1] - bd[5 * P + 1], xt[2] - bd[5 * P + 2]};
            int nearp = xsqrt(dot3(d, d)) <= bd[5 * P + 3] + eta * bd[5 * P + 4];
            if (sn >= S->node_off[P] && sn < S->node_off[P + 1]) nearp = 1;
            if (nearp) {
                if (pairs) pairs[offs[r] + cnt] = P;
                cnt++;
            }
        }
        if (!pairs) counts[r] = cnt;
    }
    free(bd);
    (void)is_near;
    return 0;
}

/* Correction rows for explicit pairs.  pair_t[npair] (target index), pair_P[npair]
 * (patch).  vals: for kernel slot k (S, D, S', D' = 0..3) rows are written at
 * vals[k][val_off[n] .. + n_p).  flags[npair]. */
int orc_rows(void *h, int64_t npair, const int64_t *pair_t, const int32_t *pair_P,
             const double *txyz, const double *tnrm, const int64_t *tself, unsigned mask,
             const int64_t *val_off, double *valS, double *valD, double *valSp, double *valDp,
             int32_t *flags) {
    orc_surface *S = h;
    /* group pairs by patch: order by patch id (counting sort) */
    int64_t *cnt = calloc(S->npatch + 1, sizeof(int64_t));
    for (int64_t n = 0; n < npair; n++) cnt[pair_P[n] + 1]++;
    for (int P = 0; P < S->npatch; P++) cnt[P + 1] += cnt[P];
    int64_t *ord = malloc(sizeof(int64_t) * (npair > 0 ? npair : 1));
    int64_t *fill = malloc(sizeof(int64_t) * (S->npatch + 1));
    memcpy(fill, cnt, sizeof(int64_t) * (S->npatch + 1));
    for (int64_t n = 0; n < npair; n++) ord[fill[pair_P[n]]++] = n;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
    for (int P = 0; P < S->npatch; P++) {
        if (cnt[P + 1] == cnt[P]) continue;
        orc_patch pd;
        if (setup_patch_of(S, P, &pd, 0)) err |= 1;
        int p = S->order[P];
        const orc_order *O = &S->ord[p];
        int np = O->np;
        int64_t o = S->node_off[P];
        real rows[4 * ORC_PMAX * (ORC_PMAX + 1) / 2];
        for (int64_t k = cnt[P]; k < cnt[P + 1]; k++) {
            int64_t n = ord[k];
            int64_t t = pair_t[n];
            int self_i = -1;
            if (tself && tself[t] >= o && tself[t] < o + np) self_i = (int)(tself[t] - o);
            int f = pair_rows(O, &pd, &S->opt, txyz + 3 * t, tnrm + 3 * t, self_i, mask,
                              S->xyz + 3 * o, S->nrm + 3 * o, S->wts + o, rows);
            if (flags) flags[n] = f | (pd.ok ? 0 : FLAG_SINGULAR);
            int64_t vo = val_off[n];
            for (int i = 0; i < np; i++) {
                if ((mask & ORC_S) && valS) valS[vo + i] = rows[i];
                if ((mask & ORC_D) && valD) valD[vo + i] = rows[np + i];
                if ((mask & ORC_SP) && valSp) valSp[vo + i] = rows[2 * np + i];
                if ((mask & ORC_DP) && valDp) valDp[vo + i] = rows[3 * np + i];
            }
        }
        patch_free(&pd);
    }
    free(cnt); free(ord); free(fill);
    return err ? -1 : 0;
}

/* ------------------------------------------------------------------------- */
/* Internals exported for the oracle's own pin tests                          */
/* ------------------------------------------------------------------------- */

int orc_solid_S(int L, const double *y, double *out /*[(L+1)^2][2]*/) {
    binom_init();
    if (L > ORC_LMAX) return -1;
    cplx S[NHFULL(ORC_LMAX)];
    real yr[3] = {y[0], y[1], y[2]};
    solid_S(L, yr, S);
    for (int i = 0; i < NHFULL(L); i++) { out[2 * i] = xcreal(S[i]); out[2 * i + 1] = xcimag(S[i]); }
    return 0;
}

int orc_solid_R(int L, const double *xyz, double *out) {
    binom_init();
    if (L > ORC_LMAX) return -1;
    cplx R[NHFULL(ORC_LMAX)];
    solid_R(L, xyz[0], xyz[1], xyz[2], R);
    for (int i = 0; i < NHFULL(L); i++) { out[2 * i] = xcreal(R[i]); out[2 * i + 1] = xcimag(R[i]); }
    return 0;
}

/* grad and Hessian of S^{(l,m)} at y: g[3][2], H[3][3][2] */
int orc_grad_hess_S(int L, const double *y, int l, int m, double *g, double *H) {
    lowdeg_init();
    cplx S[NHFULL(ORC_LMAX)];
    real yr[3] = {y[0], y[1], y[2]};
    solid_S(L, yr, S);
    cplx gg[3], HH[3][3];
    grad_S(S, L, l, m, gg);
    hess_S(S, L, l, m, HH);
    for (int a = 0; a < 3; a++) {
        g[2 * a] = xcreal(gg[a]); g[2 * a + 1] = xcimag(gg[a]);
        for (int b = 0; b < 3; b++) { H[2 * (3 * a + b)] = xcreal(HH[a][b]); H[2 * (3 * a + b) + 1] = xcimag(HH[a][b]); }
    }
    return 0;
}

double orc_T(int j, int k, int l, int m) { binom_init(); return Tcoef(j, k, l, m); }

int orc_gauss_legendre(int n, double *x, double *w) {
    if (n < 1 || n > 4 * ORC_PTMAX) return -1;
    real xr[4 * ORC_PTMAX], wr[4 * ORC_PTMAX];
    gauss_legendre(n, xr, wr);
    for (int i = 0; i < n; i++) { x[i] = xr[i]; w[i] = wr[i]; }
    return 0;
}

int orc_ssq_moments(int n, double a, double b, double *J, double *K) {
    if (n < 1 || n > 4 * ORC_PTMAX) return -1;
    real Jr[4 * ORC_PTMAX], Kr[4 * ORC_PTMAX];
    ssq_moments(n, a, b, Jr, K ? Kr : NULL);
    for (int i = 0; i < n; i++) { J[i] = Jr[i]; if (K) K[i] = Kr[i]; }
    return 0;
}

/* Singularity-swap weights on [-1, 1] for the pt Gauss-Legendre nodes: l1[q], l3[q] with
 * int f(t) / ((t - a)^2 + b^2)^{m/2} dt = sum_q l_m[q] f(t_q) for polynomials f of degree
 * < pt (m = 1, 3), lambda = V^{-T} I as in the edge rule. */
int orc_ssq_weights(int pt, double a, double b, double *l1, double *l3) {
    if (pt < 1 || pt > ORC_PTMAX) return -1;
    real tq[ORC_PTMAX], wq[ORC_PTMAX], lu[ORC_PTMAX * ORC_PTMAX], J[ORC_PTMAX], K[ORC_PTMAX];
    int piv[ORC_PTMAX];
    gauss_legendre(pt, tq, wq);
    if (vt_factor(pt, tq, lu, piv)) return -1;
    ssq_moments(pt, a, b, J, K);
    lu_solve(pt, lu, piv, 1, J);
    lu_solve(pt, lu, piv, 1, K);
    for (int q = 0; q < pt; q++) { l1[q] = J[q]; l3[q] = K[q]; }
    return 0;
}

int orc_bernstein_rho(double re, double im, double *rho) {
    *rho = bernstein_rho((real)re + I * (real)im);
    return 0;
}

int orc_lu_solve(int n, const double *A, int nrhs, double *B) {
    real *a = malloc(sizeof(real) * n * n);
    real *b = malloc(sizeof(real) * n * nrhs);
    int *piv = malloc(sizeof(int) * n);
    for (int i = 0; i < n * n; i++) a[i] = A[i];
    for (int i = 0; i < n * nrhs; i++) b[i] = B[i];
    int r = lu_factor(n, a, piv);
    if (!r) {
        lu_solve(n, a, piv, nrhs, b);
        for (int i = 0; i < n * nrhs; i++) B[i] = b[i];
    }
    free(a); free(b); free(piv);
    return r;
}

/* 1-norm condition number of patch P's fit matrix A (Sec. 5.1), or -1 on error */
double orc_patch_kappa(void *h, int P) {
    orc_surface *S = (orc_surface *)h;
    if (!S || P < 0 || P >= S->npatch) return -1.0;
    orc_patch pd;
    if (setup_patch_of(S, P, &pd, 1)) {
        patch_free(&pd);
        return -1.0;
    }
    const real k = pd.kappa1;
    patch_free(&pd);
    return k;
}

/* Patch internals for tests: frame[13] = c, R (row-major), s; vertices[9];
 * y[np*3]; ea[3*p*3]; ey[3*pt*3]; et[3*pt*3]; XD, XSp [4np*np], XS1 [np*np], XS2 [4np*np]. */
static void copy_out(double *dst, const real *src, size_t n) {
    if (dst)
        for (size_t i = 0; i < n; i++) dst[i] = src[i];
}

int orc_patch_internals(void *h, int P, double *frame, double *vert, double *y, double *ea,
                        double *ey, double *et, double *XD, double *XSp, double *XS1, double *XS2) {
    orc_surface *S = h;
    orc_patch pd;
    int r = setup_patch_of(S, P, &pd, 0);
    int np = pd.np, pt = pd.pt, p = pd.p;
    if (frame) {
        for (int a = 0; a < 3; a++) frame[a] = pd.c[a];
        for (int a = 0; a < 3; a++) for (int b = 0; b < 3; b++) frame[3 + 3 * a + b] = pd.R[a][b];
        frame[12] = pd.s;
    }
    if (vert) for (int k = 0; k < 3; k++) for (int a = 0; a < 3; a++) vert[3 * k + a] = pd.V[k][a];
    copy_out(y, pd.y, (size_t)np * 3);
    copy_out(ea, pd.ea, (size_t)3 * p * 3);
    copy_out(ey, pd.ey, (size_t)3 * pt * 3);
    copy_out(et, pd.et, (size_t)3 * pt * 3);
    copy_out(XD, pd.XD, (size_t)4 * np * np);
    copy_out(XSp, pd.XSp, (size_t)4 * np * np);
    copy_out(XS1, pd.XS1, (size_t)np * np);
    copy_out(XS2, pd.XS2, (size_t)4 * np * np);
    patch_free(&pd);
    return r;
}

/* Edge root for tests: returns converged flag; t0 as (re, im). */
int orc_edge_root(void *h, int P, int e, const double *yt, double *t0) {
    orc_surface *S = h;
    orc_patch pd;
    setup_patch_of(S, P, &pd, 0);
    cplx t;
    real yr[3] = {yt[0], yt[1], yt[2]};
    int c = edge_root(pd.ea + e * pd.p * 3, pd.p, yr, 30, &t);
    t0[0] = xcreal(t); t0[1] = xcimag(t);
    patch_free(&pd);
    return c;
}

/* Raw per-pair quantities for the Stokes-reduction pins: B^{lm} (4 reals per lm),
 * Psi^{lm}, dB^{lm} and Omega = (Omega0, Omega_vec), dOmega; target in global
 * coordinates.  Returns flags. */
int orc_pair_B(void *h, int P, const double *xt, const double *nt, int self_i,
               double *Bout, double *Psiout, double *dBout, double *Omout, double *dOmout) {
    orc_surface *S = h;
    orc_patch pd;
    if (setup_patch_of(S, P, &pd, 0)) { patch_free(&pd); return -1; }
    orc_forms F;
    int fl = pair_forms(&S->ord[pd.p], &pd, &S->opt, xt, nt, self_i, 1, &F);
    for (int lm = 0; lm < pd.np; lm++) {
        for (int c = 0; c < 4; c++) { Bout[4 * lm + c] = F.B[lm][c]; dBout[4 * lm + c] = F.Bd[lm][c]; }
        Psiout[lm] = F.Psi[lm];
    }
    for (int c = 0; c < 4; c++) { Omout[c] = F.Om[c]; dOmout[c] = F.dOm[c]; }
    patch_free(&pd);
    return fl;
}

/* H^{(l,m)} = sqrt2 Im S^{(l,m)} and grad H for 1 <= m <= l <= p at npts points
 * (basis order lm = l(l-1)/2 + m - 1): H[npts][np], gH[npts][np][3]. */
int orc_basis_batch(int p, int64_t npts, const double *y, double *H, double *gH) {
    lowdeg_init();
    int np = p * (p + 1) / 2;
    for (int64_t n = 0; n < npts; n++) {
        cplx S[NHFULL(ORC_LMAX)];
        real yr[3] = {y[3 * n], y[3 * n + 1], y[3 * n + 2]};
        solid_S(p, yr, S);
        int lm = 0;
        for (int l = 1; l <= p; l++)
            for (int m = 1; m <= l; m++, lm++) {
                cplx g[3];
                grad_S(S, p, l, m, g);
                H[n * np + lm] = xsqrt(2.0) * xcimag(S[HIDX(l, m)]);
                for (int a = 0; a < 3; a++) gH[(n * np + lm) * 3 + a] = xsqrt(2.0) * xcimag(g[a]);
            }
    }
    return 0;
}

/* Binary64 (0) or binary128 (1) arithmetic in this build. */
int orc_real_kind(void) { return sizeof(real) > sizeof(double) ? 1 : 0; }
