// Per-order constant tables of librrq, computed once per order on the host.
//
//  * Gauss-Legendre rules (edge nodes t_q, the upsampled rule, the Omega_0 panel rule);
//  * the reciprocal node differences of the dual Vandermonde solve that turns the
//    singularity-swap moments into weights (Sec. 3.4);
//  * Lup: Lagrange basis of the edge nodes at the upsampled nodes (barycentric form);
//  * Eint: the node interpolant evaluated at the edge samples and the vertices
//    (Koornwinder-Dubiner basis on the reference triangle, solved with complete
//    pivoting);
//  * Legendre tables for the edge coefficients;
//  * rrq_ref_nodes: a reference node set and its interpolatory weights for callers.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "rrq_internal.cuh"

namespace {

// Rotation of Rn_l^m (Rn_l^m = R_l^m / sqrt((l-m)!(l+m)!)) by +90 degrees about the Y axis:
// Rn_l^m(Ry(90) a) = sum_k Delta_{mk} Rn_l^k(a) with
//     Delta_{mk} = 2^{-l} sum_s (-1)^{k-m+s} binom(l+k, k-m+s) binom(l-k, s),
// Wigner's small-d formula at beta = pi/2 carried over to this normalisation (the
// half-angle powers all become 2^{-1/2}).  The sum is of integers below 2^53, so every
// entry is exact in double.  The -90 degree rotation is (-1)^{k-m} Delta_{mk}.  Both are
// stored folded for coefficient sets with c_{-k} = (-1)^k conj(c_k) (see OrderTables).
void rotation_tables(double *D) {
    long long bn[2 * RRQ_PMAX + 1][2 * RRQ_PMAX + 1];
    for (int n = 0; n <= 2 * RRQ_PMAX; n++)
        for (int k = 0; k <= 2 * RRQ_PMAX; k++)
            bn[n][k] = k == 0 ? 1 : (k > n ? 0 : bn[n - 1][k - 1] + (k <= n - 1 ? bn[n - 1][k] : 0));
    for (int l = 0; l <= RRQ_PMAX; l++) {
        auto delta = [&](int m, int k) {
            long long acc = 0;
            for (int s = 0; s <= l - k; s++) {
                const int a = k - m + s;
                if (a < 0 || a > l + k) continue;
                const long long t = bn[l + k][a] * bn[l - k][s];
                acc += ((k - m + s) & 1) ? -t : t;
            }
            return ldexp((double)acc, -l);
        };
        const int n1 = (l + 1) * (l + 1), n2 = l * l;
        double *Am = D + rot_off(l), *Bm = Am + n1, *Ap = Bm + n2, *Bp = Ap + n1;
        for (int sgn = 0; sgn < 2; sgn++) {
            double *A = sgn ? Ap : Am, *B = sgn ? Bp : Bm;
            auto d = [&](int m, int k) { return (sgn || !((k - m) & 1)) ? delta(m, k) : -delta(m, k); };
            for (int m = 0; m <= l; m++) {
                A[m * (l + 1)] = d(m, 0);
                for (int k = 1; k <= l; k++) {
                    const double pk = d(m, k), nk = (k & 1) ? -d(m, -k) : d(m, -k);
                    A[m * (l + 1) + k] = pk + nk;
                    if (m >= 1) B[(m - 1) * l + (k - 1)] = pk - nk;
                }
            }
        }
    }
}

// Gauss-Legendre on [-1,1]: Newton on P_n from Tricomi's initial approximation.
void gl_rule(int n, double *x, double *w) {
    for (int k = 1; k <= n; k++) {
        double th = M_PI * (4.0 * k - 1.0) / (4.0 * n + 2.0);
        double z = (1.0 - (n - 1.0) / (8.0 * n * n * n)) * cos(th);
        double dp = 0;
        for (int it = 0; it < 60; it++) {
            double pm = 1.0, pc = z;
            for (int j = 2; j <= n; j++) {
                double pn = ((2.0 * j - 1.0) * z * pc - (j - 1.0) * pm) / j;
                pm = pc;
                pc = pn;
            }
            if (n == 1) { pc = z; pm = 1.0; }
            dp = n * (pm - z * pc) / (1.0 - z * z);
            double dz = pc / dp;
            z -= dz;
            if (fabs(dz) <= 1e-17) break;
        }
        {
            double pm = 1.0, pc = z;
            for (int j = 2; j <= n; j++) {
                double pn = ((2.0 * j - 1.0) * z * pc - (j - 1.0) * pm) / j;
                pm = pc;
                pc = pn;
            }
            if (n == 1) { pc = z; pm = 1.0; }
            dp = n * (pm - z * pc) / (1.0 - z * z);
        }
        // ascending order
        x[n - k] = z;
        w[n - k] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

void legendre_vals(int n, double t, double *P, double *dP) {
    P[0] = 1.0;
    dP[0] = 0.0;
    if (n > 1) { P[1] = t; dP[1] = 1.0; }
    for (int k = 2; k < n; k++) {
        P[k] = ((2.0 * k - 1.0) * t * P[k - 1] - (k - 1.0) * P[k - 2]) / k;
        dP[k] = dP[k - 2] + (2.0 * k - 1.0) * P[k - 1];
    }
}

// Koornwinder-Dubiner basis of total degree <= deg at (u, v); ordering a-major.
void dubiner_basis(int deg, double u, double v, double *out) {
    const double xs = 2.0 * u - 1.0 + v, ws = 1.0 - v, eta = 2.0 * v - 1.0;
    double La[RRQ_PMAX + 2];
    La[0] = 1.0;
    if (deg >= 1) La[1] = xs;
    for (int a = 2; a <= deg; a++) La[a] = ((2.0 * a - 1.0) * xs * La[a - 1] - (a - 1.0) * ws * ws * La[a - 2]) / a;
    int idx = 0;
    for (int a = 0; a <= deg; a++) {
        const double al = 2.0 * a + 1.0;
        double Jb[RRQ_PMAX + 2];
        Jb[0] = 1.0;
        if (deg - a >= 1) Jb[1] = 0.5 * ((al + 2.0) * eta + al);
        for (int n = 2; n <= deg - a; n++) {
            // Jacobi P_n^{(al,0)} three-term recurrence
            double b = n - 1.0;
            double a1 = 2.0 * (b + 1.0) * (b + al + 1.0) * (2.0 * b + al);
            double a2 = (2.0 * b + al + 1.0) * al * al;
            double a3 = (2.0 * b + al) * (2.0 * b + al + 1.0) * (2.0 * b + al + 2.0);
            double a4 = 2.0 * (b + al) * b * (2.0 * b + al + 2.0);
            Jb[n] = ((a2 + a3 * eta) * Jb[n - 1] - a4 * Jb[n - 2]) / a1;
        }
        for (int b = 0; b <= deg - a; b++) out[idx++] = La[a] * Jb[b];
    }
}

// Solve M X = B (n x n, nrhs columns, row-major) by Gauss-Jordan with complete pivoting.
int solve_complete_pivot(int n, std::vector<double> M, int nrhs, std::vector<double> &B) {
    std::vector<int> colperm(n);
    for (int i = 0; i < n; i++) colperm[i] = i;
    for (int k = 0; k < n; k++) {
        int pr = k, pc = k;
        double best = -1;
        for (int i = k; i < n; i++)
            for (int j = k; j < n; j++)
                if (fabs(M[i * n + j]) > best) { best = fabs(M[i * n + j]); pr = i; pc = j; }
        if (best <= 0) return -1;
        if (pr != k) {
            for (int j = 0; j < n; j++) std::swap(M[k * n + j], M[pr * n + j]);
            for (int c = 0; c < nrhs; c++) std::swap(B[k * nrhs + c], B[pr * nrhs + c]);
        }
        if (pc != k) {
            for (int i = 0; i < n; i++) std::swap(M[i * n + k], M[i * n + pc]);
            std::swap(colperm[k], colperm[pc]);
        }
        double piv = M[k * n + k];
        for (int j = 0; j < n; j++) M[k * n + j] /= piv;
        for (int c = 0; c < nrhs; c++) B[k * nrhs + c] /= piv;
        for (int i = 0; i < n; i++) {
            if (i == k) continue;
            double f = M[i * n + k];
            if (f == 0.0) continue;
            for (int j = 0; j < n; j++) M[i * n + j] -= f * M[k * n + j];
            for (int c = 0; c < nrhs; c++) B[i * nrhs + c] -= f * B[k * nrhs + c];
        }
    }
    // undo the column permutation: unknown colperm[k] is row k of B
    std::vector<double> X(B.size());
    for (int k = 0; k < n; k++)
        for (int c = 0; c < nrhs; c++) X[colperm[k] * nrhs + c] = B[k * nrhs + c];
    B.swap(X);
    return 0;
}

}  // namespace

int rrq_host_order_tables(int p, int pt, double rho0, const double *ref_uv, OrderTables *T) {
    if (p < 2 || p > RRQ_PMAX || pt != 2 * p) return -1;
    memset(T, 0, sizeof(*T));
    T->p = p;
    T->np = p * (p + 1) / 2;
    T->pt = pt;
    T->nup = 2 * pt;
    T->njk = (p + 1) * (p + 2) / 2;
    T->rho0 = rho0 > 0 ? rho0 : pow(10.0, 5.0 / pt);
    gl_rule(pt, T->tq, T->wq);
    gl_rule(T->nup, T->tu, T->wu);
    gl_rule(RRQ_NOM, T->tom, T->wom);
    // reciprocal node differences of the dual Bjorck-Pereyra Vandermonde solve (rrq_pairs.cuh)
    for (int k = 0; k < pt; k++)
        for (int i = 0; i < pt; i++) T->BPr[k * pt + i] = (i > k) ? 1.0 / (T->tq[i] - T->tq[i - k - 1]) : 0.0;
    // Lup[s][q] by the barycentric formula
    std::vector<double> bw(pt);
    for (int q = 0; q < pt; q++) {
        double prod = 1.0;
        for (int r = 0; r < pt; r++)
            if (r != q) prod *= (T->tq[q] - T->tq[r]);
        bw[q] = 1.0 / prod;
    }
    for (int s = 0; s < T->nup; s++) {
        double x = T->tu[s], sum = 0;
        for (int q = 0; q < pt; q++) sum += bw[q] / (x - T->tq[q]);
        for (int q = 0; q < pt; q++) T->Lup[s * pt + q] = (bw[q] / (x - T->tq[q])) / sum;
    }
    // node interpolant at edge samples and vertices
    const int np = T->np, deg = p - 1;
    std::vector<double> V(np * np);  // V[b][i] = psi_b(node i)  (transposed Vandermonde)
    double psi[RRQ_NPMAX];
    for (int i = 0; i < np; i++) {
        dubiner_basis(deg, ref_uv[2 * i], ref_uv[2 * i + 1], psi);
        for (int b = 0; b < np; b++) V[b * np + i] = psi[b];
    }
    const int nrow = 3 * pt + 3;
    std::vector<double> R(np * nrow);  // R[b][row] = psi_b(sample row)
    for (int e = 0; e < 3; e++)
        for (int q = 0; q < pt; q++) {
            double s = 0.5 * (1.0 + T->tq[q]), u, v;
            if (e == 0) { u = s; v = 0.0; }
            else if (e == 1) { u = 1.0 - s; v = s; }
            else { u = 0.0; v = 1.0 - s; }
            dubiner_basis(deg, u, v, psi);
            for (int b = 0; b < np; b++) R[b * nrow + e * pt + q] = psi[b];
        }
    const double vtx[3][2] = {{0, 0}, {1, 0}, {0, 1}};
    for (int k = 0; k < 3; k++) {
        dubiner_basis(deg, vtx[k][0], vtx[k][1], psi);
        for (int b = 0; b < np; b++) R[b * nrow + 3 * pt + k] = psi[b];
    }
    if (solve_complete_pivot(np, V, nrow, R)) return -2;  // R[i][row] = l_i(sample row)
    for (int row = 0; row < nrow; row++)
        for (int i = 0; i < np; i++) T->Eint[row * np + i] = R[i * nrow + row];
    double P[RRQ_PMAX], dP[RRQ_PMAX];
    for (int q = 0; q < pt; q++) {
        legendre_vals(p, T->tq[q], P, dP);
        for (int n = 0; n < p; n++) {
            T->LegW[n * pt + q] = 0.5 * (2.0 * n + 1.0) * T->wq[q] * P[n];
            T->dLeg[q * p + n] = dP[n];
        }
    }
    for (int s = 0; s < T->nup; s++) {
        legendre_vals(p, T->tu[s], P, dP);
        for (int n = 0; n < p; n++) T->LegU[s * p + n] = P[n];
    }
    // the factors of the translated line integrals: C_{j,l} = int_0^1 t^{j-2} (1-t)^{l-j} dt
    // (Thm. dlp1form) and D_{j,l} = int_0^1 t^{j-1} (1-t)^{l-j} dt (Thm. cslp1form)
    {
        double f[2 * RRQ_PMAX + 2];
        f[0] = 1.0;
        for (int n = 1; n < 2 * RRQ_PMAX + 2; n++) f[n] = f[n - 1] * n;
        for (int l = 0; l <= RRQ_PMAX; l++)
            for (int j = 0; j <= RRQ_PMAX; j++) {
                const bool in = j >= 1 && j <= l;
                T->Djl[l * (RRQ_PMAX + 1) + j] = in ? f[j - 1] * f[l - j] / f[l] : 0.0;
                T->Cjl[l * (RRQ_PMAX + 1) + j] = (in && j >= 2) ? f[j - 2] * f[l - j] / f[l - 1] : 0.0;
            }
    }
    rotation_tables(T->Drot);
    // monomial coefficients of P_n by (n+1) P_{n+1} = (2n+1) t P_n - n P_{n-1}
    for (int i = 0; i < p * p; i++) T->L2M[i] = 0.0;
    T->L2M[0] = 1.0;
    if (p > 1) T->L2M[1 * p + 1] = 1.0;
    for (int n = 1; n + 1 < p; n++)
        for (int k = 0; k < p; k++) {
            double v = -(double)n * T->L2M[(n - 1) * p + k];
            if (k > 0) v += (2.0 * n + 1.0) * T->L2M[n * p + k - 1];
            T->L2M[(n + 1) * p + k] = v / (n + 1.0);
        }
    // monomial coefficients of the node Lagrange functions: Vm[i][ab] = u_i^a v_i^b, Mmon = Vm^{-1}
    {
        std::vector<double> Vm(np * np), I(np * np, 0.0);
        for (int i = 0; i < np; i++) {
            int ab = 0;
            for (int a = 0; a < p; a++)
                for (int b = 0; a + b < p; b++, ab++)
                    Vm[i * np + ab] = pow(ref_uv[2 * i], a) * pow(ref_uv[2 * i + 1], b);
            I[i * np + i] = 1.0;
        }
        if (solve_complete_pivot(np, Vm, np, I)) return -2;
        for (int i = 0; i < np * np; i++) T->Mmon[i] = I[i];
    }
    return 0;
}

extern "C" rrq_status rrq_ref_nodes(int32_t p, double *uv, double *w) {
    if (p < 2 || p > RRQ_PMAX || !uv) return RRQ_ERR_ARG;
    // 1-D Gauss-Legendre points on [0, 1], blended onto the triangle (i + j + k = p - 1)
    double x[RRQ_PMAX], xw[RRQ_PMAX], g[RRQ_PMAX];
    gl_rule(p, x, xw);
    for (int i = 0; i < p; i++) g[i] = 0.5 * (x[i] + 1.0);
    const int n = p - 1, np = p * (p + 1) / 2;
    int r = 0;
    for (int i = 0; i <= n; i++)
        for (int j = 0; j <= n - i; j++, r++) {
            const int k = n - i - j;
            uv[2 * r] = (1.0 + 2.0 * g[j] - g[i] - g[k]) / 3.0;
            uv[2 * r + 1] = (1.0 + 2.0 * g[k] - g[i] - g[j]) / 3.0;
        }
    if (!w) return RRQ_OK;
    // interpolatory weights: V^T w = moments in the orthogonal basis (1/2 for the constant)
    std::vector<double> VT(np * np), B(np, 0.0);
    double psi[RRQ_NPMAX];
    for (int i = 0; i < np; i++) {
        dubiner_basis(n, uv[2 * i], uv[2 * i + 1], psi);
        for (int b = 0; b < np; b++) VT[b * np + i] = psi[b];
    }
    B[0] = 0.5;
    if (solve_complete_pivot(np, VT, 1, B)) return RRQ_ERR_ARG;
    for (int i = 0; i < np; i++) w[i] = B[i];
    return RRQ_OK;
}
