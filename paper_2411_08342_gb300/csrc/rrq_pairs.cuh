// Per-pair (target, patch) work: Sec. 4 Steps 4-8 for S, D, S', D' in one pass.
// One warp per pair, pairs grouped by patch so the patch data stays in L2.
//
//   Step 4  harmonic table S^{(n,q)}(y'), its gradient (and Hessian for D') at the
//           target in the patch frame;
//   u       +e_z for a target that is a node of the patch, else the better of +-e_z
//           by min over nodes and edge samples of u.(y'-y)/|y'-y|;
//   Step 5  per edge: complex root t0 of |y(t)-y'|^2 (Newton from the chord root),
//           singularity-swap moments by recurrence and modified weights
//           lambda = U^T I (Sec. 2.4, 3.4), or an upsampled Gauss rule when t0 is
//           outside the Bernstein ellipse of radius rho0;
//           Omega_0 (eq. solidangle; its sign such that (1/4pi) d omega_0 =
//           -grad G . nu da as Thm. dlp1form requires) on Gauss panels graded toward
//           Re t0, and its nu' derivative (eq. dprimelineintegrals);
//   Step 6  Q^{(j,k)}, V^{(j,k)}, Omega (eqs. lineintegrals, qjkdef2) and for D' their
//           nu' derivatives, k >= 0 only (k < 0 by conjugation);
//   Step 7  translations (eqs. cdlp1dintegral, cslp1formrep) and I[gamma] (eq. gammalmdef);
//   Step 8  rows through the precomputed fit matrices (matrix-build remark of Sec. 4),
//           principal-value jump on self pairs, minus the smooth rule.
#pragma once
#include <math.h>

#include "rrq_internal.cuh"

namespace rrqk {

constexpr int WARPS = 4;

template <int P>
struct PairSm {
    static constexpr int NP = P * (P + 1) / 2, PT = 2 * P, NJK = (P + 1) * (P + 2) / 2, NS = 3 * PT, NUP = 2 * PT;
    static constexpr int YT = 0, NUT = 3, XT = 6, NT = 9, FR = 12;   // FR: 16
    static constexpr int EA = 28;                                     // 9P
    static constexpr int DQ = EA + 9 * P;                             // NS*3
    static constexpr int TAU = DQ + 3 * NS;                           // NS*3
    static constexpr int RINV = TAU + 3 * NS;                         // NS
    static constexpr int OM1 = RINV + NS;                             // NS
    static constexpr int OM3 = OM1 + NS;                              // NS
    static constexpr int MOM = OM3 + NS;                              // 3*2*PT
    static constexpr int UP = MOM + 6 * PT;                           // 2*NUP
    static constexpr int T0 = UP + 2 * NUP;                           // 3*4 (re, im, conv, ssq)
    static constexpr int ST = T0 + 12;                                // NJK complex
    static constexpr int GST = ST + 2 * NJK;                          // NJK*3 complex
    static constexpr int HST = GST + 6 * NJK;                         // NJK*6 complex
    static constexpr int Q = HST + 12 * NJK;                          // NJK*4 complex
    static constexpr int DQQ = Q + 8 * NJK;                           // NJK*4 complex
    static constexpr int V = DQQ + 8 * NJK;                           // NJK complex
    static constexpr int OM = V + 2 * NJK;                            // 8
    static constexpr int B = OM + 8;                                  // NP*4
    static constexpr int BD = B + 4 * NP;                             // NP*4
    static constexpr int PSI = BD + 4 * NP;                           // NP
    static constexpr int WV = PSI + NP;                               // NS*12 premultiplied sample vectors
    static constexpr int EM = WV + 12 * NS;                           // 3*P*3 monomial edge coefficients
    static constexpr int TOTAL = EM + 9 * P + 2;
};

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_min(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ cd sqrt_c(cd z) {
    double r = sqrt(z.x * z.x + z.y * z.y);
    double re = sqrt(fmax(0.5 * (r + z.x), 0.0));
    double im = sqrt(fmax(0.5 * (r - z.x), 0.0));
    return mkc(re, z.y < 0 ? -im : im);
}

// Table of Rn_n^q (0 <= q <= n <= P), column m = lane computed by the warp.
template <int P>
__device__ __forceinline__ void target_table(const double *y, cd *S, int lane) {
    if (lane <= P) {
        const double X = y[1], Y = y[2], Z = y[0], r2 = X * X + Y * Y + Z * Z;
        const int m = lane;
        cd w = mkc(1.0, 0.0);
        for (int k = 1; k <= m; k++) w = cscale(cmul(w, mkc(X, Y)), 1.0 / (2.0 * k));
        cd prev = mkc(0.0, 0.0), cur = w;
        S[jk_index(m, m)] = cur;
        for (int l = m; l < P; l++) {
            cd nxt = cscale(csub(cscale(cur, (2.0 * l + 1.0) * Z), cscale(prev, r2)), 1.0 / ((l - m + 1.0) * (l + m + 1.0)));
            S[jk_index(l + 1, m)] = nxt;
            prev = cur;
            cur = nxt;
        }
    }
}

__device__ __forceinline__ cd tget(const cd *S, int n, int q) {
    if (n < 0) return mkc(0, 0);
    int aq = q < 0 ? -q : q;
    if (aq > n) return mkc(0, 0);
    cd v = S[jk_index(n, aq)];
    if (q < 0) {
        v.y = -v.y;
        if (aq & 1) { v.x = -v.x; v.y = -v.y; }
    }
    return v;
}

// conjugation rule for k < 0 applied to a stored k >= 0 quantity
__device__ __forceinline__ cd kflip(cd v, int k) {
    if (k >= 0) return v;
    v.y = -v.y;
    if ((-k) & 1) { v.x = -v.x; v.y = -v.y; }
    return v;
}

// acc += a * b (complex), as four fused multiply-adds
__device__ __forceinline__ void cfma(cd &acc, const cd a, const cd b) {
    acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}

__device__ __forceinline__ void edge_eval_real(const double *ea, int p, double t, double y[3], double dy[3]) {
    double Pm = 1.0, Pc = t, dPm = 0.0, dPc = 1.0;
    for (int a = 0; a < 3; a++) { y[a] = ea[a]; dy[a] = 0.0; }
    if (p > 1)
        for (int a = 0; a < 3; a++) { y[a] += ea[3 + a] * t; dy[a] += ea[3 + a]; }
    for (int n = 1; n + 1 < p; n++) {
        double Pn = ((2.0 * n + 1.0) * t * Pc - n * Pm) / (n + 1.0);
        double dPn = dPm + (2.0 * n + 1.0) * Pc;
        for (int a = 0; a < 3; a++) { y[a] += ea[3 * (n + 1) + a] * Pn; dy[a] += ea[3 * (n + 1) + a] * dPn; }
        Pm = Pc; Pc = Pn; dPm = dPc; dPc = dPn;
    }
}

__device__ __forceinline__ void edge_eval_cplx(const double *ea, int p, cd t, cd y[3], cd dy[3]) {
    cd Pm = mkc(1, 0), Pc = t, dPm = mkc(0, 0), dPc = mkc(1, 0);
    for (int a = 0; a < 3; a++) { y[a] = mkc(ea[a], 0); dy[a] = mkc(0, 0); }
    if (p > 1)
        for (int a = 0; a < 3; a++) { y[a] = cadd(y[a], cscale(t, ea[3 + a])); dy[a].x += ea[3 + a]; }
    for (int n = 1; n + 1 < p; n++) {
        cd Pn = cscale(csub(cscale(cmul(t, Pc), 2.0 * n + 1.0), cscale(Pm, (double)n)), 1.0 / (n + 1.0));
        cd dPn = cadd(dPm, cscale(Pc, 2.0 * n + 1.0));
        for (int a = 0; a < 3; a++) {
            y[a] = cadd(y[a], cscale(Pn, ea[3 * (n + 1) + a]));
            dy[a] = cadd(dy[a], cscale(dPn, ea[3 * (n + 1) + a]));
        }
        Pm = Pc; Pc = Pn; dPm = dPc; dPc = dPn;
    }
}

template <int P>
__device__ void process_pair(const OrderTables *__restrict__ tab, const PairItem item, const PatchData &pd,
                             const int64_t *__restrict__ node_off, const double *__restrict__ xyz,
                             const double *__restrict__ nrm, const double *__restrict__ wts,
                             const double *__restrict__ txyz, const double *__restrict__ tnrm,
                             const int64_t *__restrict__ tself, uint32_t mask, int newton_max, double *vS,
                             double *vD, double *vSp, double *vDp, int32_t *col, double *sw, int lane,
                             unsigned int *bc) {
    using Z = PairSm<P>;
    constexpr int NP = Z::NP, PT = Z::PT, NJK = Z::NJK, NS = Z::NS, NUP = Z::NUP;
    const bool wantDP = (mask & RRQ_DP) != 0;
    const int pid = item.P;
    const int64_t t = item.t;
    const size_t ps = (size_t)pid;
    double *fr = sw + Z::FR, *yt = sw + Z::YT, *nut = sw + Z::NUT, *ea = sw + Z::EA;
    double *dq = sw + Z::DQ, *tau = sw + Z::TAU, *rinv = sw + Z::RINV, *om1 = sw + Z::OM1, *om3 = sw + Z::OM3;
    double *mom = sw + Z::MOM, *up = sw + Z::UP, *t0s = sw + Z::T0;
    cd *St = reinterpret_cast<cd *>(sw + Z::ST), *gSt = reinterpret_cast<cd *>(sw + Z::GST);
    cd *HSt = reinterpret_cast<cd *>(sw + Z::HST), *Qs = reinterpret_cast<cd *>(sw + Z::Q);
    cd *dQs = reinterpret_cast<cd *>(sw + Z::DQQ), *Vs = reinterpret_cast<cd *>(sw + Z::V);
    double *Om = sw + Z::OM, *Bs = sw + Z::B, *Bds = sw + Z::BD, *Psis = sw + Z::PSI;

    if (lane < 13) fr[lane] = pd.frame[ps * PD_FRAME + lane];
    if (lane < 3) { sw[Z::XT + lane] = txyz[3 * t + lane]; sw[Z::NT + lane] = tnrm[3 * t + lane]; }
    for (int w = lane; w < 9 * P; w += 32) ea[w] = pd.ea[ps * pd_ea() + w];
    __syncwarp();
    if (lane < 3) {
        double sy = 0, sn = 0;
        for (int a = 0; a < 3; a++) {
            sy += fr[3 + 3 * a + lane] * (sw[Z::XT + a] - fr[a]);
            sn += fr[3 + 3 * a + lane] * sw[Z::NT + a];
        }
        yt[lane] = fr[12] * sy;
        nut[lane] = sn;
    }
    const int64_t o = node_off[pid];
    int self_i = -1;
    if (tself) {
        int64_t sn = tself[t];
        if (sn >= o && sn < o + NP) self_i = (int)(sn - o);
    }
    __syncwarp();
    // edge samples: d = y' - y(t_q), tangent, 1/|d|
    for (int q = lane; q < NS; q += 32) {
        const double *ey = pd.ey + ps * pd_ey() + 3 * q;
        const double *et = pd.et + ps * pd_ey() + 3 * q;
        double d0 = yt[0] - ey[0], d1 = yt[1] - ey[1], d2 = yt[2] - ey[2];
        dq[3 * q] = d0; dq[3 * q + 1] = d1; dq[3 * q + 2] = d2;
        tau[3 * q] = et[0]; tau[3 * q + 1] = et[1]; tau[3 * q + 2] = et[2];
        rinv[q] = 1.0 / sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    }
    // Step 4: harmonics at the target
    target_table<P>(yt, St, lane);
    __syncwarp();
    for (int jk = lane; jk < NJK; jk += 32) {
        int j = 0;
        while (jk_index(j + 1, 0) <= jk) j++;
        int k = jk - jk_index(j, 0);
        cd a = tget(St, j - 1, k - 1), b = tget(St, j - 1, k + 1);
        gSt[3 * jk + 0] = tget(St, j - 1, k);
        gSt[3 * jk + 1] = cscale(csub(a, b), 0.5);
        gSt[3 * jk + 2] = cmuli(cscale(cadd(a, b), 0.5));
        if (wantDP) {
            cd r0 = tget(St, j - 2, k), rm1 = tget(St, j - 2, k - 1), rp1 = tget(St, j - 2, k + 1);
            cd rm2 = tget(St, j - 2, k - 2), rp2 = tget(St, j - 2, k + 2);
            cd *H = HSt + 6 * jk;
            H[0] = r0;
            H[1] = cscale(csub(rm1, rp1), 0.5);
            H[2] = cmuli(cscale(cadd(rm1, rp1), 0.5));
            H[3] = cscale(cadd(csub(rm2, cscale(r0, 2.0)), rp2), 0.25);
            H[4] = cmuli(cscale(csub(rm2, rp2), 0.25));
            H[5] = cscale(cadd(cadd(rm2, cscale(r0, 2.0)), rp2), -0.25);
        }
    }
    // choice of u among +-e_z
    double mplus = 2.0, mminus = 2.0;
    for (int s = lane; s < NP + NS; s += 32) {
        double dz, dl;
        if (s < NP) {
            const double *yn = pd.ynode + ps * pd_ynode() + 3 * s;
            double d0 = yt[0] - yn[0], d1 = yt[1] - yn[1];
            dz = yt[2] - yn[2];
            dl = sqrt(d0 * d0 + d1 * d1 + dz * dz);
        } else {
            int q = s - NP;
            dz = dq[3 * q + 2];
            dl = sqrt(dq[3 * q] * dq[3 * q] + dq[3 * q + 1] * dq[3 * q + 1] + dz * dz);
        }
        if (dl != 0.0) {
            double cz = dz / dl;
            mplus = fmin(mplus, cz);
            mminus = fmin(mminus, -cz);
        }
    }
    mplus = warp_min(mplus);
    mminus = warp_min(mminus);
    const double uz = (self_i < 0 && mminus > mplus) ? -1.0 : 1.0;
    unsigned int fl_upoor = ((uz > 0 ? mplus : mminus) < -0.5) ? 1u : 0u;
    // Step 5: roots and moments, one lane per edge
    if (lane < 3) {
        const int e = lane;
        const double *ce = ea + 9 * e * P / 3;  // ea laid [e][n][a]: offset e*P*3
        double ym[3], yp[3];
        for (int a = 0; a < 3; a++) {
            double sp = 0, sm = 0;
            for (int n = 0; n < P; n++) {
                sp += ce[3 * n + a];
                sm += ((n & 1) ? -1.0 : 1.0) * ce[3 * n + a];
            }
            yp[a] = sp;
            ym[a] = sm;
        }
        double c[3], b[3], w[3];
        for (int a = 0; a < 3; a++) { c[a] = 0.5 * (yp[a] + ym[a]); b[a] = 0.5 * (yp[a] - ym[a]); w[a] = yt[a] - c[a]; }
        double bw0 = b[1] * w[2] - b[2] * w[1], bw1 = b[2] * w[0] - b[0] * w[2], bw2 = b[0] * w[1] - b[1] * w[0];
        double bb = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
        cd tt = mkc((b[0] * w[0] + b[1] * w[1] + b[2] * w[2]) / bb, sqrt(bw0 * bw0 + bw1 * bw1 + bw2 * bw2) / bb);
        int conv = 0;
        // an edge whose chord root lies well outside the Bernstein ellipse rho0 takes the
        // upsampled rule whatever the exact root is: the root is not refined
        bool skip = false;
        {
            cd zm1 = mkc(tt.x - 1.0, tt.y), zp1 = mkc(tt.x + 1.0, tt.y);
            cd wv = cadd(tt, cmul(sqrt_c(zm1), sqrt_c(zp1)));
            double rc = sqrt(cabs2(wv));
            if (rc < 1.0) rc = 1.0 / rc;
            if (rc > 1.5 * tab->rho0 && tt.y > 0.0) { skip = true; conv = 1; }
        }
        for (int it = 0; it < (skip ? 0 : newton_max); it++) {
            cd y[3], dy[3];
            edge_eval_cplx(ce, P, tt, y, dy);
            cd g = mkc(0, 0), gp = mkc(0, 0);
            for (int a = 0; a < 3; a++) {
                cd r = mkc(y[a].x - yt[a], y[a].y);
                g = cadd(g, cmul(r, r));
                gp = cadd(gp, cscale(cmul(r, dy[a]), 2.0));
            }
            if (gp.x == 0.0 && gp.y == 0.0) break;
            cd dt = cdivz(g, gp);
            tt = csub(tt, dt);
            double at = sqrt(cabs2(tt));
            if (sqrt(cabs2(dt)) <= 1e-14 * (at > 1.0 ? at : 1.0)) { conv = 1; break; }
        }
        if (tt.y < 0) tt.y = -tt.y;
        // Bernstein radius
        cd zm1 = mkc(tt.x - 1.0, tt.y), zp1 = mkc(tt.x + 1.0, tt.y);
        cd wv = cadd(tt, cmul(sqrt_c(zm1), sqrt_c(zp1)));
        double rho = sqrt(cabs2(wv));
        if (rho < 1.0) rho = 1.0 / rho;
        int ssq = conv && rho < tab->rho0 && tt.y > 0.0;
        t0s[4 * e] = tt.x;
        t0s[4 * e + 1] = tt.y;
        t0s[4 * e + 2] = conv;
        t0s[4 * e + 3] = ssq;
        if (ssq) {
            const double a = tt.x, bi = tt.y, c0 = a * a + bi * bi;
            const double sp = sqrt((1 - a) * (1 - a) + bi * bi), sm = sqrt((1 + a) * (1 + a) + bi * bi);
            double *J = mom + 2 * PT * e, *K = J + PT;
            J[0] = asinh((1 - a) / bi) + asinh((1 + a) / bi);
            J[1] = (sp - sm) + a * J[0];
            for (int i = 2; i < PT; i++) {
                double br = ((i - 1) & 1) ? sp + sm : sp - sm;
                J[i] = (br + (2.0 * i - 1.0) * a * J[i - 1] - (i - 1.0) * c0 * J[i - 2]) / i;
            }
            if (wantDP) {
                K[0] = ((1 - a) / sp + (1 + a) / sm) / (bi * bi);
                K[1] = (1.0 / sm - 1.0 / sp) + a * K[0];
                for (int i = 0; i + 2 < PT; i++) K[i + 2] = J[i] + 2.0 * a * K[i + 1] - c0 * K[i];
            }
        }
    }
    __syncwarp();
    unsigned int fl_newton = 0, fl_onedge = 0, n_ssq = 0, n_far = 0;
    for (int e = 0; e < 3; e++) {
        const double tr = t0s[4 * e], ti = t0s[4 * e + 1];
        const int conv = (int)t0s[4 * e + 2], ssq = (int)t0s[4 * e + 3];
        if (!conv) fl_newton = 1;
        if (conv && ti < 1e-14 && fabs(tr) <= 1.0) fl_onedge = 1;
        if (ssq) {
            n_ssq++;
            if (lane < PT) {
                const double *J = mom + 2 * PT * e, *K = J + PT;
                double l1 = 0, l3 = 0;
                for (int i = 0; i < PT; i++) {
                    double u = tab->U[i * PT + lane];
                    l1 += u * J[i];
                    if (wantDP) l3 += u * K[i];
                }
                double dtr = tab->tq[lane] - tr;
                double ratio = sqrt(dtr * dtr + ti * ti) * rinv[e * PT + lane];
                om1[e * PT + lane] = l1 * ratio;
                om3[e * PT + lane] = wantDP ? l3 * ratio * ratio * ratio : 0.0;
            }
        } else {
            n_far++;
            if (lane < NUP) {
                const double *yu = pd.eyu + ps * pd_eyu() + 3 * (e * NUP + lane);
                double d0 = yt[0] - yu[0], d1 = yt[1] - yu[1], d2 = yt[2] - yu[2];
                double r2 = d0 * d0 + d1 * d1 + d2 * d2, r = sqrt(r2);
                double k1 = tab->wu[lane] / r;
                up[lane] = k1;
                up[NUP + lane] = k1 / r2;
            }
            __syncwarp();
            if (lane < PT) {
                double s1 = 0, s3 = 0;
                for (int s = 0; s < NUP; s++) {
                    double L = tab->Lup[s * PT + lane];
                    s1 += L * up[s];
                    s3 += L * up[NUP + s];
                }
                om1[e * PT + lane] = s1;
                om3[e * PT + lane] = s3;
            }
            __syncwarp();
        }
    }
    // monomial coefficients of the three edges (for Horner evaluation on the panels)
    double *em = sw + Z::EM;
    for (int w = lane; w < 9 * P; w += 32) {
        const int e = w / (3 * P), rem = w % (3 * P), k = rem / 3, a = rem % 3;
        double v = 0.0;
        for (int n = k; n < P; n++) v = fma(ea[(e * P + n) * 3 + a], tab->L2M[n * P + k], v);
        em[w] = v;
    }
    __syncwarp();
    // Omega_0 and d Omega_0 / d nu' on graded panels
    double o0 = 0.0, do0 = 0.0;
    const double nxu0 = uz * nut[1], nxu1 = -uz * nut[0], nuu = nut[2] * uz;
    for (int e = 0; e < 3; e++) {
        const double *cm = em + 3 * P * e;
        const double tr = t0s[4 * e], ti = t0s[4 * e + 1];
        double c, sig;
        if (t0s[4 * e + 2] != 0.0) {
            c = fmin(fmax(tr, -1.0), 1.0);
            double dr = tr - c;
            sig = sqrt(dr * dr + ti * ti);
            if (sig < 1e-14) sig = 1e-14;
        } else {
            c = 0.0;
            sig = 4.0;
        }
        const double lo = fmax(c - 0.5 * sig, -1.0), hi = fmin(c + 0.5 * sig, 1.0);
        int nl = 0, nr = 0;
        if (lo > -1.0) { double y = lo, len = sig; while (y > -1.0 && nl < 127) { y -= len; len *= 2; nl++; } }
        if (hi < 1.0) { double x = hi, len = sig; while (x < 1.0 && nr < 127) { x += len; len *= 2; nr++; } }
        const int npan = nl + 1 + nr;
        for (int idx = lane; idx < npan * RRQ_NOM; idx += 32) {
            const int pan = idx / RRQ_NOM, g = idx % RRQ_NOM;
            double a0, a1;
            if (pan < nl) {
                int k = nl - pan;  // left panel k: [y_k, y_{k-1}]
                double yk = lo, len = sig, ykm1 = lo;
                for (int s2 = 1; s2 <= k; s2++) { ykm1 = yk; yk -= len; len *= 2; }
                a0 = fmax(yk, -1.0);
                a1 = ykm1;
            } else if (pan == nl) {
                a0 = lo;
                a1 = hi;
            } else {
                int k = pan - nl;
                double xk = hi, len = sig, xkm1 = hi;
                for (int s2 = 1; s2 <= k; s2++) { xkm1 = xk; xk += len; len *= 2; }
                a0 = xkm1;
                a1 = fmin(xk, 1.0);
            }
            const double mid = 0.5 * (a0 + a1), half = 0.5 * (a1 - a0);
            const double tt = fma(half, tab->tom[g], mid), wg = half * tab->wom[g];
            double y0 = cm[3 * (P - 1)], y1 = cm[3 * (P - 1) + 1], y2 = cm[3 * (P - 1) + 2];
            double dy0 = 0.0, dy1 = 0.0, dy2 = 0.0;
            for (int k = P - 2; k >= 0; k--) {
                dy0 = fma(dy0, tt, y0); dy1 = fma(dy1, tt, y1); dy2 = fma(dy2, tt, y2);
                y0 = fma(y0, tt, cm[3 * k]); y1 = fma(y1, tt, cm[3 * k + 1]); y2 = fma(y2, tt, cm[3 * k + 2]);
            }
            const double d0 = yt[0] - y0, d1 = yt[1] - y1, d2 = yt[2] - y2;
            const double r2 = fma(d0, d0, fma(d1, d1, d2 * d2));
            const double ir = rsqrt(r2), r = r2 * ir;
            const double E = fma(uz, d2, r);
            const double iE = 1.0 / E, inv = ir * iE;
            const double N = uz * (d1 * dy0 - d0 * dy1);
            o0 = fma(-wg * N, inv, o0);
            if (wantDP) {
                const double nd = fma(nut[0], d0, fma(nut[1], d1, nut[2] * d2));
                const double v = inv * ((nxu0 * dy0 + nxu1 * dy1) - N * iE * (nuu + nd * ir) - nd * N * ir * ir);
                do0 = fma(-wg, v, do0);
            }
        }
    }
    o0 = warp_sum(o0);
    if (wantDP) do0 = warp_sum(do0);
    // Omega vector and its derivative
    double ov[3] = {0, 0, 0}, dov[3] = {0, 0, 0};
    for (int q = lane; q < NS; q += 32) {
        const double nd = nut[0] * dq[3 * q] + nut[1] * dq[3 * q + 1] + nut[2] * dq[3 * q + 2];
        for (int a = 0; a < 3; a++) {
            ov[a] -= om1[q] * tau[3 * q + a];
            dov[a] += om3[q] * nd * tau[3 * q + a];
        }
    }
    for (int a = 0; a < 3; a++) {
        ov[a] = warp_sum(ov[a]);
        if (wantDP) dov[a] = warp_sum(dov[a]);
    }
    if (lane == 0) {
        Om[0] = o0; Om[1] = ov[0]; Om[2] = ov[1]; Om[3] = ov[2];
        Om[4] = do0; Om[5] = dov[0]; Om[6] = dov[1]; Om[7] = dov[2];
    }
    // per-sample premultiplied vectors: w1 d, w1 (tau x d), w1 nu', w3 (nu'.d) d
    double *wv = sw + Z::WV;
    for (int q = lane; q < NS; q += 32) {
        const double w1 = om1[q], w3 = om3[q];
        const double d0 = dq[3 * q], d1 = dq[3 * q + 1], d2 = dq[3 * q + 2];
        const double t0 = tau[3 * q], t1 = tau[3 * q + 1], t2 = tau[3 * q + 2];
        const double w3n = w3 * (nut[0] * d0 + nut[1] * d1 + nut[2] * d2);
        double *o = wv + 12 * q;
        o[0] = w1 * d0; o[1] = w1 * d1; o[2] = w1 * d2;
        o[3] = w1 * (t1 * d2 - t2 * d1); o[4] = w1 * (t2 * d0 - t0 * d2); o[5] = w1 * (t0 * d1 - t1 * d0);
        o[6] = w1 * nut[0]; o[7] = w1 * nut[1]; o[8] = w1 * nut[2];
        o[9] = w3n * d0; o[10] = w3n * d1; o[11] = w3n * d2;
    }
    __syncwarp();
    // Step 6: line integrals, one lane per (j, k >= 0), j >= 1
    const cd *eg = pd.eg + ps * pd_eg();
    const cd *eh = pd.eh + ps * pd_eg();
    for (int jk = 1 + lane; jk < NJK; jk += 32) {
        const bool hj = jk >= 3;  // j >= 2
        double Vr = 0, Vi = 0;
        double Q0r = 0, Q0i = 0, Q1r = 0, Q1i = 0, Q2r = 0, Q2i = 0, Q3r = 0, Q3i = 0;
        double D0r = 0, D0i = 0, D1r = 0, D1i = 0, D2r = 0, D2i = 0, D3r = 0, D3i = 0;
        double E0r = 0, E0i = 0, E1r = 0, E1i = 0, E2r = 0, E2i = 0, E3r = 0, E3i = 0;
        for (int q = 0; q < NS; q++) {
            const double *o = wv + 12 * q;
            const cd *g = eg + ((size_t)q * NJK + jk) * 3;
            const cd g0 = g[0], g1 = g[1], g2 = g[2];
            Vr = fma(g0.x, o[3], fma(g1.x, o[4], fma(g2.x, o[5], Vr)));
            Vi = fma(g0.y, o[3], fma(g1.y, o[4], fma(g2.y, o[5], Vi)));
            if (hj) {
                const cd *h = eh + ((size_t)q * NJK + jk) * 3;
                const cd h0 = h[0], h1 = h[1], h2 = h[2];
                const double a0 = o[0], a1 = o[1], a2 = o[2];
                // (0, w1 d)(0, h) = (-(w1 d).h, (w1 d) x h)
                Q0r = fma(-a0, h0.x, fma(-a1, h1.x, fma(-a2, h2.x, Q0r)));
                Q0i = fma(-a0, h0.y, fma(-a1, h1.y, fma(-a2, h2.y, Q0i)));
                Q1r = fma(a1, h2.x, fma(-a2, h1.x, Q1r));
                Q1i = fma(a1, h2.y, fma(-a2, h1.y, Q1i));
                Q2r = fma(a2, h0.x, fma(-a0, h2.x, Q2r));
                Q2i = fma(a2, h0.y, fma(-a0, h2.y, Q2i));
                Q3r = fma(a0, h1.x, fma(-a1, h0.x, Q3r));
                Q3i = fma(a0, h1.y, fma(-a1, h0.y, Q3i));
                if (wantDP) {
                    // sum_q w1 h (the nu' factor is applied after the sum) and
                    // sum_q w3 (nu'.d) (0,d)(0,h)
                    const double w1 = om1[q], m0 = o[9], m1 = o[10], m2 = o[11];
                    D0r = fma(w1, h0.x, D0r); D0i = fma(w1, h0.y, D0i);     // H1 (3 complex, in D0..D2)
                    D1r = fma(w1, h1.x, D1r); D1i = fma(w1, h1.y, D1i);
                    D2r = fma(w1, h2.x, D2r); D2i = fma(w1, h2.y, D2i);
                    E0r = fma(-m0, h0.x, fma(-m1, h1.x, fma(-m2, h2.x, E0r)));
                    E0i = fma(-m0, h0.y, fma(-m1, h1.y, fma(-m2, h2.y, E0i)));
                    E1r = fma(m1, h2.x, fma(-m2, h1.x, E1r));
                    E1i = fma(m1, h2.y, fma(-m2, h1.y, E1i));
                    E2r = fma(m2, h0.x, fma(-m0, h2.x, E2r));
                    E2i = fma(m2, h0.y, fma(-m0, h2.y, E2i));
                    E3r = fma(m0, h1.x, fma(-m1, h0.x, E3r));
                    E3i = fma(m0, h1.y, fma(-m1, h0.y, E3i));
                }
            }
        }
        if (wantDP) {
            // dQ = (0,nu')(0,H1) - (0, w3 (nu'.d) d)(0,h) summed
            const double n0 = nut[0], n1 = nut[1], n2 = nut[2];
            const double a0 = -(n0 * D0r + n1 * D1r + n2 * D2r) - E0r, b0 = -(n0 * D0i + n1 * D1i + n2 * D2i) - E0i;
            const double a1 = (n1 * D2r - n2 * D1r) - E1r, b1 = (n1 * D2i - n2 * D1i) - E1i;
            const double a2 = (n2 * D0r - n0 * D2r) - E2r, b2 = (n2 * D0i - n0 * D2i) - E2i;
            const double a3 = (n0 * D1r - n1 * D0r) - E3r, b3 = (n0 * D1i - n1 * D0i) - E3i;
            D0r = a0; D0i = b0; D1r = a1; D1i = b1; D2r = a2; D2i = b2; D3r = a3; D3i = b3;
        }
        Vs[jk] = mkc(Vr, Vi);
        Qs[4 * jk] = mkc(Q0r, Q0i); Qs[4 * jk + 1] = mkc(Q1r, Q1i); Qs[4 * jk + 2] = mkc(Q2r, Q2i); Qs[4 * jk + 3] = mkc(Q3r, Q3i);
        dQs[4 * jk] = mkc(D0r, D0i); dQs[4 * jk + 1] = mkc(D1r, D1i); dQs[4 * jk + 2] = mkc(D2r, D2i); dQs[4 * jk + 3] = mkc(D3r, D3i);
    }
    __syncwarp();
    // Step 7: translations, one lane per (l, m), 1 <= m <= l <= P
    constexpr double FACT[2 * RRQ_PMAX + 2] = {1.0, 1.0, 2.0, 6.0, 24.0, 120.0, 720.0, 5040.0, 40320.0, 362880.0,
                                               3628800.0, 39916800.0, 479001600.0, 6227020800.0, 87178291200.0,
                                               1307674368000.0, 20922789888000.0, 355687428096000.0};
    const double inv4pi = 0.07957747154594767, sq2 = 1.4142135623730951;
    for (int lm = lane; lm < NP; lm += 32) {
        int l = 1;
        while ((l + 1) * l / 2 <= lm) l++;
        const int m = lm - l * (l - 1) / 2 + 1;
        // only imaginary parts are needed (B = sqrt2 Im(...)): Im(a b) = a.x b.y + a.y b.x
        double Ib0 = 0, Ib1 = 0, Ib2 = 0, Ib3 = 0, Ip = 0, dI0 = 0, dI1 = 0, dI2 = 0, dI3 = 0;
        for (int j = 1; j <= l; j++) {
            const double Dj = FACT[j - 1] * FACT[l - j] / FACT[l];
            const double Cj = j >= 2 ? FACT[j - 2] * FACT[l - j] / FACT[l - 1] : 0.0;
            const int kmin = max(-j, m - (l - j)), kmax = min(j, m + (l - j));
            for (int k = kmin; k <= kmax; k++) {
                const int ak = k < 0 ? -k : k;
                const int jkx = jk_index(j, ak);
                const cd Sv = tget(St, l - j, m - k);
                const cd v = kflip(Vs[jkx], k);
                Ip = fma(Dj, fma(v.x, Sv.y, v.y * Sv.x), Ip);
                if (j >= 2) {
                    const cd q0 = kflip(Qs[4 * jkx], k), q1 = kflip(Qs[4 * jkx + 1], k);
                    const cd q2 = kflip(Qs[4 * jkx + 2], k), q3 = kflip(Qs[4 * jkx + 3], k);
                    const cd cs = cscale(Sv, Cj);
                    Ib0 = fma(q0.x, cs.y, fma(q0.y, cs.x, Ib0));
                    Ib1 = fma(q1.x, cs.y, fma(q1.y, cs.x, Ib1));
                    Ib2 = fma(q2.x, cs.y, fma(q2.y, cs.x, Ib2));
                    Ib3 = fma(q3.x, cs.y, fma(q3.y, cs.x, Ib3));
                    if (wantDP) {
                        // d/dnu' of S^{(l-j, m-k)}(y') = grad . nu'
                        const int n = l - j, qq = m - k, aq = qq < 0 ? -qq : qq;
                        cd dS = mkc(0, 0);
                        if (aq <= n) {
                            const cd *gg = gSt + 3 * jk_index(n, aq);
                            dS = cadd(cadd(cscale(gg[0], nut[0]), cscale(gg[1], nut[1])), cscale(gg[2], nut[2]));
                            dS = kflip(dS, qq);
                        }
                        const cd c2 = cscale(dS, Cj);
                        const cd e0 = kflip(dQs[4 * jkx], k), e1 = kflip(dQs[4 * jkx + 1], k);
                        const cd e2 = kflip(dQs[4 * jkx + 2], k), e3 = kflip(dQs[4 * jkx + 3], k);
                        dI0 = fma(e0.x, cs.y, fma(e0.y, cs.x, fma(q0.x, c2.y, fma(q0.y, c2.x, dI0))));
                        dI1 = fma(e1.x, cs.y, fma(e1.y, cs.x, fma(q1.x, c2.y, fma(q1.y, c2.x, dI1))));
                        dI2 = fma(e2.x, cs.y, fma(e2.y, cs.x, fma(q2.x, c2.y, fma(q2.y, c2.x, dI2))));
                        dI3 = fma(e3.x, cs.y, fma(e3.y, cs.x, fma(q3.x, c2.y, fma(q3.y, c2.x, dI3))));
                    }
                }
            }
        }
        // I[gamma] = (1/4pi) Omega (0, grad S^{(l,m)}(y')), real quaternion times complex vector
        const cd *g = gSt + 3 * jk_index(l, m);
        const double W0 = Om[0], W1 = Om[1], W2 = Om[2], W3 = Om[3];
        const cd G0 = cscale(cadd(cadd(cscale(g[0], W1), cscale(g[1], W2)), cscale(g[2], W3)), -1.0);
        const cd G1 = cadd(cscale(g[0], W0), csub(cscale(g[2], W2), cscale(g[1], W3)));
        const cd G2 = cadd(cscale(g[1], W0), csub(cscale(g[0], W3), cscale(g[2], W1)));
        const cd G3 = cadd(cscale(g[2], W0), csub(cscale(g[1], W1), cscale(g[0], W2)));
        const double f = sq2 * inv4pi;
        Bs[4 * lm] = f * (Ib0 + G0.y);
        Bs[4 * lm + 1] = f * (Ib1 + G1.y);
        Bs[4 * lm + 2] = f * (Ib2 + G2.y);
        Bs[4 * lm + 3] = f * (Ib3 + G3.y);
        const cd Slm = St[jk_index(l, m)];
        Psis[lm] = f * (Ip + Slm.y * Om[0]);
        if (wantDP) {
            const double X0 = Om[4], X1 = Om[5], X2 = Om[6], X3 = Om[7];
            const cd E0 = cscale(cadd(cadd(cscale(g[0], X1), cscale(g[1], X2)), cscale(g[2], X3)), -1.0);
            const cd E1 = cadd(cscale(g[0], X0), csub(cscale(g[2], X2), cscale(g[1], X3)));
            const cd E2 = cadd(cscale(g[1], X0), csub(cscale(g[0], X3), cscale(g[2], X1)));
            const cd E3 = cadd(cscale(g[2], X0), csub(cscale(g[1], X1), cscale(g[0], X2)));
            const cd *H = HSt + 6 * jk_index(l, m);
            cd hn[3];
            hn[0] = cadd(cadd(cscale(H[0], nut[0]), cscale(H[1], nut[1])), cscale(H[2], nut[2]));
            hn[1] = cadd(cadd(cscale(H[1], nut[0]), cscale(H[3], nut[1])), cscale(H[4], nut[2]));
            hn[2] = cadd(cadd(cscale(H[2], nut[0]), cscale(H[4], nut[1])), cscale(H[5], nut[2]));
            const cd F0 = cscale(cadd(cadd(cscale(hn[0], W1), cscale(hn[1], W2)), cscale(hn[2], W3)), -1.0);
            const cd F1 = cadd(cscale(hn[0], W0), csub(cscale(hn[2], W2), cscale(hn[1], W3)));
            const cd F2 = cadd(cscale(hn[1], W0), csub(cscale(hn[0], W3), cscale(hn[2], W1)));
            const cd F3 = cadd(cscale(hn[2], W0), csub(cscale(hn[1], W1), cscale(hn[0], W2)));
            Bds[4 * lm] = f * (dI0 + E0.y + F0.y);
            Bds[4 * lm + 1] = f * (dI1 + E1.y + F1.y);
            Bds[4 * lm + 2] = f * (dI2 + E2.y + F2.y);
            Bds[4 * lm + 3] = f * (dI3 + E3.y + F3.y);
        }
    }
    __syncwarp();
    // Step 8: rows, one lane per node i
    const double *XD = pd.XD + ps * pd_X(), *XSp = pd.XSp + ps * pd_X(), *XS2 = pd.XS2 + ps * pd_X();
    const double *XS1 = pd.XS1 + ps * pd_XS1();
    const double sc = fr[12], Lsc = 1.0 / sc;
    const double n0 = nut[0], n1 = nut[1], n2 = nut[2];
    const double xt0 = sw[Z::XT], xt1 = sw[Z::XT + 1], xt2 = sw[Z::XT + 2];
    const double gn0 = sw[Z::NT], gn1 = sw[Z::NT + 1], gn2 = sw[Z::NT + 2];
    for (int i = lane; i < NP; i += 32) {
        double rS = 0, rD = 0, rSp = 0, rDp = 0;
        for (int lm = 0; lm < NP; lm++) {
            const double B0 = Bs[4 * lm], B1 = Bs[4 * lm + 1], B2 = Bs[4 * lm + 2], B3 = Bs[4 * lm + 3];
            const double x0 = XD[(0 * NP + lm) * NP + i], x1 = XD[(1 * NP + lm) * NP + i];
            const double x2 = XD[(2 * NP + lm) * NP + i], x3 = XD[(3 * NP + lm) * NP + i];
            rD -= B0 * x0 - B1 * x1 - B2 * x2 - B3 * x3;
            if (wantDP)
                rDp -= Bds[4 * lm] * x0 - Bds[4 * lm + 1] * x1 - Bds[4 * lm + 2] * x2 - Bds[4 * lm + 3] * x3;
            if (mask & RRQ_SP) {
                const double w0 = XSp[(0 * NP + lm) * NP + i], w1 = XSp[(1 * NP + lm) * NP + i];
                const double w2 = XSp[(2 * NP + lm) * NP + i], w3 = XSp[(3 * NP + lm) * NP + i];
                const double nB = n0 * B1 + n1 * B2 + n2 * B3;
                const double c0 = n1 * B3 - n2 * B2, c1 = n2 * B1 - n0 * B3, c2 = n0 * B2 - n1 * B1;
                rSp += nB * w0 + (B0 * n0 + c0) * w1 + (B0 * n1 + c1) * w2 + (B0 * n2 + c2) * w3;
            }
            if (mask & RRQ_S) {
                const double g0 = XS2[(0 * NP + lm) * NP + i], g1 = XS2[(1 * NP + lm) * NP + i];
                const double g2 = XS2[(2 * NP + lm) * NP + i], g3 = XS2[(3 * NP + lm) * NP + i];
                rS += Psis[lm] * XS1[lm * NP + i] - (B0 * g0 - B1 * g1 - B2 * g2 - B3 * g3);
            }
        }
        rS *= Lsc;
        rDp *= sc;
        if (i == self_i) {
            rD -= 0.5;
            rSp += 0.5;
        } else {
            const double *xs = xyz + 3 * (o + i), *ns = nrm + 3 * (o + i);
            const double d0 = xt0 - xs[0], d1 = xt1 - xs[1], d2 = xt2 - xs[2];
            const double r2 = d0 * d0 + d1 * d1 + d2 * d2, r = sqrt(r2), r3 = r2 * r;
            const double wk = wts[o + i] * inv4pi;
            const double dns = d0 * ns[0] + d1 * ns[1] + d2 * ns[2];
            const double dnt = d0 * gn0 + d1 * gn1 + d2 * gn2;
            rS -= wk / r;
            rD -= wk * dns / r3;
            rSp += wk * dnt / r3;
            rDp -= wk * ((gn0 * ns[0] + gn1 * ns[1] + gn2 * ns[2]) / r3 - 3.0 * dns * dnt / (r3 * r2));
        }
        const int64_t dst = item.off + i;
        col[dst] = (int32_t)(o + i);
        if ((mask & RRQ_S) && vS) vS[dst] = rS;
        if ((mask & RRQ_D) && vD) vD[dst] = rD;
        if ((mask & RRQ_SP) && vSp) vSp[dst] = rSp;
        if ((mask & RRQ_DP) && vDp) vDp[dst] = rDp;
    }
    if (lane == 0) {
        if (fl_newton) atomicAdd(&bc[0], 1u);
        if (fl_onedge) atomicAdd(&bc[1], 1u);
        if (fl_upoor) atomicAdd(&bc[2], 1u);
        atomicAdd(&bc[3], n_ssq);
        atomicAdd(&bc[4], n_far);
    }
    __syncwarp();
}

template <int P>
__global__ void __launch_bounds__(32 * WARPS) k_pairs(const OrderTables *__restrict__ tab, const PairItem *__restrict__ items,
                                                      int64_t nitems, PatchData pd, const int64_t *__restrict__ node_off,
                                                      const double *__restrict__ xyz, const double *__restrict__ nrm,
                                                      const double *__restrict__ wts, const double *__restrict__ txyz,
                                                      const double *__restrict__ tnrm, const int64_t *__restrict__ tself,
                                                      uint32_t mask, int newton_max, double *vS, double *vD, double *vSp,
                                                      double *vDp, int32_t *col, BuildCounters *cnt) {
    extern __shared__ double smraw[];
    __shared__ unsigned int bc[5];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if (threadIdx.x < 5) bc[threadIdx.x] = 0;
    __syncthreads();
    double *sw = smraw + (size_t)wib * PairSm<P>::TOTAL;
    for (int64_t it = (int64_t)blockIdx.x * WARPS + wib; it < nitems; it += (int64_t)gridDim.x * WARPS) {
        process_pair<P>(tab, items[it], pd, node_off, xyz, nrm, wts, txyz, tnrm, tself, mask, newton_max, vS, vD,
                        vSp, vDp, col, sw, lane, bc);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (bc[0]) atomicAdd(&cnt->newton_fail, (unsigned long long)bc[0]);
        if (bc[1]) atomicAdd(&cnt->on_edge, (unsigned long long)bc[1]);
        if (bc[2]) atomicAdd(&cnt->u_poor, (unsigned long long)bc[2]);
        if (bc[3]) atomicAdd(&cnt->ssq_edges, (unsigned long long)bc[3]);
        if (bc[4]) atomicAdd(&cnt->far_edges, (unsigned long long)bc[4]);
    }
}

template <int P>
cudaError_t launch_pairs_p(const OrderTables *d_tab, const PairItem *d_items, int64_t nitems, PatchData pd,
                           const int64_t *d_node_off, const double *d_xyz, const double *d_nrm, const double *d_wts,
                           const double *d_txyz, const double *d_tnrm, const int64_t *d_tself, uint32_t mask,
                           int newton_max, double *vS, double *vD, double *vSp, double *vDp, int32_t *col,
                           BuildCounters *cnt, cudaStream_t st) {
    const size_t bytes = sizeof(double) * PairSm<P>::TOTAL * WARPS;
    cudaError_t e = cudaFuncSetAttribute(k_pairs<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    if (nitems <= 0) return cudaSuccess;
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pairs<P>, 32 * WARPS, bytes);
    if (per_sm < 1) per_sm = 1;
    int64_t want = (nitems + WARPS - 1) / WARPS;
    int64_t grid = (int64_t)nsm * per_sm * 8;
    if (grid > want) grid = want;
    k_pairs<P><<<(unsigned)grid, 32 * WARPS, bytes, st>>>(d_tab, d_items, nitems, pd, d_node_off, d_xyz, d_nrm, d_wts,
                                                          d_txyz, d_tnrm, d_tself, mask, newton_max, vS, vD, vSp, vDp,
                                                          col, cnt);
    RRQ_COUNT_LAUNCH();
    return cudaGetLastError();
}

}  // namespace rrqk
