// Per-pair (target, patch) work: Sec. 4 Steps 4-8 for S, D, S', D' in one pass.
// Shared helpers and the per-pair shared-memory layout; the kernel is in
// rrq_pairs_tile.cuh (pairs grouped by patch so the patch data stays in L2).
//
//   Step 4  harmonic table S^{(n,q)}(y'), its gradient (and Hessian for D') at the
//           target in the patch frame;
//   u       +e_z for a target that is a node of the patch; else, if the target's
//           footprint along e_z lies in the patch, the side it is on; else the better of
//           +-e_z by min over nodes and edge samples of u.(y'-y)/|y'-y|;
//   Step 5  per edge: complex root t0 of |y(t)-y'|^2 (Newton from the chord root),
//           singularity-swap moments by recurrence and weights lambda solving
//           V^T lambda = I (Sec. 2.4, 3.4), or an upsampled Gauss rule when t0 is
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

// Per-pair shared-memory layout (in doubles).  Regions whose lifetimes do not overlap share
// space, so that more pairs' CTAs fit on an SM:
//   header YT, NUT, XT, NT, FR                 whole tile
//   ST, GST (target harmonics, gradients)     phases C/D .. L
//   OM (Omega_0, Omega and nu' derivatives)   H .. L
//   R: WV (premultiplied sample vectors)      H .. K, holding before H the edge
//      coefficients EA (A .. D) and after K the nu'-derivative table DST and (mixed)
//      the split target table STF (L0 .. L), then the row vectors B, BD, BP, PSI
//      (L .. M) when they fit
//   early scratch after WV: DQ, TAU, RINV, OM1, OM3, UP/MOM, T0, EM   C .. H
//   line integrals Q, DQQ, V over the early scratch                     K .. L
//   B, BD, BP, PSI after the line integrals when they do not fit in WV  L .. M
// Every region starts at an even double offset and TOTAL is even, so that the (hi, lo)
// float4 views of the mixed path are 16-byte aligned.
template <int P>
struct PairSm {
    static constexpr int NP = P * (P + 1) / 2, PT = 2 * P, NJK = (P + 1) * (P + 2) / 2, NS = 3 * PT, NUP = 2 * PT;
    static constexpr int ev(int x) { return (x + 1) & ~1; }
    static constexpr int mx(int a, int b) { return a > b ? a : b; }
    static constexpr int YT = 0, NUT = 3, XT = 6, NT = 9, FR = 12;   // FR: 16
    static constexpr int ST = 28;                                     // NJK complex
    static constexpr int GST = ST + 2 * NJK;                          // NJK*3 complex
    static constexpr int OM = GST + 6 * NJK;                          // 8
    static constexpr int R = OM + 8;
    static constexpr int WV = R;                                      // NS*12
    static constexpr int EA = R;                                      // 9P
    static constexpr int DST = R;                                     // NJK complex
    static constexpr int STF = R + 2 * NJK;                           // NJK complex (mixed)
    static constexpr int DQ = R + 12 * NS;                            // NS*3
    static constexpr int TAU = DQ + 3 * NS;                           // NS*3
    static constexpr int RINV = TAU + 3 * NS;                         // NS
    static constexpr int OM1 = RINV + NS;                             // NS
    static constexpr int OM3 = OM1 + NS;                              // NS
    // per edge e: either the SSQ moments J, K (2*PT) or the upsampled kernel values
    // (2*NUP), never both, at UP + 2*NUP*e
    static constexpr int UP = OM3 + NS;                               // 3*2*NUP
    static constexpr int MOM = UP;
    static constexpr int T0 = UP + 6 * NUP;                           // 3*4 (re, im, conv, ssq)
    static constexpr int EM = T0 + 12;                                // 3*P*3 monomial edge coefficients
    static constexpr int EEND = EM + 9 * P;
    static constexpr int Q = DQ;                                      // NJK*4 complex
    static constexpr int DQQ = Q + 8 * NJK;                           // NJK*4 complex
    static constexpr int V = DQQ + 8 * NJK;                           // NJK complex
    static constexpr int QEND = V + 2 * NJK;
    static constexpr bool OUT_IN_WV = 4 * NJK + 13 * NP <= 12 * NS;
    static constexpr int B = OUT_IN_WV ? R + 4 * NJK : ev(QEND);    // NP*4
    static constexpr int BD = B + 4 * NP;                             // NP*4
    static constexpr int BP = BD + 4 * NP;                            // NP*4: (0, nu') B
    static constexpr int PSI = BP + 4 * NP;                           // NP
    static constexpr int TOTAL = ev(mx(mx(EEND, QEND), PSI + NP));
    static_assert(9 * P <= 12 * NS && 4 * NJK <= 12 * NS, "region R too small");
    // rotation-based translation only, appended: the second buffer of the nine coefficient
    // sets (18 NJK), e^{ik theta} and e^{ik(phi + 90)} for k = 0..P, rho^n / n!, and nu' in
    // the rotated frame
    static constexpr int RY = TOTAL;
    static constexpr int RPH = RY + 18 * NJK;
    static constexpr int RRP = RPH + 4 * (P + 1);
    static constexpr int RNU = RRP + P + 1;
    static constexpr int TOTAL_ROT = ev(RNU + 3);
};

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
// sum over each half (16 lanes) of the warp; every lane of the warp takes part
__device__ __forceinline__ double half_warp_sum(double v) {
    for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
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

// 1/n for n = 0 .. 2 RRQ_PMAX + 1 (entry 0 unused)
__device__ __forceinline__ double rcp_small(int n) {
    constexpr double R[2 * RRQ_PMAX + 2] = {0.0,      1.0,      1.0 / 2,  1.0 / 3,  1.0 / 4,  1.0 / 5,  1.0 / 6,
                                            1.0 / 7,  1.0 / 8,  1.0 / 9,  1.0 / 10, 1.0 / 11, 1.0 / 12, 1.0 / 13,
                                            1.0 / 14, 1.0 / 15, 1.0 / 16, 1.0 / 17, 1.0 / 18, 1.0 / 19, 1.0 / 20,
                                            1.0 / 21, 1.0 / 22, 1.0 / 23, 1.0 / 24, 1.0 / 25, 1.0 / 26, 1.0 / 27,
                                            1.0 / 28, 1.0 / 29};
    static_assert(2 * RRQ_PMAX + 2 == 30, "extend the table with the order limit");
    return R[n];
}

// Singularity-swap weights from the moments: solves V^T lam = mom in place, V[q][i] = x_q^i
// (x the PT edge nodes), so that sum_q lam_q F(x_q) = sum_i c_i mom_i for the monomial
// coefficients c of the interpolant of F (Sec. 3.4).  The dual algorithm of Bjorck and
// Pereyra (Math. Comp. 24, 1970): Newton-form differences, then back to the power basis,
// with the reciprocal node differences rd[k][i] = 1/(x_i - x_{i-k-1}) tabulated.  It is
// accurate to rounding for Gauss-Legendre nodes even where cond(V) ~ 1e10 (PT = 24),
// whereas a product with an explicitly formed inverse cancels.
template <int PT>
__device__ __forceinline__ void dual_vandermonde_solve(double *mom, const double *x, const double *rd) {
    if constexpr (PT <= 12) {
        // in registers, fully unrolled
        double a[PT];
#pragma unroll
        for (int i = 0; i < PT; i++) a[i] = mom[i];
#pragma unroll
        for (int k = 0; k < PT - 1; k++) {
            const double xk = x[k];
#pragma unroll
            for (int i = PT - 1; i > k; i--) a[i] = fma(-xk, a[i - 1], a[i]);
        }
#pragma unroll
        for (int k = PT - 2; k >= 0; k--) {
#pragma unroll
            for (int i = k + 1; i < PT; i++) a[i] *= rd[k * PT + i];
#pragma unroll
            for (int i = k; i < PT - 1; i++) a[i] -= a[i + 1];
        }
#pragma unroll
        for (int i = 0; i < PT; i++) mom[i] = a[i];
    } else {
        // higher orders: in place (shared memory), the same steps
        for (int k = 0; k < PT - 1; k++) {
            const double xk = x[k];
            for (int i = PT - 1; i > k; i--) mom[i] = fma(-xk, mom[i - 1], mom[i]);
        }
        for (int k = PT - 2; k >= 0; k--) {
            for (int i = k + 1; i < PT; i++) mom[i] *= rd[k * PT + i];
            for (int i = k; i < PT - 1; i++) mom[i] -= mom[i + 1];
        }
    }
}

// Table of Rn_n^q (0 <= q <= n <= P), column m = lane computed by the warp.
template <int P>
__device__ __forceinline__ void target_table(const double *y, cd *S, int lane) {
    if (lane <= P) {
        const double X = y[1], Y = y[2], Z = y[0], r2 = X * X + Y * Y + Z * Z;
        const int m = lane;
        cd w = mkc(1.0, 0.0);
        for (int k = 1; k <= m; k++) w = cscale(cmul(w, mkc(X, Y)), 0.5 * rcp_small(k));
        cd prev = mkc(0.0, 0.0), cur = w;
        S[jk_index(m, m)] = cur;
        for (int l = m; l < P; l++) {
            cd nxt = cscale(csub(cscale(cur, (2.0 * l + 1.0) * Z), cscale(prev, r2)), rcp_small(l - m + 1) * rcp_small(l + m + 1));
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
        cd Pn = cscale(csub(cscale(cmul(t, Pc), 2.0 * n + 1.0), cscale(Pm, (double)n)), rcp_small(n + 1));
        cd dPn = cadd(dPm, cscale(Pc, 2.0 * n + 1.0));
        for (int a = 0; a < 3; a++) {
            y[a] = cadd(y[a], cscale(Pn, ea[3 * (n + 1) + a]));
            dy[a] = cadd(dy[a], cscale(dPn, ea[3 * (n + 1) + a]));
        }
        Pm = Pc; Pc = Pn; dPm = dPc; dPc = dPn;
    }
}

}  // namespace rrqk
