// Per-patch, source-only work (Sec. 4, Steps 1-3 in the matrix-build variant):
//   * patch frame: origin at the vertex mean, e_z normal to the vertex plane, e_x along
//     the longest edge, lengths scaled so the longest edge is 1 (Sec. 4, Sec. 5.1);
//   * edge curves: node interpolant at the edge Gauss nodes, Legendre coefficients,
//     tangents, samples at the upsampled nodes;
//   * Step 3: grad S^{(j,k)} and (Hess S^{(j,k)}) tau at the 3 ptilde edge samples;
//   * Steps 1-2: the quaternion harmonic system (eq. dlpdensitylinearsystem2) solved
//     as an n_p x n_p quaternion system by Gaussian elimination with pivoting on the
//     quaternion modulus, for the right-hand sides (e_i, 0) [D] and (0, nu_i e_i) [S'];
//     the scalar SLP system (eq. slpdensitylinearsystem) by LU with partial pivoting;
//     and X_S2 = X_D Hn A_S^{-1} for the intermediate density of Thm. slpreduction.
//   * when requested, kappa_1(A) of the quaternion system in the paper's normalisation
//     (the conditioning study of Sec. 5.1).
// One CTA per patch; everything lives in shared memory.
#include <math.h>

#include "rrq_internal.cuh"

namespace {

// complex double -> (re.hi, re.lo, im.hi, im.lo) as float pairs (about 48 bits)
// x as (hi, lo) float pair
__device__ __forceinline__ float2 split2f(double x) {
    const float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(x - (double)h));
}

__device__ __forceinline__ float4 split4(cd v) {
    const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
    return make_float4(rh, __double2float_rn(v.x - (double)rh), ih, __double2float_rn(v.y - (double)ih));
}

struct q4 {
    double s, x, y, z;
};

__device__ __forceinline__ q4 qmul(const q4 &a, const q4 &b) {
    q4 r;
    r.s = a.s * b.s - (a.x * b.x + a.y * b.y + a.z * b.z);
    r.x = a.s * b.x + b.s * a.x + (a.y * b.z - a.z * b.y);
    r.y = a.s * b.y + b.s * a.y + (a.z * b.x - a.x * b.z);
    r.z = a.s * b.z + b.s * a.z + (a.x * b.y - a.y * b.x);
    return r;
}
__device__ __forceinline__ q4 qsub(const q4 &a, const q4 &b) {
    q4 r = {a.s - b.s, a.x - b.x, a.y - b.y, a.z - b.z};
    return r;
}
__device__ __forceinline__ double qnorm2(const q4 &a) { return a.s * a.s + a.x * a.x + a.y * a.y + a.z * a.z; }
__device__ __forceinline__ q4 qinv(const q4 &a) {
    double n = qnorm2(a);
    q4 r = {a.s / n, -a.x / n, -a.y / n, -a.z / n};
    return r;
}

// Table of Rn_n^q (unit-translation normalisation) for 0 <= q <= n <= L at the S
// coordinates of y: S(x,y,z) = Rn(y,z,x).
// d_lm = sqrt((l-m)! (l+m)!) for the lm-th fit harmonic (l = 1..p, m = 1..l, l-major):
// the paper's R_l^m over the device's Rn_l^m.
__device__ __forceinline__ double paper_norm(int lm) {
    int l = 1;
    while ((l + 1) * l / 2 <= lm) l++;
    const int m = lm - l * (l - 1) / 2 + 1;
    double f = 1.0;
    for (int k = 2; k <= l - m; k++) f *= k;
    for (int k = 2; k <= l + m; k++) f *= k;
    return sqrt(f);
}

template <int L>
__device__ void harmonic_table(const double *y, cd *S) {
    const double X = y[1], Y = y[2], Z = y[0];
    const double r2 = X * X + Y * Y + Z * Z;
    cd w = mkc(1.0, 0.0);
    for (int m = 0; m <= L; m++) {
        if (m > 0) w = cscale(cmul(w, mkc(X, Y)), 1.0 / (2.0 * m));
        S[jk_index(m, m)] = w;
        if (m < L) S[jk_index(m + 1, m)] = cscale(w, Z);
        for (int l = m + 1; l < L; l++) {
            cd a = cscale(S[jk_index(l, m)], (2.0 * l + 1.0) * Z);
            cd b = cscale(S[jk_index(l - 1, m)], r2);
            S[jk_index(l + 1, m)] = cscale(csub(a, b), 1.0 / ((l - m + 1.0) * (l + m + 1.0)));
        }
    }
}

__device__ __forceinline__ cd hget(const cd *S, int n, int q) {
    if (n < 0) return mkc(0, 0);
    int aq = q < 0 ? -q : q;
    if (aq > n) return mkc(0, 0);
    cd v = S[jk_index(n, aq)];
    if (q < 0) {
        v = cconj(v);
        if (aq & 1) v = mkc(-v.x, -v.y);
    }
    return v;
}

// grad of S^{(j,k)} in (x,y,z) from the table (ladder rules with X=y, Y=z, Z=x)
__device__ __forceinline__ void hgrad(const cd *S, int j, int k, cd g[3]) {
    cd a = hget(S, j - 1, k - 1), b = hget(S, j - 1, k + 1);
    g[0] = hget(S, j - 1, k);                         // d/dx = d/dZ
    g[1] = cscale(csub(a, b), 0.5);                   // d/dy = d/dX
    g[2] = cmuli(cscale(cadd(a, b), 0.5));            // d/dz = d/dY
}

// Hessian of S^{(j,k)}: H[0]=xx, H[1]=xy, H[2]=xz, H[3]=yy, H[4]=yz, H[5]=zz
__device__ __forceinline__ void hhess(const cd *S, int j, int k, cd H[6]) {
    cd r0 = hget(S, j - 2, k), rm1 = hget(S, j - 2, k - 1), rp1 = hget(S, j - 2, k + 1);
    cd rm2 = hget(S, j - 2, k - 2), rp2 = hget(S, j - 2, k + 2);
    H[0] = r0;                                                        // ZZ
    H[1] = cscale(csub(rm1, rp1), 0.5);                               // ZX
    H[2] = cmuli(cscale(cadd(rm1, rp1), 0.5));                        // ZY
    H[3] = cscale(cadd(csub(rm2, cscale(r0, 2.0)), rp2), 0.25);       // XX
    H[4] = cmuli(cscale(csub(rm2, rp2), 0.25));                       // XY
    H[5] = cscale(cadd(cadd(rm2, cscale(r0, 2.0)), rp2), -0.25);      // YY
}

template <int P>
struct PreSizes {
    static constexpr int NP = P * (P + 1) / 2, PT = 2 * P, NJK = (P + 1) * (P + 2) / 2, NUP = 2 * PT;
    static constexpr int NS = 3 * PT + 3;
    // phase B layout (doubles)
    static constexpr int M_OFF = 0;                         // NP*NP quaternions
    static constexpr int W_OFF = M_OFF + 4 * NP * NP;        // NP*2NP quaternions
    static constexpr int AS_OFF = W_OFF + 8 * NP * NP;       // NP*NP
    static constexpr int ASI_OFF = AS_OFF + NP * NP;         // NP*NP
    static constexpr int HN_OFF = ASI_OFF + NP * NP;         // NP*NP
    static constexpr int TMP_OFF = HN_OFF + NP * NP;         // NP*NP
    static constexpr int TAB_OFF = TMP_OFF + NP * NP;        // NP*NJK complex (node tables)
    // orders above 8: only the quaternion factor of the fit matrix stays in shared memory;
    // above 12 it is kept in global memory (PatchData::lu) and shared memory holds the
    // scalar system only
    static constexpr bool BIGP = P > 8;
    static constexpr bool GLU = P > 12;
    static constexpr int PHASEB = GLU ? NP * NP : BIGP ? 4 * NP * NP : TAB_OFF + 2 * NP * NJK;
    static constexpr int PHASEA = 2 * 3 * PT * NJK;          // edge tables
    static constexpr int BIG = PHASEB > PHASEA ? PHASEB : PHASEA;
    // persistent small arrays
    static constexpr int SX_OFF = BIG;                       // NP*3 global xyz
    static constexpr int SN_OFF = SX_OFF + 3 * NP;           // NP*3 global normals
    static constexpr int SNL_OFF = SN_OFF + 3 * NP;          // NP*3 local normals
    static constexpr int SG_OFF = SNL_OFF + 3 * NP;          // NS*3 global samples
    static constexpr int EY_OFF = SG_OFF + 3 * NS;           // 3PT*3 local samples
    static constexpr int EA_OFF = EY_OFF + 9 * PT;           // 3*P*3 coefficients
    static constexpr int YN_OFF = EA_OFF + 9 * P;            // NP*3 local nodes
    static constexpr int FR_OFF = YN_OFF + 3 * NP;           // 16 frame
    static constexpr int LB_OFF = FR_OFF + 16;               // NP quaternions (elimination multipliers)
    static constexpr int TOTAL = LB_OFF + 4 * NP + 8;
    static constexpr size_t BYTES = sizeof(double) * TOTAL;
};

// (l, m) of the lm-th fit harmonic (l = 1..p, m = 1..l, l-major)
__device__ __forceinline__ void lm_of(int lm, int &l, int &m) {
    l = 1;
    while ((l + 1) * l / 2 <= lm) l++;
    m = lm - l * (l - 1) / 2 + 1;
}

// Steps 1-2 for orders above 8, where the 4 n_p x 4 n_p system no longer fits in shared memory
// beside its right-hand sides: the quaternion matrix is factored in place in shared memory
// (above order 12, where the factor alone exceeds shared memory, in the patch's slice of
// PatchData::lu, which stays in L2 while the CTA works on it)
// (P A = L U, pivoting on the quaternion modulus, multipliers kept below the diagonal), and
// each right-hand side is solved by one thread with its work vector in the output array
// itself (X_D, X_S' in global memory, element (comp, row) of column c at
// [(comp n_p + row) n_p + c], coalesced across threads).  The scalar SLP system is factored
// the same way in the freed shared memory, its inverse solved into X_S1, and
// X_S2 = X_D (Hn A_S^{-1}) formed from global memory.  Node harmonic tables are rebuilt per
// node in per-thread local arrays where they are needed.
template <int P>
__device__ void fit_big(double *sm, const double *syn, const double *snl, const PatchData &pd, int pid, int tid,
                        int nth, int &s_bad) {
    constexpr int NP = P * (P + 1) / 2, NJK = (P + 1) * (P + 2) / 2;
    const double sq2 = 1.4142135623730951;
    q4 *Mq = PreSizes<P>::GLU ? reinterpret_cast<q4 *>(pd.lu + (size_t)pid * pd_lu(pd.pmax))
                              : reinterpret_cast<q4 *>(sm);  // [NP][NP]
    __shared__ int s_pv[NP];
    __shared__ double s_red[NP];
    __shared__ double s_anorm;
    __shared__ int s_k;
    double *gXD = pd.XD + (size_t)pid * pd_X(pd.pmax), *gXSp = pd.XSp + (size_t)pid * pd_X(pd.pmax);
    double *gXS2 = pd.XS2 + (size_t)pid * pd_X(pd.pmax), *gXS1 = pd.XS1 + (size_t)pid * pd_XS1(pd.pmax);
    // the system matrix: row i (node), column lm, entry (0, grad H^{(l,m)}(y_i))
    for (int i = tid; i < NP; i += nth) {
        cd tb[NJK];
        harmonic_table<P>(syn + 3 * i, tb);
        for (int lm = 0; lm < NP; lm++) {
            int l, m;
            lm_of(lm, l, m);
            cd g[3];
            hgrad(tb, l, m, g);
            q4 e = {0.0, sq2 * g[0].y, sq2 * g[1].y, sq2 * g[2].y};
            Mq[i * NP + lm] = e;
        }
    }
    __syncthreads();
    // ||A||_1 (kappa_1 in the paper's normalisation, as for the lower orders)
    if (pd.kappa) {
        for (int lm = tid; lm < NP; lm += nth) {
            double a = 0;
            for (int i = 0; i < NP; i++) {
                const q4 e = Mq[i * NP + lm];
                a += fabs(e.x) + fabs(e.y) + fabs(e.z);
            }
            s_red[lm] = a * paper_norm(lm);
        }
        __syncthreads();
        if (tid == 0) {
            double a = 0;
            for (int lm = 0; lm < NP; lm++) a = fmax(a, s_red[lm]);
            s_anorm = a;
        }
    }
    // factorisation
    for (int k = 0; k < NP; k++) {
        if (tid == 0) {
            int pr = k;
            double best = qnorm2(Mq[k * NP + k]);
            for (int r = k + 1; r < NP; r++) {
                const double v = qnorm2(Mq[r * NP + k]);
                if (v > best) { best = v; pr = r; }
            }
            if (!(best > 0.0)) s_bad = 1;
            s_pv[k] = pr;
            s_k = pr;
        }
        __syncthreads();
        if (s_bad) break;
        const int pr = s_k;
        if (pr != k)
            for (int j = tid; j < NP; j += nth) {
                const q4 t = Mq[k * NP + j];
                Mq[k * NP + j] = Mq[pr * NP + j];
                Mq[pr * NP + j] = t;
            }
        __syncthreads();
        const q4 inv = qinv(Mq[k * NP + k]);
        for (int r = k + 1 + tid; r < NP; r += nth) Mq[r * NP + k] = qmul(Mq[r * NP + k], inv);
        __syncthreads();
        const int w = NP - k - 1;
        for (int f = tid; f < w * w; f += nth) {
            const int r = k + 1 + f / w, j = k + 1 + f % w;
            Mq[r * NP + j] = qsub(Mq[r * NP + j], qmul(Mq[r * NP + k], Mq[k * NP + j]));
        }
        __syncthreads();
    }
    if (!s_bad) {
        // right-hand sides: column c < NP is (e_c, 0) [D], c >= NP is (0, nu_r e_r), r = c - NP [S']
        for (int c = tid; c < 2 * NP; c += nth) {
            double *X = c < NP ? gXD + c : gXSp + (c - NP);
            const size_t cs = (size_t)NP * NP;  // stride between components
            auto ld = [&](int row) {
                q4 v = {X[(size_t)row * NP], X[cs + (size_t)row * NP], X[2 * cs + (size_t)row * NP],
                        X[3 * cs + (size_t)row * NP]};
                return v;
            };
            auto st = [&](int row, const q4 &v) {
                X[(size_t)row * NP] = v.s;
                X[cs + (size_t)row * NP] = v.x;
                X[2 * cs + (size_t)row * NP] = v.y;
                X[3 * cs + (size_t)row * NP] = v.z;
            };
            const int r0 = c < NP ? c : c - NP;
            for (int row = 0; row < NP; row++) {
                q4 v = {0.0, 0.0, 0.0, 0.0};
                if (row == r0) {
                    if (c < NP) v.s = 1.0;
                    else { v.x = snl[3 * r0]; v.y = snl[3 * r0 + 1]; v.z = snl[3 * r0 + 2]; }
                }
                st(row, v);
            }
            // row interchanges in factorisation order, then L y = P b
            for (int k = 0; k < NP; k++) {
                const int pr = s_pv[k];
                if (pr != k) {
                    const q4 a = ld(k), b = ld(pr);
                    st(k, b);
                    st(pr, a);
                }
            }
            for (int k = 0; k < NP; k++) {
                const q4 yk = ld(k);
                for (int r = k + 1; r < NP; r++) st(r, qsub(ld(r), qmul(Mq[r * NP + k], yk)));
            }
            // U x = y
            for (int k = NP - 1; k >= 0; k--) {
                q4 acc = ld(k);
                for (int j = k + 1; j < NP; j++) acc = qsub(acc, qmul(Mq[k * NP + j], ld(j)));
                st(k, qmul(qinv(Mq[k * NP + k]), acc));
            }
        }
    }
    __syncthreads();
    // ||A^{-1}||_1 from the columns of X_D (as for the lower orders)
    if (pd.kappa) {
        for (int i = tid; i < NP; i += nth) {
            double a = 0;
            for (int c = 0; c < 4; c++)
                for (int lm = 0; lm < NP; lm++) a += fabs(gXD[((size_t)c * NP + lm) * NP + i]) / paper_norm(lm);
            s_red[i] = a;
        }
        __syncthreads();
        if (tid == 0) {
            double a = 0;
            for (int i = 0; i < NP; i++) a = fmax(a, s_red[i]);
            pd.kappa[pid] = (s_bad || !(a == a)) ? INFINITY : s_anorm * a;
        }
    }
    // scalar SLP system A_S[i][lm] = grad H^{(l,m)}(y_i) . nu_i, factored in the freed space
    double *AS = sm;
    for (int i = tid; i < NP; i += nth) {
        cd tb[NJK];
        harmonic_table<P>(syn + 3 * i, tb);
        const double *nu = snl + 3 * i;
        for (int lm = 0; lm < NP; lm++) {
            int l, m;
            lm_of(lm, l, m);
            cd g[3];
            hgrad(tb, l, m, g);
            AS[i * NP + lm] = sq2 * (g[0].y * nu[0] + g[1].y * nu[1] + g[2].y * nu[2]);
        }
    }
    __syncthreads();
    for (int k = 0; k < NP; k++) {
        if (tid == 0) {
            int pr = k;
            double best = fabs(AS[k * NP + k]);
            for (int r = k + 1; r < NP; r++)
                if (fabs(AS[r * NP + k]) > best) { best = fabs(AS[r * NP + k]); pr = r; }
            if (!(best > 0.0)) s_bad = 1;
            s_pv[k] = pr;
            s_k = pr;
        }
        __syncthreads();
        if (s_bad) break;
        const int pr = s_k;
        if (pr != k)
            for (int j = tid; j < NP; j += nth) {
                const double t = AS[k * NP + j];
                AS[k * NP + j] = AS[pr * NP + j];
                AS[pr * NP + j] = t;
            }
        __syncthreads();
        const double pinv = 1.0 / AS[k * NP + k];
        for (int r = k + 1 + tid; r < NP; r += nth) AS[r * NP + k] *= pinv;
        __syncthreads();
        const int w = NP - k - 1;
        for (int f = tid; f < w * w; f += nth) {
            const int r = k + 1 + f / w, j = k + 1 + f % w;
            AS[r * NP + j] -= AS[r * NP + k] * AS[k * NP + j];
        }
        __syncthreads();
    }
    if (!s_bad)
        for (int c = tid; c < NP; c += nth) {
            // column c of A_S^{-1} into X_S1[row][c]
            double *X = gXS1 + c;
            for (int row = 0; row < NP; row++) X[(size_t)row * NP] = row == c ? 1.0 : 0.0;
            for (int k = 0; k < NP; k++) {
                const int pr = s_pv[k];
                if (pr != k) {
                    const double a = X[(size_t)k * NP];
                    X[(size_t)k * NP] = X[(size_t)pr * NP];
                    X[(size_t)pr * NP] = a;
                }
            }
            for (int k = 0; k < NP; k++) {
                const double yk = X[(size_t)k * NP];
                for (int r = k + 1; r < NP; r++) X[(size_t)r * NP] -= AS[r * NP + k] * yk;
            }
            for (int k = NP - 1; k >= 0; k--) {
                double acc = X[(size_t)k * NP];
                for (int j = k + 1; j < NP; j++) acc -= AS[k * NP + j] * X[(size_t)j * NP];
                X[(size_t)k * NP] = acc / AS[k * NP + k];
            }
        }
    __syncthreads();
    // TMP = Hn A_S^{-1}, Hn[i][k] = sqrt2 Im S^{(l,m)}(y_i), in the freed space
    double *TMP = sm;
    for (int i = tid; i < NP; i += nth) {
        cd tb[NJK];
        harmonic_table<P>(syn + 3 * i, tb);
        double hn[NP];
        for (int k = 0; k < NP; k++) {
            int l, m;
            lm_of(k, l, m);
            hn[k] = sq2 * tb[jk_index(l, m)].y;
        }
        for (int j = 0; j < NP; j++) {
            double a = 0;
            for (int k = 0; k < NP; k++) a += hn[k] * gXS1[(size_t)k * NP + j];
            TMP[i * NP + j] = a;
        }
    }
    __syncthreads();
    // X_S2 = X_D TMP, and the double-float copies of the mixed path
    for (int w = tid; w < 4 * NP * NP; w += nth) {
        const int row = w / NP, i = w % NP;
        double a = 0;
        for (int k = 0; k < NP; k++) a += gXD[(size_t)row * NP + k] * TMP[k * NP + i];
        gXS2[w] = a;
        if (pd.XD2) {
            const size_t o2 = (size_t)pid * pd_X(pd.pmax) + w;
            pd.XD2[o2] = split2f(gXD[w]);
            pd.XSp2[o2] = split2f(gXSp[w]);
            pd.XS22[o2] = split2f(a);
        }
    }
    if (pd.XS12)
        for (int w = tid; w < NP * NP; w += nth) pd.XS12[(size_t)pid * pd_XS1(pd.pmax) + w] = split2f(gXS1[w]);
}

template <int P>
__global__ void __launch_bounds__(256) k_precompute(const OrderTables *__restrict__ tab,
                                                    const int32_t *__restrict__ plist, int n,
                                                    const int64_t *__restrict__ node_off,
                                                    const double *__restrict__ xyz,
                                                    const double *__restrict__ nrm, PatchData pd) {
    using Z = PreSizes<P>;
    constexpr int NP = Z::NP, PT = Z::PT, NJK = Z::NJK, NS = Z::NS, NUP = Z::NUP;
    extern __shared__ double sm[];
    const int b = blockIdx.x;
    if (b >= n) return;
    const int pid = plist[b];
    const int tid = threadIdx.x, nth = blockDim.x;
    const int64_t o = node_off[pid];
    double *sx = sm + Z::SX_OFF, *sn = sm + Z::SN_OFF, *sg = sm + Z::SG_OFF, *sey = sm + Z::EY_OFF;
    double *sea = sm + Z::EA_OFF, *syn = sm + Z::YN_OFF, *fr = sm + Z::FR_OFF, *snl = sm + Z::SNL_OFF;
    __shared__ int s_bad;
    if (tid == 0) s_bad = 0;
    for (int i = tid; i < 3 * NP; i += nth) {
        sx[i] = xyz[3 * o + i];
        sn[i] = nrm[3 * o + i];
    }
    __syncthreads();
    // node interpolant at edge Gauss nodes and vertices (global coordinates)
    for (int w = tid; w < NS * 3; w += nth) {
        int row = w / 3, a = w % 3;
        double s = 0;
        for (int i = 0; i < NP; i++) s += tab->Eint[row * NP + i] * sx[3 * i + a];
        sg[w] = s;
    }
    __syncthreads();
    if (tid == 0) {
        const double *V0 = sg + 3 * (3 * PT), *V1 = V0 + 3, *V2 = V0 + 6;
        double c[3], e01[3], e12[3], e20[3], e02[3];
        for (int a = 0; a < 3; a++) {
            c[a] = (V0[a] + V1[a] + V2[a]) / 3.0;
            e01[a] = V1[a] - V0[a];
            e12[a] = V2[a] - V1[a];
            e20[a] = V0[a] - V2[a];
            e02[a] = V2[a] - V0[a];
        }
        double nz[3] = {e01[1] * e02[2] - e01[2] * e02[1], e01[2] * e02[0] - e01[0] * e02[2],
                        e01[0] * e02[1] - e01[1] * e02[0]};
        double nzl = sqrt(nz[0] * nz[0] + nz[1] * nz[1] + nz[2] * nz[2]);
        double L0 = sqrt(e01[0] * e01[0] + e01[1] * e01[1] + e01[2] * e01[2]);
        double L1 = sqrt(e12[0] * e12[0] + e12[1] * e12[1] + e12[2] * e12[2]);
        double L2 = sqrt(e20[0] * e20[0] + e20[1] * e20[1] + e20[2] * e20[2]);
        const double *exs = e01;
        double Lm = L0;
        if (L1 > Lm) { Lm = L1; exs = e12; }
        if (L2 > Lm) { Lm = L2; exs = e20; }
        if (!(nzl > 0.0) || !(Lm > 0.0)) s_bad = 1;
        double ez[3] = {nz[0] / nzl, nz[1] / nzl, nz[2] / nzl};
        double ex[3] = {exs[0] / Lm, exs[1] / Lm, exs[2] / Lm};
        double ey[3] = {ez[1] * ex[2] - ez[2] * ex[1], ez[2] * ex[0] - ez[0] * ex[2], ez[0] * ex[1] - ez[1] * ex[0]};
        for (int a = 0; a < 3; a++) {
            fr[a] = c[a];
            fr[3 + 3 * a + 0] = ex[a];
            fr[3 + 3 * a + 1] = ey[a];
            fr[3 + 3 * a + 2] = ez[a];
        }
        fr[12] = 1.0 / Lm;
        double rp = 0;
        for (int i = 0; i < NP + 3; i++) {
            const double *q = i < NP ? sx + 3 * i : V0 + 3 * (i - NP);
            double d0 = q[0] - c[0], d1 = q[1] - c[1], d2 = q[2] - c[2];
            double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
            rp = r > rp ? r : rp;
        }
        double *bd = pd.bounds + (size_t)pid * PD_BOUNDS;
        bd[0] = c[0]; bd[1] = c[1]; bd[2] = c[2]; bd[3] = rp; bd[4] = Lm;
    }
    __syncthreads();
    for (int i = tid; i < 16; i += nth) pd.frame[(size_t)pid * PD_FRAME + i] = i < 13 ? fr[i] : 0.0;
    const double sc = fr[12];
    // local coordinates of nodes, normals, edge samples
    for (int w = tid; w < NP * 3; w += nth) {
        int i = w / 3, bb = w % 3;
        double sy = 0, sv = 0;
        for (int a = 0; a < 3; a++) {
            sy += fr[3 + 3 * a + bb] * (sx[3 * i + a] - fr[a]);
            sv += fr[3 + 3 * a + bb] * sn[3 * i + a];
        }
        syn[w] = sc * sy;
        snl[w] = sv;
    }
    __syncthreads();
    for (int w = tid; w < 3 * PT * 3; w += nth) {
        int q = w / 3, bb = w % 3;
        double sy = 0;
        for (int a = 0; a < 3; a++) sy += fr[3 + 3 * a + bb] * (sg[3 * q + a] - fr[a]);
        sey[w] = sc * sy;
    }
    __syncthreads();
    // Legendre coefficients of the edges: a_n = (2n+1)/2 sum_q w_q y(t_q) P_n(t_q)
    for (int w = tid; w < 3 * P * 3; w += nth) {
        int e = w / (3 * P), rem = w % (3 * P), nn = rem / 3, a = rem % 3;
        double s = 0;
        for (int q = 0; q < PT; q++) s += tab->LegW[nn * PT + q] * sey[3 * (e * PT + q) + a];
        sea[w] = s;
    }
    __syncthreads();
    double *g_ea = pd.ea + (size_t)pid * pd_ea(pd.pmax);
    double *g_ey = pd.ey + (size_t)pid * pd_ey(pd.pmax);
    double *g_et = pd.et + (size_t)pid * pd_ey(pd.pmax);
    double *g_eyu = pd.eyu + (size_t)pid * pd_eyu(pd.pmax);
    double *g_yn = pd.ynode + (size_t)pid * pd_ynode(pd.pmax);
    for (int w = tid; w < 9 * P; w += nth) g_ea[w] = sea[w];
    for (int w = tid; w < 9 * PT; w += nth) g_ey[w] = sey[w];
    for (int w = tid; w < 3 * NP; w += nth) g_yn[w] = syn[w];
    // monomial coefficients of the local node interpolant X(u, v) = sum_ab xm[ab] u^a v^b
    double *g_xm = pd.xm + (size_t)pid * pd_ynode(pd.pmax);
    for (int w = tid; w < 3 * NP; w += nth) {
        const int ab = w / 3, a = w % 3;
        double v = 0.0;
        for (int i = 0; i < NP; i++) v = fma(tab->Mmon[ab * NP + i], syn[3 * i + a], v);
        g_xm[w] = v;
    }
    for (int w = tid; w < 3 * PT * 3; w += nth) {
        int q = w / 3, a = w % 3, e = q / PT, qq = q % PT;
        double s = 0;
        for (int nn = 0; nn < P; nn++) s += sea[(e * P + nn) * 3 + a] * tab->dLeg[qq * P + nn];
        g_et[w] = s;
    }
    for (int w = tid; w < 3 * NUP * 3; w += nth) {
        int q = w / 3, a = w % 3, e = q / NUP, ss = q % NUP;
        double s = 0;
        for (int nn = 0; nn < P; nn++) s += sea[(e * P + nn) * 3 + a] * tab->LegU[ss * P + nn];
        g_eyu[w] = s;
    }
    // Step 3: harmonics at the edge samples
    cd *etab = reinterpret_cast<cd *>(sm);  // phase A: [3PT][NJK]
    for (int q = tid; q < 3 * PT; q += nth) harmonic_table<P>(sey + 3 * q, etab + q * NJK);
    __syncthreads();
    cd *g_eg = pd.eg + (size_t)pid * pd_eg(pd.pmax);
    cd *g_eh = pd.eh + (size_t)pid * pd_eg(pd.pmax);
    __syncthreads();
    for (int w = tid; w < 3 * PT * NJK; w += nth) {
        int q = w / NJK, jk = w % NJK;
        int j = 0;
        while (jk_index(j + 1, 0) <= jk) j++;
        int k = jk - jk_index(j, 0);
        cd g[3] = {mkc(0, 0), mkc(0, 0), mkc(0, 0)}, hv[3] = {mkc(0, 0), mkc(0, 0), mkc(0, 0)};
        if (j >= 1) hgrad(etab + q * NJK, j, k, g);
        if (j >= 2) {
            cd H[6];
            hhess(etab + q * NJK, j, k, H);
            // g_et is global; reconstruct tau from coefficients for this sample
            int e = q / PT, qq = q % PT;
            double tau[3];
            for (int a = 0; a < 3; a++) {
                double s = 0;
                for (int nn = 0; nn < P; nn++) s += sea[(e * P + nn) * 3 + a] * tab->dLeg[qq * P + nn];
                tau[a] = s;
            }
            hv[0] = cadd(cadd(cscale(H[0], tau[0]), cscale(H[1], tau[1])), cscale(H[2], tau[2]));
            hv[1] = cadd(cadd(cscale(H[1], tau[0]), cscale(H[3], tau[1])), cscale(H[4], tau[2]));
            hv[2] = cadd(cadd(cscale(H[2], tau[0]), cscale(H[4], tau[1])), cscale(H[5], tau[2]));
        }
        for (int a = 0; a < 3; a++) {
            g_eg[(size_t)w * 3 + a] = g[a];
            g_eh[(size_t)w * 3 + a] = hv[a];
            if (pd.eg2) {
                pd.eg2[(size_t)pid * pd_eg(pd.pmax) + (size_t)w * 3 + a] = split4(g[a]);
                pd.eh2[(size_t)pid * pd_eg(pd.pmax) + (size_t)w * 3 + a] = split4(hv[a]);
            }
        }
    }
    __syncthreads();
    if constexpr (!Z::BIGP) {
    // Steps 1-2: fit systems.  Node harmonic tables first.
    double *M = sm + Z::M_OFF, *W = sm + Z::W_OFF, *AS = sm + Z::AS_OFF, *ASI = sm + Z::ASI_OFF;
    double *HN = sm + Z::HN_OFF, *TMP = sm + Z::TMP_OFF;
    cd *ntab = reinterpret_cast<cd *>(sm + Z::TAB_OFF);
    for (int i = tid; i < NP; i += nth) harmonic_table<P>(syn + 3 * i, ntab + i * NJK);
    __syncthreads();
    const double sq2 = 1.4142135623730951;
    for (int w = tid; w < NP * NP; w += nth) {
        int i = w / NP, lm = w % NP;
        int l = 1;
        while ((l + 1) * l / 2 <= lm) l++;
        int m = lm - l * (l - 1) / 2 + 1;
        cd g[3];
        hgrad(ntab + i * NJK, l, m, g);
        double F1 = sq2 * g[0].y, F2 = sq2 * g[1].y, F3 = sq2 * g[2].y;
        double *q = M + 4 * w;
        q[0] = 0.0; q[1] = F1; q[2] = F2; q[3] = F3;
        const double *nu = snl + 3 * i;
        AS[w] = F1 * nu[0] + F2 * nu[1] + F3 * nu[2];
        HN[w] = sq2 * ntab[i * NJK + jk_index(l, m)].y;
        ASI[w] = (i == lm) ? 1.0 : 0.0;
    }
    for (int w = tid; w < NP * 2 * NP; w += nth) {
        int r = w / (2 * NP), c = w % (2 * NP);
        double *q = W + 4 * w;
        q[0] = q[1] = q[2] = q[3] = 0.0;
        if (c < NP && r == c) q[0] = 1.0;
        if (c >= NP && r == c - NP) { q[1] = snl[3 * r]; q[2] = snl[3 * r + 1]; q[3] = snl[3 * r + 2]; }
    }
    __syncthreads();
    // Conditioning (Sec. 5.1): kappa_1(A) = ||A||_1 ||A^{-1}||_1 in the paper's normalisation
    // R_l^m = d_lm Rn_l^m.  Every column (lm, component) of A holds the three components of
    // d_lm grad H^{(l,m)} at the nodes, so ||A||_1 = max_lm d_lm sum_i (|F1| + |F2| + |F3|).
    // TMP is free until the scalar fit is done.
    __shared__ double s_anorm;
    if (pd.kappa) {
        for (int lm = tid; lm < NP; lm += nth) {
            double s = 0;
            for (int i = 0; i < NP; i++) {
                const double *q = M + 4 * (i * NP + lm);
                s += fabs(q[1]) + fabs(q[2]) + fabs(q[3]);
            }
            TMP[lm] = s * paper_norm(lm);
        }
        __syncthreads();
        if (tid == 0) {
            double a = 0;
            for (int lm = 0; lm < NP; lm++) a = fmax(a, TMP[lm]);
            s_anorm = a;
        }
    }
    // quaternion Gaussian elimination (left multiplication: sum_j M_rj c_j = W_r)
    __shared__ int s_piv;
    q4 *Mq = reinterpret_cast<q4 *>(M), *Wq = reinterpret_cast<q4 *>(W), *Lq = reinterpret_cast<q4 *>(sm + Z::LB_OFF);
    for (int k = 0; k < NP; k++) {
        if (tid == 0) {
            int pr = k;
            double best = qnorm2(Mq[k * NP + k]);
            for (int r = k + 1; r < NP; r++) {
                double v = qnorm2(Mq[r * NP + k]);
                if (v > best) { best = v; pr = r; }
            }
            if (!(best > 0.0)) s_bad = 1;
            s_piv = pr;
        }
        __syncthreads();
        const int pr = s_piv;
        if (pr != k) {
            for (int j = tid; j < NP; j += nth) { q4 t = Mq[k * NP + j]; Mq[k * NP + j] = Mq[pr * NP + j]; Mq[pr * NP + j] = t; }
            for (int j = tid; j < 2 * NP; j += nth) { q4 t = Wq[k * 2 * NP + j]; Wq[k * 2 * NP + j] = Wq[pr * 2 * NP + j]; Wq[pr * 2 * NP + j] = t; }
        }
        __syncthreads();
        if (s_bad) break;
        const q4 inv = qinv(Mq[k * NP + k]);
        for (int r = k + 1 + tid; r < NP; r += nth) Lq[r] = qmul(Mq[r * NP + k], inv);
        __syncthreads();
        const int rows = NP - k - 1, cols = (NP - k - 1) + 2 * NP;
        for (int w = tid; w < rows * cols; w += nth) {
            int r = k + 1 + w / cols, c = w % cols;
            if (c < NP - k - 1) {
                int j = k + 1 + c;
                Mq[r * NP + j] = qsub(Mq[r * NP + j], qmul(Lq[r], Mq[k * NP + j]));
            } else {
                int j = c - (NP - k - 1);
                Wq[r * 2 * NP + j] = qsub(Wq[r * 2 * NP + j], qmul(Lq[r], Wq[k * 2 * NP + j]));
            }
        }
        __syncthreads();
    }
    // back substitution, one right-hand side per thread: c_k = M_kk^{-1} (W_k - sum M_kj c_j)
    if (!s_bad) {
        for (int c = tid; c < 2 * NP; c += nth) {
            for (int k = NP - 1; k >= 0; k--) {
                q4 acc = Wq[k * 2 * NP + c];
                for (int j = k + 1; j < NP; j++) acc = qsub(acc, qmul(Mq[k * NP + j], Wq[j * 2 * NP + c]));
                Wq[k * 2 * NP + c] = qmul(qinv(Mq[k * NP + k]), acc);
            }
        }
    }
    __syncthreads();
    // ||A^{-1}||_1: column (i, 0) of A^{-1} is the fit of a unit density at node i, column
    // (i, r) for r > 0 is that fit right-multiplied by a unit quaternion (the system is
    // left-multiplication by quaternions), which only permutes and negates components.
    // Coefficients in the paper's normalisation are the device ones divided by d_lm.
    if (pd.kappa) {
        for (int i = tid; i < NP; i += nth) {
            double s = 0;
            for (int lm = 0; lm < NP; lm++) {
                const double *q = W + 4 * (lm * 2 * NP + i);
                s += (fabs(q[0]) + fabs(q[1]) + fabs(q[2]) + fabs(q[3])) / paper_norm(lm);
            }
            TMP[NP + i] = s;
        }
        __syncthreads();
        if (tid == 0) {
            double a = 0;
            for (int i = 0; i < NP; i++) a = fmax(a, TMP[NP + i]);
            pd.kappa[pid] = (s_bad || !(a == a)) ? INFINITY : s_anorm * a;
        }
    }
    // scalar fit: LU with partial pivoting on A_S, identity right-hand sides
    // (the exit test reads s_bad only after a barrier, so that all threads leave together)
    for (int k = 0; k < NP; k++) {
        if (tid == 0) {
            int pr = k;
            double best = fabs(AS[k * NP + k]);
            for (int r = k + 1; r < NP; r++)
                if (fabs(AS[r * NP + k]) > best) { best = fabs(AS[r * NP + k]); pr = r; }
            if (!(best > 0.0)) s_bad = 1;
            s_piv = pr;
        }
        __syncthreads();
        if (s_bad) break;
        const int pr = s_piv;
        if (pr != k)
            for (int j = tid; j < NP; j += nth) {
                double t = AS[k * NP + j]; AS[k * NP + j] = AS[pr * NP + j]; AS[pr * NP + j] = t;
                t = ASI[k * NP + j]; ASI[k * NP + j] = ASI[pr * NP + j]; ASI[pr * NP + j] = t;
            }
        __syncthreads();
        const double piv = AS[k * NP + k];
        const int rows = NP - k - 1;
        for (int w = tid; w < rows * 2 * NP; w += nth) {
            int r = k + 1 + w / (2 * NP), c = w % (2 * NP);
            double f = AS[r * NP + k] / piv;
            if (c < NP) {
                if (c > k) AS[r * NP + c] -= f * AS[k * NP + c];
            } else {
                ASI[r * NP + (c - NP)] -= f * ASI[k * NP + (c - NP)];
            }
        }
        __syncthreads();
        for (int r = k + 1 + tid; r < NP; r += nth) AS[r * NP + k] = 0.0;
        __syncthreads();
    }
    if (!s_bad)
        for (int c = tid; c < NP; c += nth)
            for (int k = NP - 1; k >= 0; k--) {
                double acc = ASI[k * NP + c];
                for (int j = k + 1; j < NP; j++) acc -= AS[k * NP + j] * ASI[j * NP + c];
                ASI[k * NP + c] = acc / AS[k * NP + k];
            }
    __syncthreads();
    // TMP = Hn A_S^{-1}
    for (int w = tid; w < NP * NP; w += nth) {
        int i = w / NP, j = w % NP;
        double s = 0;
        for (int k = 0; k < NP; k++) s += HN[i * NP + k] * ASI[k * NP + j];
        TMP[w] = s;
    }
    __syncthreads();
    double *gXD = pd.XD + (size_t)pid * pd_X(pd.pmax), *gXSp = pd.XSp + (size_t)pid * pd_X(pd.pmax);
    double *gXS2 = pd.XS2 + (size_t)pid * pd_X(pd.pmax), *gXS1 = pd.XS1 + (size_t)pid * pd_XS1(pd.pmax);
    for (int w = tid; w < 4 * NP * NP; w += nth) {
        int row = w / NP, i = w % NP;       // row = comp * NP + lm
        int comp = row / NP, lm = row % NP;
        const double *qd = W + 4 * (lm * 2 * NP + i);
        const double *qs = W + 4 * (lm * 2 * NP + NP + i);
        gXD[w] = qd[comp];
        gXSp[w] = qs[comp];
        double s = 0;
        for (int k = 0; k < NP; k++) s += W[4 * (lm * 2 * NP + k) + comp] * TMP[k * NP + i];
        gXS2[w] = s;
        if (pd.XD2) {
            const size_t o2 = (size_t)pid * pd_X(pd.pmax) + w;
            pd.XD2[o2] = split2f(qd[comp]);
            pd.XSp2[o2] = split2f(qs[comp]);
            pd.XS22[o2] = split2f(s);
        }
    }
    for (int w = tid; w < NP * NP; w += nth) {
        gXS1[w] = ASI[w];
        if (pd.XS12) pd.XS12[(size_t)pid * pd_XS1(pd.pmax) + w] = split2f(ASI[w]);
    }
    } else {
        fit_big<P>(sm, syn, snl, pd, pid, tid, nth, s_bad);
    }
    if (tid == 0) pd.status[pid] = s_bad;
}

template <int P>
cudaError_t launch_pre(const OrderTables *d_tab, const int32_t *d_plist, int n, const int64_t *d_node_off,
                       const double *d_xyz, const double *d_nrm, PatchData pd, cudaStream_t st) {
    size_t bytes = PreSizes<P>::BYTES;
    cudaError_t e = cudaFuncSetAttribute(k_precompute<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    if (n <= 0) return cudaSuccess;
    k_precompute<P><<<n, 256, bytes, st>>>(d_tab, d_plist, n, d_node_off, d_xyz, d_nrm, pd);
    RRQ_COUNT_LAUNCH();
    return cudaGetLastError();
}

}  // namespace

cudaError_t rrq_launch_precompute(int p, const OrderTables *d_tab, const int32_t *d_plist, int n,
                                  const int64_t *d_node_off, const double *d_xyz, const double *d_nrm,
                                  PatchData pd, cudaStream_t st) {
    switch (p) {
        case 2: return launch_pre<2>(d_tab, d_plist, n, d_node_off, d_xyz, d_nrm, pd, st);
        case 3: return launch_pre<3>(d_tab, d_plist, n, d_node_off, d_xyz, d_nrm, pd, st);
        case 4: return launch_pre<4>(d_tab, d_plist, n, d_node_off, d_xyz, d_nrm, pd, st);
        case 5: return launch_pre<5>(d_tab, d_plist, n, d_node_off, d_xyz, d_nrm, pd, st);
        case 6: return launch_pre<6>(d_tab, d_plist, n, d_node_off, d_xyz, d_nrm, pd, st);
        case 7: return launch_pre<7>(d_tab, d_plist, n, d_node_off, d_xyz, d_nrm, pd, st);
        case 8: return launch_pre<8>(d_tab, d_plist, n, d_node_off, d_xyz, d_nrm, pd, st);
        case 9: return launch_pre<9>(d_tab, d_plist, n, d_node_off, d_xyz, d_nrm, pd, st);
        case 10: return launch_pre<10>(d_tab, d_plist, n, d_node_off, d_xyz, d_nrm, pd, st);
        case 11: return launch_pre<11>(d_tab, d_plist, n, d_node_off, d_xyz, d_nrm, pd, st);
        case 12: return launch_pre<12>(d_tab, d_plist, n, d_node_off, d_xyz, d_nrm, pd, st);
        case 13: return launch_pre<13>(d_tab, d_plist, n, d_node_off, d_xyz, d_nrm, pd, st);
        case 14: return launch_pre<14>(d_tab, d_plist, n, d_node_off, d_xyz, d_nrm, pd, st);
        default: return cudaErrorInvalidValue;
    }
}
