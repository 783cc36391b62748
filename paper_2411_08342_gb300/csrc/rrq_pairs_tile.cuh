// Tiled form of the per-pair kernel: one CTA takes a tile of T consecutive pair items
// (grouped by patch) and every phase of Sec. 4 Steps 4-8 runs over the flattened
// (pair, item) index space with all threads of the CTA, so that warp instructions
// carry full lanes (a warp per pair leaves lanes idle wherever a phase has fewer than
// 32 items: 3 edges, p+1 columns, n_p basis functions, ...).  Phases that end in a
// per-pair reduction (choice of u, Omega_0 panels, Omega vector) run warp-per-pair.
// Each phase is one step of the per-pair algorithm summarised in rrq_pairs.cuh.
#pragma once
#include "rrq_pairs.cuh"

namespace rrqk {

template <int P>
struct TileCfg {
    static constexpr int THREADS = 128;
};

// double-float accumulator: value = h + l (two FP32 numbers, about 48 bits)
struct dfa {
    float h, l;
};

// acc += (ah + al) * (bh + bl): exact FP32 product by FMA, compensated (TwoSum) sum
__device__ __forceinline__ void dfmac(dfa &acc, float ah, float al, float bh, float bl) {
    const float p = ah * bh;
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    const float s = acc.h + p;
    const float bb = s - acc.h;
    const float err = (acc.h - (s - bb)) + (p - bb);
    acc.h = s;
    acc.l += err + e;
}

__device__ __forceinline__ double dfval(const dfa &a) { return (double)a.h + (double)a.l; }

// (hi, lo) with |lo| <= ulp(hi) / 2 (fast two-sum)
__device__ __forceinline__ dfa dfnorm(const dfa &a) {
    const float s = a.h + a.l;
    return dfa{s, a.l - (s - a.h)};
}

// Double-float values (h + l, |l| <= ulp(h)/2) for the mixed path's Omega_0 panels.
__device__ __forceinline__ dfa dfs(double x) {
    const float h = __double2float_rn(x);
    return dfa{h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ dfa dfadd(dfa a, dfa b) {
    const float s = a.h + b.h, bb = s - a.h;
    const float e = (a.h - (s - bb)) + (b.h - bb) + a.l + b.l;
    const float t = s + e;
    return dfa{t, e - (t - s)};
}
__device__ __forceinline__ dfa dfneg(dfa a) { return dfa{-a.h, -a.l}; }
__device__ __forceinline__ dfa dfmul(dfa a, dfa b) {
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
    const float t = p + e;
    return dfa{t, e - (t - p)};
}
// a * b + c
__device__ __forceinline__ dfa dffma(dfa a, dfa b, dfa c) { return dfadd(dfmul(a, b), c); }
// 1/a: the FP32 reciprocal corrected by one Newton step in double-float
__device__ __forceinline__ dfa dfrcp(dfa a) {
    const float y = 1.0f / a.h;
    const float e = fmaf(-a.h, y, 1.0f) - a.l * y;   // 1 - a y to double-float accuracy
    const float c = y * e, t = y + c;
    return dfa{t, c - (t - y)};
}
// 1/sqrt(a), a > 0: rsqrtf corrected by one Newton step (y + y (1 - a y^2) / 2)
__device__ __forceinline__ dfa dfrsqrt(dfa a) {
    const float y = rsqrtf(a.h);
    const dfa yy = dfmul(dfa{y, 0.0f}, dfa{y, 0.0f});
    const dfa ay2 = dfmul(a, yy);
    const float e = (1.0f - ay2.h) - ay2.l;
    const float c = 0.5f * y * e, t = y + c;
    return dfa{t, c - (t - y)};
}

// acc += Im(a b) for complex numbers stored as (re.hi, re.lo, im.hi, im.lo)
__device__ __forceinline__ void dfim(dfa &acc, const float4 a, const float4 b) {
    dfmac(acc, a.x, a.y, b.z, b.w);
    dfmac(acc, a.z, a.w, b.x, b.y);
}

// complex (re, im) double-float pair of two accumulators
__device__ __forceinline__ float4 dfc(const dfa &re, const dfa &im) {
    const dfa r = dfnorm(re), i = dfnorm(im);
    return make_float4(r.h, r.l, i.h, i.l);
}

// conjugation rules of tget / kflip for double-float complex tables
__device__ __forceinline__ float4 kflip4(float4 v, int k) {
    if (k >= 0) return v;
    v.z = -v.z;
    v.w = -v.w;
    if ((-k) & 1) { v.x = -v.x; v.y = -v.y; v.z = -v.z; v.w = -v.w; }
    return v;
}
__device__ __forceinline__ float4 tget4(const float4 *S, int n, int q) {
    if (n < 0) return make_float4(0.f, 0.f, 0.f, 0.f);
    const int aq = q < 0 ? -q : q;
    if (aq > n) return make_float4(0.f, 0.f, 0.f, 0.f);
    return kflip4(S[jk_index(n, aq)], q);
}

__device__ __forceinline__ float4 split4c(cd v) {
    const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
    return make_float4(rh, __double2float_rn(v.x - (double)rh), ih, __double2float_rn(v.y - (double)ih));
}
__device__ __forceinline__ float2 split2d(double x) {
    const float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(x - (double)h));
}

// Item f of phase K: (pair, harmonic jk) with the j >= 2 harmonics (jk >= 3) of all pairs
// first, then the two j = 1 harmonics of all pairs.
template <int NJK>
__device__ __forceinline__ void kitem(int f, int nt, int &pl, int &jk) {
    constexpr int N2 = NJK - 3;
    if (f < nt * N2) {
        pl = f / N2;
        jk = 3 + f % N2;
    } else {
        const int g = f - nt * N2;
        pl = g >> 1;
        jk = 1 + (g & 1);
    }
}

template <int P, bool MIX, int T, bool EVAL, bool ROT>
__global__ void __launch_bounds__(128) k_pairs_tile(const PairArgs a, unsigned long long *tile_ctr) {
    const OrderTables *__restrict__ tab = a.tab;
    const PairItem *__restrict__ items = a.items;
    const int64_t nitems = a.nitems;
    const PatchData &pd = a.pd;
    const int64_t *__restrict__ node_off = a.node_off;
    const int64_t *__restrict__ col_off = a.pd.col_off ? a.pd.col_off : a.node_off;
    const double *__restrict__ xyz = a.xyz, *__restrict__ nrm = a.nrm, *__restrict__ wts = a.wts;
    const double *__restrict__ txyz = a.txyz, *__restrict__ tnrm = a.tnrm;
    const int64_t *__restrict__ tself = a.tself;
    const uint32_t mask = a.mask;
    double *vS = a.val[0], *vD = a.val[1], *vSp = a.val[2], *vDp = a.val[3];
    int32_t *col = a.col;
    BuildCounters *cnt = a.cnt;
    using Z = PairSm<P>;
    constexpr int NP = Z::NP, PT = Z::PT, NJK = Z::NJK, NS = Z::NS, NUP = Z::NUP;
    extern __shared__ __align__(16) double smraw[];
    __shared__ unsigned int bc[5];
    __shared__ PairItem s_item[T];
    __shared__ int64_t s_base;
    __shared__ int s_self[T];
    __shared__ double s_uz[T];
    __shared__ double s_h0[3 * T], s_h1[3 * T];  // Omega_0 and its nu' derivative per (pair, edge)
    const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nth >> 5;
    const bool wantDP = (mask & RRQ_DP) != 0;
    // kernel groups of the row phase that this build needs
    __shared__ int s_grp[3];
    int ngrp = 0;
    {
        int g[3], n = 0;
        if (mask & (RRQ_D | RRQ_DP)) g[n++] = 0;
        if (mask & RRQ_SP) g[n++] = 1;
        if (mask & RRQ_S) g[n++] = 2;
        if (tid < n) s_grp[tid] = g[tid];
        ngrp = n;
    }
    if (tid < 5) bc[tid] = 0;
    const double inv4pi = 0.07957747154594767, sq2 = 1.4142135623730951;
    constexpr int STRIDE = ROT ? Z::TOTAL_ROT : Z::TOTAL;   // doubles per pair
#define SW(pl) (smraw + (size_t)(pl) * STRIDE)
    // tiles of T consecutive items: grid-stride, or (persistent launch) fetched from a counter
    for (int64_t tile = blockIdx.x;; tile += gridDim.x) {
        __syncthreads();
        if (tid == 0) s_base = (tile_ctr ? (int64_t)atomicAdd(tile_ctr, 1ULL) : tile) * T;
        __syncthreads();
        const int64_t base = s_base;
        if (base >= nitems) break;
        const int nt = (int)min((int64_t)T, nitems - base);
        if (tid < nt) s_item[tid] = items[base + tid];
        __syncthreads();
        // A: frame, target, normal, edge coefficients
        for (int f = tid; f < nt * (19 + 9 * P); f += nth) {
            const int pl = f / (19 + 9 * P), it = f % (19 + 9 * P);
            double *sw = SW(pl);
            const PairItem im = s_item[pl];
            if (it < 13) sw[Z::FR + it] = pd.frame[(size_t)im.P * PD_FRAME + it];
            else if (it < 16) sw[Z::XT + it - 13] = txyz[3 * im.t + it - 13];
            else if (it < 19) sw[Z::NT + it - 16] = tnrm[3 * im.t + it - 16];
            else sw[Z::EA + it - 19] = pd.ea[(size_t)im.P * pd_ea(pd.pmax) + it - 19];
        }
        __syncthreads();
        // B: target in the patch frame; self index
        for (int f = tid; f < nt * 4; f += nth) {
            const int pl = f >> 2, b = f & 3;
            double *sw = SW(pl);
            const PairItem im = s_item[pl];
            if (b < 3) {
                const double *fr = sw + Z::FR;
                double sy = 0, sn = 0;
                for (int a = 0; a < 3; a++) {
                    sy += fr[3 + 3 * a + b] * (sw[Z::XT + a] - fr[a]);
                    sn += fr[3 + 3 * a + b] * sw[Z::NT + a];
                }
                sw[Z::YT + b] = fr[12] * sy;
                sw[Z::NUT + b] = sn;
                if (MIX) reinterpret_cast<float2 *>(sw + Z::FR + 13)[b] = split2d(sn);
            } else {
                const int64_t o = node_off[im.P];
                int si = -1;
                if (tself) {
                    const int64_t sn = tself[im.t];
                    if (sn >= o && sn < o + NP) si = (int)(sn - o);
                }
                s_self[pl] = si;
            }
        }
        __syncthreads();
        // C: edge samples (d, tau, 1/|d|) and target harmonic columns
        for (int f = tid; f < nt * (NS + P + 1); f += nth) {
            const int pl = f / (NS + P + 1), it = f % (NS + P + 1);
            double *sw = SW(pl);
            const size_t ps = (size_t)s_item[pl].P;
            const double *yt = sw + Z::YT;
            if (it < NS) {
                const int q = it;
                const double *ey = pd.ey + ps * pd_ey(pd.pmax) + 3 * q;
                const double *et = pd.et + ps * pd_ey(pd.pmax) + 3 * q;
                const double d0 = yt[0] - ey[0], d1 = yt[1] - ey[1], d2 = yt[2] - ey[2];
                double *dq = sw + Z::DQ, *tau = sw + Z::TAU;
                dq[3 * q] = d0; dq[3 * q + 1] = d1; dq[3 * q + 2] = d2;
                tau[3 * q] = et[0]; tau[3 * q + 1] = et[1]; tau[3 * q + 2] = et[2];
                sw[Z::RINV + q] = rsqrt(d0 * d0 + d1 * d1 + d2 * d2);
            } else {
                target_table<P>(yt, reinterpret_cast<cd *>(sw + Z::ST), it - NS);
            }
        }
        __syncthreads();
        // D: target gradients (the Hessians are formed where they are used, phase L); monomial
        // edge coefficients
        for (int f = tid; f < nt * (NJK + 9 * P); f += nth) {
            const int pl = f / (NJK + 9 * P), it = f % (NJK + 9 * P);
            double *sw = SW(pl);
            if (it < NJK) {
                const int jk = it;
                const cd *St = reinterpret_cast<const cd *>(sw + Z::ST);
                cd *gSt = reinterpret_cast<cd *>(sw + Z::GST);
                int j = 0;
                while (jk_index(j + 1, 0) <= jk) j++;
                const int k = jk - jk_index(j, 0);
                const cd a = tget(St, j - 1, k - 1), b = tget(St, j - 1, k + 1);
                gSt[3 * jk + 0] = tget(St, j - 1, k);
                gSt[3 * jk + 1] = cscale(csub(a, b), 0.5);
                gSt[3 * jk + 2] = cmuli(cscale(cadd(a, b), 0.5));
            } else {
                const int w = it - NJK;
                const int e = w / (3 * P), rem = w % (3 * P), kk = rem / 3, a = rem % 3;
                const double *ea = sw + Z::EA;
                double v = 0.0;
                for (int n = kk; n < P; n++) v = fma(ea[(e * P + n) * 3 + a], tab->L2M[n * P + kk], v);
                if (MIX) reinterpret_cast<float2 *>(sw + Z::EM)[w] = split2d(v);  // (hi, lo) for the panels
                else sw[Z::EM + w] = v;
            }
        }
        __syncthreads();
        // E: choice of u (warp per pair)
        // +e_z for a node of the patch (exterior limit); the side the target is on when its
        // footprint along e_z lies in the patch (k_uside); otherwise the better of +-e_z by
        // the smallest u.(y'-y)/|y'-y| over nodes and edge samples
        for (int pl = warp; pl < nt; pl += nwarp) {
            double *sw = SW(pl);
            const size_t ps = (size_t)s_item[pl].P;
            const int side = s_self[pl] < 0 ? pd.uside[base + pl] : 0;
            if (side != 0) {
                if (lane == 0) s_uz[pl] = (double)side;
                continue;
            }
            const double *yt = sw + Z::YT, *dq = sw + Z::DQ;
            double mplus = 2.0, mminus = 2.0;
            for (int s2 = lane; s2 < NP + NS; s2 += 32) {
                double dz, dl2;
                if (s2 < NP) {
                    const double *yn = pd.ynode + ps * pd_ynode(pd.pmax) + 3 * s2;
                    const double d0 = yt[0] - yn[0], d1 = yt[1] - yn[1];
                    dz = yt[2] - yn[2];
                    dl2 = d0 * d0 + d1 * d1 + dz * dz;
                } else {
                    const int q = s2 - NP;
                    dz = dq[3 * q + 2];
                    dl2 = dq[3 * q] * dq[3 * q] + dq[3 * q + 1] * dq[3 * q + 1] + dz * dz;
                }
                if (dl2 != 0.0) {
                    const double cz = dz * rsqrt(dl2);
                    mplus = fmin(mplus, cz);
                    mminus = fmin(mminus, -cz);
                }
            }
            mplus = warp_min(mplus);
            mminus = warp_min(mminus);
            const double uz = (s_self[pl] < 0 && mminus > mplus) ? -1.0 : 1.0;
            if (lane == 0) {
                s_uz[pl] = uz;
                if ((uz > 0 ? mplus : mminus) < -0.5) atomicAdd(&bc[2], 1u);
            }
        }
        // F: complex roots (from k_roots), singularity-swap moments and weights, one thread per (pair, edge)
        for (int f = tid; f < nt * 3; f += nth) {
            const int pl = f / 3, e = f % 3;
            double *sw = SW(pl);
            const EdgeRoot rt = pd.roots[(base + pl) * 3 + e];
            const int conv = rt.z != 0.0, ssq = rt.w != 0.0;
            double *t0s = sw + Z::T0;
            t0s[4 * e] = rt.x;
            t0s[4 * e + 1] = rt.y;
            t0s[4 * e + 2] = rt.z;
            t0s[4 * e + 3] = rt.w;
            if (!conv) atomicAdd(&bc[0], 1u);
            if (conv && rt.y < 1e-14 && fabs(rt.x) <= 1.0) atomicAdd(&bc[1], 1u);
            atomicAdd(ssq ? &bc[3] : &bc[4], 1u);
            if (ssq) {
                const double a = rt.x, bi = rt.y, c0 = a * a + bi * bi;
                const double sp = sqrt((1 - a) * (1 - a) + bi * bi), sm = sqrt((1 + a) * (1 + a) + bi * bi);
                double *J = sw + Z::MOM + 2 * NUP * e, *K = J + PT;
                J[0] = asinh((1 - a) / bi) + asinh((1 + a) / bi);
                J[1] = (sp - sm) + a * J[0];
                for (int i = 2; i < PT; i++) {
                    const double br = ((i - 1) & 1) ? sp + sm : sp - sm;
                    J[i] = (br + (2.0 * i - 1.0) * a * J[i - 1] - (i - 1.0) * c0 * J[i - 2]) * rcp_small(i);
                }
                if (wantDP) {
                    K[0] = ((1 - a) / sp + (1 + a) / sm) / (bi * bi);
                    K[1] = (1.0 / sm - 1.0 / sp) + a * K[0];
                    for (int i = 0; i + 2 < PT; i++) K[i + 2] = J[i] + 2.0 * a * K[i + 1] - c0 * K[i];
                }
            }
        }
        __syncthreads();
        // singularity-swap weights lambda = V^{-T} (J or K) in place, one thread per
        // (pair, edge, m); then G1: upsampled kernel values of the edges that take the
        // direct rule (disjoint edges, same scratch)
        if (tid < nt * 6) {
            const int pl = tid / 6, e = (tid >> 1) % 3, m3 = tid & 1;
            double *sw = SW(pl);
            if (sw[Z::T0 + 4 * e + 3] != 0.0 && (m3 == 0 || wantDP))
                dual_vandermonde_solve<PT>(sw + Z::MOM + 2 * NUP * e + m3 * PT, tab->tq, tab->BPr);
        }
        for (int f = tid; f < nt * 3 * NUP; f += nth) {
            const int pl = f / (3 * NUP), rem = f % (3 * NUP), e = rem / NUP, s2 = rem % NUP;
            double *sw = SW(pl);
            if (sw[Z::T0 + 4 * e + 3] != 0.0) continue;
            const double *yt = sw + Z::YT;
            const double *yu = pd.eyu + (size_t)s_item[pl].P * pd_eyu(pd.pmax) + 3 * (e * NUP + s2);
            const double d0 = yt[0] - yu[0], d1 = yt[1] - yu[1], d2 = yt[2] - yu[2];
            const double r2 = d0 * d0 + d1 * d1 + d2 * d2, r = sqrt(r2);
            const double k1 = tab->wu[s2] / r;
            double *up = sw + Z::UP + 2 * NUP * e;
            up[s2] = k1;
            up[NUP + s2] = k1 / r2;
        }
        __syncthreads();
        // G2: modified weights, one thread per (pair, edge, node)
        for (int f = tid; f < nt * 3 * PT; f += nth) {
            const int pl = f / (3 * PT), rem = f % (3 * PT), e = rem / PT, q = rem % PT;
            double *sw = SW(pl);
            const double *t0s = sw + Z::T0;
            double w1, w3;
            if (t0s[4 * e + 3] != 0.0) {
                // lambda (phase F) for m = 1 and m = 3
                const double *J = sw + Z::MOM + 2 * NUP * e, *K = J + PT;
                const double l1 = J[q], l3 = wantDP ? K[q] : 0.0;
                const double dtr = tab->tq[q] - t0s[4 * e], ti = t0s[4 * e + 1];
                const double ratio = sqrt(dtr * dtr + ti * ti) * sw[Z::RINV + e * PT + q];
                w1 = l1 * ratio;
                w3 = wantDP ? l3 * ratio * ratio * ratio : 0.0;
            } else {
                const double *up = sw + Z::UP + 2 * NUP * e;
                double s1 = 0, s3 = 0;
                for (int s2 = 0; s2 < NUP; s2++) {
                    const double L = tab->Lup[s2 * PT + q];
                    s1 = fma(L, up[s2], s1);
                    s3 = fma(L, up[NUP + s2], s3);
                }
                w1 = s1;
                w3 = s3;
            }
            sw[Z::OM1 + e * PT + q] = w1;
            sw[Z::OM3 + e * PT + q] = w3;
        }
        __syncthreads();
        // H, in three parts.  (1) premultiplied per-sample vectors w1 d, w1 (tau x d), w1 nu',
        // w3 (nu'.d) d, one thread per (pair, sample)
        for (int f = tid; f < nt * NS; f += nth) {
            const int pl = f / NS, q = f % NS;
            double *sw = SW(pl);
            const double *nut = sw + Z::NUT, *dq = sw + Z::DQ, *tau = sw + Z::TAU;
            const double w1 = sw[Z::OM1 + q], w3 = sw[Z::OM3 + q];
            const double d0 = dq[3 * q], d1 = dq[3 * q + 1], d2 = dq[3 * q + 2];
            const double t0 = tau[3 * q], t1 = tau[3 * q + 1], t2 = tau[3 * q + 2];
            const double w3n = w3 * (nut[0] * d0 + nut[1] * d1 + nut[2] * d2);
            double vv[12];
            vv[0] = w1 * d0; vv[1] = w1 * d1; vv[2] = w1 * d2;
            vv[3] = w1 * (t1 * d2 - t2 * d1); vv[4] = w1 * (t2 * d0 - t0 * d2); vv[5] = w1 * (t0 * d1 - t1 * d0);
            vv[6] = w1; vv[7] = 0.0; vv[8] = 0.0;
            vv[9] = w3n * d0; vv[10] = w3n * d1; vv[11] = w3n * d2;
            if (!MIX && wantDP) {
                // FP64 with D': w3 (nu'.d) and d itself, for the shared product (0, d)(0, h)
                vv[7] = w3n;
                vv[9] = d0; vv[10] = d1; vv[11] = d2;
            }
            double *wv = sw + Z::WV;
            if (MIX) {
                // the same 12 numbers as (hi, lo) float pairs, in the same slot
                float *of = reinterpret_cast<float *>(wv + 12 * q);
                for (int i = 0; i < 12; i++) {
                    const float hi = __double2float_rn(vv[i]);
                    of[2 * i] = hi;
                    of[2 * i + 1] = __double2float_rn(vv[i] - (double)hi);
                }
            } else {
                double *o = wv + 12 * q;
                for (int i = 0; i < 12; i++) o[i] = vv[i];
            }
        }
        // (2) Omega_0 on graded panels, one half-warp per (pair, edge): an edge away from the
        // target has one panel of RRQ_NOM = 16 points, which fills a half-warp, and the
        // half-warps share the edges evenly whatever the tile size; per-edge partial sums in
        // shared memory
        for (int pe0 = 2 * warp; pe0 < nt * 3; pe0 += 2 * nwarp) {
            const int pe = pe0 + (lane >> 4), hl = lane & 15;
            double o0 = 0.0, do0 = 0.0;
            if (pe < nt * 3) {
            const int pl = pe / 3, e = pe % 3;
            double *sw = SW(pl);
            const double *yt = sw + Z::YT, *nut = sw + Z::NUT, *t0s = sw + Z::T0, *em = sw + Z::EM;
            const double uz = s_uz[pl];
            const double nxu0 = uz * nut[1], nxu1 = -uz * nut[0], nuu = nut[2] * uz;
            {
                const double *cm = em + 3 * P * e;
                const double tr = t0s[4 * e], ti = t0s[4 * e + 1];
                double c, sig;
                if (t0s[4 * e + 2] != 0.0) {
                    c = fmin(fmax(tr, -1.0), 1.0);
                    const double dr = tr - c;
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
                if (MIX) {
                    // the same panels and sums in double-float on the FP32 pipes (about 48 bits)
                    const float2 *cmf = reinterpret_cast<const float2 *>(em) + 3 * P * e;
                    const dfa ytf[3] = {dfs(yt[0]), dfs(yt[1]), dfs(yt[2])};
                    const dfa lof = dfs(lo), hif = dfs(hi), sigf = dfs(sig);
                    const float2 *nf = reinterpret_cast<const float2 *>(sw + Z::FR + 13);
                    const dfa n0 = {nf[0].x, nf[0].y}, n1 = {nf[1].x, nf[1].y}, n2 = {nf[2].x, nf[2].y};
                    const float uzf = (float)uz;
                    dfa a0acc = {0.0f, 0.0f}, a1acc = {0.0f, 0.0f};
                    for (int idx = hl; idx < npan * RRQ_NOM; idx += 16) {
                        const int pan = idx / RRQ_NOM, g = idx % RRQ_NOM;
                        dfa a0, a1;
                        if (pan < nl) {
                            const float pk = ldexpf(1.0f, nl - pan);
                            // pk - 1 and pk/2 - 1 exactly, as (hi, lo) pairs
                            a0 = dfadd(lof, dfneg(dfmul(dfadd(dfa{pk, 0.0f}, dfa{-1.0f, 0.0f}), sigf)));
                            if (a0.h + a0.l < -1.0f) a0 = dfa{-1.0f, 0.0f};
                            a1 = dfadd(lof, dfneg(dfmul(dfadd(dfa{0.5f * pk, 0.0f}, dfa{-1.0f, 0.0f}), sigf)));
                        } else if (pan == nl) {
                            a0 = lof;
                            a1 = hif;
                        } else {
                            const float pk = ldexpf(1.0f, pan - nl);
                            a0 = dfadd(hif, dfmul(dfadd(dfa{0.5f * pk, 0.0f}, dfa{-1.0f, 0.0f}), sigf));
                            a1 = dfadd(hif, dfmul(dfadd(dfa{pk, 0.0f}, dfa{-1.0f, 0.0f}), sigf));
                            if (a1.h + a1.l > 1.0f) a1 = dfa{1.0f, 0.0f};
                        }
                        const dfa mid = dfmul(dfa{0.5f, 0.0f}, dfadd(a0, a1));
                        const dfa half = dfmul(dfa{0.5f, 0.0f}, dfadd(a1, dfneg(a0)));
                        const dfa tt = dffma(half, dfs(tab->tom[g]), mid), wg = dfmul(half, dfs(tab->wom[g]));
                        dfa y[3], dy[3];
                        for (int c = 0; c < 3; c++) {
                            const float2 top = cmf[3 * (P - 1) + c];
                            y[c] = dfa{top.x, top.y};
                            dy[c] = dfa{0.0f, 0.0f};
                        }
                        for (int k = P - 2; k >= 0; k--)
                            for (int c = 0; c < 3; c++) {
                                dy[c] = dffma(dy[c], tt, y[c]);
                                const float2 ck = cmf[3 * k + c];
                                y[c] = dffma(y[c], tt, dfa{ck.x, ck.y});
                            }
                        const dfa d0 = dfadd(ytf[0], dfneg(y[0])), d1 = dfadd(ytf[1], dfneg(y[1]));
                        const dfa d2 = dfadd(ytf[2], dfneg(y[2]));
                        const dfa r2 = dfadd(dfmul(d0, d0), dfadd(dfmul(d1, d1), dfmul(d2, d2)));
                        const dfa ir = dfrsqrt(r2), r = dfmul(r2, ir);
                        const dfa E = dfadd(r, dfmul(dfa{uzf, 0.0f}, d2));
                        const dfa iE = dfrcp(E), inv = dfmul(ir, iE);
                        const dfa N = dfmul(dfa{uzf, 0.0f}, dfadd(dfmul(d1, dy[0]), dfneg(dfmul(d0, dy[1]))));
                        a0acc = dfadd(a0acc, dfneg(dfmul(dfmul(wg, N), inv)));
                        if (wantDP) {
                            const dfa nd = dfadd(dfmul(n0, d0), dfadd(dfmul(n1, d1), dfmul(n2, d2)));
                            // (nu' x u) . tau with u = uz e_z: uz (nu'_y tau_x - nu'_x tau_y)
                            const dfa nxt = dfmul(dfa{uzf, 0.0f}, dfadd(dfmul(n1, dy[0]), dfneg(dfmul(n0, dy[1]))));
                            const dfa t1 = dfmul(dfmul(N, iE), dfadd(dfmul(dfa{uzf, 0.0f}, n2), dfmul(nd, ir)));
                            const dfa t2 = dfmul(dfmul(nd, N), dfmul(ir, ir));
                            const dfa v = dfmul(inv, dfadd(nxt, dfneg(dfadd(t1, t2))));
                            a1acc = dfadd(a1acc, dfneg(dfmul(wg, v)));
                        }
                    }
                    o0 = dfval(a0acc);
                    do0 = dfval(a1acc);
                } else
                for (int idx = hl; idx < npan * RRQ_NOM; idx += 16) {
                    const int pan = idx / RRQ_NOM, g = idx % RRQ_NOM;
                    // panel k away from the central one spans (2^(k-1) - 1) sig .. (2^k - 1) sig
                    // beyond lo (or hi): widths sig, 2 sig, 4 sig, ...
                    double a0, a1;
                    if (pan < nl) {
                        const double pk = ldexp(1.0, nl - pan);
                        a0 = fmax(lo - (pk - 1.0) * sig, -1.0);
                        a1 = lo - (0.5 * pk - 1.0) * sig;
                    } else if (pan == nl) {
                        a0 = lo;
                        a1 = hi;
                    } else {
                        const double pk = ldexp(1.0, pan - nl);
                        a0 = hi + (0.5 * pk - 1.0) * sig;
                        a1 = fmin(hi + (pk - 1.0) * sig, 1.0);
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
            }
            o0 = half_warp_sum(o0);
            if (wantDP) do0 = half_warp_sum(do0);
            if (hl == 0 && pe < nt * 3) {
                s_h0[pe] = o0;
                s_h1[pe] = do0;
            }
        }
        __syncthreads();
        // (3) Omega_0 summed over the edges in order, the Omega vector, warp per pair
        for (int pl = warp; pl < nt; pl += nwarp) {
            double *sw = SW(pl);
            const double *nut = sw + Z::NUT;
            const double o0 = s_h0[3 * pl] + s_h0[3 * pl + 1] + s_h0[3 * pl + 2];
            const double do0 = s_h1[3 * pl] + s_h1[3 * pl + 1] + s_h1[3 * pl + 2];
            const double *dq = sw + Z::DQ, *tau = sw + Z::TAU, *om1 = sw + Z::OM1, *om3 = sw + Z::OM3;
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
                double *Om = sw + Z::OM;
                Om[0] = o0; Om[1] = ov[0]; Om[2] = ov[1]; Om[3] = ov[2];
                Om[4] = do0; Om[5] = dov[0]; Om[6] = dov[1]; Om[7] = dov[2];
            }
        }
        __syncthreads();
        // K: line integrals, one thread per (pair, (j, k >= 0)), j >= 1; the items with j >= 2
        // (V, Q, dQ) come first and the cheap j = 1 items (V only) last, so that warps do not
        // mix the two
        if (MIX) {
            for (int f = tid; f < nt * (NJK - 1); f += nth) {
                int pl, jk;
                kitem<NJK>(f, nt, pl, jk);
                double *sw = SW(pl);
                const size_t ps = (size_t)s_item[pl].P;
                const float *wf = reinterpret_cast<const float *>(sw + Z::WV);
                const double *nut = sw + Z::NUT;
                const float4 *eg = pd.eg2 + ps * pd_eg(pd.pmax);
                const float4 *eh = pd.eh2 + ps * pd_eg(pd.pmax);
                const bool hj = jk >= 3;
                dfa Vr = {0, 0}, Vi = {0, 0}, Q0r = {0, 0}, Q0i = {0, 0}, Q1r = {0, 0}, Q1i = {0, 0}, Q2r = {0, 0}, Q2i = {0, 0};
                dfa Q3r = {0, 0}, Q3i = {0, 0}, D0r = {0, 0}, D0i = {0, 0}, D1r = {0, 0}, D1i = {0, 0}, D2r = {0, 0}, D2i = {0, 0};
                dfa E0r = {0, 0}, E0i = {0, 0}, E1r = {0, 0}, E1i = {0, 0}, E2r = {0, 0}, E2i = {0, 0}, E3r = {0, 0}, E3i = {0, 0};
                for (int q = 0; q < NS; q++) {
                    const float *o = wf + 24 * q;
                    const float4 *g = eg + ((size_t)q * NJK + jk) * 3;
                    const float4 g0 = g[0], g1 = g[1], g2 = g[2];
                    // V += g . (w1 tau x d): values 3, 4, 5
                    dfmac(Vr, o[6], o[7], g0.x, g0.y); dfmac(Vr, o[8], o[9], g1.x, g1.y); dfmac(Vr, o[10], o[11], g2.x, g2.y);
                    dfmac(Vi, o[6], o[7], g0.z, g0.w); dfmac(Vi, o[8], o[9], g1.z, g1.w); dfmac(Vi, o[10], o[11], g2.z, g2.w);
                    if (hj) {
                        const float4 *h = eh + ((size_t)q * NJK + jk) * 3;
                        const float4 h0 = h[0], h1 = h[1], h2 = h[2];
                        const float a0h = o[0], a0l = o[1], a1h = o[2], a1l = o[3], a2h = o[4], a2l = o[5];
                        // (0, w1 d)(0, h) = (-(w1 d).h, (w1 d) x h)
                        dfmac(Q0r, -a0h, -a0l, h0.x, h0.y); dfmac(Q0r, -a1h, -a1l, h1.x, h1.y); dfmac(Q0r, -a2h, -a2l, h2.x, h2.y);
                        dfmac(Q0i, -a0h, -a0l, h0.z, h0.w); dfmac(Q0i, -a1h, -a1l, h1.z, h1.w); dfmac(Q0i, -a2h, -a2l, h2.z, h2.w);
                        dfmac(Q1r, a1h, a1l, h2.x, h2.y); dfmac(Q1r, -a2h, -a2l, h1.x, h1.y);
                        dfmac(Q1i, a1h, a1l, h2.z, h2.w); dfmac(Q1i, -a2h, -a2l, h1.z, h1.w);
                        dfmac(Q2r, a2h, a2l, h0.x, h0.y); dfmac(Q2r, -a0h, -a0l, h2.x, h2.y);
                        dfmac(Q2i, a2h, a2l, h0.z, h0.w); dfmac(Q2i, -a0h, -a0l, h2.z, h2.w);
                        dfmac(Q3r, a0h, a0l, h1.x, h1.y); dfmac(Q3r, -a1h, -a1l, h0.x, h0.y);
                        dfmac(Q3i, a0h, a0l, h1.z, h1.w); dfmac(Q3i, -a1h, -a1l, h0.z, h0.w);
                        if (wantDP) {
                            const float w1h = o[12], w1l = o[13];
                            const float m0h = o[18], m0l = o[19], m1h = o[20], m1l = o[21], m2h = o[22], m2l = o[23];
                            dfmac(D0r, w1h, w1l, h0.x, h0.y); dfmac(D0i, w1h, w1l, h0.z, h0.w);
                            dfmac(D1r, w1h, w1l, h1.x, h1.y); dfmac(D1i, w1h, w1l, h1.z, h1.w);
                            dfmac(D2r, w1h, w1l, h2.x, h2.y); dfmac(D2i, w1h, w1l, h2.z, h2.w);
                            dfmac(E0r, -m0h, -m0l, h0.x, h0.y); dfmac(E0r, -m1h, -m1l, h1.x, h1.y); dfmac(E0r, -m2h, -m2l, h2.x, h2.y);
                            dfmac(E0i, -m0h, -m0l, h0.z, h0.w); dfmac(E0i, -m1h, -m1l, h1.z, h1.w); dfmac(E0i, -m2h, -m2l, h2.z, h2.w);
                            dfmac(E1r, m1h, m1l, h2.x, h2.y); dfmac(E1r, -m2h, -m2l, h1.x, h1.y);
                            dfmac(E1i, m1h, m1l, h2.z, h2.w); dfmac(E1i, -m2h, -m2l, h1.z, h1.w);
                            dfmac(E2r, m2h, m2l, h0.x, h0.y); dfmac(E2r, -m0h, -m0l, h2.x, h2.y);
                            dfmac(E2i, m2h, m2l, h0.z, h0.w); dfmac(E2i, -m0h, -m0l, h2.z, h2.w);
                            dfmac(E3r, m0h, m0l, h1.x, h1.y); dfmac(E3r, -m1h, -m1l, h0.x, h0.y);
                            dfmac(E3i, m0h, m0l, h1.z, h1.w); dfmac(E3i, -m1h, -m1l, h0.z, h0.w);
                        }
                    }
                }
                // results stay double-float: (re.hi, re.lo, im.hi, im.lo) per complex value
                float4 *Vf = reinterpret_cast<float4 *>(sw + Z::V), *Qf = reinterpret_cast<float4 *>(sw + Z::Q);
                float4 *dQf = reinterpret_cast<float4 *>(sw + Z::DQQ);
                Vf[jk] = dfc(Vr, Vi);
                Qf[4 * jk] = dfc(Q0r, Q0i); Qf[4 * jk + 1] = dfc(Q1r, Q1i);
                Qf[4 * jk + 2] = dfc(Q2r, Q2i); Qf[4 * jk + 3] = dfc(Q3r, Q3i);
                if (wantDP) {
                    // dQ = (0, nu')(0, sum w1 h) - sum (0, w3 (nu'.d) d)(0, h), components as in FP64
                    const float2 *nf = reinterpret_cast<const float2 *>(sw + Z::FR + 13);
                    const float2 n0 = nf[0], n1 = nf[1], n2 = nf[2];
                    dfa a0r = {-E0r.h, -E0r.l}, a0i = {-E0i.h, -E0i.l};
                    dfmac(a0r, -n0.x, -n0.y, D0r.h, D0r.l); dfmac(a0r, -n1.x, -n1.y, D1r.h, D1r.l); dfmac(a0r, -n2.x, -n2.y, D2r.h, D2r.l);
                    dfmac(a0i, -n0.x, -n0.y, D0i.h, D0i.l); dfmac(a0i, -n1.x, -n1.y, D1i.h, D1i.l); dfmac(a0i, -n2.x, -n2.y, D2i.h, D2i.l);
                    dfa a1r = {-E1r.h, -E1r.l}, a1i = {-E1i.h, -E1i.l};
                    dfmac(a1r, n1.x, n1.y, D2r.h, D2r.l); dfmac(a1r, -n2.x, -n2.y, D1r.h, D1r.l);
                    dfmac(a1i, n1.x, n1.y, D2i.h, D2i.l); dfmac(a1i, -n2.x, -n2.y, D1i.h, D1i.l);
                    dfa a2r = {-E2r.h, -E2r.l}, a2i = {-E2i.h, -E2i.l};
                    dfmac(a2r, n2.x, n2.y, D0r.h, D0r.l); dfmac(a2r, -n0.x, -n0.y, D2r.h, D2r.l);
                    dfmac(a2i, n2.x, n2.y, D0i.h, D0i.l); dfmac(a2i, -n0.x, -n0.y, D2i.h, D2i.l);
                    dfa a3r = {-E3r.h, -E3r.l}, a3i = {-E3i.h, -E3i.l};
                    dfmac(a3r, n0.x, n0.y, D1r.h, D1r.l); dfmac(a3r, -n1.x, -n1.y, D0r.h, D0r.l);
                    dfmac(a3i, n0.x, n0.y, D1i.h, D1i.l); dfmac(a3i, -n1.x, -n1.y, D0i.h, D0i.l);
                    dQf[4 * jk] = dfc(a0r, a0i); dQf[4 * jk + 1] = dfc(a1r, a1i);
                    dQf[4 * jk + 2] = dfc(a2r, a2i); dQf[4 * jk + 3] = dfc(a3r, a3i);
                }
            }
        } else
        for (int f = tid; f < nt * (NJK - 1); f += nth) {
            int pl, jk;
            kitem<NJK>(f, nt, pl, jk);
            double *sw = SW(pl);
            const size_t ps = (size_t)s_item[pl].P;
            const double *wv = sw + Z::WV, *nut = sw + Z::NUT;
            const cd *eg = pd.eg + ps * pd_eg(pd.pmax);
            const cd *eh = pd.eh + ps * pd_eg(pd.pmax);
            const bool hj = jk >= 3;
            double Vr = 0, Vi = 0;
            double Q0r = 0, Q0i = 0, Q1r = 0, Q1i = 0, Q2r = 0, Q2i = 0, Q3r = 0, Q3i = 0;
            double D0r = 0, D0i = 0, D1r = 0, D1i = 0, D2r = 0, D2i = 0;
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
                    if (wantDP) {
                        // Q and E are sums of the same product (0, d)(0, h) = (-d.h, d x h),
                        // weighted by w1 and by w3 (nu'.d): form it once
                        const double w1 = o[6], sn = o[7], d0 = o[9], d1 = o[10], d2 = o[11];
                        const double r0r = -fma(d0, h0.x, fma(d1, h1.x, d2 * h2.x));
                        const double r0i = -fma(d0, h0.y, fma(d1, h1.y, d2 * h2.y));
                        const double r1r = fma(d1, h2.x, -d2 * h1.x), r1i = fma(d1, h2.y, -d2 * h1.y);
                        const double r2r = fma(d2, h0.x, -d0 * h2.x), r2i = fma(d2, h0.y, -d0 * h2.y);
                        const double r3r = fma(d0, h1.x, -d1 * h0.x), r3i = fma(d0, h1.y, -d1 * h0.y);
                        Q0r = fma(w1, r0r, Q0r); Q0i = fma(w1, r0i, Q0i); Q1r = fma(w1, r1r, Q1r); Q1i = fma(w1, r1i, Q1i);
                        Q2r = fma(w1, r2r, Q2r); Q2i = fma(w1, r2i, Q2i); Q3r = fma(w1, r3r, Q3r); Q3i = fma(w1, r3i, Q3i);
                        E0r = fma(sn, r0r, E0r); E0i = fma(sn, r0i, E0i); E1r = fma(sn, r1r, E1r); E1i = fma(sn, r1i, E1i);
                        E2r = fma(sn, r2r, E2r); E2i = fma(sn, r2i, E2i); E3r = fma(sn, r3r, E3r); E3i = fma(sn, r3i, E3i);
                        D0r = fma(w1, h0.x, D0r); D0i = fma(w1, h0.y, D0i);
                        D1r = fma(w1, h1.x, D1r); D1i = fma(w1, h1.y, D1i);
                        D2r = fma(w1, h2.x, D2r); D2i = fma(w1, h2.y, D2i);
                    } else {
                        const double a0 = o[0], a1 = o[1], a2 = o[2];
                        Q0r = fma(-a0, h0.x, fma(-a1, h1.x, fma(-a2, h2.x, Q0r)));
                        Q0i = fma(-a0, h0.y, fma(-a1, h1.y, fma(-a2, h2.y, Q0i)));
                        Q1r = fma(a1, h2.x, fma(-a2, h1.x, Q1r));
                        Q1i = fma(a1, h2.y, fma(-a2, h1.y, Q1i));
                        Q2r = fma(a2, h0.x, fma(-a0, h2.x, Q2r));
                        Q2i = fma(a2, h0.y, fma(-a0, h2.y, Q2i));
                        Q3r = fma(a0, h1.x, fma(-a1, h0.x, Q3r));
                        Q3i = fma(a0, h1.y, fma(-a1, h0.y, Q3i));
                    }
                }
            }
            cd *Vs = reinterpret_cast<cd *>(sw + Z::V), *Qs = reinterpret_cast<cd *>(sw + Z::Q);
            cd *dQs = reinterpret_cast<cd *>(sw + Z::DQQ);
            Vs[jk] = mkc(Vr, Vi);
            Qs[4 * jk] = mkc(Q0r, Q0i); Qs[4 * jk + 1] = mkc(Q1r, Q1i);
            Qs[4 * jk + 2] = mkc(Q2r, Q2i); Qs[4 * jk + 3] = mkc(Q3r, Q3i);
            if (wantDP) {
                const double n0 = nut[0], n1 = nut[1], n2 = nut[2];
                dQs[4 * jk] = mkc(-(n0 * D0r + n1 * D1r + n2 * D2r) - E0r, -(n0 * D0i + n1 * D1i + n2 * D2i) - E0i);
                dQs[4 * jk + 1] = mkc((n1 * D2r - n2 * D1r) - E1r, (n1 * D2i - n2 * D1i) - E1i);
                dQs[4 * jk + 2] = mkc((n2 * D0r - n0 * D2r) - E2r, (n2 * D0i - n0 * D2i) - E2i);
                dQs[4 * jk + 3] = mkc((n0 * D1r - n1 * D0r) - E3r, (n0 * D1i - n1 * D0i) - E3i);
            }
        }
        __syncthreads();
        // L0: nu' derivative of the target harmonics, dS^{(n,q)} = grad S^{(n,q)}(y') . nu', per
        // (pair, (n, q >= 0)), into the per-sample vectors' space (dead after phase K)
        // (mixed: the target harmonics as double-float pairs too, beside it)
        if ((wantDP || MIX) && !ROT) {
            for (int f = tid; f < nt * NJK; f += nth) {
                const int pl = f / NJK, jk = f % NJK;
                double *sw = SW(pl);
                const double *nut = sw + Z::NUT;
                const cd *gg = reinterpret_cast<const cd *>(sw + Z::GST) + 3 * jk;
                const cd dS = mkc(fma(gg[0].x, nut[0], fma(gg[1].x, nut[1], gg[2].x * nut[2])),
                                  fma(gg[0].y, nut[0], fma(gg[1].y, nut[1], gg[2].y * nut[2])));
                if (MIX) {
                    reinterpret_cast<float4 *>(sw + Z::DST)[jk] = split4c(dS);
                    reinterpret_cast<float4 *>(sw + Z::STF)[jk] = split4c(reinterpret_cast<const cd *>(sw + Z::ST)[jk]);
                } else {
                    reinterpret_cast<cd *>(sw + Z::DST)[jk] = dS;
                }
            }
            __syncthreads();
        }
        // I[gamma] (eq. gammalmdef) and the row vectors B, (0, nu') B, Psi, dB/dnu' of one (pair, (l, m))
        // from its nine translated sums (imaginary parts)
        auto finish_lm = [&](double *sw, int l, int m, int lm, double Ib0, double Ib1, double Ib2, double Ib3,
                             double Ip, double dI0, double dI1, double dI2, double dI3) {
            const double *nut = sw + Z::NUT, *Om = sw + Z::OM;
            const cd *St = reinterpret_cast<const cd *>(sw + Z::ST), *gSt = reinterpret_cast<const cd *>(sw + Z::GST);
            const cd *g = gSt + 3 * jk_index(l, m);
            const double W0 = Om[0], W1 = Om[1], W2 = Om[2], W3 = Om[3];
            const cd G0 = cscale(cadd(cadd(cscale(g[0], W1), cscale(g[1], W2)), cscale(g[2], W3)), -1.0);
            const cd G1 = cadd(cscale(g[0], W0), csub(cscale(g[2], W2), cscale(g[1], W3)));
            const cd G2 = cadd(cscale(g[1], W0), csub(cscale(g[0], W3), cscale(g[2], W1)));
            const cd G3 = cadd(cscale(g[2], W0), csub(cscale(g[1], W1), cscale(g[0], W2)));
            const double fct = sq2 * inv4pi;
            double *Bs = sw + Z::B, *Bds = sw + Z::BD;
            const double B0 = fct * (Ib0 + G0.y), B1 = fct * (Ib1 + G1.y), B2 = fct * (Ib2 + G2.y), B3 = fct * (Ib3 + G3.y);
            // (0, nu') B, whose product with the S' fit gives the S' row (eq. sprime1formrep)
            const double n0 = nut[0], n1 = nut[1], n2 = nut[2];
            const double Bp0 = n0 * B1 + n1 * B2 + n2 * B3, Bp1 = B0 * n0 + (n1 * B3 - n2 * B2);
            const double Bp2 = B0 * n1 + (n2 * B1 - n0 * B3), Bp3 = B0 * n2 + (n0 * B2 - n1 * B1);
            const double psi = fct * (Ip + St[jk_index(l, m)].y * Om[0]);
            if (MIX) {
                // rows in double-float: the row phase reads (hi, lo) pairs in the same slots
                float2 *Bf = reinterpret_cast<float2 *>(Bs) + 4 * lm, *Bpf = reinterpret_cast<float2 *>(sw + Z::BP) + 4 * lm;
                Bf[0] = split2d(B0); Bf[1] = split2d(B1); Bf[2] = split2d(B2); Bf[3] = split2d(B3);
                Bpf[0] = split2d(Bp0); Bpf[1] = split2d(Bp1); Bpf[2] = split2d(Bp2); Bpf[3] = split2d(Bp3);
                reinterpret_cast<float2 *>(sw + Z::PSI)[lm] = split2d(psi);
            } else {
                Bs[4 * lm] = B0; Bs[4 * lm + 1] = B1; Bs[4 * lm + 2] = B2; Bs[4 * lm + 3] = B3;
                double *Bp = sw + Z::BP + 4 * lm;
                Bp[0] = Bp0; Bp[1] = Bp1; Bp[2] = Bp2; Bp[3] = Bp3;
                sw[Z::PSI + lm] = psi;
            }
            if (wantDP) {
                const double X0 = Om[4], X1 = Om[5], X2 = Om[6], X3 = Om[7];
                const cd E0 = cscale(cadd(cadd(cscale(g[0], X1), cscale(g[1], X2)), cscale(g[2], X3)), -1.0);
                const cd E1 = cadd(cscale(g[0], X0), csub(cscale(g[2], X2), cscale(g[1], X3)));
                const cd E2 = cadd(cscale(g[1], X0), csub(cscale(g[0], X3), cscale(g[2], X1)));
                const cd E3 = cadd(cscale(g[2], X0), csub(cscale(g[1], X1), cscale(g[0], X2)));
                // Hessian of S^{(l,m)} at y' by the ladder rules applied twice: the second
                // derivatives of Rn_l^m are combinations of Rn_{l-2}^{m-2 .. m+2}
                cd H[6];
                {
                    const cd r0 = tget(St, l - 2, m), rm1 = tget(St, l - 2, m - 1), rp1 = tget(St, l - 2, m + 1);
                    const cd rm2 = tget(St, l - 2, m - 2), rp2 = tget(St, l - 2, m + 2);
                    H[0] = r0;
                    H[1] = cscale(csub(rm1, rp1), 0.5);
                    H[2] = cmuli(cscale(cadd(rm1, rp1), 0.5));
                    H[3] = cscale(cadd(csub(rm2, cscale(r0, 2.0)), rp2), 0.25);
                    H[4] = cmuli(cscale(csub(rm2, rp2), 0.25));
                    H[5] = cscale(cadd(cadd(rm2, cscale(r0, 2.0)), rp2), -0.25);
                }
                cd hn[3];
                hn[0] = cadd(cadd(cscale(H[0], nut[0]), cscale(H[1], nut[1])), cscale(H[2], nut[2]));
                hn[1] = cadd(cadd(cscale(H[1], nut[0]), cscale(H[3], nut[1])), cscale(H[4], nut[2]));
                hn[2] = cadd(cadd(cscale(H[2], nut[0]), cscale(H[4], nut[1])), cscale(H[5], nut[2]));
                const cd F0 = cscale(cadd(cadd(cscale(hn[0], W1), cscale(hn[1], W2)), cscale(hn[2], W3)), -1.0);
                const cd F1 = cadd(cscale(hn[0], W0), csub(cscale(hn[2], W2), cscale(hn[1], W3)));
                const cd F2 = cadd(cscale(hn[1], W0), csub(cscale(hn[0], W3), cscale(hn[2], W1)));
                const cd F3 = cadd(cscale(hn[2], W0), csub(cscale(hn[1], W1), cscale(hn[0], W2)));
                const double d0 = fct * (dI0 + E0.y + F0.y), d1 = fct * (dI1 + E1.y + F1.y);
                const double d2 = fct * (dI2 + E2.y + F2.y), d3 = fct * (dI3 + E3.y + F3.y);
                if (MIX) {
                    float2 *Bdf = reinterpret_cast<float2 *>(Bds) + 4 * lm;
                    Bdf[0] = split2d(d0); Bdf[1] = split2d(d1); Bdf[2] = split2d(d2); Bdf[3] = split2d(d3);
                } else {
                    Bds[4 * lm] = d0; Bds[4 * lm + 1] = d1; Bds[4 * lm + 2] = d2; Bds[4 * lm + 3] = d3;
                }
            }
        };
        // L: translations and I[gamma], one thread per (pair, (l, m)); items ordered with
        // the largest l first and the pair index fastest, so that the lanes of a warp
        // run loops of similar length.  The factors C_{j,l}, D_{j,l} multiply each j's sum.
        if constexpr (!ROT)
        for (int f = tid; f < nt * NP; f += nth) {
            const int pl = f % nt, lm = NP - 1 - f / nt;
            double *sw = SW(pl);
            const cd *St = reinterpret_cast<const cd *>(sw + Z::ST), *Qs = reinterpret_cast<const cd *>(sw + Z::Q);
            const cd *dQs = reinterpret_cast<const cd *>(sw + Z::DQQ), *Vs = reinterpret_cast<const cd *>(sw + Z::V);
            const cd *dSt = reinterpret_cast<const cd *>(sw + Z::DST);
            int l = 1;
            while ((l + 1) * l / 2 <= lm) l++;
            const int m = lm - l * (l - 1) / 2 + 1;
            double Ib0 = 0, Ib1 = 0, Ib2 = 0, Ib3 = 0, Ip = 0, dI0 = 0, dI1 = 0, dI2 = 0, dI3 = 0;
            if (MIX) {
                // the same sums in double-float on the FP32 pipes; each j's sums in FP64 after
                const float4 *Stf = reinterpret_cast<const float4 *>(sw + Z::STF);
                const float4 *dStf = reinterpret_cast<const float4 *>(sw + Z::DST);
                const float4 *Qf = reinterpret_cast<const float4 *>(sw + Z::Q);
                const float4 *dQf = reinterpret_cast<const float4 *>(sw + Z::DQQ);
                const float4 *Vf = reinterpret_cast<const float4 *>(sw + Z::V);
                for (int j = 1; j <= l; j++) {
                    const int kmin = max(-j, m - (l - j)), kmax = min(j, m + (l - j));
                    dfa ip = {0, 0}, b0 = {0, 0}, b1 = {0, 0}, b2 = {0, 0}, b3 = {0, 0};
                    dfa e0s = {0, 0}, e1s = {0, 0}, e2s = {0, 0}, e3s = {0, 0};
                    for (int k = kmin; k <= kmax; k++) {
                        const int ak = k < 0 ? -k : k;
                        const int jkx = jk_index(j, ak);
                        const float4 Sv = tget4(Stf, l - j, m - k);
                        dfim(ip, kflip4(Vf[jkx], k), Sv);
                        if (j >= 2) {
                            const float4 q0 = kflip4(Qf[4 * jkx], k), q1 = kflip4(Qf[4 * jkx + 1], k);
                            const float4 q2 = kflip4(Qf[4 * jkx + 2], k), q3 = kflip4(Qf[4 * jkx + 3], k);
                            dfim(b0, q0, Sv); dfim(b1, q1, Sv); dfim(b2, q2, Sv); dfim(b3, q3, Sv);
                            if (wantDP) {
                                const float4 dS = tget4(dStf, l - j, m - k);
                                dfim(e0s, kflip4(dQf[4 * jkx], k), Sv); dfim(e0s, q0, dS);
                                dfim(e1s, kflip4(dQf[4 * jkx + 1], k), Sv); dfim(e1s, q1, dS);
                                dfim(e2s, kflip4(dQf[4 * jkx + 2], k), Sv); dfim(e2s, q2, dS);
                                dfim(e3s, kflip4(dQf[4 * jkx + 3], k), Sv); dfim(e3s, q3, dS);
                            }
                        }
                    }
                    Ip = fma(tab->Djl[l * (RRQ_PMAX + 1) + j], dfval(ip), Ip);
                    if (j >= 2) {
                        const double Cj = tab->Cjl[l * (RRQ_PMAX + 1) + j];
                        Ib0 = fma(Cj, dfval(b0), Ib0); Ib1 = fma(Cj, dfval(b1), Ib1);
                        Ib2 = fma(Cj, dfval(b2), Ib2); Ib3 = fma(Cj, dfval(b3), Ib3);
                        if (wantDP) {
                            dI0 = fma(Cj, dfval(e0s), dI0); dI1 = fma(Cj, dfval(e1s), dI1);
                            dI2 = fma(Cj, dfval(e2s), dI2); dI3 = fma(Cj, dfval(e3s), dI3);
                        }
                    }
                }
            } else
            for (int j = 1; j <= l; j++) {
                const double Dj = tab->Djl[l * (RRQ_PMAX + 1) + j];
                const int kmin = max(-j, m - (l - j)), kmax = min(j, m + (l - j));
                double ip = 0, b0 = 0, b1 = 0, b2 = 0, b3 = 0, e0s = 0, e1s = 0, e2s = 0, e3s = 0;
                for (int k = kmin; k <= kmax; k++) {
                    const int ak = k < 0 ? -k : k;
                    const int jkx = jk_index(j, ak);
                    const cd Sv = tget(St, l - j, m - k);
                    const cd v = kflip(Vs[jkx], k);
                    ip = fma(v.x, Sv.y, fma(v.y, Sv.x, ip));
                    if (j >= 2) {
                        const cd q0 = kflip(Qs[4 * jkx], k), q1 = kflip(Qs[4 * jkx + 1], k);
                        const cd q2 = kflip(Qs[4 * jkx + 2], k), q3 = kflip(Qs[4 * jkx + 3], k);
                        b0 = fma(q0.x, Sv.y, fma(q0.y, Sv.x, b0));
                        b1 = fma(q1.x, Sv.y, fma(q1.y, Sv.x, b1));
                        b2 = fma(q2.x, Sv.y, fma(q2.y, Sv.x, b2));
                        b3 = fma(q3.x, Sv.y, fma(q3.y, Sv.x, b3));
                        if (wantDP) {
                            const cd dS = tget(dSt, l - j, m - k);
                            const cd e0 = kflip(dQs[4 * jkx], k), e1 = kflip(dQs[4 * jkx + 1], k);
                            const cd e2 = kflip(dQs[4 * jkx + 2], k), e3 = kflip(dQs[4 * jkx + 3], k);
                            e0s = fma(e0.x, Sv.y, fma(e0.y, Sv.x, fma(q0.x, dS.y, fma(q0.y, dS.x, e0s))));
                            e1s = fma(e1.x, Sv.y, fma(e1.y, Sv.x, fma(q1.x, dS.y, fma(q1.y, dS.x, e1s))));
                            e2s = fma(e2.x, Sv.y, fma(e2.y, Sv.x, fma(q2.x, dS.y, fma(q2.y, dS.x, e2s))));
                            e3s = fma(e3.x, Sv.y, fma(e3.y, Sv.x, fma(q3.x, dS.y, fma(q3.y, dS.x, e3s))));
                        }
                    }
                }
                Ip = fma(Dj, ip, Ip);
                if (j >= 2) {
                    const double Cj = tab->Cjl[l * (RRQ_PMAX + 1) + j];
                    Ib0 = fma(Cj, b0, Ib0); Ib1 = fma(Cj, b1, Ib1); Ib2 = fma(Cj, b2, Ib2); Ib3 = fma(Cj, b3, Ib3);
                    if (wantDP) {
                        dI0 = fma(Cj, e0s, dI0); dI1 = fma(Cj, e1s, dI1); dI2 = fma(Cj, e2s, dI2); dI3 = fma(Cj, e3s, dI3);
                    }
                }
            }
            finish_lm(sw, l, m, lm, Ib0, Ib1, Ib2, Ib3, Ip, dI0, dI1, dI2, dI3);
        }
        if constexpr (ROT) {
            // Rotation-based translation (Sec. 2.3, the remark on fast translation), O(p^3) per
            // pair: rotate the nine coefficient sets (set 0..3: the components of Q, 4..7: those
            // of dQ/dnu', 8: V) so that y' lies on the polar axis of the harmonics, translate
            // along that axis, where Rn_n^q(rho e_z) = rho^n / n! for q = 0 and 0 otherwise so
            // that only the k = m terms remain, and rotate the results back.  With (theta, phi)
            // the polar angles of y' in the harmonics' frame (X, Y, Z) = (y, z, x),
            //   U = Ry(-theta) Rz(-phi) = Rz(90) Ry(90) Rz(-theta) Ry(-90) Rz(-phi - 90),
            //   U^-1 = Rz(phi + 90) Ry(90) Rz(theta) Ry(-90) Rz(-90):
            // z rotations are the phases e^{ik alpha}, the two fixed Y rotations the exact
            // tables Delta+- (tab->Drot).  Every set keeps c_{-k} = (-1)^k conj(c_k), so only
            // k >= 0 is held; the nu' derivative of the translation kernel, on the axis,
            // couples k' = m', m' -+ 1 only (ladder rules of Rn).  Stages R0 .. R6.
            auto cset = [&](double *sw, int s, int jk) -> double * {
                return s < 4 ? sw + Z::Q + 2 * (4 * jk + s)
                             : (s < 8 ? sw + Z::DQQ + 2 * (4 * jk + s - 4) : sw + Z::V + 2 * jk);
            };
            // folded product with a rotation table: (Delta v)_m for v at stride vs (doubles)
            auto fold = [&](const double *D, int j, int m, const double *v, int vs) -> cd {
                const double *A = D + m * (j + 1);
                double re = 0.0, im = 0.0;
                for (int k = 0; k <= j; k++) re = fma(A[k], v[k * vs], re);
                if (m >= 1) {
                    const double *B = D + (j + 1) * (j + 1) + (m - 1) * j;
                    for (int k = 1; k <= j; k++) im = fma(B[k - 1], v[k * vs + 1], im);
                }
                return mkc(re, im);
            };
            auto dec = [](int jk, int &j, int &m) {
                j = 0;
                while ((j + 1) * (j + 2) / 2 <= jk) j++;
                m = jk - j * (j + 1) / 2;
            };
            const double *Drot = tab->Drot;
            const int nset = nt * 9 * NJK;
            // R0: angles, the phases e^{ik theta}, e^{ik (phi + 90)}, rho^n / n!, U nu'
            if (tid < nt) {
                double *sw = SW(tid);
                const double *yt = sw + Z::YT, *nut = sw + Z::NUT;
                const double ax = yt[1], ay = yt[2], az = yt[0];
                const double rxy = sqrt(ax * ax + ay * ay), rho = sqrt(rxy * rxy + az * az);
                const double cph = rxy > 0.0 ? ax / rxy : 1.0, sph = rxy > 0.0 ? ay / rxy : 0.0;
                const double cth = rho > 0.0 ? az / rho : 1.0, sth = rho > 0.0 ? rxy / rho : 0.0;
                cd *eth = reinterpret_cast<cd *>(sw + Z::RPH), *eph = eth + (P + 1);
                cd wt = mkc(1.0, 0.0), wp = mkc(1.0, 0.0);
                const cd st = mkc(cth, sth), sp = mkc(-sph, cph);
                for (int k = 0; k <= P; k++) {
                    eth[k] = wt;
                    eph[k] = wp;
                    wt = cmul(wt, st);
                    wp = cmul(wp, sp);
                }
                double *rp = sw + Z::RRP;
                rp[0] = 1.0;
                for (int n = 1; n <= P; n++) rp[n] = rp[n - 1] * rho * rcp_small(n);
                const double nx = nut[1], ny = nut[2], nz = nut[0];
                const double x1 = cph * nx + sph * ny, y1 = cph * ny - sph * nx;
                sw[Z::RNU] = cth * x1 - sth * nz;
                sw[Z::RNU + 1] = y1;
                sw[Z::RNU + 2] = sth * x1 + cth * nz;
            }
            __syncthreads();
            // R1: c <- Rz(-phi - 90) c, in place
            for (int f = tid; f < nset; f += nth) {
                const int pl = f % nt, r = f / nt, s = r % 9, jk = r / 9;
                int j, k;
                dec(jk, j, k);
                if ((s >= 4 && s < 8 && !wantDP) || j < (s == 8 ? 1 : 2)) continue;
                double *sw = SW(pl);
                double *c = cset(sw, s, jk);
                const cd e = reinterpret_cast<const cd *>(sw + Z::RPH)[P + 1 + k];
                const double re = c[0], im = c[1];
                c[0] = fma(re, e.x, im * e.y);
                c[1] = fma(im, e.x, -re * e.y);
            }
            __syncthreads();
            // R2: y = Rz(-theta) Ry(-90) c, into the second buffer (set-major)
            for (int f = tid; f < nset; f += nth) {
                const int pl = f % nt, r = f / nt, s = r % 9, jk = NJK - 1 - r / 9;
                int j, m;
                dec(jk, j, m);
                if ((s >= 4 && s < 8 && !wantDP) || j < (s == 8 ? 1 : 2)) continue;
                double *sw = SW(pl);
                const cd y = fold(Drot + rot_off(j), j, m, cset(sw, s, jk - m), s == 8 ? 2 : 8);
                const cd e = reinterpret_cast<const cd *>(sw + Z::RPH)[m];
                reinterpret_cast<cd *>(sw + Z::RY)[s * NJK + jk] = cmul(y, cconj(e));
            }
            __syncthreads();
            // R3: c' = Rz(90) Ry(90) y, back into the sets
            for (int f = tid; f < nset; f += nth) {
                const int pl = f % nt, r = f / nt, s = r % 9, jk = NJK - 1 - r / 9;
                int j, m;
                dec(jk, j, m);
                if ((s >= 4 && s < 8 && !wantDP) || j < (s == 8 ? 1 : 2)) continue;
                double *sw = SW(pl);
                const int n1 = (j + 1) * (j + 1) + j * j;
                const cd y = fold(Drot + rot_off(j) + n1, j, m, sw + Z::RY + 2 * (s * NJK + jk - m), 2);
                double *c = cset(sw, s, jk);
                const int q = m & 3;   // times i^m
                c[0] = q == 0 ? y.x : (q == 1 ? -y.y : (q == 2 ? -y.x : y.y));
                c[1] = q == 0 ? y.y : (q == 1 ? y.x : (q == 2 ? -y.y : -y.x));
            }
            __syncthreads();
            // R4: translation along the axis, O'_{l m'} = sum_j W_{j,l} rho^{l-j}/(l-j)! c'_{j m'}
            // (W = C for Q and dQ, D for V), plus for dQ the nu' derivative term acting on Q;
            // then times (-i)^{m'} (the Rz(-90) that starts the inverse rotation)
            for (int f = tid; f < nset; f += nth) {
                const int pl = f % nt, r = f / nt, t = r % 9, jk = NJK - 1 - r / 9;
                int l, mq;
                dec(jk, l, mq);
                if ((t >= 4 && t < 8 && !wantDP) || l < 1) continue;
                double *sw = SW(pl);
                const double *rp = sw + Z::RRP;
                const double *Wl = (t == 8 ? tab->Djl : tab->Cjl) + l * (RRQ_PMAX + 1);
                double ax = 0.0, ay = 0.0;
                for (int j = max(t == 8 ? 1 : 2, mq); j <= l; j++) {
                    const double w = Wl[j] * rp[l - j];
                    const double *c = cset(sw, t, jk_index(j, mq));
                    ax = fma(w, c[0], ax);
                    ay = fma(w, c[1], ay);
                }
                if (t >= 4 && t < 8) {
                    // grad Rn_n^q(rho e_z) . nu~ = rho^{n-1}/(n-1)! times nu~_z (q = 0),
                    // (nu~_x + i nu~_y)/2 (q = 1), (-nu~_x + i nu~_y)/2 (q = -1); q = m' - k'
                    const double nx = sw[Z::RNU], ny = sw[Z::RNU + 1], nz = sw[Z::RNU + 2];
                    for (int j = 2; j < l; j++) {
                        const double w = Wl[j] * rp[l - j - 1];
                        if (mq <= j) {
                            const double *c = cset(sw, t - 4, jk_index(j, mq));
                            ax = fma(w * nz, c[0], ax);
                            ay = fma(w * nz, c[1], ay);
                        }
                        if (mq - 1 <= j) {
                            cd cv;
                            if (mq >= 1) {
                                const double *c = cset(sw, t - 4, jk_index(j, mq - 1));
                                cv = mkc(c[0], c[1]);
                            } else {   // c'_{j,-1} = -conj(c'_{j,1})
                                const double *c = cset(sw, t - 4, jk_index(j, 1));
                                cv = mkc(-c[0], c[1]);
                            }
                            const double gx = 0.5 * w * nx, gy = 0.5 * w * ny;
                            ax = fma(gx, cv.x, fma(-gy, cv.y, ax));
                            ay = fma(gx, cv.y, fma(gy, cv.x, ay));
                        }
                        if (mq + 1 <= j) {
                            const double *c = cset(sw, t - 4, jk_index(j, mq + 1));
                            const double gx = -0.5 * w * nx, gy = 0.5 * w * ny;
                            ax = fma(gx, c[0], fma(-gy, c[1], ax));
                            ay = fma(gx, c[1], fma(gy, c[0], ay));
                        }
                    }
                }
                const int q = mq & 3;   // times (-i)^{m'}
                cd o;
                o.x = q == 0 ? ax : (q == 1 ? ay : (q == 2 ? -ax : -ay));
                o.y = q == 0 ? ay : (q == 1 ? -ax : (q == 2 ? -ay : ax));
                reinterpret_cast<cd *>(sw + Z::RY)[t * NJK + jk] = o;
            }
            __syncthreads();
            // R5: Rz(theta) Ry(-90), from the second buffer into the sets
            for (int f = tid; f < nset; f += nth) {
                const int pl = f % nt, r = f / nt, t = r % 9, jk = NJK - 1 - r / 9;
                int l, m;
                dec(jk, l, m);
                if ((t >= 4 && t < 8 && !wantDP) || l < 1) continue;
                double *sw = SW(pl);
                const cd y = fold(Drot + rot_off(l), l, m, sw + Z::RY + 2 * (t * NJK + jk - m), 2);
                const cd e = reinterpret_cast<const cd *>(sw + Z::RPH)[m];
                const cd o = cmul(y, e);
                double *c = cset(sw, t, jk);
                c[0] = o.x;
                c[1] = o.y;
            }
            __syncthreads();
            // R6: per (pair, (l, m)), m >= 1: the nine sums, Im of Rz(phi + 90) Ry(90) applied to
            // each set, then I[gamma] and the row vectors
            for (int f = tid; f < nt * NP; f += nth) {
                const int pl = f % nt, lm = NP - 1 - f / nt;
                double *sw = SW(pl);
                int l = 1;
                while ((l + 1) * l / 2 <= lm) l++;
                const int m = lm - l * (l - 1) / 2 + 1;
                const double *D = Drot + rot_off(l) + (l + 1) * (l + 1) + l * l;
                const cd e = reinterpret_cast<const cd *>(sw + Z::RPH)[P + 1 + m];
                double o[9];
#pragma unroll
                for (int t = 0; t < 9; t++) {
                    o[t] = 0.0;
                    if (t >= 4 && t < 8 && !wantDP) continue;
                    const cd u = fold(D, l, m, cset(sw, t, jk_index(l, 0)), t == 8 ? 2 : 8);
                    o[t] = fma(e.y, u.x, e.x * u.y);
                }
                finish_lm(sw, l, m, lm, o[0], o[1], o[2], o[3], o[8], o[4], o[5], o[6], o[7]);
            }
        }
        __syncthreads();
        // M (density-given evaluation, Step 8 for a given density): per pair the fit coefficients
        // of the density against B, Bd, (0, nu')B, Psi, then the jump and the smooth rule over the
        // patch's nodes; one warp per pair, one result per (pair, kernel)
        if (EVAL) {
            for (int pl = warp; pl < nt; pl += nwarp) {
                const double *sw = SW(pl);
                const PairItem im = s_item[pl];
                const double *c = a.coef + (size_t)im.P * (13 * RRQ_NPMAX);
                const double *cD = c, *cSp = c + 4 * RRQ_NPMAX, *cS2 = c + 8 * RRQ_NPMAX, *cS1 = c + 12 * RRQ_NPMAX;
                const double *Bs = sw + Z::B, *Bds = sw + Z::BD, *Bp = sw + Z::BP, *Psis = sw + Z::PSI;
                double qD = 0, qDp = 0, qSp = 0, qS = 0;
                for (int lm = lane; lm < NP; lm += 32) {
                    const double B0 = Bs[4 * lm], B1 = Bs[4 * lm + 1], B2 = Bs[4 * lm + 2], B3 = Bs[4 * lm + 3];
                    qD -= B0 * cD[lm] - B1 * cD[NP + lm] - B2 * cD[2 * NP + lm] - B3 * cD[3 * NP + lm];
                    if (wantDP)
                        qDp -= Bds[4 * lm] * cD[lm] - Bds[4 * lm + 1] * cD[NP + lm] - Bds[4 * lm + 2] * cD[2 * NP + lm] -
                               Bds[4 * lm + 3] * cD[3 * NP + lm];
                    qSp += Bp[4 * lm] * cSp[lm] + Bp[4 * lm + 1] * cSp[NP + lm] + Bp[4 * lm + 2] * cSp[2 * NP + lm] +
                           Bp[4 * lm + 3] * cSp[3 * NP + lm];
                    qS += Psis[lm] * cS1[lm] -
                          (B0 * cS2[lm] - B1 * cS2[NP + lm] - B2 * cS2[2 * NP + lm] - B3 * cS2[3 * NP + lm]);
                }
                const double sc = sw[Z::FR + 12];
                const int64_t o = node_off[im.P];
                double mD = 0, mDp = 0, mSp = 0, mS = 0;
                for (int i = lane; i < NP; i += 32) {
                    const double sg = a.sigma[o + i];
                    if (i == s_self[pl]) {
                        mD -= 0.5 * sg;
                        mSp += 0.5 * sg;
                    } else {
                        const double *xs = xyz + 3 * (o + i), *ns = nrm + 3 * (o + i);
                        const double d0 = sw[Z::XT] - xs[0], d1 = sw[Z::XT + 1] - xs[1], d2 = sw[Z::XT + 2] - xs[2];
                        const double gn0 = sw[Z::NT], gn1 = sw[Z::NT + 1], gn2 = sw[Z::NT + 2];
                        const double ri = rsqrt(d0 * d0 + d1 * d1 + d2 * d2), ri2 = ri * ri, ri3 = ri2 * ri;
                        const double wk = wts[o + i] * inv4pi * sg;
                        const double dns = d0 * ns[0] + d1 * ns[1] + d2 * ns[2];
                        const double dnt = d0 * gn0 + d1 * gn1 + d2 * gn2;
                        mS -= wk * ri;
                        mD -= wk * dns * ri3;
                        mSp += wk * dnt * ri3;
                        mDp -= wk * ri3 * ((gn0 * ns[0] + gn1 * ns[1] + gn2 * ns[2]) - 3.0 * dns * dnt * ri2);
                    }
                }
                qD = warp_sum(qD); qDp = warp_sum(qDp); qSp = warp_sum(qSp); qS = warp_sum(qS);
                mD = warp_sum(mD); mDp = warp_sum(mDp); mSp = warp_sum(mSp); mS = warp_sum(mS);
                if (lane == 0) {
                    const int64_t q = im.pad;
                    if (a.res[0]) a.res[0][q] = qS * (1.0 / sc) + mS;
                    if (a.res[1]) a.res[1][q] = qD + mD;
                    if (a.res[2]) a.res[2][q] = qSp + mSp;
                    if (a.res[3]) a.res[3][q] = qDp * sc + mDp;
                }
            }
        } else
        {
        // M: rows through the fit matrices (Step 8), jump and smooth subtraction, one thread per
        // (kernel group, pair, node) for the groups {D, D'} (X_D), {S'} (X_S'), {S} (X_S2, X_S1)
        // fit-matrix terms of the lm-th harmonic at one node, FP64 (fused into the sums)
        auto term_d = [&](double &r0, double &r1, const double *B, const double *Bd, double x0, double x1, double x2,
                          double x3) {
            r0 = fma(B[3], x3, fma(B[2], x2, fma(B[1], x1, fma(-B[0], x0, r0))));
            if (wantDP) r1 = fma(Bd[3], x3, fma(Bd[2], x2, fma(Bd[1], x1, fma(-Bd[0], x0, r1))));
        };
        auto term_sp = [&](double &r0, const double *Bp, double x0, double x1, double x2, double x3) {
            r0 = fma(Bp[3], x3, fma(Bp[2], x2, fma(Bp[1], x1, fma(Bp[0], x0, r0))));
        };
        auto term_s = [&](double &r0, const double *B, double psi, double xs1, double g0, double g1, double g2,
                          double g3) {
            r0 = fma(B[3], g3, fma(B[2], g2, fma(B[1], g1, fma(-B[0], g0, fma(psi, xs1, r0)))));
        };
        // the same in double-float with the (hi, lo) fit matrices
        auto mterm_d = [&](dfa &a0, dfa &a1, const float2 *Bf, const float2 *Bdf, float2 x0, float2 x1, float2 x2,
                           float2 x3) {
            dfmac(a0, -Bf[0].x, -Bf[0].y, x0.x, x0.y); dfmac(a0, Bf[1].x, Bf[1].y, x1.x, x1.y);
            dfmac(a0, Bf[2].x, Bf[2].y, x2.x, x2.y); dfmac(a0, Bf[3].x, Bf[3].y, x3.x, x3.y);
            if (wantDP) {
                dfmac(a1, -Bdf[0].x, -Bdf[0].y, x0.x, x0.y); dfmac(a1, Bdf[1].x, Bdf[1].y, x1.x, x1.y);
                dfmac(a1, Bdf[2].x, Bdf[2].y, x2.x, x2.y); dfmac(a1, Bdf[3].x, Bdf[3].y, x3.x, x3.y);
            }
        };
        auto mterm_sp = [&](dfa &a0, const float2 *Bpf, float2 x0, float2 x1, float2 x2, float2 x3) {
            dfmac(a0, Bpf[0].x, Bpf[0].y, x0.x, x0.y); dfmac(a0, Bpf[1].x, Bpf[1].y, x1.x, x1.y);
            dfmac(a0, Bpf[2].x, Bpf[2].y, x2.x, x2.y); dfmac(a0, Bpf[3].x, Bpf[3].y, x3.x, x3.y);
        };
        auto mterm_s = [&](dfa &a0, const float2 *Bf, float2 psi, float2 xs1, float2 g0, float2 g1, float2 g2,
                           float2 g3) {
            dfmac(a0, psi.x, psi.y, xs1.x, xs1.y);
            dfmac(a0, -Bf[0].x, -Bf[0].y, g0.x, g0.y); dfmac(a0, Bf[1].x, Bf[1].y, g1.x, g1.y);
            dfmac(a0, Bf[2].x, Bf[2].y, g2.x, g2.y); dfmac(a0, Bf[3].x, Bf[3].y, g3.x, g3.y);
        };
        // jump on self pairs, else minus the smooth rule; then the CSR entries of (pair, node)
        auto finish_row = [&](int pl, int grp, int i, double r0, double r1) {
            const double *sw = SW(pl);
            const PairItem im = s_item[pl];
            const int64_t o = node_off[im.P];
            const int64_t dst = im.off + i;
            if (i == s_self[pl]) {
                if (grp == 0) r0 -= 0.5;
                if (grp == 1) r0 += 0.5;
            } else {
                const double *xs = xyz + 3 * (o + i), *ns = nrm + 3 * (o + i);
                const double d0 = sw[Z::XT] - xs[0], d1 = sw[Z::XT + 1] - xs[1], d2 = sw[Z::XT + 2] - xs[2];
                const double gn0 = sw[Z::NT], gn1 = sw[Z::NT + 1], gn2 = sw[Z::NT + 2];
                const double ri = rsqrt(d0 * d0 + d1 * d1 + d2 * d2), ri2 = ri * ri, ri3 = ri2 * ri;
                const double wk = wts[o + i] * inv4pi;
                const double dns = d0 * ns[0] + d1 * ns[1] + d2 * ns[2];
                const double dnt = d0 * gn0 + d1 * gn1 + d2 * gn2;
                if (grp == 0) {
                    r0 -= wk * dns * ri3;
                    r1 -= wk * ri3 * ((gn0 * ns[0] + gn1 * ns[1] + gn2 * ns[2]) - 3.0 * dns * dnt * ri2);
                } else if (grp == 1) {
                    r0 += wk * dnt * ri3;
                } else {
                    r0 -= wk * ri;
                }
            }
            if (grp == s_grp[0]) col[dst] = (int32_t)(col_off[im.P] + i);
            if (grp == 0) {
                if ((mask & RRQ_D) && vD) vD[dst] = r0;
                if ((mask & RRQ_DP) && vDp) vDp[dst] = r1;
            } else if (grp == 1) {
                if (vSp) vSp[dst] = r0;
            } else if (vS) {
                vS[dst] = r0;
            }
        };
        for (int f = tid; f < nt * NP * ngrp; f += nth) {
            const int grp = s_grp[f / (nt * NP)], rem = f % (nt * NP), pl = rem / NP, i = rem % NP;
            const double *sw = SW(pl);
            const size_t ps = (size_t)s_item[pl].P;
            const double sc = sw[Z::FR + 12];
            double r0 = 0, r1 = 0;
            if (MIX) {
                dfa a0 = {0, 0}, a1 = {0, 0};
                if (grp == 0) {
                    const float2 *X = pd.XD2 + ps * pd_X(pd.pmax);
                    for (int lm = 0; lm < NP; lm++)
                        mterm_d(a0, a1, reinterpret_cast<const float2 *>(sw + Z::B) + 4 * lm,
                                reinterpret_cast<const float2 *>(sw + Z::BD) + 4 * lm, X[(0 * NP + lm) * NP + i],
                                X[(1 * NP + lm) * NP + i], X[(2 * NP + lm) * NP + i], X[(3 * NP + lm) * NP + i]);
                } else if (grp == 1) {
                    const float2 *X = pd.XSp2 + ps * pd_X(pd.pmax);
                    for (int lm = 0; lm < NP; lm++)
                        mterm_sp(a0, reinterpret_cast<const float2 *>(sw + Z::BP) + 4 * lm, X[(0 * NP + lm) * NP + i],
                                 X[(1 * NP + lm) * NP + i], X[(2 * NP + lm) * NP + i], X[(3 * NP + lm) * NP + i]);
                } else {
                    const float2 *X = pd.XS22 + ps * pd_X(pd.pmax), *X1 = pd.XS12 + ps * pd_XS1(pd.pmax);
                    for (int lm = 0; lm < NP; lm++)
                        mterm_s(a0, reinterpret_cast<const float2 *>(sw + Z::B) + 4 * lm,
                                reinterpret_cast<const float2 *>(sw + Z::PSI)[lm], X1[lm * NP + i],
                                X[(0 * NP + lm) * NP + i], X[(1 * NP + lm) * NP + i], X[(2 * NP + lm) * NP + i],
                                X[(3 * NP + lm) * NP + i]);
                }
                r0 = dfval(a0);
                r1 = dfval(a1);
            } else if (grp == 0) {
                const double *X = pd.XD + ps * pd_X(pd.pmax);
                for (int lm = 0; lm < NP; lm++)
                    term_d(r0, r1, sw + Z::B + 4 * lm, sw + Z::BD + 4 * lm, X[(0 * NP + lm) * NP + i],
                           X[(1 * NP + lm) * NP + i], X[(2 * NP + lm) * NP + i], X[(3 * NP + lm) * NP + i]);
            } else if (grp == 1) {
                const double *X = pd.XSp + ps * pd_X(pd.pmax);
                for (int lm = 0; lm < NP; lm++)
                    term_sp(r0, sw + Z::BP + 4 * lm, X[(0 * NP + lm) * NP + i], X[(1 * NP + lm) * NP + i],
                            X[(2 * NP + lm) * NP + i], X[(3 * NP + lm) * NP + i]);
            } else {
                const double *X = pd.XS2 + ps * pd_X(pd.pmax), *X1 = pd.XS1 + ps * pd_XS1(pd.pmax);
                for (int lm = 0; lm < NP; lm++)
                    term_s(r0, sw + Z::B + 4 * lm, sw[Z::PSI + lm], X1[lm * NP + i], X[(0 * NP + lm) * NP + i],
                           X[(1 * NP + lm) * NP + i], X[(2 * NP + lm) * NP + i], X[(3 * NP + lm) * NP + i]);
            }
            finish_row(pl, grp, i, grp == 2 ? r0 * (1.0 / sc) : r0, r1 * sc);
        }
        }
    }
#undef SW
    __syncthreads();
    if (tid == 0) {
        if (bc[0]) atomicAdd(&cnt->newton_fail, (unsigned long long)bc[0]);
        if (bc[1]) atomicAdd(&cnt->on_edge, (unsigned long long)bc[1]);
        if (bc[2]) atomicAdd(&cnt->u_poor, (unsigned long long)bc[2]);
        if (bc[3]) atomicAdd(&cnt->ssq_edges, (unsigned long long)bc[3]);
        if (bc[4]) atomicAdd(&cnt->far_edges, (unsigned long long)bc[4]);
    }
}

// Step 5, complex preimage t0 of every (pair, edge): Newton on sum_a (y_a(t) - y'_a)^2
// from the root of the straight chord (|dt| <= 1e-14 max(1,|t|), newton_max steps), Im t0 >= 0;
// an edge for which a bound shows that no root lies in the ellipse E_rho0 takes the
// upsampled rule without Newton and keeps the chord root.  One thread per (pair, edge), so
// the Newton chains of many pairs overlap.
template <int P>
__global__ void __launch_bounds__(128) k_roots(const OrderTables *__restrict__ tab, const PairItem *__restrict__ items,
                                               int64_t nitems, PatchData pd, const double *__restrict__ txyz,
                                               int newton_max) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nitems * 3) return;
    const int64_t n = idx / 3;
    const int e = (int)(idx % 3);
    const PairItem im = items[n];
    const double *fr = pd.frame + (size_t)im.P * PD_FRAME;
    double yt[3];
    for (int b = 0; b < 3; b++) {
        double sy = 0;
        for (int a = 0; a < 3; a++) sy += fr[3 + 3 * a + b] * (txyz[3 * im.t + a] - fr[a]);
        yt[b] = fr[12] * sy;
    }
    double ce[3 * P];
    for (int i = 0; i < 3 * P; i++) ce[i] = pd.ea[(size_t)im.P * pd_ea(pd.pmax) + 3 * P * e + i];
    double ym[3], yp[3];
    for (int a = 0; a < 3; a++) {
        double sp = 0, sm = 0;
        for (int k = 0; k < P; k++) {
            sp += ce[3 * k + a];
            sm += ((k & 1) ? -1.0 : 1.0) * ce[3 * k + a];
        }
        yp[a] = sp;
        ym[a] = sm;
    }
    double c[3], b[3], w[3];
    for (int a = 0; a < 3; a++) { c[a] = 0.5 * (yp[a] + ym[a]); b[a] = 0.5 * (yp[a] - ym[a]); w[a] = yt[a] - c[a]; }
    const double bw0 = b[1] * w[2] - b[2] * w[1], bw1 = b[2] * w[0] - b[0] * w[2], bw2 = b[0] * w[1] - b[1] * w[0];
    const double bb = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
    cd tt = mkc((b[0] * w[0] + b[1] * w[1] + b[2] * w[2]) / bb, sqrt(bw0 * bw0 + bw1 * bw1 + bw2 * bw2) / bb);
    int conv = 0;
    bool skip = false;
    {
        // Newton is skipped only where no root can lie in the Bernstein ellipse E_rho0, so that
        // the rule is the one the root would select.  With the chord c + b t of the edge,
        // f(t) = sum_a (y_a(t) - y'_a)^2 = |b|^2 (t - tt)(t - conj tt) + 2 (b t - w).d(t) + d.d,
        // with d(t) = sum_{n >= 2} a_n (P_n(t) - e_n(t)) the deviation from the chord (e_n = 1
        // for even n, t for odd n).  On and inside E_rho0: |P_n| <= rho0^n (Laplace's integral),
        // |e_n| <= |t| <= A0 = (rho0 + 1/rho0)/2, so |d| <= D = sum_{n>=2} |a_n| (rho0^n + A0);
        // and |t - tt| >= the gap between the
        // confocal ellipses through tt and E_rho0, (rc + 1/rc - rho0 - 1/rho0)/2.  No root
        // there if |b|^2 gap^2 > 2 (|b| A0 + |w|) D + D^2.
        const cd zm1 = mkc(tt.x - 1.0, tt.y), zp1 = mkc(tt.x + 1.0, tt.y);
        const cd wv = cadd(tt, cmul(sqrt_c(zm1), sqrt_c(zp1)));
        double rc = sqrt(cabs2(wv));
        if (rc < 1.0) rc = 1.0 / rc;
        const double r0 = tab->rho0, A0 = 0.5 * (r0 + 1.0 / r0);
        if (rc > r0 && tt.y > 0.0) {
            double D = 0.0, rn = r0;
            for (int k = 2; k < P; k++) {
                rn *= r0;
                const double an = sqrt(ce[3 * k] * ce[3 * k] + ce[3 * k + 1] * ce[3 * k + 1] + ce[3 * k + 2] * ce[3 * k + 2]);
                D += an * (rn + A0);
            }
            const double gap = 0.5 * (rc + 1.0 / rc - r0 - 1.0 / r0);
            const double wn = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
            if (bb * gap * gap > 2.0 * (sqrt(bb) * A0 + wn) * D + D * D) { skip = true; conv = 1; }
        }
    }
    for (int it = 0; it < (skip ? 0 : newton_max); it++) {
        cd y[3], dy[3];
        edge_eval_cplx(ce, P, tt, y, dy);
        cd g = mkc(0, 0), gp = mkc(0, 0);
        for (int a = 0; a < 3; a++) {
            const cd r = mkc(y[a].x - yt[a], y[a].y);
            g = cadd(g, cmul(r, r));
            gp = cadd(gp, cscale(cmul(r, dy[a]), 2.0));
        }
        if (gp.x == 0.0 && gp.y == 0.0) break;
        const double rq = 1.0 / (gp.x * gp.x + gp.y * gp.y);
        const cd dt = mkc((g.x * gp.x + g.y * gp.y) * rq, (g.y * gp.x - g.x * gp.y) * rq);
        tt = csub(tt, dt);
        const double at2 = cabs2(tt);
        if (cabs2(dt) <= 1e-28 * (at2 > 1.0 ? at2 : 1.0)) { conv = 1; break; }
    }
    if (tt.y < 0) tt.y = -tt.y;
    const cd zm1 = mkc(tt.x - 1.0, tt.y), zp1 = mkc(tt.x + 1.0, tt.y);
    const cd wv = cadd(tt, cmul(sqrt_c(zm1), sqrt_c(zp1)));
    double rho = sqrt(cabs2(wv));
    if (rho < 1.0) rho = 1.0 / rho;
    const int ssq = conv && rho < tab->rho0 && tt.y > 0.0;
    pd.roots[idx] = EdgeRoot{tt.x, tt.y, (double)conv, (double)ssq};
}

// Side of patch P on which the target lies along the frame axis e_z, one thread per pair
// item: Newton for the footprint (u, v) with X_xy(u, v) = y'_xy on the monomial form of
// the local node interpolant, from the barycentric coordinates of y'_xy in the
// projected vertex triangle (|du| + |dv| <= 1e-14 (1 + |u| + |v|), 30 steps).  +1 when
// the footprint lies in the reference triangle (tolerance 1e-12) and y'_z >= X_z(u, v),
// -1 when below, 0 when outside, not converged, or the target is a node of the patch.
template <int P>
__global__ void __launch_bounds__(128) k_uside(const PairItem *__restrict__ items, int64_t nitems, PatchData pd,
                                               const int64_t *__restrict__ node_off,
                                               const double *__restrict__ txyz, const int64_t *__restrict__ tself) {
    constexpr int NP = P * (P + 1) / 2;
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nitems) return;
    const PairItem im = items[n];
    int8_t side = 0;
    const int64_t o = node_off[im.P];
    const bool self = tself && tself[im.t] >= o && tself[im.t] < o + NP;
    if (!self) {
        const double *fr = pd.frame + (size_t)im.P * PD_FRAME;
        double yt[3];
        for (int b = 0; b < 3; b++) {
            double sy = 0;
            for (int a = 0; a < 3; a++) sy += fr[3 + 3 * a + b] * (txyz[3 * im.t + a] - fr[a]);
            yt[b] = fr[12] * sy;
        }
        const double *xm = pd.xm + (size_t)im.P * pd_ynode(pd.pmax);
        // vertices X(0,0) = xm[00], X(1,0) = sum_a xm[a0], X(0,1) = sum_b xm[0b]
        double v0[2] = {xm[0], xm[1]}, v1[2] = {0, 0}, v2[2] = {0, 0};
        {
            int ab = 0;
            for (int a = 0; a < P; a++)
                for (int b = 0; a + b < P; b++, ab++) {
                    if (b == 0) { v1[0] += xm[3 * ab]; v1[1] += xm[3 * ab + 1]; }
                    if (a == 0) { v2[0] += xm[3 * ab]; v2[1] += xm[3 * ab + 1]; }
                }
        }
        const double a11 = v1[0] - v0[0], a12 = v2[0] - v0[0], a21 = v1[1] - v0[1], a22 = v2[1] - v0[1];
        const double det = a11 * a22 - a12 * a21;
        if (det != 0.0) {
            const double rx = yt[0] - v0[0], ry = yt[1] - v0[1];
            double u = (a22 * rx - a12 * ry) / det, v = (a11 * ry - a21 * rx) / det;
            bool conv = false;
            for (int it = 0; it < 30; it++) {
                // X_xy and its derivatives at (u, v): powers by recurrence
                double X0 = 0, X1 = 0, Xu0 = 0, Xu1 = 0, Xv0 = 0, Xv1 = 0;
                double ua = 1.0, ua1 = 0.0;  // u^a, a u^(a-1)
                int ab = 0;
                for (int a = 0; a < P; a++) {
                    double vb = 1.0, vb1 = 0.0;  // v^b, b v^(b-1)
                    for (int b = 0; a + b < P; b++, ab++) {
                        const double c0 = xm[3 * ab], c1 = xm[3 * ab + 1];
                        const double m = ua * vb, mu = ua1 * vb, mv = ua * vb1;
                        X0 = fma(c0, m, X0); X1 = fma(c1, m, X1);
                        Xu0 = fma(c0, mu, Xu0); Xu1 = fma(c1, mu, Xu1);
                        Xv0 = fma(c0, mv, Xv0); Xv1 = fma(c1, mv, Xv1);
                        vb1 = vb * (b + 1);
                        vb *= v;
                    }
                    ua1 = ua * (a + 1);
                    ua *= u;
                }
                const double dj = Xu0 * Xv1 - Xv0 * Xu1;
                if (dj == 0.0) break;
                const double fx = X0 - yt[0], fy = X1 - yt[1];
                const double du = (Xv1 * fx - Xv0 * fy) / dj, dv = (Xu0 * fy - Xu1 * fx) / dj;
                u -= du;
                v -= dv;
                if (fabs(du) + fabs(dv) <= 1e-14 * (1.0 + fabs(u) + fabs(v))) { conv = true; break; }
            }
            const double tol = 1e-12;
            if (conv && u >= -tol && v >= -tol && u + v <= 1.0 + tol) {
                double Xz = 0.0, ua = 1.0;
                int ab = 0;
                for (int a = 0; a < P; a++) {
                    double vb = 1.0;
                    for (int b = 0; a + b < P; b++, ab++) {
                        Xz = fma(xm[3 * ab + 2], ua * vb, Xz);
                        vb *= v;
                    }
                    ua *= u;
                }
                side = yt[2] >= Xz ? 1 : -1;
            }
        }
    }
    pd.uside[n] = side;
}

template <int P, bool MIX, int T, bool EVAL = false, bool ROT = false>
cudaError_t launch_pairs_tile(const PairArgs &a, const PairShape &shape, cudaStream_t st) {
    constexpr int NTH = TileCfg<P>::THREADS;
    const size_t bytes = sizeof(double) * (ROT ? PairSm<P>::TOTAL_ROT : PairSm<P>::TOTAL) * T;
    cudaError_t e = cudaFuncSetAttribute(k_pairs_tile<P, MIX, T, EVAL, ROT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    if (a.nitems <= 0) return cudaSuccess;
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pairs_tile<P, MIX, T, EVAL, ROT>, NTH, bytes);
    if (per_sm < 1) per_sm = 1;
    k_roots<P><<<(unsigned)((a.nitems * 3 + 127) / 128), 128, 0, st>>>(a.tab, a.items, a.nitems, a.pd, a.txyz,
                                                                       a.newton_max);
    RRQ_COUNT_LAUNCH();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_uside<P><<<(unsigned)((a.nitems + 127) / 128), 128, 0, st>>>(a.items, a.nitems, a.pd, a.node_off, a.txyz,
                                                                   a.tself);
    RRQ_COUNT_LAUNCH();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t want = (a.nitems + T - 1) / T;
    int64_t grid = (int64_t)nsm * per_sm * (shape.persistent ? 1 : 16);
    if (grid > want) grid = want;
    unsigned long long *ctr = shape.persistent ? shape.tile_ctr : nullptr;
    if (shape.persistent) {
        if (!ctr) return cudaErrorInvalidValue;
        e = cudaMemsetAsync(ctr, 0, sizeof(unsigned long long), st);
        if (e != cudaSuccess) return e;
    }
    k_pairs_tile<P, MIX, T, EVAL, ROT><<<(unsigned)grid, NTH, bytes, st>>>(a, ctr);
    RRQ_COUNT_LAUNCH();
    return cudaGetLastError();
}

// Tile of the rotation-based translation: of the compiled tiles, the one that keeps the most
// pairs resident per SM with its larger per-pair scratch (228 KB of shared memory per SM,
// 1 KB reserved per CTA).
template <int P, int... Ts>
constexpr int rot_tile() {
    int best = 0, bt = 0;
    for (int t : {Ts...}) {
        const int per_sm = (228 * 1024) / (t * PairSm<P>::TOTAL_ROT * 8 + 1024);
        if (t * per_sm > best) {
            best = t * per_sm;
            bt = t;
        }
    }
    return bt;
}

// Dispatch on the tile size among the compiled ones (Ts, the first being the default).  The
// rotation-based translation (a.rot) is compiled for FP64 and one tile (rot_tile).
template <int P, int... Ts>
cudaError_t launch_pairs_order(bool mixed, const PairArgs &a, const PairShape &shape, cudaStream_t st) {
    constexpr int tiles[] = {Ts...};
    if (a.rot)
        return mixed ? cudaErrorInvalidValue : launch_pairs_tile<P, false, rot_tile<P, Ts...>(), false, true>(a, shape, st);
    const int T = shape.tile ? shape.tile : tiles[0];
    cudaError_t e = cudaErrorInvalidValue;
    ((T == Ts ? (void)(e = mixed ? launch_pairs_tile<P, true, Ts>(a, shape, st)
                                 : launch_pairs_tile<P, false, Ts>(a, shape, st))
              : (void)0),
     ...);
    return e;
}

// Density-given evaluation (FP64), with the tile sizes of the matrix build.
template <int P, int... Ts>
cudaError_t launch_pairs_eval_order(const PairArgs &a, const PairShape &shape, cudaStream_t st) {
    constexpr int tiles[] = {Ts...};
    const int T = shape.tile ? shape.tile : tiles[0];
    cudaError_t e = cudaErrorInvalidValue;
    ((T == Ts ? (void)(e = launch_pairs_tile<P, false, Ts, true>(a, shape, st)) : (void)0), ...);
    return e;
}

template <int... Ts>
int tiles_of(int out[4]) {
    constexpr int tiles[] = {Ts...};
    int n = 0;
    for (int t : tiles)
        if (n < 4) out[n++] = t;
    return n;
}

}  // namespace rrqk
