// Internal definitions shared by the librrq CUDA translation units.
//
// Harmonic normalisation used on the device.  The paper's regular solid harmonics
// R_l^m (eq. rlmdef) are rescaled to Rn_l^m = R_l^m / sqrt((l-m)!(l+m)!), which turns
// the translation coefficients T_{jk,lm} of eq. (tjklmdef) into 1:
//     Rn_l^m(a + b) = sum_{j,k} Rn_j^k(a) Rn_{l-j}^{m-k}(b),
// and gives ladder rules for derivatives (the j = 1 terms of that expansion):
//     d/dZ Rn_l^m = Rn_{l-1}^m,  d/dX Rn_l^m = (Rn_{l-1}^{m-1} - Rn_{l-1}^{m+1})/2,
//     d/dY Rn_l^m = i (Rn_{l-1}^{m-1} + Rn_{l-1}^{m+1})/2,
// with Rn_l^{-m} = (-1)^m conj(Rn_l^m).  The basis S^{(l,m)}(x,y,z) = Rn_l^m(y,z,x)
// (eq. slmdef) and H^{(l,m)} = sqrt2 Im S^{(l,m)} (eq. hlmslmconnection) then differ
// from the paper's by a constant factor per (l,m), which leaves every correction row
// unchanged: the rows depend only on the span of the basis.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rrq.h"

#define RRQ_PTMAX (2 * RRQ_PMAX)
#define RRQ_NPMAX (RRQ_PMAX * (RRQ_PMAX + 1) / 2)
#define RRQ_NJKMAX ((RRQ_PMAX + 1) * (RRQ_PMAX + 2) / 2)
#define RRQ_NOM 16

struct cd {
    double x, y;
};

__host__ __device__ __forceinline__ cd mkc(double a, double b) { cd r; r.x = a; r.y = b; return r; }
__host__ __device__ __forceinline__ cd cadd(cd a, cd b) { return mkc(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ cd csub(cd a, cd b) { return mkc(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ cd cmul(cd a, cd b) { return mkc(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__host__ __device__ __forceinline__ cd cscale(cd a, double s) { return mkc(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ cd cconj(cd a) { return mkc(a.x, -a.y); }
__host__ __device__ __forceinline__ cd cmuli(cd a) { return mkc(-a.y, a.x); }  // i * a
__host__ __device__ __forceinline__ double cabs2(cd a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ cd cdivz(cd a, cd b) {
    double d = b.x * b.x + b.y * b.y;
    return mkc((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

// index of (n, q), 0 <= q <= n, in a triangular harmonic table
__host__ __device__ __forceinline__ int jk_index(int n, int q) { return n * (n + 1) / 2 + q; }

// Per-order constant tables (computed on the host by rrq_tables.cu).
struct OrderTables {
    int p, np, pt, nup, njk;
    double rho0;
    double tq[RRQ_PTMAX], wq[RRQ_PTMAX];            // edge Gauss-Legendre nodes/weights
    double BPr[RRQ_PTMAX * RRQ_PTMAX];              // [k][i] 1/(tq[i] - tq[i-k-1]), i > k: dual Vandermonde solve
    double tu[2 * RRQ_PTMAX], wu[2 * RRQ_PTMAX];    // upsampled Gauss-Legendre rule
    double Lup[2 * RRQ_PTMAX * RRQ_PTMAX];          // [s][q] Lagrange basis of tq at tu[s]
    double tom[RRQ_NOM], wom[RRQ_NOM];              // Gauss-Legendre rule per Omega_0 panel
    double Eint[(3 * RRQ_PTMAX + 3) * RRQ_NPMAX];   // [row][i]: node -> edge samples, then vertices
    double LegW[RRQ_PMAX * RRQ_PTMAX];              // [n][q] (2n+1)/2 w_q P_n(t_q)
    double dLeg[RRQ_PTMAX * RRQ_PMAX];              // [q][n] P_n'(t_q)
    double LegU[2 * RRQ_PTMAX * RRQ_PMAX];          // [s][n] P_n(tu_s)
    double L2M[RRQ_PMAX * RRQ_PMAX];                // [n][k] coefficient of t^k in P_n(t)
    double Mmon[RRQ_NPMAX * RRQ_NPMAX];             // [ab][i] coefficient of u^a v^b in the node
                                                    // Lagrange function l_i (ab a-major, a + b < p)
    double Cjl[(RRQ_PMAX + 1) * (RRQ_PMAX + 1)];    // [l][j] C_{j,l} = (j-2)!(l-j)!/(l-1)!, j >= 2
    double Djl[(RRQ_PMAX + 1) * (RRQ_PMAX + 1)];    // [l][j] D_{j,l} = (j-1)!(l-j)!/l!, j >= 1
    // Rotation of the degree-l harmonics by -90 and +90 degrees about the Y axis of their own
    // frame, Rn_l^m(Ry(+-90) a) = sum_k Delta^{+-}_{mk} Rn_l^k(a), folded for coefficient sets
    // with c_{-k} = (-1)^k conj(c_k): Re y_m = sum_{k>=0} A_{mk} Re c_k, Im y_m = sum_{k>=1}
    // B_{mk} Im c_k.  Per degree l at rot_off(l): A- [(l+1)^2], B- [l^2], A+, B+ (row-major,
    // B indexed from 1).  Used by the rotation-based translation (Sec. 2.3).
    double Drot[2 * ((RRQ_PMAX + 1) * RRQ_PMAX * (2 * RRQ_PMAX + 1) / 3 + (RRQ_PMAX + 1) * RRQ_PMAX + RRQ_PMAX + 1)];
};

// offset of degree l in OrderTables::Drot
__host__ __device__ __forceinline__ constexpr int rot_off(int l) {
    return 2 * ((l - 1) * l * (2 * l - 1) / 3 + l * (l - 1) + l);
}

// Complex preimage of one (pair, edge): Re t0, Im t0, converged (0/1), singularity swap (0/1).
struct EdgeRoot {
    double x, y, z, w;
};

// Device-side per-patch data; per-patch strides are those of the largest order pmax of the
// build (pd_*(pmax) below), the layout inside a patch is that of the patch's own order.
struct PatchData {
    int npatch;
    int pmax;
    double *frame;   // [P][16]  c[3], R[3][3] (R[a][b] = b-th frame vector, component a), s
    double *bounds;  // [P][5]   c_P[3], R_P, d_P (global coordinates, for the near list)
    double *ynode;   // [P][NPMAX*3] local node coordinates
    double *ea;      // [P][3*PMAX*3] local Legendre coefficients of the 3 edges, [e][n][a]
    double *ey;      // [P][3*PTMAX*3] local edge samples at the Gauss nodes, [e*pt+q][a]
    double *et;      // [P][3*PTMAX*3] tangents dy/dt at the edge samples
    double *eyu;     // [P][3*2PTMAX*3] local edge samples at the upsampled nodes
    cd *eg;          // [P][3*PTMAX][NJKMAX][3] grad S^{(j,k)} at edge samples
    cd *eh;          // [P][3*PTMAX][NJKMAX][3] (Hess S^{(j,k)}) tau at edge samples
    float4 *eg2;     // same as eg as (re.hi, re.lo, im.hi, im.lo) float pairs, or NULL
    float4 *eh2;     // same as eh as float pairs, or NULL
    double *XD;      // [P][4*NPMAX][NPMAX] quaternion fit of (mu, 0):    row c*np+lm, col i
    double *XSp;     // [P][4*NPMAX][NPMAX] quaternion fit of (0, sigma nu)
    double *XS2;     // [P][4*NPMAX][NPMAX] quaternion fit of the intermediate density
    double *XS1;     // [P][NPMAX][NPMAX]   scalar fit A_S^{-1}
    float2 *XD2, *XSp2, *XS22, *XS12;  // the four fit matrices as (hi, lo) float pairs, or NULL
    int *status;     // [P] 0 ok, nonzero = singular fit / degenerate patch
    double *kappa;   // [P] 1-norm condition number of the fit matrix A (Sec. 5.1), or NULL
    double *lu;      // [P][4*NPMAX*NPMAX] quaternion LU factor of the fit for orders above 12
                     // (too large for shared memory there), or NULL
    double *xm;      // [P][NPMAX*3] monomial coefficients [ab][a] of the local node interpolant
    EdgeRoot *roots;  // [pair item][3 edges]: (Re t0, Im t0, converged, singularity swap)
    int8_t *uside;    // [pair item] side of the patch the target is on along e_z (+1, -1), 0 = unknown
    const int64_t *col_off;  // [P] first CSR column of the patch's nodes, or NULL = node_off
};

static const size_t PD_FRAME = 16, PD_BOUNDS = 5;
// Per-patch strides of the PatchData arrays, for the largest order pm of the build.
__host__ __device__ __forceinline__ size_t pd_np(int pm) { return (size_t)pm * (pm + 1) / 2; }
__host__ __device__ __forceinline__ size_t pd_ynode(int pm) { return pd_np(pm) * 3; }
__host__ __device__ __forceinline__ size_t pd_ea(int pm) { return (size_t)3 * pm * 3; }
__host__ __device__ __forceinline__ size_t pd_ey(int pm) { return (size_t)3 * 2 * pm * 3; }
__host__ __device__ __forceinline__ size_t pd_eyu(int pm) { return (size_t)3 * 4 * pm * 3; }
__host__ __device__ __forceinline__ size_t pd_eg(int pm) { return (size_t)3 * 2 * pm * ((pm + 1) * (pm + 2) / 2) * 3; }
__host__ __device__ __forceinline__ size_t pd_X(int pm) { return 4 * pd_np(pm) * pd_np(pm); }
__host__ __device__ __forceinline__ size_t pd_XS1(int pm) { return pd_np(pm) * pd_np(pm); }
__host__ __device__ __forceinline__ size_t pd_lu(int pm) { return pm > 12 ? 4 * pd_np(pm) * pd_np(pm) : 0; }

// Pair work item: target, patch, offset of the first CSR entry of the pair, and the
// pair's index in target-major order (near-list order).
struct PairItem {
    int64_t t;
    int64_t off;
    int32_t P;
    int32_t pad;
};

// Device counters of a build.
struct BuildCounters {
    unsigned long long newton_fail, on_edge, u_poor, ssq_edges, far_edges;
};

// Kernel launches issued by the library on this host thread since the last reset
// (reported in rrq_diag.kernel_launches).
int64_t &rrq_launch_counter();
#define RRQ_COUNT_LAUNCH() (++rrq_launch_counter())

// Host entry points implemented in the individual translation units.
int rrq_host_order_tables(int p, int pt, double rho0, const double *ref_uv, OrderTables *out);
cudaError_t rrq_launch_precompute(int p, const OrderTables *d_tab, const int32_t *d_plist, int n,
                                  const int64_t *d_node_off, const double *d_xyz, const double *d_nrm,
                                  PatchData pd, cudaStream_t st);
// Arguments of the per-pair stage of one order (Sec. 4 Steps 4-8 for every pair item).
struct PairArgs {
    const OrderTables *tab;
    const PairItem *items;
    int64_t nitems;
    PatchData pd;
    const int64_t *node_off;
    const double *xyz, *nrm, *wts, *txyz, *tnrm;
    const int64_t *tself;
    uint32_t mask;
    int newton_max;
    double *val[4];       // S, D, S', D' values (NULL = not built)
    int32_t *col;
    BuildCounters *cnt;
    // density-given evaluation (rrq_evaluate_near) instead of rows: per patch the fit
    // coefficients of the density, [P][13 NPMAX] = X_D sigma (4 NPMAX), X_S' sigma, X_S2 sigma,
    // X_S1 sigma (NPMAX); the density; one result per (pair in target-major order, kernel)
    const double *coef;
    const double *sigma;
    double *res[4];
    int rot;              // 1: rotation-based translation (FP64 matrix build, the default tile)
};

// Launch shape of the per-pair stage.
struct PairShape {
    int tile;                       // pairs per CTA; 0 = the order's default
    int persistent;                 // 1: one wave of CTAs fetching tiles from tile_ctr; 0: grid-stride over 16 waves
    unsigned long long *tile_ctr;   // device counter for persistent launches (zeroed by the launcher)
};

// Roots and pair kernels of order p; mixed = line integrals in double-float (needs pd.eg2, pd.eh2).
cudaError_t rrq_launch_pairs(int p, bool mixed, const PairArgs &a, PairShape shape, cudaStream_t st);
// The same stage in density-given evaluation form (FP64, PairArgs.coef/sigma/res, item.pad =
// the pair's index in target-major order).
cudaError_t rrq_launch_pairs_eval(int p, const PairArgs &a, PairShape shape, cudaStream_t st);
// Tile sizes compiled for order p (the first is the default); returns their number.
int rrq_pair_tiles(int p, int tiles[4]);
