// C ABI of librrq (include/rrq.h): argument checks, device memory, orchestration of
// the near list (K1), the per-patch precompute (K2), CSR row pointers and pair items
// (K4), the per-pair kernel (K3), and the corrected-operator apply (K5).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "rrq_host.h"





static thread_local char g_err[RRQ_ERR_LEN] = "";
char *rrq_err_buf() { return g_err; }
void set_err(const char *what, cudaError_t e) { snprintf(g_err, RRQ_ERR_LEN, "%s: %s", what, cudaGetErrorString(e)); }

#define RRQ_DECL_PAIRS(P)                                                                              \
    cudaError_t rrq_launch_pairs_p##P(bool, const PairArgs &, const PairShape &, cudaStream_t); \
    int rrq_pair_tiles_p##P(int out[4]);                                                                  \
    cudaError_t rrq_launch_pairs_eval_p##P(const PairArgs &, const PairShape &, cudaStream_t);
RRQ_DECL_PAIRS(2)
RRQ_DECL_PAIRS(3)
RRQ_DECL_PAIRS(4)
RRQ_DECL_PAIRS(5)
RRQ_DECL_PAIRS(6)
RRQ_DECL_PAIRS(7)
RRQ_DECL_PAIRS(8)
RRQ_DECL_PAIRS(9)
RRQ_DECL_PAIRS(10)
RRQ_DECL_PAIRS(11)
RRQ_DECL_PAIRS(12)
RRQ_DECL_PAIRS(13)
RRQ_DECL_PAIRS(14)
#undef RRQ_DECL_PAIRS

cudaError_t rrq_launch_pairs(int p, bool mixed, const PairArgs &a, PairShape shape, cudaStream_t st) {
    switch (p) {
#define RRQ_CASE(P) \
    case P: return rrq_launch_pairs_p##P(mixed, a, shape, st);
        RRQ_CASE(2) RRQ_CASE(3) RRQ_CASE(4) RRQ_CASE(5) RRQ_CASE(6) RRQ_CASE(7) RRQ_CASE(8)
        RRQ_CASE(9) RRQ_CASE(10) RRQ_CASE(11) RRQ_CASE(12) RRQ_CASE(13) RRQ_CASE(14)
#undef RRQ_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t rrq_launch_pairs_eval(int p, const PairArgs &a, PairShape shape, cudaStream_t st) {
    switch (p) {
#define RRQ_CASE(P) \
    case P: return rrq_launch_pairs_eval_p##P(a, shape, st);
        RRQ_CASE(2) RRQ_CASE(3) RRQ_CASE(4) RRQ_CASE(5) RRQ_CASE(6) RRQ_CASE(7) RRQ_CASE(8)
        RRQ_CASE(9) RRQ_CASE(10) RRQ_CASE(11) RRQ_CASE(12) RRQ_CASE(13) RRQ_CASE(14)
#undef RRQ_CASE
        default: return cudaErrorInvalidValue;
    }
}

int rrq_pair_tiles(int p, int tiles[4]) {
    switch (p) {
#define RRQ_CASE(P) \
    case P: return rrq_pair_tiles_p##P(tiles);
        RRQ_CASE(2) RRQ_CASE(3) RRQ_CASE(4) RRQ_CASE(5) RRQ_CASE(6) RRQ_CASE(7) RRQ_CASE(8)
        RRQ_CASE(9) RRQ_CASE(10) RRQ_CASE(11) RRQ_CASE(12) RRQ_CASE(13) RRQ_CASE(14)
#undef RRQ_CASE
        default: return 0;
    }
}

namespace {

constexpr int kMaxChecked = 8;
struct CheckedArrays {
    const double *a[kMaxChecked];
    int64_t n[kMaxChecked];
    int count;
};

// Sets bit k of *bad when array k holds a NaN or an infinity: blockIdx.y selects the
// array, grid-stride over its elements, one warp vote per warp.
__global__ void __launch_bounds__(256) k_nonfinite(CheckedArrays arr, unsigned *bad) {
    const int k = blockIdx.y;
    const double *__restrict__ a = arr.a[k];
    const int64_t n = a ? arr.n[k] : 0;
    bool any = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        any |= !isfinite(a[i]);
    if (__any_sync(0xffffffffu, any) && (threadIdx.x & 31) == 0) atomicOr(bad, 1u << k);
}

}  // namespace

rrq_status check_finite(cudaStream_t st, unsigned *d_flag, const double *const arrays[], const int64_t sizes[],
                        const char *const names[], int n) {
    if (n > kMaxChecked) return RRQ_ERR_ARG;
    CheckedArrays arr{};
    int64_t most = 0;
    for (int a = 0; a < n; a++) {
        arr.a[a] = sizes[a] > 0 ? arrays[a] : nullptr;
        arr.n[a] = sizes[a];
        most = std::max(most, sizes[a]);
    }
    arr.count = n;
    CK(cudaMemsetAsync(d_flag, 0, sizeof(unsigned), st));
    if (most > 0) {
        const int64_t blocks = std::min<int64_t>((most + 255) / 256, 152 * 2);
        k_nonfinite<<<dim3((unsigned)blocks, (unsigned)n), 256, 0, st>>>(arr, d_flag);
        RRQ_COUNT_LAUNCH();
        CK(cudaGetLastError());
    }
    unsigned h = 0;
    CK(cudaMemcpyAsync(&h, d_flag, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int a = 0; a < n; a++)
        if (h & (1u << a)) {
            snprintf(rrq_err_buf(), RRQ_ERR_LEN, "non-finite value (NaN or infinity) in the %s", names[a]);
            return RRQ_ERR_ARG;
        }
    return RRQ_OK;
}

rrq_status prepare_inputs(rrq_ctx *ctx, Scratch &s, const rrq_surface *surf, const rrq_targets *targ, bool on_host,
                          bool need_targets, Inputs &in) {
    if (!surf || surf->npatch < 1 || !surf->order || !surf->node_off || !surf->xyz || !surf->nrm || !surf->wts)
        return RRQ_ERR_ARG;
    if (need_targets && (!targ || targ->ntarg < 0 || (targ->ntarg > 0 && (!targ->xyz || !targ->nrm))))
        return RRQ_ERR_ARG;
    in.npatch = surf->npatch;
    in.h_order.resize(in.npatch);
    in.h_node_off.resize(in.npatch + 1);
    if (on_host) {
        memcpy(in.h_order.data(), surf->order, sizeof(int32_t) * in.npatch);
        memcpy(in.h_node_off.data(), surf->node_off, sizeof(int64_t) * (in.npatch + 1));
    } else {
        CK(cudaMemcpyAsync(in.h_order.data(), surf->order, sizeof(int32_t) * in.npatch, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(in.h_node_off.data(), surf->node_off, sizeof(int64_t) * (in.npatch + 1),
                           cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    if (in.h_node_off[0] != 0) return RRQ_ERR_ARG;
    for (int P = 0; P < in.npatch; P++) {
        int p = in.h_order[P];
        if (p < 2 || p > RRQ_PMAX || !surf->ref_uv[p]) return RRQ_ERR_ARG;
        if (in.h_node_off[P + 1] - in.h_node_off[P] != np_of(p)) return RRQ_ERR_ARG;
    }
    in.nnode = in.h_node_off[in.npatch];
    in.ntarg = need_targets ? targ->ntarg : 0;
    if (in.nnode >= (int64_t)INT32_MAX) return RRQ_ERR_ARG;
    cudaError_t err = cudaSuccess;
    in.order = upload(s, surf->order, in.npatch, on_host, &err);
    in.node_off = upload(s, surf->node_off, in.npatch + 1, on_host, &err);
    in.xyz = upload(s, surf->xyz, 3 * in.nnode, on_host, &err);
    in.nrm = upload(s, surf->nrm, 3 * in.nnode, on_host, &err);
    in.wts = upload(s, surf->wts, in.nnode, on_host, &err);
    if (need_targets) {
        in.txyz = upload(s, targ->xyz, 3 * in.ntarg, on_host, &err);
        in.tnrm = upload(s, targ->nrm, 3 * in.ntarg, on_host, &err);
        in.tself = targ->self_node ? upload(s, targ->self_node, in.ntarg, on_host, &err) : nullptr;
    } else {
        in.txyz = in.tnrm = nullptr;
        in.tself = nullptr;
    }
    if (err != cudaSuccess) {
        set_err("input upload", err);
        return err == cudaErrorMemoryAllocation ? RRQ_ERR_OOM : RRQ_ERR_CUDA;
    }
    unsigned *flag = (unsigned *)Scratch::alloc(&s, sizeof(unsigned));
    if (!flag) return RRQ_ERR_OOM;
    const double *arrays[5] = {in.xyz, in.nrm, in.wts, in.txyz, in.tnrm};
    const int64_t sizes[5] = {3 * in.nnode, 3 * in.nnode, in.nnode, 3 * in.ntarg, 3 * in.ntarg};
    return check_finite(s.st, flag, arrays, sizes, kInputNames, need_targets ? 5 : 3);
}

rrq_status order_tables(rrq_ctx *ctx, int p, const double *ref_uv, double rho0) {
    const int np = np_of(p);
    std::vector<double> key(ref_uv, ref_uv + 2 * np);
    if (ctx->d_tab[p] && ctx->tab_key[p] == key && ctx->tab_rho0[p] == rho0) return RRQ_OK;
    OrderTables h;
    if (rrq_host_order_tables(p, 2 * p, rho0, ref_uv, &h)) return RRQ_ERR_ARG;
    if (!ctx->d_tab[p]) CK(cudaMalloc(&ctx->d_tab[p], sizeof(OrderTables)));
    CK(cudaMemcpyAsync(ctx->d_tab[p], &h, sizeof(OrderTables), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->tab_key[p] = key;
    ctx->tab_rho0[p] = rho0;
    return RRQ_OK;
}


extern "C" {

const char *rrq_status_string(rrq_status s) {
    switch (s) {
        case RRQ_OK: return "ok";
        case RRQ_ERR_ARG: return "invalid argument";
        case RRQ_ERR_CUDA: return "CUDA error";
        case RRQ_ERR_OOM: return "out of device memory";
        case RRQ_ERR_DEGENERATE: return "degenerate patch or singular fit";
        case RRQ_ERR_UNSUPPORTED: return "unsupported option";
        case RRQ_WARN_ROOTFIND: return "ok, some edges used the fallback rule";
        default: return "unknown status";
    }
}

const char *rrq_last_error(void) { return rrq_err_buf(); }

rrq_status rrq_ctx_create(rrq_ctx **ctx, int device, void *cuda_stream) {
    if (!ctx) return RRQ_ERR_ARG;
    *ctx = nullptr;
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return RRQ_ERR_ARG;
    CK(cudaSetDevice(device));
    rrq_ctx *c = new rrq_ctx();
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    memset(&c->diag, 0, sizeof(c->diag));
    for (int p = 0; p <= RRQ_PMAX; p++) { c->d_tab[p] = nullptr; c->tab_rho0[p] = -1; }
    memset(c->tune_tile, 0, sizeof(c->tune_tile));
    memset(c->tune_pers, 0, sizeof(c->tune_pers));
    for (int i = 0; i < 4; i++) cudaEventCreate(&c->ev[i]);
    // keep freed stream-ordered memory in the pool between builds
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    *ctx = c;
    return RRQ_OK;
}

void rrq_ctx_destroy(rrq_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (int p = 0; p <= RRQ_PMAX; p++)
        if (ctx->d_tab[p]) cudaFree(ctx->d_tab[p]);
    for (int i = 0; i < 4; i++) cudaEventDestroy(ctx->ev[i]);
    delete ctx;
}

rrq_status rrq_last_diagnostics(rrq_ctx *ctx, rrq_diag *diag) {
    if (!ctx || !diag) return RRQ_ERR_ARG;
    *diag = ctx->diag;
    return RRQ_OK;
}

}  // extern "C"


namespace {

// Everything a build needs before the per-pair stage: device inputs, per-order tables,
// per-patch data (Steps 1-3, precompute kernels), near list and pair items grouped by
// (order, patch), CSR row pointers and entry count.  Stage times go to ctx->diag.
struct Prep {
    Inputs in;
    std::vector<std::vector<int32_t>> plist;
    PatchData pd{};
    NearBuffers nb{};
    int64_t *rowptr = nullptr;  // [ntarg + 1]; cudaMallocAsync'd when rowptr_for_caller, else scratch
    PairItem *items = nullptr;
    std::vector<int64_t> h_roff;
    int64_t nnz = 0;
    BuildCounters *d_cnt = nullptr;
    bool mixed = false;
    bool rot = false;      // rotation-based translation
    int newton_max = 30;
    double kappa_max = 0;  // max over patches of kappa_1(A)
};

// Device arrays of the per-patch data (every array the precompute kernels write) in the
// scratch arena; a failed allocation marks the arena failed.
void alloc_patch_data(Scratch &s, size_t NPc, bool mixed, PatchData &pd) {
    pd.frame = (double *)Scratch::alloc(&s, sizeof(double) * NPc * PD_FRAME);
    pd.bounds = (double *)Scratch::alloc(&s, sizeof(double) * NPc * PD_BOUNDS);
    pd.ynode = (double *)Scratch::alloc(&s, sizeof(double) * NPc * pd_ynode(pd.pmax));
    pd.xm = (double *)Scratch::alloc(&s, sizeof(double) * NPc * pd_ynode(pd.pmax));
    pd.ea = (double *)Scratch::alloc(&s, sizeof(double) * NPc * pd_ea(pd.pmax));
    pd.ey = (double *)Scratch::alloc(&s, sizeof(double) * NPc * pd_ey(pd.pmax));
    pd.et = (double *)Scratch::alloc(&s, sizeof(double) * NPc * pd_ey(pd.pmax));
    pd.eyu = (double *)Scratch::alloc(&s, sizeof(double) * NPc * pd_eyu(pd.pmax));
    pd.eg = (cd *)Scratch::alloc(&s, sizeof(cd) * NPc * pd_eg(pd.pmax));
    pd.eh = (cd *)Scratch::alloc(&s, sizeof(cd) * NPc * pd_eg(pd.pmax));
    pd.eg2 = mixed ? (float4 *)Scratch::alloc(&s, sizeof(float4) * NPc * pd_eg(pd.pmax)) : nullptr;
    pd.eh2 = mixed ? (float4 *)Scratch::alloc(&s, sizeof(float4) * NPc * pd_eg(pd.pmax)) : nullptr;
    if (mixed) {
        pd.XD2 = (float2 *)Scratch::alloc(&s, sizeof(float2) * NPc * pd_X(pd.pmax));
        pd.XSp2 = (float2 *)Scratch::alloc(&s, sizeof(float2) * NPc * pd_X(pd.pmax));
        pd.XS22 = (float2 *)Scratch::alloc(&s, sizeof(float2) * NPc * pd_X(pd.pmax));
        pd.XS12 = (float2 *)Scratch::alloc(&s, sizeof(float2) * NPc * pd_XS1(pd.pmax));
    }
    pd.XD = (double *)Scratch::alloc(&s, sizeof(double) * NPc * pd_X(pd.pmax));
    pd.XSp = (double *)Scratch::alloc(&s, sizeof(double) * NPc * pd_X(pd.pmax));
    pd.XS2 = (double *)Scratch::alloc(&s, sizeof(double) * NPc * pd_X(pd.pmax));
    pd.XS1 = (double *)Scratch::alloc(&s, sizeof(double) * NPc * pd_XS1(pd.pmax));
    pd.status = (int *)Scratch::alloc(&s, sizeof(int) * NPc);
    pd.kappa = (double *)Scratch::alloc(&s, sizeof(double) * NPc);
    pd.lu = pd_lu(pd.pmax) ? (double *)Scratch::alloc(&s, sizeof(double) * NPc * pd_lu(pd.pmax)) : nullptr;
}

rrq_status build_prep(rrq_ctx *ctx, Scratch &s, const rrq_surface *surf, const rrq_targets *targ, const rrq_options &o,
                      bool rowptr_for_caller, Prep &pr) {
    const double eta = o.eta > 0 ? o.eta : 1.0;
    pr.newton_max = o.newton_max > 0 ? o.newton_max : 30;
    if (o.precision != 0 && o.precision != 1) return RRQ_ERR_ARG;
    if (o.translation != 0 && o.translation != 1) return RRQ_ERR_ARG;
    if (o.translation == 1 && o.precision != 0) {
        snprintf(rrq_err_buf(), RRQ_ERR_LEN, "rotation-based translation: FP64 builds only (precision = 0)");
        return RRQ_ERR_UNSUPPORTED;
    }
    pr.mixed = o.precision == 1;
    pr.rot = o.translation == 1;
    const bool mixed = pr.mixed;
    Inputs &in = pr.in;
    rrq_status rs = prepare_inputs(ctx, s, surf, targ, o.inputs_on_host != 0, true, in);
    if (rs != RRQ_OK) return rs;
    if (o.ptilde != 0)
        for (int P = 0; P < in.npatch; P++)
            if (o.ptilde != 2 * in.h_order[P]) return RRQ_ERR_UNSUPPORTED;
    // per-order tables and patch lists
    int pmax = 0;
    std::vector<std::vector<int32_t>> &plist = pr.plist;
    plist.assign(RRQ_PMAX + 1, {});
    for (int P = 0; P < in.npatch; P++) {
        plist[in.h_order[P]].push_back(P);
        pmax = std::max(pmax, in.h_order[P]);
    }
    for (int p = 2; p <= RRQ_PMAX; p++)
        if (!plist[p].empty()) {
            rs = order_tables(ctx, p, surf->ref_uv[p], o.rho0);
            if (rs != RRQ_OK) return rs;
        }
    // patch data
    const size_t NPc = in.npatch;
    PatchData &pd = pr.pd;
    pd.npatch = in.npatch;
    pd.pmax = pmax;
    alloc_patch_data(s, NPc, mixed, pd);
    std::vector<int32_t> rank(in.npatch);
    std::vector<int32_t> order_major;
    order_major.reserve(in.npatch);
    for (int p = 2; p <= RRQ_PMAX; p++)
        for (int32_t P : plist[p]) order_major.push_back(P);
    for (int r = 0; r < in.npatch; r++) rank[order_major[r]] = r;
    int32_t *d_plists = (int32_t *)Scratch::alloc(&s, sizeof(int32_t) * in.npatch);
    int32_t *d_rank = (int32_t *)Scratch::alloc(&s, sizeof(int32_t) * in.npatch);
    pr.d_cnt = (BuildCounters *)Scratch::alloc(&s, sizeof(BuildCounters));
    if (s.failed) return RRQ_ERR_OOM;
    CK(cudaMemcpyAsync(d_plists, order_major.data(), sizeof(int32_t) * in.npatch, cudaMemcpyHostToDevice, s.st));
    CK(cudaMemcpyAsync(d_rank, rank.data(), sizeof(int32_t) * in.npatch, cudaMemcpyHostToDevice, s.st));
    CK(cudaMemsetAsync(pr.d_cnt, 0, sizeof(BuildCounters), s.st));
    CK(cudaEventRecord(ctx->ev[0], s.st));
    {
        int start = 0;
        for (int p = 2; p <= RRQ_PMAX; p++) {
            int n = (int)plist[p].size();
            if (n) CK(rrq_launch_precompute(p, ctx->d_tab[p], d_plists + start, n, in.node_off, in.xyz, in.nrm, pd, s.st));
            start += n;
        }
    }
    CK(cudaEventRecord(ctx->ev[1], s.st));
    CK(rrq_near_build(pd.bounds, in.npatch, in.node_off, in.txyz, in.tself, in.ntarg, eta, &Scratch::alloc, &s, &pr.nb,
                      s.st));
    if (s.failed) return RRQ_ERR_OOM;
    if (rowptr_for_caller)
        CK(cudaMallocAsync(&pr.rowptr, sizeof(int64_t) * (in.ntarg + 1), s.st));
    else
        pr.rowptr = (int64_t *)Scratch::alloc(&s, sizeof(int64_t) * (in.ntarg + 1));
    if (!pr.rowptr) return RRQ_ERR_OOM;
    int64_t *roff = nullptr;
    cudaError_t e = rrq_items_build(&pr.nb, in.ntarg, in.order, d_rank, in.npatch, &Scratch::alloc, &s, pr.rowptr,
                                    &pr.items, &roff, s.st);
    if (e != cudaSuccess || s.failed) {
        set_err("pair items", e);
        return s.failed ? RRQ_ERR_OOM : RRQ_ERR_CUDA;
    }
    // sizes: nnz and the item range of every order
    pr.h_roff.assign(in.npatch + 1, 0);
    CK(cudaMemcpyAsync(&pr.nnz, pr.rowptr + in.ntarg, sizeof(int64_t), cudaMemcpyDeviceToHost, s.st));
    CK(cudaMemcpyAsync(pr.h_roff.data(), roff, sizeof(int64_t) * (in.npatch + 1), cudaMemcpyDeviceToHost, s.st));
    std::vector<int> h_status(in.npatch);
    std::vector<double> h_kappa(in.npatch);
    CK(cudaMemcpyAsync(h_status.data(), pd.status, sizeof(int) * in.npatch, cudaMemcpyDeviceToHost, s.st));
    CK(cudaMemcpyAsync(h_kappa.data(), pd.kappa, sizeof(double) * in.npatch, cudaMemcpyDeviceToHost, s.st));
    CK(cudaEventRecord(ctx->ev[2], s.st));
    CK(cudaStreamSynchronize(s.st));
    pr.kappa_max = *std::max_element(h_kappa.begin(), h_kappa.end());
    for (int P = 0; P < in.npatch; P++)
        if (h_status[P]) return RRQ_ERR_DEGENERATE;
    return RRQ_OK;
}

}  // namespace

extern "C" rrq_status rrq_build_corrections(rrq_ctx *ctx, const rrq_surface *surf, const rrq_targets *targ,
                                            uint32_t kernel_mask, const rrq_options *opt, rrq_csr *out) {
    if (!ctx || !out) return RRQ_ERR_ARG;
    memset(out, 0, sizeof(*out));
    if (kernel_mask == 0 || (kernel_mask & ~15u)) return RRQ_ERR_ARG;
    rrq_options o;
    memset(&o, 0, sizeof(o));
    if (opt) o = *opt;
    CK(cudaSetDevice(ctx->device));
    memset(&ctx->diag, 0, sizeof(ctx->diag));
    rrq_launch_counter() = 0;
    Scratch s;
    s.st = ctx->stream;
    Prep pr;
    rrq_status rs = build_prep(ctx, s, surf, targ, o, true, pr);
    if (rs != RRQ_OK) {
        if (pr.rowptr) cudaFreeAsync(pr.rowptr, s.st);
        return rs;
    }
    const Inputs &in = pr.in;
    const std::vector<std::vector<int32_t>> &plist = pr.plist;
    const PatchData &pd = pr.pd;
    const NearBuffers &nb = pr.nb;
    int64_t *d_rowptr = pr.rowptr;
    PairItem *items = pr.items;
    const std::vector<int64_t> &h_roff = pr.h_roff;
    const int64_t nnz = pr.nnz;
    BuildCounters *d_cnt = pr.d_cnt;
    const bool mixed = pr.mixed;
    const int newton_max = pr.newton_max;
    cudaError_t e = cudaSuccess;
    int32_t *col = nullptr;
    double *vals[4] = {nullptr, nullptr, nullptr, nullptr};
    bool oom = cudaMallocAsync(&col, sizeof(int32_t) * (nnz > 0 ? nnz : 1), s.st) != cudaSuccess;
    for (int k = 0; k < 4 && !oom; k++)
        if (kernel_mask & (1u << k)) oom = cudaMallocAsync(&vals[k], sizeof(double) * (nnz > 0 ? nnz : 1), s.st) != cudaSuccess;
    if (oom) {
        cudaGetLastError();
        cudaFreeAsync(d_rowptr, s.st);
        if (col) cudaFreeAsync(col, s.st);
        for (int k = 0; k < 4; k++)
            if (vals[k]) cudaFreeAsync(vals[k], s.st);
        return RRQ_ERR_OOM;
    }
    EdgeRoot *roots = (EdgeRoot *)Scratch::alloc(&s, sizeof(EdgeRoot) * 3 * (nb.npairs > 0 ? nb.npairs : 1));
    int8_t *uside = (int8_t *)Scratch::alloc(&s, sizeof(int8_t) * (nb.npairs > 0 ? nb.npairs : 1));
    unsigned long long *tile_ctr = (unsigned long long *)Scratch::alloc(&s, sizeof(unsigned long long) * (RRQ_PMAX + 1));
    if (!roots || !uside || !tile_ctr) oom = true;
    if (oom) {
        cudaFreeAsync(d_rowptr, s.st);
        cudaFreeAsync(col, s.st);
        for (int k = 0; k < 4; k++)
            if (vals[k]) cudaFreeAsync(vals[k], s.st);
        return RRQ_ERR_OOM;
    }
    {
        int start = 0;
        for (int p = 2; p <= RRQ_PMAX; p++) {
            int n = (int)plist[p].size();
            if (n) {
                int64_t i0 = h_roff[start], i1 = h_roff[start + n];
                PatchData pdo = pd;
                pdo.roots = roots + 3 * i0;
                pdo.uside = uside + i0;
                PairArgs pa = {ctx->d_tab[p], items + i0, i1 - i0, pdo, in.node_off, in.xyz, in.nrm, in.wts,
                               in.txyz, in.tnrm, in.tself, kernel_mask, newton_max,
                               {vals[0], vals[1], vals[2], vals[3]}, col, d_cnt};
                pa.rot = pr.rot;
                const PairShape shape{ctx->tune_tile[mixed][p], ctx->tune_pers[mixed][p], tile_ctr + p};
                e = rrq_launch_pairs(p, mixed, pa, shape, s.st);
                if (e != cudaSuccess) break;
            }
            start += n;
        }
    }
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev[3], s.st);
    BuildCounters hc;
    memset(&hc, 0, sizeof(hc));
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, d_cnt, sizeof(hc), cudaMemcpyDeviceToHost, s.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s.st);
    if (e != cudaSuccess) {
        set_err("pair kernel", e);
        cudaFreeAsync(d_rowptr, s.st);
        cudaFreeAsync(col, s.st);
        for (int k = 0; k < 4; k++)
            if (vals[k]) cudaFreeAsync(vals[k], s.st);
        return RRQ_ERR_CUDA;
    }
    out->nrows = in.ntarg;
    out->nnz = nnz;
    out->npairs = nb.npairs;
    out->kernel_mask = kernel_mask;
    out->rowptr = d_rowptr;
    out->col = col;
    for (int k = 0; k < 4; k++) out->val[k] = vals[k];
    ctx->diag.npairs = nb.npairs;
    ctx->diag.newton_fail = (int64_t)hc.newton_fail;
    ctx->diag.on_edge = (int64_t)hc.on_edge;
    ctx->diag.u_poor = (int64_t)hc.u_poor;
    ctx->diag.ssq_edges = (int64_t)hc.ssq_edges;
    ctx->diag.far_edges = (int64_t)hc.far_edges;
    float ms = 0;
    cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]);
    ctx->diag.ms_precompute = ms;
    cudaEventElapsedTime(&ms, ctx->ev[1], ctx->ev[2]);
    ctx->diag.ms_near = ms;
    cudaEventElapsedTime(&ms, ctx->ev[2], ctx->ev[3]);
    ctx->diag.ms_pairs = ms;
    ctx->diag.kernel_launches = rrq_launch_counter();
    ctx->diag.kappa_max = pr.kappa_max;
    return hc.newton_fail > 0 ? RRQ_WARN_ROOTFIND : RRQ_OK;
}

namespace {
__global__ void k_rebase(int64_t *rowptr, int64_t n, int64_t first) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) rowptr[i] -= first;
}
}  // namespace

namespace {

// Fit coefficients of the density on every patch (Sec. 4 Step 2 for a given density):
// [P][13 NPMAX] = X_D sigma_P (4 n_p rows), X_S' sigma_P, X_S2 sigma_P, X_S1 sigma_P (n_p rows).
__global__ void k_patch_coef(const int32_t *__restrict__ order, const int64_t *__restrict__ node_off, PatchData pd,
                             const double *__restrict__ sig, double *__restrict__ coef) {
    const int P = blockIdx.x;
    const int p = order[P], np = p * (p + 1) / 2;
    const double *s = sig + node_off[P];
    double *c = coef + (size_t)P * (13 * RRQ_NPMAX);
    for (int r = threadIdx.x; r < 13 * np; r += blockDim.x) {
        const double *X;
        double *dst;
        int row;
        if (r < 12 * np) {
            const int blk = r / (4 * np);
            row = r % (4 * np);
            X = (blk == 0 ? pd.XD : blk == 1 ? pd.XSp : pd.XS2) + (size_t)P * pd_X(pd.pmax);
            dst = c + blk * 4 * RRQ_NPMAX;
        } else {
            row = r - 12 * np;
            X = pd.XS1 + (size_t)P * pd_XS1(pd.pmax);
            dst = c + 12 * RRQ_NPMAX;
        }
        double v = 0.0;
        for (int i = 0; i < np; i++) v = fma(X[row * np + i], s[i], v);
        dst[row] = v;
    }
}

// out[t] = sum of the pair results of target t, in near-list order
__global__ void k_pair_reduce(const int64_t *__restrict__ poff, int64_t ntarg, const double *__restrict__ res,
                              double *__restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntarg) return;
    double v = 0.0;
    for (int64_t q = poff[t]; q < poff[t + 1]; q++) v += res[q];
    out[t] = v;
}

}  // namespace

extern "C" rrq_status rrq_evaluate_near(rrq_ctx *ctx, const rrq_surface *surf, const rrq_targets *targ,
                                        uint32_t kernel_mask, const double *density, double *out[4],
                                        const rrq_options *opt) {
    if (!ctx || !density || !out) return RRQ_ERR_ARG;
    if (kernel_mask == 0 || (kernel_mask & ~15u)) return RRQ_ERR_ARG;
    for (int k = 0; k < 4; k++)
        if ((kernel_mask & (1u << k)) && !out[k]) return RRQ_ERR_ARG;
    rrq_options o;
    memset(&o, 0, sizeof(o));
    if (opt) o = *opt;
    if (o.precision != 0 || o.translation != 0) return RRQ_ERR_UNSUPPORTED;
    CK(cudaSetDevice(ctx->device));
    memset(&ctx->diag, 0, sizeof(ctx->diag));
    rrq_launch_counter() = 0;
    Scratch s;
    s.st = ctx->stream;
    Prep pr;
    rrq_status rs = build_prep(ctx, s, surf, targ, o, false, pr);
    if (rs != RRQ_OK) return rs;
    const Inputs &in = pr.in;
    const int64_t npairs = pr.nb.npairs;
    if (npairs >= (int64_t)INT32_MAX) return RRQ_ERR_UNSUPPORTED;
    const bool on_host = o.inputs_on_host != 0;
    cudaError_t err = cudaSuccess;
    const double *d_sig = upload(s, density, in.nnode, on_host, &err);
    double *coef = (double *)Scratch::alloc(&s, sizeof(double) * (size_t)in.npatch * 13 * RRQ_NPMAX);
    EdgeRoot *roots = (EdgeRoot *)Scratch::alloc(&s, sizeof(EdgeRoot) * 3 * (npairs > 0 ? npairs : 1));
    int8_t *uside = (int8_t *)Scratch::alloc(&s, sizeof(int8_t) * (npairs > 0 ? npairs : 1));
    unsigned long long *tile_ctr = (unsigned long long *)Scratch::alloc(&s, sizeof(unsigned long long) * (RRQ_PMAX + 1));
    double *res[4] = {nullptr, nullptr, nullptr, nullptr}, *dout[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int k = 0; k < 4; k++)
        if (kernel_mask & (1u << k)) {
            res[k] = (double *)Scratch::alloc(&s, sizeof(double) * (npairs > 0 ? npairs : 1));
            dout[k] = on_host ? (double *)Scratch::alloc(&s, sizeof(double) * (in.ntarg > 0 ? in.ntarg : 1)) : out[k];
        }
    if (err != cudaSuccess || s.failed) return RRQ_ERR_OOM;
    k_patch_coef<<<in.npatch, 128, 0, s.st>>>(in.order, in.node_off, pr.pd, d_sig, coef);
    RRQ_COUNT_LAUNCH();
    CK(cudaGetLastError());
    int start = 0;
    for (int p = 2; p <= RRQ_PMAX; p++) {
        const int n = (int)pr.plist[p].size();
        if (n) {
            const int64_t i0 = pr.h_roff[start], i1 = pr.h_roff[start + n];
            PatchData pdo = pr.pd;
            pdo.roots = roots + 3 * i0;
            pdo.uside = uside + i0;
            const PairArgs pa = {ctx->d_tab[p], pr.items + i0, i1 - i0, pdo, in.node_off, in.xyz, in.nrm, in.wts,
                                 in.txyz, in.tnrm, in.tself, kernel_mask, pr.newton_max,
                                 {nullptr, nullptr, nullptr, nullptr}, nullptr, pr.d_cnt,
                                 coef, d_sig, {res[0], res[1], res[2], res[3]}};
            CK(rrq_launch_pairs_eval(p, pa, PairShape{ctx->tune_tile[0][p], ctx->tune_pers[0][p], tile_ctr + p}, s.st));
        }
        start += n;
    }
    for (int k = 0; k < 4; k++)
        if (res[k] && in.ntarg > 0) {
            k_pair_reduce<<<(unsigned)((in.ntarg + 255) / 256), 256, 0, s.st>>>(pr.nb.poff, in.ntarg, res[k], dout[k]);
            RRQ_COUNT_LAUNCH();
            CK(cudaGetLastError());
        }
    CK(cudaEventRecord(ctx->ev[3], s.st));
    if (on_host)
        for (int k = 0; k < 4; k++)
            if (dout[k] && in.ntarg > 0)
                CK(cudaMemcpyAsync(out[k], dout[k], sizeof(double) * in.ntarg, cudaMemcpyDeviceToHost, s.st));
    BuildCounters hc;
    CK(cudaMemcpyAsync(&hc, pr.d_cnt, sizeof(hc), cudaMemcpyDeviceToHost, s.st));
    CK(cudaStreamSynchronize(s.st));
    ctx->diag.npairs = npairs;
    ctx->diag.newton_fail = (int64_t)hc.newton_fail;
    ctx->diag.on_edge = (int64_t)hc.on_edge;
    ctx->diag.u_poor = (int64_t)hc.u_poor;
    ctx->diag.ssq_edges = (int64_t)hc.ssq_edges;
    ctx->diag.far_edges = (int64_t)hc.far_edges;
    float ms = 0;
    cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]);
    ctx->diag.ms_precompute = ms;
    cudaEventElapsedTime(&ms, ctx->ev[1], ctx->ev[2]);
    ctx->diag.ms_near = ms;
    cudaEventElapsedTime(&ms, ctx->ev[2], ctx->ev[3]);
    ctx->diag.ms_pairs = ms;
    ctx->diag.kernel_launches = rrq_launch_counter();
    ctx->diag.kappa_max = pr.kappa_max;
    return hc.newton_fail > 0 ? RRQ_WARN_ROOTFIND : RRQ_OK;
}

namespace {

// Device address of a caller buffer: itself for device or managed memory, the mapped
// address for page-locked host memory; false for memory the device cannot address.
bool device_address(void *p, void **dp) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) {
        *dp = p;
        return true;
    }
    if (a.type == cudaMemoryTypeHost && a.devicePointer) {
        *dp = a.devicePointer;
        return true;
    }
    return false;
}

}  // namespace

extern "C" rrq_status rrq_build_corrections_into(rrq_ctx *ctx, const rrq_surface *surf, const rrq_targets *targ,
                                                 uint32_t kernel_mask, const rrq_options *opt, int64_t *rowptr,
                                                 int32_t *col, double *val[4], int64_t capacity, int64_t *nnz_out,
                                                 int64_t *npairs_out) {
    if (!ctx || !rowptr || !col || !val || capacity < 0) return RRQ_ERR_ARG;
    if (kernel_mask == 0 || (kernel_mask & ~15u)) return RRQ_ERR_ARG;
    rrq_options o;
    memset(&o, 0, sizeof(o));
    if (opt) o = *opt;
    CK(cudaSetDevice(ctx->device));
    // every output buffer must be addressable by the kernels that write it
    void *d_col = nullptr, *d_val[4] = {nullptr, nullptr, nullptr, nullptr}, *d_rp = nullptr;
    bool ok = device_address(col, &d_col) && device_address(rowptr, &d_rp);
    for (int k = 0; k < 4 && ok; k++)
        if (kernel_mask & (1u << k)) ok = val[k] && device_address(val[k], &d_val[k]);
    if (!ok) {
        snprintf(rrq_err_buf(), RRQ_ERR_LEN,
                 "rrq_build_corrections_into: an output buffer is neither device memory nor page-locked host memory");
        return RRQ_ERR_ARG;
    }
    memset(&ctx->diag, 0, sizeof(ctx->diag));
    rrq_launch_counter() = 0;
    Scratch s;
    s.st = ctx->stream;
    Prep pr;
    rrq_status rs = build_prep(ctx, s, surf, targ, o, false, pr);
    if (rs != RRQ_OK) return rs;
    if (nnz_out) *nnz_out = pr.nnz;
    if (npairs_out) *npairs_out = pr.nb.npairs;
    if (pr.nnz > capacity) {
        snprintf(rrq_err_buf(), RRQ_ERR_LEN, "rrq_build_corrections_into: %lld entries exceed the capacity %lld",
                 (long long)pr.nnz, (long long)capacity);
        return RRQ_ERR_ARG;
    }
    const NearBuffers &nb = pr.nb;
    EdgeRoot *roots = (EdgeRoot *)Scratch::alloc(&s, sizeof(EdgeRoot) * 3 * (nb.npairs > 0 ? nb.npairs : 1));
    int8_t *uside = (int8_t *)Scratch::alloc(&s, sizeof(int8_t) * (nb.npairs > 0 ? nb.npairs : 1));
    unsigned long long *tile_ctr = (unsigned long long *)Scratch::alloc(&s, sizeof(unsigned long long) * (RRQ_PMAX + 1));
    if (!roots || !uside || !tile_ctr) return RRQ_ERR_OOM;
    cudaError_t e = cudaSuccess;
    int start = 0;
    for (int p = 2; p <= RRQ_PMAX && e == cudaSuccess; p++) {
        const int n = (int)pr.plist[p].size();
        if (n) {
            const int64_t i0 = pr.h_roff[start], i1 = pr.h_roff[start + n];
            PatchData pdo = pr.pd;
            pdo.roots = roots + 3 * i0;
            pdo.uside = uside + i0;
            PairArgs pa = {ctx->d_tab[p], pr.items + i0, i1 - i0, pdo, pr.in.node_off, pr.in.xyz, pr.in.nrm,
                           pr.in.wts, pr.in.txyz, pr.in.tnrm, pr.in.tself, kernel_mask, pr.newton_max,
                           {(double *)d_val[0], (double *)d_val[1], (double *)d_val[2], (double *)d_val[3]},
                           (int32_t *)d_col, pr.d_cnt};
            pa.rot = pr.rot;
            const PairShape shape{ctx->tune_tile[pr.mixed][p], ctx->tune_pers[pr.mixed][p], tile_ctr + p};
            e = rrq_launch_pairs(p, pr.mixed, pa, shape, s.st);
        }
        start += n;
    }
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev[3], s.st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(rowptr, pr.rowptr, sizeof(int64_t) * (pr.in.ntarg + 1), cudaMemcpyDefault, s.st);
    BuildCounters hc;
    memset(&hc, 0, sizeof(hc));
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, pr.d_cnt, sizeof(hc), cudaMemcpyDeviceToHost, s.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s.st);
    if (e != cudaSuccess) {
        set_err("pair kernel", e);
        return RRQ_ERR_CUDA;
    }
    ctx->diag.npairs = nb.npairs;
    ctx->diag.newton_fail = (int64_t)hc.newton_fail;
    ctx->diag.on_edge = (int64_t)hc.on_edge;
    ctx->diag.u_poor = (int64_t)hc.u_poor;
    ctx->diag.ssq_edges = (int64_t)hc.ssq_edges;
    ctx->diag.far_edges = (int64_t)hc.far_edges;
    float ms = 0;
    cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]);
    ctx->diag.ms_precompute = ms;
    cudaEventElapsedTime(&ms, ctx->ev[1], ctx->ev[2]);
    ctx->diag.ms_near = ms;
    cudaEventElapsedTime(&ms, ctx->ev[2], ctx->ev[3]);
    ctx->diag.ms_pairs = ms;
    ctx->diag.kernel_launches = rrq_launch_counter();
    ctx->diag.kappa_max = pr.kappa_max;
    return hc.newton_fail > 0 ? RRQ_WARN_ROOTFIND : RRQ_OK;
}

extern "C" rrq_status rrq_fit_condition(rrq_ctx *ctx, const rrq_surface *surf, double *kappa, int32_t on_host) {
    if (!ctx || !kappa) return RRQ_ERR_ARG;
    CK(cudaSetDevice(ctx->device));
    Scratch s;
    s.st = ctx->stream;
    Inputs in;
    rrq_status rs = prepare_inputs(ctx, s, surf, nullptr, on_host != 0, false, in);
    if (rs != RRQ_OK) return rs;
    std::vector<std::vector<int32_t>> plist(RRQ_PMAX + 1);
    std::vector<int32_t> order_major;
    for (int P = 0; P < in.npatch; P++) plist[in.h_order[P]].push_back(P);
    for (int p = 2; p <= RRQ_PMAX; p++)
        if (!plist[p].empty()) {
            rs = order_tables(ctx, p, surf->ref_uv[p], 0.0);
            if (rs != RRQ_OK) return rs;
            order_major.insert(order_major.end(), plist[p].begin(), plist[p].end());
        }
    PatchData pd{};
    pd.npatch = in.npatch;
    for (int p = 2; p <= RRQ_PMAX; p++)
        if (!plist[p].empty()) pd.pmax = p;
    alloc_patch_data(s, in.npatch, false, pd);
    int32_t *d_plists = (int32_t *)Scratch::alloc(&s, sizeof(int32_t) * in.npatch);
    if (s.failed) return RRQ_ERR_OOM;
    CK(cudaMemcpyAsync(d_plists, order_major.data(), sizeof(int32_t) * in.npatch, cudaMemcpyHostToDevice, s.st));
    int start = 0;
    for (int p = 2; p <= RRQ_PMAX; p++) {
        const int n = (int)plist[p].size();
        if (n) CK(rrq_launch_precompute(p, ctx->d_tab[p], d_plists + start, n, in.node_off, in.xyz, in.nrm, pd, s.st));
        start += n;
    }
    CK(cudaMemcpyAsync(kappa, pd.kappa, sizeof(double) * in.npatch,
                       on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s.st));
    CK(cudaStreamSynchronize(s.st));
    return RRQ_OK;
}

extern "C" rrq_status rrq_csr_copy(rrq_ctx *ctx, const rrq_csr *csr, int64_t *rowptr, int32_t *col, double *val[4],
                                   int32_t dst_on_host) {
    if (!ctx || !csr) return RRQ_ERR_ARG;
    CK(cudaSetDevice(ctx->device));
    cudaMemcpyKind kind = dst_on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    // a batch view indexes the batch's col/val arrays: its entries start at rowptr[0]
    int64_t first = 0;
    if ((csr->kernel_mask & RRQ_CSR_VIEW) && csr->rowptr) {
        CK(cudaMemcpyAsync(&first, csr->rowptr, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    if (rowptr && csr->rowptr) CK(cudaMemcpyAsync(rowptr, csr->rowptr, sizeof(int64_t) * (csr->nrows + 1), kind, ctx->stream));
    if (col && csr->col && csr->nnz)
        CK(cudaMemcpyAsync(col, csr->col + first, sizeof(int32_t) * csr->nnz, kind, ctx->stream));
    for (int k = 0; k < 4; k++)
        if (val && val[k] && csr->val[k] && csr->nnz)
            CK(cudaMemcpyAsync(val[k], csr->val[k] + first, sizeof(double) * csr->nnz, kind, ctx->stream));
    if (rowptr && csr->rowptr && first != 0 && !dst_on_host) {
        k_rebase<<<(unsigned)((csr->nrows + 256) / 256), 256, 0, ctx->stream>>>(rowptr, csr->nrows + 1, first);
        CK(cudaGetLastError());
    }
    CK(cudaStreamSynchronize(ctx->stream));
    if (rowptr && csr->rowptr && first != 0 && dst_on_host)
        for (int64_t i = 0; i <= csr->nrows; i++) rowptr[i] -= first;
    return RRQ_OK;
}

extern "C" rrq_status rrq_csr_free(rrq_ctx *ctx, rrq_csr *csr) {
    if (!ctx || !csr || (csr->kernel_mask & RRQ_CSR_VIEW)) return RRQ_ERR_ARG;
    CK(cudaSetDevice(ctx->device));
    if (csr->rowptr) cudaFreeAsync(csr->rowptr, ctx->stream);
    if (csr->col) cudaFreeAsync(csr->col, ctx->stream);
    for (int k = 0; k < 4; k++)
        if (csr->val[k]) cudaFreeAsync(csr->val[k], ctx->stream);
    memset(csr, 0, sizeof(*csr));
    return RRQ_OK;
}

// ------------------------------------------------------------------------------------
// Apply (Sec. 5, eq. dlpsplitting): smooth direct sum over all nodes plus the correction
// row, fused in one kernel per tile of targets; and the correction alone (SpMV).
// ------------------------------------------------------------------------------------
namespace {

constexpr int APPLY_TILE = 256;
constexpr double kInv4Pi = 0.07957747154594767;

// Kernel values without the 1/(4 pi) factor: d = x_t - x_j, ri = 1/|d|, n = source
// normal, m = target normal (Sec. 1, eqs. slpdef-dprimelpdef).
template <int K, typename T>
__device__ __forceinline__ T kernel_value(T d0, T d1, T d2, T ri, T n0, T n1, T n2, T m0, T m1, T m2) {
    const T ri3 = ri * ri * ri;
    if (K == RRQ_S) return ri;
    if (K == RRQ_D) return (d0 * n0 + d1 * n1 + d2 * n2) * ri3;
    if (K == RRQ_SP) return -(d0 * m0 + d1 * m1 + d2 * m2) * ri3;
    const T dn = d0 * n0 + d1 * n1 + d2 * n2, dm = d0 * m0 + d1 * m1 + d2 * m2;
    return (m0 * n0 + m1 * n1 + m2 * n2) * ri3 - T(3) * dn * dm * ri3 * ri * ri;
}

// x as a (hi, lo) FP32 pair
__device__ __forceinline__ void split2(double x, float &h, float &l) {
    h = __double2float_rn(x);
    l = __double2float_rn(x - (double)h);
}

// |x_t - x_j|^2 in FP32 from (hi, lo) pairs; the differences of the hi parts are exact
// for close points, so close distances keep ~1e-7 relative accuracy
__device__ __forceinline__ float split_r2(const float th[3], const float tl[3], const float sh[3], const float sl[3],
                                          float d[3]) {
    for (int a = 0; a < 3; a++) d[a] = (th[a] - sh[a]) + (tl[a] - sl[a]);
    return fmaf(d[0], d[0], fmaf(d[1], d[1], d[2] * d[2]));
}

// Sum over the CSR row of target t of val[q] sigma[col[q]] (one warp; lanes stride the
// row, four independent loads in flight per lane), plus, when MIXED, the smooth terms of
// the row's nodes closer than r_c in FP64 (see rrq_apply).  Returns the warp sum in
// every lane.
template <int K, bool MIXED>
__device__ __forceinline__ double row_sum(int64_t a, int64_t b, const int32_t *__restrict__ col,
                                          const double *__restrict__ val, const double *__restrict__ sig,
                                          const double *__restrict__ xyz, const double *__restrict__ nrm,
                                          const double *__restrict__ wts, const double x[3], const double m[3],
                                          int64_t self, float rc2, int lane) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int64_t q = a + lane;
    for (; q + 96 < b; q += 128) {
        const double v0 = __ldcs(val + q), v1 = __ldcs(val + q + 32), v2 = __ldcs(val + q + 64),
                     v3 = __ldcs(val + q + 96);
        const int32_t c0 = __ldcs(col + q), c1 = __ldcs(col + q + 32), c2 = __ldcs(col + q + 64),
                      c3 = __ldcs(col + q + 96);
        s0 = fma(v0, __ldg(sig + c0), s0);
        s1 = fma(v1, __ldg(sig + c1), s1);
        s2 = fma(v2, __ldg(sig + c2), s2);
        s3 = fma(v3, __ldg(sig + c3), s3);
    }
    for (; q < b; q += 32) s0 = fma(__ldcs(val + q), __ldg(sig + __ldcs(col + q)), s0);
    double s = (s0 + s1) + (s2 + s3);
    if (MIXED) {
        float th[3], tl[3];
        for (int c = 0; c < 3; c++) split2(x[c], th[c], tl[c]);
        for (int64_t r = a + lane; r < b; r += 32) {
            const int32_t j = __ldg(col + r);
            if (j == self) continue;
            float sh[3], sl[3], d[3];
            for (int c = 0; c < 3; c++) split2(__ldg(xyz + 3 * j + c), sh[c], sl[c]);
            if (split_r2(th, tl, sh, sl, d) >= rc2) continue;
            const double d0 = x[0] - xyz[3 * j], d1 = x[1] - xyz[3 * j + 1], d2 = x[2] - xyz[3 * j + 2];
            const double ri = rsqrt(d0 * d0 + d1 * d1 + d2 * d2);
            const double kv = kernel_value<K, double>(d0, d1, d2, ri, nrm[3 * j], nrm[3 * j + 1], nrm[3 * j + 2], m[0],
                                                      m[1], m[2]);
            s = fma(kv, wts[j] * __ldg(sig + j) * kInv4Pi, s);
        }
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// One kernel per apply: the block's APPLY_TILE targets (one per thread) sum the smooth
// rule over all nodes, staged through shared memory tile by tile (the coincident node
// skipped); then its eight warps walk the block's CSR rows (row_sum) and every target
// adds its row.  FP64: every term in FP64.  MIXED: terms with |x_t - x_j| >= r_c in FP32
// (coordinates as (hi, lo) FP32 pairs, Kahan-compensated sums per source tile, FP64
// across tiles), the closer ones -- all in the target's row -- in FP64 with the row.
template <int K, bool MIXED>
__global__ void __launch_bounds__(APPLY_TILE) k_apply_fused(
    const double *__restrict__ xyz, const double *__restrict__ nrm, const double *__restrict__ wts,
    const double *__restrict__ sig, int64_t nnode, const double *__restrict__ txyz, const double *__restrict__ tnrm,
    const int64_t *__restrict__ tself, int64_t ntarg, const int64_t *__restrict__ rowptr,
    const int32_t *__restrict__ col, const double *__restrict__ val, float rc2, double *__restrict__ out) {
    constexpr bool kNeedN = (K == RRQ_D || K == RRQ_DP);
    typedef typename std::conditional<MIXED, float, double>::type R;
    __shared__ R sx[APPLY_TILE * 3], sxl[MIXED ? APPLY_TILE * 3 : 1], sn[kNeedN ? APPLY_TILE * 3 : 1], sw[APPLY_TILE];
    __shared__ double srow[APPLY_TILE];
    const int64_t t0 = (int64_t)blockIdx.x * APPLY_TILE;
    const int64_t t = t0 + threadIdx.x;
    const bool act = t < ntarg;
    double x[3] = {0, 0, 0}, m[3] = {0, 0, 0};
    int64_t self = -1;
    if (act) {
        for (int a = 0; a < 3; a++) { x[a] = txyz[3 * t + a]; m[a] = tnrm[3 * t + a]; }
        if (tself) self = tself[t];
    }
    float th[3], tl[3], mf[3];
    for (int a = 0; a < 3; a++) {
        split2(x[a], th[a], tl[a]);
        mf[a] = __double2float_rn(m[a]);
    }
    double acc = 0.0;
    for (int64_t base = 0; base < nnode; base += APPLY_TILE) {
        __syncthreads();
        const int64_t j = base + threadIdx.x;
        if (j < nnode) {
            for (int a = 0; a < 3; a++) {
                if (MIXED) {
                    float h, l;
                    split2(xyz[3 * j + a], h, l);
                    sx[3 * threadIdx.x + a] = h;
                    sxl[3 * threadIdx.x + a] = l;
                } else {
                    sx[3 * threadIdx.x + a] = (R)xyz[3 * j + a];
                }
                if (kNeedN) sn[3 * threadIdx.x + a] = (R)nrm[3 * j + a];
            }
            sw[threadIdx.x] = (R)(wts[j] * sig[j] * kInv4Pi);
        }
        __syncthreads();
        const int nt = (int)min((int64_t)APPLY_TILE, nnode - base);
        if (!act) continue;
        if (MIXED) {
            float s = 0.0f, c = 0.0f;
            for (int k = 0; k < nt; k++) {
                float d[3];
                const float r2 = split_r2(th, tl, (const float *)sx + 3 * k, (const float *)sxl + 3 * k, d);
                const float ri = rsqrtf(r2);
                const float n0 = kNeedN ? (float)sn[3 * k] : 0.f, n1 = kNeedN ? (float)sn[3 * k + 1] : 0.f,
                            n2 = kNeedN ? (float)sn[3 * k + 2] : 0.f;
                const float kv = kernel_value<K, float>(d[0], d[1], d[2], ri, n0, n1, n2, mf[0], mf[1], mf[2]);
                const float term = r2 < rc2 ? 0.0f : kv * (float)sw[k];  // close sources: FP64 with the row
                const float y = term - c;                               // Kahan step
                const float tt = s + y;
                c = (tt - s) - y;
                s = tt;
            }
            acc += (double)s - (double)c;
        } else {
            for (int k = 0; k < nt; k++) {
                if (base + k == self) continue;
                const double d0 = x[0] - (double)sx[3 * k], d1 = x[1] - (double)sx[3 * k + 1],
                             d2 = x[2] - (double)sx[3 * k + 2];
                const double ri = rsqrt(d0 * d0 + d1 * d1 + d2 * d2);
                const double n0 = kNeedN ? (double)sn[3 * k] : 0.0, n1 = kNeedN ? (double)sn[3 * k + 1] : 0.0,
                             n2 = kNeedN ? (double)sn[3 * k + 2] : 0.0;
                acc = fma(kernel_value<K, double>(d0, d1, d2, ri, n0, n1, n2, m[0], m[1], m[2]), (double)sw[k], acc);
            }
        }
    }
    if (val) {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int i = warp; i < APPLY_TILE; i += APPLY_TILE / 32) {
            const int64_t r = t0 + i;
            double v = 0.0;
            if (r < ntarg) {
                double xr[3] = {0, 0, 0}, mr[3] = {0, 0, 0};
                if (MIXED)
                    for (int a = 0; a < 3; a++) { xr[a] = txyz[3 * r + a]; mr[a] = tnrm[3 * r + a]; }
                v = row_sum<K, MIXED>(rowptr[r], rowptr[r + 1], col, val, sig, xyz, nrm, wts, xr, mr,
                                      (MIXED && tself) ? tself[r] : -1, rc2, lane);
            }
            if (lane == 0) srow[i] = v;
        }
        __syncthreads();
        acc += srow[threadIdx.x];
    }
    if (act) out[t] = acc;
}

// out[t] = (accumulate ? out[t] : 0) + sum over row t of val[q] sigma[col[q]]: one warp
// per row (row_sum).  HBM bound: 12 bytes per entry plus the row pointers.
__global__ void __launch_bounds__(256) k_spmv(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                                             const double *__restrict__ val, const double *__restrict__ sig,
                                             int64_t nrows, int accumulate, double *__restrict__ out) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= nrows) return;
    const double none[3] = {0, 0, 0};
    const double s = row_sum<RRQ_S, false>(rowptr[row], rowptr[row + 1], col, val, sig, nullptr, nullptr, nullptr,
                                           none, none, -1, 0.f, lane);
    if (lane == 0) out[row] = accumulate ? out[row] + s : s;
}

// smallest spread (largest node-to-node distance) over the patches, as ordered bits
__global__ void k_patch_spread(const int64_t *__restrict__ node_off, int npatch, const double *__restrict__ xyz,
                               unsigned long long *__restrict__ out) {
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= npatch) return;
    const int64_t a = node_off[P], b = node_off[P + 1];
    double m = 0.0;
    for (int64_t i = a; i < b; i++)
        for (int64_t k = i + 1; k < b; k++) {
            const double d0 = xyz[3 * i] - xyz[3 * k], d1 = xyz[3 * i + 1] - xyz[3 * k + 1], d2 = xyz[3 * i + 2] - xyz[3 * k + 2];
            m = fmax(m, d0 * d0 + d1 * d1 + d2 * d2);
        }
    atomicMin(out, (unsigned long long)__double_as_longlong(sqrt(m)));
}

template <bool MIXED>
cudaError_t launch_apply(int kernel, const Inputs &in, const double *sig, const rrq_csr *corr, const double *val,
                         float rc2, double *out, cudaStream_t st) {
    const unsigned grid = (unsigned)((in.ntarg + APPLY_TILE - 1) / APPLY_TILE);
    const int64_t *rp = corr ? corr->rowptr : nullptr;
    const int32_t *cl = corr ? corr->col : nullptr;
#define RRQ_APPLY_CASE(KK)                                                                                     \
    case KK:                                                                                                   \
        k_apply_fused<KK, MIXED><<<grid, APPLY_TILE, 0, st>>>(in.xyz, in.nrm, in.wts, sig, in.nnode, in.txyz, \
                                                              in.tnrm, in.tself, in.ntarg, rp, cl, val, rc2, out); \
        break;
    switch (kernel) {
        RRQ_APPLY_CASE(RRQ_S)
        RRQ_APPLY_CASE(RRQ_D)
        RRQ_APPLY_CASE(RRQ_SP)
        RRQ_APPLY_CASE(RRQ_DP)
        default: return cudaErrorInvalidValue;
    }
#undef RRQ_APPLY_CASE
    RRQ_COUNT_LAUNCH();
    return cudaGetLastError();
}

int kernel_slot(int32_t kernel) {
    return kernel == RRQ_S ? 0 : kernel == RRQ_D ? 1 : kernel == RRQ_SP ? 2 : kernel == RRQ_DP ? 3 : -1;
}

}  // namespace

extern "C" rrq_status rrq_apply(rrq_ctx *ctx, const rrq_surface *surf, const rrq_targets *targ, int32_t kernel,
                                const rrq_csr *corr, const double *density, double *out, const rrq_options *opt) {
    if (!ctx || !density || !out) return RRQ_ERR_ARG;
    const int kidx = kernel_slot(kernel);
    if (kidx < 0) return RRQ_ERR_ARG;
    rrq_options o;
    memset(&o, 0, sizeof(o));
    if (opt) o = *opt;
    if (o.precision != 0 && o.precision != 1) return RRQ_ERR_ARG;
    CK(cudaSetDevice(ctx->device));
    Scratch s;
    s.st = ctx->stream;
    Inputs in;
    rrq_status rs = prepare_inputs(ctx, s, surf, targ, o.inputs_on_host != 0, true, in);
    if (rs != RRQ_OK) return rs;
    const double *val = nullptr;
    if (corr) {
        if (corr->nrows != in.ntarg || !(corr->kernel_mask & (uint32_t)kernel)) return RRQ_ERR_ARG;
        val = corr->val[kidx];
    }
    cudaError_t err = cudaSuccess;
    const double *d_sig = upload(s, density, in.nnode, o.inputs_on_host != 0, &err);
    double *d_out = out;
    if (o.inputs_on_host) d_out = (double *)Scratch::alloc(&s, sizeof(double) * (in.ntarg > 0 ? in.ntarg : 1));
    if (err != cudaSuccess || s.failed) return RRQ_ERR_OOM;
    const bool mixed = o.precision == 1;
    if (mixed && !val) {
        snprintf(rrq_err_buf(), RRQ_ERR_LEN, "rrq_apply: precision = 1 needs the correction CSR");
        return RRQ_ERR_ARG;
    }
    float rc2 = 0.0f;
    if (mixed && in.ntarg > 0) {
        // r_c = eta x the smallest node spread of a patch
        unsigned long long *red = (unsigned long long *)Scratch::alloc(&s, sizeof(unsigned long long));
        if (!red) return RRQ_ERR_OOM;
        const unsigned long long init = 0x7FF0000000000000ULL;  // +inf
        CK(cudaMemcpyAsync(red, &init, sizeof(init), cudaMemcpyHostToDevice, s.st));
        k_patch_spread<<<(unsigned)((in.npatch + 127) / 128), 128, 0, s.st>>>(in.node_off, in.npatch, in.xyz, red);
        RRQ_COUNT_LAUNCH();
        CK(cudaGetLastError());
        unsigned long long h = 0;
        CK(cudaMemcpyAsync(&h, red, sizeof(h), cudaMemcpyDeviceToHost, s.st));
        CK(cudaStreamSynchronize(s.st));
        double rc;
        memcpy(&rc, &h, sizeof(rc));
        rc *= (o.eta > 0 ? o.eta : 1.0);
        rc2 = (float)(rc * rc);
    }
    if (in.ntarg > 0) {
        CK(cudaEventRecord(ctx->ev[0], s.st));
        if (mixed)
            CK(launch_apply<true>(kernel, in, d_sig, corr, val, rc2, d_out, s.st));
        else
            CK(launch_apply<false>(kernel, in, d_sig, corr, val, rc2, d_out, s.st));
        CK(cudaEventRecord(ctx->ev[1], s.st));
    }
    if (o.inputs_on_host && in.ntarg > 0)
        CK(cudaMemcpyAsync(out, d_out, sizeof(double) * in.ntarg, cudaMemcpyDeviceToHost, s.st));
    CK(cudaStreamSynchronize(s.st));
    if (in.ntarg > 0) {
        float ms = 0;
        cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]);
        ctx->diag.ms_apply_smooth = ms;
    }
    return RRQ_OK;
}

extern "C" rrq_status rrq_apply_correction(rrq_ctx *ctx, const rrq_csr *corr, int32_t kernel, const double *density,
                                           int64_t nnode, double *out, int32_t accumulate, int32_t on_host) {
    if (!ctx || !corr || !density || !out || nnode < 0) return RRQ_ERR_ARG;
    const int kidx = kernel_slot(kernel);
    if (kidx < 0 || !(corr->kernel_mask & (uint32_t)kernel) || !corr->val[kidx] || corr->nrows < 0) return RRQ_ERR_ARG;
    if (corr->nrows > 0 && (!corr->rowptr || !corr->col)) return RRQ_ERR_ARG;
    CK(cudaSetDevice(ctx->device));
    Scratch s;
    s.st = ctx->stream;
    cudaError_t err = cudaSuccess;
    const double *d_sig = upload(s, density, (size_t)nnode, on_host != 0, &err);
    double *d_out = out;
    if (on_host) {
        d_out = (double *)Scratch::alloc(&s, sizeof(double) * (corr->nrows > 0 ? corr->nrows : 1));
        if (d_out && accumulate && corr->nrows > 0)
            err = cudaMemcpyAsync(d_out, out, sizeof(double) * corr->nrows, cudaMemcpyHostToDevice, s.st);
    }
    if (err != cudaSuccess || s.failed) return RRQ_ERR_OOM;
    if (corr->nrows > 0) {
        CK(cudaEventRecord(ctx->ev[0], s.st));
        k_spmv<<<(unsigned)((corr->nrows * 32 + 255) / 256), 256, 0, s.st>>>(corr->rowptr, corr->col,
                                                                              corr->val[kidx], d_sig, corr->nrows,
                                                                              accumulate, d_out);
        RRQ_COUNT_LAUNCH();
        CK(cudaGetLastError());
        CK(cudaEventRecord(ctx->ev[1], s.st));
        if (on_host) CK(cudaMemcpyAsync(out, d_out, sizeof(double) * corr->nrows, cudaMemcpyDeviceToHost, s.st));
    }
    CK(cudaStreamSynchronize(s.st));
    if (corr->nrows > 0) {
        float ms = 0;
        cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]);
        ctx->diag.ms_apply_spmv = ms;
    }
    return RRQ_OK;
}

// ------------------------------------------------------------------------------------
// FMA throughput microbenchmark (roofline denominator for the ALU-bound build).
// ------------------------------------------------------------------------------------
namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T *out, int iters, T a, T b) {
    T x0 = (T)threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < 8; u++) {
            x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
            x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
        }
    }
    T s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
    if (s == (T)-1.2345) out[0] = s;  // keeps the chains alive
}

template <typename T>
rrq_status fma_peak(rrq_ctx *ctx, double *tflops) {
    int nsm = 0;
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
    T *d = nullptr;
    CK(cudaMallocAsync(&d, sizeof(T), ctx->stream));
    const int blocks = nsm * 8, threads = 256, iters = 4096;
    k_fma_peak<T><<<blocks, threads, 0, ctx->stream>>>(d, 64, (T)0.999, (T)0.001);  // warm-up
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, ctx->stream);
    k_fma_peak<T><<<blocks, threads, 0, ctx->stream>>>(d, iters, (T)0.999, (T)0.001);
    cudaEventRecord(e1, ctx->stream);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(d, ctx->stream);
    if (e != cudaSuccess) { set_err("peak kernel", e); return RRQ_ERR_CUDA; }
    double flops = 2.0 * 64.0 * iters * (double)blocks * threads;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return RRQ_OK;
}

}  // namespace

extern "C" rrq_status rrq_measure_fma_peak(rrq_ctx *ctx, int32_t fp32, double *tflops) {
    if (!ctx || !tflops) return RRQ_ERR_ARG;
    CK(cudaSetDevice(ctx->device));
    return fp32 ? fma_peak<float>(ctx, tflops) : fma_peak<double>(ctx, tflops);
}

// ------------------------------------------------------------------------------------
// Allocation-free variant of rrq_build_corrections.  All scratch (order tables, patch
// data, near list, pair items, counters) lives in one file-scope device array that every
// GPU loading this library keeps until the process exits; the caller provides the CSR
// output buffers.  No cudaMalloc / cudaMallocAsync / cudaFree is called.
// ------------------------------------------------------------------------------------
namespace {

static __device__ __align__(256) unsigned char g_rrq_static_scratch[RRQ_STATIC_SCRATCH_BYTES];

struct StaticArena {
    unsigned char *base;
    size_t used, cap;
    bool failed;
    size_t wanted;
    static void *alloc(void *self, size_t bytes) {
        StaticArena *a = static_cast<StaticArena *>(self);
        size_t off = (a->used + 255) & ~(size_t)255;
        if (bytes == 0) bytes = 16;
        if (off + bytes > a->cap) {
            a->failed = true;
            a->wanted = off + bytes;
            return nullptr;
        }
        a->used = off + bytes;
        return a->base + off;
    }
};

}  // namespace

extern "C" rrq_status rrq_build_corrections_static(rrq_ctx *ctx, const rrq_surface *surf, const rrq_targets *targ,
                                                   uint32_t kernel_mask, const rrq_options *opt, int64_t *rowptr,
                                                   int32_t *col, double *val[4], int64_t capacity, int64_t *nnz_out,
                                                   int64_t *npairs_out) {
    if (!ctx || !rowptr || !col || !val || capacity < 0) return RRQ_ERR_ARG;
    if (kernel_mask == 0 || (kernel_mask & ~15u)) return RRQ_ERR_ARG;
    for (int k = 0; k < 4; k++)
        if ((kernel_mask & (1u << k)) && !val[k]) return RRQ_ERR_ARG;
    rrq_options o;
    memset(&o, 0, sizeof(o));
    if (opt) o = *opt;
    if (o.inputs_on_host) {
        snprintf(rrq_err_buf(), RRQ_ERR_LEN, "rrq_build_corrections_static: inputs must be device pointers");
        return RRQ_ERR_ARG;
    }
    if (o.precision != 0) {
        snprintf(rrq_err_buf(), RRQ_ERR_LEN, "rrq_build_corrections_static: FP64 only (precision = 0)");
        return RRQ_ERR_UNSUPPORTED;
    }
    if (o.translation != 0) {
        snprintf(rrq_err_buf(), RRQ_ERR_LEN, "rrq_build_corrections_static: direct translation only (translation = 0)");
        return RRQ_ERR_UNSUPPORTED;
    }
    const double eta = o.eta > 0 ? o.eta : 1.0;
    const int newton_max = o.newton_max > 0 ? o.newton_max : 30;
    CK(cudaSetDevice(ctx->device));
    // device address of the array on the current device, looked up on every call (no
    // allocation; valid for the device's current context)
    void *scratch_base = nullptr;
    CK(cudaGetSymbolAddress(&scratch_base, g_rrq_static_scratch));
    memset(&ctx->diag, 0, sizeof(ctx->diag));
    rrq_launch_counter() = 0;
    StaticArena ar;
    ar.base = static_cast<unsigned char *>(scratch_base);
    ar.used = 0;
    ar.cap = RRQ_STATIC_SCRATCH_BYTES;
    ar.failed = false;
    ar.wanted = 0;
    cudaStream_t st = ctx->stream;
    // inputs (device pointers): sizes and orders read back to the host
    if (!surf || surf->npatch < 1 || !surf->order || !surf->node_off || !surf->xyz || !surf->nrm || !surf->wts)
        return RRQ_ERR_ARG;
    if (!targ || targ->ntarg < 0 || (targ->ntarg > 0 && (!targ->xyz || !targ->nrm))) return RRQ_ERR_ARG;
    const int npatch = surf->npatch;
    const int64_t ntarg = targ->ntarg;
    std::vector<int32_t> h_order(npatch);
    std::vector<int64_t> h_node_off(npatch + 1);
    CK(cudaMemcpyAsync(h_order.data(), surf->order, sizeof(int32_t) * npatch, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(h_node_off.data(), surf->node_off, sizeof(int64_t) * (npatch + 1), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h_node_off[0] != 0) return RRQ_ERR_ARG;
    std::vector<std::vector<int32_t>> plist(RRQ_PMAX + 1);
    int pmax = 0;
    for (int P = 0; P < npatch; P++) {
        int p = h_order[P];
        if (p < 2 || p > RRQ_PMAX || !surf->ref_uv[p]) return RRQ_ERR_ARG;
        if (h_node_off[P + 1] - h_node_off[P] != np_of(p)) return RRQ_ERR_ARG;
        if (o.ptilde != 0 && o.ptilde != 2 * p) return RRQ_ERR_UNSUPPORTED;
        plist[p].push_back(P);
        pmax = std::max(pmax, p);
    }
    // order tables, built on the host and copied into the arena
    OrderTables *tabs[RRQ_PMAX + 1] = {nullptr};
    std::vector<OrderTables> htab(RRQ_PMAX + 1);
    for (int p = 2; p <= RRQ_PMAX; p++)
        if (!plist[p].empty()) {
            if (rrq_host_order_tables(p, 2 * p, o.rho0, surf->ref_uv[p], &htab[p])) return RRQ_ERR_ARG;
            tabs[p] = (OrderTables *)StaticArena::alloc(&ar, sizeof(OrderTables));
            if (!tabs[p]) break;
            CK(cudaMemcpyAsync(tabs[p], &htab[p], sizeof(OrderTables), cudaMemcpyHostToDevice, st));
        }
    const size_t NPc = npatch;
    PatchData pd{};
    pd.npatch = npatch;
    pd.pmax = pmax;
    pd.frame = (double *)StaticArena::alloc(&ar, sizeof(double) * NPc * PD_FRAME);
    pd.bounds = (double *)StaticArena::alloc(&ar, sizeof(double) * NPc * PD_BOUNDS);
    pd.ynode = (double *)StaticArena::alloc(&ar, sizeof(double) * NPc * pd_ynode(pd.pmax));
    pd.xm = (double *)StaticArena::alloc(&ar, sizeof(double) * NPc * pd_ynode(pd.pmax));
    pd.ea = (double *)StaticArena::alloc(&ar, sizeof(double) * NPc * pd_ea(pd.pmax));
    pd.ey = (double *)StaticArena::alloc(&ar, sizeof(double) * NPc * pd_ey(pd.pmax));
    pd.et = (double *)StaticArena::alloc(&ar, sizeof(double) * NPc * pd_ey(pd.pmax));
    pd.eyu = (double *)StaticArena::alloc(&ar, sizeof(double) * NPc * pd_eyu(pd.pmax));
    pd.eg = (cd *)StaticArena::alloc(&ar, sizeof(cd) * NPc * pd_eg(pd.pmax));
    pd.eh = (cd *)StaticArena::alloc(&ar, sizeof(cd) * NPc * pd_eg(pd.pmax));
    pd.eg2 = nullptr;
    pd.eh2 = nullptr;
    pd.XD = (double *)StaticArena::alloc(&ar, sizeof(double) * NPc * pd_X(pd.pmax));
    pd.XSp = (double *)StaticArena::alloc(&ar, sizeof(double) * NPc * pd_X(pd.pmax));
    pd.XS2 = (double *)StaticArena::alloc(&ar, sizeof(double) * NPc * pd_X(pd.pmax));
    pd.XS1 = (double *)StaticArena::alloc(&ar, sizeof(double) * NPc * pd_XS1(pd.pmax));
    pd.lu = pd_lu(pd.pmax) ? (double *)StaticArena::alloc(&ar, sizeof(double) * NPc * pd_lu(pd.pmax)) : nullptr;
    pd.status = (int *)StaticArena::alloc(&ar, sizeof(int) * NPc);
    pd.kappa = (double *)StaticArena::alloc(&ar, sizeof(double) * NPc);
    int32_t *d_plists = (int32_t *)StaticArena::alloc(&ar, sizeof(int32_t) * npatch);
    int32_t *d_rank = (int32_t *)StaticArena::alloc(&ar, sizeof(int32_t) * npatch);
    BuildCounters *d_cnt = (BuildCounters *)StaticArena::alloc(&ar, sizeof(BuildCounters));
    unsigned *d_flag = (unsigned *)StaticArena::alloc(&ar, sizeof(unsigned));
    if (ar.failed) {
        snprintf(rrq_err_buf(), RRQ_ERR_LEN, "rrq_build_corrections_static: needs more than %zu bytes of scratch (maximum %zu)",
                 ar.wanted, (size_t)RRQ_STATIC_SCRATCH_BYTES);
        return RRQ_ERR_ARG;
    }
    {
        const int64_t nnode = h_node_off[npatch];
        const double *arrays[5] = {surf->xyz, surf->nrm, surf->wts, targ->xyz, targ->nrm};
        const int64_t sizes[5] = {3 * nnode, 3 * nnode, nnode, 3 * ntarg, 3 * ntarg};
        rrq_status rs = check_finite(st, d_flag, arrays, sizes, kInputNames, 5);
        if (rs != RRQ_OK) return rs;
    }
    std::vector<int32_t> rank(npatch), order_major;
    order_major.reserve(npatch);
    for (int p = 2; p <= RRQ_PMAX; p++)
        for (int32_t P : plist[p]) order_major.push_back(P);
    for (int r = 0; r < npatch; r++) rank[order_major[r]] = r;
    CK(cudaMemcpyAsync(d_plists, order_major.data(), sizeof(int32_t) * npatch, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_rank, rank.data(), sizeof(int32_t) * npatch, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(d_cnt, 0, sizeof(BuildCounters), st));
    {
        int start = 0;
        for (int p = 2; p <= RRQ_PMAX; p++) {
            int n = (int)plist[p].size();
            if (n) CK(rrq_launch_precompute(p, tabs[p], d_plists + start, n, surf->node_off, surf->xyz, surf->nrm, pd, st));
            start += n;
        }
    }
    NearBuffers nb;
    cudaError_t e = rrq_near_build(pd.bounds, npatch, surf->node_off, targ->xyz, targ->self_node, ntarg, eta,
                                   &StaticArena::alloc, &ar, &nb, st);
    PairItem *items = nullptr;
    int64_t *roff = nullptr;
    if (e == cudaSuccess && !ar.failed)
        e = rrq_items_build(&nb, ntarg, surf->order, d_rank, npatch, &StaticArena::alloc, &ar, rowptr, &items, &roff, st);
    if (ar.failed) {
        cudaStreamSynchronize(st);
        snprintf(rrq_err_buf(), RRQ_ERR_LEN, "rrq_build_corrections_static: needs more than %zu bytes of scratch (maximum %zu)",
                 ar.wanted, (size_t)RRQ_STATIC_SCRATCH_BYTES);
        return RRQ_ERR_ARG;
    }
    CK(e);
    int64_t nnz = 0;
    std::vector<int64_t> h_roff(npatch + 1);
    std::vector<int> h_status(npatch);
    CK(cudaMemcpyAsync(&nnz, rowptr + ntarg, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(h_roff.data(), roff, sizeof(int64_t) * (npatch + 1), cudaMemcpyDeviceToHost, st));
    std::vector<double> h_kappa(npatch);
    CK(cudaMemcpyAsync(h_status.data(), pd.status, sizeof(int) * npatch, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(h_kappa.data(), pd.kappa, sizeof(double) * npatch, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const double kappa_max = *std::max_element(h_kappa.begin(), h_kappa.end());
    if (nnz_out) *nnz_out = nnz;
    if (npairs_out) *npairs_out = nb.npairs;
    for (int P = 0; P < npatch; P++)
        if (h_status[P]) return RRQ_ERR_DEGENERATE;
    if (nnz > capacity) {
        snprintf(rrq_err_buf(), RRQ_ERR_LEN, "rrq_build_corrections_static: %lld entries exceed the output capacity %lld",
                 (long long)nnz, (long long)capacity);
        return RRQ_ERR_ARG;
    }
    pd.roots = (EdgeRoot *)StaticArena::alloc(&ar, sizeof(EdgeRoot) * 3 * (nb.npairs > 0 ? nb.npairs : 1));
    pd.uside = (int8_t *)StaticArena::alloc(&ar, sizeof(int8_t) * (nb.npairs > 0 ? nb.npairs : 1));
    if (ar.failed) {
        snprintf(rrq_err_buf(), RRQ_ERR_LEN, "rrq_build_corrections_static: needs more than %zu bytes of scratch (maximum %zu)",
                 ar.wanted, (size_t)RRQ_STATIC_SCRATCH_BYTES);
        return RRQ_ERR_ARG;
    }
    {
        int start = 0;
        for (int p = 2; p <= RRQ_PMAX; p++) {
            int n = (int)plist[p].size();
            if (n) {
                int64_t i0 = h_roff[start], i1 = h_roff[start + n];
                PatchData pdo = pd;
                pdo.roots = pd.roots + 3 * i0;
                pdo.uside = pd.uside + i0;
                const PairArgs pa = {tabs[p], items + i0, i1 - i0, pdo, surf->node_off, surf->xyz, surf->nrm,
                                     surf->wts, targ->xyz, targ->nrm, targ->self_node, kernel_mask, newton_max,
                                     {(kernel_mask & RRQ_S) ? val[0] : nullptr, (kernel_mask & RRQ_D) ? val[1] : nullptr,
                                      (kernel_mask & RRQ_SP) ? val[2] : nullptr,
                                      (kernel_mask & RRQ_DP) ? val[3] : nullptr},
                                     col, d_cnt};
                CK(rrq_launch_pairs(p, false, pa, PairShape{0, 0, nullptr}, st));
            }
            start += n;
        }
    }
    BuildCounters hc;
    CK(cudaMemcpyAsync(&hc, d_cnt, sizeof(hc), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    ctx->diag.npairs = nb.npairs;
    ctx->diag.newton_fail = (int64_t)hc.newton_fail;
    ctx->diag.on_edge = (int64_t)hc.on_edge;
    ctx->diag.u_poor = (int64_t)hc.u_poor;
    ctx->diag.ssq_edges = (int64_t)hc.ssq_edges;
    ctx->diag.far_edges = (int64_t)hc.far_edges;
    ctx->diag.kernel_launches = rrq_launch_counter();
    ctx->diag.kappa_max = kappa_max;
    return hc.newton_fail > 0 ? RRQ_WARN_ROOTFIND : RRQ_OK;
}
