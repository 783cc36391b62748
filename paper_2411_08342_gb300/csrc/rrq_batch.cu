// Batched build of many surfaces (include/rrq.h, rrq_batch_*).  The paper builds one
// surface at a time; here the surfaces of a batch are concatenated (patches, nodes,
// targets), each keeps its own near list, and the value computation of the whole
// batch -- per-patch precompute of every order, then per order one root kernel and
// one persistent pair kernel over the pairs of all surfaces -- is recorded once as a
// CUDA graph and replayed by rrq_batch_execute.  The per-pair arithmetic is the same
// as in rrq_build_corrections (same kernels); only the CSR columns are made local to
// each surface (PatchData.col_off).
#include <algorithm>
#include <chrono>

#include "rrq_host.h"

struct rrq_batch {
    int device = 0;
    int32_t nsurf = 0;
    uint32_t mask = 0;
    bool mixed = false;
    int newton_max = 30;
    int npatch = 0;
    int64_t nrows = 0, nnode = 0, nnz = 0, npairs = 0;
    std::vector<int64_t> row_start, node_start, patch_start, nnz_start, pair_count;
    std::vector<void *> mem;  // owned device allocations
    int32_t *order = nullptr, *plists = nullptr;
    int64_t *node_off = nullptr, *col_off = nullptr, *tself = nullptr, *rowptr = nullptr;
    double *xyz = nullptr, *nrm = nullptr, *wts = nullptr, *txyz = nullptr, *tnrm = nullptr;
    int32_t *col = nullptr;
    double *val[4] = {nullptr, nullptr, nullptr, nullptr};
    PairItem *items = nullptr;
    EdgeRoot *roots = nullptr;
    int8_t *uside = nullptr;
    BuildCounters *cnt = nullptr;
    unsigned long long *tile_ctr = nullptr;  // [RRQ_PMAX + 1]
    PatchData pd{};
    OrderTables *tab[RRQ_PMAX + 1] = {};
    int pl_start[RRQ_PMAX + 1] = {}, pl_count[RRQ_PMAX + 1] = {};
    int64_t it0[RRQ_PMAX + 1] = {}, it1[RRQ_PMAX + 1] = {};
    int tile[RRQ_PMAX + 1] = {}, persistent[RRQ_PMAX + 1] = {};
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_kernels = 0;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    double ms_create = 0, ms_autotune = 0, ms_last = 0;
    double kappa_max = 0;  // max over all patches of kappa_1(A)

    void *alloc(size_t bytes) {
        void *p = nullptr;
        if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        mem.push_back(p);
        return p;
    }
    static void *alloc_cb(void *self, size_t bytes) { return static_cast<rrq_batch *>(self)->alloc(bytes); }
    ~rrq_batch() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (void *p : mem) cudaFree(p);
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
        if (cap) cudaStreamDestroy(cap);
    }
};

namespace {

// Global node id of a target that is a node of its own surface, else -1.
__global__ void k_self_global(const int64_t *__restrict__ src, int64_t n, int64_t nnode_s, int64_t node0,
                              int64_t *__restrict__ dst) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int64_t s = src ? src[t] : -1;
    dst[t] = (s >= 0 && s < nnode_s) ? s + node0 : -1;
}

// Append one surface's near list to the batch list (patch ids made global).
__global__ void k_near_merge(const int64_t *__restrict__ poff, const int32_t *__restrict__ pairs, int64_t ntarg,
                             int64_t npairs, int64_t pair0, int32_t patch0, int64_t *__restrict__ gpoff,
                             int32_t *__restrict__ gpairs) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ntarg) gpoff[i] = poff[i] + pair0;
    if (i < npairs) gpairs[pair0 + i] = pairs[i] + patch0;
}

unsigned blocks(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

template <typename T>
cudaError_t put(T *dst, const T *src, size_t n, bool on_host, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    return cudaMemcpyAsync(dst, src, sizeof(T) * n, on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st);
}

PairArgs pair_args(const rrq_batch *b, int p) {
    PatchData pdo = b->pd;
    pdo.roots = b->roots + 3 * b->it0[p];
    pdo.uside = b->uside + b->it0[p];
    return PairArgs{b->tab[p], b->items + b->it0[p], b->it1[p] - b->it0[p], pdo, b->node_off, b->xyz, b->nrm, b->wts,
                    b->txyz, b->tnrm, b->tself, b->mask, b->newton_max, {b->val[0], b->val[1], b->val[2], b->val[3]},
                    b->col, b->cnt};
}

// Time every compiled tile size and both schedules of order p on a sample of its pairs
// (the sample's values are recomputed by every execution).
cudaError_t autotune_order(rrq_batch *b, int p, cudaStream_t st) {
    int tiles[4];
    const int nt = rrq_pair_tiles(p, tiles);
    PairArgs a = pair_args(b, p);
    a.nitems = std::min<int64_t>(a.nitems, 65536);
    float best = 1e30f;
    for (int i = 0; i < nt; i++)
        for (int pers = 1; pers >= 0; pers--) {
            const PairShape sh{tiles[i], pers, b->tile_ctr + p};
            float ms = 0;
            for (int rep = 0; rep < 2; rep++) {
                cudaError_t e = cudaEventRecord(b->ev[0], st);
                if (e == cudaSuccess) e = rrq_launch_pairs(p, b->mixed, a, sh, st);
                if (e == cudaSuccess) e = cudaEventRecord(b->ev[1], st);
                if (e == cudaSuccess) e = cudaEventSynchronize(b->ev[1]);
                if (e != cudaSuccess) return e;
                cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]);
            }
            if (ms < best) {
                best = ms;
                b->tile[p] = tiles[i];
                b->persistent[p] = pers;
            }
        }
    return cudaSuccess;
}

rrq_status create_impl(rrq_ctx *ctx, rrq_batch *b, int32_t nsurf, const rrq_surface *surfs, const rrq_targets *targs,
                       uint32_t kernel_mask, const rrq_options &o, uint32_t flags) {
    const bool on_host = o.inputs_on_host != 0;
    cudaStream_t st = ctx->stream;
    Scratch s;
    s.st = st;
    // inputs of every surface (device views) and the batch layout
    std::vector<Inputs> in(nsurf);
    b->row_start.assign(nsurf + 1, 0);
    b->node_start.assign(nsurf + 1, 0);
    b->patch_start.assign(nsurf + 1, 0);
    const double *ref[RRQ_PMAX + 1] = {};
    for (int k = 0; k < nsurf; k++) {
        rrq_status rs = prepare_inputs(ctx, s, &surfs[k], &targs[k], on_host, true, in[k]);
        if (rs != RRQ_OK) return rs;
        if (o.ptilde != 0)
            for (int P = 0; P < in[k].npatch; P++)
                if (o.ptilde != 2 * in[k].h_order[P]) return RRQ_ERR_UNSUPPORTED;
        for (int P = 0; P < in[k].npatch; P++) {
            const int p = in[k].h_order[P];
            const double *r = surfs[k].ref_uv[p];
            if (!ref[p]) ref[p] = r;
            else if (ref[p] != r && memcmp(ref[p], r, sizeof(double) * 2 * np_of(p)) != 0) {
                snprintf(rrq_err_buf(), RRQ_ERR_LEN, "rrq_batch_create: surfaces use different reference nodes for p = %d",
                         p);
                return RRQ_ERR_ARG;
            }
        }
        b->row_start[k + 1] = b->row_start[k] + in[k].ntarg;
        b->node_start[k + 1] = b->node_start[k] + in[k].nnode;
        b->patch_start[k + 1] = b->patch_start[k] + in[k].npatch;
    }
    b->nrows = b->row_start[nsurf];
    b->nnode = b->node_start[nsurf];
    if (b->patch_start[nsurf] >= INT32_MAX || b->nnode >= INT32_MAX) return RRQ_ERR_ARG;
    b->npatch = (int)b->patch_start[nsurf];
    const size_t NP = b->npatch;
    for (int p = 2; p <= RRQ_PMAX; p++)
        if (ref[p]) {
            rrq_status rs = order_tables(ctx, p, ref[p], o.rho0);
            if (rs != RRQ_OK) return rs;
            b->tab[p] = ctx->d_tab[p];
        }
    // batch-owned copies of the inputs
    b->order = (int32_t *)b->alloc(sizeof(int32_t) * NP);
    b->node_off = (int64_t *)b->alloc(sizeof(int64_t) * (NP + 1));
    b->col_off = (int64_t *)b->alloc(sizeof(int64_t) * NP);
    b->xyz = (double *)b->alloc(sizeof(double) * 3 * b->nnode);
    b->nrm = (double *)b->alloc(sizeof(double) * 3 * b->nnode);
    b->wts = (double *)b->alloc(sizeof(double) * b->nnode);
    b->txyz = (double *)b->alloc(sizeof(double) * 3 * b->nrows);
    b->tnrm = (double *)b->alloc(sizeof(double) * 3 * b->nrows);
    b->tself = (int64_t *)b->alloc(sizeof(int64_t) * b->nrows);
    if (!b->order || !b->node_off || !b->col_off || !b->xyz || !b->nrm || !b->wts || !b->txyz || !b->tnrm || !b->tself)
        return RRQ_ERR_OOM;
    std::vector<int32_t> h_order(NP);
    std::vector<int64_t> h_node_off(NP + 1), h_col_off(NP);
    for (int k = 0; k < nsurf; k++)
        for (int P = 0; P < in[k].npatch; P++) {
            const size_t g = b->patch_start[k] + P;
            h_order[g] = in[k].h_order[P];
            h_node_off[g] = in[k].h_node_off[P] + b->node_start[k];
            h_col_off[g] = in[k].h_node_off[P];
        }
    h_node_off[NP] = b->nnode;
    CK(cudaMemcpyAsync(b->order, h_order.data(), sizeof(int32_t) * NP, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(b->node_off, h_node_off.data(), sizeof(int64_t) * (NP + 1), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(b->col_off, h_col_off.data(), sizeof(int64_t) * NP, cudaMemcpyHostToDevice, st));
    for (int k = 0; k < nsurf; k++) {
        // prepare_inputs has already moved host inputs to the device
        const int64_t n0 = b->node_start[k], r0 = b->row_start[k];
        CK(put(b->xyz + 3 * n0, in[k].xyz, 3 * in[k].nnode, false, st));
        CK(put(b->nrm + 3 * n0, in[k].nrm, 3 * in[k].nnode, false, st));
        CK(put(b->wts + n0, in[k].wts, in[k].nnode, false, st));
        CK(put(b->txyz + 3 * r0, in[k].txyz, 3 * in[k].ntarg, false, st));
        CK(put(b->tnrm + 3 * r0, in[k].tnrm, 3 * in[k].ntarg, false, st));
        if (in[k].ntarg > 0) {
            k_self_global<<<blocks(in[k].ntarg, 256), 256, 0, st>>>(in[k].tself, in[k].ntarg, in[k].nnode, n0,
                                                                    b->tself + r0);
            CK(cudaGetLastError());
        }
    }
    // per-patch data and the order-major patch lists
    PatchData &pd = b->pd;
    pd.npatch = b->npatch;
    pd.pmax = 0;
    std::vector<int32_t> order_major;
    order_major.reserve(NP);
    std::vector<int32_t> rank(NP);
    for (int p = 2; p <= RRQ_PMAX; p++) {
        b->pl_start[p] = (int)order_major.size();
        for (size_t P = 0; P < NP; P++)
            if (h_order[P] == p) order_major.push_back((int32_t)P);
        b->pl_count[p] = (int)order_major.size() - b->pl_start[p];
        if (b->pl_count[p]) pd.pmax = p;
    }
    for (size_t r = 0; r < NP; r++) rank[order_major[r]] = (int32_t)r;
    pd.frame = (double *)b->alloc(sizeof(double) * NP * PD_FRAME);
    pd.bounds = (double *)b->alloc(sizeof(double) * NP * PD_BOUNDS);
    pd.ynode = (double *)b->alloc(sizeof(double) * NP * pd_ynode(pd.pmax));
    pd.xm = (double *)b->alloc(sizeof(double) * NP * pd_ynode(pd.pmax));
    pd.ea = (double *)b->alloc(sizeof(double) * NP * pd_ea(pd.pmax));
    pd.ey = (double *)b->alloc(sizeof(double) * NP * pd_ey(pd.pmax));
    pd.et = (double *)b->alloc(sizeof(double) * NP * pd_ey(pd.pmax));
    pd.eyu = (double *)b->alloc(sizeof(double) * NP * pd_eyu(pd.pmax));
    pd.eg = (cd *)b->alloc(sizeof(cd) * NP * pd_eg(pd.pmax));
    pd.eh = (cd *)b->alloc(sizeof(cd) * NP * pd_eg(pd.pmax));
    pd.eg2 = b->mixed ? (float4 *)b->alloc(sizeof(float4) * NP * pd_eg(pd.pmax)) : nullptr;
    pd.eh2 = b->mixed ? (float4 *)b->alloc(sizeof(float4) * NP * pd_eg(pd.pmax)) : nullptr;
    if (b->mixed) {
        pd.XD2 = (float2 *)b->alloc(sizeof(float2) * NP * pd_X(pd.pmax));
        pd.XSp2 = (float2 *)b->alloc(sizeof(float2) * NP * pd_X(pd.pmax));
        pd.XS22 = (float2 *)b->alloc(sizeof(float2) * NP * pd_X(pd.pmax));
        pd.XS12 = (float2 *)b->alloc(sizeof(float2) * NP * pd_XS1(pd.pmax));
        if (!pd.XD2 || !pd.XSp2 || !pd.XS22 || !pd.XS12) return RRQ_ERR_OOM;
    }
    pd.XD = (double *)b->alloc(sizeof(double) * NP * pd_X(pd.pmax));
    pd.XSp = (double *)b->alloc(sizeof(double) * NP * pd_X(pd.pmax));
    pd.XS2 = (double *)b->alloc(sizeof(double) * NP * pd_X(pd.pmax));
    pd.XS1 = (double *)b->alloc(sizeof(double) * NP * pd_XS1(pd.pmax));
    pd.lu = pd_lu(pd.pmax) ? (double *)b->alloc(sizeof(double) * NP * pd_lu(pd.pmax)) : nullptr;
    pd.status = (int *)b->alloc(sizeof(int) * NP);
    pd.kappa = (double *)b->alloc(sizeof(double) * NP);
    pd.col_off = b->col_off;
    b->plists = (int32_t *)b->alloc(sizeof(int32_t) * NP);
    int32_t *d_rank = (int32_t *)Scratch::alloc(&s, sizeof(int32_t) * NP);
    b->cnt = (BuildCounters *)b->alloc(sizeof(BuildCounters));
    b->tile_ctr = (unsigned long long *)b->alloc(sizeof(unsigned long long) * (RRQ_PMAX + 1));
    if (!pd.frame || !pd.bounds || !pd.ynode || !pd.xm || !pd.ea || !pd.ey || !pd.et || !pd.eyu || !pd.eg || !pd.eh ||
        (b->mixed && (!pd.eg2 || !pd.eh2)) || !pd.XD || !pd.XSp || !pd.XS2 || !pd.XS1 || !pd.status || !pd.kappa || !b->plists ||
        !d_rank || !b->cnt || !b->tile_ctr)
        return RRQ_ERR_OOM;
    CK(cudaMemcpyAsync(b->plists, order_major.data(), sizeof(int32_t) * NP, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_rank, rank.data(), sizeof(int32_t) * NP, cudaMemcpyHostToDevice, st));
    // the patch bounds feed the near lists: precompute once here (the graph repeats it)
    for (int p = 2; p <= RRQ_PMAX; p++)
        if (b->pl_count[p])
            CK(rrq_launch_precompute(p, b->tab[p], b->plists + b->pl_start[p], b->pl_count[p], b->node_off, b->xyz,
                                     b->nrm, pd, st));
    std::vector<int> h_status(NP);
    std::vector<double> h_kappa(NP);
    CK(cudaMemcpyAsync(h_status.data(), pd.status, sizeof(int) * NP, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(h_kappa.data(), pd.kappa, sizeof(double) * NP, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    b->kappa_max = *std::max_element(h_kappa.begin(), h_kappa.end());
    for (size_t P = 0; P < NP; P++)
        if (h_status[P]) return RRQ_ERR_DEGENERATE;
    // near list of every surface, merged into one list over the batch
    const double eta = o.eta > 0 ? o.eta : 1.0;
    std::vector<NearBuffers> nbs(nsurf);
    b->pair_count.assign(nsurf, 0);
    int64_t npairs = 0;
    for (int k = 0; k < nsurf; k++) {
        const int64_t P0 = b->patch_start[k], r0 = b->row_start[k];
        CK(rrq_near_build(pd.bounds + P0 * PD_BOUNDS, in[k].npatch, b->node_off + P0, b->txyz + 3 * r0, b->tself + r0,
                          in[k].ntarg, eta, &Scratch::alloc, &s, &nbs[k], st));
        b->pair_count[k] = nbs[k].npairs;
        npairs += nbs[k].npairs;
    }
    if (s.failed) return RRQ_ERR_OOM;
    b->npairs = npairs;
    NearBuffers g;
    g.npairs = npairs;
    g.poff = (int64_t *)Scratch::alloc(&s, sizeof(int64_t) * (b->nrows + 1));
    g.pairs = (int32_t *)Scratch::alloc(&s, sizeof(int32_t) * (npairs > 0 ? npairs : 1));
    if (s.failed) return RRQ_ERR_OOM;
    {
        int64_t pair0 = 0;
        for (int k = 0; k < nsurf; k++) {
            const int64_t n = std::max(in[k].ntarg, nbs[k].npairs);
            if (n > 0) {
                k_near_merge<<<blocks(n, 256), 256, 0, st>>>(nbs[k].poff, nbs[k].pairs, in[k].ntarg, nbs[k].npairs,
                                                             pair0, (int32_t)b->patch_start[k],
                                                             g.poff + b->row_start[k], g.pairs);
                CK(cudaGetLastError());
            }
            pair0 += nbs[k].npairs;
        }
        CK(cudaMemcpyAsync(g.poff + b->nrows, &npairs, sizeof(int64_t), cudaMemcpyHostToDevice, st));
    }
    // CSR row pointers of the batch and the pair items grouped by (order, patch)
    b->rowptr = (int64_t *)b->alloc(sizeof(int64_t) * (b->nrows + 1));
    if (!b->rowptr) return RRQ_ERR_OOM;
    int64_t *roff = nullptr;
    CK(rrq_items_build(&g, b->nrows, b->order, d_rank, b->npatch, &rrq_batch::alloc_cb, b, b->rowptr, &b->items, &roff,
                       st));
    std::vector<int64_t> h_roff(NP + 1);
    CK(cudaMemcpyAsync(h_roff.data(), roff, sizeof(int64_t) * (NP + 1), cudaMemcpyDeviceToHost, st));
    b->nnz_start.assign(nsurf + 1, 0);
    for (int k = 0; k <= nsurf; k++)
        CK(cudaMemcpyAsync(&b->nnz_start[k], b->rowptr + b->row_start[k], sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    b->nnz = b->nnz_start[nsurf];
    for (int p = 2; p <= RRQ_PMAX; p++) {
        b->it0[p] = h_roff[b->pl_start[p]];
        b->it1[p] = h_roff[b->pl_start[p] + b->pl_count[p]];
    }
    b->col = (int32_t *)b->alloc(sizeof(int32_t) * (b->nnz > 0 ? b->nnz : 1));
    for (int k = 0; k < 4; k++)
        if (kernel_mask & (1u << k)) b->val[k] = (double *)b->alloc(sizeof(double) * (b->nnz > 0 ? b->nnz : 1));
    b->roots = (EdgeRoot *)b->alloc(sizeof(EdgeRoot) * 3 * (npairs > 0 ? npairs : 1));
    b->uside = (int8_t *)b->alloc(sizeof(int8_t) * (npairs > 0 ? npairs : 1));
    if (!b->col || !b->roots || !b->uside) return RRQ_ERR_OOM;
    for (int k = 0; k < 4; k++)
        if ((kernel_mask & (1u << k)) && !b->val[k]) return RRQ_ERR_OOM;
    // launch shapes: defaults (persistent) or measured
    for (int p = 2; p <= RRQ_PMAX; p++) {
        int tiles[4];
        if (b->pl_count[p] && rrq_pair_tiles(p, tiles) > 0) {
            b->tile[p] = tiles[0];
            b->persistent[p] = 1;
        }
    }
    CK(cudaMemsetAsync(b->cnt, 0, sizeof(BuildCounters), st));
    if (flags & RRQ_BATCH_AUTOTUNE) {
        const auto t0 = std::chrono::steady_clock::now();
        for (int p = 2; p <= RRQ_PMAX; p++)
            if (b->it1[p] > b->it0[p]) CK(autotune_order(b, p, st));
        b->ms_autotune = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        // later builds on this context use the measured shapes
        for (int p = 2; p <= RRQ_PMAX; p++)
            if (b->it1[p] > b->it0[p]) {
                ctx->tune_tile[b->mixed][p] = b->tile[p];
                ctx->tune_pers[b->mixed][p] = b->persistent[p];
            }
    }
    // record the value computation as one graph (on a private stream)
    CK(cudaStreamSynchronize(st));
    CK(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
    rrq_launch_counter() = 0;
    CK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed));
    cudaError_t e = cudaMemsetAsync(b->cnt, 0, sizeof(BuildCounters), b->cap);
    for (int p = 2; p <= RRQ_PMAX && e == cudaSuccess; p++)
        if (b->pl_count[p])
            e = rrq_launch_precompute(p, b->tab[p], b->plists + b->pl_start[p], b->pl_count[p], b->node_off, b->xyz,
                                      b->nrm, pd, b->cap);
    for (int p = 2; p <= RRQ_PMAX && e == cudaSuccess; p++)
        if (b->it1[p] > b->it0[p])
            e = rrq_launch_pairs(p, b->mixed, pair_args(b, p), PairShape{b->tile[p], b->persistent[p], b->tile_ctr + p},
                                 b->cap);
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(b->cap, &graph);
    b->graph = graph;
    if (e != cudaSuccess || e2 != cudaSuccess) {
        set_err("graph capture", e != cudaSuccess ? e : e2);
        return RRQ_ERR_CUDA;
    }
    CK(cudaGraphInstantiate(&b->exec, b->graph, 0));
    size_t nn = 0;
    CK(cudaGraphGetNodes(b->graph, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    CK(cudaGraphGetNodes(b->graph, nodes.data(), &nn));
    for (cudaGraphNode_t n : nodes) {
        cudaGraphNodeType ty;
        if (cudaGraphNodeGetType(n, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) b->graph_kernels++;
    }
    return RRQ_OK;
}

}  // namespace

extern "C" rrq_status rrq_batch_create(rrq_ctx *ctx, int32_t nsurf, const rrq_surface *surfs, const rrq_targets *targs,
                                       uint32_t kernel_mask, const rrq_options *opt, uint32_t flags,
                                       rrq_batch **out) {
    if (!ctx || !out || nsurf < 1 || !surfs || !targs) return RRQ_ERR_ARG;
    *out = nullptr;
    if (kernel_mask == 0 || (kernel_mask & ~15u) || (flags & ~(uint32_t)RRQ_BATCH_AUTOTUNE)) return RRQ_ERR_ARG;
    rrq_options o;
    memset(&o, 0, sizeof(o));
    if (opt) o = *opt;
    if (o.precision != 0 && o.precision != 1) return RRQ_ERR_ARG;
    if (o.translation != 0) return RRQ_ERR_UNSUPPORTED;
    CK(cudaSetDevice(ctx->device));
    const auto t0 = std::chrono::steady_clock::now();
    rrq_batch *b = new rrq_batch();
    b->device = ctx->device;
    b->nsurf = nsurf;
    b->mask = kernel_mask;
    b->mixed = o.precision == 1;
    b->newton_max = o.newton_max > 0 ? o.newton_max : 30;
    if (cudaEventCreate(&b->ev[0]) != cudaSuccess || cudaEventCreate(&b->ev[1]) != cudaSuccess) {
        delete b;
        return RRQ_ERR_CUDA;
    }
    const rrq_status rs = create_impl(ctx, b, nsurf, surfs, targs, kernel_mask, o, flags);
    if (rs != RRQ_OK) {
        cudaStreamSynchronize(ctx->stream);
        delete b;
        return rs;
    }
    b->ms_create = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = b;
    return RRQ_OK;
}

extern "C" rrq_status rrq_batch_execute(rrq_ctx *ctx, rrq_batch *b) {
    if (!ctx || !b || !b->exec || ctx->device != b->device) return RRQ_ERR_ARG;
    CK(cudaSetDevice(ctx->device));
    memset(&ctx->diag, 0, sizeof(ctx->diag));
    CK(cudaEventRecord(b->ev[0], ctx->stream));
    CK(cudaGraphLaunch(b->exec, ctx->stream));
    CK(cudaEventRecord(b->ev[1], ctx->stream));
    BuildCounters hc;
    CK(cudaMemcpyAsync(&hc, b->cnt, sizeof(hc), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    float ms = 0;
    cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]);
    b->ms_last = ms;
    ctx->diag.npairs = b->npairs;
    ctx->diag.newton_fail = (int64_t)hc.newton_fail;
    ctx->diag.on_edge = (int64_t)hc.on_edge;
    ctx->diag.u_poor = (int64_t)hc.u_poor;
    ctx->diag.ssq_edges = (int64_t)hc.ssq_edges;
    ctx->diag.far_edges = (int64_t)hc.far_edges;
    ctx->diag.ms_pairs = ms;
    ctx->diag.kernel_launches = b->graph_kernels;
    ctx->diag.kappa_max = b->kappa_max;
    return hc.newton_fail > 0 ? RRQ_WARN_ROOTFIND : RRQ_OK;
}

extern "C" rrq_status rrq_batch_csr(const rrq_batch *b, int32_t surf, rrq_csr *view, int64_t *row_start,
                                    int64_t *node_start) {
    if (!b || !view || surf < -1 || surf >= b->nsurf) return RRQ_ERR_ARG;
    memset(view, 0, sizeof(*view));
    const int k0 = surf < 0 ? 0 : surf, k1 = surf < 0 ? b->nsurf : surf + 1;
    view->nrows = b->row_start[k1] - b->row_start[k0];
    view->nnz = b->nnz_start[k1] - b->nnz_start[k0];
    for (int k = k0; k < k1; k++) view->npairs += b->pair_count[k];
    view->kernel_mask = b->mask | RRQ_CSR_VIEW;
    view->rowptr = b->rowptr + b->row_start[k0];
    view->col = b->col;
    for (int k = 0; k < 4; k++) view->val[k] = b->val[k];
    if (row_start)
        for (int k = 0; k <= b->nsurf; k++) row_start[k] = b->row_start[k];
    if (node_start)
        for (int k = 0; k <= b->nsurf; k++) node_start[k] = b->node_start[k];
    return RRQ_OK;
}

extern "C" rrq_status rrq_batch_info_get(const rrq_batch *b, rrq_batch_info *info) {
    if (!b || !info) return RRQ_ERR_ARG;
    memset(info, 0, sizeof(*info));
    info->nsurf = b->nsurf;
    info->nrows = b->nrows;
    info->nnode = b->nnode;
    info->nnz = b->nnz;
    info->npairs = b->npairs;
    info->graph_kernels = b->graph_kernels;
    for (int p = 0; p <= RRQ_PMAX; p++) {
        info->tile[p] = b->tile[p];
        info->persistent[p] = b->persistent[p];
    }
    info->ms_create = b->ms_create;
    info->ms_autotune = b->ms_autotune;
    info->ms_last_execute = b->ms_last;
    return RRQ_OK;
}

extern "C" void rrq_batch_destroy(rrq_batch *b) {
    if (!b) return;
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    delete b;
}

extern "C" rrq_status rrq_autotune(rrq_ctx *ctx, const rrq_surface *surf, const rrq_targets *targ, uint32_t kernel_mask,
                                   const rrq_options *opt) {
    rrq_batch *b = nullptr;
    const rrq_status rs = rrq_batch_create(ctx, 1, surf, targ, kernel_mask, opt, RRQ_BATCH_AUTOTUNE, &b);
    if (rs != RRQ_OK) return rs;
    rrq_batch_destroy(b);
    return RRQ_OK;
}
