// Host-side pieces shared by the librrq translation units that implement the C ABI:
// the context, the stream-ordered scratch allocator, error reporting, input checks and
// uploads, per-order table caching, and the near-list / pair-item builders of rrq_near.cu.
#pragma once
#include <stdio.h>
#include <string.h>

#include <vector>

#include "rrq_internal.cuh"

// near list: pairs[poff[t] .. poff[t+1]) are the patches near target t
struct NearBuffers {
    int64_t *poff;
    int32_t *pairs;
    int64_t npairs;
};
typedef void *(*rrq_alloc_fn)(void *ctx, size_t bytes);
cudaError_t rrq_near_build(const double *d_bounds, int npatch, const int64_t *d_node_off, const double *d_txyz,
                           const int64_t *d_tself, int64_t ntarg, double eta, rrq_alloc_fn alloc, void *actx,
                           NearBuffers *out, cudaStream_t st);
cudaError_t rrq_items_build(const NearBuffers *nb, int64_t ntarg, const int32_t *d_order, const int32_t *d_rank,
                            int npatch, rrq_alloc_fn alloc, void *actx, int64_t *d_rowptr, PairItem **items_out,
                            int64_t **rank_off_out, cudaStream_t st);

// last error message of the calling host thread (rrq_last_error)
constexpr size_t RRQ_ERR_LEN = 512;
char *rrq_err_buf();
void set_err(const char *what, cudaError_t e);

struct rrq_ctx {
    int device;
    cudaStream_t stream;
    rrq_diag diag;
    cudaEvent_t ev[4];
    // cached per-order tables
    OrderTables *d_tab[RRQ_PMAX + 1];
    std::vector<double> tab_key[RRQ_PMAX + 1];
    double tab_rho0[RRQ_PMAX + 1];
    // launch shapes of the per-pair stage measured by the autotuner, per [mixed][order]
    // (tile 0 = not tuned: the order's default tile, grid-stride schedule)
    int tune_tile[2][RRQ_PMAX + 1];
    int tune_pers[2][RRQ_PMAX + 1];
};

// scratch allocator: stream-ordered allocations freed together
struct Scratch {
    cudaStream_t st;
    std::vector<void *> ptrs;
    bool failed = false;
    static void *alloc(void *self, size_t bytes) {
        Scratch *s = static_cast<Scratch *>(self);
        void *p = nullptr;
        if (bytes == 0) bytes = 16;
        if (cudaMallocAsync(&p, bytes, s->st) != cudaSuccess) {
            s->failed = true;
            cudaGetLastError();
            return nullptr;
        }
        s->ptrs.push_back(p);
        return p;
    }
    ~Scratch() {
        for (void *p : ptrs) cudaFreeAsync(p, st);
    }
};

#define CK(call)                                   \
    do {                                           \
        cudaError_t _e = (call);                   \
        if (_e != cudaSuccess) {                   \
            set_err(#call, _e);                    \
            return _e == cudaErrorMemoryAllocation ? RRQ_ERR_OOM : RRQ_ERR_CUDA; \
        }                                          \
    } while (0)


inline int np_of(int p) { return p * (p + 1) / 2; }

// device views of the inputs (copies when they were host pointers)
struct Inputs {
    int npatch;
    int64_t nnode, ntarg;
    std::vector<int32_t> h_order;
    std::vector<int64_t> h_node_off;
    const int32_t *order;
    const int64_t *node_off;
    const double *xyz, *nrm, *wts, *txyz, *tnrm;
    const int64_t *tself;
};

template <typename T>
const T *upload(Scratch &s, const T *h, size_t n, bool on_host, cudaError_t *err) {
    if (!on_host || n == 0) return h;
    T *d = (T *)Scratch::alloc(&s, sizeof(T) * n);
    if (!d) { *err = cudaErrorMemoryAllocation; return nullptr; }
    cudaError_t e = cudaMemcpyAsync(d, h, sizeof(T) * n, cudaMemcpyHostToDevice, s.st);
    if (e != cudaSuccess) *err = e;
    return d;
}

// Checks the inputs and makes device views of them; a NaN or infinity in the node
// positions, normals, weights, target positions or target normals gives RRQ_ERR_ARG.
rrq_status prepare_inputs(rrq_ctx *ctx, Scratch &s, const rrq_surface *surf, const rrq_targets *targ, bool on_host,
                          bool need_targets, Inputs &in);
// One device pass over each of the n arrays (sizes in doubles); RRQ_ERR_ARG, with the
// array's name in rrq_last_error(), if one holds a non-finite value.  d_flag: one
// unsigned of device scratch.  Synchronises st.
rrq_status check_finite(cudaStream_t st, unsigned *d_flag, const double *const arrays[], const int64_t sizes[],
                        const char *const names[], int n);
static const char *const kInputNames[5] = {"node positions", "node normals", "smooth weights", "target positions",
                                          "target normals"};
// per-order constant tables, cached in the context by (reference nodes, rho0)
rrq_status order_tables(rrq_ctx *ctx, int p, const double *ref_uv, double rho0);
