/*
 * rrq.h -- C ABI of librrq: near-field quadrature corrections for the Laplace
 * single/double layer potentials and their normal derivatives (S, D, S', D') on
 * triangulated surfaces in 3D, by recursive reduction quadrature (Jiang & Zhu,
 * arXiv 2411.08342), computed on one NVIDIA GB300 (sm_103a).
 *
 * What is computed.  For a target r' and a source patch P the correction row is
 *     row_K(r', P)[i] = RRQ_K(r', P)[i] - K(r', x_i) w_i      (i = 0 .. n_p-1)
 * where RRQ_K(r', P) is the row vector that maps the density values at the n_p
 * nodes x_i of P to the integral over P of the kernel K against the harmonic fit of
 * the density (Sec. 3, Thms. 3.2-3.5; Sec. 4 Steps 1-8 and the matrix-build remark),
 * and K(r', x_i) w_i is the smooth-rule weight (omitted for the node that coincides
 * with the target).  The kernels are (Sec. 1, eqs. slpdef-dprimelpdef):
 *     S : G = 1/(4 pi |r'-r|)          D : dG/dnu (source normal)
 *     S': dG/dnu' (target normal)      D': d^2 G / dnu' dnu
 * On-surface targets that are nodes of P get the principal value for D and S'
 * (the line integrals give the exterior limit; the jump 1/2 is applied), S and D'
 * are continuous.  The correction matrix has one row per target and is stored as
 * CSR; the columns of a row are the nodes of its near patches in ascending patch
 * id, each patch's nodes in node order.  Near patches of a target t are those with
 * |x_t - c_P| <= R_P + eta d_P (c_P: vertex mean, R_P: largest distance from c_P to
 * the nodes and vertices, d_P: longest vertex-to-vertex edge), plus the patch that
 * contains t as a node (Sec. 4, remark on near-target identification).
 *
 * Geometry.  Patch P of order p (2 <= p <= RRQ_PMAX) has n_p = p(p+1)/2 nodes: the
 * images of the reference nodes ref_uv[p] (points (u,v) strictly inside the triangle
 * (0,0),(1,0),(0,1), unisolvent for total degree p-1).  The patch surface is the
 * degree p-1 interpolant of its node positions; its boundary is the image of the
 * triangle's edges, oriented counter-clockwise about the outward normal.
 *
 * Conventions for every function:
 *   - return RRQ_OK (0) on success, a negative rrq_status on error; no function
 *     aborts the process; rrq_status_string() names a status;
 *   - pointers are borrowed for the duration of the call only;
 *   - input arrays are device pointers unless rrq_options.inputs_on_host = 1;
 *   - all work is enqueued on the context's CUDA stream; functions that return
 *     sizes or diagnostics synchronise that stream first;
 *   - there is no CPU fallback: without a usable sm_103a device every entry point
 *     that computes returns RRQ_ERR_CUDA.
 */
#ifndef RRQ_H
#define RRQ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RRQ_PMAX 14

typedef int32_t rrq_status;
enum {
    RRQ_OK = 0,
    RRQ_ERR_ARG = -1,          /* NULL pointer, size or order out of range, or a NaN or
                                  infinity in the node positions, normals, weights, target
                                  positions or target normals (checked on the device) */
    RRQ_ERR_CUDA = -2,         /* a CUDA call failed (message in rrq_last_error) */
    RRQ_ERR_OOM = -3,          /* device allocation failed */
    RRQ_ERR_DEGENERATE = -4,   /* a patch is degenerate or its fit matrix is singular */
    RRQ_ERR_UNSUPPORTED = -5,  /* option combination not implemented (e.g. ptilde != 2p) */
    RRQ_WARN_ROOTFIND = 1      /* success, but some pairs used the fallback edge rule */
};

/* Kernel selection bits (rrq_build_corrections kernel_mask; rrq_apply kernel). */
enum { RRQ_S = 1, RRQ_D = 2, RRQ_SP = 4, RRQ_DP = 8 };

typedef struct rrq_ctx rrq_ctx;

/* One surface.  All arrays are read only. */
typedef struct {
    int32_t npatch;                 /* number of patches, >= 1 */
    const int32_t *order;           /* [npatch] order p of each patch */
    const int64_t *node_off;        /* [npatch+1] first node of each patch; node_off[0] = 0,
                                       node_off[P+1] - node_off[P] = n_p(order[P]) */
    const double *xyz;              /* [nnode][3] node positions */
    const double *nrm;              /* [nnode][3] unit outward normals at the nodes */
    const double *wts;              /* [nnode] smooth-rule weights (reference weight x area element) */
    const double *ref_uv[RRQ_PMAX + 1]; /* ref_uv[p]: [n_p][2] reference nodes of order p
                                       (host memory always); NULL for unused orders */
} rrq_surface;

/* Targets.  self_node[t] = global node id if target t is a surface node, else -1. */
typedef struct {
    int64_t ntarg;                  /* >= 0 */
    const double *xyz;              /* [ntarg][3] */
    const double *nrm;              /* [ntarg][3] unit normal nu' at the target (used by S', D') */
    const int64_t *self_node;       /* [ntarg], or NULL = no target is a node */
} rrq_targets;

typedef struct {
    int32_t inputs_on_host;  /* 1: surface/target arrays are host pointers (copied in) */
    int32_t ptilde;          /* Gauss-Legendre nodes per edge; 0 = 2p (only 2p is implemented) */
    double rho0;             /* singularity-swap used when the Bernstein radius of the
                                complex preimage t0 is below rho0; 0 = 10^(5/ptilde) */
    int32_t newton_max;      /* Newton iterations for t0; 0 = 30 */
    double eta;              /* near factor; 0 = 1 */
    int32_t precision;       /* 0: FP64 throughout (default).  1: mixed -- the line
                                integrals of Step 6 (sums over the 3 ptilde edge nodes), the
                                translation sums of Step 7 and the fit contraction of Step 8
                                are accumulated in double-float arithmetic (pairs of FP32
                                numbers, exact FMA products, compensated sums: about 48 bits)
                                on the FP32 pipes; roots, singularity-swap recurrences and
                                weights, Omega_0, target harmonics and the smooth subtraction
                                stay FP64.  In rrq_apply: the smooth sum beyond r_c in FP32
                                (see rrq_apply) */
    int32_t translation;     /* Step 7.  0: the translation sums of eqs. l2ltranslation2-3 term
                                by term, O(p^4) per pair (default).  1: the O(p^3) scheme of
                                the remark on fast translation in Sec. 2.3 -- rotate the line
                                integrals so that the target lies on the polar axis, translate
                                along it, rotate back.  The same rows up to rounding.  Only
                                for FP64 matrix builds (rrq_build_corrections,
                                rrq_build_corrections_into; with precision = 1:
                                RRQ_ERR_UNSUPPORTED; values other than 0, 1: RRQ_ERR_ARG);
                                rrq_evaluate_near, rrq_batch_create and
                                rrq_build_corrections_static return RRQ_ERR_UNSUPPORTED for
                                any value but 0; rrq_apply ignores it */
} rrq_options;

/* CSR correction matrix in device memory owned by the library (rrq_csr_free). */
typedef struct {
    int64_t nrows;           /* = ntarg */
    int64_t nnz;             /* entries per kernel */
    int64_t npairs;          /* near (target, patch) pairs */
    uint32_t kernel_mask;    /* kernels whose val[] is filled */
    int64_t *rowptr;         /* [nrows+1] device */
    int32_t *col;            /* [nnz] device, global node ids */
    double *val[4];          /* [nnz] device each, for S, D, S', D' (NULL if not built) */
} rrq_csr;

/* Counters of the last build (pairs per category). */
typedef struct {
    int64_t npairs;
    int64_t newton_fail;     /* an edge root did not converge: upsampled edge rule used */
    int64_t on_edge;         /* target numerically on a patch edge: row unreliable */
    int64_t u_poor;          /* no unit vector u kept min u.(r'-r)/|r'-r| above -1/2 */
    int64_t ssq_edges;       /* edges evaluated by singularity swap */
    int64_t far_edges;       /* edges evaluated by the upsampled Gauss rule */
    double ms_near, ms_precompute, ms_pairs;  /* stage times of the last build (ms) */
    int64_t kernel_launches; /* CUDA kernels the last build launched */
    double ms_apply_smooth, ms_apply_spmv;    /* kernel time of the last rrq_apply and of the
                                                 last rrq_apply_correction (ms) */
    double kappa_max;        /* largest 1-norm condition number kappa_1(A) of a patch's fit
                                matrix A (eq. dlpdensitylinearsystem2) in the last build, in
                                the paper's harmonic normalisation (Sec. 5.1); INFINITY if a
                                fit was singular */
} rrq_diag;

/* A reference node set for order p (2 <= p <= RRQ_PMAX) on the triangle
 * {u, v >= 0, u + v <= 1}: uv [n_p][2], n_p = p(p+1)/2, the blend of the p Gauss-Legendre
 * points of [0, 1] onto the triangle (strictly interior nodes, ordered i-major over the
 * barycentric index triples i + j + k = p - 1), and, if w is not NULL, w [n_p] the
 * interpolatory weights (exact for total degree < p, summing to 1/2).  Any other node set
 * may be passed in rrq_surface.ref_uv; this one is what the test workloads use.  Host
 * memory, no GPU work. */
rrq_status rrq_ref_nodes(int32_t p, double *uv, double *w);

/* Create a context on CUDA device `device`, enqueuing on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream). */
rrq_status rrq_ctx_create(rrq_ctx **ctx, int device, void *cuda_stream);
void rrq_ctx_destroy(rrq_ctx *ctx);

/* Build the correction matrices for the kernels in kernel_mask (RRQ_S|RRQ_D|...)
 * (Sec. 4 Steps 1-8 with the matrix-build remark; Sec. 3.6 for S', 3.7 for D';
 * Sec. 5 eq. dlpsplitting for the correction = RRQ - smooth).  On success *out holds
 * device buffers allocated by the library; free them with rrq_csr_free.  Synchronises
 * the context stream.  Errors: RRQ_ERR_ARG for invalid sizes/orders/pointers,
 * RRQ_ERR_DEGENERATE if a patch has zero area or a singular fit, RRQ_ERR_OOM,
 * RRQ_ERR_CUDA; RRQ_WARN_ROOTFIND (> 0) when some pairs used the fallback rule. */
rrq_status rrq_build_corrections(rrq_ctx *ctx, const rrq_surface *surf, const rrq_targets *targ,
                                 uint32_t kernel_mask, const rrq_options *opt, rrq_csr *out);

/* Copy a CSR (built by rrq_build_corrections, or a batch view) into caller buffers:
 * rowptr [nrows+1] (rebased to start at 0), col [nnz], val[k] [nnz] for each built
 * kernel k (NULL entries are skipped).
 * dst_on_host = 1 for host buffers (pinned or pageable), 0 for device buffers.
 * Synchronises the context stream. */
rrq_status rrq_csr_copy(rrq_ctx *ctx, const rrq_csr *csr, int64_t *rowptr, int32_t *col,
                        double *val[4], int32_t dst_on_host);

/* Free the device buffers of a CSR built by this context and zero the struct
 * (RRQ_ERR_ARG for a batch view). */
rrq_status rrq_csr_free(rrq_ctx *ctx, rrq_csr *csr);

/* Apply one corrected operator (Sec. 5, eq. dlpsplitting):
 *   out[t] = sum_{j : x_j != target t} K(x_t, x_j) w_j density[j] + sum_j C[t][j] density[j]
 * with K the kernel `kernel` (one of RRQ_S, RRQ_D, RRQ_SP, RRQ_DP) and C its correction
 * CSR (NULL: the smooth sum alone).  density [nnode] and out [ntarg] follow
 * inputs_on_host.  One fused kernel: each block of targets sums the smooth rule over all
 * nodes (a direct O(ntarg * nnode) sum; no fast multipole method) and then adds its
 * targets' CSR rows.  With rrq_options.precision = 1 the smooth terms of nodes at least
 * r_c from the target run in FP32 (coordinates as (hi, lo) FP32 pairs so that x_t - x_j
 * keeps ~1e-7 relative accuracy, compensated FP32 sums per tile of sources, FP64 across
 * tiles) and the closer ones, which all lie in the target's CSR row, in FP64 with the
 * row (r_c = eta x the smallest node spread of a patch; the CSR is then required).
 * rrq_last_diagnostics reports the kernel time as ms_apply_smooth. */
rrq_status rrq_apply(rrq_ctx *ctx, const rrq_surface *surf, const rrq_targets *targ, int32_t kernel,
                     const rrq_csr *corr, const double *density, double *out, const rrq_options *opt);

/* The correction alone (Sec. 5, eq. dlpsplitting: the sparse part that is added to a
 * smooth-rule sum computed elsewhere, e.g. by a fast multipole method):
 *   out[t] = (accumulate ? out[t] : 0) + sum_j C[t][j] density[j],   t < corr->nrows,
 * with C the CSR of `kernel` in corr (a build's CSR or a batch view).  density [nnode]
 * (nnode > every column index) and out [nrows] are host memory when on_host != 0, else
 * device memory.  One warp per row; HBM bound.  Synchronises the context stream;
 * rrq_last_diagnostics reports the kernel time as ms_apply_spmv. */
rrq_status rrq_apply_correction(rrq_ctx *ctx, const rrq_csr *corr, int32_t kernel, const double *density,
                                int64_t nnode, double *out, int32_t accumulate, int32_t on_host);

/* Density-given near evaluation (Sec. 4 Steps 1-8 with Step 2 for a given density, as the
 * paper evaluates close targets without storing the matrix):
 *     out[k][t] = sum_j C_k[t][j] density[j]        for every kernel k in kernel_mask
 * i.e. the correction of rrq_build_corrections applied to `density`, computed without the
 * CSR: per patch the fit coefficients X sigma are formed once, then per (target, patch)
 * pair only the B . (X sigma) products (O(p^2) per pair instead of O(p^4)), the jump and
 * the smooth rule.  out[k] ([ntarg], device or host as inputs_on_host; indexed S, D, S',
 * D') must be non-NULL for every requested kernel.  FP64 only (precision = 1 gives
 * RRQ_ERR_UNSUPPORTED).  The smooth sum over all nodes is not included: rrq_apply with a
 * NULL CSR gives it.  Synchronises the context stream; diagnostics as for a build. */
rrq_status rrq_evaluate_near(rrq_ctx *ctx, const rrq_surface *surf, const rrq_targets *targ, uint32_t kernel_mask,
                             const double *density, double *out[4], const rrq_options *opt);

/* Conditioning of the density fits (Sec. 5.1): for every patch P of `surf`, kappa[P] =
 * kappa_1(A) = ||A||_1 ||A^{-1}||_1 of its quaternion harmonic system (eq.
 * dlpdensitylinearsystem2, the 4 n_p x 4 n_p real block form) in the paper's
 * normalisation of the harmonics (R_l^m of eq. rlmdef, H^{(l,m)} = sqrt2 Im S^{(l,m)}),
 * on the patch scaled, translated and rotated as in Step 1; INFINITY where the fit is
 * singular or the patch degenerate.  Runs the per-patch precompute only (no targets).
 * With on_host != 0 the surface arrays and kappa ([npatch] doubles, caller-owned) are
 * host memory, else device memory.  Synchronises the context stream. */
rrq_status rrq_fit_condition(rrq_ctx *ctx, const rrq_surface *surf, double *kappa, int32_t on_host);

/* Counters and stage timings of the last rrq_build_corrections on this context. */
rrq_status rrq_last_diagnostics(rrq_ctx *ctx, rrq_diag *diag);

/* Allocation-free build.  The paper has no counterpart to this entry point; it exists
 * for callers that must not allocate device memory during a call: applications that
 * reserve all device memory up front in their own allocator (a cudaMalloc would fail
 * or fragment their pool), loops that forbid allocation after start-up, and plug-in
 * hosts whose device footprint must not change once running.
 *
 * It computes exactly what rrq_build_corrections computes, with the same kernels, but
 * takes every scratch buffer from one static device array of RRQ_STATIC_SCRATCH_BYTES
 * (64 MiB) that each GPU loading this library holds until the process exits; the
 * per-patch data take about 0.15 MB at a largest order of 6, 0.35 MB at 8 and 1.3 MB at
 * 12, plus the near list and the order tables (e.g. a few hundred patches), larger
 * problems are rejected with RRQ_ERR_ARG and a message in rrq_last_error().  It calls
 * no cudaMalloc, cudaFree or allocating library routine.
 *   - inputs: device pointers only (inputs_on_host = 1 is rejected);
 *   - FP64 only: rrq_options.precision other than 0 gives RRQ_ERR_UNSUPPORTED; the
 *     launch shapes are the orders' defaults (the context's tuned shapes are not used);
 *   - outputs (device, caller-owned): rowptr [ntarg+1], col [capacity], val[k]
 *     [capacity] for every kernel k in kernel_mask (S, D, S', D' order);
 *   - *nnz_out and *npairs_out (host, may be NULL) receive the entry and pair counts;
 *     when nnz exceeds capacity nothing is written to col/val and RRQ_ERR_ARG is
 *     returned with *nnz_out set, so the caller can retry with larger buffers;
 *   - every call looks up the array's device address on the current device
 *     (cudaGetSymbolAddress, which allocates nothing), and reads sizes back to the host,
 *     synchronising the context stream several times before it returns;
 *   - every call reuses the same array and leaves the last call's contents in it; what
 *     must start at zero is cleared by each call.  Calls whose GPU work overlaps (two
 *     streams, two threads, two contexts on one device) race on the array: serialise
 *     them. */
#define RRQ_STATIC_SCRATCH_BYTES ((size_t)64 << 20)
rrq_status rrq_build_corrections_static(rrq_ctx *ctx, const rrq_surface *surf, const rrq_targets *targ,
                                        uint32_t kernel_mask, const rrq_options *opt, int64_t *rowptr,
                                        int32_t *col, double *val[4], int64_t capacity, int64_t *nnz_out,
                                        int64_t *npairs_out);

/* Build into caller-owned buffers that the device can address: device memory, managed
 * memory, or page-locked host memory (cudaHostAlloc, or cudaHostRegister'ed and mapped),
 * which the per-pair kernels then write directly, so that no copy of the matrices
 * follows the build.  Same values as rrq_build_corrections (same kernels).
 *   - rowptr [ntarg+1], col [capacity], val[k] [capacity] for every kernel k in
 *     kernel_mask (the others may be NULL); CSR layout as rrq_csr;
 *   - inputs as rrq_options.inputs_on_host says; other options as for a build;
 *   - *nnz_out, *npairs_out (may be NULL): entries per kernel and near pairs.
 * If an output buffer is not device-addressable (plain pageable host memory) nothing is
 * launched and RRQ_ERR_ARG is returned; if the entries exceed capacity, *nnz_out is set,
 * nothing beyond the near list is computed and RRQ_ERR_ARG is returned (call again with
 * a larger capacity).  Synchronises the context stream. */
rrq_status rrq_build_corrections_into(rrq_ctx *ctx, const rrq_surface *surf, const rrq_targets *targ,
                                      uint32_t kernel_mask, const rrq_options *opt, int64_t *rowptr,
                                      int32_t *col, double *val[4], int64_t capacity, int64_t *nnz_out,
                                      int64_t *npairs_out);

/* ---- Batched build of many surfaces (the paper has no counterpart: it builds one
 * surface at a time).  A batch plan takes nsurf surfaces, each with its own targets,
 * patch counts and orders, and runs the same per-patch and per-pair computation as
 * rrq_build_corrections over all of them at once:
 *   - rrq_batch_create checks and copies the inputs into batch-owned device memory,
 *     computes the patch bounds, builds every surface's near list (a target sees only
 *     the patches of its own surface), the CSR structure of the whole batch and the
 *     pair work list (grouped by order, then patch), then records the value
 *     computation -- per-patch precompute of every order, then for every order one
 *     root kernel and one persistent pair kernel over the pairs of all surfaces (S, D,
 *     S', D' in one pass per pair) -- as one CUDA graph.  With RRQ_BATCH_AUTOTUNE in
 *     `flags` it first times the compiled tile sizes (pairs per CTA) and both schedules
 *     (persistent / 16 waves) of every order on a sample of that order's pairs and
 *     records the fastest; otherwise each order takes its default shape, persistent;
 *   - rrq_batch_execute launches that graph once and synchronises: afterwards the
 *     batch CSR holds the corrections of every surface.  Executing again recomputes
 *     the same values (the graph reads only batch-owned copies of the inputs);
 *   - the result is ONE CSR over the concatenated targets: rows row_start[s] ..
 *     row_start[s+1]-1 belong to surface s, and their columns are node ids LOCAL to
 *     surface s, so rrq_batch_csr(b, s, &view) gives a CSR view of surface s that
 *     rrq_apply accepts together with that surface and its targets.  Views alias the
 *     batch's memory: never pass them to rrq_csr_free; they live until
 *     rrq_batch_destroy.
 * All surfaces must use the same reference nodes for a given order (RRQ_ERR_ARG
 * otherwise).  Each targets' self_node holds node ids of its own surface.  Options and
 * errors as rrq_build_corrections; rrq_batch_create synchronises the context stream.
 * rrq_last_diagnostics after rrq_batch_execute reports that execution (counters;
 * ms_pairs = device time of the whole graph, precompute included; kernel_launches =
 * kernel nodes in the graph). */
typedef struct rrq_batch rrq_batch;
enum { RRQ_BATCH_AUTOTUNE = 1 };
/* Set in rrq_csr.kernel_mask of a view: its rowptr values index the batch's col/val
 * arrays (rowptr[0] may be nonzero) and rrq_csr_free refuses it. */
#define RRQ_CSR_VIEW 0x80000000u

typedef struct {
    int32_t nsurf;
    int64_t nrows, nnode, nnz, npairs;   /* totals over the batch */
    int32_t graph_kernels;               /* kernel nodes in the recorded graph */
    int32_t tile[RRQ_PMAX + 1];          /* pairs per CTA chosen for order p (0: order absent) */
    int32_t persistent[RRQ_PMAX + 1];    /* 1: one wave of CTAs fetching tiles from a counter */
    double ms_create, ms_autotune;       /* host wall time of rrq_batch_create and of its tuning */
    double ms_last_execute;              /* device time of the last rrq_batch_execute */
} rrq_batch_info;

rrq_status rrq_batch_create(rrq_ctx *ctx, int32_t nsurf, const rrq_surface *surfs, const rrq_targets *targs,
                            uint32_t kernel_mask, const rrq_options *opt, uint32_t flags, rrq_batch **out);
rrq_status rrq_batch_execute(rrq_ctx *ctx, rrq_batch *batch);
/* surf in [0, nsurf): view of that surface's rows; surf = -1: the whole batch.
 * row_start, node_start (may be NULL): [nsurf+1] host arrays of first rows / nodes. */
rrq_status rrq_batch_csr(const rrq_batch *batch, int32_t surf, rrq_csr *view, int64_t *row_start,
                         int64_t *node_start);
rrq_status rrq_batch_info_get(const rrq_batch *batch, rrq_batch_info *info);
void rrq_batch_destroy(rrq_batch *batch);

/* Autotune the per-pair stage for this problem (no counterpart in the paper): times every
 * compiled tile size and both schedules of every order present on a sample of the
 * problem's pairs (as rrq_batch_create with RRQ_BATCH_AUTOTUNE on one surface) and keeps
 * the fastest shape per order and precision (rrq_options.precision) in the context;
 * later rrq_build_corrections calls on this context launch with those shapes.  The
 * computed values do not depend on the shape.  A batch created with RRQ_BATCH_AUTOTUNE
 * stores its measured shapes the same way.  Synchronises the context stream. */
rrq_status rrq_autotune(rrq_ctx *ctx, const rrq_surface *surf, const rrq_targets *targ, uint32_t kernel_mask,
                        const rrq_options *opt);

/* Measured fused-multiply-add throughput of this device in TFLOP/s (2 flops per FMA),
 * FP64 (fp32 = 0) or FP32 (fp32 = 1): 8 independent dependency chains per thread,
 * 8 blocks of 256 threads per SM, timed with CUDA events.  Used as the roofline
 * denominator of the ALU-bound correction build.  Synchronises the context stream. */
rrq_status rrq_measure_fma_peak(rrq_ctx *ctx, int32_t fp32, double *tflops);

/* Human-readable name of a status; message of the last CUDA error on this thread. */
const char *rrq_status_string(rrq_status s);
const char *rrq_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
