// Near-pair list (the paper leaves near-target identification to a standard spatial
// search, Sec. 4 remark; this is a uniform grid of cell size max_P(R_P + eta d_P)):
//   1. patches are binned by the cell of their centre c_P (count, scan, fill);
//   2. each target scans the 27 cells around it and keeps P with
//      |x_t - c_P| <= R_P + eta d_P, plus the patch it is a node of;
//   3. counts are scanned into pair offsets, the pairs are written and each row is
//      sorted by patch id (so the CSR column order is deterministic);
//   4. CSR row lengths are n_p summed over the row's patches; pair work items carry
//      the target, the patch and the offset of their n_p entries, and are grouped by
//      a caller-given patch rank (order-major) for the per-order launches.
#include <math.h>
#include <string.h>

#include "rrq_internal.cuh"

__global__ void rrq_widen_int(const int *in, int64_t *out, int64_t n);
__global__ void rrq_narrow_int(const int64_t *in, int *out, int64_t n);

int64_t &rrq_launch_counter() {
    static thread_local int64_t n = 0;
    return n;
}

static double bits_to_double(long long b) {
    double d;
    memcpy(&d, &b, sizeof(d));
    return d;
}

namespace {

constexpr int SCAN_BLOCK = 1024;

__global__ void k_scan_block(const int64_t *__restrict__ in, int64_t *__restrict__ out, int64_t n,
                             int64_t *__restrict__ block_sums) {
    __shared__ int64_t s[SCAN_BLOCK];
    int64_t i = (int64_t)blockIdx.x * SCAN_BLOCK + threadIdx.x;
    int64_t v = i < n ? in[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < SCAN_BLOCK; off <<= 1) {
        int64_t t = threadIdx.x >= off ? s[threadIdx.x - off] : 0;
        __syncthreads();
        s[threadIdx.x] += t;
        __syncthreads();
    }
    if (i < n) out[i] = s[threadIdx.x] - v;  // exclusive
    if (threadIdx.x == SCAN_BLOCK - 1) block_sums[blockIdx.x] = s[threadIdx.x];
}

__global__ void k_scan_add(int64_t *__restrict__ out, int64_t n, const int64_t *__restrict__ block_off) {
    int64_t i = (int64_t)blockIdx.x * SCAN_BLOCK + threadIdx.x;
    if (i < n) out[i] += block_off[blockIdx.x];
}

__global__ void k_patch_reach(const double *__restrict__ bounds, int npatch, double eta,
                              unsigned long long *__restrict__ red /* [7]: h, lo3, hi3 as ordered bits */) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npatch) return;
    const double *b = bounds + (size_t)i * PD_BOUNDS;
    double reach = b[3] + eta * b[4];
    atomicMax(&red[0], (unsigned long long)__double_as_longlong(reach));
    for (int a = 0; a < 3; a++) {
        // order-preserving map of doubles to unsigned integers
        long long bits = __double_as_longlong(b[a]);
        unsigned long long key = bits < 0 ? ~(unsigned long long)bits : ((unsigned long long)bits | 0x8000000000000000ULL);
        atomicMin(&red[1 + a], key);
        atomicMax(&red[4 + a], key);
    }
}

struct Grid {
    double lo[3];
    double h;
    int n[3];
};

__device__ __forceinline__ int cell_coord(double x, double lo, double h) { return (int)floor((x - lo) / h); }

__global__ void k_bin_count(const double *__restrict__ bounds, int npatch, Grid g, int *__restrict__ cnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npatch) return;
    const double *b = bounds + (size_t)i * PD_BOUNDS;
    int cx = min(max(cell_coord(b[0], g.lo[0], g.h), 0), g.n[0] - 1);
    int cy = min(max(cell_coord(b[1], g.lo[1], g.h), 0), g.n[1] - 1);
    int cz = min(max(cell_coord(b[2], g.lo[2], g.h), 0), g.n[2] - 1);
    atomicAdd(&cnt[((size_t)cz * g.n[1] + cy) * g.n[0] + cx], 1);
}

__global__ void k_bin_fill(const double *__restrict__ bounds, int npatch, Grid g, int *__restrict__ cursor,
                           int32_t *__restrict__ items) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npatch) return;
    const double *b = bounds + (size_t)i * PD_BOUNDS;
    int cx = min(max(cell_coord(b[0], g.lo[0], g.h), 0), g.n[0] - 1);
    int cy = min(max(cell_coord(b[1], g.lo[1], g.h), 0), g.n[1] - 1);
    int cz = min(max(cell_coord(b[2], g.lo[2], g.h), 0), g.n[2] - 1);
    int pos = atomicAdd(&cursor[((size_t)cz * g.n[1] + cy) * g.n[0] + cx], 1);
    items[pos] = i;
}

__device__ int patch_of_node(const int64_t *__restrict__ node_off, int npatch, int64_t node) {
    int lo = 0, hi = npatch - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (node_off[mid] <= node) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// pass 0: count; pass 1: fill + sort
template <int PASS>
__global__ void k_near(const double *__restrict__ txyz, const int64_t *__restrict__ tself, int64_t ntarg,
                       const double *__restrict__ bounds, const int64_t *__restrict__ node_off, int npatch,
                       double eta, Grid g, const int *__restrict__ cell_start, const int32_t *__restrict__ cell_items,
                       int64_t *__restrict__ cnt, const int64_t *__restrict__ off, int32_t *__restrict__ pairs) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntarg) return;
    const double x = txyz[3 * t], y = txyz[3 * t + 1], z = txyz[3 * t + 2];
    int selfP = -1;
    if (tself) {
        int64_t sn = tself[t];
        if (sn >= 0 && sn < node_off[npatch]) selfP = patch_of_node(node_off, npatch, sn);
    }
    int cx = cell_coord(x, g.lo[0], g.h), cy = cell_coord(y, g.lo[1], g.h), cz = cell_coord(z, g.lo[2], g.h);
    int64_t c = 0, base = PASS ? off[t] : 0;
    bool self_found = false;
    for (int dz = -1; dz <= 1; dz++) {
        int zz = cz + dz;
        if (zz < 0 || zz >= g.n[2]) continue;
        for (int dy = -1; dy <= 1; dy++) {
            int yy = cy + dy;
            if (yy < 0 || yy >= g.n[1]) continue;
            for (int dx = -1; dx <= 1; dx++) {
                int xx = cx + dx;
                if (xx < 0 || xx >= g.n[0]) continue;
                size_t cell = ((size_t)zz * g.n[1] + yy) * g.n[0] + xx;
                for (int k = cell_start[cell]; k < cell_start[cell + 1]; k++) {
                    int P = cell_items[k];
                    const double *b = bounds + (size_t)P * PD_BOUNDS;
                    double d0 = x - b[0], d1 = y - b[1], d2 = z - b[2];
                    bool nearp = sqrt(d0 * d0 + d1 * d1 + d2 * d2) <= b[3] + eta * b[4];
                    if (P == selfP) { nearp = true; self_found = true; }
                    if (nearp) {
                        if (PASS) pairs[base + c] = P;
                        c++;
                    }
                }
            }
        }
    }
    if (selfP >= 0 && !self_found) {
        if (PASS) pairs[base + c] = selfP;
        c++;
    }
    if (!PASS) {
        cnt[t] = c;
    } else {
        // insertion sort of the row by patch id
        for (int64_t i = 1; i < c; i++) {
            int32_t v = pairs[base + i];
            int64_t j = i - 1;
            while (j >= 0 && pairs[base + j] > v) {
                pairs[base + j + 1] = pairs[base + j];
                j--;
            }
            pairs[base + j + 1] = v;
        }
    }
}

__global__ void k_row_len(const int64_t *__restrict__ poff, const int32_t *__restrict__ pairs, int64_t ntarg,
                          const int32_t *__restrict__ order, int64_t *__restrict__ rowlen) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntarg) return;
    int64_t s = 0;
    for (int64_t k = poff[t]; k < poff[t + 1]; k++) {
        int p = order[pairs[k]];
        s += p * (p + 1) / 2;
    }
    rowlen[t] = s;
}

// per pair: count by patch rank
__global__ void k_rank_count(const int32_t *__restrict__ pairs, int64_t npairs, const int32_t *__restrict__ rank,
                             int64_t *__restrict__ cnt) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= npairs) return;
    atomicAdd((unsigned long long *)&cnt[rank[pairs[k]]], 1ULL);
}

__global__ void k_items(const int64_t *__restrict__ poff, const int32_t *__restrict__ pairs, int64_t ntarg,
                        const int32_t *__restrict__ order, const int64_t *__restrict__ rowptr,
                        const int32_t *__restrict__ rank, int64_t *__restrict__ cursor, PairItem *__restrict__ items) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntarg) return;
    int64_t o = rowptr[t];
    for (int64_t k = poff[t]; k < poff[t + 1]; k++) {
        int P = pairs[k];
        int p = order[P];
        int64_t pos = (int64_t)atomicAdd((unsigned long long *)&cursor[rank[P]], 1ULL);
        PairItem it;
        it.t = t;
        it.off = o;
        it.P = P;
        it.pad = (int32_t)k;  // index of the pair in target-major order
        items[pos] = it;
        o += p * (p + 1) / 2;
    }
}

}  // namespace

// Exclusive scan of n int64 values (in -> out, may alias); returns the total in *total_dev
// position out[n] (out must hold n+1 entries).  tmp: scratch of >= 2*ceil(n/1024)+2 int64.
cudaError_t rrq_scan_exclusive(const int64_t *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t st);

cudaError_t rrq_scan_exclusive(const int64_t *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t st) {
    // out[0..n] with out[n] = total
    if (n <= 0) {
        return cudaMemsetAsync(out, 0, sizeof(int64_t), st);
    }
    int64_t nb = (n + SCAN_BLOCK - 1) / SCAN_BLOCK;
    int64_t *bsum = tmp, *boff = tmp + nb + 1;
    k_scan_block<<<(unsigned)nb, SCAN_BLOCK, 0, st>>>(in, out, n, bsum);
    RRQ_COUNT_LAUNCH();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (nb > 1) {
        e = rrq_scan_exclusive(bsum, boff, nb, tmp + 2 * nb + 2, st);
        if (e != cudaSuccess) return e;
        k_scan_add<<<(unsigned)nb, SCAN_BLOCK, 0, st>>>(out, n, boff);
        RRQ_COUNT_LAUNCH();
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        // total = boff[nb]
        return cudaMemcpyAsync(out + n, boff + nb, sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
    }
    return cudaMemcpyAsync(out + n, bsum, sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
}

int64_t rrq_scan_tmp_size(int64_t n) {
    int64_t tot = 0;
    while (n > 1) {
        int64_t nb = (n + SCAN_BLOCK - 1) / SCAN_BLOCK;
        tot += 2 * nb + 2;
        n = nb;
    }
    return tot + 4;
}

// ---------------------------------------------------------------------------------
// Host orchestration of the near list.  Scratch comes from the caller's allocator.
// ---------------------------------------------------------------------------------
struct NearBuffers {
    int64_t *poff;      // [ntarg+1] pair offsets
    int32_t *pairs;     // [npairs]
    int64_t npairs;
};

typedef void *(*rrq_alloc_fn)(void *ctx, size_t bytes);

cudaError_t rrq_near_build(const double *d_bounds, int npatch, const int64_t *d_node_off, const double *d_txyz,
                           const int64_t *d_tself, int64_t ntarg, double eta, rrq_alloc_fn alloc, void *actx,
                           NearBuffers *out, cudaStream_t st) {
    unsigned long long *red = (unsigned long long *)alloc(actx, 8 * sizeof(unsigned long long));
    if (!red) return cudaErrorMemoryAllocation;
    unsigned long long init[8];
    init[0] = 0ULL;
    for (int a = 0; a < 3; a++) { init[1 + a] = ~0ULL; init[4 + a] = 0ULL; }
    init[7] = 0ULL;
    cudaError_t e = cudaMemcpyAsync(red, init, sizeof(init), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    k_patch_reach<<<(npatch + 255) / 256, 256, 0, st>>>(d_bounds, npatch, eta, red);
    RRQ_COUNT_LAUNCH();
    unsigned long long hred[8];
    e = cudaMemcpyAsync(hred, red, sizeof(hred), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    Grid g;
    double h = bits_to_double((long long)hred[0]);
    double lo[3], hi[3];
    for (int a = 0; a < 3; a++) {
        unsigned long long kl = hred[1 + a], kh = hred[4 + a];
        long long bl = (kl & 0x8000000000000000ULL) ? (long long)(kl & 0x7FFFFFFFFFFFFFFFULL) : (long long)~kl;
        long long bh = (kh & 0x8000000000000000ULL) ? (long long)(kh & 0x7FFFFFFFFFFFFFFFULL) : (long long)~kh;
        lo[a] = bits_to_double(bl);
        hi[a] = bits_to_double(bh);
    }
    if (!(h > 0) || !isfinite(h)) return cudaErrorInvalidValue;
    for (;;) {
        double tot = 1;
        for (int a = 0; a < 3; a++) {
            g.n[a] = (int)floor((hi[a] - lo[a]) / h) + 1;
            tot *= g.n[a];
        }
        if (tot <= (double)(1 << 24)) break;
        h *= 1.5;
    }
    g.h = h;
    for (int a = 0; a < 3; a++) g.lo[a] = lo[a];
    size_t ncell = (size_t)g.n[0] * g.n[1] * g.n[2];
    int *cell_cnt = (int *)alloc(actx, sizeof(int) * (ncell + 1));
    int32_t *cell_items = (int32_t *)alloc(actx, sizeof(int32_t) * npatch);
    int64_t *cell_tmp = (int64_t *)alloc(actx, sizeof(int64_t) * (ncell + 1) * 2);
    int64_t *scan_tmp = (int64_t *)alloc(actx, sizeof(int64_t) * rrq_scan_tmp_size((int64_t)ncell + ntarg + 2));
    if (!cell_cnt || !cell_items || !cell_tmp || !scan_tmp) return cudaErrorMemoryAllocation;
    cudaMemsetAsync(cell_cnt, 0, sizeof(int) * (ncell + 1), st);
    k_bin_count<<<(npatch + 255) / 256, 256, 0, st>>>(d_bounds, npatch, g, cell_cnt);
    RRQ_COUNT_LAUNCH();
    // scan in int64 then narrow (ncell <= 2^24, npatch < 2^31)
    // widen counts
    {
        int64_t *wide = cell_tmp, *wscan = cell_tmp + (ncell + 1);
        rrq_widen_int<<<(unsigned)((ncell + 255) / 256), 256, 0, st>>>(cell_cnt, wide, (int64_t)ncell);
        RRQ_COUNT_LAUNCH();
        e = rrq_scan_exclusive(wide, wscan, (int64_t)ncell, scan_tmp, st);
        if (e != cudaSuccess) return e;
        rrq_narrow_int<<<(unsigned)((ncell + 1 + 255) / 256), 256, 0, st>>>(wscan, cell_cnt, (int64_t)ncell + 1);
        RRQ_COUNT_LAUNCH();
    }
    int *cursor = (int *)alloc(actx, sizeof(int) * (ncell + 1));
    if (!cursor) return cudaErrorMemoryAllocation;
    cudaMemcpyAsync(cursor, cell_cnt, sizeof(int) * (ncell + 1), cudaMemcpyDeviceToDevice, st);
    k_bin_fill<<<(npatch + 255) / 256, 256, 0, st>>>(d_bounds, npatch, g, cursor, cell_items);
    RRQ_COUNT_LAUNCH();
    int64_t *cnt = (int64_t *)alloc(actx, sizeof(int64_t) * (ntarg + 1));
    out->poff = (int64_t *)alloc(actx, sizeof(int64_t) * (ntarg + 1));
    if (!cnt || !out->poff) return cudaErrorMemoryAllocation;
    unsigned tb = (unsigned)((ntarg + 127) / 128);
    if (ntarg > 0) {
        k_near<0><<<tb, 128, 0, st>>>(d_txyz, d_tself, ntarg, d_bounds, d_node_off, npatch, eta, g, cell_cnt,
                                      cell_items, cnt, nullptr, nullptr);
        RRQ_COUNT_LAUNCH();
    }
    e = rrq_scan_exclusive(cnt, out->poff, ntarg, scan_tmp, st);
    if (e != cudaSuccess) return e;
    int64_t np_h = 0;
    cudaMemcpyAsync(&np_h, out->poff + ntarg, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    out->npairs = np_h;
    out->pairs = (int32_t *)alloc(actx, sizeof(int32_t) * (np_h > 0 ? np_h : 1));
    if (!out->pairs) return cudaErrorMemoryAllocation;
    if (ntarg > 0) {
        k_near<1><<<tb, 128, 0, st>>>(d_txyz, d_tself, ntarg, d_bounds, d_node_off, npatch, eta, g, cell_cnt,
                                      cell_items, nullptr, out->poff, out->pairs);
        RRQ_COUNT_LAUNCH();
    }
    return cudaGetLastError();
}

__global__ void rrq_widen_int(const int *in, int64_t *out, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[i];
}
__global__ void rrq_narrow_int(const int64_t *in, int *out, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (int)in[i];
}

// CSR row pointers and pair items grouped by patch rank.
cudaError_t rrq_items_build(const NearBuffers *nb, int64_t ntarg, const int32_t *d_order, const int32_t *d_rank,
                            int npatch, rrq_alloc_fn alloc, void *actx, int64_t *d_rowptr /*[ntarg+1]*/,
                            PairItem **items_out, int64_t **rank_off_out /*[npatch+1] device*/, cudaStream_t st) {
    int64_t *rowlen = (int64_t *)alloc(actx, sizeof(int64_t) * (ntarg + 1));
    int64_t *scan_tmp = (int64_t *)alloc(actx, sizeof(int64_t) * rrq_scan_tmp_size(ntarg + npatch + 2));
    int64_t *rcnt = (int64_t *)alloc(actx, sizeof(int64_t) * (npatch + 1));
    int64_t *roff = (int64_t *)alloc(actx, sizeof(int64_t) * (npatch + 1));
    PairItem *items = (PairItem *)alloc(actx, sizeof(PairItem) * (nb->npairs > 0 ? nb->npairs : 1));
    if (!rowlen || !scan_tmp || !rcnt || !roff || !items) return cudaErrorMemoryAllocation;
    unsigned tb = (unsigned)((ntarg + 127) / 128);
    if (ntarg > 0) {
        k_row_len<<<tb, 128, 0, st>>>(nb->poff, nb->pairs, ntarg, d_order, rowlen);
        RRQ_COUNT_LAUNCH();
    }
    cudaError_t e = rrq_scan_exclusive(rowlen, d_rowptr, ntarg, scan_tmp, st);
    if (e != cudaSuccess) return e;
    cudaMemsetAsync(rcnt, 0, sizeof(int64_t) * (npatch + 1), st);
    if (nb->npairs > 0) {
        k_rank_count<<<(unsigned)((nb->npairs + 255) / 256), 256, 0, st>>>(nb->pairs, nb->npairs, d_rank, rcnt);
        RRQ_COUNT_LAUNCH();
    }
    e = rrq_scan_exclusive(rcnt, roff, npatch, scan_tmp, st);
    if (e != cudaSuccess) return e;
    int64_t *cursor = rcnt;  // reuse
    cudaMemcpyAsync(cursor, roff, sizeof(int64_t) * (npatch + 1), cudaMemcpyDeviceToDevice, st);
    if (ntarg > 0) {
        k_items<<<tb, 128, 0, st>>>(nb->poff, nb->pairs, ntarg, d_order, d_rowptr, d_rank, cursor, items);
        RRQ_COUNT_LAUNCH();
    }
    *items_out = items;
    *rank_off_out = roff;
    return cudaGetLastError();
}
