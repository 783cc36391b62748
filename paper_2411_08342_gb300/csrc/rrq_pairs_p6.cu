// Instantiation of the per-pair kernel for patch order p = 6.
#include "rrq_pairs_tile.cuh"

cudaError_t rrq_launch_pairs_p6(const OrderTables *d_tab, const PairItem *d_items, int64_t nitems, PatchData pd,
                                 const int64_t *d_node_off, const double *d_xyz, const double *d_nrm,
                                 const double *d_wts, const double *d_txyz, const double *d_tnrm,
                                 const int64_t *d_tself, uint32_t mask, int newton_max, double *vS, double *vD,
                                 double *vSp, double *vDp, int32_t *col, BuildCounters *cnt, cudaStream_t st) {
    return rrqk::launch_pairs_tile<6, false>(d_tab, d_items, nitems, pd, d_node_off, d_xyz, d_nrm, d_wts, d_txyz, d_tnrm,
                                    d_tself, mask, newton_max, vS, vD, vSp, vDp, col, cnt, st);
}

cudaError_t rrq_launch_pairs_mix_p6(const OrderTables *d_tab, const PairItem *d_items, int64_t nitems, PatchData pd,
                                     const int64_t *d_node_off, const double *d_xyz, const double *d_nrm,
                                     const double *d_wts, const double *d_txyz, const double *d_tnrm,
                                     const int64_t *d_tself, uint32_t mask, int newton_max, double *vS, double *vD,
                                     double *vSp, double *vDp, int32_t *col, BuildCounters *cnt, cudaStream_t st) {
    return rrqk::launch_pairs_tile<6, true>(d_tab, d_items, nitems, pd, d_node_off, d_xyz, d_nrm, d_wts, d_txyz,
                                         d_tnrm, d_tself, mask, newton_max, vS, vD, vSp, vDp, col, cnt, st);
}
