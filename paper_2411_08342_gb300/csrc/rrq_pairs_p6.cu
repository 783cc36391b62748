// Instantiation of the per-pair stage for patch order p = 6: tiles of 6, 5, 4, 3 pairs per CTA
// (the first is the default), FP64 and mixed line integrals.
#include "rrq_pairs_tile.cuh"

cudaError_t rrq_launch_pairs_p6(bool mixed, const PairArgs &a, const PairShape &shape, cudaStream_t st) {
    return rrqk::launch_pairs_order<6, 6, 5, 4, 3>(mixed, a, shape, st);
}

cudaError_t rrq_launch_pairs_eval_p6(const PairArgs &a, const PairShape &shape, cudaStream_t st) {
    return rrqk::launch_pairs_eval_order<6, 6, 5, 4, 3>(a, shape, st);
}

int rrq_pair_tiles_p6(int out[4]) { return rrqk::tiles_of<6, 5, 4, 3>(out); }
