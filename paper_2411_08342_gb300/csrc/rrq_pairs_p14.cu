// Instantiation of the per-pair stage for patch order p = 14: tiles of 2 pairs per CTA
// (the first is the default), FP64 and mixed line integrals.
#include "rrq_pairs_tile.cuh"

cudaError_t rrq_launch_pairs_p14(bool mixed, const PairArgs &a, const PairShape &shape, cudaStream_t st) {
    return rrqk::launch_pairs_order<14, 2>(mixed, a, shape, st);
}

cudaError_t rrq_launch_pairs_eval_p14(const PairArgs &a, const PairShape &shape, cudaStream_t st) {
    return rrqk::launch_pairs_eval_order<14, 2>(a, shape, st);
}

int rrq_pair_tiles_p14(int out[4]) { return rrqk::tiles_of<2>(out); }
