// Instantiation of the per-pair stage for patch order p = 2: tiles of 8, 4 pairs per CTA
// (the first is the default), FP64 and mixed line integrals.
#include "rrq_pairs_tile.cuh"

cudaError_t rrq_launch_pairs_p2(bool mixed, const PairArgs &a, const PairShape &shape, cudaStream_t st) {
    return rrqk::launch_pairs_order<2, 8, 4>(mixed, a, shape, st);
}

cudaError_t rrq_launch_pairs_eval_p2(const PairArgs &a, const PairShape &shape, cudaStream_t st) {
    return rrqk::launch_pairs_eval_order<2, 8, 4>(a, shape, st);
}

int rrq_pair_tiles_p2(int out[4]) { return rrqk::tiles_of<8, 4>(out); }
