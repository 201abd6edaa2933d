// Instantiation of the tile-fused batched stage kernels of one velocity-solve
// arithmetic and order, selected at build time: DG_SUFFIX (launcher name),
// DG_PREAL (velocity-solve arithmetic), DG_P (order, 1..3); every tile
// shape.  build.py compiles this file once per combination; dg_dispatch.cu
// maps the run-time order to it.
#include "dg_batch.cuh"

#define DGSWE_BT_PASTE(a, b, c, d) a##b##c##d
#define DGSWE_BT_NAME(WHAT, SUFFIX, P) DGSWE_BT_PASTE(WHAT, SUFFIX, _p, P)

namespace dgswe {

cudaError_t DGSWE_BT_NAME(batch_tile_launch_, DG_SUFFIX, DG_P)(int shape, int grid, const BatchArgs& a,
                                                               cudaStream_t s) {
  return batch_tile_launch_p<DG_PREAL, DG_P>(shape, grid, a, s);
}

cudaError_t DGSWE_BT_NAME(batch_tile_occupancy_, DG_SUFFIX, DG_P)(int shape, int* blocks_per_sm) {
  return batch_tile_occupancy_p<DG_PREAL, DG_P>(shape, blocks_per_sm);
}

}  // namespace dgswe
