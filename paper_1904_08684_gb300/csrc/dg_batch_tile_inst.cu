// One instantiation of the tile-fused batched stage kernel, selected at
// build time: DG_SUFFIX (launcher name), DG_PREAL (velocity-solve
// arithmetic); all tile shapes.  build.py compiles this file once per
// arithmetic.
#include "dg_batch.cuh"

#define DGSWE_BT_PASTE(a, b) a##b
#define DGSWE_BT_NAME(WHAT, SUFFIX) DGSWE_BT_PASTE(WHAT, SUFFIX)

namespace dgswe {

cudaError_t DGSWE_BT_NAME(batch_tile_launch_, DG_SUFFIX)(int shape, int grid, const BatchArgs& a, cudaStream_t s) {
  if (shape == 1) return batch_tile_launch_shape<DG_PREAL, 16, 8>(grid, a, s);
  if (shape == 2) return batch_tile_launch_shape<DG_PREAL, 8, 4>(grid, a, s);
  return batch_tile_launch_shape<DG_PREAL, 8, 8>(grid, a, s);
}

cudaError_t DGSWE_BT_NAME(batch_tile_occupancy_, DG_SUFFIX)(int shape, int* blocks_per_sm) {
  if (shape == 1) return batch_tile_occupancy_shape<DG_PREAL, 16, 8>(blocks_per_sm);
  if (shape == 2) return batch_tile_occupancy_shape<DG_PREAL, 8, 4>(blocks_per_sm);
  return batch_tile_occupancy_shape<DG_PREAL, 8, 8>(blocks_per_sm);
}

}  // namespace dgswe
