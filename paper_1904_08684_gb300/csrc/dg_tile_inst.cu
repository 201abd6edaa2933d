// One instantiation of the tile-fused FP32 stage kernel, selected at build
// time: DG_SUFFIX (launcher name), DG_PREAL (velocity-solve arithmetic),
// DG_P (order).  build.py compiles this file once per combination.
#include "dg_tile.cuh"

namespace dgswe {

cudaError_t DGSWE_TILE_NAME(DG_SUFFIX, DG_P)(int shape, const StageParams<float>& sp, cudaStream_t s) {
  return launch_tile_p<DG_P, DG_PREAL>(shape, sp, s);
}

}  // namespace dgswe
