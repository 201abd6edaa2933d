// One instantiation of the stage kernels, selected at build time:
//   DG_SUFFIX (launcher name), DG_REAL / DG_PREAL (state and velocity-solve
//   arithmetic), DG_FEAT (0 uniform mesh, 1 general features), DG_P (order).
// build.py compiles this file once per combination.
#include "dg_launch.cuh"

namespace dgswe {

cudaError_t DGSWE_STAGE_NAME(DG_SUFFIX, DG_P)(int mode, int block, const void* params, cudaStream_t s) {
  return launch_stage_p<DG_P, DG_REAL, DG_PREAL, DG_FEAT>(mode, block, params, s);
}

}  // namespace dgswe
