// One instantiation of the batched persistent stage kernel, selected at build
// time: DG_SUFFIX, DG_REAL / DG_PREAL (state and velocity-solve arithmetic),
// DG_MODE (0 evaluation, 1 stage).  build.py compiles this file once per
// combination.
#include "dg_batch.cuh"

#define DGSWE_BATCH_PASTE(a, b, c, d) a##b##c##d
#define DGSWE_BATCH_NAME(WHAT, SUFFIX, M) DGSWE_BATCH_PASTE(WHAT, SUFFIX, _m, M)

namespace dgswe {

cudaError_t DGSWE_BATCH_NAME(batch_launch_, DG_SUFFIX, DG_MODE)(int grid, int block, const BatchArgs& a,
                                                              cudaStream_t s) {
  batch_kernel<DG_REAL, DG_PREAL, DG_MODE><<<grid, block, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t DGSWE_BATCH_NAME(batch_occupancy_, DG_SUFFIX, DG_MODE)(int block, int* blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, batch_kernel<DG_REAL, DG_PREAL, DG_MODE>,
                                                       block, 0);
}

}  // namespace dgswe
