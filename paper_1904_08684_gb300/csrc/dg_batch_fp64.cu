// Batched persistent stage kernel, double state / double velocity solve.
#include "dg_batch.cuh"
namespace dgswe {
DGSWE_DEFINE_BATCH(fp64, double, double)
}  // namespace dgswe
