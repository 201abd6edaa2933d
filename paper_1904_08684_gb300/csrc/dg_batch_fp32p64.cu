// Batched persistent stage kernel, float state / double velocity solve.
#include "dg_batch.cuh"
namespace dgswe {
DGSWE_DEFINE_BATCH(fp32p64, float, double)
}  // namespace dgswe
