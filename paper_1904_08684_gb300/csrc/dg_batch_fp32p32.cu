// Batched persistent stage kernel, float state / float velocity solve.
#include "dg_batch.cuh"
namespace dgswe {
DGSWE_DEFINE_BATCH(fp32p32, float, float)
}  // namespace dgswe
