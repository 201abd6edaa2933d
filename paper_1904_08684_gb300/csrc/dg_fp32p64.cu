// FP32 state and contractions, FP64 velocity solve.
#include "dg_launch.cuh"
namespace dgswe {
DGSWE_DEFINE_LAUNCHERS(fp32p64, float, double)
}  // namespace dgswe
