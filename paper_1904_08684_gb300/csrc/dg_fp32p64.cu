// FP32 state and contractions, FP64 velocity solve.
#include "dg_launch.cuh"
namespace dgswe {
DGSWE_DEFINE_STAGE(fp32p64, float, double, 0)
DGSWE_DEFINE_AUX(fp32p64, float, double)
}  // namespace dgswe
