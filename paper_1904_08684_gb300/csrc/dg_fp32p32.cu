// FP32 everywhere, including the velocity solve (evaluated alternative).
#include "dg_launch.cuh"
namespace dgswe {
DGSWE_DEFINE_STAGE(fp32p32, float, float, 0)
DGSWE_DEFINE_AUX(fp32p32, float, float)
}  // namespace dgswe
