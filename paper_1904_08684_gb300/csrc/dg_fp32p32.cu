// FP32 everywhere, including the velocity solve (evaluated alternative).
#include "dg_launch.cuh"
namespace dgswe {
DGSWE_DEFINE_LAUNCHERS(fp32p32, float, float)
}  // namespace dgswe
