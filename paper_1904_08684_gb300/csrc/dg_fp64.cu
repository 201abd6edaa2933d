// FP64 instantiations: state, contractions and velocity solve in double.
#include "dg_launch.cuh"
namespace dgswe {
DGSWE_DEFINE_LAUNCHERS(fp64, double, double)
}  // namespace dgswe
