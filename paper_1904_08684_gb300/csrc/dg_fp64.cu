// FP64 instantiations: state, contractions and velocity solve in double.
#include "dg_launch.cuh"
namespace dgswe {
DGSWE_DEFINE_STAGE(fp64, double, double, 0)
DGSWE_DEFINE_AUX(fp64, double, double)
}  // namespace dgswe
