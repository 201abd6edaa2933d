// General meshes, §3.1 body force and Dirichlet edges: double state, double velocity solve.
#include "dg_launch.cuh"
namespace dgswe {
DGSWE_DEFINE_STAGE(fp64_gen, double, double, 1)
}  // namespace dgswe
