// General meshes, §3.1 body force and Dirichlet edges: float state, double velocity solve.
#include "dg_launch.cuh"
namespace dgswe {
DGSWE_DEFINE_STAGE(fp32p64_gen, float, double, 1)
}  // namespace dgswe
