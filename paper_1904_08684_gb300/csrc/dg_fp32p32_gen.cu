// General meshes, §3.1 body force and Dirichlet edges: float state, float velocity solve.
#include "dg_launch.cuh"
namespace dgswe {
DGSWE_DEFINE_STAGE(fp32p32_gen, float, float, 1)
}  // namespace dgswe
