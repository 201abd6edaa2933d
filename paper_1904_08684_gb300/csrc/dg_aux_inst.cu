// Set-up (bathymetry fields) and diagnostics kernels of one arithmetic and
// order, selected at build time by DG_SUFFIX, DG_REAL, DG_PREAL, DG_P.
// build.py compiles this file once per combination.
#include "dg_launch.cuh"

namespace dgswe {

cudaError_t DGSWE_STATIC_NAME(DG_SUFFIX, DG_P)(const Mesh& m, double gg, const double* hb64, void* hb, void* hbt,
                                               void* ghb, void* lin, cudaStream_t s) {
  return launch_static_p<DG_P, DG_REAL>(m, gg, hb64, hb, hbt, ghb, lin, s);
}

cudaError_t DGSWE_DIAG_NAME(DG_SUFFIX, DG_P)(const Mesh& m, const void* w, const void* hb, double det, double gg,
                                             double* partial, cudaStream_t s) {
  return launch_diag_p<DG_P, DG_REAL, DG_PREAL>(m, w, hb, det, gg, partial, s);
}

}  // namespace dgswe
