// dg_launch.cuh -- launch entry points shared by the per-precision
// translation units (each one instantiates the kernels for one arithmetic).
#pragma once

#include <cuda_runtime.h>

#include <cmath>

#include "dg_kernels.cuh"

namespace dgswe {

// arithmetic of one context: state/contractions and velocity solve
enum Arith { ARITH_FP64 = 0, ARITH_FP32_P64 = 1, ARITH_FP32_P32 = 2 };

// Launch one stage_kernel.  params points to a StageParams<double> (FP64) or
// StageParams<float>.  Returns the launch error.
cudaError_t launch_diag(int arith, int p, const Mesh& m, const void* w, const void* hb, double det, double g,
                        double* partial, cudaStream_t s);

template <class Real>
inline long long grid_for(long long E, int block) {
  return (E + block - 1) / block;
}

// stage launchers of one arithmetic and feature set (one translation unit each)
#define DGSWE_DEFINE_STAGE(SUFFIX, REAL, PREAL, FEAT)                                                     \
  template <int P, int MODE>                                                                               \
  static cudaError_t stage_##SUFFIX##_pm(int block, const void* params, cudaStream_t s) {                  \
    const StageParams<REAL>& sp = *static_cast<const StageParams<REAL>*>(params);                          \
    const long long g = (sp.m.E + block - 1) / block;                                                      \
    stage_kernel<P, REAL, PREAL, MODE, FEAT><<<(unsigned)g, block, 0, s>>>(sp);                            \
    return cudaGetLastError();                                                                             \
  }                                                                                                        \
  template <int P>                                                                                         \
  static cudaError_t stage_##SUFFIX##_p(int mode, int block, const void* params, cudaStream_t s) {         \
    if (mode == MODE_EVAL) return stage_##SUFFIX##_pm<P, MODE_EVAL>(block, params, s);                     \
    if (mode == MODE_STAGE) return stage_##SUFFIX##_pm<P, MODE_STAGE>(block, params, s);                   \
    return stage_##SUFFIX##_pm<P, MODE_RHS>(block, params, s);                                             \
  }                                                                                                        \
  cudaError_t stage_##SUFFIX(int p, int mode, int block, const void* params, cudaStream_t s) {             \
    switch (p) {                                                                                           \
      case 1: return stage_##SUFFIX##_p<1>(mode, block, params, s);                                        \
      case 2: return stage_##SUFFIX##_p<2>(mode, block, params, s);                                        \
      case 3: return stage_##SUFFIX##_p<3>(mode, block, params, s);                                        \
      case 4: return stage_##SUFFIX##_p<4>(mode, block, params, s);                                        \
    }                                                                                                      \
    return cudaErrorInvalidValue;                                                                          \
  }

// set-up and diagnostics launchers of one arithmetic
#define DGSWE_DEFINE_AUX(SUFFIX, REAL, PREAL)                                                              \
  cudaError_t static_##SUFFIX(int p, const Mesh& m, double gg, const double* hb64, void* hb, void* hbt,    \
                              void* ghb, void* lin, cudaStream_t s) {                                      \
    const unsigned g = (unsigned)((m.E + 127) / 128);                                                      \
    REAL *a = (REAL*)hb, *b = (REAL*)hbt, *c = (REAL*)ghb, *d = (REAL*)lin;                                \
    switch (p) {                                                                                           \
      case 1: static_kernel<1, REAL><<<g, 128, 0, s>>>(m, gg, hb64, a, b, c, d); break;                    \
      case 2: static_kernel<2, REAL><<<g, 128, 0, s>>>(m, gg, hb64, a, b, c, d); break;                    \
      case 3: static_kernel<3, REAL><<<g, 128, 0, s>>>(m, gg, hb64, a, b, c, d); break;                    \
      case 4: static_kernel<4, REAL><<<g, 128, 0, s>>>(m, gg, hb64, a, b, c, d); break;                    \
      default: return cudaErrorInvalidValue;                                                               \
    }                                                                                                      \
    return cudaGetLastError();                                                                             \
  }                                                                                                        \
  cudaError_t diag_##SUFFIX(int p, const Mesh& m, const void* w, const void* hb, double det, double gg,    \
                            double* partial, cudaStream_t s) {                                             \
    const unsigned g = (unsigned)((m.E + 127) / 128);                                                      \
    const REAL *a = (const REAL*)w, *b = (const REAL*)hb;                                                  \
    switch (p) {                                                                                           \
      case 1: diag_kernel<1, REAL, PREAL><<<g, 128, 0, s>>>(m, a, b, det, gg, partial); break;             \
      case 2: diag_kernel<2, REAL, PREAL><<<g, 128, 0, s>>>(m, a, b, det, gg, partial); break;             \
      case 3: diag_kernel<3, REAL, PREAL><<<g, 128, 0, s>>>(m, a, b, det, gg, partial); break;             \
      case 4: diag_kernel<4, REAL, PREAL><<<g, 128, 0, s>>>(m, a, b, det, gg, partial); break;             \
      default: return cudaErrorInvalidValue;                                                               \
    }                                                                                                      \
    return cudaGetLastError();                                                                             \
  }

cudaError_t stage_fp64(int p, int mode, int block, const void* params, cudaStream_t s);
cudaError_t stage_fp32p64(int p, int mode, int block, const void* params, cudaStream_t s);
cudaError_t stage_fp32p32(int p, int mode, int block, const void* params, cudaStream_t s);
cudaError_t stage_fp64_gen(int p, int mode, int block, const void* params, cudaStream_t s);
cudaError_t stage_fp32p64_gen(int p, int mode, int block, const void* params, cudaStream_t s);
cudaError_t stage_fp32p32_gen(int p, int mode, int block, const void* params, cudaStream_t s);
// static fields of the bathymetry; lin (FP64 contexts only, else null):
// [2][K][K][E] matrices of the terms linear in xi
cudaError_t static_fp64(int p, const Mesh& m, double g, const double* hb64, void* hb, void* hbt, void* ghb, void* lin,
                        cudaStream_t s);
cudaError_t static_fp32p64(int p, const Mesh& m, double g, const double* hb64, void* hb, void* hbt, void* ghb,
                           void* lin, cudaStream_t s);
cudaError_t static_fp32p32(int p, const Mesh& m, double g, const double* hb64, void* hb, void* hbt, void* ghb,
                           void* lin, cudaStream_t s);

// fill the derived geometry of a uniform mesh
inline Mesh make_mesh(int nx, int ny, double x0, double y0, double Lx, double Ly, bool periodic) {
  Mesh m;
  m.nx = nx;
  m.ny = ny;
  m.E = 2LL * nx * ny;
  m.x0 = x0;
  m.y0 = y0;
  m.geo = nullptr;
  m.hx = Lx / nx;
  m.hy = Ly / ny;
  m.diag = std::hypot(m.hx, m.hy);
  m.ndx = m.hy / m.diag;
  m.ndy = m.hx / m.diag;
  m.periodic = periodic ? 1 : 0;
  return m;
}
cudaError_t diag_fp64(int p, const Mesh& m, const void* w, const void* hb, double det, double g, double* partial,
                      cudaStream_t s);
cudaError_t diag_fp32p64(int p, const Mesh& m, const void* w, const void* hb, double det, double g,
                         double* partial, cudaStream_t s);
cudaError_t diag_fp32p32(int p, const Mesh& m, const void* w, const void* hb, double det, double g,
                         double* partial, cudaStream_t s);

}  // namespace dgswe
