// dg_launch.cuh -- launch entry points of the stage, set-up and diagnostics
// kernels, shared by the instantiation units and the host API.
#pragma once

#include <cuda_runtime.h>

#include <cmath>

#include "dg_kernels.cuh"

namespace dgswe {

// arithmetic of one context: state/contractions and velocity solve
enum Arith { ARITH_FP64 = 0, ARITH_FP32_P64 = 1, ARITH_FP32_P32 = 2, ARITH_FP32_PDF = 3, ARITH_FP32_PIR = 4 };

// arithmetic of a configuration (precision and velocity-solve precision)
inline int arith_of(int precision, int proj_precision) {
  if (precision == 0) return ARITH_FP64;
  switch (proj_precision) {
    case 1: return ARITH_FP32_P32;
    case 2: return ARITH_FP32_PDF;
    case 3: return ARITH_FP32_PIR;
    default: return ARITH_FP32_P64;
  }
}

// Stage launchers.  Each (arithmetic, feature set, order) combination is
// compiled separately from dg_stage_inst.cu (build flags select it), so the
// build runs many small compilations in parallel; the per-arithmetic
// dispatchers stage_<suffix>(p, ...) live in dg_dispatch.cu.
#define DGSWE_PASTE4(a, b, c, d) a##b##c##d
#define DGSWE_STAGE_NAME(SUFFIX, P) DGSWE_PASTE4(stage_, SUFFIX, _p, P)
#define DGSWE_DECLARE_STAGE_P(SUFFIX, P) \
  cudaError_t DGSWE_STAGE_NAME(SUFFIX, P)(int mode, int block, const void* params, cudaStream_t s);

template <int P, class REAL, class PREAL, int FEAT, int MODE>
cudaError_t launch_stage_pm(int block, const void* params, cudaStream_t s) {
  const StageParams<REAL>& sp = *static_cast<const StageParams<REAL>*>(params);
  long long g = (sp.m.E + block - 1) / block;
  if (std::is_same<REAL, float>::value) {
    // FP32 state: a persistent grid of the resident CTAs (no partial last
    // wave; measured 2-10 % faster).  FP64 keeps one CTA per element block
    // (the capped grid measured 0.8 % slower there).
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stage_kernel<P, REAL, PREAL, MODE, FEAT>, block, 0);
    if (e != cudaSuccess) return e;
    const long long resident = (long long)sms * (per_sm > 0 ? per_sm : 1);
    if (g > resident) g = resident;
  }
  stage_kernel<P, REAL, PREAL, MODE, FEAT><<<(unsigned)g, block, 0, s>>>(sp);
  return cudaGetLastError();
}

template <int P, class REAL, class PREAL, int FEAT>
cudaError_t launch_stage_p(int mode, int block, const void* params, cudaStream_t s) {
  if (mode == MODE_EVAL) return launch_stage_pm<P, REAL, PREAL, FEAT, MODE_EVAL>(block, params, s);
  if (mode == MODE_STAGE) return launch_stage_pm<P, REAL, PREAL, FEAT, MODE_STAGE>(block, params, s);
  return launch_stage_pm<P, REAL, PREAL, FEAT, MODE_RHS>(block, params, s);
}

// Set-up (bathymetry fields) and diagnostics launchers of one arithmetic
// and order, compiled separately from dg_aux_inst.cu; the dispatchers
// static_<suffix>(p, ...) and diag_<suffix>(p, ...) live in dg_dispatch.cu.
#define DGSWE_STATIC_NAME(SUFFIX, P) DGSWE_PASTE4(static_, SUFFIX, _p, P)
#define DGSWE_DIAG_NAME(SUFFIX, P) DGSWE_PASTE4(diag_, SUFFIX, _p, P)
#define DGSWE_DECLARE_AUX_P(SUFFIX, P)                                                                   \
  cudaError_t DGSWE_STATIC_NAME(SUFFIX, P)(const Mesh& m, double gg, const double* hb64, void* hb, void* hbt, \
                                           void* ghb, void* lin, cudaStream_t s);                         \
  cudaError_t DGSWE_DIAG_NAME(SUFFIX, P)(const Mesh& m, const void* w, const void* hb, double det, double gg, \
                                         double* partial, cudaStream_t s);
#define DGSWE_DECLARE_AUX_ALL(SUFFIX) \
  DGSWE_DECLARE_AUX_P(SUFFIX, 0)      \
  DGSWE_DECLARE_AUX_P(SUFFIX, 1)      \
  DGSWE_DECLARE_AUX_P(SUFFIX, 2)      \
  DGSWE_DECLARE_AUX_P(SUFFIX, 3)      \
  DGSWE_DECLARE_AUX_P(SUFFIX, 4)
DGSWE_DECLARE_AUX_ALL(fp64)
DGSWE_DECLARE_AUX_ALL(fp32p64)
DGSWE_DECLARE_AUX_ALL(fp32p32)
DGSWE_DECLARE_AUX_ALL(fp32pdf)
DGSWE_DECLARE_AUX_ALL(fp32pir)

template <int P, class REAL>
cudaError_t launch_static_p(const Mesh& m, double gg, const double* hb64, void* hb, void* hbt, void* ghb, void* lin,
                            cudaStream_t s) {
  const unsigned g = (unsigned)((m.E + 127) / 128);
  static_kernel<P, REAL><<<g, 128, 0, s>>>(m, gg, hb64, (REAL*)hb, (REAL*)hbt, (REAL*)ghb, (REAL*)lin);
  return cudaGetLastError();
}

template <int P, class REAL, class PREAL>
cudaError_t launch_diag_p(const Mesh& m, const void* w, const void* hb, double det, double gg, double* partial,
                          cudaStream_t s) {
  const unsigned g = (unsigned)((m.E + 127) / 128);
  diag_kernel<P, REAL, PREAL><<<g, 128, 0, s>>>(m, (const REAL*)w, (const REAL*)hb, det, gg, partial);
  return cudaGetLastError();
}

#define DGSWE_DECLARE_STAGE_ALL(SUFFIX) \
  DGSWE_DECLARE_STAGE_P(SUFFIX, 0)      \
  DGSWE_DECLARE_STAGE_P(SUFFIX, 1)      \
  DGSWE_DECLARE_STAGE_P(SUFFIX, 2)      \
  DGSWE_DECLARE_STAGE_P(SUFFIX, 3)      \
  DGSWE_DECLARE_STAGE_P(SUFFIX, 4)
DGSWE_DECLARE_STAGE_ALL(fp64)
DGSWE_DECLARE_STAGE_ALL(fp32p64)
DGSWE_DECLARE_STAGE_ALL(fp32p32)
DGSWE_DECLARE_STAGE_ALL(fp32pdf)
DGSWE_DECLARE_STAGE_ALL(fp32pir)
DGSWE_DECLARE_STAGE_ALL(fp64_gen)
DGSWE_DECLARE_STAGE_ALL(fp32p64_gen)
DGSWE_DECLARE_STAGE_ALL(fp32p32_gen)

cudaError_t stage_fp64(int p, int mode, int block, const void* params, cudaStream_t s);
cudaError_t stage_fp32p64(int p, int mode, int block, const void* params, cudaStream_t s);
cudaError_t stage_fp32p32(int p, int mode, int block, const void* params, cudaStream_t s);
cudaError_t stage_fp32pdf(int p, int mode, int block, const void* params, cudaStream_t s);
cudaError_t stage_fp32pir(int p, int mode, int block, const void* params, cudaStream_t s);
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
cudaError_t static_fp32pdf(int p, const Mesh& m, double g, const double* hb64, void* hb, void* hbt, void* ghb,
                           void* lin, cudaStream_t s);
cudaError_t static_fp32pir(int p, const Mesh& m, double g, const double* hb64, void* hb, void* hbt, void* ghb,
                           void* lin, cudaStream_t s);

// static bathymetry matrix of the mixed solve: ahb [K(K+1)/2][E] low parts
cudaError_t static_ahb(int p, const Mesh& m, const double* hb64, float* ahb, cudaStream_t s);

// FP64 element-major [F][E][K] <-> context-precision SoA [F][K][E] on the device
template <class Real>
__global__ void aos_to_soa_kernel(const double* __restrict__ a, Real* __restrict__ b, long long E, int K, int F) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  for (int f = 0; f < F; ++f)
    for (int i = 0; i < K; ++i) b[((long long)f * K + i) * E + e] = Real(a[((long long)f * E + e) * K + i]);
}
template <class Real>
__global__ void soa_to_aos_kernel(const Real* __restrict__ b, double* __restrict__ a, long long E, int K, int F) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  for (int f = 0; f < F; ++f)
    for (int i = 0; i < K; ++i) a[((long long)f * E + e) * K + i] = double(b[((long long)f * K + i) * E + e]);
}

// Three element-major FP64 arrays [E][K] (xi, q_x, q_y) that the device reads
// or writes directly in host memory (page-locked and mapped), <-> the
// context-precision SoA state [3][K][E].  One thread per host word, in the
// host arrays' order, so that the traffic over the host link is coalesced
// (the device side, scattered by K rows, merges in L2).  A null field is
// skipped.
struct HostFields {
  double* f[3];
};
template <class Real>
__global__ void __launch_bounds__(256) fields_to_soa_kernel(HostFields a, Real* __restrict__ b, long long E, int K) {
  const long long n = E * K;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < 3 * n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(idx / n);
    const long long r = idx - f * n, e = r / K;
    const int i = (int)(r - e * K);
    if (a.f[f]) b[((long long)f * K + i) * E + e] = Real(a.f[f][r]);
  }
}
template <class Real>
__global__ void __launch_bounds__(256) soa_to_fields_kernel(const Real* __restrict__ b, HostFields a, long long E,
                                                           int K) {
  const long long n = E * K;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < 3 * n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(idx / n);
    const long long r = idx - f * n, e = r / K;
    const int i = (int)(r - e * K);
    if (a.f[f]) a.f[f][r] = double(b[((long long)f * K + i) * E + e]);
  }
}
inline unsigned fields_grid(long long E, int K) {
  const long long blocks = (3 * E * K + 255) / 256;
  return (unsigned)(blocks < 4096 ? (blocks > 0 ? blocks : 1) : 4096);
}

// Device address of a host array of `bytes` bytes that kernels may access in
// place: page-locked memory mapped into the device's address space
// (cudaHostAlloc, cudaHostRegister), checked at its first and last byte;
// null for any other memory (pageable arrays go through copies instead).
inline double* mapped_host(const double* p, size_t bytes) {
  if (!p || bytes == 0) return nullptr;
  cudaPointerAttributes a0, a1;
  if (cudaPointerGetAttributes(&a0, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  const char* last = (const char*)p + bytes - 1;
  if (cudaPointerGetAttributes(&a1, last) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a0.type != cudaMemoryTypeHost || a1.type != cudaMemoryTypeHost || !a0.devicePointer || !a1.devicePointer)
    return nullptr;
  if ((const char*)a1.devicePointer - (const char*)a0.devicePointer != (long long)bytes - 1) return nullptr;
  return (double*)a0.devicePointer;
}

// The three fields' device addresses (n doubles each; null stays null) when
// every non-null field is mapped host memory and at least one is given
inline bool mapped_fields(double* const* p, long long n, HostFields& hf) {
  bool any = false;
  for (int f = 0; f < 3; ++f) {
    hf.f[f] = nullptr;
    if (!p[f]) continue;
    hf.f[f] = mapped_host(p[f], sizeof(double) * (size_t)n);
    if (!hf.f[f]) return false;
    any = true;
  }
  return any;
}

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
  m.fhx = float(m.hx);
  m.fhy = float(m.hy);
  m.fdiag = float(m.diag);
  m.fndx = float(m.ndx);
  m.fndy = float(m.ndy);
  return m;
}
cudaError_t diag_fp64(int p, const Mesh& m, const void* w, const void* hb, double det, double g, double* partial,
                      cudaStream_t s);
cudaError_t diag_fp32p64(int p, const Mesh& m, const void* w, const void* hb, double det, double g,
                         double* partial, cudaStream_t s);
cudaError_t diag_fp32p32(int p, const Mesh& m, const void* w, const void* hb, double det, double g,
                         double* partial, cudaStream_t s);
cudaError_t diag_fp32pdf(int p, const Mesh& m, const void* w, const void* hb, double det, double g,
                         double* partial, cudaStream_t s);
cudaError_t diag_fp32pir(int p, const Mesh& m, const void* w, const void* hb, double det, double g,
                         double* partial, cudaStream_t s);

}  // namespace dgswe
