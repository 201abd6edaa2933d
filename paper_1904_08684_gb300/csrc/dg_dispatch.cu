// Order (and mode) dispatch of the separately compiled launchers:
// stage_<suffix>(p, ...) calls stage_<suffix>_p<p> (dg_stage_inst.cu),
// static_/diag_<suffix>(p, ...) call *_p<p> (dg_aux_inst.cu) and
// batch_launch_<suffix>(mode, ...) calls batch_launch_<suffix>_m<mode>
// (dg_batch_inst.cu).  Orders outside 0..4 return cudaErrorInvalidValue.
#include "dg_batch.cuh"
#include "dg_launch.cuh"
#include "dg_tile.cuh"

namespace dgswe {

#define DGSWE_DISPATCH(SUFFIX)                                                                  \
  cudaError_t stage_##SUFFIX(int p, int mode, int block, const void* params, cudaStream_t s) {         \
    switch (p) {                                                                                      \
      case 0: return stage_##SUFFIX##_p0(mode, block, params, s);                                      \
      case 1: return stage_##SUFFIX##_p1(mode, block, params, s);                                      \
      case 2: return stage_##SUFFIX##_p2(mode, block, params, s);                                      \
      case 3: return stage_##SUFFIX##_p3(mode, block, params, s);                                      \
      case 4: return stage_##SUFFIX##_p4(mode, block, params, s);                                      \
    }                                                                                                 \
    return cudaErrorInvalidValue;                                                                     \
  }

DGSWE_DISPATCH(fp64)
DGSWE_DISPATCH(fp32p64)
DGSWE_DISPATCH(fp32p32)
DGSWE_DISPATCH(fp64_gen)
DGSWE_DISPATCH(fp32p64_gen)
DGSWE_DISPATCH(fp32p32_gen)
DGSWE_DISPATCH(fp32pdf)
DGSWE_DISPATCH(fp32pir)

#define DGSWE_TILE_DISPATCH(SUFFIX)                                                                   \
  cudaError_t tile_##SUFFIX(int p, int shape, const StageParams<float>& sp, cudaStream_t s) {          \
    switch (p) {                                                                                      \
      case 0: return tile_##SUFFIX##_p0(shape, sp, s);                                                \
      case 1: return tile_##SUFFIX##_p1(shape, sp, s);                                                \
      case 2: return tile_##SUFFIX##_p2(shape, sp, s);                                                \
      case 3: return tile_##SUFFIX##_p3(shape, sp, s);                                                \
      case 4: return tile_##SUFFIX##_p4(shape, sp, s);                                                \
    }                                                                                                 \
    return cudaErrorInvalidValue;                                                                     \
  }
#define DGSWE_BATCH_TILE_DISPATCH(SUFFIX)                                                                \
  cudaError_t batch_tile_launch_##SUFFIX(int p, int shape, int grid, const BatchArgs& a, cudaStream_t s) { \
    switch (p) {                                                                                        \
      case 1: return batch_tile_launch_##SUFFIX##_p1(shape, grid, a, s);                                \
      case 2: return batch_tile_launch_##SUFFIX##_p2(shape, grid, a, s);                                \
      case 3: return batch_tile_launch_##SUFFIX##_p3(shape, grid, a, s);                                \
    }                                                                                                   \
    return cudaErrorInvalidValue;                                                                       \
  }                                                                                                     \
  cudaError_t batch_tile_occupancy_##SUFFIX(int p, int shape, int* blocks_per_sm) {                     \
    switch (p) {                                                                                        \
      case 1: return batch_tile_occupancy_##SUFFIX##_p1(shape, blocks_per_sm);                          \
      case 2: return batch_tile_occupancy_##SUFFIX##_p2(shape, blocks_per_sm);                          \
      case 3: return batch_tile_occupancy_##SUFFIX##_p3(shape, blocks_per_sm);                          \
    }                                                                                                   \
    return cudaErrorInvalidValue;                                                                       \
  }
DGSWE_BATCH_TILE_DISPATCH(fp32p64)
DGSWE_BATCH_TILE_DISPATCH(fp32p32)
DGSWE_BATCH_TILE_DISPATCH(fp32pdf)
DGSWE_BATCH_TILE_DISPATCH(fp32pir)

DGSWE_TILE_DISPATCH(fp32p64)
DGSWE_TILE_DISPATCH(fp32p32)
DGSWE_TILE_DISPATCH(fp32pdf)
DGSWE_TILE_DISPATCH(fp32pir)
cudaError_t tile_fp32pdf_p4(int, const StageParams<float>&, cudaStream_t) { return cudaErrorInvalidValue; }

// the double-float velocity solve is built for p <= 3: its p = 4 entries
// reject the call
cudaError_t stage_fp32pdf_p4(int, int, const void*, cudaStream_t) { return cudaErrorInvalidValue; }
cudaError_t static_fp32pdf_p4(const Mesh&, double, const double*, void*, void*, void*, void*, cudaStream_t) {
  return cudaErrorInvalidValue;
}
cudaError_t diag_fp32pdf_p4(const Mesh&, const void*, const void*, double, double, double*, cudaStream_t) {
  return cudaErrorInvalidValue;
}

#define DGSWE_BATCH_DISPATCH(SUFFIX)                                                                  \
  cudaError_t batch_launch_##SUFFIX(int mode, int grid, int block, const BatchArgs& a, cudaStream_t s) { \
    return mode == MODE_EVAL ? batch_launch_##SUFFIX##_m0(grid, block, a, s)                           \
                             : batch_launch_##SUFFIX##_m1(grid, block, a, s);                          \
  }                                                                                                   \
  cudaError_t batch_occupancy_##SUFFIX(int block, int* blocks_per_sm) {                               \
    int a = 0, b = 0;                                                                                 \
    cudaError_t e = batch_occupancy_##SUFFIX##_m0(block, &a);                                         \
    if (e == cudaSuccess) e = batch_occupancy_##SUFFIX##_m1(block, &b);                               \
    *blocks_per_sm = a < b ? a : b;                                                                   \
    return e;                                                                                         \
  }

#define DGSWE_AUX_DISPATCH(SUFFIX)                                                                     \
  cudaError_t static_##SUFFIX(int p, const Mesh& m, double gg, const double* hb64, void* hb, void* hbt,         \
                              void* ghb, void* lin, cudaStream_t s) {                                           \
    switch (p) {                                                                                                \
      case 0: return static_##SUFFIX##_p0(m, gg, hb64, hb, hbt, ghb, lin, s);                                   \
      case 1: return static_##SUFFIX##_p1(m, gg, hb64, hb, hbt, ghb, lin, s);                                   \
      case 2: return static_##SUFFIX##_p2(m, gg, hb64, hb, hbt, ghb, lin, s);                                   \
      case 3: return static_##SUFFIX##_p3(m, gg, hb64, hb, hbt, ghb, lin, s);                                   \
      case 4: return static_##SUFFIX##_p4(m, gg, hb64, hb, hbt, ghb, lin, s);                                   \
    }                                                                                                           \
    return cudaErrorInvalidValue;                                                                               \
  }                                                                                                             \
  cudaError_t diag_##SUFFIX(int p, const Mesh& m, const void* w, const void* hb, double det, double gg,         \
                            double* partial, cudaStream_t s) {                                                  \
    switch (p) {                                                                                                \
      case 0: return diag_##SUFFIX##_p0(m, w, hb, det, gg, partial, s);                                         \
      case 1: return diag_##SUFFIX##_p1(m, w, hb, det, gg, partial, s);                                         \
      case 2: return diag_##SUFFIX##_p2(m, w, hb, det, gg, partial, s);                                         \
      case 3: return diag_##SUFFIX##_p3(m, w, hb, det, gg, partial, s);                                         \
      case 4: return diag_##SUFFIX##_p4(m, w, hb, det, gg, partial, s);                                         \
    }                                                                                                           \
    return cudaErrorInvalidValue;                                                                               \
  }

// set-up and diagnostics
DGSWE_AUX_DISPATCH(fp64)
DGSWE_AUX_DISPATCH(fp32p64)
DGSWE_AUX_DISPATCH(fp32p32)
DGSWE_AUX_DISPATCH(fp32pdf)
DGSWE_AUX_DISPATCH(fp32pir)

// static bathymetry matrix of the mixed solve (the low parts of its FP64 sums; at
// p = 4 also the FP32 parts, see ahb_keeps_hi)
cudaError_t static_ahb(int p, const Mesh& m, const double* hb64, float* ahb, cudaStream_t s) {
  const unsigned g = (unsigned)((m.E + 127) / 128);
  switch (p) {
    case 0: ahb_kernel<0><<<g, 128, 0, s>>>(m.E, hb64, ahb); break;
    case 1: ahb_kernel<1><<<g, 128, 0, s>>>(m.E, hb64, ahb); break;
    case 2: ahb_kernel<2><<<g, 128, 0, s>>>(m.E, hb64, ahb); break;
    case 3: ahb_kernel<3><<<g, 128, 0, s>>>(m.E, hb64, ahb); break;
    case 4: ahb_kernel<4><<<g, 128, 0, s>>>(m.E, hb64, ahb); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// batched persistent kernel: mode 0 = evaluation, 1 = stage
DGSWE_BATCH_DISPATCH(fp64)
DGSWE_BATCH_DISPATCH(fp32p64)
DGSWE_BATCH_DISPATCH(fp32p32)
DGSWE_BATCH_DISPATCH(fp32pdf)
DGSWE_BATCH_DISPATCH(fp32pir)

}  // namespace dgswe
