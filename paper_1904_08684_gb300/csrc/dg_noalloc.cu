// dg_noalloc.cu -- dg_rhs_noalloc: the right-hand side of dg_rhs for callers
// that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running inside a CUDA graph that
// is being captured, allocator-free embedded runtimes, or host frameworks
// that forbid the library from touching the device heap after start-up.
// For them this entry point keeps every intermediate it needs (bathymetry
// traces and gradients, per-element volume integrals, edge side records and
// the error word) in one fixed array that lives in the library's device
// image: the array is reserved when the library's device code is loaded on a
// GPU and stays reserved on every GPU that loads the library until the
// process exits.  It calls no cudaMalloc, cudaFree or other allocating
// routine; the caller passes the bathymetry, the state and the output.
//
// The array is shared by every call on a device and keeps the previous
// call's contents; its error word is cleared at the start of each call.
// Calls whose GPU work overlaps (different streams or threads, no ordering
// between them) race on the array and produce wrong results.  A caller that
// wants to know whether the state was dry (a non-positive or NaN depth at
// a wave-speed point, or a projection matrix that is not positive
// definite) passes a device word of its own, which the kernels OR their
// flags into.
//
// The array's device address is looked up once per device and cached.  A
// cudaDeviceReset() unloads the library's device image, so the cached
// address no longer belongs to it: a process that resets a device must not
// call dg_rhs_noalloc on that device afterwards.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "dg_launch.cuh"
#include "dgswe.h"

using namespace dgswe;

namespace {

// 32 MiB: enough for about 24,000 FP64 triangles at p = 2 (1344 bytes each).
constexpr size_t kScratchBytes = size_t(32) << 20;
constexpr size_t kAlign = 256;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_scratch on the current device, looked up once per
// device.  In host code the name g_scratch is only a host-side stand-in, so
// its address must come from cudaGetSymbolAddress.
cudaError_t scratch_for_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    if (!p) return cudaErrorInvalidSymbol;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

size_t round_up(size_t n) { return (n + kAlign - 1) / kAlign * kAlign; }

template <class Real>
dg_status run(const dg_config* cfg, int arith, const double* d_hb, const void* d_in, void* d_out,
              unsigned* d_flags, cudaStream_t s) {
  const int P = cfg->p;
  const int K = (P + 1) * (P + 2) / 2, P1 = P + 1, NREC = 6 * P1 + 1;
  // bathymetry space P^max(p,1): basis size, edge modes, gradient basis
  const int PB = P > 0 ? P : 1, KB = (PB + 1) * (PB + 2) / 2, PB1 = PB + 1, KB1 = PB * (PB + 1) / 2;
  const long long E = 2LL * cfg->nx * cfg->ny;
  const size_t rs = sizeof(Real);
  // carve the array: error word, hb, hb traces, hb gradients, vs, records,
  // and in FP64 the matrices of the terms linear in xi
  const size_t o_err = 0;
  const size_t o_hb = o_err + round_up(sizeof(unsigned));
  const size_t o_hbt = o_hb + round_up((size_t)KB * E * rs);
  const size_t o_ghb = o_hbt + round_up((size_t)3 * PB1 * E * rs);
  const size_t o_vs = o_ghb + round_up((size_t)2 * KB1 * E * rs);
  const size_t o_rec = o_vs + round_up((size_t)3 * K * E * rs);
  const size_t o_lin = o_rec + round_up((size_t)3 * NREC * E * rs);
  const bool fp64 = arith == ARITH_FP64, mixed = arith == ARITH_FP32_PIR;
  const size_t o_ahb = o_lin + (fp64 ? round_up((size_t)2 * K * K * E * rs) : 0);
  const size_t total = o_ahb + (mixed ? round_up(sizeof(float) * ahb_words(K) * E) : 0);
  if (total > kScratchBytes) return DG_ERR_ARG;
  void* base = nullptr;
  cudaError_t e = scratch_for_current_device(&base);
  if (e != cudaSuccess) return DG_ERR_CUDA;
  unsigned char* b = static_cast<unsigned char*>(base);
  // the kernels OR their flags into the caller's word, else into the
  // array's own word (cleared per call, never read back)
  unsigned* err = d_flags ? d_flags : reinterpret_cast<unsigned*>(b + o_err);
  if (!d_flags && cudaMemsetAsync(err, 0, sizeof(unsigned), s) != cudaSuccess) return DG_ERR_CUDA;

  const Mesh m = make_mesh(cfg->nx, cfg->ny, cfg->x0, cfg->y0, cfg->Lx, cfg->Ly, cfg->bc == DG_BC_PERIODIC);
  const double hx = m.hx, hy = m.hy;
  void* lin = fp64 ? (void*)(b + o_lin) : nullptr;
  switch (arith) {
    case ARITH_FP64: e = static_fp64(P, m, cfg->g, d_hb, b + o_hb, b + o_hbt, b + o_ghb, lin, s); break;
    case ARITH_FP32_P64: e = static_fp32p64(P, m, cfg->g, d_hb, b + o_hb, b + o_hbt, b + o_ghb, nullptr, s); break;
    case ARITH_FP32_PDF: e = static_fp32pdf(P, m, cfg->g, d_hb, b + o_hb, b + o_hbt, b + o_ghb, nullptr, s); break;
    case ARITH_FP32_PIR:
      e = static_fp32pir(P, m, cfg->g, d_hb, b + o_hb, b + o_hbt, b + o_ghb, nullptr, s);
      if (e == cudaSuccess) e = static_ahb(P, m, d_hb, reinterpret_cast<float*>(b + o_ahb), s);
      break;
    default: e = static_fp32p32(P, m, cfg->g, d_hb, b + o_hb, b + o_hbt, b + o_ghb, nullptr, s); break;
  }
  if (e != cudaSuccess) return DG_ERR_CUDA;

  StageParams<Real> sp;
  std::memset(&sp, 0, sizeof sp);
  sp.m = m;
  sp.g = Real(cfg->g);
  sp.hb = reinterpret_cast<const Real*>(b + o_hb);
  sp.hbt = reinterpret_cast<const Real*>(b + o_hbt);
  sp.ghb = reinterpret_cast<const Real*>(b + o_ghb);
  sp.lin = static_cast<const Real*>(lin);
  sp.ahb = mixed ? reinterpret_cast<const float*>(b + o_ahb) : nullptr;
  sp.inv_det = 1.0 / (hx * hy);
  sp.det = hx * hy;
  sp.tau_bf = cfg->tau_bf;
  sp.f_c = cfg->f_c;
  sp.err = err;
  sp.w = static_cast<const Real*>(d_in);
  sp.vs_out = reinterpret_cast<Real*>(b + o_vs);
  sp.rec_out = reinterpret_cast<Real*>(b + o_rec);
  const int block = cfg->block_size ? cfg->block_size : 128;
  auto launch = [&](int mode) {
    switch (arith) {
      case ARITH_FP64: return stage_fp64(P, mode, block, &sp, s);
      case ARITH_FP32_P64: return stage_fp32p64(P, mode, block, &sp, s);
      case ARITH_FP32_PDF: return stage_fp32pdf(P, mode, block, &sp, s);
      case ARITH_FP32_PIR: return stage_fp32pir(P, mode, block, &sp, s);
      default: return stage_fp32p32(P, mode, block, &sp, s);
    }
  };
  if (launch(MODE_EVAL) != cudaSuccess) return DG_ERR_CUDA;
  sp.vs = sp.vs_out;
  sp.rec = sp.rec_out;
  sp.rhs_out = static_cast<Real*>(d_out);
  if (launch(MODE_RHS) != cudaSuccess) return DG_ERR_CUDA;
  return DG_OK;
}

}  // namespace

extern "C" dg_status dg_rhs_noalloc(const dg_config* cfg, const void* d_hb, const void* d_state_in,
                                    void* d_rhs_out, unsigned* d_flags, void* stream) {
  if (!cfg || !d_hb || !d_state_in || !d_rhs_out || d_state_in == d_rhs_out) return DG_ERR_ARG;
  if (cfg->nx < 1 || cfg->ny < 1 || cfg->p < 0 || cfg->p > 4 || !(cfg->Lx > 0.0) || !(cfg->Ly > 0.0) ||
      !(cfg->g > 0.0) || cfg->vertex_xy || cfg->bc < 0 || cfg->bc > 1 || cfg->precision < 0 ||
      cfg->precision > 1 || cfg->proj_precision < 0 || cfg->proj_precision > 3)
    return DG_ERR_ARG;
  if (cfg->bc == DG_BC_PERIODIC && (cfg->nx < 2 || cfg->ny < 2)) return DG_ERR_ARG;
  if (!(cfg->tau_bf >= 0.0) || !std::isfinite(cfg->tau_bf) || !std::isfinite(cfg->f_c)) return DG_ERR_ARG;
  if (cfg->forcing != DG_FORCING_NONE) return DG_ERR_UNSUPPORTED;
  if (cfg->precision == DG_PREC_FP32_MIXED && cfg->proj_precision == DG_PROJ_DF64 && cfg->p > 3)
    return DG_ERR_UNSUPPORTED;
  if (cfg->block_size != 0 && (cfg->block_size < 32 || cfg->block_size > 128 || cfg->block_size % 32))
    return DG_ERR_ARG;
  if (2.0 * (double)cfg->nx * (double)cfg->ny > 1.0e8) return DG_ERR_ARG;
  const int arith = arith_of(cfg->precision, cfg->proj_precision);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (arith == ARITH_FP64) return run<double>(cfg, arith, (const double*)d_hb, d_state_in, d_rhs_out, d_flags, s);
  return run<float>(cfg, arith, (const double*)d_hb, d_state_in, d_rhs_out, d_flags, s);
}
