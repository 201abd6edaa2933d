// dgswe_api.cu -- C-ABI of libdgswe (declared in include/dgswe.h): contexts,
// device buffers, graph-captured time steps, set-up projection, diagnostics.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <exception>
#include <new>
#include <vector>

#include "dg_launch.cuh"
#include "dg_nvtx.h"
#include "dg_tile.cuh"
#include "dgswe.h"

using namespace dgswe;

namespace {

struct GraphSlot {
  cudaGraphExec_t exec = nullptr;
};

}  // namespace

struct dg_ctx {
  dg_config cfg;
  int P, K, K1, P1, NREC;
  int KB, PB1, KB1;        // bathymetry space P^max(p,1): basis, edge modes, gradient basis
  long long E;
  int arith;
  bool tiled;  // FP32 time steps by the tile-fused stage kernel
  size_t rsz;  // bytes per Real
  Mesh mesh;
  double inv_det, det, cfl_num;
  cudaStream_t stream;   // caller's stream
  cudaStream_t cap;      // private stream used only for graph capture
  // device buffers
  void* w[3];            // state w0 (step start / result), w1, w2 (stage outputs)
  void* vs[2];           // volume+source integrals of the evaluated state
  void* rec[2];          // side records of the evaluated state
  void* hb;              // [K][E]
  void* hbt;             // [3][PB1][E]
  void* ghb;             // [2][KB1][E]
  void* lin;             // FP64 only: [2][K][K][E] terms linear in xi
  float* ahb;            // mixed solve only: [ahb_words(K)][E] bathymetry matrix parts
  double* geo;           // general meshes: [NGEO][E] per-element geometry
  double* vq;            // forcing: volume Gauss rule [3][nqv]
  double* eq;            // forcing: edge Gauss rule [nqe][7]
  int nqv, nqe;
  double* scal;          // [0],[1]: wave-speed slots, [2]: t, [3]: last dt
  unsigned* err;
  double* partial;       // diagnostics partial sums
  double* stage;         // FP64 AoS staging buffer [3][E][K] for host copies
  void* rhs_vs;          // scratch of dg_rhs
  void* rhs_rec;
  unsigned* rhs_err;     // error word of dg_rhs (kept apart from the time loop's)
  int ep;                // eval buffer holding the current state's evaluation
  int lc;                // wave-speed slot of the current state
  bool evaluated;
  GraphSlot graph[2][2];
};

namespace {

int K_of(int p) { return (p + 1) * (p + 2) / 2; }
// basis size of the bathymetry space P^max(p,1)
int KB_of(int p) { return K_of(p > 1 ? p : 1); }

// Status of a failed CUDA call.  A failed allocation also leaves the
// runtime's last-error slot set; it is cleared here, so that the next
// launch check (cudaGetLastError) of a later call does not report it again.
dg_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return DG_OK;
  if (e == cudaErrorMemoryAllocation) {
    (void)cudaGetLastError();
    return DG_ERR_OOM;
  }
  return DG_ERR_CUDA;
}

#define CK(x)                                 \
  do {                                        \
    cudaError_t _e = (x);                     \
    if (_e != cudaSuccess) return cuda_status(_e); \
  } while (0)

dg_status validate(const dg_config* c) {
  if (!c) return DG_ERR_ARG;
  if (c->nx < 1 || c->ny < 1 || c->p < 0 || c->p > 4) return DG_ERR_ARG;
  if (!(c->Lx > 0.0) || !(c->Ly > 0.0) || !(c->g > 0.0)) return DG_ERR_ARG;
  if (c->rk_order < 1 || c->rk_order > 3) return DG_ERR_ARG;
  if (c->bc < 0 || c->bc > 2 || c->precision < 0 || c->precision > 1) return DG_ERR_ARG;
  if (c->proj_precision < 0 || c->proj_precision > 3) return DG_ERR_ARG;
  if (!(c->dt > 0.0) && !(c->cfl > 0.0)) return DG_ERR_ARG;
  if (!(c->tau_bf >= 0.0) || !std::isfinite(c->tau_bf) || !std::isfinite(c->f_c)) return DG_ERR_ARG;
  // the stage kernels are compiled for at most 128 threads per block
  if (c->block_size != 0 && (c->block_size < 32 || c->block_size > 128 || c->block_size % 32)) return DG_ERR_ARG;
  if (c->bc == DG_BC_PERIODIC && (c->nx < 2 || c->ny < 2)) return DG_ERR_ARG;
  if (c->forcing < 0 || c->forcing > 1) return DG_ERR_ARG;
  if (c->tile_shape < -1 || c->tile_shape > 3) return DG_ERR_ARG;
  if (c->bc == DG_BC_DIRICHLET && c->forcing != DG_FORCING_MANUFACTURED) return DG_ERR_UNSUPPORTED;
  if (c->vertex_xy && c->bc == DG_BC_PERIODIC) return DG_ERR_UNSUPPORTED;
  // the double-float and mixed solves are built for uniform meshes without
  // forcing (double-float: p <= 3)
  if (c->precision == DG_PREC_FP32_MIXED && (c->proj_precision == DG_PROJ_DF64 || c->proj_precision == DG_PROJ_MIXED) &&
      (c->vertex_xy || c->forcing != DG_FORCING_NONE || c->bc == DG_BC_DIRICHLET))
    return DG_ERR_UNSUPPORTED;
  if (c->precision == DG_PREC_FP32_MIXED && c->proj_precision == DG_PROJ_DF64 && c->p > 3) return DG_ERR_UNSUPPORTED;
  if (2.0 * (double)c->nx * (double)c->ny > 4.0e9) return DG_ERR_ARG;
  return DG_OK;
}

cudaError_t launch_stage_any(const dg_ctx* c, int mode, const void* params, cudaStream_t s) {
  const int block = c->cfg.block_size ? c->cfg.block_size : 128;
  // general meshes, forcing and Dirichlet edges use the general kernels
  const bool gen = c->geo || c->cfg.forcing != DG_FORCING_NONE || c->cfg.bc == DG_BC_DIRICHLET;
  switch (c->arith) {
    case ARITH_FP64: return (gen ? stage_fp64_gen : stage_fp64)(c->P, mode, block, params, s);
    case ARITH_FP32_P64: return (gen ? stage_fp32p64_gen : stage_fp32p64)(c->P, mode, block, params, s);
    case ARITH_FP32_PDF: return stage_fp32pdf(c->P, mode, block, params, s);
    case ARITH_FP32_PIR: return stage_fp32pir(c->P, mode, block, params, s);
    default: return (gen ? stage_fp32p32_gen : stage_fp32p32)(c->P, mode, block, params, s);
  }
}

template <class Real>
StageParams<Real> base_params(const dg_ctx* c) {
  StageParams<Real> sp;
  std::memset(&sp, 0, sizeof sp);
  sp.m = c->mesh;
  sp.g = Real(c->cfg.g);
  sp.hb = (const Real*)c->hb;
  sp.hbt = (const Real*)c->hbt;
  sp.ghb = (const Real*)c->ghb;
  sp.lin = (const Real*)c->lin;
  sp.ahb = c->ahb;
  sp.forcing = c->cfg.forcing == DG_FORCING_MANUFACTURED;
  sp.dirichlet = c->cfg.bc == DG_BC_DIRICHLET;
  sp.t_now = c->scal + 2;
  sp.c_eval = 0.0;
  sp.vq = c->vq;
  sp.nqv = c->nqv;
  sp.eq = c->eq;
  sp.nqe = c->nqe;
  sp.dt_fixed = c->cfg.dt > 0.0 ? c->cfg.dt : 0.0;
  sp.cfl_num = c->cfl_num;
  sp.inv_det = c->inv_det;
  sp.det = c->det;
  sp.tau_bf = c->cfg.tau_bf;
  sp.f_c = c->cfg.f_c;
  sp.err = c->err;
  return sp;
}

cudaError_t launch_tile_any(const dg_ctx* c, const StageParams<float>& sp, cudaStream_t s) {
  // launcher index: tile_shape 1..3 -> 0..2; the default (0) takes 8 x 8
  // tiles, 8 x 4 at p = 4 (its shared memory leaves more resident CTAs)
  const int shape = c->cfg.tile_shape > 1 ? c->cfg.tile_shape - 1 : (c->cfg.tile_shape == 0 && c->P == 4 ? 2 : 0);
  switch (c->arith) {
    case ARITH_FP32_P64: return tile_fp32p64(c->P, shape, sp, s);
    case ARITH_FP32_PDF: return tile_fp32pdf(c->P, shape, sp, s);
    case ARITH_FP32_PIR: return tile_fp32pir(c->P, shape, sp, s);
    default: return tile_fp32p32(c->P, shape, sp, s);
  }
}

// Tiled contexts evaluate a state inside the stage that consumes it: after
// dg_init or dg_set_state only the step's CFL maximum is needed (slot lc).
dg_status launch_wave_speed(dg_ctx* c, cudaStream_t s) {
  CK(cudaMemsetAsync(c->scal + c->lc, 0, sizeof(double), s));
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  long long g = (c->E + 255) / 256;
  if (g > 4LL * sms) g = 4LL * sms;
  wave_speed_kernel<float><<<(unsigned)g, 256, 0, s>>>(c->mesh, float(c->cfg.g), c->K, (const float*)c->w[0],
                                                       (const float*)c->hb, c->scal + c->lc);
  CK(cudaGetLastError());
  return DG_OK;
}

// Evaluation of the state in buffer w into (vs[ep], rec[ep]) and its wave
// speed into slot lc.
template <class Real>
dg_status launch_eval_t(dg_ctx* c, cudaStream_t s) {
  CK(cudaMemsetAsync(c->scal + c->lc, 0, sizeof(double), s));
  StageParams<Real> sp = base_params<Real>(c);
  sp.w = (const Real*)c->w[0];
  sp.vs_out = (Real*)c->vs[c->ep];
  sp.rec_out = (Real*)c->rec[c->ep];
  sp.lam_next = c->scal + c->lc;
  CK(launch_stage_any(c, MODE_EVAL, &sp, s));
  return DG_OK;
}

// Shu-Osher coefficients of SSP-RK1/2/3: w_{s+1} = a_s w_0 + b_s (w_s + dt R(w_s))
const double RK_A[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.5, 0.0}, {0.0, 0.75, 1.0 / 3.0}};
const double RK_B[3][3] = {{1.0, 0.0, 0.0}, {1.0, 0.5, 0.0}, {1.0, 0.25, 2.0 / 3.0}};
// time of each stage's output state, in units of dt after the step start
const double RK_C[3][3] = {{1.0, 0.0, 0.0}, {1.0, 1.0, 0.0}, {1.0, 0.5, 1.0}};

// End of a time step: t += dt (fixed, or from the step's wave-speed slot);
// the step's dt is kept in dt_out.  One thread, launched after the last stage
// so that every stage reads a constant step time.
__global__ void advance_time_kernel(double* t, double* dt_out, double dt_fixed, double cfl_num, const double* lam) {
  const double dt = dt_fixed > 0.0 ? dt_fixed : cfl_num / lam[0];
  *t += dt;
  *dt_out = dt;
}

// Launch one full time step from eval parity ep, wave-speed slot lc.
template <class Real>
dg_status launch_step_t(const dg_ctx* c, int ep, int lc, cudaStream_t s) {
  const int S = c->cfg.rk_order;
  const bool adaptive = !(c->cfg.dt > 0.0);
  if (adaptive) CK(cudaMemsetAsync(c->scal + (1 - lc), 0, sizeof(double), s));
  for (int st = 0; st < S; ++st) {
    StageParams<Real> sp = base_params<Real>(c);
    if constexpr (std::is_same<Real, float>::value) {
      if (c->tiled) {
        sp.w = (const float*)(st == 0 ? c->w[0] : c->w[st]);
        sp.wout = (float*)(st == S - 1 ? c->w[0] : c->w[st + 1]);
        sp.w0 = (const float*)c->w[0];
        sp.alpha = RK_A[S - 1][st];
        sp.beta = RK_B[S - 1][st];
        sp.lam = c->scal + lc;
        if (st == S - 1 && adaptive) sp.lam_next = c->scal + (1 - lc);
        CK(launch_tile_any(c, sp, s));
        continue;
      }
    }
    sp.w = (const Real*)(st == 0 ? c->w[0] : c->w[st]);
    sp.wout = (Real*)(st == S - 1 ? c->w[0] : c->w[st + 1]);
    sp.w0 = (const Real*)c->w[0];
    sp.alpha = RK_A[S - 1][st];
    sp.beta = RK_B[S - 1][st];
    const int pin = (ep + st) & 1;
    sp.vs = (const Real*)c->vs[pin];
    sp.rec = (const Real*)c->rec[pin];
    sp.vs_out = (Real*)c->vs[1 - pin];
    sp.rec_out = (Real*)c->rec[1 - pin];
    sp.lam = c->scal + lc;
    sp.c_eval = RK_C[S - 1][st];
    if (st == S - 1 && adaptive) sp.lam_next = c->scal + (1 - lc);
    CK(launch_stage_any(c, MODE_STAGE, &sp, s));
  }
  advance_time_kernel<<<1, 1, 0, s>>>(c->scal + 2, c->scal + 3, c->cfg.dt > 0.0 ? c->cfg.dt : 0.0, c->cfl_num,
                                      c->scal + lc);
  CK(cudaGetLastError());
  return DG_OK;
}

dg_status launch_step(const dg_ctx* c, int ep, int lc, cudaStream_t s) {
  return c->arith == ARITH_FP64 ? launch_step_t<double>(c, ep, lc, s) : launch_step_t<float>(c, ep, lc, s);
}

dg_status launch_eval(dg_ctx* c, cudaStream_t s) {
  if (c->tiled) return launch_wave_speed(c, s);
  return c->arith == ARITH_FP64 ? launch_eval_t<double>(c, s) : launch_eval_t<float>(c, s);
}

dg_status ensure_evaluated(dg_ctx* c) {
  if (c->evaluated) return DG_OK;
  dg_status st = launch_eval(c, c->stream);
  if (st != DG_OK) return st;
  c->evaluated = true;
  return DG_OK;
}

dg_status get_graph(dg_ctx* c, cudaGraphExec_t* out) {
  GraphSlot& g = c->graph[c->ep][c->lc];
  if (!g.exec) {
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
    dg_status st = launch_step(c, c->ep, c->lc, c->cap);
    cudaError_t ce = cudaStreamEndCapture(c->cap, &graph);
    if (st != DG_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    CK(ce);
    ce = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(ce);
  }
  *out = g.exec;
  return DG_OK;
}

void advance_parity(dg_ctx* c) {
  c->ep = (c->ep + c->cfg.rk_order) & 1;
  if (!(c->cfg.dt > 0.0)) c->lc = 1 - c->lc;
}

dg_status read_err(dg_ctx* c) {
  unsigned h = 0;
  CK(cudaMemcpyAsync(&h, c->err, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (h) {
    // report once: clear the word so the context can be inspected and reused
    CK(cudaMemsetAsync(c->err, 0, sizeof(unsigned), c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  if (h & ERRF_NONFINITE) return DG_ERR_NONFINITE;
  if (h & ERRF_DRY) return DG_ERR_DRY;
  return DG_OK;
}

// host AoS FP64 [E][K] -> device SoA FP64 [K][E] (staging through a pinned
// or pageable host transpose)
dg_status upload_soa(const double* host, long long E, int K, double* dev, cudaStream_t s) {
  std::vector<double> t;
  try {
    t.resize((size_t)E * K);
  } catch (const std::exception&) {   // no C++ exception crosses the C ABI
    return DG_ERR_OOM;
  }
  for (long long e = 0; e < E; ++e)
    for (int i = 0; i < K; ++i) t[(size_t)i * E + e] = host[(size_t)e * K + i];
  CK(cudaMemcpyAsync(dev, t.data(), sizeof(double) * t.size(), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  return DG_OK;
}

__global__ void cvt_kernel_f(const double* __restrict__ a, float* __restrict__ b, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = float(a[i]);
}


// device FP64 -> context precision
dg_status store_real(const dg_ctx* c, const double* src, void* dst, long long n, cudaStream_t s) {
  if (c->arith == ARITH_FP64) {
    CK(cudaMemcpyAsync(dst, src, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  } else if (n > 0) {
    cvt_kernel_f<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, (float*)dst, n);
    CK(cudaGetLastError());
  }
  return DG_OK;
}
void free_ctx(dg_ctx* c) {
  if (!c) return;
  for (auto& row : c->graph)
    for (auto& g : row)
      if (g.exec) cudaGraphExecDestroy(g.exec);
  void* bufs[] = {c->w[0], c->w[1], c->w[2], c->vs[0], c->vs[1], c->rec[0], c->rec[1], c->hb, c->hbt,
                  c->ghb, c->lin, c->ahb, c->geo, c->vq, c->eq, c->scal, c->err, c->partial, c->rhs_vs, c->rhs_rec,
                  c->rhs_err, c->stage};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (c->cap) cudaStreamDestroy(c->cap);
  delete c;
}

// Per-element geometry of a general quad-split mesh from its vertices:
// G = adj(B)^T, |det B|, 1/|det B|, outward unit normal and length of each
// local edge (edge n runs from vertex n+1 to n+2), vertex a1; and the smallest
// inscribed-circle diameter.  Rejects clockwise or degenerate triangles.
dg_status build_geometry(const dg_config* cfg, std::vector<double>& geo, double* dmin) {
  const int nx = cfg->nx, ny = cfg->ny;
  const long long E = 2LL * nx * ny;
  geo.assign((size_t)NGEO * E, 0.0);
  const double* v = cfg->vertex_xy;
  auto vx = [&](int i, int j) { return v[2 * ((size_t)j * (nx + 1) + i)]; };
  auto vy = [&](int i, int j) { return v[2 * ((size_t)j * (nx + 1) + i) + 1]; };
  double dm = 1e300;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i)
      for (int t = 0; t < 2; ++t) {
        const long long e = 2LL * ((long long)j * nx + i) + t;
        double x[3], y[3];
        if (t == 0) {
          x[0] = vx(i, j); y[0] = vy(i, j);
          x[1] = vx(i + 1, j); y[1] = vy(i + 1, j);
          x[2] = vx(i, j + 1); y[2] = vy(i, j + 1);
        } else {
          x[0] = vx(i + 1, j + 1); y[0] = vy(i + 1, j + 1);
          x[1] = vx(i, j + 1); y[1] = vy(i, j + 1);
          x[2] = vx(i + 1, j); y[2] = vy(i + 1, j);
        }
        const double B11 = x[1] - x[0], B12 = x[2] - x[0], B21 = y[1] - y[0], B22 = y[2] - y[0];
        const double det = B11 * B22 - B12 * B21;
        if (!(det > 0.0) || !std::isfinite(det)) return DG_ERR_ARG;
        geo[GEO_G11 * E + e] = B22;
        geo[GEO_G12 * E + e] = -B21;
        geo[GEO_G21 * E + e] = -B12;
        geo[GEO_G22 * E + e] = B11;
        geo[GEO_DET * E + e] = det;
        geo[GEO_IDET * E + e] = 1.0 / det;
        double per = 0.0;
        for (int n = 0; n < 3; ++n) {
          const int a = (n + 1) % 3, b = (n + 2) % 3;
          const double tx = x[b] - x[a], ty = y[b] - y[a], len = std::hypot(tx, ty);
          geo[(GEO_EDGE + 3 * n) * E + e] = ty / len;
          geo[(GEO_EDGE + 3 * n + 1) * E + e] = -tx / len;
          geo[(GEO_EDGE + 3 * n + 2) * E + e] = len;
          per += len;
        }
        geo[GEO_A1X * E + e] = x[0];
        geo[GEO_A1Y * E + e] = y[0];
        dm = std::min(dm, 2.0 * det / per);
      }
  *dmin = dm;
  return DG_OK;
}

// Gauss-Legendre nodes/weights on [0, 1] (Newton on P_n, three-term recurrence)
void gauss01(int n, double* s, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
    for (int it = 0; it < 60; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-17) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    s[i] = 0.5 * (1.0 + z);
    w[i] = 1.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Rules for the non-polynomial data of the §3.1 test: collapsed Gauss rule
// on the triangle with ceil((3p+2)/2)+1 points per direction, Gauss rule on
// edges with ceil((3p+1)/2)+1 points (the counts of the reference scheme's
// exact-integration rules), edge rows carrying L_0..L_4 at each node.
void build_rules(int p, std::vector<double>& vq, std::vector<double>& eq, int* nqv, int* nqe) {
  const int nv = (3 * p + 3) / 2 + 1, ne = (3 * p + 2) / 2 + 1;
  double s[16], w[16];
  gauss01(nv, s, w);
  *nqv = nv * nv;
  vq.assign((size_t)3 * nv * nv, 0.0);
  for (int a = 0; a < nv; ++a)
    for (int b = 0; b < nv; ++b) {
      const int q = a * nv + b;
      vq[q] = s[a];
      vq[nv * nv + q] = (1.0 - s[a]) * s[b];
      vq[2 * nv * nv + q] = w[a] * w[b] * (1.0 - s[a]);
    }
  gauss01(ne, s, w);
  *nqe = ne;
  eq.assign((size_t)7 * ne, 0.0);
  for (int q = 0; q < ne; ++q) {
    const double z = 2.0 * s[q] - 1.0;
    double pm = 1.0, pc = z;
    eq[7 * q] = s[q];
    eq[7 * q + 1] = w[q];
    eq[7 * q + 2] = 1.0;
    eq[7 * q + 3] = std::sqrt(3.0) * z;
    for (int j = 1; j + 1 <= 4; ++j) {
      const double pn = ((2 * j + 1) * z * pc - j * pm) / (j + 1);
      pm = pc;
      pc = pn;
      eq[7 * q + 2 + j + 1] = std::sqrt(2.0 * (j + 1) + 1.0) * pn;
    }
  }
}

// Common part of dg_init / dg_init_device: d_fields = device FP64 SoA
// [4][K][E] (hb, xi, qx, qy), owned by the caller of this helper.
dg_status create(const dg_config* cfg, const double* d_hb, const double* d_xi, const double* d_qx,
                 const double* d_qy, void* stream, dg_ctx** out) {
  dg_ctx* c = new (std::nothrow) dg_ctx;
  if (!c) return DG_ERR_OOM;
  std::memset(c, 0, sizeof *c);
  c->cfg = *cfg;
  c->P = cfg->p;
  c->K = K_of(cfg->p);
  c->K1 = K_of(cfg->p - 1);
  c->P1 = cfg->p + 1;
  c->NREC = 6 * c->P1 + 1;
  c->KB = KB_of(cfg->p);
  c->PB1 = std::max(cfg->p, 1) + 1;
  c->KB1 = K_of(std::max(cfg->p, 1) - 1);
  c->E = 2LL * cfg->nx * cfg->ny;
  c->arith = arith_of(cfg->precision, cfg->proj_precision);
  c->rsz = c->arith == ARITH_FP64 ? sizeof(double) : sizeof(float);
  // the tile kernel covers FP32 uniform meshes without forcing (periodic or
  // walls); by default with the mixed and FP32 solves at p <= 3, and with
  // the FP32 solve at p = 4 (1.47x the per-element kernel on 2048^2 quads;
  // the mixed solve's p = 4 tile kernel spills and measured 1.6x slower than
  // its per-element kernel, and with the FP64 and double-float solves the
  // halo's extra solves cost more than the traffic the tiles save)
  const bool light_solve = cfg->proj_precision == DG_PROJ_MIXED || cfg->proj_precision == DG_PROJ_FP32;
  const bool tile_default = (cfg->p <= 3 && light_solve) || (cfg->p == 4 && cfg->proj_precision == DG_PROJ_FP32);
  c->tiled = c->arith != ARITH_FP64 && !cfg->vertex_xy && cfg->forcing == DG_FORCING_NONE &&
             cfg->bc != DG_BC_DIRICHLET && (cfg->tile_shape > 0 || (cfg->tile_shape == 0 && tile_default));
  c->stream = (cudaStream_t)stream;
  const double hx = cfg->Lx / cfg->nx, hy = cfg->Ly / cfg->ny;
  c->mesh = make_mesh(cfg->nx, cfg->ny, cfg->x0, cfg->y0, cfg->Lx, cfg->Ly, cfg->bc == DG_BC_PERIODIC);
  c->det = hx * hy;
  c->inv_det = 1.0 / c->det;
  // smallest inscribed-circle diameter 4 area / perimeter (all triangles equal)
  double dmin = 4.0 * (0.5 * c->det) / (hx + hy + std::hypot(hx, hy));
  std::vector<double> geo_h;
  if (cfg->vertex_xy) {
    dg_status gs;
    try {
      gs = build_geometry(cfg, geo_h, &dmin);
    } catch (const std::exception&) {
      gs = DG_ERR_OOM;
    }
    if (gs != DG_OK) {
      delete c;
      return gs;
    }
  }
  c->cfg.vertex_xy = nullptr;   // the caller's array is not kept
  c->cfl_num = cfg->cfl * dmin / (2.0 * cfg->p + 1.0);
  const long long E = c->E;
  const size_t st = (size_t)3 * c->K * E * c->rsz;
  dg_status s = DG_OK;
  auto alloc = [&](void** p, size_t n) {
    if (s != DG_OK) return;
    cudaError_t e = cudaMalloc(p, n);
    if (e != cudaSuccess) s = cuda_status(e);
  };
  for (int i = 0; i < 3; ++i) alloc(&c->w[i], st);
  // the per-element kernels hand volume integrals and side records from one
  // launch to the next; the tile-fused kernels keep them in shared memory
  for (int i = 0; i < 2 && !c->tiled; ++i) {
    alloc(&c->vs[i], st);
    alloc(&c->rec[i], (size_t)3 * c->NREC * E * c->rsz);
  }
  alloc(&c->hb, (size_t)c->KB * E * c->rsz);
  alloc(&c->hbt, (size_t)3 * c->PB1 * E * c->rsz);
  alloc(&c->ghb, (size_t)2 * c->KB1 * E * c->rsz);
  if (c->arith == ARITH_FP64) alloc(&c->lin, (size_t)2 * c->K * c->K * E * c->rsz);
  if (c->arith == ARITH_FP32_PIR) alloc((void**)&c->ahb, sizeof(float) * ahb_words(c->K) * E);
  if (!geo_h.empty()) alloc((void**)&c->geo, sizeof(double) * geo_h.size());
  std::vector<double> vq_h, eq_h;
  if (cfg->forcing == DG_FORCING_MANUFACTURED) {
    try {
      build_rules(cfg->p, vq_h, eq_h, &c->nqv, &c->nqe);
    } catch (const std::exception&) {
      free_ctx(c);
      return DG_ERR_OOM;
    }
    alloc((void**)&c->vq, sizeof(double) * vq_h.size());
    alloc((void**)&c->eq, sizeof(double) * eq_h.size());
  }
  alloc((void**)&c->scal, 4 * sizeof(double));
  alloc((void**)&c->err, sizeof(unsigned));
  alloc((void**)&c->partial, sizeof(double) * 2 * (size_t)((E + 127) / 128));
  if (s == DG_OK) {
    cudaError_t e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) s = cuda_status(e);
  }
  if (s != DG_OK) {
    free_ctx(c);
    return s;
  }
  cudaStream_t ss = c->stream;
  cudaError_t ce = cudaMemsetAsync(c->scal, 0, 4 * sizeof(double), ss);
  if (ce == cudaSuccess && c->geo) {
    ce = cudaMemcpy(c->geo, geo_h.data(), sizeof(double) * geo_h.size(), cudaMemcpyHostToDevice);
    c->mesh.geo = c->geo;
  }
  if (ce == cudaSuccess && c->vq) ce = cudaMemcpy(c->vq, vq_h.data(), sizeof(double) * vq_h.size(), cudaMemcpyHostToDevice);
  if (ce == cudaSuccess && c->eq) ce = cudaMemcpy(c->eq, eq_h.data(), sizeof(double) * eq_h.size(), cudaMemcpyHostToDevice);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(c->err, 0, sizeof(unsigned), ss);
  if (ce != cudaSuccess) {
    free_ctx(c);
    return cuda_status(ce);
  }
  const long long KE = (long long)c->K * E;
  char* w0 = (char*)c->w[0];
  if ((s = store_real(c, d_xi, w0, KE, ss)) != DG_OK || (s = store_real(c, d_qx, w0 + KE * c->rsz, KE, ss)) != DG_OK ||
      (s = store_real(c, d_qy, w0 + 2 * KE * c->rsz, KE, ss)) != DG_OK) {
    free_ctx(c);
    return s;
  }
  cudaError_t le;
  switch (c->arith) {
    case ARITH_FP64: le = static_fp64(c->P, c->mesh, cfg->g, d_hb, c->hb, c->hbt, c->ghb, c->lin, ss); break;
    case ARITH_FP32_P64:
      le = static_fp32p64(c->P, c->mesh, cfg->g, d_hb, c->hb, c->hbt, c->ghb, nullptr, ss);
      break;
    case ARITH_FP32_PDF:
      le = static_fp32pdf(c->P, c->mesh, cfg->g, d_hb, c->hb, c->hbt, c->ghb, nullptr, ss);
      break;
    case ARITH_FP32_PIR:
      le = static_fp32pir(c->P, c->mesh, cfg->g, d_hb, c->hb, c->hbt, c->ghb, nullptr, ss);
      if (le == cudaSuccess) le = static_ahb(c->P, c->mesh, d_hb, c->ahb, ss);
      break;
    default: le = static_fp32p32(c->P, c->mesh, cfg->g, d_hb, c->hb, c->hbt, c->ghb, nullptr, ss); break;
  }
  if (le == cudaSuccess) le = cudaStreamSynchronize(ss);
  if (le != cudaSuccess) {
    free_ctx(c);
    return cuda_status(le);
  }
  *out = c;
  return DG_OK;
}

}  // namespace

// ===========================================================================
extern "C" {

int dg_num_basis(int p) { return (p < 0 || p > 4) ? 0 : K_of(p); }

int dg_num_basis_bathymetry(int p) { return (p < 0 || p > 4) ? 0 : KB_of(p); }

long long dg_num_elements(const dg_config* cfg) {
  if (!cfg || cfg->nx < 1 || cfg->ny < 1) return 0;
  return 2LL * cfg->nx * cfg->ny;
}

const char* dg_status_str(dg_status s) {
  switch (s) {
    case DG_OK: return "DG_OK";
    case DG_ERR_ARG: return "DG_ERR_ARG";
    case DG_ERR_UNSUPPORTED: return "DG_ERR_UNSUPPORTED";
    case DG_ERR_OOM: return "DG_ERR_OOM";
    case DG_ERR_CUDA: return "DG_ERR_CUDA";
    case DG_ERR_DRY: return "DG_ERR_DRY";
    case DG_ERR_NONFINITE: return "DG_ERR_NONFINITE";
    case DG_ERR_TIMEOUT: return "DG_ERR_TIMEOUT";
  }
  return "DG_ERR_UNKNOWN";
}

dg_status dg_init_device(const dg_config* cfg, const void* d_hb, const void* d_xi, const void* d_qx,
                         const void* d_qy, void* stream, dg_ctx** out) {
  dgswe::NvtxRange nvtx_range("dg_init_device");
  dg_status s = validate(cfg);
  if (s != DG_OK) return s;
  if (!d_hb || !d_xi || !d_qx || !d_qy || !out) return DG_ERR_ARG;
  return create(cfg, (const double*)d_hb, (const double*)d_xi, (const double*)d_qx, (const double*)d_qy, stream,
                out);
}

dg_status dg_init(const dg_config* cfg, const double* hb, const double* xi, const double* qx, const double* qy,
                  void* stream, dg_ctx** out) {
  dgswe::NvtxRange nvtx_range("dg_init");
  dg_status s = validate(cfg);
  if (s != DG_OK) return s;
  if (!hb || !xi || !qx || !qy || !out) return DG_ERR_ARG;
  const int K = K_of(cfg->p), KB = KB_of(cfg->p);
  const long long E = 2LL * cfg->nx * cfg->ny;
  double* tmp = nullptr;
  cudaError_t e = cudaMalloc(&tmp, sizeof(double) * (size_t)(KB + 3 * K) * E);
  if (e != cudaSuccess) return cuda_status(e);
  cudaStream_t ss = (cudaStream_t)stream;
  // layout of tmp: h_b [KB][E], then xi, qx, qy [K][E] each
  double* dst[4] = {tmp, tmp + (size_t)KB * E, tmp + (size_t)(KB + K) * E, tmp + (size_t)(KB + 2 * K) * E};
  const double* src[4] = {hb, xi, qx, qy};
  for (int f = 0; f < 4 && s == DG_OK; ++f) s = upload_soa(src[f], E, f == 0 ? KB : K, dst[f], ss);
  if (s == DG_OK) s = create(cfg, dst[0], dst[1], dst[2], dst[3], stream, out);
  cudaStreamSynchronize(ss);
  cudaFree(tmp);
  return s;
}

void dg_destroy(dg_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  free_ctx(ctx);
}

dg_status dg_rhs(dg_ctx* c, const void* d_in, void* d_out) {
  dgswe::NvtxRange nvtx_range("dg_rhs");
  if (!c || !d_in || !d_out || d_in == d_out) return DG_ERR_ARG;
  const long long E = c->E;
  // each buffer on its own: a failed allocation leaves the others for a retry
  if (!c->rhs_vs) CK(cudaMalloc(&c->rhs_vs, (size_t)3 * c->K * E * c->rsz));
  if (!c->rhs_rec) CK(cudaMalloc(&c->rhs_rec, (size_t)3 * c->NREC * E * c->rsz));
  if (!c->rhs_err) CK(cudaMalloc((void**)&c->rhs_err, sizeof(unsigned)));
  if (c->arith == ARITH_FP64) {
    StageParams<double> sp = base_params<double>(c);
    sp.err = c->rhs_err;
    sp.w = (const double*)d_in;
    sp.vs_out = (double*)c->rhs_vs;
    sp.rec_out = (double*)c->rhs_rec;
    CK(launch_stage_any(c, MODE_EVAL, &sp, c->stream));
    sp.vs = (const double*)c->rhs_vs;
    sp.rec = (const double*)c->rhs_rec;
    sp.rhs_out = (double*)d_out;
    CK(launch_stage_any(c, MODE_RHS, &sp, c->stream));
  } else {
    StageParams<float> sp = base_params<float>(c);
    sp.err = c->rhs_err;
    sp.w = (const float*)d_in;
    sp.vs_out = (float*)c->rhs_vs;
    sp.rec_out = (float*)c->rhs_rec;
    CK(launch_stage_any(c, MODE_EVAL, &sp, c->stream));
    sp.vs = (const float*)c->rhs_vs;
    sp.rec = (const float*)c->rhs_rec;
    sp.rhs_out = (float*)d_out;
    CK(launch_stage_any(c, MODE_RHS, &sp, c->stream));
  }
  return DG_OK;
}

dg_status dg_run(dg_ctx* c, int nsteps, double* t_out) {
  dgswe::NvtxRange nvtx_range("dg_run");
  if (!c || nsteps < 0) return DG_ERR_ARG;
  dg_status s = ensure_evaluated(c);
  if (s != DG_OK) return s;
  for (int k = 0; k < nsteps; ++k) {
    cudaGraphExec_t g;
    if ((s = get_graph(c, &g)) != DG_OK) return s;
    CK(cudaGraphLaunch(g, c->stream));
    advance_parity(c);
  }
  if ((s = read_err(c)) != DG_OK) return s;
  if (t_out) {
    CK(cudaMemcpyAsync(t_out, c->scal + 2, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  return DG_OK;
}

dg_status dg_rk_step(dg_ctx* c, double* dt_used) {
  dgswe::NvtxRange nvtx_range("dg_rk_step");
  if (!c) return DG_ERR_ARG;
  dg_status s = ensure_evaluated(c);
  if (s != DG_OK) return s;
  if ((s = launch_step(c, c->ep, c->lc, c->stream)) != DG_OK) return s;
  advance_parity(c);
  if (dt_used) {
    CK(cudaMemcpyAsync(dt_used, c->scal + 3, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  return DG_OK;
}

dg_status dg_state_device(dg_ctx* c, void** d_state) {
  if (!c || !d_state) return DG_ERR_ARG;
  *d_state = c->w[0];
  return DG_OK;
}

// Host state arrays that are page-locked and mapped are read or written in
// place by one conversion kernel (over the host link, no copy engine and no
// staging buffer).  Other host arrays go through a device staging buffer
// (allocated on first use, kept with the context): the caller's
// element-major arrays are copied as they are and transposed on the device.
static dg_status ensure_stage(dg_ctx* c) {
  if (!c->stage) CK(cudaMalloc((void**)&c->stage, sizeof(double) * 3 * (size_t)c->K * c->E));
  return DG_OK;
}

dg_status dg_get_state(dg_ctx* c, double* xi, double* qx, double* qy) {
  dgswe::NvtxRange nvtx_range("dg_get_state");
  if (!c) return DG_ERR_ARG;
  const long long E = c->E, KE = (long long)c->K * E;
  double* dst[3] = {xi, qx, qy};
  dgswe::HostFields hf;
  if (mapped_fields(dst, KE, hf)) {
    const unsigned gf = dgswe::fields_grid(E, c->K);
    if (c->arith == ARITH_FP64)
      dgswe::soa_to_fields_kernel<double><<<gf, 256, 0, c->stream>>>((const double*)c->w[0], hf, E, c->K);
    else
      dgswe::soa_to_fields_kernel<float><<<gf, 256, 0, c->stream>>>((const float*)c->w[0], hf, E, c->K);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->stream));
    return DG_OK;
  }
  dg_status s = ensure_stage(c);
  if (s != DG_OK) return s;
  const unsigned g = (unsigned)((E + 127) / 128);
  if (c->arith == ARITH_FP64)
    soa_to_aos_kernel<double><<<g, 128, 0, c->stream>>>((const double*)c->w[0], c->stage, E, c->K, 3);
  else
    soa_to_aos_kernel<float><<<g, 128, 0, c->stream>>>((const float*)c->w[0], c->stage, E, c->K, 3);
  CK(cudaGetLastError());
  for (int f = 0; f < 3; ++f)
    if (dst[f])
      CK(cudaMemcpyAsync(dst[f], c->stage + (size_t)f * KE, sizeof(double) * KE, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return DG_OK;
}

dg_status dg_set_state(dg_ctx* c, const double* xi, const double* qx, const double* qy, double t) {
  dgswe::NvtxRange nvtx_range("dg_set_state");
  if (!c || !xi || !qx || !qy) return DG_ERR_ARG;
  const long long E = c->E, KE = (long long)c->K * E;
  double* src[3] = {const_cast<double*>(xi), const_cast<double*>(qx), const_cast<double*>(qy)};
  dgswe::HostFields hf;
  if (mapped_fields(src, KE, hf)) {
    const unsigned gf = dgswe::fields_grid(E, c->K);
    if (c->arith == ARITH_FP64)
      dgswe::fields_to_soa_kernel<double><<<gf, 256, 0, c->stream>>>(hf, (double*)c->w[0], E, c->K);
    else
      dgswe::fields_to_soa_kernel<float><<<gf, 256, 0, c->stream>>>(hf, (float*)c->w[0], E, c->K);
  } else {
    dg_status s = ensure_stage(c);
    if (s != DG_OK) return s;
    for (int f = 0; f < 3; ++f)
      CK(cudaMemcpyAsync(c->stage + (size_t)f * KE, src[f], sizeof(double) * KE, cudaMemcpyHostToDevice, c->stream));
    const unsigned g = (unsigned)((E + 127) / 128);
    if (c->arith == ARITH_FP64)
      aos_to_soa_kernel<double><<<g, 128, 0, c->stream>>>(c->stage, (double*)c->w[0], E, c->K, 3);
    else
      aos_to_soa_kernel<float><<<g, 128, 0, c->stream>>>(c->stage, (float*)c->w[0], E, c->K, 3);
  }
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(c->scal + 2, &t, sizeof(double), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->evaluated = false;
  return DG_OK;
}

dg_status dg_diagnostics(dg_ctx* c, double* mass, double* energy) {
  if (!c) return DG_ERR_ARG;
  const long long nb = (c->E + 127) / 128;
  cudaError_t e;
  switch (c->arith) {
    case ARITH_FP64: e = diag_fp64(c->P, c->mesh, c->w[0], c->hb, c->det, c->cfg.g, c->partial, c->stream); break;
    case ARITH_FP32_P64:
      e = diag_fp32p64(c->P, c->mesh, c->w[0], c->hb, c->det, c->cfg.g, c->partial, c->stream);
      break;
    case ARITH_FP32_PDF:
      e = diag_fp32pdf(c->P, c->mesh, c->w[0], c->hb, c->det, c->cfg.g, c->partial, c->stream);
      break;
    case ARITH_FP32_PIR:
      e = diag_fp32pir(c->P, c->mesh, c->w[0], c->hb, c->det, c->cfg.g, c->partial, c->stream);
      break;
    default: e = diag_fp32p32(c->P, c->mesh, c->w[0], c->hb, c->det, c->cfg.g, c->partial, c->stream); break;
  }
  CK(e);
  std::vector<double> h;
  try {
    h.resize((size_t)2 * nb);
  } catch (const std::exception&) {
    (void)cudaStreamSynchronize(c->stream);
    return DG_ERR_OOM;
  }
  CK(cudaMemcpyAsync(h.data(), c->partial, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  double m = 0.0, en = 0.0;
  for (long long b = 0; b < nb; ++b) {
    m += h[2 * b];
    en += h[2 * b + 1];
  }
  if (mass) *mass = m;
  if (energy) *energy = en;
  return DG_OK;
}

}  // extern "C"
