// dg_batch_api.cu -- C-ABI of batched instances (include/dgswe.h, dg_batch_*):
// arenas, work items, graph-captured steps and the block-size autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <climits>
#include <cstring>
#include <exception>
#include <new>
#include <vector>

#include "dg_batch.cuh"
#include "dg_launch.cuh"
#include "dg_nvtx.h"
#include "dgswe.h"

using namespace dgswe;

namespace {

int K_of(int p) { return (p + 1) * (p + 2) / 2; }

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

#define CK(x)                                          \
  do {                                                 \
    cudaError_t _e = (x);                              \
    if (_e != cudaSuccess) return cuda_status(_e);     \
  } while (0)

size_t align256(size_t n) { return (n + 255) / 256 * 256; }

const double RK_B[3][3] = {{1.0, 0.0, 0.0}, {1.0, 0.5, 0.0}, {1.0, 0.25, 2.0 / 3.0}};

struct HostInst {
  dg_config cfg;
  int p, K, K1, P1, NREC;
  long long E;
  size_t o_state, o_rec, o_hb, o_hbt, o_ghb, o_lin, o_ahb;  // byte offsets in the arenas
  size_t o_stage;                                            // offset (doubles) of its staging slice
};

// Instance record of dg_batch_step_host's per-group kernels (one row of
// blocks per instance: blockIdx.y)
struct XferInst {
  double* stage;     // its staging slice [3][E][K], FP64 element-major
  void* state;       // its state [3][K][E] in the batch's precision
  const void* hb;    // its h_b coefficients (the first E are the element means)
  long long E;
  int K, i;          // coefficients per field; instance index
  float g;
};

// staging slices <-> states of a group's instances: a transpose through
// shared memory, 256 elements of one field at a time, coalesced on both
// sides (the slice's [E][K] run of those elements, the state's K rows);
// one padding word per 32 breaks the bank conflicts of the K-strided
// accesses
constexpr int kXferTile = 256;
constexpr int kXferWords = kXferTile * 15;   // K <= 15
__device__ __forceinline__ int xfer_pad(int j) { return j + (j >> 5); }

template <class Real>
__global__ void __launch_bounds__(kXferTile) group_in_kernel(const XferInst* __restrict__ t, int first) {
  __shared__ double tile[kXferWords + kXferWords / 32];
  const XferInst x = t[first + blockIdx.y];
  const int K = x.K, tid = threadIdx.x;
  Real* w = static_cast<Real*>(x.state);
  for (long long e0 = (long long)blockIdx.x * kXferTile; e0 < x.E; e0 += (long long)gridDim.x * kXferTile) {
    const int ne = (int)(x.E - e0 < kXferTile ? x.E - e0 : kXferTile);
    for (int f = 0; f < 3; ++f) {
      const double* src = x.stage + ((long long)f * x.E + e0) * K;
      for (int j = tid; j < ne * K; j += kXferTile) tile[xfer_pad(j)] = src[j];
      __syncthreads();
      if (tid < ne)
        for (int k = 0; k < K; ++k) w[((long long)f * K + k) * x.E + e0 + tid] = Real(tile[xfer_pad(tid * K + k)]);
      __syncthreads();
    }
  }
}
template <class Real>
__global__ void __launch_bounds__(kXferTile) group_out_kernel(const XferInst* __restrict__ t, int first) {
  __shared__ double tile[kXferWords + kXferWords / 32];
  const XferInst x = t[first + blockIdx.y];
  const int K = x.K, tid = threadIdx.x;
  const Real* w = static_cast<const Real*>(x.state);
  for (long long e0 = (long long)blockIdx.x * kXferTile; e0 < x.E; e0 += (long long)gridDim.x * kXferTile) {
    const int ne = (int)(x.E - e0 < kXferTile ? x.E - e0 : kXferTile);
    for (int f = 0; f < 3; ++f) {
      if (tid < ne)
        for (int k = 0; k < K; ++k) tile[xfer_pad(tid * K + k)] = double(w[((long long)f * K + k) * x.E + e0 + tid]);
      __syncthreads();
      double* dst = x.stage + ((long long)f * x.E + e0) * K;
      for (int j = tid; j < ne * K; j += kXferTile) dst[j] = tile[xfer_pad(j)];
      __syncthreads();
    }
  }
}
// CFL maxima of a group's FP32 states into lam_row[i] (zeroed by the caller),
// with the operations of wave_speed_kernel<float>
__global__ void __launch_bounds__(256) group_wave_speed_kernel(const XferInst* __restrict__ t, int first,
                                                               double* lam_row) {
  const XferInst x = t[first + blockIdx.y];
  const float* w = static_cast<const float*>(x.state);
  const float* hb = static_cast<const float*>(x.hb);
  double l = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < x.E; e += (long long)gridDim.x * blockDim.x) {
    const float H0 = w[e] + hb[e];
    l = fmax(l, double(element_wave_speed_H(H0, w[(long long)x.K * x.E + e], w[2LL * x.K * x.E + e], x.g)));
  }
  l = block_max(l);
  if (threadIdx.x == 0) atomic_max_nonneg(lam_row + x.i, l);
}

}  // namespace

struct dg_batch {
  int n = 0;
  int arith = 0;
  size_t rsz = 0;
  int S = 0;
  bool adaptive = false;
  cudaStream_t stream = nullptr, cap = nullptr;
  std::vector<HostInst> inst;
  size_t sz_state = 0, sz_rec = 0;
  void* w[3] = {nullptr, nullptr, nullptr};
  void* vs[2] = {nullptr, nullptr};
  void* rec[2] = {nullptr, nullptr};
  void* hb = nullptr;
  void* hbt = nullptr;
  void* ghb = nullptr;
  void* lin = nullptr;          // FP64 batches only
  void* ahb = nullptr;          // mixed-solve batches only
  double* stage = nullptr;      // FP64 staging for get/set state: one slice per instance
  size_t stage_n = 0;
  size_t stage_total = 0;       // doubles of all slices
  double* lam = nullptr;        // [2][n]
  double* t = nullptr;          // [n]
  unsigned* err = nullptr;
  unsigned* counters = nullptr; // one per launch of a step (+ evaluation): [1 + 3 S]
  BatchInst* d_inst = nullptr;
  BatchItem* d_items = nullptr;
  int n_items = 0;
  int block = 0, grid = 0;     // per-element: elements per item, persistent grid
  bool tiled = false;           // FP32: tile-fused stage kernels, one launch per order class
  int cls_shape[4] = {0, 0, 0, 0};   // tiled, per order p = 1..3: tile shape index
  int cls_begin[4] = {0, 0, 0, 0};   //   its items [cls_begin, cls_end)
  int cls_end[4] = {0, 0, 0, 0};
  int cls_grid[4] = {0, 0, 0, 0};    //   its persistent grid
  int ep = 0, lc = 0;
  bool evaluated = false;
  cudaGraphExec_t graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  std::vector<int> item_lo, item_hi;  // per instance: its work items [lo, hi)
  // dg_batch_step_host: copy streams, events and per-group work counters
  // (created on first use)
  cudaStream_t s_up = nullptr, s_down = nullptr;
  std::vector<cudaEvent_t> ev_up, ev_done;
  cudaEvent_t ev_start = nullptr, ev_end = nullptr;
  unsigned* pcount = nullptr;         // [groups][S]
  XferInst* xfer = nullptr;           // [n] per-instance records, in group order
  long long dofs = 0;
};

namespace {

// tile-fused launch of items [lo, hi) of order class p on `grid` CTAs
cudaError_t launch_tile_range(const dg_batch* b, int p, int lo, int hi, int grid, BatchArgs a, cudaStream_t s) {
  a.item_begin = lo;
  a.n_items = hi;
  const int shape = b->cls_shape[p];
  switch (b->arith) {
    case ARITH_FP32_P64: return batch_tile_launch_fp32p64(p, shape, grid, a, s);
    case ARITH_FP32_PDF: return batch_tile_launch_fp32pdf(p, shape, grid, a, s);
    case ARITH_FP32_PIR: return batch_tile_launch_fp32pir(p, shape, grid, a, s);
    default: return batch_tile_launch_fp32p32(p, shape, grid, a, s);
  }
}

// tile-fused launch of order class p (items [cls_begin[p], cls_end[p]))
cudaError_t launch_tile_class(const dg_batch* b, int p, const BatchArgs& a, cudaStream_t s) {
  return launch_tile_range(b, p, b->cls_begin[p], b->cls_end[p], b->cls_grid[p], a, s);
}

cudaError_t launch_batch(const dg_batch* b, int mode, const BatchArgs& a, cudaStream_t s) {
  switch (b->arith) {
    case ARITH_FP64: return batch_launch_fp64(mode, b->grid, b->block, a, s);
    case ARITH_FP32_P64: return batch_launch_fp32p64(mode, b->grid, b->block, a, s);
    case ARITH_FP32_PDF: return batch_launch_fp32pdf(mode, b->grid, b->block, a, s);
    case ARITH_FP32_PIR: return batch_launch_fp32pir(mode, b->grid, b->block, a, s);
    default: return batch_launch_fp32p32(mode, b->grid, b->block, a, s);
  }
}

BatchArgs base_args(const dg_batch* b) {
  BatchArgs a;
  std::memset(&a, 0, sizeof a);
  a.inst = b->d_inst;
  a.items = b->d_items;
  a.n_items = b->n_items;
  a.n_inst = b->n;
  a.err = b->err;
  return a;
}

// CFL maximum of instance i's current state into its slot of lam row lc
// (tile-fused batches; the slot zeroed by the caller)
cudaError_t launch_wave_speed(const dg_batch* b, int i, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const HostInst& h = b->inst[i];
  long long g = (h.E + 255) / 256;
  if (g > 4LL * sms) g = 4LL * sms;
  const Mesh m = make_mesh(h.cfg.nx, h.cfg.ny, h.cfg.x0, h.cfg.y0, h.cfg.Lx, h.cfg.Ly, h.cfg.bc == DG_BC_PERIODIC);
  wave_speed_kernel<float><<<(unsigned)g, 256, 0, s>>>(m, float(h.cfg.g), h.K, (const float*)((char*)b->w[0] + h.o_state),
                                                       (const float*)((char*)b->hb + h.o_hb),
                                                       b->lam + (size_t)b->lc * b->n + i);
  return cudaGetLastError();
}

dg_status launch_eval(dg_batch* b, cudaStream_t s) {
  CK(cudaMemsetAsync(b->counters, 0, sizeof(unsigned), s));
  CK(cudaMemsetAsync(b->lam + (size_t)b->lc * b->n, 0, sizeof(double) * b->n, s));
  if (b->tiled) {
    // the tile-fused stages evaluate their own input: only the first step's
    // CFL maximum of every instance is needed
    for (int i = 0; i < b->n; ++i) CK(launch_wave_speed(b, i, s));
    return DG_OK;
  }
  BatchArgs a = base_args(b);
  a.counter = b->counters;
  a.pin = b->ep;
  a.lc = b->lc;
  CK(launch_batch(b, MODE_EVAL, a, s));
  return DG_OK;
}

// One step: every stage is one persistent launch (per-element batches) or
// one per order class present (tile-fused batches, p = 3 first).  With
// cls_ms (tile-fused only; not while capturing) each class launch is timed
// with events and its milliseconds added to cls_ms[p].
dg_status launch_step(const dg_batch* b, int ep, int lc, cudaStream_t s, double* cls_ms = nullptr) {
  CK(cudaMemsetAsync(b->counters + 1, 0, sizeof(unsigned) * 3 * b->S, s));
  if (b->adaptive) CK(cudaMemsetAsync(b->lam + (size_t)(1 - lc) * b->n, 0, sizeof(double) * b->n, s));
  cudaEvent_t ev[2] = {nullptr, nullptr};
  if (cls_ms) {
    CK(cudaEventCreate(&ev[0]));
    const cudaError_t ce = cudaEventCreate(&ev[1]);
    if (ce != cudaSuccess) {
      cudaEventDestroy(ev[0]);
      return cuda_status(ce);
    }
  }
  dg_status st_out = DG_OK;
  for (int st = 0; st < b->S && st_out == DG_OK; ++st) {
    BatchArgs a = base_args(b);
    a.win = st == 0 ? 0 : st;
    a.wout = st == b->S - 1 ? 0 : st + 1;
    a.pin = (ep + st) & 1;
    a.beta = RK_B[b->S - 1][st];
    a.alpha = 1.0 - a.beta;
    a.lc = lc;
    a.last = st == b->S - 1;
    if (!b->tiled) {
      a.counter = b->counters + 1 + st;
      const cudaError_t ce = launch_batch(b, MODE_STAGE, a, s);
      if (ce != cudaSuccess) st_out = cuda_status(ce);
      continue;
    }
    for (int p = 3; p >= 1 && st_out == DG_OK; --p) {
      if (b->cls_end[p] <= b->cls_begin[p]) continue;
      a.counter = b->counters + 1 + 3 * st + (p - 1);
      cudaError_t ce = cls_ms ? cudaEventRecord(ev[0], s) : cudaSuccess;
      if (ce == cudaSuccess) ce = launch_tile_class(b, p, a, s);
      if (ce == cudaSuccess && cls_ms) ce = cudaEventRecord(ev[1], s);
      if (ce == cudaSuccess && cls_ms) ce = cudaEventSynchronize(ev[1]);
      float ms = 0.f;
      if (ce == cudaSuccess && cls_ms) ce = cudaEventElapsedTime(&ms, ev[0], ev[1]);
      if (ce != cudaSuccess) st_out = cuda_status(ce);
      if (cls_ms) cls_ms[p] += ms;
    }
  }
  if (ev[0]) cudaEventDestroy(ev[0]);
  if (ev[1]) cudaEventDestroy(ev[1]);
  return st_out;
}

// The stages of one step for the items [lo, hi) of order class p alone
// (tile-fused batches; whole instances): the class launches of launch_step
// restricted to those instances.  The instances are independent, so
// stepping groups of them one after another instead of stage by stage gives
// the same bits.  counters: one per stage, zeroed by the caller (with the
// next step's CFL row when adaptive) before the first group.
dg_status launch_range_step(const dg_batch* b, int p, int lo, int hi, unsigned* counters, int ep, int lc,
                            cudaStream_t s) {
  const int grid = std::max(1, std::min(b->cls_grid[p], hi - lo));
  for (int st = 0; st < b->S; ++st) {
    BatchArgs a = base_args(b);
    a.win = st == 0 ? 0 : st;
    a.wout = st == b->S - 1 ? 0 : st + 1;
    a.pin = (ep + st) & 1;
    a.beta = RK_B[b->S - 1][st];
    a.alpha = 1.0 - a.beta;
    a.lc = lc;
    a.last = st == b->S - 1;
    a.counter = counters + st;
    CK(launch_tile_range(b, p, lo, hi, grid, a, s));
  }
  return DG_OK;
}

void drop_graphs(dg_batch* b) {
  for (auto& row : b->graph)
    for (auto& g : row)
      if (g) {
        cudaGraphExecDestroy(g);
        g = nullptr;
      }
}

dg_status get_graph(dg_batch* b, cudaGraphExec_t* out) {
  cudaGraphExec_t& g = b->graph[b->ep][b->lc];
  if (!g) {
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    dg_status st = launch_step(b, b->ep, b->lc, b->cap);
    cudaError_t ce = cudaStreamEndCapture(b->cap, &graph);
    if (st != DG_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    CK(ce);
    ce = cudaGraphInstantiate(&g, graph, 0);
    cudaGraphDestroy(graph);
    CK(ce);
  }
  *out = g;
  return DG_OK;
}

// Work items of `block` elements, the most expensive order first (all p = 3
// items, then p = 2, then p = 1).  All warps of an SM then run the same
// order's code at the same time; queues that mix orders (each class spread
// evenly, so that FP64-bound and FP32-bound items overlap) measured 1.2-5x
// slower, the warps stalling on instruction fetch.
//
// The batch changes only once the new list is on the device: on any failure
// it keeps its previous items, block and graphs.
//
// Tiled batches (block = tile shape index): one item per tile of
// tile_tx x tile_ty quads, in the same order of orders.
dg_status build_items_impl(dg_batch* b, int block, const int* shapes) {
  std::vector<BatchItem> items;
  std::vector<int> lo, hi;
  int begin[4] = {0, 0, 0, 0}, end[4] = {0, 0, 0, 0};
  try {
    lo.assign(b->n, 0);
    hi.assign(b->n, 0);
    for (int p = 3; p >= 1; --p) {
      begin[p] = (int)std::min(items.size(), (size_t)INT_MAX);
      for (int i = 0; i < b->n; ++i) {
        if (b->inst[i].p != p) continue;
        lo[i] = (int)std::min(items.size(), (size_t)INT_MAX);
        if (b->tiled) {
          const int tx = tile_tx(shapes[p]), ty = tile_ty(shapes[p]);
          const long long nt = (long long)((b->inst[i].cfg.nx + tx - 1) / tx) * ((b->inst[i].cfg.ny + ty - 1) / ty);
          for (long long k = 0; k < nt; ++k) items.push_back({i, (int)k});
        } else {
          for (long long s = 0; s < b->inst[i].E; s += block) items.push_back({i, (int)s});
        }
        hi[i] = (int)std::min(items.size(), (size_t)INT_MAX);
      }
      end[p] = (int)std::min(items.size(), (size_t)INT_MAX);
    }
  } catch (const std::exception&) {   // no C++ exception crosses the C ABI
    return DG_ERR_OOM;
  }
  if (items.size() > (size_t)INT_MAX) return DG_ERR_ARG;
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int grid = 0, cls_grid[4] = {0, 0, 0, 0};
  if (b->tiled) {
    for (int p = 1; p <= 3; ++p) {
      if (end[p] <= begin[p]) continue;
      int occ = 0;
      cudaError_t e;
      switch (b->arith) {
        case ARITH_FP32_P64: e = batch_tile_occupancy_fp32p64(p, shapes[p], &occ); break;
        case ARITH_FP32_PDF: e = batch_tile_occupancy_fp32pdf(p, shapes[p], &occ); break;
        case ARITH_FP32_PIR: e = batch_tile_occupancy_fp32pir(p, shapes[p], &occ); break;
        default: e = batch_tile_occupancy_fp32p32(p, shapes[p], &occ); break;
      }
      CK(e);
      cls_grid[p] = std::max(1, std::min(end[p] - begin[p], sms * std::max(1, occ)));
    }
  } else {
    int occ = 0;
    cudaError_t e;
    switch (b->arith) {
      case ARITH_FP64: e = batch_occupancy_fp64(block, &occ); break;
      case ARITH_FP32_P64: e = batch_occupancy_fp32p64(block, &occ); break;
      case ARITH_FP32_PDF: e = batch_occupancy_fp32pdf(block, &occ); break;
      case ARITH_FP32_PIR: e = batch_occupancy_fp32pir(block, &occ); break;
      default: e = batch_occupancy_fp32p32(block, &occ); break;
    }
    CK(e);
    grid = std::max(1, std::min((int)items.size(), sms * std::max(1, occ)));
  }
  BatchItem* d_new = nullptr;
  CK(cudaMalloc(&d_new, sizeof(BatchItem) * items.size()));
  const cudaError_t ce = cudaMemcpy(d_new, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice);
  if (ce != cudaSuccess) {
    cudaFree(d_new);
    return cuda_status(ce);
  }
  // the captured graphs hold the old list's address: drop them with it
  drop_graphs(b);
  if (b->d_items) cudaFree(b->d_items);
  b->d_items = d_new;
  b->n_items = (int)items.size();
  b->item_lo.swap(lo);
  b->item_hi.swap(hi);
  b->block = block;
  b->grid = grid;
  for (int p = 0; p < 4; ++p) {
    b->cls_shape[p] = shapes ? shapes[p] : 0;
    b->cls_begin[p] = begin[p];
    b->cls_end[p] = end[p];
    b->cls_grid[p] = cls_grid[p];
  }
  return DG_OK;
}

// Per-element batches: `block` elements per work item.  Tile-fused
// batches: `block` is the tile shape index of every order class.
dg_status build_items(dg_batch* b, int block) {
  const int shapes[4] = {block, block, block, block};
  return build_items_impl(b, block, b->tiled ? shapes : nullptr);
}

void free_batch(dg_batch* b) {
  if (!b) return;
  drop_graphs(b);
  void* bufs[] = {b->w[0], b->w[1], b->w[2], b->vs[0], b->vs[1], b->rec[0], b->rec[1], b->hb, b->hbt,
                  b->ghb, b->lin, b->ahb, b->stage, b->lam, b->t, b->err, b->counters, b->d_inst, b->d_items};
  for (void* p : bufs)
    if (p) cudaFree(p);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (cudaStream_t s : {b->s_up, b->s_down})
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->ev_up) cudaEventDestroy(e);
  for (cudaEvent_t e : b->ev_done) cudaEventDestroy(e);
  for (cudaEvent_t e : {b->ev_start, b->ev_end})
    if (e) cudaEventDestroy(e);
  if (b->pcount) cudaFree(b->pcount);
  if (b->xfer) cudaFree(b->xfer);
  delete b;
}

__global__ void set_scalar_kernel(double* dst, double v) { *dst = v; }

__global__ void cvt_f(const double* __restrict__ a, float* __restrict__ b, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = float(a[i]);
}

dg_status store_real(const dg_batch* b, const double* src, void* dst, long long n, cudaStream_t s) {
  if (n <= 0) return DG_OK;
  if (b->arith == ARITH_FP64) {
    CK(cudaMemcpyAsync(dst, src, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  } else {
    cvt_f<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, (float*)dst, n);
    CK(cudaGetLastError());
  }
  return DG_OK;
}

dg_status validate_one(const dg_config* c) {
  if (c->nx < 2 || c->ny < 2 || c->p < 0 || c->p > 4) return DG_ERR_ARG;
  if (c->p == 0 || c->p == 4) return DG_ERR_UNSUPPORTED;   // the batched kernel holds p = 1..3
  if (!(c->Lx > 0.0) || !(c->Ly > 0.0) || !(c->g > 0.0)) return DG_ERR_ARG;
  if (c->rk_order < 1 || c->rk_order > 3 || c->bc < 0 || c->bc > 2) return DG_ERR_ARG;
  if (c->precision < 0 || c->precision > 1 || c->proj_precision < 0 || c->proj_precision > 3) return DG_ERR_ARG;
  if (c->tile_shape < -1 || c->tile_shape > 3) return DG_ERR_ARG;
  if (c->bc == DG_BC_DIRICHLET || c->vertex_xy || c->forcing != DG_FORCING_NONE) return DG_ERR_UNSUPPORTED;
  if (!(c->dt > 0.0) && !(c->cfl > 0.0)) return DG_ERR_ARG;
  if (2.0 * c->nx * (double)c->ny > 2.0e9) return DG_ERR_ARG;
  return DG_OK;
}

// Checks shared by both forms of dg_batch_init (no CUDA call).
dg_status validate_batch(int n, const dg_config* cfgs, const void* const* hb, const void* const* xi,
                         const void* const* qx, const void* const* qy, dg_batch** out) {
  if (n < 1 || !cfgs || !hb || !xi || !qx || !qy || !out) return DG_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    dg_status s = validate_one(&cfgs[i]);
    if (s != DG_OK) return s;
    if (!hb[i] || !xi[i] || !qx[i] || !qy[i]) return DG_ERR_ARG;
    if (cfgs[i].precision != cfgs[0].precision || cfgs[i].proj_precision != cfgs[0].proj_precision ||
        cfgs[i].rk_order != cfgs[0].rk_order || (cfgs[i].dt > 0.0) != (cfgs[0].dt > 0.0) ||
        (cfgs[i].tile_shape >= 0) != (cfgs[0].tile_shape >= 0))
      return DG_ERR_ARG;
  }
  return DG_OK;
}

// Source of one instance's FP64 input fields on the device, SoA [Kb][E]
// (h_b) and [K][E] (xi, qx, qy): the caller's device arrays, or the caller's
// host AoS arrays transposed and uploaded into one staging buffer that is
// reused for every instance (stream order keeps the previous instance's
// conversion ahead of the next upload).
struct InputSource {
  const void* const* f[4];
  bool host;
  double* stage;
  size_t stage_n;
  dg_status get(int i, long long E, int K, int KB, const double* out[4], cudaStream_t s) {
    if (!host) {
      for (int k = 0; k < 4; ++k) out[k] = static_cast<const double*>(f[k][i]);
      return DG_OK;
    }
    const size_t need = (size_t)(KB + 3 * K) * (size_t)E;
    if (stage_n < need) {
      CK(cudaStreamSynchronize(s));
      if (stage) cudaFree(stage);
      stage = nullptr;
      stage_n = 0;
      CK(cudaMalloc((void**)&stage, sizeof(double) * need));
      stage_n = need;
    }
    std::vector<double> t;
    try {
      t.resize(need);
    } catch (const std::exception&) {   // no C++ exception crosses the C ABI
      return DG_ERR_OOM;
    }
    size_t off = 0;
    for (int k = 0; k < 4; ++k) {
      const int nk = k == 0 ? KB : K;
      const double* h = static_cast<const double*>(f[k][i]);
      for (long long e = 0; e < E; ++e)
        for (int c = 0; c < nk; ++c) t[off + (size_t)c * E + e] = h[(size_t)e * nk + c];
      out[k] = stage + off;
      off += (size_t)nk * E;
    }
    // the previous instance's kernels read the staging buffer: they run
    // first on this stream, and the copy below waits for them
    CK(cudaMemcpyAsync(stage, t.data(), sizeof(double) * need, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    return DG_OK;
  }
};

dg_status batch_create(int n, const dg_config* cfgs, InputSource& src, void* stream, dg_batch** out) {
  dg_batch* b = new (std::nothrow) dg_batch();
  if (!b) return DG_ERR_OOM;
  std::vector<BatchInst> desc;
  try {
    b->inst.reserve(n);
    desc.resize(n);
  } catch (const std::exception&) {   // no C++ exception crosses the C ABI
    delete b;
    return DG_ERR_OOM;
  }
  b->n = n;
  b->arith = arith_of(cfgs[0].precision, cfgs[0].proj_precision);
  b->rsz = b->arith == ARITH_FP64 ? 8 : 4;
  b->S = cfgs[0].rk_order;
  b->adaptive = !(cfgs[0].dt > 0.0);
  b->stream = (cudaStream_t)stream;
  // tile-fused by default with the mixed and FP32 solves (as single contexts)
  b->tiled = b->arith != ARITH_FP64 &&
             (cfgs[0].tile_shape > 0 ||
              (cfgs[0].tile_shape == 0 && (b->arith == ARITH_FP32_PIR || b->arith == ARITH_FP32_P32)));
  size_t ost = 0, orec = 0, ohb = 0, ohbt = 0, oghb = 0, olin = 0, oahb = 0;
  b->dofs = 0;
  for (int i = 0; i < n; ++i) {
    HostInst h;
    h.cfg = cfgs[i];
    h.p = cfgs[i].p;
    h.K = K_of(h.p);
    h.K1 = K_of(h.p - 1);
    h.P1 = h.p + 1;
    h.NREC = 6 * h.P1 + 1;
    h.E = 2LL * cfgs[i].nx * cfgs[i].ny;
    h.o_state = ost;
    h.o_rec = orec;
    h.o_hb = ohb;
    h.o_hbt = ohbt;
    h.o_ghb = oghb;
    h.o_lin = olin;
    h.o_ahb = oahb;
    h.o_stage = b->stage_total;
    b->stage_total += (size_t)3 * h.K * h.E;
    ost += align256((size_t)3 * h.K * h.E * b->rsz);
    orec += align256((size_t)3 * h.NREC * h.E * b->rsz);
    ohb += align256((size_t)h.K * h.E * b->rsz);
    ohbt += align256((size_t)3 * h.P1 * h.E * b->rsz);
    oghb += align256((size_t)2 * h.K1 * h.E * b->rsz);
    if (b->arith == ARITH_FP64) olin += align256((size_t)2 * h.K * h.K * h.E * b->rsz);
    if (b->arith == ARITH_FP32_PIR) oahb += align256(sizeof(float) * ahb_words(h.K) * h.E);
    b->dofs += 3LL * h.K * h.E;
    b->inst.push_back(h);
  }
  b->sz_state = ost;
  b->sz_rec = orec;
  dg_status st = DG_OK;
  auto alloc = [&](void** p, size_t bytes) {
    if (st != DG_OK) return;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) st = cuda_status(e);
  };
  for (int k = 0; k < 3; ++k) alloc(&b->w[k], ost);
  // per-element kernels hand volume integrals and side records from one
  // launch to the next; the tile-fused kernels keep them in shared memory
  for (int k = 0; k < 2 && !b->tiled; ++k) {
    alloc(&b->vs[k], ost);
    alloc(&b->rec[k], orec);
  }
  alloc(&b->hb, ohb);
  alloc(&b->hbt, ohbt);
  alloc(&b->ghb, oghb);
  if (olin) alloc(&b->lin, olin);
  if (oahb) alloc(&b->ahb, oahb);
  alloc((void**)&b->lam, sizeof(double) * 2 * n);
  alloc((void**)&b->t, sizeof(double) * n);
  alloc((void**)&b->err, sizeof(unsigned));
  alloc((void**)&b->counters, sizeof(unsigned) * 16);
  alloc((void**)&b->d_inst, sizeof(BatchInst) * n);
  if (st == DG_OK) {
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) st = cuda_status(e);
  }
  if (st != DG_OK) {
    free_batch(b);
    return st;
  }
  cudaStream_t s = b->stream;
  cudaError_t e = cudaMemsetAsync(b->lam, 0, sizeof(double) * 2 * n, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->t, 0, sizeof(double) * n, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->err, 0, sizeof(unsigned), s);
  for (int i = 0; i < n && e == cudaSuccess && st == DG_OK; ++i) {
    const HostInst& h = b->inst[i];
    BatchInst& d = desc[i];
    std::memset(&d, 0, sizeof d);
    const double hx = h.cfg.Lx / h.cfg.nx, hy = h.cfg.Ly / h.cfg.ny;
    d.m = make_mesh(h.cfg.nx, h.cfg.ny, h.cfg.x0, h.cfg.y0, h.cfg.Lx, h.cfg.Ly, h.cfg.bc == DG_BC_PERIODIC);
    d.g = h.cfg.g;
    d.inv_det = 1.0 / (hx * hy);
    d.det = hx * hy;
    d.tau_bf = h.cfg.tau_bf;
    d.f_c = h.cfg.f_c;
    const double dmin = 4.0 * (0.5 * hx * hy) / (hx + hy + std::hypot(hx, hy));
    d.cfl_num = h.cfg.cfl * dmin / (2.0 * h.p + 1.0);
    d.dt_fixed = h.cfg.dt > 0.0 ? h.cfg.dt : 0.0;
    for (int k = 0; k < 3; ++k) d.w[k] = (char*)b->w[k] + h.o_state;
    for (int k = 0; k < 2; ++k) {
      d.vs[k] = (char*)b->vs[k] + h.o_state;
      d.rec[k] = (char*)b->rec[k] + h.o_rec;
    }
    d.hb = (char*)b->hb + h.o_hb;
    d.hbt = (char*)b->hbt + h.o_hbt;
    d.ghb = (char*)b->ghb + h.o_ghb;
    d.lin = b->lin ? (char*)b->lin + h.o_lin : nullptr;
    d.ahb = b->ahb ? (const float*)((char*)b->ahb + h.o_ahb) : nullptr;
    d.lam = b->lam + i;
    d.t = b->t + i;
    d.p = h.p;
    const long long KE = (long long)h.K * h.E;
    char* w0 = (char*)d.w[0];
    const double* in[4];
    if ((st = src.get(i, h.E, h.K, h.K, in, s)) != DG_OK) break;
    if ((st = store_real(b, in[1], w0, KE, s)) != DG_OK) break;
    if ((st = store_real(b, in[2], w0 + KE * b->rsz, KE, s)) != DG_OK) break;
    if ((st = store_real(b, in[3], w0 + 2 * KE * b->rsz, KE, s)) != DG_OK) break;
    void *ph = (void*)d.hb, *pt = (void*)d.hbt, *pg = (void*)d.ghb, *pl = (void*)d.lin;
    const double* hbi = in[0];
    switch (b->arith) {
      case ARITH_FP64: e = static_fp64(h.p, d.m, h.cfg.g, hbi, ph, pt, pg, pl, s); break;
      case ARITH_FP32_P64: e = static_fp32p64(h.p, d.m, h.cfg.g, hbi, ph, pt, pg, nullptr, s); break;
      case ARITH_FP32_PDF: e = static_fp32pdf(h.p, d.m, h.cfg.g, hbi, ph, pt, pg, nullptr, s); break;
      case ARITH_FP32_PIR:
        e = static_fp32pir(h.p, d.m, h.cfg.g, hbi, ph, pt, pg, nullptr, s);
        if (e == cudaSuccess) e = static_ahb(h.p, d.m, hbi, (float*)d.ahb, s);
        break;
      default: e = static_fp32p32(h.p, d.m, h.cfg.g, hbi, ph, pt, pg, nullptr, s); break;
    }
  }
  if (e == cudaSuccess && st == DG_OK)
    e = cudaMemcpyAsync(b->d_inst, desc.data(), sizeof(BatchInst) * n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess || st != DG_OK) {
    free_batch(b);
    return st != DG_OK ? st : cuda_status(e);
  }
  if ((st = build_items(b, b->tiled ? (cfgs[0].tile_shape > 1 ? cfgs[0].tile_shape - 1 : 0) : 128)) != DG_OK) {
    free_batch(b);
    return st;
  }
  *out = b;
  return DG_OK;
}

}  // namespace

extern "C" {

dg_status dg_batch_init(int n, const dg_config* cfgs, const double* const* hb, const double* const* xi,
                        const double* const* qx, const double* const* qy, void* stream, dg_batch** out) {
  dgswe::NvtxRange nvtx_range("dg_batch_init");
  const void* const* f[4] = {(const void* const*)hb, (const void* const*)xi, (const void* const*)qx,
                             (const void* const*)qy};
  dg_status s = validate_batch(n, cfgs, f[0], f[1], f[2], f[3], out);
  if (s != DG_OK) return s;
  InputSource src = {{f[0], f[1], f[2], f[3]}, true, nullptr, 0};
  s = batch_create(n, cfgs, src, stream, out);
  if (src.stage) {
    cudaStreamSynchronize((cudaStream_t)stream);
    cudaFree(src.stage);
  }
  return s;
}

dg_status dg_batch_init_device(int n, const dg_config* cfgs, const void* const* d_hb, const void* const* d_xi,
                               const void* const* d_qx, const void* const* d_qy, void* stream, dg_batch** out) {
  dgswe::NvtxRange nvtx_range("dg_batch_init_device");
  dg_status s = validate_batch(n, cfgs, d_hb, d_xi, d_qx, d_qy, out);
  if (s != DG_OK) return s;
  InputSource src = {{d_hb, d_xi, d_qx, d_qy}, false, nullptr, 0};
  return batch_create(n, cfgs, src, stream, out);
}

void dg_batch_destroy(dg_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  free_batch(b);
}

long long dg_batch_dofs(const dg_batch* b) { return b ? b->dofs : 0; }

dg_status dg_batch_set_block(dg_batch* b, int block) {
  if (!b) return DG_ERR_ARG;
  if (b->tiled ? (block < 1 || block > kTileShapes) : (block < 32 || block > 128 || block % 32)) return DG_ERR_ARG;
  CK(cudaStreamSynchronize(b->stream));
  return build_items(b, b->tiled ? block - 1 : block);
}

dg_status dg_batch_run(dg_batch* b, int nsteps, double* t_out) {
  dgswe::NvtxRange nvtx_range("dg_batch_run");
  if (!b || nsteps < 0) return DG_ERR_ARG;
  if (!b->evaluated) {
    dg_status s = launch_eval(b, b->stream);
    if (s != DG_OK) return s;
    b->evaluated = true;
  }
  for (int k = 0; k < nsteps; ++k) {
    cudaGraphExec_t g;
    dg_status s = get_graph(b, &g);
    if (s != DG_OK) return s;
    CK(cudaGraphLaunch(g, b->stream));
    b->ep = (b->ep + b->S) & 1;
    if (b->adaptive) b->lc = 1 - b->lc;
  }
  unsigned h = 0;
  CK(cudaMemcpyAsync(&h, b->err, sizeof h, cudaMemcpyDeviceToHost, b->stream));
  if (t_out) CK(cudaMemcpyAsync(t_out, b->t, sizeof(double) * b->n, cudaMemcpyDeviceToHost, b->stream));
  CK(cudaStreamSynchronize(b->stream));
  if (h) {
    CK(cudaMemsetAsync(b->err, 0, sizeof(unsigned), b->stream));
    CK(cudaStreamSynchronize(b->stream));
  }
  if (h & ERRF_NONFINITE) return DG_ERR_NONFINITE;
  if (h & ERRF_DRY) return DG_ERR_DRY;
  return DG_OK;
}

// device FP64 staging of every instance's state [3][E][K] (one slice per
// instance, allocated on first use), so that host copies of different
// instances need not wait for each other
static dg_status ensure_batch_stage(dg_batch* b, size_t doubles) {
  if (b->stage_n >= doubles) return DG_OK;
  if (b->stage) cudaFree(b->stage);
  b->stage = nullptr;
  b->stage_n = 0;
  CK(cudaMalloc((void**)&b->stage, sizeof(double) * doubles));
  b->stage_n = doubles;
  return DG_OK;
}

// Enqueue the transfer of instance i's state to host arrays (no
// synchronisation): in place for mapped page-locked arrays, else through the
// instance's staging slice.
static dg_status enqueue_get_state(dg_batch* b, int i, double* xi, double* qx, double* qy) {
  const HostInst& h = b->inst[i];
  const long long E = h.E, KE = (long long)h.K * E;
  const char* src = (const char*)b->w[0] + h.o_state;
  double* dst[3] = {xi, qx, qy};
  HostFields hf;
  if (mapped_fields(dst, KE, hf)) {
    // page-locked, mapped host arrays: written in place by one kernel
    const unsigned gf = fields_grid(E, h.K);
    if (b->arith == ARITH_FP64)
      soa_to_fields_kernel<double><<<gf, 256, 0, b->stream>>>((const double*)src, hf, E, h.K);
    else
      soa_to_fields_kernel<float><<<gf, 256, 0, b->stream>>>((const float*)src, hf, E, h.K);
    CK(cudaGetLastError());
    return DG_OK;
  }
  dg_status s = ensure_batch_stage(b, b->stage_total);
  if (s != DG_OK) return s;
  double* slice = b->stage + h.o_stage;
  // device transpose to element-major FP64, then one copy per field
  const unsigned g = (unsigned)((E + 127) / 128);
  if (b->arith == ARITH_FP64)
    soa_to_aos_kernel<double><<<g, 128, 0, b->stream>>>((const double*)src, slice, E, h.K, 3);
  else
    soa_to_aos_kernel<float><<<g, 128, 0, b->stream>>>((const float*)src, slice, E, h.K, 3);
  CK(cudaGetLastError());
  for (int f = 0; f < 3; ++f)
    if (dst[f])
      CK(cudaMemcpyAsync(dst[f], slice + (size_t)f * KE, sizeof(double) * KE, cudaMemcpyDeviceToHost, b->stream));
  return DG_OK;
}

dg_status dg_batch_get_state(dg_batch* b, int i, double* xi, double* qx, double* qy) {
  dgswe::NvtxRange nvtx_range("dg_batch_get_state");
  if (!b || i < 0 || i >= b->n) return DG_ERR_ARG;
  dg_status s = enqueue_get_state(b, i, xi, qx, qy);
  if (s != DG_OK) return s;
  CK(cudaStreamSynchronize(b->stream));
  return DG_OK;
}

dg_status dg_batch_get_states(dg_batch* b, double* const* xi, double* const* qx, double* const* qy) {
  dgswe::NvtxRange nvtx_range("dg_batch_get_states");
  if (!b || !xi || !qx || !qy) return DG_ERR_ARG;
  for (int i = 0; i < b->n; ++i) {
    dg_status s = enqueue_get_state(b, i, xi[i], qx[i], qy[i]);
    if (s != DG_OK) return s;
  }
  CK(cudaStreamSynchronize(b->stream));
  return DG_OK;
}

// Groups of dg_batch_step_host: tile-fused batches split every order class
// (p = 3 first) into runs of consecutive instances of about 1/16 of the
// batch's state bytes each (one instance at least), so that copies and
// compute overlap finely; other batches form one group.
constexpr int kStepGroups = 16;
struct StepGroup {
  int p, lo, hi;              // order class, items [lo, hi)
  std::vector<int> inst;      // its instances
};

static dg_status make_groups(const dg_batch* b, std::vector<StepGroup>& gs) {
  try {
    gs.clear();
    if (!b->tiled) {
      StepGroup g{0, 0, 0, {}};
      for (int i = 0; i < b->n; ++i) g.inst.push_back(i);
      gs.push_back(std::move(g));
      return DG_OK;
    }
    double total = 0.0;
    for (const HostInst& h : b->inst) total += 24.0 * h.K * h.E;
    const double target = total / kStepGroups;
    for (int p = 3; p >= 1; --p) {
      StepGroup g{p, 0, 0, {}};
      double bytes = 0.0;
      for (int i = 0; i < b->n; ++i) {
        if (b->inst[i].p != p) continue;
        if (g.inst.empty()) g.lo = b->item_lo[i];
        g.inst.push_back(i);
        g.hi = b->item_hi[i];
        bytes += 24.0 * b->inst[i].K * b->inst[i].E;
        if (bytes >= target) {
          gs.push_back(std::move(g));
          g = StepGroup{p, 0, 0, {}};
          bytes = 0.0;
        }
      }
      if (!g.inst.empty()) gs.push_back(std::move(g));
    }
  } catch (const std::exception&) {
    return DG_ERR_OOM;
  }
  return DG_OK;
}

// Copy streams, events and work counters of dg_batch_step_host
// (non-blocking streams: no implicit ordering with a legacy default
// stream; all ordering is by events)
static dg_status ensure_pipeline(dg_batch* b, size_t groups) {
  if (!b->s_up) CK(cudaStreamCreateWithFlags(&b->s_up, cudaStreamNonBlocking));
  if (!b->s_down) CK(cudaStreamCreateWithFlags(&b->s_down, cudaStreamNonBlocking));
  for (cudaEvent_t* e : {&b->ev_start, &b->ev_end})
    if (!*e) CK(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  try {   // reserved first, so that no push_back below can throw
    b->ev_up.reserve(groups);
    b->ev_done.reserve(groups);
  } catch (const std::exception&) {
    return DG_ERR_OOM;
  }
  while (b->ev_up.size() < groups) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreateWithFlags(&e0, cudaEventDisableTiming));
    const cudaError_t ce = cudaEventCreateWithFlags(&e1, cudaEventDisableTiming);
    if (ce != cudaSuccess) {
      cudaEventDestroy(e0);
      return cuda_status(ce);
    }
    b->ev_up.push_back(e0);
    b->ev_done.push_back(e1);
  }
  // sized once for the largest group count make_groups can give (at most
  // kStepGroups + 3: every class ends one partial group)
  if (!b->pcount) CK(cudaMalloc((void**)&b->pcount, sizeof(unsigned) * b->S * (kStepGroups + 3)));
  return DG_OK;
}

static dg_status step_host_impl(dg_batch* b, const double* const* xi_in, const double* const* qx_in,
                                const double* const* qy_in, double* const* xi_out, double* const* qx_out,
                                double* const* qy_out, double* t_out) {
  std::vector<StepGroup> gs;
  dg_status s = make_groups(b, gs);
  if (s == DG_OK && gs.size() > (size_t)(kStepGroups + 3)) s = DG_ERR_ARG;   // cannot happen: see make_groups
  if (s == DG_OK) s = ensure_batch_stage(b, b->stage_total);
  if (s == DG_OK) s = ensure_pipeline(b, gs.size());
  if (s != DG_OK) return s;
  const int ng = (int)gs.size();
  // per-instance records in group order (the groups depend only on the
  // instances' sizes: built once)
  std::vector<int> first(ng + 1, 0);
  for (int g = 0; g < ng; ++g) first[g + 1] = first[g] + (int)gs[g].inst.size();
  if (!b->xfer) {
    std::vector<XferInst> tab;
    try {
      for (const StepGroup& g : gs)
        for (int i : g.inst) {
          const HostInst& h = b->inst[i];
          tab.push_back({b->stage + h.o_stage, (char*)b->w[0] + h.o_state, (const char*)b->hb + h.o_hb, h.E, h.K, i,
                         float(h.cfg.g)});
        }
    } catch (const std::exception&) {
      return DG_ERR_OOM;
    }
    XferInst* d = nullptr;
    CK(cudaMalloc((void**)&d, sizeof(XferInst) * tab.size()));
    const cudaError_t ce = cudaMemcpy(d, tab.data(), sizeof(XferInst) * tab.size(), cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) {
      cudaFree(d);
      return cuda_status(ce);
    }
    b->xfer = d;
  }
  const cudaStream_t c = b->stream, up = b->s_up, down = b->s_down;
  // the copies start after the work already queued on the batch's stream
  CK(cudaEventRecord(b->ev_start, c));
  CK(cudaStreamWaitEvent(up, b->ev_start, 0));
  CK(cudaStreamWaitEvent(down, b->ev_start, 0));
  const double* const* in[3] = {xi_in, qx_in, qy_in};
  double* const* out[3] = {xi_out, qx_out, qy_out};
  // uploads, group by group (copy engine)
  for (int g = 0; g < ng; ++g) {
    for (int i : gs[g].inst) {
      const HostInst& h = b->inst[i];
      const long long KE = (long long)h.K * h.E;
      for (int f = 0; f < 3; ++f)
        CK(cudaMemcpyAsync(b->stage + h.o_stage + (size_t)f * KE, in[f][i], sizeof(double) * KE,
                           cudaMemcpyHostToDevice, up));
    }
    CK(cudaEventRecord(b->ev_up[g], up));
  }
  // compute: every group's state in, evaluated, stepped and out to staging
  // as soon as its upload is done; later groups' uploads and earlier
  // groups' downloads overlap it
  const int ep = b->ep, lc = b->lc;
  if (b->tiled) {
    CK(cudaMemsetAsync(b->pcount, 0, sizeof(unsigned) * b->S * ng, c));
    CK(cudaMemsetAsync(b->lam + (size_t)lc * b->n, 0, sizeof(double) * b->n, c));
    if (b->adaptive) CK(cudaMemsetAsync(b->lam + (size_t)(1 - lc) * b->n, 0, sizeof(double) * b->n, c));
  }
  for (int g = 0; g < ng; ++g) {
    CK(cudaStreamWaitEvent(c, b->ev_up[g], 0));
    // the group's staging slices -> states, then (tile-fused) their CFL
    // maxima: one launch each, one row of blocks per instance
    const int ni = first[g + 1] - first[g];
    const dim3 grid((unsigned)std::max(16, 1216 / ni), (unsigned)ni);
    if (b->arith == ARITH_FP64)
      group_in_kernel<double><<<grid, 256, 0, c>>>(b->xfer, first[g]);
    else
      group_in_kernel<float><<<grid, 256, 0, c>>>(b->xfer, first[g]);
    CK(cudaGetLastError());
    if (b->tiled) {
      group_wave_speed_kernel<<<grid, 256, 0, c>>>(b->xfer, first[g], b->lam + (size_t)lc * b->n);
      CK(cudaGetLastError());
    }
    if (b->tiled) {
      s = launch_range_step(b, gs[g].p, gs[g].lo, gs[g].hi, b->pcount + (size_t)g * b->S, ep, lc, c);
    } else {
      b->evaluated = false;
      s = launch_eval(b, c);
      cudaGraphExec_t gx;
      if (s == DG_OK) s = get_graph(b, &gx);
      if (s == DG_OK) CK(cudaGraphLaunch(gx, c));
    }
    if (s != DG_OK) return s;
    if (b->arith == ARITH_FP64)
      group_out_kernel<double><<<grid, 256, 0, c>>>(b->xfer, first[g]);
    else
      group_out_kernel<float><<<grid, 256, 0, c>>>(b->xfer, first[g]);
    CK(cudaGetLastError());
    CK(cudaEventRecord(b->ev_done[g], c));
    // downloads of this group (copy engine)
    CK(cudaStreamWaitEvent(down, b->ev_done[g], 0));
    for (int i : gs[g].inst) {
      const HostInst& h = b->inst[i];
      const long long KE = (long long)h.K * h.E;
      for (int f = 0; f < 3; ++f)
        CK(cudaMemcpyAsync(out[f][i], b->stage + h.o_stage + (size_t)f * KE, sizeof(double) * KE,
                           cudaMemcpyDeviceToHost, down));
    }
  }
  CK(cudaEventRecord(b->ev_end, down));
  CK(cudaStreamWaitEvent(c, b->ev_end, 0));
  b->ep = (b->ep + b->S) & 1;
  if (b->adaptive) b->lc = 1 - b->lc;
  b->evaluated = true;
  unsigned herr = 0;
  CK(cudaMemcpyAsync(&herr, b->err, sizeof herr, cudaMemcpyDeviceToHost, c));
  if (t_out) CK(cudaMemcpyAsync(t_out, b->t, sizeof(double) * b->n, cudaMemcpyDeviceToHost, c));
  CK(cudaStreamSynchronize(c));
  if (herr) {
    CK(cudaMemsetAsync(b->err, 0, sizeof(unsigned), c));
    CK(cudaStreamSynchronize(c));
  }
  if (herr & ERRF_NONFINITE) return DG_ERR_NONFINITE;
  if (herr & ERRF_DRY) return DG_ERR_DRY;
  return DG_OK;
}

dg_status dg_batch_step_host(dg_batch* b, const double* const* xi_in, const double* const* qx_in,
                             const double* const* qy_in, double* const* xi_out, double* const* qx_out,
                             double* const* qy_out, double* t_out) {
  dgswe::NvtxRange nvtx_range("dg_batch_step_host");
  if (!b || !xi_in || !qx_in || !qy_in || !xi_out || !qx_out || !qy_out) return DG_ERR_ARG;
  for (int i = 0; i < b->n; ++i)
    if (!xi_in[i] || !qx_in[i] || !qy_in[i] || !xi_out[i] || !qx_out[i] || !qy_out[i]) return DG_ERR_ARG;
  const dg_status s = step_host_impl(b, xi_in, qx_in, qy_in, xi_out, qx_out, qy_out, t_out);
  if (s != DG_OK && s != DG_ERR_DRY && s != DG_ERR_NONFINITE) {
    // a launch failed part-way: let the copies already queued finish before
    // the caller's arrays may go away
    if (b->s_up) cudaStreamSynchronize(b->s_up);
    if (b->s_down) cudaStreamSynchronize(b->s_down);
    cudaStreamSynchronize(b->stream);
  }
  return s;
}

dg_status dg_batch_set_state(dg_batch* b, int i, const double* xi, const double* qx, const double* qy, double t) {
  dgswe::NvtxRange nvtx_range("dg_batch_set_state");
  if (!b || i < 0 || i >= b->n || !xi || !qx || !qy) return DG_ERR_ARG;
  const HostInst& h = b->inst[i];
  const long long E = h.E, KE = (long long)h.K * E;
  // asynchronous: the caller keeps its arrays unchanged until the stream is
  // synchronised (dg_batch_run does).  Page-locked, mapped host arrays are
  // read in place by one kernel; others are copied into this instance's
  // staging slice (the copies of different instances overlap) and
  // transposed on the device.
  double* src[3] = {const_cast<double*>(xi), const_cast<double*>(qx), const_cast<double*>(qy)};
  char* dst = (char*)b->w[0] + h.o_state;
  HostFields hf;
  if (mapped_fields(src, KE, hf)) {
    const unsigned gf = fields_grid(E, h.K);
    if (b->arith == ARITH_FP64)
      fields_to_soa_kernel<double><<<gf, 256, 0, b->stream>>>(hf, (double*)dst, E, h.K);
    else
      fields_to_soa_kernel<float><<<gf, 256, 0, b->stream>>>(hf, (float*)dst, E, h.K);
  } else {
    dg_status s = ensure_batch_stage(b, b->stage_total);
    if (s != DG_OK) return s;
    double* slice = b->stage + h.o_stage;
    for (int f = 0; f < 3; ++f)
      CK(cudaMemcpyAsync(slice + (size_t)f * KE, src[f], sizeof(double) * KE, cudaMemcpyHostToDevice, b->stream));
    const unsigned g = (unsigned)((E + 127) / 128);
    if (b->arith == ARITH_FP64)
      aos_to_soa_kernel<double><<<g, 128, 0, b->stream>>>(slice, (double*)dst, E, h.K, 3);
    else
      aos_to_soa_kernel<float><<<g, 128, 0, b->stream>>>(slice, (float*)dst, E, h.K, 3);
  }
  CK(cudaGetLastError());
  set_scalar_kernel<<<1, 1, 0, b->stream>>>(b->t + i, t);   // t by value: no host memory outlives the call
  CK(cudaGetLastError());
  b->evaluated = false;   // the next run re-evaluates every instance
  return DG_OK;
}

// Autotuner: times trial_steps steps at every candidate launch shape on the
// batch's own state, restoring the state after each, and keeps the fastest.
// Per-element kernels: 32, 64, 96, 128 elements per work item; tile-fused
// kernels: tiles of 8 x 8, 16 x 8 and 8 x 4 quads (128, 256 and 64 owned
// triangles per CTA; reported as tile_shape 1, 2, 3), each order class's
// launches timed separately (eager steps) so that every class keeps its own
// fastest shape.  ms_out[4] receives the time per step of each
// candidate in that order (0 where there is none).
dg_status dg_batch_autotune(dg_batch* b, int trial_steps, int* block_out, double* ms_out) {
  dgswe::NvtxRange nvtx_range("dg_batch_autotune");
  if (!b || trial_steps < 1) return DG_ERR_ARG;
  CK(cudaStreamSynchronize(b->stream));
  // snapshot of everything a step changes
  void* save = nullptr;
  double* save_t = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const int ep0 = b->ep, lc0 = b->lc;
  const int cand_el[4] = {32, 64, 96, 128}, cand_tile[4] = {0, 1, 2, -1};
  const int* cand = b->tiled ? cand_tile : cand_el;
  if (ms_out)
    for (int c = 0; c < 4; ++c) ms_out[c] = 0.0;
  double best = 1e300;
  int best_block = b->block;
  // tile-fused batches: each order class keeps the shape of its fastest launches
  double cls_best[4] = {1e300, 1e300, 1e300, 1e300};
  int cls_pick[4] = {0, 0, 0, 0};
  dg_status s = DG_OK;
  cudaError_t ce = cudaMalloc(&save, b->sz_state);
  if (ce == cudaSuccess) ce = cudaMalloc((void**)&save_t, sizeof(double) * b->n);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(save, b->w[0], b->sz_state, cudaMemcpyDeviceToDevice, b->stream);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(save_t, b->t, sizeof(double) * b->n, cudaMemcpyDeviceToDevice, b->stream);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  for (int c = 0; c < 4 && ce == cudaSuccess && s == DG_OK; ++c) {
    const int block = cand[c];
    if (block < 0) break;
    if ((s = build_items(b, block)) != DG_OK) break;
    b->evaluated = false;
    b->ep = ep0;
    b->lc = lc0;
    if ((s = dg_batch_run(b, 1, nullptr)) != DG_OK) break;   // warm-up, graph build
    float ms = 0.f;
    if (b->tiled) {
      // eager steps, every order class's launches timed on their own
      double cls_ms[4] = {0.0, 0.0, 0.0, 0.0};
      for (int k = 0; k < trial_steps && s == DG_OK; ++k) {
        s = launch_step(b, b->ep, b->lc, b->stream, cls_ms);
        b->ep = (b->ep + b->S) & 1;
        if (b->adaptive) b->lc = 1 - b->lc;
      }
      for (int p = 1; p <= 3; ++p) {
        ms += (float)cls_ms[p];
        if (b->cls_end[p] > b->cls_begin[p] && cls_ms[p] < cls_best[p]) {
          cls_best[p] = cls_ms[p];
          cls_pick[p] = block;
        }
      }
    } else {
      ce = cudaEventRecord(e0, b->stream);
      for (int k = 0; k < trial_steps && ce == cudaSuccess && s == DG_OK; ++k) {
        cudaGraphExec_t g;
        if ((s = get_graph(b, &g)) != DG_OK) break;
        ce = cudaGraphLaunch(g, b->stream);
        b->ep = (b->ep + b->S) & 1;
        if (b->adaptive) b->lc = 1 - b->lc;
      }
      if (ce == cudaSuccess && s == DG_OK) ce = cudaEventRecord(e1, b->stream);
      if (ce == cudaSuccess && s == DG_OK) ce = cudaEventSynchronize(e1);
      if (ce == cudaSuccess && s == DG_OK) ce = cudaEventElapsedTime(&ms, e0, e1);
    }
    const double per = ms / trial_steps;
    if (ms_out) ms_out[c] = per;
    if (ce == cudaSuccess && s == DG_OK && per < best) {
      best = per;
      best_block = block;
    }
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(b->w[0], save, b->sz_state, cudaMemcpyDeviceToDevice, b->stream);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(b->t, save_t, sizeof(double) * b->n, cudaMemcpyDeviceToDevice, b->stream);
  }
  const cudaError_t ce2 = cudaStreamSynchronize(b->stream);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (save) cudaFree(save);
  if (save_t) cudaFree(save_t);
  b->ep = ep0;
  b->lc = lc0;
  b->evaluated = false;   // re-evaluate the restored state
  if (s != DG_OK) return s;
  if (ce != cudaSuccess) return cuda_status(ce);
  if (ce2 != cudaSuccess) return cuda_status(ce2);
  if (b->tiled) {
    if ((s = build_items_impl(b, best_block, cls_pick)) != DG_OK) return s;
  } else if ((s = build_items(b, best_block)) != DG_OK) {
    return s;
  }
  // tile shapes are reported in dg_config.tile_shape numbering (1, 2, 3):
  // the shape of the highest order class present
  if (block_out) {
    *block_out = best_block;
    if (b->tiled)
      for (int p = 1; p <= 3; ++p)
        if (b->cls_end[p] > b->cls_begin[p]) *block_out = b->cls_shape[p] + 1;
  }
  return DG_OK;
}

int dg_batch_tile_shape(const dg_batch* b, int p) {
  if (!b || !b->tiled || p < 1 || p > 3 || b->cls_end[p] <= b->cls_begin[p]) return 0;
  return b->cls_shape[p] + 1;
}

}  // extern "C"
