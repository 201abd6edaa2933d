// dg_batch.cuh -- many independent instances (uneven mesh sizes and orders
// p = 1..3) advanced by one persistent launch per RK stage.
//
// Work items are (instance, first element) blocks of blockDim elements,
// ordered by decreasing p (the most expensive work first).  Each CTA pulls
// items from a global counter until none is left; every element's work is
// independent of which CTA does it, so results are deterministic and equal
// to the single-instance kernels (stage_element is shared).  Each instance
// has its own CFL time step: the wave-speed maximum of an item goes to its
// instance's slot.
#pragma once

#include "dg_kernels.cuh"
#include "dg_tile.cuh"

namespace dgswe {

// device descriptor of one instance
struct BatchInst {
  Mesh m;
  double g, inv_det, cfl_num, dt_fixed;
  double det, tau_bf, f_c;
  void* w[3];          // state buffers (instance's own SoA arrays)
  void* vs[2];
  void* rec[2];
  const void* hb;
  const void* hbt;
  const void* ghb;
  const void* lin;     // FP64 batches: [2][K][K][E], else null
  const float* ahb;    // mixed-solve batches: [ahb_words(K)][E] parts of A_hb, else null
  double* lam;         // slot s of this instance at lam[s * n_inst]
  double* t;
  int p;
};

struct BatchItem {
  int inst;
  int start;
};

struct BatchArgs {
  const BatchInst* inst;
  const BatchItem* items;
  int n_items, n_inst;
  unsigned* counter;   // zeroed before the launch
  unsigned* err;
  int win, wout, pin;  // state in/out buffer, evaluation buffer read (MODE_STAGE)
  double alpha, beta;
  int lc;              // wave-speed slot of the current step
  int last;            // last stage: wave speed -> slot 1-lc, t += dt
  int item_begin;      // tile-fused batches: this launch's items are
                       // [item_begin, n_items) (one order class)
};

template <class Real, class PR, int MODE>
__global__ void __launch_bounds__(128, (stage_min_blocks<3, Real, PR>())) batch_kernel(const BatchArgs a) {
  __shared__ int s_item;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = (int)atomicAdd(a.counter, 1u);
    __syncthreads();
    const int it = s_item;
    if (it >= a.n_items) break;
    const BatchItem item = a.items[it];
    const BatchInst& d = a.inst[item.inst];
    StageParams<Real> sp;
    sp.m = d.m;
    sp.g = Real(d.g);
    sp.hb = static_cast<const Real*>(d.hb);
    sp.hbt = static_cast<const Real*>(d.hbt);
    sp.ghb = static_cast<const Real*>(d.ghb);
    sp.lin = static_cast<const Real*>(d.lin);
    sp.ahb = d.ahb;
    sp.inv_det = d.inv_det;
    sp.det = d.det;
    sp.tau_bf = d.tau_bf;
    sp.f_c = d.f_c;
    sp.err = a.err;
    sp.dt_fixed = d.dt_fixed;
    sp.cfl_num = d.cfl_num;
    sp.alpha = a.alpha;
    sp.beta = a.beta;
    sp.w0 = static_cast<const Real*>(d.w[0]);
    sp.rhs_out = nullptr;
    sp.lam_clear = nullptr;
    sp.forcing = 0;
    sp.dirichlet = 0;
    sp.t_now = nullptr;
    sp.c_eval = 0.0;
    sp.vq = nullptr;
    sp.nqv = 0;
    sp.eq = nullptr;
    sp.nqe = 0;
    double* lam_target = nullptr;
    double dt = 0.0;
    if constexpr (MODE == MODE_EVAL) {
      sp.w = static_cast<const Real*>(d.w[0]);
      sp.vs = nullptr;
      sp.rec = nullptr;
      sp.vs_out = static_cast<Real*>(d.vs[a.pin]);
      sp.rec_out = static_cast<Real*>(d.rec[a.pin]);
      sp.wout = nullptr;
      sp.lam = nullptr;
      lam_target = d.lam + (long long)a.lc * a.n_inst;
    } else {
      sp.w = static_cast<const Real*>(d.w[a.win]);
      sp.wout = static_cast<Real*>(d.w[a.wout]);
      sp.vs = static_cast<const Real*>(d.vs[a.pin]);
      sp.rec = static_cast<const Real*>(d.rec[a.pin]);
      sp.vs_out = static_cast<Real*>(d.vs[1 - a.pin]);
      sp.rec_out = static_cast<Real*>(d.rec[1 - a.pin]);
      sp.lam = d.lam + (long long)a.lc * a.n_inst;
      dt = d.dt_fixed > 0.0 ? d.dt_fixed : d.cfl_num / sp.lam[0];
      if (a.last && !(d.dt_fixed > 0.0)) lam_target = d.lam + (long long)(1 - a.lc) * a.n_inst;
    }
    sp.lam_next = lam_target;
    const long long e = (long long)item.start + threadIdx.x;
    double lam_e = 0.0;
    unsigned err = 0;
    if (e < d.m.E) {
      switch (d.p) {
        case 1: stage_element<1, Real, PR, MODE, 0>(sp, e, dt, lam_e, err); break;
        case 2: stage_element<2, Real, PR, MODE, 0>(sp, e, dt, lam_e, err); break;
        default: stage_element<3, Real, PR, MODE, 0>(sp, e, dt, lam_e, err); break;
      }
    }
    if (lam_target) {
      const double l = block_max(lam_e);
      if (threadIdx.x == 0) atomic_max_nonneg(lam_target, l);
    }
    if (err) atomicOr(a.err, err);
    if (MODE == MODE_STAGE && a.last && item.start == 0 && threadIdx.x == 0) *d.t += dt;
  }
}

// Tile-fused form of the batched stage (FP32 state): one persistent launch
// per order class and RK stage, each compiled for its order P (its own
// register budget, shared memory and tile shape); work items are
// (instance, tile) pairs of that class, items [item_begin, n_items) of the
// batch's list.  The per-tile work is tile_stage_body, as in the
// single-instance tile kernel, so results equal those of single contexts.
template <class PR, int P, int TX, int TY>
__global__ void __launch_bounds__(TileShape<TX, TY>::NT, (tile_min_blocks<P, TX, TY>()))
    batch_tile_kernel(const BatchArgs a) {
  extern __shared__ float tile_smem[];
  __shared__ int s_item;
  __shared__ double s_dt;
  __shared__ TileUpdate s_up;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      // the item, its instance's step and the update constants, formed once
      // for the CTA (as tile_update forms them)
      const int it = a.item_begin + (int)atomicAdd(a.counter, 1u);
      s_item = it;
      if (it < a.n_items) {
        const BatchInst& d0 = a.inst[a.items[it].inst];
        const double dt0 = d0.dt_fixed > 0.0 ? d0.dt_fixed : d0.cfl_num / d0.lam[(long long)a.lc * a.n_inst];
        s_dt = dt0;
        s_up.c = float(dt0 * d0.inv_det);
        s_up.beta = float(a.beta);
        s_up.with_base = a.alpha != 0.0;
      }
    }
    __syncthreads();
    const int it = s_item;
    if (it >= a.n_items) break;
    const BatchItem item = a.items[it];
    const BatchInst& d = a.inst[item.inst];
    StageParams<float> sp;
    sp.m = d.m;
    sp.g = float(d.g);
    sp.hb = static_cast<const float*>(d.hb);
    sp.hbt = static_cast<const float*>(d.hbt);
    sp.ghb = static_cast<const float*>(d.ghb);
    sp.lin = nullptr;
    sp.ahb = d.ahb;
    sp.inv_det = d.inv_det;
    sp.det = d.det;
    sp.tau_bf = d.tau_bf;
    sp.f_c = d.f_c;
    sp.err = a.err;
    sp.dt_fixed = d.dt_fixed;
    sp.cfl_num = d.cfl_num;
    sp.alpha = a.alpha;
    sp.beta = a.beta;
    sp.w = static_cast<const float*>(d.w[a.win]);
    sp.wout = static_cast<float*>(d.w[a.wout]);
    sp.w0 = static_cast<const float*>(d.w[0]);
    sp.vs = sp.rec = nullptr;
    sp.vs_out = sp.rec_out = sp.rhs_out = nullptr;
    sp.lam_clear = nullptr;
    sp.forcing = 0;
    sp.dirichlet = 0;
    sp.t_now = nullptr;
    sp.c_eval = 0.0;
    sp.vq = nullptr;
    sp.nqv = 0;
    sp.eq = nullptr;
    sp.nqe = 0;
    sp.lam = d.lam + (long long)a.lc * a.n_inst;
    const double dt = s_dt;
    double* lam_target = (a.last && !(d.dt_fixed > 0.0)) ? d.lam + (long long)(1 - a.lc) * a.n_inst : nullptr;
    sp.lam_next = lam_target;
    const int tiles_x = (d.m.nx + TX - 1) / TX;
    float lam_e = 0.f;
    unsigned err = 0;
    const TileUpdate up = s_up;
    tile_stage_body<P, PR, TX, TY>(sp, item.start, tiles_x, up, tile_smem, lam_e, err);
    if (lam_target) {
      const float l = block_max_f(lam_e);
      if (threadIdx.x == 0) atomic_max_nonneg(lam_target, double(l));
    }
    if (err) atomicOr(a.err, err);
    if (a.last && item.start == 0 && threadIdx.x == 0) *d.t += dt;
  }
}

template <class PR, int P, int TX, int TY>
cudaError_t batch_tile_launch_shape(int grid, const BatchArgs& a, cudaStream_t s) {
  auto kern = batch_tile_kernel<PR, P, TX, TY>;
  const size_t smem = sizeof(float) * tile_smem_floats<P, TX, TY>();
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, TileShape<TX, TY>::NT, smem, s>>>(a);
  return cudaGetLastError();
}

template <class PR, int P, int TX, int TY>
cudaError_t batch_tile_occupancy_shape(int* blocks_per_sm) {
  auto kern = batch_tile_kernel<PR, P, TX, TY>;
  const size_t smem = sizeof(float) * tile_smem_floats<P, TX, TY>();
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kern, TileShape<TX, TY>::NT, smem);
}

// launch / occupancy of order P with tile shape index 0..2
template <class PR, int P>
cudaError_t batch_tile_launch_p(int shape, int grid, const BatchArgs& a, cudaStream_t s) {
  if (shape == 1) return batch_tile_launch_shape<PR, P, 16, 8>(grid, a, s);
  if (shape == 2) return batch_tile_launch_shape<PR, P, 8, 4>(grid, a, s);
  return batch_tile_launch_shape<PR, P, 8, 8>(grid, a, s);
}
template <class PR, int P>
cudaError_t batch_tile_occupancy_p(int shape, int* blocks_per_sm) {
  if (shape == 1) return batch_tile_occupancy_shape<PR, P, 16, 8>(blocks_per_sm);
  if (shape == 2) return batch_tile_occupancy_shape<PR, P, 8, 4>(blocks_per_sm);
  return batch_tile_occupancy_shape<PR, P, 8, 8>(blocks_per_sm);
}

// quads per tile side of each shape (kTileShapes entries)
__host__ __device__ constexpr int tile_tx(int shape) { return shape == 1 ? 16 : 8; }
__host__ __device__ constexpr int tile_ty(int shape) { return shape == 2 ? 4 : 8; }

#define DGSWE_BATCH_TILE_DECLARE_P(SUFFIX, P)                                                               \
  cudaError_t batch_tile_launch_##SUFFIX##_p##P(int shape, int grid, const BatchArgs& a, cudaStream_t s);    \
  cudaError_t batch_tile_occupancy_##SUFFIX##_p##P(int shape, int* blocks_per_sm);
#define DGSWE_BATCH_TILE_DECLARE(SUFFIX)                                                                 \
  DGSWE_BATCH_TILE_DECLARE_P(SUFFIX, 1)                                                                  \
  DGSWE_BATCH_TILE_DECLARE_P(SUFFIX, 2)                                                                  \
  DGSWE_BATCH_TILE_DECLARE_P(SUFFIX, 3)                                                                  \
  cudaError_t batch_tile_launch_##SUFFIX(int p, int shape, int grid, const BatchArgs& a, cudaStream_t s);  \
  cudaError_t batch_tile_occupancy_##SUFFIX(int p, int shape, int* blocks_per_sm);
DGSWE_BATCH_TILE_DECLARE(fp32p64)
DGSWE_BATCH_TILE_DECLARE(fp32p32)
DGSWE_BATCH_TILE_DECLARE(fp32pdf)
DGSWE_BATCH_TILE_DECLARE(fp32pir)

// Launch and occupancy of one (arithmetic, mode) instantiation; each is
// compiled separately from dg_batch_inst.cu (build flags select it), and the
// per-arithmetic dispatchers batch_launch_<suffix>(mode, ...) and
// batch_occupancy_<suffix> live in dg_dispatch.cu.
#define DGSWE_BATCH_DECLARE(SUFFIX)                                                                  \
  cudaError_t batch_launch_##SUFFIX##_m0(int grid, int block, const BatchArgs& a, cudaStream_t s);  \
  cudaError_t batch_launch_##SUFFIX##_m1(int grid, int block, const BatchArgs& a, cudaStream_t s);  \
  cudaError_t batch_occupancy_##SUFFIX##_m0(int block, int* blocks_per_sm);                         \
  cudaError_t batch_occupancy_##SUFFIX##_m1(int block, int* blocks_per_sm);                         \
  cudaError_t batch_launch_##SUFFIX(int mode, int grid, int block, const BatchArgs& a, cudaStream_t s); \
  cudaError_t batch_occupancy_##SUFFIX(int block, int* blocks_per_sm);
DGSWE_BATCH_DECLARE(fp64)
DGSWE_BATCH_DECLARE(fp32p64)
DGSWE_BATCH_DECLARE(fp32p32)
DGSWE_BATCH_DECLARE(fp32pdf)
DGSWE_BATCH_DECLARE(fp32pir)

}  // namespace dgswe
