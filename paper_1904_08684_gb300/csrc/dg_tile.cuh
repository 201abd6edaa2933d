// dg_tile.cuh -- tile-fused RK stage for FP32 state on uniform quad-split
// meshes (arXiv:1904.08684, §2.2 scheme; §2.3 mesh).
//
// One CTA owns a tile of TX x TY quads (2 TX TY triangles) and, per tile,
// evaluates the stage's input state in shared memory instead of handing
// intermediates to the next launch through HBM:
//   phase 1  every owned triangle: velocity projection (Eq. (12)), volume +
//            source integrals (Eqs. (15)-(16), r of Eq. (5)) and its three
//            side records (traces, projected edge fluxes, wave speed);
//            every halo triangle (the neighbour across a tile-boundary edge,
//            one per boundary edge): velocity projection and the one side
//            record of the shared edge -- recomputed, never read from HBM;
//   phase 2  every owned triangle: Lax-Friedrichs flux of its three edges
//            from the two side records, lift, inverse mass, SSP stage
//            update, written to HBM; on the last stage the element wave
//            speed of the new state for the next step's CFL maximum.
// HBM traffic per owned triangle and stage is therefore the state (3K), the
// RK base (3K), the bathymetry fields and the new state (3K), plus the halo
// triangles' state (one per boundary edge of the tile, read again by the
// neighbouring tile, mostly from L2).  The side records and volume integrals
// of the per-element kernels (stage_kernel) never reach HBM.
//
// The element arithmetic is the per-element kernels' own (evaluate_to,
// side_record, edge_flux_lift_at, the update of stage_element): only where
// the intermediates live differs, so the two kernel forms agree to FP32
// rounding.
#pragma once

#include <cuda_runtime.h>

#include "dg_launch.cuh"

namespace dgswe {

// Tile shape: TX x TY quads.  Thread slots: owned triangle (ii, jj, t) at
// 2 (jj TX + ii) + t, then 2 (TX + TY) halo slots: left (TY), right (TY),
// bottom (TX), top (TX).
template <int TX, int TY>
struct TileShape {
  static constexpr int NO = 2 * TX * TY;        // owned triangles
  static constexpr int NH = 2 * (TX + TY);      // halo triangles
  static constexpr int NT = NO + NH;            // threads per CTA
};

// floats of dynamic shared memory: the owned triangles' side records
// [3][NREC][NO], the halo triangles' one record each [NREC][NH], the owned
// volume integrals [3K][NO] and the owned RK base state [3K][NO]
template <int P, int TX, int TY>
__host__ __device__ constexpr int tile_smem_floats() {
  return (3 * Dims<P>::NREC + 6 * Dims<P>::K) * TileShape<TX, TY>::NO + Dims<P>::NREC * TileShape<TX, TY>::NH;
}

// 4-byte asynchronous copy global -> shared (no register is held while the
// copy is in flight); completed by cp_async_wait_all
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Resident CTAs per SM requested from the register allocator: as many as
// leave ~128 registers per thread (~80 at p <= 1, whose element work is
// small and whose shared memory leaves room for more CTAs), but no more than
// the shared memory of an SM (227 KB per CTA at most, ~228 KB per SM) holds.
template <int P, int TX, int TY>
constexpr int tile_min_blocks() {
  constexpr int threads = (TileShape<TX, TY>::NT + 31) / 32 * 32;
  constexpr int by_regs = 65536 / (threads * (P <= 1 ? 80 : 128));
  constexpr int by_smem = (228 * 1024) / (4 * tile_smem_floats<P, TX, TY>() + 1024);
  constexpr int b = by_regs < by_smem ? by_regs : by_smem;
  return b > 0 ? b : 1;
}

// Tile shapes of the launchers: index 0 = 8 x 8 quads, 1 = 16 x 8, 2 = 8 x 4
// (dg_config.tile_shape 1, 2, 3).
constexpr int kTileShapes = 3;

// Halo slot h of the tile at quad (i0, j0) with valid extent TXv x TYv: the
// element f across the tile boundary and the local edge n (1 or 2) it shares
// with the tile (the same local index on both sides).  False if there is no
// such element (a wall, an anchor outside a partial tile, or a periodic
// neighbour that lies inside the tile itself).
template <int TX, int TY>
__device__ __forceinline__ bool halo_element(const Mesh& m, int h, int i0, int j0, int TXv, int TYv, long long& f,
                                             int& n) {
  int ii, jj, t;
  if (h < TY) {              // left: across the west side of owned (0, jj, 0)
    ii = 0; jj = h; t = 0; n = 1;
    if (jj >= TYv) return false;
  } else if (h < 2 * TY) {   // right: across the east side of owned (TXv-1, jj, 1)
    ii = TXv - 1; jj = h - TY; t = 1; n = 1;
    if (jj >= TYv) return false;
  } else if (h < 2 * TY + TX) {   // bottom: across the south side of owned (ii, 0, 0)
    ii = h - 2 * TY; jj = 0; t = 0; n = 2;
    if (ii >= TXv) return false;
  } else {                   // top: across the north side of owned (ii, TYv-1, 1)
    ii = h - 2 * TY - TX; jj = TYv - 1; t = 1; n = 2;
    if (ii >= TXv) return false;
  }
  const long long e = 2LL * ((long long)(j0 + jj) * m.nx + (i0 + ii)) + t;
  f = neighbour(m, e, n);
  if (f < 0) return false;
  const long long q = f >> 1;
  const int qi = (int)(q % m.nx), qj = (int)(q / m.nx);
  return !(qi >= i0 && qi < i0 + TXv && qj >= j0 && qj < j0 + TYv);
}

// Slot of the element across local edge n of the owned triangle (ii, jj, t)
// (global index e): an owned slot, the halo slot of halo_element, or -1 on a
// wall.
template <int TX, int TY>
__device__ __forceinline__ int neighbour_slot(const Mesh& m, long long e, int ii, int jj, int t, int n, int i0,
                                              int j0, int TXv, int TYv) {
  constexpr int NO = TileShape<TX, TY>::NO;
  if (n == 0) return 2 * (jj * TX + ii) + (1 - t);
  const long long f = neighbour(m, e, n);
  if (f < 0) return -1;
  const long long q = f >> 1;
  const int di = (int)(q % m.nx) - i0, dj = (int)(q / m.nx) - j0;
  if (di >= 0 && di < TXv && dj >= 0 && dj < TYv) return 2 * (dj * TX + di) + (int)(f & 1);
  if (n == 1) return NO + (t == 0 ? jj : TY + jj);
  return NO + 2 * TY + (t == 0 ? ii : TX + ii);
}

// Per-launch (per-item in a batch) constants of the stage update, formed once
// in FP64 and rounded as stage_element rounds them: c = dt / |det B| and
// beta; with_base = (alpha != 0).
struct TileUpdate {
  float c, beta;
  bool with_base;
};
__device__ __forceinline__ TileUpdate tile_update(const StageParams<float>& sp, double dt) {
  TileUpdate u;
  u.c = float(dt * sp.inv_det);
  u.beta = float(sp.beta);
  u.with_base = sp.alpha != 0.0;
  return u;
}

// One tile of one RK stage: the stage's input state sp.w is evaluated here,
// then updated into sp.wout (w' = w0 + beta ((w - w0) + dt R),
// R = res / |det B|, as stage_element).  All threads of the CTA call it; it
// ends with a barrier, so the next tile may reuse the shared memory.
// lam_acc collects the new state's element wave speeds (sp.lam_next set).
template <int P, class PR, int TX, int TY>
__device__ __forceinline__ void tile_stage_body(const StageParams<float>& sp, int tile, int tiles_x,
                                                const TileUpdate& up, float* tile_smem, float& lam_acc,
                                                unsigned& err) {
  using D = Dims<P>;
  using TS = TileShape<TX, TY>;
  constexpr int K = D::K, NREC = D::NREC, NO = TS::NO, NH = TS::NH;
  float* s_rec = tile_smem;                   // [3][NREC][NO] owned side records
  float* s_hrec = s_rec + 3 * NREC * NO;      // [NREC][NH] halo side records
  float* s_vs = s_hrec + NREC * NH;           // [3K][NO] volume integrals
  float* s_w0 = s_vs + 3 * K * NO;            // [3K][NO] RK base state
  const int tid = threadIdx.x;
  const long long E = sp.m.E;
  const int nx = sp.m.nx, ny = sp.m.ny;
  const int i0 = (tile % tiles_x) * TX, j0 = (tile / tiles_x) * TY;
  const int TXv = min(TX, nx - i0), TYv = min(TY, ny - j0);
  // owned slot coordinates (threads tid < NO)
  const int t = tid & 1, ii = (tid >> 1) % TX, jj = (tid >> 1) / TX;
  const bool owned = tid < NO && ii < TXv && jj < TYv;
  const long long e = 2LL * ((long long)(j0 + jj) * nx + (i0 + ii)) + t;
  // the RK base state is needed only by the update of phase 2: its first
  // read from HBM is issued now, asynchronously, and lands in shared memory
  // while phase 1 computes
  const bool with_base = up.with_base;
  if (owned && with_base) {
    sfor<0, 3 * K>([&](auto k) { cp_async4(s_w0 + CV(k) * NO + tid, sp.w0 + CV(k) * E + e); });
  }
  // ---- phase 1: evaluation of the input state into shared memory.  Owned
  // and halo threads run the same code (one copy of the velocity solve in
  // the instruction stream); a halo triangle writes only the record of the
  // edge it shares with the tile (its local edge n, 1 or 2).
  long long f = e;
  int n = 0;
  const bool halo = tid >= NO && halo_element<TX, TY>(sp.m, tid - NO, i0, j0, TXv, TYv, f, n);
  if (owned || halo) {
    const int tf = (int)(f & 1);
    float w[3][K], hb[K], H[K], u[K], v[K];
    sfor<0, 3>([&](auto c) {
      sfor<0, K>([&](auto i) { w[CV(c)][CV(i)] = sp.w[(CV(c) * K + CV(i)) * E + f]; });
    });
    element_velocity<P, float, PR>(sp, f, w[0], w[1], w[2], hb, H, u, v, err);
    if (owned) volume_to<P, float, 0>(sp, f, tf, w[0], w[1], w[2], u, v, hb, 0.0, s_vs + tid, NO);
    // records: owned at s_rec (stride NO), a halo triangle's at s_hrec (stride NH)
    float* rb = owned ? s_rec + tid : s_hrec + (tid - NO);
    const int rs = owned ? NO : NH;
    if (owned) side_record<0, P, 0>(sp, f, tf, w[0], w[1], w[2], u, v, err, 0.0, rb, rs);
    if (owned || n == 1)
      side_record<1, P, 0>(sp, f, tf, w[0], w[1], w[2], u, v, err, 0.0, rb + (owned ? NREC * NO : 0), rs);
    if (owned || n == 2)
      side_record<2, P, 0>(sp, f, tf, w[0], w[1], w[2], u, v, err, 0.0, rb + (owned ? 2 * NREC * NO : 0), rs);
  }
  cp_async_wait_all();
  __syncthreads();
  // ---- phase 2: fluxes, lift, stage update of the owned triangles
  if (owned) {
    float res[3][K];
    sfor<0, 3>([&](auto f) {
      sfor<0, K>([&](auto i) { res[CV(f)][CV(i)] = s_vs[(CV(f) * K + CV(i)) * NO + tid]; });
    });
    sfor<0, 3>([&](auto nn) {
      constexpr int n = CV(nn);
      const int ns = neighbour_slot<TX, TY>(sp.m, e, ii, jj, t, n, i0, j0, TXv, TYv);
      const float* ro = s_rec + n * NREC * NO + tid;
      const float* rn = ns < 0 ? nullptr : ns < NO ? s_rec + n * NREC * NO + ns : s_hrec + (ns - NO);
      edge_flux_lift_at<n, P, 0>(sp, e, t, ro, NO, rn, ns < NO ? NO : NH, res);
    });
    const float b = up.beta, c = up.c;
    bool fin = true;
    float x0[3];
    sfor<0, 3>([&](auto f) {
      sfor<0, K>([&](auto i) {
        const long long idx = (CV(f) * K + CV(i)) * E + e;
        const float wv = sp.w[idx];
        float x;
        if (with_base) {
          const float base = s_w0[(CV(f) * K + CV(i)) * NO + tid];
          x = fmaf(b, fmaf(c, res[CV(f)][CV(i)], wv - base), base);
        } else {
          x = fmaf(c, res[CV(f)][CV(i)], wv);
        }
        fin = fin && isfinite(x);
        sp.wout[idx] = x;
        if constexpr (CV(i) == 0) x0[CV(f)] = x;
      });
    });
    if (!fin) err |= ERRF_NONFINITE;
    if (sp.lam_next) {
      const float H0 = x0[0] + sp.hb[e];
      lam_acc = fmaxf(lam_acc, element_wave_speed_H(H0, x0[1], x0[2], sp.g));
    }
  }
  __syncthreads();
}

// One RK stage of every tile (persistent grid striding over tiles).
template <int P, class PR, int TX, int TY>
__global__ void __launch_bounds__(TileShape<TX, TY>::NT, (tile_min_blocks<P, TX, TY>()))
    tile_stage_kernel(const StageParams<float> sp, int tiles_x, int n_tiles) {
  extern __shared__ float tile_smem[];
  const double dt = sp.dt_fixed > 0.0 ? sp.dt_fixed : sp.cfl_num / sp.lam[0];
  const TileUpdate up = tile_update(sp, dt);
  float lam_acc = 0.f;
  unsigned err = 0;
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x)
    tile_stage_body<P, PR, TX, TY>(sp, tile, tiles_x, up, tile_smem, lam_acc, err);
  if (sp.lam_next) {
    const float l = block_max_f(lam_acc);
    if (threadIdx.x == 0) atomic_max_nonneg(sp.lam_next, double(l));
  }
  if (err) atomicOr(sp.err, err);
}

// Largest element wave speed of a state (the CFL maximum of its step), for
// the first step after the state was set: max_e |q_bar/H_bar| + sqrt(g H_bar)
// into *lam (zeroed by the caller), with the same operations as the stage
// kernels (g in the state's precision), so that a state set from the host
// continues with the bits of an uninterrupted run.
template <class Real>
__global__ void __launch_bounds__(256) wave_speed_kernel(Mesh m, Real g, int K, const Real* __restrict__ w,
                                                         const Real* __restrict__ hb, double* lam) {
  const long long E = m.E;
  double l = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (long long)gridDim.x * blockDim.x) {
    const Real H0 = w[e] + hb[e];
    l = fmax(l, double(element_wave_speed_H(H0, w[(long long)K * E + e], w[2LL * K * E + e], g)));
  }
  l = block_max(l);
  if (threadIdx.x == 0) atomic_max_nonneg(lam, l);
}

// Launchers of one (solve arithmetic, order), compiled from dg_tile_inst.cu
// (tile shapes as kTileShapes).
#define DGSWE_TILE_NAME(SUFFIX, P) DGSWE_PASTE4(tile_, SUFFIX, _p, P)
#define DGSWE_DECLARE_TILE_P(SUFFIX, P) \
  cudaError_t DGSWE_TILE_NAME(SUFFIX, P)(int shape, const StageParams<float>& sp, cudaStream_t s);
#define DGSWE_DECLARE_TILE_ALL(SUFFIX) \
  DGSWE_DECLARE_TILE_P(SUFFIX, 0)      \
  DGSWE_DECLARE_TILE_P(SUFFIX, 1)      \
  DGSWE_DECLARE_TILE_P(SUFFIX, 2)      \
  DGSWE_DECLARE_TILE_P(SUFFIX, 3)      \
  DGSWE_DECLARE_TILE_P(SUFFIX, 4)
DGSWE_DECLARE_TILE_ALL(fp32p64)
DGSWE_DECLARE_TILE_ALL(fp32p32)
DGSWE_DECLARE_TILE_ALL(fp32pdf)
DGSWE_DECLARE_TILE_ALL(fp32pir)
cudaError_t tile_fp32p64(int p, int shape, const StageParams<float>& sp, cudaStream_t s);
cudaError_t tile_fp32p32(int p, int shape, const StageParams<float>& sp, cudaStream_t s);
cudaError_t tile_fp32pdf(int p, int shape, const StageParams<float>& sp, cudaStream_t s);
cudaError_t tile_fp32pir(int p, int shape, const StageParams<float>& sp, cudaStream_t s);

template <int P, class PR, int TX, int TY>
cudaError_t launch_tile_shape(const StageParams<float>& sp, cudaStream_t s) {
  auto kern = tile_stage_kernel<P, PR, TX, TY>;
  constexpr int NT = TileShape<TX, TY>::NT;
  const size_t smem = sizeof(float) * tile_smem_floats<P, TX, TY>();
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int dev = 0, sms = 0, per_sm = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
  if (e != cudaSuccess) return e;
  const int tiles_x = (sp.m.nx + TX - 1) / TX, tiles_y = (sp.m.ny + TY - 1) / TY;
  const long long n_tiles = (long long)tiles_x * tiles_y;
  if (n_tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  long long grid = (long long)sms * (per_sm > 0 ? per_sm : 1);
  if (grid > n_tiles) grid = n_tiles;
  kern<<<(unsigned)grid, NT, smem, s>>>(sp, tiles_x, (int)n_tiles);
  return cudaGetLastError();
}

template <int P, class PR>
cudaError_t launch_tile_p(int shape, const StageParams<float>& sp, cudaStream_t s) {
  if (shape == 1) return launch_tile_shape<P, PR, 16, 8>(sp, s);
  if (shape == 2) return launch_tile_shape<P, PR, 8, 4>(sp, s);
  return launch_tile_shape<P, PR, 8, 8>(sp, s);
}

}  // namespace dgswe
