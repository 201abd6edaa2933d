// dg_project.cu -- set-up L2 projection of sampled data onto the DG basis
// (not part of the time loop).  With the orthonormal reference basis of §2.2
// the element mass matrix is |det B| I, so the coefficients of f are
//   c_i = int_T^ (f o F_e) phi^_i,
// evaluated with a collapsed Gauss-Legendre rule of n = p + 3 points per
// direction (exact for f of degree p + 4).
#include <cuda_runtime.h>

#include <cmath>
#include <exception>
#include <vector>

#include "dg_kernels.cuh"
#include "dgswe.h"

namespace {

using dgswe::BasisMonomials;
using dgswe::sfor;

constexpr int QMAX = 64;

struct Rule {
  int Q;
  double xr[QMAX], yr[QMAX], w[QMAX];
};

// Gauss-Legendre nodes/weights on [0, 1]: Newton's method on the Legendre
// polynomial P_n, evaluated by its three-term recurrence.
void gauss01(int n, double* s, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
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

Rule make_rule(int p) {
  Rule r;
  const int n = p + 3;
  double s[16], w[16];
  gauss01(n, s, w);
  r.Q = n * n;
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      const int q = a * n + b;
      r.xr[q] = s[a];
      r.yr[q] = (1.0 - s[a]) * s[b];
      r.w[q] = w[a] * w[b] * (1.0 - s[a]);
    }
  return r;
}

struct Geo {
  int nx;
  long long E;
  double x0, y0, hx, hy;
};

// vertex a1 and the (diagonal) map B of element e of the uniform mesh
__device__ __forceinline__ void elem_map(const Geo& g, long long e, double& ax, double& ay, double& b11,
                                         double& b22) {
  const int t = (int)(e & 1);
  const long long q = e >> 1;
  const int i = (int)(q % g.nx), j = (int)(q / g.nx);
  if (t == 0) {
    ax = g.x0 + i * g.hx;
    ay = g.y0 + j * g.hy;
    b11 = g.hx;
    b22 = g.hy;
  } else {
    ax = g.x0 + (i + 1) * g.hx;
    ay = g.y0 + (j + 1) * g.hy;
    b11 = -g.hx;
    b22 = -g.hy;
  }
}

__global__ void nodes_kernel(Geo g, Rule r, double* __restrict__ xy) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.E) return;
  double ax, ay, b11, b22;
  elem_map(g, e, ax, ay, b11, b22);
  for (int q = 0; q < r.Q; ++q) {
    xy[(long long)q * g.E + e] = ax + b11 * r.xr[q];
    xy[((long long)r.Q + q) * g.E + e] = ay + b22 * r.yr[q];
  }
}

// nodes of a general mesh from per-element maps [6][E]: a1x, a1y, B11, B12, B21, B22
__global__ void nodes_kernel_map(long long E, Rule r, const double* __restrict__ map, double* __restrict__ xy) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const double ax = map[e], ay = map[E + e], b11 = map[2 * E + e], b12 = map[3 * E + e], b21 = map[4 * E + e],
               b22 = map[5 * E + e];
  for (int q = 0; q < r.Q; ++q) {
    xy[(long long)q * E + e] = ax + b11 * r.xr[q] + b12 * r.yr[q];
    xy[((long long)r.Q + q) * E + e] = ay + b21 * r.xr[q] + b22 * r.yr[q];
  }
}

template <int K>
__global__ void project_kernel(long long E, Rule r, const double* __restrict__ vals, double* __restrict__ coef) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  double c[K];
  sfor<0, K>([&](auto i) { c[decltype(i)::value] = 0.0; });
  for (int q = 0; q < r.Q; ++q) {
    const double f = r.w[q] * vals[(long long)q * E + e];
    double xp[5], yp[5];
    xp[0] = yp[0] = 1.0;
    for (int k = 1; k < 5; ++k) {
      xp[k] = xp[k - 1] * r.xr[q];
      yp[k] = yp[k - 1] * r.yr[q];
    }
    sfor<0, K>([&](auto i) {
      double phi = 0.0;
      sfor<0, 5>([&](auto a) {
        sfor<0, 5 - decltype(a)::value>([&](auto b) {
          constexpr double m = BasisMonomials::c[decltype(i)::value][decltype(a)::value][decltype(b)::value];
          if constexpr (m != 0.0) phi = fma(m, xp[decltype(a)::value] * yp[decltype(b)::value], phi);
        });
      });
      c[decltype(i)::value] = fma(f, phi, c[decltype(i)::value]);
    });
  }
  sfor<0, K>([&](auto i) { coef[(long long)decltype(i)::value * E + e] = c[decltype(i)::value]; });
}

bool geo_of(const dg_config* c, Geo* g) {
  if (!c || c->nx < 1 || c->ny < 1 || c->p < 0 || c->p > 4 || !(c->Lx > 0) || !(c->Ly > 0)) return false;
  g->nx = c->nx;
  g->E = 2LL * c->nx * c->ny;
  g->x0 = c->x0;
  g->y0 = c->y0;
  g->hx = c->Lx / c->nx;
  g->hy = c->Ly / c->ny;
  return true;
}

}  // namespace

extern "C" {

int dg_proj_num_nodes(int p) { return (p < 0 || p > 4) ? 0 : (p + 3) * (p + 3); }

dg_status dg_proj_nodes(const dg_config* cfg, void* d_xy, void* stream) {
  Geo g;
  if (!geo_of(cfg, &g) || !d_xy) return DG_ERR_ARG;
  const Rule r = make_rule(cfg->p);
  if (!cfg->vertex_xy) {
    nodes_kernel<<<(unsigned)((g.E + 127) / 128), 128, 0, (cudaStream_t)stream>>>(g, r, (double*)d_xy);
    return cudaGetLastError() == cudaSuccess ? DG_OK : DG_ERR_CUDA;
  }
  // general mesh: element maps from the vertices (set-up only)
  const int nx = cfg->nx, ny = cfg->ny;
  const long long E = g.E;
  std::vector<double> map;
  try {
    map.resize((size_t)6 * E);
  } catch (const std::exception&) {   // no C++ exception crosses the C ABI
    return DG_ERR_OOM;
  }
  const double* v = cfg->vertex_xy;
  auto vx = [&](int i, int j) { return v[2 * ((size_t)j * (nx + 1) + i)]; };
  auto vy = [&](int i, int j) { return v[2 * ((size_t)j * (nx + 1) + i) + 1]; };
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i)
      for (int t = 0; t < 2; ++t) {
        const long long e = 2LL * ((long long)j * nx + i) + t;
        const int i1 = t ? i + 1 : i, j1 = t ? j + 1 : j;
        const int i2 = t ? i : i + 1, j2 = t ? j + 1 : j;
        const int i3 = t ? i + 1 : i, j3 = t ? j : j + 1;
        map[e] = vx(i1, j1);
        map[E + e] = vy(i1, j1);
        map[2 * E + e] = vx(i2, j2) - vx(i1, j1);
        map[3 * E + e] = vx(i3, j3) - vx(i1, j1);
        map[4 * E + e] = vy(i2, j2) - vy(i1, j1);
        map[5 * E + e] = vy(i3, j3) - vy(i1, j1);
      }
  double* d = nullptr;
  if (cudaMalloc(&d, sizeof(double) * map.size()) != cudaSuccess) {
    (void)cudaGetLastError();   // clear the failed allocation from the last-error slot
    return DG_ERR_OOM;
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(d, map.data(), sizeof(double) * map.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    nodes_kernel_map<<<(unsigned)((E + 127) / 128), 128, 0, s>>>(E, r, d, (double*)d_xy);
    e = cudaGetLastError();
  }
  cudaError_t e2 = cudaStreamSynchronize(s);
  cudaFree(d);
  return (e == cudaSuccess && e2 == cudaSuccess) ? DG_OK : DG_ERR_CUDA;
}

dg_status dg_project(const dg_config* cfg, const void* d_vals, void* d_coef, void* stream) {
  Geo g;
  if (!geo_of(cfg, &g) || !d_vals || !d_coef) return DG_ERR_ARG;
  const Rule r = make_rule(cfg->p);
  const unsigned grid = (unsigned)((g.E + 127) / 128);
  cudaStream_t s = (cudaStream_t)stream;
  const double* v = (const double*)d_vals;
  double* c = (double*)d_coef;
  switch (cfg->p) {
    case 0: project_kernel<1><<<grid, 128, 0, s>>>(g.E, r, v, c); break;
    case 1: project_kernel<3><<<grid, 128, 0, s>>>(g.E, r, v, c); break;
    case 2: project_kernel<6><<<grid, 128, 0, s>>>(g.E, r, v, c); break;
    case 3: project_kernel<10><<<grid, 128, 0, s>>>(g.E, r, v, c); break;
    default: project_kernel<15><<<grid, 128, 0, s>>>(g.E, r, v, c); break;
  }
  return cudaGetLastError() == cudaSuccess ? DG_OK : DG_ERR_CUDA;
}

}  // extern "C"
