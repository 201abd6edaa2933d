// dg_kernels.cuh -- sm_103a kernels of the quadrature-free DG shallow water
// scheme (arXiv:1904.08684, §2.2).
//
// One thread owns one triangle.  All reference integrals are compile-time
// constants (dg_ref_tables.h, exact): the loops over basis functions below are
// unrolled at compile time and every zero tensor entry is dropped, so the
// arithmetic is exactly the nonzero pattern of the tensors.
//
// Data flow of one Runge-Kutta stage (one launch of stage_kernel):
//   in : state w, RK base state w0, "vs" = volume + source integrals of w,
//        per element and local edge a "side record" of w (flux, traces, wave
//        speed) -- written by the previous launch;
//   1. numerical flux on the 3 edges from the own and the neighbour's side
//      record, lifted to the element (edge integrals of Eq. (11));
//   2. R = (vs - edge) / |det B|  (diagonal mass matrix) and the SSP stage
//      w' = a w0 + b (w + dt R);
//   3. for w': velocity projection u = q/H (Eq. (12)), volume + source
//      integrals (Eqs. (15)-(16) and r of Eq. (5)) -> vs', side records ->
//      rec', element wave speed -> CFL maximum.
//   The launch boundary is the only global synchronisation: side records of
//   w' are read by neighbours in the next launch (double-buffered).
#pragma once

#include <cstdint>
#include <type_traits>

#include "dg_ref_tables.h"

namespace dgswe {

template <int B, int E, class F>
__device__ __forceinline__ void sfor(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    sfor<B + 1, E>(f);
  }
}
#define CV(x) decltype(x)::value

template <int P>
struct Dims {
  static constexpr int K = (P + 1) * (P + 2) / 2;  // basis functions
  static constexpr int P1 = P + 1;                 // Legendre modes on an edge
  static constexpr int K1 = P * (P + 1) / 2;       // basis of P^{p-1}
  static constexpr int NREC = 6 * P1 + 1;          // side record length
  // the bathymetry lives in P^max(p,1) (at p = 0 a piecewise-constant h_b
  // would lose the source g xi grad h_b): its order, basis size, edge modes
  // and the basis size of its gradient's space
  static constexpr int PB = P > 0 ? P : 1;
  static constexpr int KB = (PB + 1) * (PB + 2) / 2;
  static constexpr int PB1 = PB + 1;
  static constexpr int KB1 = PB * (PB + 1) / 2;
};

// error word bits
enum : unsigned { ERRF_DRY = 1u, ERRF_NONFINITE = 2u };

// ---------------------------------------------------------------------------
// Uniform quad-split mesh (§2.3).  Element e = 2 (j nx + i) + t.
struct Mesh {
  int nx, ny;
  long long E;
  double x0, y0;   // domain origin
  double hx, hy;   // quad sizes
  double diag;     // sqrt(hx^2 + hy^2)
  double ndx, ndy; // hy / diag, hx / diag: unit normal of the lower diagonal
  int periodic;    // 1 periodic, 0 walls
  // the same sizes rounded to FP32 once on the host: the FP32 kernels read
  // them instead of converting the doubles per use (a double -> float
  // conversion runs on GB300's FP64 pipe, 1/64 of the FP32 rate)
  float fhx, fhy, fdiag, fndx, fndy;
  // per-element geometry of a general (e.g. randomly perturbed) quad-split
  // mesh, [NGEO][E] FP64; null for the uniform mesh (computed from e)
  const double* geo;
};

// per-element geometry record (general meshes): adj(B)^T = G, |det B|,
// 1/|det B|, (n_x, n_y, |E|) of the three local edges, vertex a1
enum { GEO_G11 = 0, GEO_G12, GEO_G21, GEO_G22, GEO_DET, GEO_IDET, GEO_EDGE, GEO_A1X = GEO_EDGE + 9, GEO_A1Y,
       NGEO };

// neighbour across local edge n (same local index on the other side); -1 = wall
__device__ __forceinline__ long long neighbour(const Mesh& m, long long e, int n) {
  const int t = (int)(e & 1);
  const long long q = e >> 1;
  const int i = (int)(q % m.nx), j = (int)(q / m.nx);
  if (n == 0) return e ^ 1;
  int ii = i, jj = j;
  if (n == 1) ii += t ? 1 : -1;
  else jj += t ? 1 : -1;
  if (ii < 0 || ii >= m.nx || jj < 0 || jj >= m.ny) {
    if (!m.periodic) return -1;
    ii = (ii + m.nx) % m.nx;
    jj = (jj + m.ny) % m.ny;
  }
  return 2 * ((long long)jj * m.nx + ii) + (1 - t);
}

// a mesh size in the kernel's precision: the double, or its float copy
template <class Real>
__device__ __forceinline__ Real mesh_val(double d, float f) {
  if constexpr (std::is_same<Real, float>::value) return f;
  else return Real(d);
}

// Outward unit normal and length of local edge n.  Lower triangle: edge 0 is
// the diagonal (normal (hy, hx)/diag), edge 1 the left side (-1, 0), edge 2
// the bottom (0, -1); the upper triangle has the opposite normals.
template <int FEAT, class Real>
__device__ __forceinline__ void edge_geom(const Mesh& m, long long e, int t, int n, Real& nx, Real& ny, Real& len) {
  if (FEAT && m.geo) {
    nx = Real(m.geo[(GEO_EDGE + 3 * n) * m.E + e]);
    ny = Real(m.geo[(GEO_EDGE + 3 * n + 1) * m.E + e]);
    len = Real(m.geo[(GEO_EDGE + 3 * n + 2) * m.E + e]);
    return;
  }
  const Real s = t ? Real(-1) : Real(1);
  if (n == 0) {
    nx = s * mesh_val<Real>(m.ndx, m.fndx);
    ny = s * mesh_val<Real>(m.ndy, m.fndy);
    len = mesh_val<Real>(m.diag, m.fdiag);
  } else if (n == 1) {
    nx = -s;
    ny = Real(0);
    len = mesh_val<Real>(m.hy, m.fhy);
  } else {
    nx = Real(0);
    ny = -s;
    len = mesh_val<Real>(m.hx, m.fhx);
  }
}

// adj(B)^T of element e: diagonal (hy, hx) for the lower, -(hy, hx) for the
// upper triangle of the uniform mesh; read from the geometry record otherwise
template <int FEAT, class Real>
__device__ __forceinline__ void elem_G(const Mesh& m, long long e, int t, Real& G11, Real& G12, Real& G21,
                                       Real& G22) {
  if (FEAT && m.geo) {
    G11 = Real(m.geo[GEO_G11 * m.E + e]);
    G12 = Real(m.geo[GEO_G12 * m.E + e]);
    G21 = Real(m.geo[GEO_G21 * m.E + e]);
    G22 = Real(m.geo[GEO_G22 * m.E + e]);
    return;
  }
  const Real sgn = t ? Real(-1) : Real(1);
  G11 = sgn * mesh_val<Real>(m.hy, m.fhy);
  G22 = sgn * mesh_val<Real>(m.hx, m.fhx);
  G12 = Real(0);
  G21 = Real(0);
}

template <int FEAT>
__device__ __forceinline__ double elem_inv_det(const Mesh& m, long long e, double uniform) {
  return (FEAT && m.geo) ? m.geo[GEO_IDET * m.E + e] : uniform;
}

// affine map x = a1 + B x^ of element e (FP64)
__device__ __forceinline__ void elem_map(const Mesh& m, long long e, double& ax, double& ay, double& B11,
                                         double& B12, double& B21, double& B22) {
  if (m.geo) {
    ax = m.geo[GEO_A1X * m.E + e];
    ay = m.geo[GEO_A1Y * m.E + e];
    // G = adj(B)^T = [[B22, -B21], [-B12, B11]]
    B11 = m.geo[GEO_G22 * m.E + e];
    B22 = m.geo[GEO_G11 * m.E + e];
    B21 = -m.geo[GEO_G12 * m.E + e];
    B12 = -m.geo[GEO_G21 * m.E + e];
    return;
  }
  const int t = (int)(e & 1);
  const long long q = e >> 1;
  const int i = (int)(q % m.nx), j = (int)(q / m.nx);
  B12 = 0.0;
  B21 = 0.0;
  if (t == 0) {
    ax = m.x0 + i * m.hx;
    ay = m.y0 + j * m.hy;
    B11 = m.hx;
    B22 = m.hy;
  } else {
    ax = m.x0 + (i + 1) * m.hx;
    ay = m.y0 + (j + 1) * m.hy;
    B11 = -m.hx;
    B22 = -m.hy;
  }
}

// §3.1 analytic solution (C_a = C_t = 0.2, y_a = 0.3) and the body force F
// that makes it satisfy Eq. (2) with tau_bf = f_c = 0 on the bathymetry
// h_b = 1 + x/1000 + 2 y/1000.
__device__ __forceinline__ void ms_state(double x, double y, double t, double& xi, double& U, double& V) {
  const double S = sin(3.141592653589793 * (x + y + 0.2 * t) / 600.0);
  xi = 2.3 - 0.4 * S;
  U = 0.6 + 0.04 * S;
  V = 0.3 + 0.04 * S;
}

__device__ __forceinline__ void ms_force(double x, double y, double t, double g, double& Fx, double& Fy) {
  const double k = 3.141592653589793 / 600.0;
  const double th = k * (x + y + 0.2 * t);
  double S, C;
  sincos(th, &S, &C);
  const double xi = 2.3 - 0.4 * S, U = 0.6 + 0.04 * S, V = 0.3 + 0.04 * S;
  const double H = xi + 1.0 + x / 1000.0 + 2.0 * y / 1000.0;
  const double xix = -0.4 * k * C;                  // = d xi / dy
  const double qx = 0.04 * k * C, qt = 0.04 * 0.2 * k * C;   // dU/dx = dU/dy = dV/dx = dV/dy; dU/dt = dV/dt
  const double Hx = xix + 1.0e-3, Hy = xix + 2.0e-3;
  // F = d_t q + div(q q^T / H) + g H grad xi
  const double dUU_dx = 2.0 * U * qx / H - U * U * Hx / (H * H);
  const double dUV_dy = (qx * V + U * qx) / H - U * V * Hy / (H * H);
  const double dUV_dx = (qx * V + U * qx) / H - U * V * Hx / (H * H);
  const double dVV_dy = 2.0 * V * qx / H - V * V * Hy / (H * H);
  Fx = qt + dUU_dx + dUV_dy + g * H * xix;
  Fy = qt + dUV_dx + dVV_dy + g * H * xix;
}

// ---------------------------------------------------------------------------
// Reference-tensor contractions (compile-time unrolled, zeros skipped).

// out[n] = sum_{i, m < MLIM} T[n][i][m] a[i] b[m] for n < NOUT: the L2
// projection of the product a*b onto the first NOUT basis functions (b known
// to vanish beyond MLIM).
template <int P, int NOUT, int MLIM, class R>
__device__ __forceinline__ void tprod(const R* a, const R* b, R* out) {
  using Tb = RefTables<P>;
  constexpr int K = Tb::K;
  sfor<0, NOUT>([&](auto n) {
    R acc = R(0);
    sfor<0, K>([&](auto i) {
      R inner = R(0);
      bool any = false;
      sfor<0, MLIM>([&](auto m) {
        constexpr double t = Tb::T[CV(n)][CV(i)][CV(m)];
        if constexpr (t != 0.0) {
          inner = fma(R(t), b[CV(m)], inner);
          any = true;
        }
      });
      if (any) acc = fma(a[CV(i)], inner, acc);
    });
    out[CV(n)] = acc;
  });
}

// The four projected momentum products Pi(U u), Pi(U v), Pi(V u), Pi(V v)
// onto P^{p-1}, sharing the rows (T_n u)_i = sum_m T[n][i][m] u_m and
// (T_n v)_i between the U and V contractions.
template <int P, class R>
__device__ __forceinline__ void momentum_products(const R* U, const R* V, const R* u, const R* v, R* Puu, R* Puv,
                                                  R* Pvu, R* Pvv) {
  using Tb = RefTables<P>;
  constexpr int K = Tb::K, K1 = Dims<P>::K1;
  sfor<0, K1>([&](auto n) {
    R auu = R(0), auv = R(0), avu = R(0), avv = R(0);
    sfor<0, K>([&](auto i) {
      R ru = R(0), rv = R(0);
      bool any = false;
      sfor<0, K>([&](auto m) {
        constexpr double t = Tb::T[CV(n)][CV(i)][CV(m)];
        if constexpr (t != 0.0) {
          ru = fma(R(t), u[CV(m)], ru);
          rv = fma(R(t), v[CV(m)], rv);
          any = true;
        }
      });
      if (any) {
        auu = fma(U[CV(i)], ru, auu);
        avu = fma(V[CV(i)], ru, avu);
        auv = fma(U[CV(i)], rv, auv);
        avv = fma(V[CV(i)], rv, avv);
      }
    });
    Puu[CV(n)] = auu;
    Puv[CV(n)] = auv;
    Pvu[CV(n)] = avu;
    Pvv[CV(n)] = avv;
  });
}

// out[n] = sum_{i,m} T[n][i][m] a_i a_m for n < NOUT, using the symmetry of
// T in (i, m): sum_i a_i (T[n][i][i] a_i + 2 sum_{m>i} T[n][i][m] a_m)
template <int P, int NOUT, class R>
__device__ __forceinline__ void tprod_sym(const R* a, R* out) {
  using Tb = RefTables<P>;
  constexpr int K = Tb::K;
  sfor<0, NOUT>([&](auto n) {
    R acc = R(0);
    sfor<0, K>([&](auto i) {
      R inner = R(0);
      bool any = false;
      sfor<CV(i), K>([&](auto m) {
        constexpr double t = Tb::T[CV(n)][CV(i)][CV(m)] * (CV(m) == CV(i) ? 1.0 : 2.0);
        if constexpr (t != 0.0) {
          inner = fma(R(t), a[CV(m)], inner);
          any = true;
        }
      });
      if (any) acc = fma(a[CV(i)], inner, acc);
    });
    out[CV(n)] = acc;
  });
}

// the two edge momentum products Pi(x u_n), Pi(y u_n) sharing the inner sums
// sum_b Lam[j][a][b] u_n,b
template <int P, class R>
__device__ __forceinline__ void lprod2(const R* x, const R* y, const R* un, R* ox, R* oy) {
  using Tb = RefTables<P>;
  constexpr int P1 = Tb::P1;
  sfor<0, P1>([&](auto j) {
    R ax = R(0), ay = R(0);
    sfor<0, P1>([&](auto a) {
      R inner = R(0);
      bool any = false;
      sfor<0, P1>([&](auto b) {
        constexpr double c = Tb::Lam[CV(j)][CV(a)][CV(b)];
        if constexpr (c != 0.0) {
          inner = fma(R(c), un[CV(b)], inner);
          any = true;
        }
      });
      if (any) {
        ax = fma(x[CV(a)], inner, ax);
        ay = fma(y[CV(a)], inner, ay);
      }
    });
    ox[CV(j)] = ax;
    oy[CV(j)] = ay;
  });
}

// sum_i S[r][a][i] f[i]  (S vanishes for i beyond P^{p-1})
template <int P, int r, int a, class R>
__device__ __forceinline__ R sdot_row(const R* f) {
  using Tb = RefTables<P>;
  R acc = R(0);
  sfor<0, Dims<P>::K1>([&](auto i) {
    constexpr double s = Tb::S[r][a][CV(i)];
    if constexpr (s != 0.0) acc = fma(R(s), f[CV(i)], acc);
  });
  return acc;
}

// trace on local edge NN: tau[j] = sum_i R[NN][j][i] w[i]
template <int NN, int P, class R>
__device__ __forceinline__ void trace(const R* w, R* tau) {
  using Tb = RefTables<P>;
  constexpr int K = Tb::K, P1 = Tb::P1;
  sfor<0, P1>([&](auto j) {
    R acc = R(0);
    sfor<0, K>([&](auto i) {
      constexpr double c = Tb::R[NN][CV(j)][CV(i)];
      if constexpr (c != 0.0) acc = fma(R(c), w[CV(i)], acc);
    });
    tau[CV(j)] = acc;
  });
}

// lift on local edge n: out[a] += sum_j R[n][j][a] F[j]
template <int NN, int P, class R>
__device__ __forceinline__ void lift_sub(const R* F, R* out) {
  using Tb = RefTables<P>;
  constexpr int K = Tb::K, P1 = Tb::P1;
  sfor<0, K>([&](auto a) {
    R acc = out[CV(a)];
    sfor<0, P1>([&](auto j) {
      constexpr double c = Tb::R[NN][CV(j)][CV(a)];
      if constexpr (c != 0.0) acc = fma(R(-c), F[CV(j)], acc);
    });
    out[CV(a)] = acc;
  });
}

// 1D product projection: out[j] = sum_{a,b} Lam[j][a][b] x[a] y[b]
template <int P, class R>
__device__ __forceinline__ void lprod(const R* x, const R* y, R* out) {
  using Tb = RefTables<P>;
  constexpr int P1 = Tb::P1;
  sfor<0, P1>([&](auto j) {
    R acc = R(0);
    sfor<0, P1>([&](auto a) {
      R inner = R(0);
      bool any = false;
      sfor<0, P1>([&](auto b) {
        constexpr double c = Tb::Lam[CV(j)][CV(a)][CV(b)];
        if constexpr (c != 0.0) {
          inner = fma(R(c), y[CV(b)], inner);
          any = true;
        }
      });
      if (any) acc = fma(x[CV(a)], inner, acc);
    });
    out[CV(j)] = acc;
  });
}

// value of an edge polynomial at s = 0, 1/2, 1 (k = 0, 1, 2)
template <int P, int k, class R>
__device__ __forceinline__ R edge_point(const R* tau) {
  using Tb = RefTables<P>;
  R acc = R(0);
  sfor<0, Tb::P1>([&](auto j) {
    constexpr double c = Tb::Lpt[k][CV(j)];
    if constexpr (c != 0.0) acc = fma(R(c), tau[CV(j)], acc);
  });
  return acc;
}

// ---------------------------------------------------------------------------
// Double-float arithmetic ("df64") on the FP32 pipe: a value is hi + lo with
// |lo| <= ulp(hi)/2 (about 48 significant bits).  Built from the error-free
// transformations of Knuth (two-sum) and Dekker (two-product, here with a
// fused multiply-add), with the accurate double-double addition of
// Hida, Li and Bailey.  Explicit _rn intrinsics keep the compiler from
// contracting or reassociating the steps.
struct df64 {
  float hi, lo;
  __host__ __device__ constexpr df64() : hi(0.f), lo(0.f) {}
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr explicit df64(int a) : hi(float(a)), lo(0.f) {}
  __host__ __device__ constexpr explicit df64(float a) : hi(a), lo(0.f) {}
  // split of a double (used on compile-time constants only)
  __host__ __device__ constexpr explicit df64(double a) : hi(float(a)), lo(float(a - double(float(a)))) {}
  __device__ explicit operator float() const { return __fadd_rn(hi, lo); }
  __device__ explicit operator double() const { return double(hi) + double(lo); }
};

__device__ __forceinline__ df64 df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return df64(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
__device__ __forceinline__ df64 df_quick_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df64(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  df64 s = df_two_sum(a.hi, b.hi);
  const df64 t = df_two_sum(a.lo, b.lo);
  s = df_quick_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return df_quick_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}
__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_quick_two_sum(p, e);
}
__device__ __forceinline__ df64 operator/(df64 a, df64 b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const df64 r = a - b * df64(q1);
  return df_quick_two_sum(q1, __fdiv_rn(r.hi, b.hi));
}
__device__ __forceinline__ bool operator>(df64 a, df64 b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
// a * b + c in the arithmetic of the velocity solve (float, double, df64)
__device__ __forceinline__ double mad(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float mad(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ df64 mad(df64 a, df64 b, df64 c) { return a * b + c; }

// ---------------------------------------------------------------------------
// Sums of products in the arithmetic of the velocity solve.  For double and
// float: a fused multiply-add chain.  For df64: a compensated dot product
// (Ogita, Rump and Oishi, "Accurate sum and dot product", SIAM J. Sci.
// Comput. 26 (2005), algorithm Dot2, extended to double-float operands):
// each product is split exactly into its rounded value and its error with a
// fused multiply-add, the running sum stays in one float whose rounding
// errors are gathered by two-sum into a second float, and the two are joined
// once at the end.  The result is as accurate as a double-float evaluation,
// but a term costs 11-12 FP32 operations instead of ~27, and the dependent
// chain through the terms is one addition long.
template <class PR>
struct SolveAcc {
  PR s;
  __device__ __forceinline__ explicit SolveAcc(PR x) : s(x) {}
  __device__ __forceinline__ void add(PR a, PR b) { s = mad(a, b, s); }   // s += a b
  template <class H>
  __device__ __forceinline__ void add_c(double t, H h) { s = mad(PR(t), PR(h), s); }   // s += t h, t constant
  __device__ __forceinline__ PR get() const { return s; }
};

template <>
struct SolveAcc<df64> {
  float s, c;   // running sum and the sum of its rounding errors
  __device__ __forceinline__ explicit SolveAcc(df64 x) : s(x.hi), c(x.lo) {}
  // add p + e, where p + e is an exact product and |e| <= ulp(p)
  __device__ __forceinline__ void add_exact(float p, float e) {
    const float t = __fadd_rn(s, p);
    const float z = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
    s = t;
    c = __fadd_rn(c, __fadd_rn(err, e));
  }
  __device__ __forceinline__ void add(df64 a, df64 b) {
    const float p = __fmul_rn(a.hi, b.hi);
    const float e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, __fmaf_rn(a.hi, b.hi, -p)));
    add_exact(p, e);
  }
  // s += t h with t a compile-time constant and h a float
  __device__ __forceinline__ void add_c(double t, float h) {
    const df64 tt(t);   // split at compile time once inlined
    const float p = __fmul_rn(tt.hi, h);
    add_exact(p, __fmaf_rn(tt.lo, h, __fmaf_rn(tt.hi, h, -p)));
  }
  __device__ __forceinline__ df64 get() const { return df_two_sum(s, c); }
};

// ---------------------------------------------------------------------------
// Velocity projection (Eq. (12)): A u = U, A v = V with
// A_ab = sum_n T[n][a][b] H_n (SPD iff H > 0 on the element).

// LDL^T factorisation of A in precision PR (left-looking: column j uses
// W_k = L_jk D_k, k < j).  Hd: the depth coefficients (HT = PR, or float for
// the double-float solve, whose depth enters as the exact float it is).
// Returns false if a pivot is not positive (dry element).
template <int P, class PR, class HT>
__device__ __forceinline__ bool ldlt_factor(const HT* Hd, PR (&L)[RefTables<P>::K][RefTables<P>::K],
                                            PR* Dg, PR* rD) {
  using Tb = RefTables<P>;
  constexpr int K = Tb::K;
  bool ok = true;
  sfor<0, K>([&](auto jj) {
    constexpr int j = CV(jj);
    PR W[K > 1 ? K : 1];
    SolveAcc<PR> d(PR(0));
    sfor<0, K>([&](auto n) {
      constexpr double t = Tb::T[CV(n)][j][j];
      if constexpr (t != 0.0) d.add_c(t, Hd[CV(n)]);
    });
    sfor<0, j>([&](auto k) {
      W[CV(k)] = L[j][CV(k)] * Dg[CV(k)];
      d.add(-L[j][CV(k)], W[CV(k)]);
    });
    const PR dj = d.get();
    ok = ok && (dj > PR(0));
    Dg[j] = dj;
    rD[j] = PR(1) / dj;
    sfor<j + 1, K>([&](auto ii) {
      constexpr int i = CV(ii);
      SolveAcc<PR> a(PR(0));
      sfor<0, K>([&](auto n) {
        constexpr double t = Tb::T[CV(n)][i][j];
        if constexpr (t != 0.0) a.add_c(t, Hd[CV(n)]);
      });
      sfor<0, j>([&](auto k) { a.add(-L[i][CV(k)], W[CV(k)]); });
      L[i][j] = a.get() * rD[j];
    });
  });
  return ok;
}

// L y = b, y <- y / D, L^T x = y
template <int P, class PR, class B, class X>
__device__ __forceinline__ void ldlt_solve(const PR (&L)[RefTables<P>::K][RefTables<P>::K], const PR* rD,
                                           const B* b, X* x) {
  constexpr int K = RefTables<P>::K;
  PR y[K];
  sfor<0, K>([&](auto ii) {
    constexpr int i = CV(ii);
    SolveAcc<PR> s{PR(b[i])};
    sfor<0, i>([&](auto k) { s.add(-L[i][CV(k)], y[CV(k)]); });
    y[i] = s.get();
  });
  sfor<0, K>([&](auto rr) {
    constexpr int i = K - 1 - CV(rr);
    SolveAcc<PR> s(y[i] * rD[i]);
    sfor<i + 1, K>([&](auto k) { s.add(-L[CV(k)][i], y[CV(k)]); });
    y[i] = s.get();
    x[i] = X(y[i]);
  });
}

// Marker type of the mixed-precision solve (FP32 state only): LDL^T and both
// triangular solves in FP32, then one step of iterative refinement,
// x = x0 + A^{-1} r with the FP32 factors (Wilkinson's mixed-precision
// refinement).  The residual r = b - A x0 must be accurate to about
// eps32^2 |A| |x0| (it cancels to ~kappa eps32 |b|); A = A_hb + A_xi splits
//   A_hb = sum_n T[n][a][b] h_b,n  static: its FP64 value is kept as the
//          unevaluated sum hi + lo, hi the FP32 sum of the FP32 bathymetry
//          coefficients formed by one fixed sequence of rounded operations
//          (ahb_hi: recomputed in the solve; stored at p = 4, see
//          ahb_keeps_hi), lo = fl(A_hb - hi) stored once per context
//          (ahb_kernel), ~48 significant bits for 4 bytes per entry;
//   A_xi = sum_n T[n][a][b] xi_n   formed in FP32, whose rounding error,
//          eps32 |A_xi| |x0| <= eps32 (|xi| / H) |b|, stays below the FP32
//          rounding of the result.
// Each row of the residual is a compensated dot product on the FP32 units
// (the Dot2 scheme of Ogita, Rump and Oishi, SIAM J. Sci. Comput. 26, 2005):
// the product hi x0_b is split exactly into its rounded value and its error
// with a fused multiply-add, the rounded values are summed with Knuth's
// two-sum, and every error term -- the product and sum errors and the small
// products (lo + A_xi) x0_b -- goes to a second float, added once at the
// end.  With kappa(A) K 2^-24 << 1 the refined result is the FP64 solution
// to within FP32 rounding (an FP64 residual gives the same accuracy at ~8x
// the pipe time on GB300, whose FP64 rate is 1/64 of its FP32 rate);
// elements whose FP32 pivots fail or spread by more than 2^10 (kappa
// estimate) take the FP64 solve.
struct MixedIR {};

template <int P, class PR, class R>
__device__ __forceinline__ bool project_velocity(const R* H, const R* U, const R* V, R* u, R* v);

// number of entries of the lower triangle of a K x K matrix
__host__ __device__ constexpr int tri_size(int K) { return K * (K + 1) / 2; }

// The mixed solve's A_hb = hi + lo per entry: lo is stored; hi is recomputed
// from h_b for p <= 3 (at p = 3, 226 FMAs per triangle against 55 loads) and
// stored too at p = 4 (K = 15), where the recompute takes 636 FMAs against
// 120 loads and measured slower than the loads.  FP32 words per triangle:
__host__ __device__ constexpr bool ahb_keeps_hi(int K) { return K >= 15; }
__host__ __device__ constexpr int ahb_words(int K) { return tri_size(K) * (ahb_keeps_hi(K) ? 2 : 1); }

// compensated running sum s + c of the refinement residual
struct ResidualAcc {
  float s, c;
  __device__ __forceinline__ ResidualAcc() : s(0.f), c(0.f) {}
  __device__ __forceinline__ explicit ResidualAcc(float b) : s(b), c(0.f) {}
  // s + c -= (hi + t) x, with hi x split exactly (t = lo + A_xi is small)
  __device__ __forceinline__ void sub(float hi, float t, float x) {
    const float p = __fmul_rn(hi, x);
    const float e = __fmaf_rn(hi, x, -p);
    const float sn = __fsub_rn(s, p);
    const float z = __fsub_rn(sn, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(sn, z)), __fsub_rn(-p, z));
    s = sn;
    c = __fmaf_rn(-t, x, __fadd_rn(c, __fsub_rn(err, e)));
  }
  __device__ __forceinline__ float get() const { return __fadd_rn(s, c); }
};

// hi of entry (a, b) of A_hb from the FP32 bathymetry coefficients hb[n],
// n < K: the same rounded operations in ahb_kernel and in the solve
template <int P, int a, int b>
__device__ __forceinline__ float ahb_hi(const float* hb) {
  using Tb = RefTables<P>;
  float hi = 0.f;
  sfor<0, Tb::K>([&](auto n) {
    constexpr double t = Tb::T[CV(n)][a][b];
    if constexpr (t != 0.0) hi = __fmaf_rn(float(t), hb[CV(n)], hi);
  });
  return hi;
}

template <int P, class R>
__device__ __forceinline__ bool project_velocity_ir(const R* H, const R* xi, const R* hb, const R* U, const R* V,
                                                    R* u, R* v, const float* __restrict__ ahb, long long E) {
  using Tb = RefTables<P>;
  constexpr int K = Tb::K;
  float L[K][K], Dg[K], rD[K];
  float Hf[K];
  sfor<0, K>([&](auto n) { Hf[CV(n)] = float(H[CV(n)]); });
  const bool ok = ldlt_factor<P, float>(Hf, L, Dg, rD);
  float dmin = Dg[0], dmax = Dg[0];
  sfor<1, K>([&](auto j) {
    dmin = fminf(dmin, Dg[CV(j)]);
    dmax = fmaxf(dmax, Dg[CV(j)]);
  });
  if (!ok || !(dmax <= 1024.f * dmin)) return project_velocity<P, double>(H, U, V, u, v);
  float u0[K], v0[K];
  ldlt_solve<P>(L, rD, U, u0);
  ldlt_solve<P>(L, rD, V, v0);
  ResidualAcc ru[K], rv[K];
  sfor<0, K>([&](auto n) {
    ru[CV(n)] = ResidualAcc(float(U[CV(n)]));
    rv[CV(n)] = ResidualAcc(float(V[CV(n)]));
  });
  sfor<0, K>([&](auto aa) {
    constexpr int a = CV(aa);
    sfor<0, a + 1>([&](auto bb) {
      constexpr int b = CV(bb);
      constexpr int ab = a * (a + 1) / 2 + b;
      const float lo = ahb[(long long)ab * E];
      float hi;
      if constexpr (ahb_keeps_hi(K)) hi = ahb[(long long)(tri_size(K) + ab) * E];
      else hi = ahb_hi<P, a, b>(hb);
      float Ax = 0.f;
      sfor<0, K>([&](auto n) {
        constexpr double t = Tb::T[CV(n)][a][b];
        if constexpr (t != 0.0) Ax = __fmaf_rn(float(t), float(xi[CV(n)]), Ax);
      });
      const float t = __fadd_rn(lo, Ax);
      ru[a].sub(hi, t, u0[b]);
      rv[a].sub(hi, t, v0[b]);
      if constexpr (a != b) {
        ru[b].sub(hi, t, u0[a]);
        rv[b].sub(hi, t, v0[a]);
      }
    });
  });
  float rf[K], du[K], dv[K];
  sfor<0, K>([&](auto i) { rf[CV(i)] = ru[CV(i)].get(); });
  ldlt_solve<P>(L, rD, rf, du);
  sfor<0, K>([&](auto i) { rf[CV(i)] = rv[CV(i)].get(); });
  ldlt_solve<P>(L, rD, rf, dv);
  // explicit rounding: the last solve step leaves u0 = y rD, and a
  // contracted y rD + du would depend on the compilation context
  sfor<0, K>([&](auto i) {
    u[CV(i)] = R(__fadd_rn(u0[CV(i)], du[CV(i)]));
    v[CV(i)] = R(__fadd_rn(v0[CV(i)], dv[CV(i)]));
  });
  return true;
}

// A_hb of the mixed solve: A = sum_n T[n][a][b] h_b,n in FP64, n over the KB
// bathymetry coefficients (P^max(p,1)), for b <= a; stored is
// lo = fl(A - hi) at [ab][E] (ab = a(a+1)/2 + b) with hi = ahb_hi of the
// FP32 coefficients (the rounding of h_b that the FP32 contexts hold), or,
// where ahb_keeps_hi, hi = fl(A) stored at [K(K+1)/2 + ab][E]
template <int P>
__global__ void ahb_kernel(long long E, const double* __restrict__ hb64, float* __restrict__ ahb) {
  using D = Dims<P>;
  using Tb = RefTables<D::PB>;
  constexpr int K = D::K, KB = D::KB;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  double h[KB];
  float hf[K];
  sfor<0, KB>([&](auto i) { h[CV(i)] = hb64[CV(i) * E + e]; });
  sfor<0, K>([&](auto i) { hf[CV(i)] = float(h[CV(i)]); });
  sfor<0, K>([&](auto aa) {
    constexpr int a = CV(aa);
    sfor<0, a + 1>([&](auto bb) {
      constexpr int b = CV(bb);
      double A = 0.0;
      sfor<0, KB>([&](auto n) {
        constexpr double t = Tb::T[CV(n)][a][b];
        if constexpr (t != 0.0) A = fma(t, h[CV(n)], A);
      });
      constexpr int ab = a * (a + 1) / 2 + b;
      if constexpr (ahb_keeps_hi(K)) {
        const float hi = __double2float_rn(A);
        ahb[(long long)ab * E + e] = __double2float_rn(A - double(hi));
        ahb[(long long)(tri_size(K) + ab) * E + e] = hi;
      } else {
        const float hi = ahb_hi<P, a, b>(hf);
        ahb[(long long)ab * E + e] = __double2float_rn(A - double(hi));
      }
    });
  });
}

// Solve in precision PR (double, float, df64), or MixedIR (see above).
template <int P, class PR, class R>
__device__ __forceinline__ bool project_velocity(const R* H, const R* U, const R* V, R* u, R* v) {
  if constexpr (std::is_same<PR, MixedIR>::value) {
    // callers without the static A_hb (diagnostics) take the FP64 solve
    return project_velocity<P, double>(H, U, V, u, v);
  } else {
    using Tb = RefTables<P>;
    constexpr int K = Tb::K;
    // the depth enters the double-float solve as the exact float it is
    using HT = typename std::conditional<std::is_same<PR, df64>::value, R, PR>::type;
    HT Hd[K];
    PR L[K][K], Dg[K], rD[K];
    sfor<0, K>([&](auto n) { Hd[CV(n)] = HT(H[CV(n)]); });
    const bool ok = ldlt_factor<P, PR>(Hd, L, Dg, rD);
    ldlt_solve<P>(L, rD, U, u);
    ldlt_solve<P>(L, rD, V, v);
    return ok;
  }
}

// phi^_i(x^, y^), i < K, from the exact monomial tables
template <int K>
__device__ __forceinline__ void basis_at(double xr, double yr, double* phi) {
  double xp[5], yp[5];
  xp[0] = yp[0] = 1.0;
  for (int k = 1; k < 5; ++k) {
    xp[k] = xp[k - 1] * xr;
    yp[k] = yp[k - 1] * yr;
  }
  sfor<0, K>([&](auto i) {
    double v = 0.0;
    sfor<0, 5>([&](auto a) {
      sfor<0, 5 - CV(a)>([&](auto b) {
        constexpr double c = BasisMonomials::c[CV(i)][CV(a)][CV(b)];
        if constexpr (c != 0.0) v = mad(c, xp[CV(a)] * yp[CV(b)], v);
      });
    });
    phi[CV(i)] = v;
  });
}

// reference point of local edge NN at s in [0, 1] (counter-clockwise)
template <int NN>
__device__ __forceinline__ void edge_ref(double s, double& xr, double& yr) {
  if constexpr (NN == 0) {
    xr = 1.0 - s;
    yr = s;
  } else if constexpr (NN == 1) {
    xr = 0.0;
    yr = 1.0 - s;
  } else {
    xr = s;
    yr = 0.0;
  }
}

// ---------------------------------------------------------------------------
template <class Real>
struct StageParams {
  Mesh m;
  Real g;
  // state and RK
  const Real* w;      // [3][K][E] state entering the stage
  const Real* w0;     // [3][K][E] RK base state (read when alpha != 0)
  Real* wout;         // [3][K][E] (may alias w0: each thread reads its own
                      // element of w0 before writing it)
  double alpha, beta;  // SSP stage w' = alpha w0 + beta (w + dt R); alpha + beta = 1
  // evaluation buffers of w (read) and of wout (written)
  const Real* vs;     // [3][K][E]
  const Real* rec;    // [3 edges][NREC][E]
  Real* vs_out;
  Real* rec_out;
  // static fields
  const Real* hb;     // [K][E]
  const Real* hbt;    // [3][P1][E] bathymetry traces
  const Real* ghb;    // [2][K1][E] det-scaled bathymetry gradient coefficients
  const Real* lin;    // FP64 only: [2][K][K][E] matrices of the terms linear in xi
                      // (g xi grad h_b source + g Pi(xi h_b) pressure part)
  const float* ahb;   // mixed solve only: [ahb_words(K)][E] low parts lo (and at p = 4
                      // the FP32 parts) of the matrix A of the bathymetry,
                      // sum_n T[n][a][b] h_b,n for b <= a (row-major lower
                      // triangle; see ahb_kernel)
  // time step
  double dt_fixed;    // > 0: fixed step
  double cfl_num;     // cfl * d_min / (2p + 1)
  const double* lam;  // max wave speed of this step's initial state
  double* lam_next;   // accumulator of the evaluated state's wave speed (or null)
  double* lam_clear;  // slot zeroed by thread 0 (or null)
  double inv_det;     // 1 / |det B| (uniform mesh)
  double det;         // |det B|
  double tau_bf, f_c; // bottom friction and Coriolis (Eq. (2)); both 0 = off
  // §3.1 manufactured solution: body force in the volume, exact Dirichlet
  // data as the ghost state of boundary edges (evaluated at the stage time)
  int forcing;
  int dirichlet;
  const double* t_now; // time at the start of the step (device scalar)
  double c_eval;       // time of the evaluated state: t_now + c_eval * dt
  const double* vq;    // volume rule [3][nqv]: x^, y^, weight
  int nqv;
  const double* eq;    // edge rule [nqe][7]: s, weight, L_0(s) .. L_4(s)
  int nqe;
  unsigned* err;      // error word (ERRF_* bits)
  Real* rhs_out;      // mode MODE_RHS output [3][K][E]
};

enum { MODE_EVAL = 0, MODE_STAGE = 1, MODE_RHS = 2 };

__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  // non-negative doubles order like their bit patterns (NaN sorts above all)
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

// Boundary edge with exact Dirichlet data (§3.1 solution at the stage time):
// the ghost state is the exact (xi, U, V) with h_b+ = h_b- and u+ = q+/H+,
// so the flux is not polynomial; it is integrated with the Gauss rule sp.eq
// (the same number of points as the reference scheme) and stored as
// |E| * its Legendre coefficients in the flux slots of the side record.
template <int NN, int P, class Real>
__device__ __forceinline__ void dirichlet_flux(const StageParams<Real>& sp, long long e, Real nx, Real ny, Real len,
                                               const Real* tx, const Real* tU, const Real* tV, const Real* tu,
                                               const Real* tv, const Real* th, const Real* un, const Real* Hs,
                                               Real* rb, long long rs, double t_eval, unsigned& err) {
  constexpr int P1 = P + 1, PB1 = Dims<P>::PB1;   // h_b traces: PB1 modes
  const long long E = sp.m.E;
  const double g = double(sp.g), nxd = double(nx), nyd = double(ny);
  double ax, ay, B11, B12, B21, B22;
  elem_map(sp.m, e, ax, ay, B11, B12, B21, B22);
  auto point = [&](double s, double& x, double& y) {
    double xr, yr;
    edge_ref<NN>(s, xr, yr);
    x = ax + B11 * xr + B12 * yr;
    y = ay + B21 * xr + B22 * yr;
  };
  auto evalN = [&](const Real* tau, const double* L, int n) {
    double v = 0.0;
    for (int j = 0; j < n; ++j) v = fma(double(tau[j]), L[j], v);
    return v;
  };
  auto evalL = [&](const Real* tau, const double* L) { return evalN(tau, L, P1); };
  // wave speed: both sides at s = 0, 1/2, 1
  double lam = 0.0;
  for (int k = 0; k < 3; ++k) {
    const double s = 0.5 * k;
    double L[PB1], pp = 1.0, pc = 2.0 * s - 1.0;   // orthonormal shifted Legendre at s
    L[0] = 1.0;
    L[1] = sqrt(3.0) * pc;
    for (int j = 1; j + 1 < PB1; ++j) {
      const double pn = ((2 * j + 1) * (2.0 * s - 1.0) * pc - j * pp) / (j + 1);
      pp = pc;
      pc = pn;
      L[j + 1] = sqrt(2.0 * (j + 1) + 1.0) * pn;
    }
    const double Hin = evalN(Hs, L, PB1), unin = evalL(un, L), hbin = evalN(th, L, PB1);
    double x, y, xg, Ug, Vg;
    point(s, x, y);
    ms_state(x, y, t_eval, xg, Ug, Vg);
    const double Hg = xg + hbin;
    if (!(Hin > 0.0) || !(Hg > 0.0)) err |= ERRF_DRY;
    lam = fmax(lam, fabs(unin) + sqrt(g * Hin));
    lam = fmax(lam, fabs((Ug * nxd + Vg * nyd) / Hg) + sqrt(g * Hg));
  }
  double acc[3][P1];
  for (int f = 0; f < 3; ++f)
    for (int j = 0; j < P1; ++j) acc[f][j] = 0.0;
  for (int q = 0; q < sp.nqe; ++q) {
    const double* row = sp.eq + 7 * q;
    const double s = row[0], w = row[1];
    const double* L = row + 2;
    const double xi_m = evalL(tx, L), U_m = evalL(tU, L), V_m = evalL(tV, L);
    const double u_m = evalL(tu, L), v_m = evalL(tv, L), hb = evalN(th, L, PB1);
    double x, y, xi_p, U_p, V_p;
    point(s, x, y);
    ms_state(x, y, t_eval, xi_p, U_p, V_p);
    const double Hp = xi_p + hb, u_p = U_p / Hp, v_p = V_p / Hp;
    // A~(c).n of Eq. (8) on both sides
    const double un_m = u_m * nxd + v_m * nyd, un_p = u_p * nxd + v_p * nyd;
    const double pr_m = 0.5 * g * xi_m * (xi_m + 2.0 * hb), pr_p = 0.5 * g * xi_p * (xi_p + 2.0 * hb);
    const double fm[3] = {U_m * nxd + V_m * nyd, U_m * un_m + pr_m * nxd, V_m * un_m + pr_m * nyd};
    const double fp[3] = {U_p * nxd + V_p * nyd, U_p * un_p + pr_p * nxd, V_p * un_p + pr_p * nyd};
    const double cm[3] = {xi_m, U_m, V_m}, cp[3] = {xi_p, U_p, V_p};
    for (int f = 0; f < 3; ++f) {
      const double Fh = 0.5 * (fm[f] + fp[f]) + 0.5 * lam * (cm[f] - cp[f]);
      for (int j = 0; j < P1; ++j) acc[f][j] = fma(w * Fh, L[j], acc[f][j]);
    }
  }
  for (int f = 0; f < 3; ++f)
    for (int j = 0; j < P1; ++j) rb[(f * P1 + j) * rs] = Real(double(len) * acc[f][j]);
}

// Side record of local edge NN of element e for the state (xi, U, V, u, v):
//   [0..P1)      (|E|/2) q.n                       (flux of xi, Eq. (8))
//   [P1..2P1)    (|E|/2) (Pi(U u_n) + g/2 n_x Pi(xi (xi + 2 h_b)))
//   [2P1..3P1)   (|E|/2) (Pi(V u_n) + g/2 n_y Pi(xi (xi + 2 h_b)))
//   [3P1..6P1)   traces of xi, U, V
//   [6P1]        max over s = 0, 1/2, 1 of |u.n| + sqrt(g H)
// all edge polynomials in the orthonormal Legendre basis of the edge in the
// element's own (counter-clockwise) direction.
// The record goes to rb[k * rs], k < NREC (rs = E in HBM, the slot count in
// shared memory).
template <int NN, int P, int FEAT, class Real>
__device__ __forceinline__ void side_record(const StageParams<Real>& sp, long long e, int t, const Real* xi,
                                            const Real* U, const Real* V, const Real* u, const Real* v,
                                            unsigned& err, double t_eval, Real* rb, long long rs) {
  using D = Dims<P>;
  constexpr int P1 = D::P1, PB1 = D::PB1;
  const long long E = sp.m.E;
  Real nx, ny, len;
  edge_geom<FEAT>(sp.m, e, t, NN, nx, ny, len);
  const Real hl = Real(0.5) * len;
  const Real hg = Real(0.5) * sp.g;
  // h_b traces have PB1 >= P1 modes (one more at p = 0): all of them enter
  // the depth at the wave-speed points; the projection of xi (xi + 2 h_b)
  // onto P^p needs only the first P1 (at p = 0, the mean of h_b on the edge)
  Real tx[P1], tU[P1], tV[P1], th[PB1], xe[P1], Hs[PB1];
  trace<NN, P>(xi, tx);
  trace<NN, P>(U, tU);
  trace<NN, P>(V, tV);
  sfor<0, PB1>([&](auto j) {
    constexpr int jj = CV(j);
    th[jj] = sp.hbt[(NN * PB1 + jj) * E + e];
    if constexpr (jj < P1) {
      xe[jj] = fma(Real(2), th[jj], tx[jj]);
      Hs[jj] = tx[jj] + th[jj];
    } else {
      Hs[jj] = th[jj];
    }
  });
  Real Pp[P1], PU[P1], PV[P1], un[P1];
  lprod<P>(tx, xe, Pp);
  const bool dir_edge = FEAT && sp.dirichlet && NN != 0 && neighbour(sp.m, e, NN) < 0;
  if (NN == 0 || (FEAT && (sp.m.geo || dir_edge))) {
    // general edge (the diagonal, any edge of a general mesh, a Dirichlet edge)
    Real tu[P1], tv[P1], qn[P1];
    trace<NN, P>(u, tu);
    trace<NN, P>(v, tv);
    sfor<0, P1>([&](auto j) {
      constexpr int jj = CV(j);
      un[jj] = fma(nx, tu[jj], ny * tv[jj]);
      qn[jj] = fma(nx, tU[jj], ny * tV[jj]);
    });
    if constexpr (FEAT) {
      if (dir_edge) dirichlet_flux<NN, P>(sp, e, nx, ny, len, tx, tU, tV, tu, tv, th, un, Hs, rb, rs, t_eval, err);
    }
    if (!dir_edge) {
      lprod2<P>(tU, tV, un, PU, PV);
      sfor<0, P1>([&](auto j) {
        constexpr int jj = CV(j);
        rb[(0 * P1 + jj) * rs] = hl * qn[jj];
        rb[(1 * P1 + jj) * rs] = hl * fma(hg * nx, Pp[jj], PU[jj]);
        rb[(2 * P1 + jj) * rs] = hl * fma(hg * ny, Pp[jj], PV[jj]);
      });
    }
  } else if constexpr (NN != 0) {
    // axis-aligned: n = -s e_x (edge 1) or -s e_y (edge 2), s = +1 lower,
    // -1 upper; u.n = -s u_1 (or -s v), and the sign folds into the scale
    const Real sh = (t ? Real(1) : Real(-1)) * hl;   // -s |E|/2
    trace<NN, P>(NN == 1 ? u : v, un);               // u.n up to the sign -s
    lprod2<P>(tU, tV, un, PU, PV);
    sfor<0, P1>([&](auto j) {
      constexpr int jj = CV(j);
      if constexpr (NN == 1) {
        rb[(0 * P1 + jj) * rs] = sh * tU[jj];
        rb[(1 * P1 + jj) * rs] = sh * fma(hg, Pp[jj], PU[jj]);
        rb[(2 * P1 + jj) * rs] = sh * PV[jj];
      } else {
        rb[(0 * P1 + jj) * rs] = sh * tV[jj];
        rb[(1 * P1 + jj) * rs] = sh * PU[jj];
        rb[(2 * P1 + jj) * rs] = sh * fma(hg, Pp[jj], PV[jj]);
      }
    });
  }
  sfor<0, P1>([&](auto j) {
    constexpr int jj = CV(j);
    rb[(3 * P1 + jj) * rs] = tx[jj];
    rb[(4 * P1 + jj) * rs] = tU[jj];
    rb[(5 * P1 + jj) * rs] = tV[jj];
  });
  // wave speed of this side at s = 0, 1/2, 1 (|u.n| is sign-free)
  const Real h0 = edge_point<D::PB, 0>(Hs), h1 = edge_point<D::PB, 1>(Hs), h2 = edge_point<D::PB, 2>(Hs);
  const Real u0 = edge_point<P, 0>(un), u1 = edge_point<P, 1>(un), u2 = edge_point<P, 2>(un);
  if (!(h0 > Real(0)) || !(h1 > Real(0)) || !(h2 > Real(0))) err |= ERRF_DRY;
  const Real l0 = fabs(u0) + sqrt(sp.g * h0);
  const Real l1 = fabs(u1) + sqrt(sp.g * h1);
  const Real l2 = fabs(u2) + sqrt(sp.g * h2);
  rb[(6 * P1) * rs] = fmax(fmax(l0, l1), l2);
}

// Evaluation of one element's state: velocity projection, volume + source
// integrals -> vs_out, side records -> rec_out; returns the element wave
// speed |q_bar/H_bar| + sqrt(g H_bar) from the means (mean = sqrt(2) c_1).
// Element wave speed |q_bar / H_bar| + sqrt(g H_bar) from the first
// coefficients H_0 = xi_0 + h_b,0 (in the state's precision), U_0, V_0 of an
// element (mean = sqrt(2) c_1; the sqrt(2) cancels in the velocity).
// FP64 state: in FP64.  FP32 state: in FP32 (IEEE division and square root);
// the value only enters the maximum that sets the CFL step, and FP64
// square roots and divisions of every element cost as much FP64 pipe time
// as a third of an FP32 stage on GB300, whose FP64 rate is 1/64 of FP32.
__device__ __forceinline__ double element_wave_speed_H(double H0, double U0, double V0, double g) {
  const double um = U0 / H0, vm = V0 / H0;
  return sqrt(fma(um, um, vm * vm)) + sqrt(g * 1.4142135623730951 * H0);
}
__device__ __forceinline__ float element_wave_speed_H(float H0, float U0, float V0, float g) {
  const float um = __fdiv_rn(U0, H0), vm = __fdiv_rn(V0, H0);
  return __fadd_rn(__fsqrt_rn(__fmaf_rn(um, um, __fmul_rn(vm, vm))),
                   __fsqrt_rn(__fmul_rn(__fmul_rn(g, 1.41421356f), H0)));
}

// Depth H = xi + h_b and the velocity projection of Eq. (12) of element e.
template <int P, class Real, class PR>
__device__ __forceinline__ void element_velocity(const StageParams<Real>& sp, long long e, const Real* xi,
                                                 const Real* U, const Real* V, Real* hb, Real* H, Real* u, Real* v,
                                                 unsigned& err) {
  constexpr int K = Dims<P>::K;
  const long long E = sp.m.E;
  sfor<0, K>([&](auto i) {
    hb[CV(i)] = sp.hb[CV(i) * E + e];
    H[CV(i)] = xi[CV(i)] + hb[CV(i)];
  });
  bool solved;
  if constexpr (std::is_same<PR, MixedIR>::value)
    solved = project_velocity_ir<P>(H, xi, hb, U, V, u, v, sp.ahb + e, E);
  else
    solved = project_velocity<P, PR>(H, U, V, u, v);
  if (!solved) err |= ERRF_DRY;
}

// Volume + source integrals of element e (the velocity u, v already
// projected) to vsb[(f K + a) * vss].
template <int P, class Real, int FEAT>
__device__ __forceinline__ void volume_to(const StageParams<Real>& sp, long long e, int t, const Real* xi,
                                          const Real* U, const Real* V, const Real* u, const Real* v, const Real* hb,
                                          double t_eval, Real* vsb, long long vss) {
  using D = Dims<P>;
  constexpr int K = D::K, K1 = D::K1;
  const long long E = sp.m.E;
  // volume integrals (A~, grad phi_a) (Eqs. (15)-(16)): grad phi_a lies in
  // P^{p-1}, so only the first K1 coefficients of each projected product count
  constexpr bool kLin = std::is_same<Real, double>::value;
  constexpr int K1A = K1 > 0 ? K1 : 1;   // array extent (p = 0 has no volume term)
  Real Puu[K1A], Puv[K1A], Pvu[K1A], Pvv[K1A], Pxx[K1A];
  momentum_products<P>(U, V, u, v, Puu, Puv, Pvu, Pvv);
  // pressure 1/2 g xi (xi + 2 h_b): in FP64 the part g xi h_b, linear in xi,
  // and the source g xi grad h_b of Eq. (5) come from the static matrices
  // sp.lin (fewer FP64 operations), leaving the symmetric Pi(xi xi)
  Real Sx[K], Sy[K];
  if constexpr (kLin) {
    tprod_sym<P, K1>(xi, Pxx);
  } else {
    Real xe[K];
    sfor<0, K>([&](auto i) { xe[CV(i)] = fma(Real(2), hb[CV(i)], xi[CV(i)]); });
    tprod<P, K1, K>(xi, xe, Pxx);
    // g sum_{i,m} T[a][i][m] xi_i ghb_m, ghb = det B * coefficients of grad h_b
    constexpr int KB1 = D::KB1;   // grad h_b lies in P^{max(p,1)-1}
    Real gx[KB1], gy[KB1];
    sfor<0, KB1>([&](auto m) {
      gx[CV(m)] = sp.ghb[CV(m) * E + e];
      gy[CV(m)] = sp.ghb[(KB1 + CV(m)) * E + e];
    });
    tprod<P, K, KB1>(xi, gx, Sx);
    tprod<P, K, KB1>(xi, gy, Sy);
  }
  const Real hg = Real(0.5) * sp.g;
  Real FxU[K1A], FyV[K1A];
  sfor<0, K1>([&](auto i) {
    FxU[CV(i)] = fma(hg, Pxx[CV(i)], Puu[CV(i)]);
    FyV[CV(i)] = fma(hg, Pxx[CV(i)], Pvv[CV(i)]);
  });
  // body force of the §3.1 solution: (F, phi_a) = |det B| sum_q w_q F(x_q) phi^_a(x^_q)
  double fU[K], fV[K];
  if (FEAT && sp.forcing) {
    sfor<0, K>([&](auto a) {
      fU[CV(a)] = 0.0;
      fV[CV(a)] = 0.0;
    });
    double ax, ay, B11, B12, B21, B22;
    elem_map(sp.m, e, ax, ay, B11, B12, B21, B22);
    const double det = B11 * B22 - B12 * B21;
    for (int q = 0; q < sp.nqv; ++q) {
      const double xr = sp.vq[q], yr = sp.vq[sp.nqv + q], w = sp.vq[2 * sp.nqv + q] * det;
      double phi[K], Fx, Fy;
      basis_at<K>(xr, yr, phi);
      ms_force(ax + B11 * xr + B12 * yr, ay + B21 * xr + B22 * yr, t_eval, double(sp.g), Fx, Fy);
      sfor<0, K>([&](auto a) {
        fU[CV(a)] = fma(w * Fx, phi[CV(a)], fU[CV(a)]);
        fV[CV(a)] = fma(w * Fy, phi[CV(a)], fV[CV(a)]);
      });
    }
  }
  // (F, grad phi_a) = sum_r sum_i S[r][a][i] (G_1r F^x_i + G_2r F^y_i)
  Real G11, G12, G21, G22;
  elem_G<FEAT>(sp.m, e, t, G11, G12, G21, G22);
  const bool full_G = FEAT && sp.m.geo != nullptr;   // off-diagonal terms vanish on the uniform mesh
  sfor<0, K>([&](auto a) {
    constexpr int aa = CV(a);
    // explicit fused forms: a contracted a*b + c*d could fuse either product,
    // and the choice would depend on the kernel the code is compiled into
    Real v0 = fma(G11, sdot_row<P, 0, aa>(U), G22 * sdot_row<P, 1, aa>(V));
    Real v1 = fma(G11, sdot_row<P, 0, aa>(FxU), G22 * sdot_row<P, 1, aa>(Puv));
    Real v2 = fma(G11, sdot_row<P, 0, aa>(Pvu), G22 * sdot_row<P, 1, aa>(FyV));
    if (full_G) {
      v0 += fma(G12, sdot_row<P, 1, aa>(U), G21 * sdot_row<P, 0, aa>(V));
      v1 += fma(G12, sdot_row<P, 1, aa>(FxU), G21 * sdot_row<P, 0, aa>(Puv));
      v2 += fma(G12, sdot_row<P, 1, aa>(Pvu), G21 * sdot_row<P, 0, aa>(FyV));
    }
    if constexpr (kLin) {
      sfor<0, K>([&](auto k) {
        v1 = fma(sp.lin[((0 * K + aa) * K + CV(k)) * E + e], xi[CV(k)], v1);
        v2 = fma(sp.lin[((1 * K + aa) * K + CV(k)) * E + e], xi[CV(k)], v2);
      });
    } else {
      v1 = fma(sp.g, Sx[aa], v1);
      v2 = fma(sp.g, Sy[aa], v2);
    }
    if (FEAT && sp.forcing) {
      v1 += Real(fU[aa]);
      v2 += Real(fV[aa]);
    }
    if (sp.tau_bf != 0.0 || sp.f_c != 0.0) {
      // (-tau_bf q + f_c (V, -U), phi_a) = |det B| (-tau_bf U_a + f_c V_a, ...)
      const double det = (FEAT && sp.m.geo) ? sp.m.geo[GEO_DET * sp.m.E + e] : sp.det;
      const Real tq = Real(-sp.tau_bf * det), fq = Real(sp.f_c * det);
      v1 = fma(tq, U[aa], fma(fq, V[aa], v1));
      v2 = fma(tq, V[aa], fma(-fq, U[aa], v2));
    }
    vsb[(0 * K + aa) * vss] = v0;
    vsb[(1 * K + aa) * vss] = v1;
    vsb[(2 * K + aa) * vss] = v2;
  });
}

// Evaluation into explicit destinations: volume + source integrals to
// vsb[(f K + a) * vss], the side record of local edge n to
// recb + n NREC recs with stride recs.
template <int P, class Real, class PR, int FEAT, bool LAM = true>
__device__ __forceinline__ double evaluate_to(const StageParams<Real>& sp, long long e, int t, const Real* xi,
                                              const Real* U, const Real* V, unsigned& err, double t_eval, Real* vsb,
                                              long long vss, Real* recb, long long recs) {
  using D = Dims<P>;
  constexpr int K = D::K, NREC = D::NREC;
  Real hb[K], H[K], u[K], v[K];
  element_velocity<P, Real, PR>(sp, e, xi, U, V, hb, H, u, v, err);
  volume_to<P, Real, FEAT>(sp, e, t, xi, U, V, u, v, hb, t_eval, vsb, vss);
  side_record<0, P, FEAT>(sp, e, t, xi, U, V, u, v, err, t_eval, recb + 0LL * NREC * recs, recs);
  side_record<1, P, FEAT>(sp, e, t, xi, U, V, u, v, err, t_eval, recb + 1LL * NREC * recs, recs);
  side_record<2, P, FEAT>(sp, e, t, xi, U, V, u, v, err, t_eval, recb + 2LL * NREC * recs, recs);
  double lam_e = 0.0;
  if (LAM && sp.lam_next) lam_e = double(element_wave_speed_H(H[0], U[0], V[0], sp.g));
  return lam_e;
}

// Evaluation into the launch's HBM buffers sp.vs_out and sp.rec_out.
template <int P, class Real, class PR, int FEAT>
__device__ __forceinline__ double evaluate(const StageParams<Real>& sp, long long e, int t, const Real* xi,
                                           const Real* U, const Real* V, unsigned& err, double t_eval) {
  const long long E = sp.m.E;
  return evaluate_to<P, Real, PR, FEAT>(sp, e, t, xi, U, V, err, t_eval, sp.vs_out + e, E, sp.rec_out + e, E);
}

// Numerical flux on local edge NN and its lift: res[f][a] -= sum_j R[NN][j][a] F^_f,j
// with F^ = |E| (1/2 (A~(c-) + A~(c+)).n + 1/2 lambda (c- - c+)) (Lax-Friedrichs).
// ro, rn: the element's and the neighbour's side records of the edge (entry
// k at [k * rs]); rn = nullptr on a boundary edge.
template <int NN, int P, int FEAT, class Real>
__device__ __forceinline__ void edge_flux_lift_at(const StageParams<Real>& sp, long long e, int t, const Real* ro,
                                                  long long ros, const Real* rn, long long rns,
                                                  Real (&res)[3][Dims<P>::K]) {
  using D = Dims<P>;
  constexpr int P1 = D::P1;
  const long long E = ros, N = rns;
  Real F[3][P1];
  if (rn) {
    Real nx, ny, len;
    edge_geom<FEAT>(sp.m, e, t, NN, nx, ny, len);
    const Real lam = fmax(ro[(6 * P1) * E], rn[(6 * P1) * N]);
    const Real hl = Real(0.5) * len * lam;
    // the neighbour's polynomials run the other way (s -> 1 - s flips the sign
    // of odd Legendre modes) and its fluxes use the opposite normal
    sfor<0, 3>([&](auto ff) {
      constexpr int fv = CV(ff);
      sfor<0, P1>([&](auto j) {
        constexpr int jj = CV(j);
        constexpr bool odd = (jj & 1) != 0;
        const Real pm = ro[(fv * P1 + jj) * E], pp = rn[(fv * P1 + jj) * N];
        const Real wm = ro[((3 + fv) * P1 + jj) * E], wp = rn[((3 + fv) * P1 + jj) * N];
        const Real phi = odd ? pm + pp : pm - pp;
        const Real jmp = odd ? wm + wp : wm - wp;
        F[fv][jj] = fma(hl, jmp, phi);
      });
    });
  } else if (FEAT && sp.dirichlet) {
    // Dirichlet edge: the side record holds the full |E| F^ (see dirichlet_flux)
    sfor<0, 3>([&](auto ff) {
      sfor<0, P1>([&](auto j) { F[CV(ff)][CV(j)] = ro[(CV(ff) * P1 + CV(j)) * E]; });
    });
  } else {
    // reflective wall, mirror ghost: F^(xi) = 0 and
    // F^(q) = |E| n (Pi(q.n u.n) + g/2 Pi(xi (xi + 2 h_b)) + lambda q.n)
    Real nx, ny, len;
    edge_geom<FEAT>(sp.m, e, t, NN, nx, ny, len);
    const Real lam = ro[(6 * P1) * E];
    sfor<0, P1>([&](auto j) {
      constexpr int jj = CV(j);
      const Real pn = fma(nx, ro[(1 * P1 + jj) * E], fma(ny, ro[(2 * P1 + jj) * E], lam * ro[jj * E]));
      F[0][jj] = Real(0);
      F[1][jj] = Real(2) * nx * pn;
      F[2][jj] = Real(2) * ny * pn;
    });
  }
  lift_sub<NN, P>(F[0], res[0]);
  lift_sub<NN, P>(F[1], res[1]);
  lift_sub<NN, P>(F[2], res[2]);
}

template <int NN, int P, int FEAT, class Real>
__device__ __forceinline__ void edge_flux_lift(const StageParams<Real>& sp, long long e, int t,
                                               Real (&res)[3][Dims<P>::K]) {
  constexpr int NREC = Dims<P>::NREC;
  const long long E = sp.m.E;
  const long long f = neighbour(sp.m, e, NN);
  const Real* ro = sp.rec + (long long)NN * NREC * E + e;
  const Real* rn = f >= 0 ? sp.rec + (long long)NN * NREC * E + f : nullptr;
  edge_flux_lift_at<NN, P, FEAT>(sp, e, t, ro, E, rn, E, res);
}

template <class Real>
__device__ __forceinline__ bool finite(Real x) { return isfinite(x); }

// Work of one element in one launch: MODE_STAGE = flux, lift, RK update and
// evaluation of the new state; MODE_EVAL = evaluation only; MODE_RHS = flux
// and lift of an evaluated state, written as d_t c.  Returns the element's
// wave speed (0 unless sp.lam_next is set) through lam_e.
template <int P, class Real, class PR, int MODE, int FEAT>
__device__ __forceinline__ void stage_element(const StageParams<Real>& sp, long long e, double dt, double& lam_e,
                                              unsigned& err) {
  using D = Dims<P>;
  constexpr int K = D::K;
  const long long E = sp.m.E;
  const int t = (int)(e & 1);
  Real w[3][K];
  sfor<0, 3>([&](auto f) {
    sfor<0, K>([&](auto i) { w[CV(f)][CV(i)] = sp.w[(CV(f) * K + CV(i)) * E + e]; });
  });
  const double t_eval = (FEAT && sp.t_now) ? *sp.t_now + sp.c_eval * dt : 0.0;
  if constexpr (MODE == MODE_EVAL) {
    lam_e = evaluate<P, Real, PR, FEAT>(sp, e, t, w[0], w[1], w[2], err, t_eval);
  } else {
    Real res[3][K];
    sfor<0, 3>([&](auto f) {
      sfor<0, K>([&](auto i) { res[CV(f)][CV(i)] = sp.vs[(CV(f) * K + CV(i)) * E + e]; });
    });
    edge_flux_lift<0, P, FEAT>(sp, e, t, res);
    edge_flux_lift<1, P, FEAT>(sp, e, t, res);
    edge_flux_lift<2, P, FEAT>(sp, e, t, res);
    if constexpr (MODE == MODE_RHS) {
      const Real idet = Real(elem_inv_det<FEAT>(sp.m, e, sp.inv_det));
      sfor<0, 3>([&](auto f) {
        sfor<0, K>([&](auto i) { sp.rhs_out[(CV(f) * K + CV(i)) * E + e] = res[CV(f)][CV(i)] * idet; });
      });
    } else {
      // w' = alpha w0 + beta (w + dt R),  R = res / |det B|, alpha + beta = 1,
      // evaluated as w0 + beta ((w - w0) + dt R): a constant state stays
      // exactly constant and the result is rounded once (alpha and beta
      // themselves are never rounded to the working precision)
      const Real b = Real(sp.beta), c = Real(dt * elem_inv_det<FEAT>(sp.m, e, sp.inv_det));
      bool fin = true;
      sfor<0, 3>([&](auto f) {
        sfor<0, K>([&](auto i) {
          const long long idx = (CV(f) * K + CV(i)) * E + e;
          Real x;
          if (sp.alpha != 0.0) {
            const Real base = sp.w0[idx];
            x = fma(b, fma(c, res[CV(f)][CV(i)], w[CV(f)][CV(i)] - base), base);
          } else {
            x = fma(c, res[CV(f)][CV(i)], w[CV(f)][CV(i)]);
          }
          fin = fin && finite(x);
          w[CV(f)][CV(i)] = x;
          sp.wout[idx] = x;
        });
      });
      if (!fin) err |= ERRF_NONFINITE;
      lam_e = evaluate<P, Real, PR, FEAT>(sp, e, t, w[0], w[1], w[2], err, t_eval);
    }
  }
}

// maximum of a non-negative float over the block, valid in thread 0 (all
// threads must call); the FP32 paths keep their wave speeds in float so that
// no FP64 instruction is spent on the maximum
__device__ __forceinline__ float block_max_f(float v) {
  __shared__ float redf[32];
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) redf[wid] = v;
  __syncthreads();
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    v = lane < nw ? redf[lane] : 0.f;
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  }
  return v;
}

// maximum of v over the block, valid in thread 0 (all threads must call)
__device__ __forceinline__ double block_max(double v) {
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    v = lane < nw ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  }
  return v;
}

// One launch per RK stage (MODE_STAGE), per initial evaluation (MODE_EVAL) or
// per right-hand side (MODE_RHS).  One thread per element.  FEAT = 0 is the
// uniform-mesh path; FEAT = 1 adds general meshes, the §3.1 body force and
// Dirichlet edges (kept out of the fast path's registers and code).
// Minimum resident 128-thread blocks per SM requested from the register
// allocator (measured on GB300): FP32-state kernels run fastest at 6 (<= 80
// registers: 24 warps per SM hide more of the load latency than the spills
// to L1 cost; 6 % faster on the ensemble and 3 % on 512^2 meshes than 4
// blocks of 128 registers), except with the FP64 velocity solve, whose FP64
// LDL^T factors take two registers per entry (4 blocks: at 80 registers it
// spilled to 15 % longer steps at p = 4); FP64 at p <= 2 at 3 (their natural
// fit); FP64 at p >= 3 needs the full register file.
template <int P, class Real, class PR>
constexpr int stage_min_blocks() {
  return std::is_same<Real, float>::value ? (std::is_same<PR, double>::value ? 4 : 6) : (P <= 2 ? 3 : 1);
}

template <int P, class Real, class PR, int MODE, int FEAT>
__global__ void __launch_bounds__(128, (stage_min_blocks<P, Real, PR>())) stage_kernel(const StageParams<Real> sp) {
  double lam_acc = 0.0;
  unsigned err = 0;
  double dt = 0.0;
  if constexpr (MODE == MODE_STAGE) {
    dt = sp.dt_fixed > 0.0 ? sp.dt_fixed : sp.cfl_num / sp.lam[0];
  }
  if constexpr (std::is_same<Real, float>::value) {
    // FP32 state: grid-stride over blocks of elements (the launch caps the
    // grid at the resident CTAs)
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e - threadIdx.x < sp.m.E;
         e += (long long)gridDim.x * blockDim.x) {
      double lam_e = 0.0;
      if (e < sp.m.E) stage_element<P, Real, PR, MODE, FEAT>(sp, e, dt, lam_e, err);
      lam_acc = fmax(lam_acc, lam_e);
    }
  } else {
    // FP64: one element per thread, the grid covers the mesh
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < sp.m.E) stage_element<P, Real, PR, MODE, FEAT>(sp, e, dt, lam_acc, err);
  }
  if (sp.lam_next) {
    const double l = block_max(lam_acc);
    if (threadIdx.x == 0) atomic_max_nonneg(sp.lam_next, l);
  }
  if (err) atomicOr(sp.err, err);
  if (blockIdx.x == 0 && threadIdx.x == 0 && sp.lam_clear) *sp.lam_clear = 0.0;
}

// Static per-element fields of the bathymetry h_b in P^PB, PB = max(p, 1):
// its coefficients, its edge traces (PB + 1 Legendre modes) and the
// det-scaled gradient coefficients gh_r = sum_c G_rc (d^_c h_b) in P^{PB-1}.
// The reference tables of order PB serve the order-p indices too (the basis
// is hierarchical).
template <int P, class Real>
__global__ void static_kernel(Mesh m, double g, const double* __restrict__ hb64, Real* hb, Real* hbt, Real* ghb,
                              Real* lin) {
  using D = Dims<P>;
  constexpr int PB = D::PB;
  using Tb = RefTables<PB>;
  constexpr int K = D::K, K1 = D::K1, KB = D::KB, PB1 = D::PB1, KB1 = D::KB1;
  const long long E = m.E;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const int t = (int)(e & 1);
  double h[KB];
  sfor<0, KB>([&](auto i) {
    h[CV(i)] = hb64[CV(i) * E + e];
    hb[CV(i) * E + e] = Real(h[CV(i)]);
  });
  auto tr = [&](auto nn) {
    double tau[PB1];
    trace<CV(nn), PB>(h, tau);
    sfor<0, PB1>([&](auto j) { hbt[(CV(nn) * PB1 + CV(j)) * E + e] = Real(tau[CV(j)]); });
  };
  sfor<0, 3>(tr);
  double G[2][2];
  elem_G<1>(m, e, t, G[0][0], G[0][1], G[1][0], G[1][1]);
  // reference derivative coefficients d_c,m = sum_i S[c][i][m] h_i and the
  // det-scaled physical gradient gh_r = sum_c G_rc d_c
  double d[2][KB1];
  sfor<0, 2>([&](auto c) {
    sfor<0, KB1>([&](auto mm) {
      double acc = 0.0;
      sfor<0, KB>([&](auto i) {
        constexpr double s = Tb::S[CV(c)][CV(i)][CV(mm)];
        if constexpr (s != 0.0) acc = fma(s, h[CV(i)], acc);
      });
      d[CV(c)][CV(mm)] = acc;
    });
  });
  double gh[2][KB1];
  sfor<0, 2>([&](auto r) {
    sfor<0, KB1>([&](auto mm) {
      gh[CV(r)][CV(mm)] = G[CV(r)][0] * d[0][CV(mm)] + G[CV(r)][1] * d[1][CV(mm)];
      ghb[(CV(r) * KB1 + CV(mm)) * E + e] = Real(gh[CV(r)][CV(mm)]);
    });
  });
  if (!lin) return;
  // lin[r][a][k] (a, k < K): coefficient of xi_k in the r-momentum volume + source
  //   g sum_c G_rc sum_{i<K1} S[c][a][i] sum_m T[i][k][m] h_m  (pressure g xi h_b)
  // + g sum_m T[a][k][m] gh_r,m                              (source g xi d_r h_b)
  sfor<0, K>([&](auto a) {
    sfor<0, K>([&](auto k) {
      double pres[2] = {0.0, 0.0};
      sfor<0, 2>([&](auto c) {
        sfor<0, K1>([&](auto i) {
          constexpr double s = Tb::S[CV(c)][CV(a)][CV(i)];
          if constexpr (s != 0.0) {
            double th = 0.0;
            sfor<0, KB>([&](auto mm) {
              constexpr double tt = Tb::T[CV(i)][CV(k)][CV(mm)];
              if constexpr (tt != 0.0) th = fma(tt, h[CV(mm)], th);
            });
            pres[CV(c)] = fma(s, th, pres[CV(c)]);
          }
        });
      });
      sfor<0, 2>([&](auto r) {
        double src = 0.0;
        sfor<0, KB1>([&](auto mm) {
          constexpr double tt = Tb::T[CV(a)][CV(k)][CV(mm)];
          if constexpr (tt != 0.0) src = fma(tt, gh[CV(r)][CV(mm)], src);
        });
        const double pr = G[CV(r)][0] * pres[0] + G[CV(r)][1] * pres[1];
        lin[((CV(r) * K + CV(a)) * K + CV(k)) * E + e] = Real(g * (pr + src));
      });
    });
  });
}

// Per-block partial sums of mass and energy (FP64); reduced in a fixed order
// by diag_finish_kernel.
template <int P, class Real, class PR>
__global__ void __launch_bounds__(128) diag_kernel(Mesh m, const Real* __restrict__ w, const Real* __restrict__ hb,
                                                   double det, double g, double* partial) {
  using D = Dims<P>;
  constexpr int K = D::K;
  const long long E = m.E;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double ms = 0.0, en = 0.0;
  if (e < E) {
    Real xi[K], U[K], V[K], H[K], u[K], v[K];
    sfor<0, K>([&](auto i) {
      xi[CV(i)] = w[CV(i) * E + e];
      U[CV(i)] = w[(K + CV(i)) * E + e];
      V[CV(i)] = w[(2 * K + CV(i)) * E + e];
      H[CV(i)] = xi[CV(i)] + hb[CV(i) * E + e];
    });
    project_velocity<P, PR>(H, U, V, u, v);
    if (m.geo) det = m.geo[GEO_DET * E + e];
    ms = det * double(xi[0]) * 0.70710678118654752;
    sfor<0, K>([&](auto i) {
      en += g * double(xi[CV(i)]) * double(xi[CV(i)]) + double(U[CV(i)]) * double(u[CV(i)]) +
            double(V[CV(i)]) * double(v[CV(i)]);
    });
    en *= 0.5 * det;
  }
  __shared__ double sm[128], se[128];
  sm[threadIdx.x] = ms;
  se[threadIdx.x] = en;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sm[threadIdx.x] += sm[threadIdx.x + s];
      se[threadIdx.x] += se[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = sm[0];
    partial[2 * blockIdx.x + 1] = se[0];
  }
}

}  // namespace dgswe
