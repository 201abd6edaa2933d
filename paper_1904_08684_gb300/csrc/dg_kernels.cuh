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
};

// error word bits
enum : unsigned { ERRF_DRY = 1u, ERRF_NONFINITE = 2u };

// ---------------------------------------------------------------------------
// Uniform quad-split mesh (§2.3).  Element e = 2 (j nx + i) + t.
struct Mesh {
  int nx, ny;
  long long E;
  double hx, hy;   // quad sizes
  double diag;     // sqrt(hx^2 + hy^2)
  int periodic;    // 1 periodic, 0 reflective walls
};

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

// Outward unit normal and length of local edge n.  Lower triangle: edge 0 is
// the diagonal (normal (hy, hx)/diag), edge 1 the left side (-1, 0), edge 2
// the bottom (0, -1); the upper triangle has the opposite normals.
template <class Real>
__device__ __forceinline__ void edge_geom(const Mesh& m, int t, int n, Real& nx, Real& ny, Real& len) {
  const Real s = t ? Real(-1) : Real(1);
  if (n == 0) {
    nx = s * Real(m.hy / m.diag);
    ny = s * Real(m.hx / m.diag);
    len = Real(m.diag);
  } else if (n == 1) {
    nx = -s;
    ny = Real(0);
    len = Real(m.hy);
  } else {
    nx = Real(0);
    ny = -s;
    len = Real(m.hx);
  }
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
// Velocity projection (Eq. (12)): A u = U, A v = V with
// A_ab = sum_n T[n][a][b] H_n (SPD iff H > 0 on the element), solved by an
// LDL^T factorisation in precision PR.  Returns false if a pivot is not
// positive (dry element).
template <int P, class PR, class R>
__device__ __forceinline__ bool project_velocity(const R* H, const R* U, const R* V, R* u, R* v) {
  using Tb = RefTables<P>;
  constexpr int K = Tb::K;
  PR Hd[K], L[K][K], Dg[K], rD[K], y[K];
  sfor<0, K>([&](auto n) { Hd[CV(n)] = PR(H[CV(n)]); });
  bool ok = true;
  // left-looking LDL^T: column j uses W_k = L_jk D_k (k < j)
  sfor<0, K>([&](auto jj) {
    constexpr int j = CV(jj);
    PR W[K > 1 ? K : 1];
    PR d = PR(0);
    sfor<0, K>([&](auto n) {
      constexpr double t = Tb::T[CV(n)][j][j];
      if constexpr (t != 0.0) d = fma(PR(t), Hd[CV(n)], d);
    });
    sfor<0, j>([&](auto k) {
      W[CV(k)] = L[j][CV(k)] * Dg[CV(k)];
      d = fma(-L[j][CV(k)], W[CV(k)], d);
    });
    ok = ok && (d > PR(0));
    Dg[j] = d;
    rD[j] = PR(1) / d;
    sfor<j + 1, K>([&](auto ii) {
      constexpr int i = CV(ii);
      PR a = PR(0);
      sfor<0, K>([&](auto n) {
        constexpr double t = Tb::T[CV(n)][i][j];
        if constexpr (t != 0.0) a = fma(PR(t), Hd[CV(n)], a);
      });
      sfor<0, j>([&](auto k) { a = fma(-L[i][CV(k)], W[CV(k)], a); });
      L[i][j] = a * rD[j];
    });
  });
  // two right-hand sides: L y = b, y <- y / D, L^T x = y
  auto solve = [&](const R* b, R* x) {
    sfor<0, K>([&](auto ii) {
      constexpr int i = CV(ii);
      PR s = PR(b[i]);
      sfor<0, i>([&](auto k) { s = fma(-L[i][CV(k)], y[CV(k)], s); });
      y[i] = s;
    });
    sfor<0, K>([&](auto rr) {
      constexpr int i = K - 1 - CV(rr);
      PR s = y[i] * rD[i];
      sfor<i + 1, K>([&](auto k) { s = fma(-L[CV(k)][i], y[CV(k)], s); });
      y[i] = s;
      x[i] = R(s);
    });
  };
  solve(U, u);
  solve(V, v);
  return ok;
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
  // time step
  double dt_fixed;    // > 0: fixed step
  double cfl_num;     // cfl * d_min / (2p + 1)
  const double* lam;  // max wave speed of this step's initial state
  double* lam_next;   // accumulator of the evaluated state's wave speed (or null)
  double* lam_clear;  // slot zeroed by thread 0 (or null)
  double* t;          // time, advanced by dt by thread 0 (or null)
  double inv_det;     // 1 / |det B| (uniform mesh)
  double det;         // |det B|
  double tau_bf, f_c; // bottom friction and Coriolis (Eq. (2)); both 0 = off
  unsigned* err;      // error word (ERRF_* bits)
  Real* rhs_out;      // mode MODE_RHS output [3][K][E]
};

enum { MODE_EVAL = 0, MODE_STAGE = 1, MODE_RHS = 2 };

__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  // non-negative doubles order like their bit patterns (NaN sorts above all)
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

// Side record of local edge NN of element e for the state (xi, U, V, u, v):
//   [0..P1)      (|E|/2) q.n                       (flux of xi, Eq. (8))
//   [P1..2P1)    (|E|/2) (Pi(U u_n) + g/2 n_x Pi(xi (xi + 2 h_b)))
//   [2P1..3P1)   (|E|/2) (Pi(V u_n) + g/2 n_y Pi(xi (xi + 2 h_b)))
//   [3P1..6P1)   traces of xi, U, V
//   [6P1]        max over s = 0, 1/2, 1 of |u.n| + sqrt(g H)
// all edge polynomials in the orthonormal Legendre basis of the edge in the
// element's own (counter-clockwise) direction.
template <int NN, int P, class Real>
__device__ __forceinline__ void side_record(const StageParams<Real>& sp, long long e, int t, const Real* xi,
                                            const Real* U, const Real* V, const Real* u, const Real* v,
                                            unsigned& err) {
  using D = Dims<P>;
  constexpr int P1 = D::P1, NREC = D::NREC;
  const long long E = sp.m.E;
  Real nx, ny, len;
  edge_geom(sp.m, t, NN, nx, ny, len);
  const Real hl = Real(0.5) * len;
  const Real hg = Real(0.5) * sp.g;
  Real tx[P1], tU[P1], tV[P1], th[P1], xe[P1], Hs[P1];
  trace<NN, P>(xi, tx);
  trace<NN, P>(U, tU);
  trace<NN, P>(V, tV);
  sfor<0, P1>([&](auto j) {
    constexpr int jj = CV(j);
    th[jj] = sp.hbt[(NN * P1 + jj) * E + e];
    xe[jj] = fma(Real(2), th[jj], tx[jj]);
    Hs[jj] = tx[jj] + th[jj];
  });
  Real Pp[P1], PU[P1], PV[P1], un[P1];
  lprod<P>(tx, xe, Pp);
  Real* rb = sp.rec_out + (long long)NN * NREC * E + e;
  if constexpr (NN == 0) {
    // diagonal: n = s (hy, hx) / diag
    Real tu[P1], tv[P1], qn[P1];
    trace<NN, P>(u, tu);
    trace<NN, P>(v, tv);
    sfor<0, P1>([&](auto j) {
      constexpr int jj = CV(j);
      un[jj] = fma(nx, tu[jj], ny * tv[jj]);
      qn[jj] = fma(nx, tU[jj], ny * tV[jj]);
    });
    lprod<P>(tU, un, PU);
    lprod<P>(tV, un, PV);
    sfor<0, P1>([&](auto j) {
      constexpr int jj = CV(j);
      rb[(0 * P1 + jj) * E] = hl * qn[jj];
      rb[(1 * P1 + jj) * E] = hl * fma(hg * nx, Pp[jj], PU[jj]);
      rb[(2 * P1 + jj) * E] = hl * fma(hg * ny, Pp[jj], PV[jj]);
    });
  } else {
    // axis-aligned: n = -s e_x (edge 1) or -s e_y (edge 2), s = +1 lower,
    // -1 upper; u.n = -s u_1 (or -s v), and the sign folds into the scale
    const Real sh = (t ? Real(1) : Real(-1)) * hl;   // -s |E|/2
    trace<NN, P>(NN == 1 ? u : v, un);               // u.n up to the sign -s
    lprod<P>(tU, un, PU);
    lprod<P>(tV, un, PV);
    sfor<0, P1>([&](auto j) {
      constexpr int jj = CV(j);
      if constexpr (NN == 1) {
        rb[(0 * P1 + jj) * E] = sh * tU[jj];
        rb[(1 * P1 + jj) * E] = sh * fma(hg, Pp[jj], PU[jj]);
        rb[(2 * P1 + jj) * E] = sh * PV[jj];
      } else {
        rb[(0 * P1 + jj) * E] = sh * tV[jj];
        rb[(1 * P1 + jj) * E] = sh * PU[jj];
        rb[(2 * P1 + jj) * E] = sh * fma(hg, Pp[jj], PV[jj]);
      }
    });
  }
  sfor<0, P1>([&](auto j) {
    constexpr int jj = CV(j);
    rb[(3 * P1 + jj) * E] = tx[jj];
    rb[(4 * P1 + jj) * E] = tU[jj];
    rb[(5 * P1 + jj) * E] = tV[jj];
  });
  // wave speed of this side at s = 0, 1/2, 1 (|u.n| is sign-free)
  const Real h0 = edge_point<P, 0>(Hs), h1 = edge_point<P, 1>(Hs), h2 = edge_point<P, 2>(Hs);
  const Real u0 = edge_point<P, 0>(un), u1 = edge_point<P, 1>(un), u2 = edge_point<P, 2>(un);
  if (!(h0 > Real(0)) || !(h1 > Real(0)) || !(h2 > Real(0))) err |= ERRF_DRY;
  const Real l0 = fabs(u0) + sqrt(sp.g * h0);
  const Real l1 = fabs(u1) + sqrt(sp.g * h1);
  const Real l2 = fabs(u2) + sqrt(sp.g * h2);
  rb[(6 * P1) * E] = fmax(fmax(l0, l1), l2);
}

// Evaluation of one element's state: velocity projection, volume + source
// integrals -> vs_out, side records -> rec_out; returns the element wave
// speed |q_bar/H_bar| + sqrt(g H_bar) from the means (mean = sqrt(2) c_1).
template <int P, class Real, class PR>
__device__ __forceinline__ double evaluate(const StageParams<Real>& sp, long long e, int t, const Real* xi,
                                           const Real* U, const Real* V, unsigned& err) {
  using D = Dims<P>;
  constexpr int K = D::K, K1 = D::K1;
  const long long E = sp.m.E;
  Real hb[K], H[K], u[K], v[K];
  sfor<0, K>([&](auto i) {
    hb[CV(i)] = sp.hb[CV(i) * E + e];
    H[CV(i)] = xi[CV(i)] + hb[CV(i)];
  });
  if (!project_velocity<P, PR>(H, U, V, u, v)) err |= ERRF_DRY;

  // volume integrals (A~, grad phi_a) (Eqs. (15)-(16)): grad phi_a lies in
  // P^{p-1}, so only the first K1 coefficients of each projected product count
  Real xe[K];
  sfor<0, K>([&](auto i) { xe[CV(i)] = fma(Real(2), hb[CV(i)], xi[CV(i)]); });
  Real Puu[K1], Puv[K1], Pvu[K1], Pvv[K1], Pxx[K1];
  momentum_products<P>(U, V, u, v, Puu, Puv, Pvu, Pvv);
  tprod<P, K1, K>(xi, xe, Pxx);
  const Real hg = Real(0.5) * sp.g;
  Real FxU[K1], FyV[K1];
  sfor<0, K1>([&](auto i) {
    FxU[CV(i)] = fma(hg, Pxx[CV(i)], Puu[CV(i)]);
    FyV[CV(i)] = fma(hg, Pxx[CV(i)], Pvv[CV(i)]);
  });
  // source g xi grad h_b of Eq. (5): g sum_{i,m} T[a][i][m] xi_i ghb_m, with
  // ghb = det B * (coefficients of grad h_b), which live in P^{p-1}
  Real gx[K1], gy[K1];
  sfor<0, K1>([&](auto m) {
    gx[CV(m)] = sp.ghb[CV(m) * E + e];
    gy[CV(m)] = sp.ghb[(K1 + CV(m)) * E + e];
  });
  Real Sx[K], Sy[K];
  tprod<P, K, K1>(xi, gx, Sx);
  tprod<P, K, K1>(xi, gy, Sy);
  // adj(B)^T of the uniform mesh is diagonal: (hy, hx) lower, -(hy, hx) upper
  const Real sgn = t ? Real(-1) : Real(1);
  const Real G11 = sgn * Real(sp.m.hy), G22 = sgn * Real(sp.m.hx);
  sfor<0, K>([&](auto a) {
    constexpr int aa = CV(a);
    Real v0 = G11 * sdot_row<P, 0, aa>(U) + G22 * sdot_row<P, 1, aa>(V);
    Real v1 = G11 * sdot_row<P, 0, aa>(FxU) + G22 * sdot_row<P, 1, aa>(Puv);
    Real v2 = G11 * sdot_row<P, 0, aa>(Pvu) + G22 * sdot_row<P, 1, aa>(FyV);
    v1 = fma(sp.g, Sx[aa], v1);
    v2 = fma(sp.g, Sy[aa], v2);
    if (sp.tau_bf != 0.0 || sp.f_c != 0.0) {
      // (-tau_bf q + f_c (V, -U), phi_a) = |det B| (-tau_bf U_a + f_c V_a, ...)
      const Real tq = Real(-sp.tau_bf * sp.det), fq = Real(sp.f_c * sp.det);
      v1 = fma(tq, U[aa], fma(fq, V[aa], v1));
      v2 = fma(tq, V[aa], fma(-fq, U[aa], v2));
    }
    sp.vs_out[(0 * K + aa) * E + e] = v0;
    sp.vs_out[(1 * K + aa) * E + e] = v1;
    sp.vs_out[(2 * K + aa) * E + e] = v2;
  });
  side_record<0, P>(sp, e, t, xi, U, V, u, v, err);
  side_record<1, P>(sp, e, t, xi, U, V, u, v, err);
  side_record<2, P>(sp, e, t, xi, U, V, u, v, err);
  double lam_e = 0.0;
  if (sp.lam_next) {
    const double Hm = double(H[0]);
    const double um = double(U[0]) / Hm, vm = double(V[0]) / Hm;
    lam_e = sqrt(um * um + vm * vm) + sqrt(double(sp.g) * 1.4142135623730951 * Hm);
  }
  return lam_e;
}

// Numerical flux on local edge NN and its lift: res[f][a] -= sum_j R[NN][j][a] F^_f,j
// with F^ = |E| (1/2 (A~(c-) + A~(c+)).n + 1/2 lambda (c- - c+)) (Lax-Friedrichs).
template <int NN, int P, class Real>
__device__ __forceinline__ void edge_flux_lift(const StageParams<Real>& sp, long long e, int t,
                                               Real (&res)[3][Dims<P>::K]) {
  using D = Dims<P>;
  constexpr int P1 = D::P1, NREC = D::NREC;
  const long long E = sp.m.E;
  const Real* ro = sp.rec + (long long)NN * NREC * E + e;
  const long long f = neighbour(sp.m, e, NN);
  Real F[3][P1];
  if (f >= 0) {
    const Real* rn = sp.rec + (long long)NN * NREC * E + f;
    Real nx, ny, len;
    edge_geom(sp.m, t, NN, nx, ny, len);
    const Real lam = fmax(ro[(6 * P1) * E], rn[(6 * P1) * E]);
    const Real hl = Real(0.5) * len * lam;
    // the neighbour's polynomials run the other way (s -> 1 - s flips the sign
    // of odd Legendre modes) and its fluxes use the opposite normal
    sfor<0, 3>([&](auto ff) {
      constexpr int fv = CV(ff);
      sfor<0, P1>([&](auto j) {
        constexpr int jj = CV(j);
        constexpr bool odd = (jj & 1) != 0;
        const Real pm = ro[(fv * P1 + jj) * E], pp = rn[(fv * P1 + jj) * E];
        const Real wm = ro[((3 + fv) * P1 + jj) * E], wp = rn[((3 + fv) * P1 + jj) * E];
        const Real phi = odd ? pm + pp : pm - pp;
        const Real jmp = odd ? wm + wp : wm - wp;
        F[fv][jj] = fma(hl, jmp, phi);
      });
    });
  } else {
    // reflective wall, mirror ghost: F^(xi) = 0 and
    // F^(q) = |E| n (Pi(q.n u.n) + g/2 Pi(xi (xi + 2 h_b)) + lambda q.n)
    Real nx, ny, len;
    edge_geom(sp.m, t, NN, nx, ny, len);
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

template <class Real>
__device__ __forceinline__ bool finite(Real x) { return isfinite(x); }

// Work of one element in one launch: MODE_STAGE = flux, lift, RK update and
// evaluation of the new state; MODE_EVAL = evaluation only; MODE_RHS = flux
// and lift of an evaluated state, written as d_t c.  Returns the element's
// wave speed (0 unless sp.lam_next is set) through lam_e.
template <int P, class Real, class PR, int MODE>
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
  if constexpr (MODE == MODE_EVAL) {
    lam_e = evaluate<P, Real, PR>(sp, e, t, w[0], w[1], w[2], err);
  } else {
    Real res[3][K];
    sfor<0, 3>([&](auto f) {
      sfor<0, K>([&](auto i) { res[CV(f)][CV(i)] = sp.vs[(CV(f) * K + CV(i)) * E + e]; });
    });
    edge_flux_lift<0, P>(sp, e, t, res);
    edge_flux_lift<1, P>(sp, e, t, res);
    edge_flux_lift<2, P>(sp, e, t, res);
    if constexpr (MODE == MODE_RHS) {
      const Real idet = Real(sp.inv_det);
      sfor<0, 3>([&](auto f) {
        sfor<0, K>([&](auto i) { sp.rhs_out[(CV(f) * K + CV(i)) * E + e] = res[CV(f)][CV(i)] * idet; });
      });
    } else {
      // w' = alpha w0 + beta (w + dt R),  R = res / |det B|, alpha + beta = 1,
      // evaluated as w0 + beta ((w - w0) + dt R): a constant state stays
      // exactly constant and the result is rounded once (alpha and beta
      // themselves are never rounded to the working precision)
      const Real b = Real(sp.beta), c = Real(dt * sp.inv_det);
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
      lam_e = evaluate<P, Real, PR>(sp, e, t, w[0], w[1], w[2], err);
    }
  }
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
// per right-hand side (MODE_RHS).  One thread per element.
template <int P, class Real, class PR, int MODE>
__global__ void __launch_bounds__(128) stage_kernel(const StageParams<Real> sp) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double lam_e = 0.0;
  unsigned err = 0;
  double dt = 0.0;
  if constexpr (MODE == MODE_STAGE) {
    dt = sp.dt_fixed > 0.0 ? sp.dt_fixed : sp.cfl_num / sp.lam[0];
  }
  if (e < sp.m.E) stage_element<P, Real, PR, MODE>(sp, e, dt, lam_e, err);
  if (sp.lam_next) {
    const double l = block_max(lam_e);
    if (threadIdx.x == 0) atomic_max_nonneg(sp.lam_next, l);
  }
  if (err) atomicOr(sp.err, err);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (sp.lam_clear) *sp.lam_clear = 0.0;
    if (sp.t) *sp.t += dt;
  }
}

// Static per-element fields of the bathymetry: edge traces and the
// det-scaled gradient coefficients  ghb_r = G_rr * (d^_r h_b) (uniform mesh).
template <int P, class Real>
__global__ void static_kernel(Mesh m, const double* __restrict__ hb64, Real* hb, Real* hbt, Real* ghb) {
  using D = Dims<P>;
  using Tb = RefTables<P>;
  constexpr int K = D::K, P1 = D::P1, K1 = D::K1;
  const long long E = m.E;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const int t = (int)(e & 1);
  double h[K];
  sfor<0, K>([&](auto i) {
    h[CV(i)] = hb64[CV(i) * E + e];
    hb[CV(i) * E + e] = Real(h[CV(i)]);
  });
  auto tr = [&](auto nn) {
    double tau[P1];
    trace<CV(nn), P>(h, tau);
    sfor<0, P1>([&](auto j) { hbt[(CV(nn) * P1 + CV(j)) * E + e] = Real(tau[CV(j)]); });
  };
  sfor<0, 3>(tr);
  const double sgn = t ? -1.0 : 1.0;
  const double G[2] = {sgn * m.hy, sgn * m.hx};
  sfor<0, 2>([&](auto r) {
    sfor<0, K1>([&](auto mm) {
      double acc = 0.0;
      sfor<0, K>([&](auto i) {
        constexpr double s = Tb::S[CV(r)][CV(i)][CV(mm)];
        if constexpr (s != 0.0) acc = fma(s, h[CV(i)], acc);
      });
      ghb[(CV(r) * K1 + CV(mm)) * E + e] = Real(G[CV(r)] * acc);
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
