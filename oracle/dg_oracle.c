/*
 * dg_oracle.c -- plain FP64 CPU reference for the quadrature-free DG
 * discretisation of the 2D shallow water equations (arXiv:1904.08684).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file:
 * only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark load it.  It shares no code, table or helper with the CUDA path.
 *
 * What it computes (paper §2.2): the semi-discrete DG system, discrete weak
 * form Eqs. (11)-(12) ("variational_disc_1/2"):
 *     (d_t c, phi)_e - (A~(c,u), grad phi)_e + <A^(c,u,c+,u+,n), phi>_de
 *         = (r(c), phi)_e,                         c = (xi, U, V)
 *     (u H, psi)_e = (q, psi)_e,                   u = (u, v), H = xi + h_b
 * with the flux A~ of Eq. (8) and the source r of Eq. (5).  The paper
 * evaluates every integral of polynomials exactly ("quadrature-free", §1 and
 * §2.2); this oracle therefore evaluates the same integrals with Gauss rules
 * that are exact for the polynomial degrees involved (3p for every
 * integrand), pointwise, in physical coordinates.  It never forms the
 * reference triple-product tensors, edge-restriction matrices or the
 * orientation sign rule that the fast path uses, and it never assumes the
 * basis is orthonormal (mass matrices are assembled and Cholesky-factored).
 *
 * Readings of the paper where it is silent or garbled:
 *  - basis phi_ei = phi^_i o F_e^-1 (§2.2, below Eq. (14)); the mass matrix is
 *    then |det B_e| I for the printed orthonormal basis;
 *  - vertices of every triangle are counter-clockwise so det B_e > 0;
 *  - degree-4 functions (p = 4) = Gram-Schmidt of x^4, x^3y, x^2y^2, xy^3, y^4
 *    against the ten printed functions;
 *  - Lax-Friedrichs flux (§2.2, after Eq. (12)):
 *        A^ = 1/2 (A~(c-)n + A~(c+)n) + 1/2 lambda (c- - c+),
 *    lambda = max over both sides and the edge points s = 0, 1/2, 1 of
 *    |u.n| + sqrt(g H)  (one constant per edge);
 *  - reflective wall ghost: xi+ = xi-, hb+ = hb-, q+ = q- - 2 (q-.n) n and
 *    likewise for u; periodic: quads wrap modulo nx, ny;
 *  - time stepping (not stated; §3.1 gives only a fixed dt): SSP Runge-Kutta
 *    of order 1, 2, 3 in Shu-Osher form; dt either fixed or
 *    cfl * d_min / ((2p+1) max_e lambda_e), lambda_e from element means,
 *    d_min the smallest inscribed-circle diameter.
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXK 15
#define OR_MAXQ1 16

enum { OR_OK = 0, OR_ERR_ARG = 1, OR_ERR_DRY = 5, OR_ERR_NONFINITE = 6 };
enum { OR_BC_PERIODIC = 0, OR_BC_REFLECTIVE = 1, OR_BC_DIRICHLET = 2 };

typedef struct {
  int nx, ny;
  double x0, y0, Lx, Ly;
  const double* vertex_xy; /* optional (nx+1)*(ny+1)*2, row j major */
  int p;
  double g;
  int bc;
  int rk_order;
  double cfl, dt;
  double tau_bf, f_c; /* bottom friction and Coriolis of Eq. (2), default 0 */
  int manufactured;   /* 1: §3.1 analytic solution supplies forcing F and
                         Dirichlet boundary data */
  int quad_extra;     /* extra Gauss points per direction (exactness checks) */
} or_config;

/* ---------------------------------------------------------------------- */
/* Polynomials on the reference triangle as monomial tables c[a][b] x^a y^b */
typedef struct { double c[5][5]; } poly2;

static double poly_eval(const poly2* P, double x, double y) {
  double s = 0.0, xa = 1.0;
  for (int a = 0; a < 5; ++a) {
    double yb = 1.0;
    for (int b = 0; a + b < 5; ++b) {
      s += P->c[a][b] * xa * yb;
      yb *= y;
    }
    xa *= x;
  }
  return s;
}
static double poly_dx(const poly2* P, double x, double y) {
  double s = 0.0, xa = 1.0;
  for (int a = 1; a < 5; ++a) {
    double yb = 1.0;
    for (int b = 0; a + b < 5; ++b) {
      s += a * P->c[a][b] * xa * yb;
      yb *= y;
    }
    xa *= x;
  }
  return s;
}
static double poly_dy(const poly2* P, double x, double y) {
  double s = 0.0, xa = 1.0;
  for (int a = 0; a < 5; ++a) {
    double yb = 1.0;
    for (int b = 1; a + b < 5; ++b) {
      s += b * P->c[a][b] * xa * yb;
      yb *= y;
    }
    xa *= x;
  }
  return s;
}

/* ---------------------------------------------------------------------- */
/* Gauss-Legendre rule on [0,1] by Newton iteration on P_n (no tables).    */
static void gauss_legendre01(int n, double* s, double* w) {
  for (int i = 0; i < n; ++i) {
    double x = cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (x * p1 - p0) / (x * x - 1.0);
      double dx = p1 / dp;
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (x * p1 - p0) / (x * x - 1.0);
    }
    s[i] = 0.5 * (1.0 - x);
    w[i] = 1.0 / ((1.0 - x * x) * dp * dp);
  }
}

/* Collapsed (Duffy) rule on the reference triangle {x,y>=0, x+y<=1}:
 * x = a, y = (1-a) b, weight w_a w_b (1-a); exact for total degree <= 2n-2. */
typedef struct { int n; double x[OR_MAXQ1 * OR_MAXQ1], y[OR_MAXQ1 * OR_MAXQ1], w[OR_MAXQ1 * OR_MAXQ1]; } tri_rule;

static void make_tri_rule(int n, tri_rule* R) {
  double s[OR_MAXQ1], w[OR_MAXQ1];
  gauss_legendre01(n, s, w);
  R->n = n * n;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      int q = i * n + j;
      R->x[q] = s[i];
      R->y[q] = (1.0 - s[i]) * s[j];
      R->w[q] = w[i] * w[j] * (1.0 - s[i]);
    }
}

/* ---------------------------------------------------------------------- */
/* The reference basis printed in §2.2 (functions 1..10, orders 0..3).     */
static void set_printed_basis(poly2* B) {
  memset(B, 0, sizeof(poly2) * 10);
  double r;
  B[0].c[0][0] = sqrt(2.0);                                        /* phi_1 */
  B[1].c[0][0] = 2.0; B[1].c[1][0] = -6.0;                         /* phi_2 */
  r = sqrt(12.0);                                                  /* phi_3 */
  B[2].c[0][0] = r; B[2].c[1][0] = -r; B[2].c[0][1] = -2.0 * r;
  r = sqrt(6.0);                                                   /* phi_4 */
  B[3].c[0][0] = r; B[3].c[1][0] = -8.0 * r; B[3].c[2][0] = 10.0 * r;
  r = sqrt(3.0);                                                   /* phi_5 */
  B[4].c[0][0] = -r; B[4].c[1][0] = -4.0 * r; B[4].c[2][0] = 5.0 * r;
  B[4].c[0][1] = 12.0 * r; B[4].c[0][2] = -15.0 * r;
  r = sqrt(45.0);                                                  /* phi_6 */
  B[5].c[0][0] = r; B[5].c[1][0] = -4.0 * r; B[5].c[2][0] = 3.0 * r;
  B[5].c[0][1] = -4.0 * r; B[5].c[1][1] = 8.0 * r; B[5].c[0][2] = 3.0 * r;
  r = sqrt(8.0);                                                   /* phi_7 */
  B[6].c[0][0] = -r; B[6].c[1][0] = 15.0 * r; B[6].c[2][0] = -45.0 * r;
  B[6].c[3][0] = 35.0 * r;
  r = sqrt(24.0);                                                  /* phi_8 */
  B[7].c[0][0] = -r; B[7].c[1][0] = 13.0 * r; B[7].c[2][0] = -33.0 * r;
  B[7].c[3][0] = 21.0 * r; B[7].c[0][1] = 2.0 * r; B[7].c[1][1] = -24.0 * r;
  B[7].c[2][1] = 42.0 * r;
  r = sqrt(40.0);                                                  /* phi_9 */
  B[8].c[0][0] = -r; B[8].c[1][0] = 9.0 * r; B[8].c[2][0] = -15.0 * r;
  B[8].c[3][0] = 7.0 * r; B[8].c[0][1] = 6.0 * r; B[8].c[1][1] = -48.0 * r;
  B[8].c[2][1] = 42.0 * r; B[8].c[0][2] = -6.0 * r; B[8].c[1][2] = 42.0 * r;
  r = sqrt(56.0);                                                  /* phi_10 */
  B[9].c[0][0] = -r; B[9].c[1][0] = 3.0 * r; B[9].c[2][0] = -3.0 * r;
  B[9].c[3][0] = r; B[9].c[0][1] = 12.0 * r; B[9].c[1][1] = -24.0 * r;
  B[9].c[2][1] = 12.0 * r; B[9].c[0][2] = -30.0 * r; B[9].c[1][2] = 30.0 * r;
  B[9].c[0][3] = 20.0 * r;
}

/* Degree-4 completion (p = 4 is beyond the printed basis): modified
 * Gram-Schmidt of x^4, x^3y, x^2y^2, xy^3, y^4 against the previous
 * functions, inner products by a rule exact for degree 8. */
static double tri_inner(const poly2* A, const poly2* B, const tri_rule* R) {
  double s = 0.0;
  for (int q = 0; q < R->n; ++q) s += R->w[q] * poly_eval(A, R->x[q], R->y[q]) * poly_eval(B, R->x[q], R->y[q]);
  return s;
}
static void set_degree4_basis(poly2* B) {
  tri_rule R;
  make_tri_rule(7, &R);
  for (int k = 0; k < 5; ++k) {
    poly2 m;
    memset(&m, 0, sizeof m);
    m.c[4 - k][k] = 1.0;
    for (int j = 0; j < 10 + k; ++j) {
      double h = tri_inner(&m, &B[j], &R);
      for (int a = 0; a < 5; ++a)
        for (int b = 0; b < 5; ++b) m.c[a][b] -= h * B[j].c[a][b];
    }
    double nrm = sqrt(tri_inner(&m, &m, &R));
    for (int a = 0; a < 5; ++a)
      for (int b = 0; b < 5; ++b) m.c[a][b] /= nrm;
    B[10 + k] = m;
  }
}

/* ---------------------------------------------------------------------- */
typedef struct {
  or_config cfg;
  int K, E;
  int Kb;            /* bathymetry functions: K(max(p, 1)) */
  poly2 basis[OR_MAXK];
  tri_rule vol;      /* exact for degree 3p (plus margin) */
  tri_rule proj;     /* rule for projecting non-polynomial data */
  int ne;            /* edge rule points */
  double es[OR_MAXQ1], ew[OR_MAXQ1];
  double* vx;        /* (nx+1)*(ny+1) vertex coordinates */
  double* vy;
  /* per element geometry */
  double* ax;        /* 3 vertices */
  double* ay;
  double* B;         /* 4: B11 B12 B21 B22 */
  double* det;
  int* nb;           /* 3 neighbours, -1 on a wall */
  double* shx;       /* 3 periodic shifts: neighbour frame = x + shift */
  double* shy;
  double dmin;
  int threads;
} or_ctx;

static int nthreads(const or_ctx* h) {
#ifdef _OPENMP
  return h->threads > 0 ? h->threads : omp_get_max_threads();
#else
  (void)h;
  return 1;
#endif
}

static int K_of(int p) { return (p + 1) * (p + 2) / 2; }

static void vertex(const or_ctx* h, int i, int j, double* x, double* y) {
  const int nx = h->cfg.nx;
  *x = h->vx[j * (nx + 1) + i];
  *y = h->vy[j * (nx + 1) + i];
}

/* Element numbering e = 2 (j nx + i) + t.  Lower triangle t = 0:
 * (v_ij, v_i+1j, v_ij+1); upper t = 1: (v_i+1j+1, v_ij+1, v_i+1j).  Both
 * counter-clockwise; local edge n is the edge opposite local vertex n:
 * edge 0 = a2->a3, edge 1 = a3->a1, edge 2 = a1->a2.  The diagonal of each
 * quad runs from v_i+1j to v_ij+1 (§2.3: two differently oriented triangles
 * per quad). */
static void build_mesh(or_ctx* h) {
  const int nx = h->cfg.nx, ny = h->cfg.ny;
  const int E = h->E;
  h->vx = malloc(sizeof(double) * (nx + 1) * (ny + 1));
  h->vy = malloc(sizeof(double) * (nx + 1) * (ny + 1));
  for (int j = 0; j <= ny; ++j)
    for (int i = 0; i <= nx; ++i) {
      int v = j * (nx + 1) + i;
      if (h->cfg.vertex_xy) {
        h->vx[v] = h->cfg.vertex_xy[2 * v];
        h->vy[v] = h->cfg.vertex_xy[2 * v + 1];
      } else {
        h->vx[v] = h->cfg.x0 + h->cfg.Lx * i / nx;
        h->vy[v] = h->cfg.y0 + h->cfg.Ly * j / ny;
      }
    }
  h->ax = malloc(sizeof(double) * 3 * E);
  h->ay = malloc(sizeof(double) * 3 * E);
  h->B = malloc(sizeof(double) * 4 * E);
  h->det = malloc(sizeof(double) * E);
  h->nb = malloc(sizeof(int) * 3 * E);
  h->shx = malloc(sizeof(double) * 3 * E);
  h->shy = malloc(sizeof(double) * 3 * E);
  const int periodic = h->cfg.bc == OR_BC_PERIODIC;
  double dmin = 1e300;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i)
      for (int t = 0; t < 2; ++t) {
        int e = 2 * (j * nx + i) + t;
        double x[3], y[3];
        if (t == 0) {
          vertex(h, i, j, &x[0], &y[0]);
          vertex(h, i + 1, j, &x[1], &y[1]);
          vertex(h, i, j + 1, &x[2], &y[2]);
        } else {
          vertex(h, i + 1, j + 1, &x[0], &y[0]);
          vertex(h, i, j + 1, &x[1], &y[1]);
          vertex(h, i + 1, j, &x[2], &y[2]);
        }
        for (int k = 0; k < 3; ++k) {
          h->ax[3 * e + k] = x[k];
          h->ay[3 * e + k] = y[k];
        }
        /* B_e = [a2 - a1, a3 - a1] (§2.2, affine map F_e) */
        double B11 = x[1] - x[0], B12 = x[2] - x[0];
        double B21 = y[1] - y[0], B22 = y[2] - y[0];
        h->B[4 * e + 0] = B11;
        h->B[4 * e + 1] = B12;
        h->B[4 * e + 2] = B21;
        h->B[4 * e + 3] = B22;
        h->det[e] = B11 * B22 - B12 * B21;
        double area = 0.5 * fabs(h->det[e]);
        double per = 0.0;
        for (int k = 0; k < 3; ++k) {
          int k1 = (k + 1) % 3;
          per += hypot(x[k1] - x[k], y[k1] - y[k]);
        }
        double d = 4.0 * area / per;
        if (d < dmin) dmin = d;
        /* neighbours: edge 0 <-> the other triangle of the quad; edge 1 <->
         * the quad to the left (t=0) / right (t=1); edge 2 <-> the quad
         * below (t=0) / above (t=1).  A neighbour's matching local edge has
         * the same index. */
        int ni[3], nj[3], nt = 1 - t;
        ni[0] = i; nj[0] = j;
        if (t == 0) { ni[1] = i - 1; nj[1] = j; ni[2] = i; nj[2] = j - 1; }
        else { ni[1] = i + 1; nj[1] = j; ni[2] = i; nj[2] = j + 1; }
        for (int n = 0; n < 3; ++n) {
          double sx = 0.0, sy = 0.0;
          int ii = ni[n], jj = nj[n];
          int wall = 0;
          if (ii < 0) { if (periodic) { ii += nx; sx = h->cfg.Lx; } else wall = 1; }
          if (ii >= nx) { if (periodic) { ii -= nx; sx = -h->cfg.Lx; } else wall = 1; }
          if (jj < 0) { if (periodic) { jj += ny; sy = h->cfg.Ly; } else wall = 1; }
          if (jj >= ny) { if (periodic) { jj -= ny; sy = -h->cfg.Ly; } else wall = 1; }
          h->nb[3 * e + n] = wall ? -1 : 2 * (jj * nx + ii) + nt;
          h->shx[3 * e + n] = sx;
          h->shy[3 * e + n] = sy;
        }
      }
  h->dmin = dmin;
}

/* map physical point to reference coordinates of element e: x^ = B^-1 (x - a1) */
static void to_ref(const or_ctx* h, int e, double x, double y, double* xr, double* yr) {
  const double* B = h->B + 4 * e;
  double dx = x - h->ax[3 * e], dy = y - h->ay[3 * e];
  double d = h->det[e];
  *xr = (B[3] * dx - B[1] * dy) / d;
  *yr = (-B[2] * dx + B[0] * dy) / d;
}

static double eval_field(const or_ctx* h, const double* coef, int e, double xr, double yr) {
  double s = 0.0;
  for (int i = 0; i < h->K; ++i) s += coef[e * h->K + i] * poly_eval(&h->basis[i], xr, yr);
  return s;
}

/* bathymetry lives in P^max(p,1): with p = 0 a piecewise-constant h_b would
 * drop the g xi grad h_b source of Eq. (5) entirely */
static double eval_hb(const or_ctx* h, const double* hb, int e, double xr, double yr) {
  double s = 0.0;
  for (int i = 0; i < h->Kb; ++i) s += hb[e * h->Kb + i] * poly_eval(&h->basis[i], xr, yr);
  return s;
}

/* physical gradient of basis function i at reference point: B^-T grad^ phi^ */
static void grad_phys(const or_ctx* h, int e, int i, double xr, double yr, double* gx, double* gy) {
  const double* B = h->B + 4 * e;
  double d = h->det[e];
  double g1 = poly_dx(&h->basis[i], xr, yr), g2 = poly_dy(&h->basis[i], xr, yr);
  *gx = (B[3] * g1 - B[2] * g2) / d;
  *gy = (-B[1] * g1 + B[0] * g2) / d;
}

/* Cholesky solve of the dense SPD n x n system A x = b (A overwritten).
 * Returns 0 if A is not positive definite. */
static int chol_solve(int n, double* A, double* b, int nrhs) {
  for (int j = 0; j < n; ++j) {
    double s = A[j * n + j];
    for (int k = 0; k < j; ++k) s -= A[j * n + k] * A[j * n + k];
    if (!(s > 0.0)) return 0;
    double l = sqrt(s);
    A[j * n + j] = l;
    for (int i = j + 1; i < n; ++i) {
      double t = A[i * n + j];
      for (int k = 0; k < j; ++k) t -= A[i * n + k] * A[j * n + k];
      A[i * n + j] = t / l;
    }
  }
  for (int r = 0; r < nrhs; ++r) {
    double* x = b + r * n;
    for (int i = 0; i < n; ++i) {
      double t = x[i];
      for (int k = 0; k < i; ++k) t -= A[i * n + k] * x[k];
      x[i] = t / A[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double t = x[i];
      for (int k = i + 1; k < n; ++k) t -= A[k * n + i] * x[k];
      x[i] = t / A[i * n + i];
    }
  }
  return 1;
}

/* ---------------------------------------------------------------------- */
/* §3.1 manufactured solution (C_a = C_t = 0.2, y_a = 0.3) and the body
 * force F that makes it satisfy Eq. (2) with tau_bf = f_c = 0.            */
static const double MS_CA = 0.2, MS_CT = 0.2, MS_YA = 0.3;

static void ms_state(double x, double y, double t, double* xi, double* U, double* V, double* hb) {
  double S = sin(M_PI * (x + y + MS_CT * t) / 600.0);
  *xi = 2.0 + MS_YA - 2.0 * MS_CA * S;
  *U = 2.0 * MS_YA + MS_CA * MS_CT * S;
  *V = MS_YA + MS_CA * MS_CT * S;
  *hb = 1.0 + x / 1000.0 + 2.0 * y / 1000.0;
}

static void ms_force(double x, double y, double t, double g, double* Fx, double* Fy) {
  double th = M_PI * (x + y + MS_CT * t) / 600.0;
  double S = sin(th), C = cos(th);
  double thx = M_PI / 600.0, tht = M_PI * MS_CT / 600.0;
  double xi = 2.0 + MS_YA - 2.0 * MS_CA * S;
  double U = 2.0 * MS_YA + MS_CA * MS_CT * S;
  double V = MS_YA + MS_CA * MS_CT * S;
  double hb = 1.0 + x / 1000.0 + 2.0 * y / 1000.0;
  double H = xi + hb;
  double xix = -2.0 * MS_CA * C * thx, xiy = xix;
  double Ux = MS_CA * MS_CT * C * thx, Uy = Ux, Ut = MS_CA * MS_CT * C * tht;
  double Vx = Ux, Vy = Ux, Vt = Ut;
  double Hx = xix + 1.0 / 1000.0, Hy = xiy + 2.0 / 1000.0;
  /* F = d_t q + div(q q^T / H) + g H grad xi */
  double dUU_dx = 2.0 * U * Ux / H - U * U * Hx / (H * H);
  double dUV_dy = (Uy * V + U * Vy) / H - U * V * Hy / (H * H);
  double dUV_dx = (Ux * V + U * Vx) / H - U * V * Hx / (H * H);
  double dVV_dy = 2.0 * V * Vy / H - V * V * Hy / (H * H);
  *Fx = Ut + dUU_dx + dUV_dy + g * H * xix;
  *Fy = Vt + dUV_dx + dVV_dy + g * H * xiy;
}

/* ---------------------------------------------------------------------- */
void* or_create(const or_config* cfg) {
  if (!cfg || cfg->nx < 1 || cfg->ny < 1 || cfg->p < 0 || cfg->p > 4) return NULL;
  if (cfg->bc == OR_BC_PERIODIC && (cfg->nx < 2 || cfg->ny < 2)) return NULL;
  or_ctx* h = calloc(1, sizeof(or_ctx));
  h->cfg = *cfg;
  h->cfg.vertex_xy = NULL;
  h->K = K_of(cfg->p);
  h->Kb = K_of(cfg->p > 1 ? cfg->p : 1);
  h->E = 2 * cfg->nx * cfg->ny;
  set_printed_basis(h->basis);
  if (cfg->p == 4) set_degree4_basis(h->basis);
  int p = cfg->p;
  int qe = cfg->quad_extra < 0 ? 0 : (cfg->quad_extra > 4 ? 4 : cfg->quad_extra);
  make_tri_rule((3 * p + 2 + 1) / 2 + 1 + qe, &h->vol);
  make_tri_rule(p + 6, &h->proj);
  h->ne = (3 * p + 1 + 1) / 2 + 1 + qe;
  gauss_legendre01(h->ne, h->es, h->ew);
  h->cfg.vertex_xy = cfg->vertex_xy;
  build_mesh(h);
  h->cfg.vertex_xy = NULL;
  h->threads = 0;
  return h;
}

void or_destroy(void* hv) {
  or_ctx* h = hv;
  if (!h) return;
  free(h->vx); free(h->vy); free(h->ax); free(h->ay); free(h->B); free(h->det);
  free(h->nb); free(h->shx); free(h->shy);
  free(h);
}

void or_set_threads(void* hv, int n) { ((or_ctx*)hv)->threads = n; }
/* threads the element loops run on (the set count, else OpenMP's default) */
int or_threads(void* hv) { return nthreads((or_ctx*)hv); }
int or_num_elems(void* hv) { return ((or_ctx*)hv)->E; }
int or_K(void* hv) { return ((or_ctx*)hv)->K; }
int or_Kb(void* hv) { return ((or_ctx*)hv)->Kb; }
double or_dmin(void* hv) { return ((or_ctx*)hv)->dmin; }

/* basis monomial tables, K x 5 x 5 (coefficient of x^a y^b at [i][a][b]) */
void or_basis_table(void* hv, double* out) {
  or_ctx* h = hv;
  for (int i = 0; i < h->K; ++i) memcpy(out + 25 * i, h->basis[i].c, sizeof(double) * 25);
}

/* per element: 3 vertices (x,y), det B, 3 neighbours, 3 shifts */
void or_geometry(void* hv, double* verts, double* det, int* nb) {
  or_ctx* h = hv;
  for (int e = 0; e < h->E; ++e) {
    for (int k = 0; k < 3; ++k) {
      verts[6 * e + 2 * k] = h->ax[3 * e + k];
      verts[6 * e + 2 * k + 1] = h->ay[3 * e + k];
      nb[3 * e + k] = h->nb[3 * e + k];
    }
    det[e] = h->det[e];
  }
}

/* value of field coef at physical (x, y) inside element e */
double or_eval_point(void* hv, const double* coef, int e, double x, double y) {
  or_ctx* h = hv;
  double xr, yr;
  to_ref(h, e, x, y, &xr, &yr);
  return eval_field(h, coef, e, xr, yr);
}

/* quadrature nodes for projecting point data: E x Q x 2 physical coords */
int or_num_proj_nodes(void* hv) { return ((or_ctx*)hv)->proj.n; }
static void proj_nodes_elem(const or_ctx* h, int e, double* xy) {
  const int Q = h->proj.n;
  const double* B = h->B + 4 * e;
  for (int q = 0; q < Q; ++q) {
    double xr = h->proj.x[q], yr = h->proj.y[q];
    xy[q * 2] = h->ax[3 * e] + B[0] * xr + B[1] * yr;
    xy[q * 2 + 1] = h->ay[3 * e] + B[2] * xr + B[3] * yr;
  }
}
void or_proj_nodes(void* hv, double* xy) {
  or_ctx* h = hv;
  for (int e = 0; e < h->E; ++e) proj_nodes_elem(h, e, xy + (size_t)e * h->proj.n * 2);
}
/* the same for the n listed elements only: n x Q x 2 */
void or_proj_nodes_sub(void* hv, const int* elems, int n, double* xy) {
  or_ctx* h = hv;
  for (int i = 0; i < n; ++i) proj_nodes_elem(h, elems[i], xy + (size_t)i * h->proj.n * 2);
}

/* L2 projection of point data (Q values at the element's or_proj_nodes) onto
 * the first nf basis functions: solve M c = (f, phi) with the quadrature mass
 * matrix of element e. */
static int project_elem(const or_ctx* h, int nf, int e, const double* vals, double* coef) {
  const int K = nf, Q = h->proj.n;
  double M[OR_MAXK * OR_MAXK], b[OR_MAXK];
  memset(M, 0, sizeof M);
  memset(b, 0, sizeof b);
  for (int q = 0; q < Q; ++q) {
    double phi[OR_MAXK];
    for (int i = 0; i < K; ++i) phi[i] = poly_eval(&h->basis[i], h->proj.x[q], h->proj.y[q]);
    double w = h->proj.w[q] * fabs(h->det[e]);
    for (int a = 0; a < K; ++a) {
      b[a] += w * vals[q] * phi[a];
      for (int c = 0; c < K; ++c) M[a * K + c] += w * phi[a] * phi[c];
    }
  }
  if (!chol_solve(K, M, b, 1)) return 0;
  for (int a = 0; a < K; ++a) coef[a] = b[a];
  return 1;
}

/* every element: vals E x Q, coef E x nf */
int or_project_n(void* hv, int nf, const double* vals, double* coef) {
  or_ctx* h = hv;
  if (nf < 1 || nf > OR_MAXK) return OR_ERR_ARG;
  const size_t Q = (size_t)h->proj.n;
  int ok = 1;
#pragma omp parallel for schedule(static) reduction(&& : ok) num_threads(nthreads(h))
  for (int e = 0; e < h->E; ++e)
    if (!project_elem(h, nf, e, vals + (size_t)e * Q, coef + (size_t)e * nf)) ok = 0;
  return ok ? OR_OK : OR_ERR_ARG;
}
int or_project(void* hv, const double* vals, double* coef) { return or_project_n(hv, ((or_ctx*)hv)->K, vals, coef); }
int or_project_hb(void* hv, const double* vals, double* coef) { return or_project_n(hv, ((or_ctx*)hv)->Kb, vals, coef); }

/* the n listed elements: vals n x Q; rows elems[i] of coef (E x nf) */
int or_project_sub(void* hv, int nf, const int* elems, int n, const double* vals, double* coef) {
  or_ctx* h = hv;
  if (nf < 1 || nf > OR_MAXK) return OR_ERR_ARG;
  const size_t Q = (size_t)h->proj.n;
  int ok = 1;
#pragma omp parallel for schedule(static) reduction(&& : ok) num_threads(nthreads(h))
  for (int i = 0; i < n; ++i)
    if (!project_elem(h, nf, elems[i], vals + (size_t)i * Q, coef + (size_t)elems[i] * nf)) ok = 0;
  return ok ? OR_OK : OR_ERR_ARG;
}

/* u-projection of Eq. (12) on one element: (u H, psi) = (q, psi). */
static int project_u_elem(const or_ctx* h, int e, const double* hb, const double* xi, const double* U,
                          const double* V, double* u, double* v) {
  const int K = h->K, Q = h->vol.n;
  double M[OR_MAXK * OR_MAXK], b[2 * OR_MAXK];
  memset(M, 0, sizeof M);
  memset(b, 0, sizeof b);
  const double ad = fabs(h->det[e]);
  for (int q = 0; q < Q; ++q) {
    double xr = h->vol.x[q], yr = h->vol.y[q];
    double phi[OR_MAXK];
    for (int i = 0; i < K; ++i) phi[i] = poly_eval(&h->basis[i], xr, yr);
    double H = eval_field(h, xi, e, xr, yr) + eval_hb(h, hb, e, xr, yr);
    double Uq = eval_field(h, U, e, xr, yr), Vq = eval_field(h, V, e, xr, yr);
    double w = h->vol.w[q] * ad;
    for (int a = 0; a < K; ++a) {
      b[a] += w * Uq * phi[a];
      b[K + a] += w * Vq * phi[a];
      for (int c = 0; c < K; ++c) M[a * K + c] += w * H * phi[a] * phi[c];
    }
  }
  if (!chol_solve(K, M, b, 2)) return 0;
  for (int a = 0; a < K; ++a) {
    u[e * K + a] = b[a];
    v[e * K + a] = b[K + a];
  }
  return 1;
}

int or_project_u(void* hv, const double* hb, const double* xi, const double* U, const double* V, double* u,
                 double* v) {
  or_ctx* h = hv;
  int ok = 1;
#pragma omp parallel for schedule(static) reduction(&& : ok) num_threads(nthreads(h))
  for (int e = 0; e < h->E; ++e)
    if (!project_u_elem(h, e, hb, xi, U, V, u, v)) ok = 0;
  return ok ? OR_OK : OR_ERR_DRY;
}

/* A~(c,u) . n for one point, Eq. (8) */
static void flux_n(double g, double xi, double U, double V, double u, double v, double hb, double nx, double ny,
                   double* f) {
  double H = xi + hb;
  double pr = 0.5 * g * xi * (H + hb);
  f[0] = U * nx + V * ny;
  f[1] = (U * u + pr) * nx + U * v * ny;
  f[2] = V * u * nx + (V * v + pr) * ny;
}

/* The traces of element e's fields on its local edge n at physical point
 * (x, y), and of the exterior state (neighbour, wall ghost or Dirichlet). */
typedef struct { double xi, U, V, u, v, hb; } pstate;

static void interior_state(const or_ctx* h, int e, double x, double y, const double* hb, const double* xi,
                           const double* U, const double* V, const double* u, const double* v, pstate* s) {
  double xr, yr;
  to_ref(h, e, x, y, &xr, &yr);
  s->xi = eval_field(h, xi, e, xr, yr);
  s->U = eval_field(h, U, e, xr, yr);
  s->V = eval_field(h, V, e, xr, yr);
  s->u = eval_field(h, u, e, xr, yr);
  s->v = eval_field(h, v, e, xr, yr);
  s->hb = eval_hb(h, hb, e, xr, yr);
}

static void exterior_state(const or_ctx* h, int e, int n, double x, double y, double t, double nx, double ny,
                           const pstate* in, const double* hb, const double* xi, const double* U, const double* V,
                           const double* u, const double* v, pstate* s) {
  int f = h->nb[3 * e + n];
  if (f >= 0) {
    interior_state(h, f, x + h->shx[3 * e + n], y + h->shy[3 * e + n], hb, xi, U, V, u, v, s);
    return;
  }
  if (h->cfg.manufactured || h->cfg.bc == OR_BC_DIRICHLET) {
    double hbx;
    ms_state(x, y, t, &s->xi, &s->U, &s->V, &hbx);
    s->hb = in->hb;
    double H = s->xi + s->hb;
    s->u = s->U / H;
    s->v = s->V / H;
    return;
  }
  /* reflective wall: mirror the normal component */
  double qn = in->U * nx + in->V * ny, un = in->u * nx + in->v * ny;
  s->xi = in->xi;
  s->hb = in->hb;
  s->U = in->U - 2.0 * qn * nx;
  s->V = in->V - 2.0 * qn * ny;
  s->u = in->u - 2.0 * un * nx;
  s->v = in->v - 2.0 * un * ny;
}

/* Right-hand side d_t c of one element (Eq. (11) solved with the mass
 * matrix).  u, v must hold the projected velocity of e and its neighbours.
 * Returns 0 on a non-positive depth in the wave-speed evaluation. */
static int rhs_elem(const or_ctx* h, int e, const double* hb, const double* xi, const double* U, const double* V,
                    const double* u, const double* v, double t, double* R0, double* R1, double* R2) {
  const int K = h->K;
  const double g = h->cfg.g;
  const double ad = fabs(h->det[e]);
  double res[3][OR_MAXK];
  memset(res, 0, sizeof res);
  /* volume: (A~, grad phi) + (r, phi) */
  for (int q = 0; q < h->vol.n; ++q) {
    double xr = h->vol.x[q], yr = h->vol.y[q];
    double w = h->vol.w[q] * ad;
    double Xi = eval_field(h, xi, e, xr, yr), Uq = eval_field(h, U, e, xr, yr), Vq = eval_field(h, V, e, xr, yr);
    double uq = eval_field(h, u, e, xr, yr), vq = eval_field(h, v, e, xr, yr), hbq = eval_hb(h, hb, e, xr, yr);
    double H = Xi + hbq;
    double pr = 0.5 * g * Xi * (H + hbq);
    double A[3][2] = {{Uq, Vq}, {Uq * uq + pr, Uq * vq}, {Vq * uq, Vq * vq + pr}};
    /* grad h_b from its polynomial */
    double hbx = 0.0, hby = 0.0;
    for (int i = 0; i < h->Kb; ++i) {
      double gx, gy;
      grad_phys(h, e, i, xr, yr, &gx, &gy);
      hbx += hb[e * h->Kb + i] * gx;
      hby += hb[e * h->Kb + i] * gy;
    }
    double r[3] = {0.0, g * Xi * hbx - h->cfg.tau_bf * Uq + h->cfg.f_c * Vq,
                   g * Xi * hby - h->cfg.tau_bf * Vq - h->cfg.f_c * Uq};
    if (h->cfg.manufactured) {
      double xp = h->ax[3 * e] + h->B[4 * e] * xr + h->B[4 * e + 1] * yr;
      double yp = h->ay[3 * e] + h->B[4 * e + 2] * xr + h->B[4 * e + 3] * yr;
      double Fx, Fy;
      ms_force(xp, yp, t, g, &Fx, &Fy);
      r[1] += Fx;
      r[2] += Fy;
    }
    for (int pp = 0; pp < K; ++pp) {
      double gx, gy;
      grad_phys(h, e, pp, xr, yr, &gx, &gy);
      double ph = poly_eval(&h->basis[pp], xr, yr);
      for (int w3 = 0; w3 < 3; ++w3) res[w3][pp] += w * (A[w3][0] * gx + A[w3][1] * gy + r[w3] * ph);
    }
  }
  /* edges: - <A^, phi> */
  for (int n = 0; n < 3; ++n) {
    int k1 = (n + 1) % 3, k2 = (n + 2) % 3;
    double Px = h->ax[3 * e + k1], Py = h->ay[3 * e + k1];
    double Qx = h->ax[3 * e + k2], Qy = h->ay[3 * e + k2];
    double len = hypot(Qx - Px, Qy - Py);
    double nx = (Qy - Py) / len, ny = -(Qx - Px) / len;
    /* lambda: max over both sides at s = 0, 1/2, 1 */
    double lam = 0.0;
    for (int k = 0; k < 3; ++k) {
      double s = 0.5 * k;
      double x = Px + s * (Qx - Px), y = Py + s * (Qy - Py);
      pstate a, b;
      interior_state(h, e, x, y, hb, xi, U, V, u, v, &a);
      exterior_state(h, e, n, x, y, t, nx, ny, &a, hb, xi, U, V, u, v, &b);
      double Ha = a.xi + a.hb, Hb = b.xi + b.hb;
      if (!(Ha > 0.0) || !(Hb > 0.0)) return 0;
      double la = fabs(a.u * nx + a.v * ny) + sqrt(g * Ha);
      double lb = fabs(b.u * nx + b.v * ny) + sqrt(g * Hb);
      if (la > lam) lam = la;
      if (lb > lam) lam = lb;
    }
    for (int q = 0; q < h->ne; ++q) {
      double s = h->es[q];
      double x = Px + s * (Qx - Px), y = Py + s * (Qy - Py);
      pstate a, b;
      interior_state(h, e, x, y, hb, xi, U, V, u, v, &a);
      exterior_state(h, e, n, x, y, t, nx, ny, &a, hb, xi, U, V, u, v, &b);
      double fa[3], fb[3];
      flux_n(g, a.xi, a.U, a.V, a.u, a.v, a.hb, nx, ny, fa);
      flux_n(g, b.xi, b.U, b.V, b.u, b.v, b.hb, nx, ny, fb);
      double ca[3] = {a.xi, a.U, a.V}, cb[3] = {b.xi, b.U, b.V};
      double xr, yr;
      to_ref(h, e, x, y, &xr, &yr);
      double w = h->ew[q] * len;
      for (int pp = 0; pp < K; ++pp) {
        double ph = poly_eval(&h->basis[pp], xr, yr);
        for (int w3 = 0; w3 < 3; ++w3) {
          double Fhat = 0.5 * (fa[w3] + fb[w3]) + 0.5 * lam * (ca[w3] - cb[w3]);
          res[w3][pp] -= w * Fhat * ph;
        }
      }
    }
  }
  /* mass matrix by quadrature and solve */
  double M[OR_MAXK * OR_MAXK];
  memset(M, 0, sizeof M);
  for (int q = 0; q < h->vol.n; ++q) {
    double phi[OR_MAXK];
    for (int i = 0; i < K; ++i) phi[i] = poly_eval(&h->basis[i], h->vol.x[q], h->vol.y[q]);
    for (int a = 0; a < K; ++a)
      for (int c = 0; c < K; ++c) M[a * K + c] += h->vol.w[q] * ad * phi[a] * phi[c];
  }
  double rhs[3 * OR_MAXK];
  for (int w3 = 0; w3 < 3; ++w3)
    for (int pp = 0; pp < K; ++pp) rhs[w3 * K + pp] = res[w3][pp];
  chol_solve(K, M, rhs, 3);
  for (int pp = 0; pp < K; ++pp) {
    R0[e * K + pp] = rhs[pp];
    R1[e * K + pp] = rhs[K + pp];
    R2[e * K + pp] = rhs[2 * K + pp];
  }
  return 1;
}

/* RHS for all elements, or for the listed ones (elems != NULL).  u and v are
 * projected where needed (listed elements and their neighbours). */
int or_rhs(void* hv, const double* hb, const double* xi, const double* U, const double* V, double t,
           const int* elems, int nelem, double* R0, double* R1, double* R2) {
  or_ctx* h = hv;
  const int E = h->E, K = h->K;
  double* u = calloc((size_t)E * K, sizeof(double));
  double* v = calloc((size_t)E * K, sizeof(double));
  int ok = 1;
  if (!elems) {
#pragma omp parallel for schedule(static) reduction(&& : ok) num_threads(nthreads(h))
    for (int e = 0; e < E; ++e)
      if (!project_u_elem(h, e, hb, xi, U, V, u, v)) ok = 0;
    if (ok) {
#pragma omp parallel for schedule(static) reduction(&& : ok) num_threads(nthreads(h))
      for (int e = 0; e < E; ++e)
        if (!rhs_elem(h, e, hb, xi, U, V, u, v, t, R0, R1, R2)) ok = 0;
    }
  } else {
    char* need = calloc(E, 1);
    for (int k = 0; k < nelem; ++k) {
      int e = elems[k];
      if (e < 0 || e >= E) { ok = 0; continue; }
      need[e] = 1;
      for (int n = 0; n < 3; ++n)
        if (h->nb[3 * e + n] >= 0) need[h->nb[3 * e + n]] = 1;
    }
    if (ok) {
#pragma omp parallel for schedule(static) reduction(&& : ok) num_threads(nthreads(h))
      for (int e = 0; e < E; ++e)
        if (need[e] && !project_u_elem(h, e, hb, xi, U, V, u, v)) ok = 0;
    }
    if (ok) {
#pragma omp parallel for schedule(static) reduction(&& : ok) num_threads(nthreads(h))
      for (int k = 0; k < nelem; ++k)
        if (!rhs_elem(h, elems[k], hb, xi, U, V, u, v, t, R0, R1, R2)) ok = 0;
    }
    free(need);
  }
  free(u);
  free(v);
  return ok ? OR_OK : OR_ERR_DRY;
}

/* element means (by quadrature) -> lambda_e = |u_bar| + sqrt(g H_bar) */
double or_max_wave_speed(void* hv, const double* hb, const double* xi, const double* U, const double* V) {
  or_ctx* h = hv;
  double lmax = 0.0;
  for (int e = 0; e < h->E; ++e) {
    double sH = 0.0, sU = 0.0, sV = 0.0, sw = 0.0;
    for (int q = 0; q < h->vol.n; ++q) {
      double xr = h->vol.x[q], yr = h->vol.y[q], w = h->vol.w[q];
      sH += w * (eval_field(h, xi, e, xr, yr) + eval_hb(h, hb, e, xr, yr));
      sU += w * eval_field(h, U, e, xr, yr);
      sV += w * eval_field(h, V, e, xr, yr);
      sw += w;
    }
    double Hm = sH / sw, um = sU / sH, vm = sV / sH;
    double l = sqrt(um * um + vm * vm) + sqrt(h->cfg.g * Hm);
    if (l > lmax) lmax = l;
  }
  return lmax;
}

double or_cfl_dt(void* hv, const double* hb, const double* xi, const double* U, const double* V) {
  or_ctx* h = hv;
  double lmax = or_max_wave_speed(hv, hb, xi, U, V);
  return h->cfg.cfl * h->dmin / ((2.0 * h->cfg.p + 1.0) * lmax);
}

/* SSP Runge-Kutta in Shu-Osher form: stage s computes
 *   w_{s+1} = alpha_s w_0 + beta_s (w_s + dt R(w_s)),
 * RK1: (0,1); RK2: (0,1), (1/2,1/2); RK3: (0,1), (3/4,1/4), (1/3,2/3).
 * Stage times: RK2 t, t+dt; RK3 t, t+dt, t+dt/2. */
int or_run(void* hv, const double* hb, double* xi, double* U, double* V, int nsteps, double* t_io,
           double* dt_last) {
  or_ctx* h = hv;
  const size_t N = (size_t)h->E * h->K;
  const int S = h->cfg.rk_order;
  static const double al[3][3] = {{0, 0, 0}, {0, 0.5, 0}, {0, 0.75, 1.0 / 3.0}};
  static const double be[3][3] = {{1, 0, 0}, {1, 0.5, 0}, {1, 0.25, 2.0 / 3.0}};
  static const double ct[3][3] = {{0, 0, 0}, {0, 1, 0}, {0, 1, 0.5}};
  if (S < 1 || S > 3) return OR_ERR_ARG;
  double* w0 = malloc(3 * N * sizeof(double));
  double* ws = malloc(3 * N * sizeof(double));
  double* R = malloc(3 * N * sizeof(double));
  double t = *t_io;
  int st = OR_OK;
  for (int step = 0; step < nsteps && st == OR_OK; ++step) {
    double dt = h->cfg.dt > 0 ? h->cfg.dt : or_cfl_dt(hv, hb, xi, U, V);
    if (dt_last) *dt_last = dt;
    memcpy(w0, xi, N * sizeof(double));
    memcpy(w0 + N, U, N * sizeof(double));
    memcpy(w0 + 2 * N, V, N * sizeof(double));
    memcpy(ws, w0, 3 * N * sizeof(double));
    for (int s = 0; s < S; ++s) {
      st = or_rhs(hv, hb, ws, ws + N, ws + 2 * N, t + ct[S - 1][s] * dt, NULL, 0, R, R + N, R + 2 * N);
      if (st != OR_OK) break;
      double a = al[S - 1][s], b = be[S - 1][s];
      for (size_t k = 0; k < 3 * N; ++k) ws[k] = a * w0[k] + b * (ws[k] + dt * R[k]);
    }
    if (st != OR_OK) break;
    for (size_t k = 0; k < 3 * N; ++k)
      if (!isfinite(ws[k])) { st = OR_ERR_NONFINITE; break; }
    memcpy(xi, ws, N * sizeof(double));
    memcpy(U, ws + N, N * sizeof(double));
    memcpy(V, ws + 2 * N, N * sizeof(double));
    t += dt;
  }
  *t_io = t;
  free(w0);
  free(ws);
  free(R);
  return st;
}

/* mass = integral of xi; energy = 1/2 integral of (g xi^2 + U u + V v) */
int or_diagnostics(void* hv, const double* hb, const double* xi, const double* U, const double* V, double* mass,
                   double* energy) {
  or_ctx* h = hv;
  const int E = h->E, K = h->K;
  double* u = malloc(sizeof(double) * E * K);
  double* v = malloc(sizeof(double) * E * K);
  int st = or_project_u(hv, hb, xi, U, V, u, v);
  double* me = malloc(sizeof(double) * E);
  double* ee = malloc(sizeof(double) * E);
#pragma omp parallel for schedule(static) num_threads(nthreads(h))
  for (int e = 0; e < E; ++e) {
    double m = 0.0, en = 0.0, ad = fabs(h->det[e]);
    for (int q = 0; q < h->vol.n; ++q) {
      double xr = h->vol.x[q], yr = h->vol.y[q], w = h->vol.w[q] * ad;
      double X = eval_field(h, xi, e, xr, yr);
      m += w * X;
      en += 0.5 * w *
            (h->cfg.g * X * X + eval_field(h, U, e, xr, yr) * eval_field(h, u, e, xr, yr) +
             eval_field(h, V, e, xr, yr) * eval_field(h, v, e, xr, yr));
    }
    me[e] = m;
    ee[e] = en;
  }
  double M = 0.0, En = 0.0;
  for (int e = 0; e < E; ++e) {
    M += me[e];
    En += ee[e];
  }
  *mass = M;
  *energy = En;
  free(u); free(v); free(me); free(ee);
  return st;
}

/* §3.1: L2 errors of xi, U, V against the manufactured solution at time t */
void or_ms_errors(void* hv, const double* xi, const double* U, const double* V, double t, double* err) {
  or_ctx* h = hv;
  double s[3] = {0, 0, 0};
  for (int e = 0; e < h->E; ++e) {
    double ad = fabs(h->det[e]);
    const double* B = h->B + 4 * e;
    for (int q = 0; q < h->proj.n; ++q) {
      double xr = h->proj.x[q], yr = h->proj.y[q], w = h->proj.w[q] * ad;
      double x = h->ax[3 * e] + B[0] * xr + B[1] * yr, y = h->ay[3 * e] + B[2] * xr + B[3] * yr;
      double ex[3], hbx;
      ms_state(x, y, t, &ex[0], &ex[1], &ex[2], &hbx);
      double d0 = eval_field(h, xi, e, xr, yr) - ex[0];
      double d1 = eval_field(h, U, e, xr, yr) - ex[1];
      double d2 = eval_field(h, V, e, xr, yr) - ex[2];
      s[0] += w * d0 * d0;
      s[1] += w * d1 * d1;
      s[2] += w * d2 * d2;
    }
  }
  for (int k = 0; k < 3; ++k) err[k] = sqrt(s[k]);
}

/* §3.1 manufactured state and force at points, for pins */
void or_ms_point(double x, double y, double t, double g, double* out) {
  ms_state(x, y, t, &out[0], &out[1], &out[2], &out[3]);
  ms_force(x, y, t, g, &out[4], &out[5]);
}
