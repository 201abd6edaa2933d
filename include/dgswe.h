/*
 * dgswe.h -- C-ABI of libdgswe, a GB300 (sm_103a) implementation of the
 * explicit right-hand side and Runge-Kutta stage update of the
 * quadrature-free discontinuous Galerkin scheme for the 2D shallow water
 * equations of Hajduk, Kuckuk et al., arXiv:1904.08684.
 *
 * Method (paper §2.1-2.2):
 *   unknowns c = (xi, U, V) (surface elevation, discharge q = (U, V)), with
 *   total depth H = xi + h_b; the velocity u = q/H is a second DG field
 *   obtained element by element from (u H, psi) = (q, psi)  (Eq. (12));
 *   the flux A~ of Eq. (8) is then polynomial, so every integral of the weak
 *   form Eq. (11) is evaluated exactly from precomputed reference tensors;
 *   the numerical flux is Lax-Friedrichs with one wave speed per edge,
 *   lambda = max over both sides and the points s = 0, 1/2, 1 of
 *   |u.n| + sqrt(g H).
 * Mesh (paper §2.3): nx x ny quads over [x0, x0+Lx] x [y0, y0+Ly], each split
 *   into two triangles along the diagonal from vertex (i+1, j) to (i, j+1);
 *   element e = 2 (j nx + i) + t, t = 0 lower triangle (v_ij, v_i+1j,
 *   v_ij+1), t = 1 upper triangle (v_i+1j+1, v_ij+1, v_i+1j), both
 *   counter-clockwise so det B_e > 0.
 * Basis (paper §2.2): on element e, phi_ei = phi^_i o F_e^-1 with the
 *   orthonormal reference functions printed in §2.2 (K = 1, 3, 6, 10 for
 *   p = 0, 1, 2, 3); p = 4 continues them by Gram-Schmidt of x^4, x^3 y,
 *   x^2 y^2, x y^3, y^4 (K = 15).  The mass matrix is |det B_e| I.  The
 *   bathymetry h_b is a DG field of order max(p, 1).
 * Time stepping (not stated in the paper; §3.1 uses a fixed dt): SSP
 *   Runge-Kutta of order 1, 2 or 3 in Shu-Osher form; dt either fixed or
 *   cfl * d_min / ((2p+1) max_e (|u_e| + sqrt(g H_e))) with element means and
 *   d_min the smallest inscribed-circle diameter, evaluated on the device at
 *   the start of every step.
 *
 * Conventions for every entry point:
 *   - Host arrays are FP64, element-major ("AoS"): coefficient i of element e
 *     at [e * K + i].  The caller owns them; the library copies what it needs.
 *   - Device arrays are structure-of-arrays ("SoA"): field f, coefficient i,
 *     element e at [(f * K + i) * E + e], in the context's precision (double
 *     for DG_PREC_FP64, float for DG_PREC_FP32_MIXED).  The caller owns device
 *     arrays it passes in; the library owns the buffers it allocates until
 *     dg_destroy.
 *   - All device work is ordered on the stream given to dg_init (NULL = the
 *     legacy default stream).  Entry points that return host data
 *     synchronise that stream.
 *   - A context or batch is used by one host thread at a time; distinct
 *     contexts are independent of each other.
 *   - No C++ exception crosses this boundary; every failure is a dg_status
 *     (a failed host allocation is DG_ERR_OOM, like a device one).
 *     After DG_ERR_DRY or DG_ERR_NONFINITE the context stays valid so the
 *     state can be inspected; after DG_ERR_CUDA it should be destroyed.
 */
#ifndef DGSWE_H
#define DGSWE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DG_OK = 0,
  DG_ERR_ARG = 1,         /* invalid argument (null pointer, size, value)    */
  DG_ERR_UNSUPPORTED = 2, /* valid configuration this build does not provide */
  DG_ERR_OOM = 3,         /* device (or host) allocation failed              */
  DG_ERR_CUDA = 4,        /* a CUDA runtime call failed                      */
  DG_ERR_DRY = 5,         /* H <= 0 met: projection matrix not SPD or a
                             wave-speed point with non-positive depth      */
  DG_ERR_NONFINITE = 6,   /* a NaN or Inf appeared in the state              */
  DG_ERR_TIMEOUT = 7      /* reserved: a bounded device wait gave up         */
} dg_status;

typedef enum { DG_BC_PERIODIC = 0, DG_BC_REFLECTIVE = 1, DG_BC_DIRICHLET = 2 } dg_bc;
typedef enum { DG_PREC_FP64 = 0, DG_PREC_FP32_MIXED = 1 } dg_precision;
/* Arithmetic of the velocity solve (u = q/H, Eq. (12)) of DG_PREC_FP32_MIXED:
 * FP64 (default); FP32; double-float (pairs of FP32 numbers, ~48 significant
 * bits, on the FP32 units; p <= 3); or MIXED: FP32 LDL^T and solves plus one
 * step of iterative refinement whose residual is accurate to ~48 bits (a
 * compensated FP32 dot product; the static bathymetry matrix is its FP32
 * part, recomputed, plus a stored FP32 low part), which returns the FP64 solution to within FP32 rounding
 * while the FP32 factors hold (elements whose FP32 pivots fail or spread by
 * more than 2^10 take the FP64 solve).  DF64 and MIXED: uniform meshes
 * without forcing only. */
typedef enum { DG_PROJ_FP64 = 0, DG_PROJ_FP32 = 1, DG_PROJ_DF64 = 2, DG_PROJ_MIXED = 3 } dg_proj_precision;
/* §3.1 convergence test of the paper: xi = 2.3 - 0.4 S, U = 0.6 + 0.04 S,
 * V = 0.3 + 0.04 S, S = sin(pi (x + y + 0.2 t) / 600), on the bathymetry
 * h_b = 1 + x/1000 + 2 y/1000 (which the caller projects), with the body force
 * F of Eq. (2) that makes it exact (tau_bf = f_c = 0).  The force enters the
 * volume term through the reference scheme's Gauss rule
 * (ceil((3p+2)/2)+1 points per direction, collapsed), the boundary data the
 * edge term through ceil((3p+1)/2)+1 Gauss points. */
typedef enum { DG_FORCING_NONE = 0, DG_FORCING_MANUFACTURED = 1 } dg_forcing;

typedef struct {
  int nx, ny;              /* quads; E = 2 nx ny triangles                      */
  double x0, y0, Lx, Ly;   /* domain                                            */
  const double* vertex_xy; /* NULL: uniform mesh; else (nx+1)(ny+1) vertices
                              (x, y), row j major (vertex (i, j) at
                              [2 (j (nx+1) + i)]): a general quad-split mesh
                              with the same topology (e.g. the randomly
                              perturbed meshes of §3.1); walls or Dirichlet
                              only, every triangle counter-clockwise; the
                              array is read by dg_init and not kept           */
  int p;                   /* polynomial order, 0..4 (p = 0: the first-order
                              finite-volume Lax-Friedrichs scheme)             */
  double g;                /* gravitational acceleration                        */
  int bc;                  /* dg_bc; DG_BC_DIRICHLET needs DG_FORCING_MANUFACTURED
                              (the only boundary data source)                 */
  int precision;           /* dg_precision                                      */
  int rk_order;            /* 1, 2 or 3 (SSP Runge-Kutta)                       */
  double cfl;              /* used when dt <= 0                                 */
  double dt;               /* > 0: fixed step                                   */
  int proj_precision;      /* dg_proj_precision: arithmetic of the u = q/H
                              solve in DG_PREC_FP32_MIXED (FP64 by default;
                              DG_PREC_FP64 always solves in FP64)             */
  int block_size;          /* threads per block of the stage kernels: 0 (=128),
                              32, 64, 96 or 128                               */
  double tau_bf;           /* bottom friction coefficient of Eq. (2) (>= 0)    */
  double f_c;              /* Coriolis coefficient of Eq. (2)                  */
  int forcing;             /* dg_forcing: DG_FORCING_MANUFACTURED adds the
                              body force of the §3.1 analytic solution and,
                              with DG_BC_DIRICHLET, uses that solution as the
                              boundary data                                    */
  int tile_shape;          /* kernel form of the time step for DG_PREC_FP32_MIXED
                              on uniform meshes without forcing (other
                              configurations ignore it): 1, 2, 3 = tile-fused
                              stages over 8 x 8, 16 x 8 or 8 x 4 quads,
                              intermediates in shared memory; -1 = one thread
                              per triangle with the intermediates in HBM;
                              0 (default) = 8 x 8 tiles at p <= 3 with the
                              MIXED and FP32 solves, 8 x 4 tiles at p = 4
                              with the FP32 solve, one thread per triangle
                              otherwise (measured faster there).
                              Both give the same scheme (agreeing to FP32
                              rounding); dg_rhs always uses the latter       */
} dg_config;

typedef struct dg_ctx dg_ctx;

/* Number of basis functions K = (p+1)(p+2)/2 of P^p on a triangle (paper
 * §2.2, the counts K = 1, 3, 6, 10 of the printed basis; p = 4 continues the
 * basis, which the paper prints up to order 3); 0 for p outside 0..4. */
int dg_num_basis(int p);

/* Number of bathymetry coefficients Kb per element (h_b enters the source
 * r(c) of Eq. (5) and the pressure term of Eq. (16); the paper leaves its
 * representation open): h_b is a DG field of P^max(p,1) (at
 * p = 0 a piecewise-constant h_b would drop the source g xi grad h_b), so
 * Kb = K for p >= 1 and 3 for p = 0. */
int dg_num_basis_bathymetry(int p);

/* Number of triangles 2 nx ny of a configuration: each quad of the
 * block-structured grid is split into two triangles (paper §2.3); 0 if
 * invalid. */
long long dg_num_elements(const dg_config* cfg);

/* Create a context (paper §2.2 discrete unknowns c_ei, Eqs. (13)-(14)).
 * hb: bathymetry coefficients, host FP64 AoS [E][Kb], Kb =
 * dg_num_basis_bathymetry(p) (h_b is a DG field of order max(p, 1); the
 * caller L2-projects it, see dg_project with that order).  xi, qx, qy: the
 * initial state, host FP64 AoS [E][K].  stream: a cudaStream_t or NULL.
 * Allocates every device buffer the time loop needs; *out receives the
 * context.  Errors: DG_ERR_ARG, DG_ERR_UNSUPPORTED, DG_ERR_OOM, DG_ERR_CUDA. */
dg_status dg_init(const dg_config* cfg, const double* hb, const double* xi, const double* qx,
                  const double* qy, void* stream, dg_ctx** out);

/* As dg_init (paper §2.2, Eqs. (13)-(14)), but hb, xi, qx, qy are DEVICE
 * arrays, FP64 SoA [Kb][E] (h_b) and [K][E] (one field each), e.g. the
 * output of dg_project.  They are copied; the caller keeps ownership.
 * Errors: DG_ERR_ARG, DG_ERR_UNSUPPORTED, DG_ERR_OOM, DG_ERR_CUDA. */
dg_status dg_init_device(const dg_config* cfg, const void* d_hb, const void* d_xi, const void* d_qx,
                         const void* d_qy, void* stream, dg_ctx** out);

/* Semi-discrete right-hand side (paper §2.2, Eq. (11) with the u-projection of
 * Eq. (12)): d_rhs_out = M^-1 [ (A~, grad phi) - <A^, phi> + (r, phi) ] for
 * the state d_state_in.  Both device SoA [3][K][E] (fields xi, U, V) in the
 * context's precision; they must not overlap.  Uses the context's scratch
 * buffers (allocated on the first call); does not change the context's own
 * state.  Asynchronous: a dry or non-finite input is not reported, and it
 * does not touch the error state that dg_run reports. */
dg_status dg_rhs(dg_ctx* ctx, const void* d_state_in, void* d_rhs_out);

/* One SSP-RK step of the context's state (the paper states no time
 * integrator, §3.1 uses a fixed dt; this library takes SSP Runge-Kutta in
 * Shu-Osher form, each stage w' = a w0 + b (w + dt R(w)) with R of dg_rhs).  Launched
 * asynchronously on the context's stream.  If dt_used is not NULL the stream
 * is synchronised and *dt_used receives the step's dt.  Dry or non-finite
 * states are flagged on the device and reported by the next dg_run.
 * Errors: DG_ERR_ARG (ctx NULL), DG_ERR_CUDA. */
dg_status dg_rk_step(dg_ctx* ctx, double* dt_used);

/* nsteps SSP-RK steps (as dg_rk_step), each launched as one
 * captured CUDA graph; nsteps = 0 only reads the error word and time.
 * Synchronises the stream once at the end, reads the device error word and
 * (if t_out is not NULL) the simulation time.  Returns DG_ERR_DRY (H <= 0 met;
 * the paper does not treat dry cells) or DG_ERR_NONFINITE if a kernel flagged one since the last
 * report; the word is then cleared and the context stays usable.
 * Errors: DG_ERR_ARG (ctx NULL, nsteps < 0), DG_ERR_DRY, DG_ERR_NONFINITE,
 * DG_ERR_OOM, DG_ERR_CUDA. */
dg_status dg_run(dg_ctx* ctx, int nsteps, double* t_out);

/* Copy the state, the coefficients c_ei of xi, q_x, q_y (paper §2.2,
 * Eqs. (13)-(14)), to host FP64 AoS arrays [E][K] (each may be NULL; the
 * caller owns them).  Page-locked arrays mapped into the device's address
 * space (cudaHostAlloc, cudaHostRegister; both ends of each array checked)
 * are written in place by one conversion kernel over the host link; other
 * arrays receive copies from a device staging buffer (allocated on first
 * use).  Synchronises the stream.
 * Errors: DG_ERR_ARG, DG_ERR_OOM (staging buffer), DG_ERR_CUDA. */
dg_status dg_get_state(dg_ctx* ctx, double* xi, double* qx, double* qy);

/* Replace the state (coefficients of Eqs. (13)-(14), host FP64 AoS [E][K],
 * all three required, copied; mapped page-locked arrays are read in place
 * as at dg_get_state) and the time t.  The next step re-evaluates the new
 * state.  Synchronises the stream.
 * Errors: DG_ERR_ARG, DG_ERR_OOM, DG_ERR_CUDA. */
dg_status dg_set_state(dg_ctx* ctx, const double* xi, const double* qx, const double* qy, double t);

/* Device pointer of the context's state (coefficients of Eqs. (13)-(14)),
 * SoA [3][K][E] in its precision; owned by the context, valid until
 * dg_destroy.  Errors: DG_ERR_ARG. */
dg_status dg_state_device(dg_ctx* ctx, void** d_state);

/* mass = sum_e integral xi (the quantity the continuity equation of Eq. (1)
 * conserves, paper §2.1); energy = 1/2 sum_e integral (g xi^2 + U u + V v)
 * with u from the projection of Eq. (12) (not in the paper: the usual
 * shallow-water energy relative to the rest state), both accumulated in
 * FP64 in a fixed order (deterministic).  Synchronises the stream.
 * Errors: DG_ERR_ARG, DG_ERR_OOM, DG_ERR_CUDA. */
dg_status dg_diagnostics(dg_ctx* ctx, double* mass, double* energy);

/* Set-up projection (not on the time-stepping path; the paper does not state
 * how initial data are projected; this is the L2 projection onto the basis
 * of §2.2): nodes of the library's Gauss rule on every element, so that
 * a caller can sample any function there and L2-project it.
 * dg_proj_num_nodes gives Q (0 for p outside 0..4); dg_proj_nodes writes
 * device FP64 [2][Q][E] (x then y); dg_project turns device FP64 samples
 * [Q][E] into device FP64 SoA coefficients [K][E].  Caller-owned device
 * arrays; asynchronous on stream.  Errors: DG_ERR_ARG, DG_ERR_CUDA. */
int dg_proj_num_nodes(int p);
dg_status dg_proj_nodes(const dg_config* cfg, void* d_xy, void* stream);
dg_status dg_project(const dg_config* cfg, const void* d_vals, void* d_coef, void* stream);

/* Flag bits that dg_rhs_noalloc ORs into the caller's optional word. */
enum { DG_FLAG_DRY = 1u /* a non-positive (or NaN) depth at a wave-speed point, or a velocity-projection
                           matrix that is not positive definite: the result is not meaningful */ };

/* dg_rhs_noalloc: the same right-hand side as dg_rhs, computed without
 * allocating any device memory.  The paper has no counterpart; this is an
 * interface for callers that cannot call cudaMalloc -- code that runs while a
 * CUDA graph is being captured, runtimes with a fixed device-memory budget
 * fixed at start-up, or hosts that forbid libraries from growing the device
 * heap -- and therefore cannot create a dg_ctx (dg_init allocates).
 *   cfg:        mesh, order, boundary, precision as for dg_init (p = 0..4,
 *               uniform mesh, periodic or reflective walls, no forcing);
 *               dt, cfl, rk_order are ignored.
 *   d_hb:       device FP64 SoA [Kb][E] bathymetry coefficients (input),
 *               Kb = dg_num_basis_bathymetry(p).
 *   d_state_in: device SoA [3][K][E] state in cfg's precision (input).
 *   d_rhs_out:  device SoA [3][K][E] (output), must not overlap d_state_in.
 *   d_flags:    NULL, or a caller-owned device word into which the call ORs
 *               DG_FLAG_DRY (stream-ordered; the call does not clear it, so
 *               the caller zeroes it and reads it after synchronising).  With
 *               NULL a dry state is not reported: the call returns DG_OK and
 *               the output holds whatever the arithmetic gave.
 *   stream:     cudaStream_t or NULL; the call is asynchronous on it.
 * Intermediates live in one fixed 32 MiB array inside the library's device
 * image, reserved on every GPU that loads the library until the process
 * exits.  A mesh needs about (K + 3(p+1) + p(p+1) + 3K + 3(6p+7)) words per
 * triangle, plus 2K^2 in FP64, plus K(K+1)/2 FP32 words (twice that at p = 4)
 * with DG_PROJ_MIXED
 * (8 bytes FP64, 4 bytes FP32, each block rounded up to 256 bytes); meshes
 * that do not fit are rejected with DG_ERR_ARG before any GPU work (about
 * 24,000 triangles at p = 2 in FP64).  The first call on a device looks up
 * the array's device address once (cudaGetSymbolAddress) and caches it; make
 * that first call before any stream capture.  A cudaDeviceReset() unloads
 * the array with the library's device image: do not call this entry point on
 * a device after resetting it.  Every call shares the array, which keeps the
 * previous call's contents; calls whose GPU work overlaps race and give wrong
 * results.
 * Errors: DG_ERR_ARG (invalid or too large), DG_ERR_UNSUPPORTED (forcing),
 * DG_ERR_CUDA. */
dg_status dg_rhs_noalloc(const dg_config* cfg, const void* d_hb, const void* d_state_in, void* d_rhs_out,
                         unsigned* d_flags, void* stream);

/* ---- batched instances -------------------------------------------------
 * Many independent problems of uneven size and order (ensembles of
 * bathymetries and initial states) advanced together: per RK stage one
 * persistent kernel launch covers every instance (per-element kernels), or
 * one per order class present (tile-fused FP32 kernels, each compiled for
 * its order), each instance keeps its own CFL
 * time step and time, and each step is one captured CUDA graph.  The
 * per-instance arithmetic is the single-instance scheme above (same kernels'
 * element code), so results equal those of separate dg_init contexts. */
typedef struct dg_batch dg_batch;

/* n instances of the scheme of paper §2.2 (the initial coefficients of
 * Eqs. (13)-(14) per instance; batching is not in the paper).  cfgs[i] as
 * for dg_init with p = 1..3, nx, ny >= 2, uniform meshes without forcing
 * (else DG_ERR_UNSUPPORTED).  All instances share precision,
 * proj_precision, rk_order, fixed-vs-CFL time stepping and the kernel form
 * (tile_shape >= 0 or -1; else DG_ERR_ARG); the kernel form and initial
 * tile shape are cfgs[0]'s (default: tile-fused with the MIXED and FP32
 * solves).  hb[i], xi[i], qx[i], qy[i]: HOST FP64 AoS arrays [E_i][K_i]
 * (as for dg_init; caller-owned, copied: each instance is transposed and
 * uploaded through one reused staging buffer).  Synchronises the stream.
 * Errors: DG_ERR_ARG (checked before any CUDA call), DG_ERR_UNSUPPORTED
 * (p = 0 or 4, Dirichlet, general meshes, forcing), DG_ERR_OOM,
 * DG_ERR_CUDA. */
dg_status dg_batch_init(int n, const dg_config* cfgs, const double* const* hb, const double* const* xi,
                        const double* const* qx, const double* const* qy, void* stream, dg_batch** out);

/* As dg_batch_init, but d_hb[i], d_xi[i], d_qx[i], d_qy[i] are DEVICE FP64
 * SoA [K_i][E_i] arrays (e.g. the output of dg_project; caller-owned,
 * copied).  The resulting batch is identical to the host form's. */
dg_status dg_batch_init_device(int n, const dg_config* cfgs, const void* const* d_hb, const void* const* d_xi,
                               const void* const* d_qx, const void* const* d_qy, void* stream, dg_batch** out);

/* nsteps SSP-RK steps (the time stepping of dg_rk_step) of every instance,
 * each with its own CFL step; t_out (NULL or n doubles) receives each
 * instance's time.  Synchronises the stream once at the end and reports
 * DG_ERR_DRY / DG_ERR_NONFINITE as dg_run does.  Errors: DG_ERR_ARG,
 * DG_ERR_DRY, DG_ERR_NONFINITE, DG_ERR_OOM, DG_ERR_CUDA. */
dg_status dg_batch_run(dg_batch* b, int nsteps, double* t_out);

/* state of instance i (coefficients of Eqs. (13)-(14)) as host FP64 AoS
 * [E_i][K_i] arrays (each may be NULL).  Mapped page-locked arrays are
 * written in place by one conversion kernel (as dg_get_state); others are
 * copied from the staging area described at dg_batch_set_state (allocated
 * by the first such call).  Synchronises the stream.  Errors: DG_ERR_ARG, DG_ERR_OOM,
 * DG_ERR_CUDA. */
dg_status dg_batch_get_state(dg_batch* b, int i, double* xi, double* qx, double* qy);

/* every instance's state (coefficients of Eqs. (13)-(14)) at once: xi[i],
 * qx[i], qy[i] as for dg_batch_get_state(b, i, ...) (host arrays of
 * n_instances pointers; the caller owns them and the arrays they point to;
 * any entry may be NULL), the transfers of all instances enqueued back to
 * back and the stream synchronised once.
 * Errors as dg_batch_get_state (DG_ERR_ARG also for a NULL pointer array);
 * on an error some instances may have been written. */
dg_status dg_batch_get_states(dg_batch* b, double* const* xi, double* const* qx, double* const* qy);

/* One SSP-RK step (as dg_rk_step: the scheme of paper §2.2 with this
 * library's SSP Runge-Kutta time step) of every instance from host states to host
 * states, as dg_batch_set_state(b, i, xi_in[i], qx_in[i], qy_in[i], t_i)
 * for every i (t_i its current time), dg_batch_run(b, 1, t_out) and
 * dg_batch_get_states(b, xi_out, qx_out, qy_out) would do, with the same
 * bits: host FP64 AoS [E_i][K_i] arrays behind arrays of n_instances
 * pointers (none NULL; the caller owns all; out may alias in).  Pipelined
 * (tile-fused batches; one group otherwise): every order class is cut into
 * runs of consecutive instances of about 1/16 of the batch's state bytes;
 * a run's state goes up by copy engine into the staging area (allocated on
 * first use, as at dg_batch_set_state), is evaluated and advanced by its
 * own stage launches and comes back by copy engine, while later runs go up
 * and earlier ones come down; page-locked arrays copy fastest.
 * Synchronises the stream.  t_out (n_instances doubles) may be NULL.
 * Errors: DG_ERR_ARG, DG_ERR_OOM, DG_ERR_DRY, DG_ERR_NONFINITE (as
 * dg_batch_run: the step was taken and the word cleared), DG_ERR_CUDA. */
dg_status dg_batch_step_host(dg_batch* b, const double* const* xi_in, const double* const* qx_in,
                             const double* const* qy_in, double* const* xi_out, double* const* qx_out,
                             double* const* qy_out, double* t_out);

/* replace the state of instance i (coefficients of Eqs. (13)-(14), host FP64
 * AoS [E_i][K_i] arrays, all three required) and its model time t; the next
 * dg_batch_run re-evaluates the batch.  Asynchronous on the batch's stream
 * (the copies of successive calls overlap): the arrays must stay unchanged
 * until the stream is synchronised -- dg_batch_run, dg_batch_get_state and
 * every other synchronising call do.  Mapped page-locked arrays are read in
 * place by one conversion kernel (as dg_get_state); for other arrays the
 * first such call allocates a device staging area for every instance's
 * FP64 state (kept until dg_batch_destroy).  Errors: DG_ERR_ARG, DG_ERR_OOM,
 * DG_ERR_CUDA. */
dg_status dg_batch_set_state(dg_batch* b, int i, const double* xi, const double* qx, const double* qy, double t);

/* Autotuner of the batched launch (not in the paper; it changes only the
 * launch shape, never the arithmetic): times trial_steps steps of each
 * candidate shape, restoring the state after each, and keeps the fastest.
 * Candidates: tile-fused batches (FP32, tile_shape >= 0) tiles of 8 x 8,
 * 16 x 8 and 8 x 4 quads (128, 256, 64 triangles per CTA; tile_shape 1, 2,
 * 3);
 * per-element batches 32, 64, 96 and 128 elements per work item (one thread
 * per element).  Tile-fused batches run one launch per order class and
 * stage, and every class keeps the shape of its own fastest launches (see
 * dg_batch_tile_shape).  *block_out (may be NULL) receives the chosen
 * element count, or the tile shape of the highest order class, and ms_out
 * (NULL or 4 doubles) the ms per step of each candidate in that order (all
 * classes on that shape; 0 where there is none).  State and times are
 * unchanged on return.  Errors: DG_ERR_ARG, DG_ERR_OOM, DG_ERR_CUDA. */
dg_status dg_batch_autotune(dg_batch* b, int trial_steps, int* block_out, double* ms_out);

/* set the launch shape of the batch (not in the paper): a tile shape 1..3
 * (numbered as dg_config.tile_shape) for tile-fused batches, else 32, 64, 96 or 128 elements per work item;
 * DG_ERR_ARG otherwise.  On any error the batch keeps its previous setting.
 * Synchronises the stream. */
dg_status dg_batch_set_block(dg_batch* b, int block);

/* tile shape (dg_config.tile_shape numbering, 1..3) of the order-p class of
 * a tile-fused batch; 0 for a per-element batch, a NULL batch, or an order
 * without instances (not in the paper) */
int dg_batch_tile_shape(const dg_batch* b, int p);

/* degrees of freedom updated per RK stage: sum over instances of 3 K E (the
 * coefficients of xi, q_x, q_y of Eqs. (13)-(14)); 0 for NULL */
long long dg_batch_dofs(const dg_batch* b);

/* Release every resource of the batch (NULL is ignored); synchronises its
 * stream first. */
void dg_batch_destroy(dg_batch* b);

/* Release every resource of the context (NULL is ignored); synchronises its
 * stream first. */
void dg_destroy(dg_ctx* ctx);

/* Static string naming a status ("DG_ERR_UNKNOWN" for other values). */
const char* dg_status_str(dg_status s);

#ifdef __cplusplus
}
#endif

#endif /* DGSWE_H */
