/* Plain C99 user of the library's C ABI: compiles against include/dgswe.h
 * alone and links libdgswe.so.  It exercises only calls that validate their
 * arguments on the host, so it runs without a GPU. */
#include <stdio.h>
#include <string.h>

#include "dgswe.h"

int main(void) {
  int fails = 0;
  if (dg_num_basis(2) != 6 || dg_num_basis(5) != 0) fails++;
  if (dg_num_basis_bathymetry(0) != 3) fails++;
  if (strcmp(dg_status_str(DG_ERR_DRY), "DG_ERR_DRY") != 0) fails++;

  dg_config cfg;
  memset(&cfg, 0, sizeof cfg);
  cfg.nx = 4;
  cfg.ny = 4;
  cfg.Lx = 1.0;
  cfg.Ly = 1.0;
  cfg.p = 2;
  cfg.g = 9.81;
  cfg.bc = DG_BC_PERIODIC;
  cfg.precision = DG_PREC_FP64;
  cfg.rk_order = 3;
  cfg.cfl = 0.2;
  if (dg_num_elements(&cfg) != 32) fails++;

  double z[1] = {0.0};
  dg_ctx* ctx = NULL;
  cfg.rk_order = 4; /* invalid: rejected before any CUDA call */
  if (dg_init(&cfg, z, z, z, z, NULL, &ctx) != DG_ERR_ARG || ctx != NULL) fails++;
  cfg.rk_order = 3;
  cfg.bc = DG_BC_DIRICHLET; /* needs the manufactured forcing */
  if (dg_init(&cfg, z, z, z, z, NULL, &ctx) != DG_ERR_UNSUPPORTED) fails++;

  /* batch calls: the host-array form validates before any CUDA call */
  const double* zp[1] = {z};
  double* outp[1] = {z};
  dg_batch* b = NULL;
  cfg.bc = DG_BC_PERIODIC;
  cfg.p = 4; /* the batched kernels hold p = 1..3 */
  if (dg_batch_init(1, &cfg, zp, zp, zp, zp, NULL, &b) != DG_ERR_UNSUPPORTED || b != NULL) fails++;
  if (dg_batch_get_states(NULL, outp, outp, outp) != DG_ERR_ARG) fails++;
  if (dg_batch_step_host(NULL, zp, zp, zp, outp, outp, outp, NULL) != DG_ERR_ARG) fails++;

  printf("%s\n", fails ? "FAIL" : "OK");
  return fails;
}
