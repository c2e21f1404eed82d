/* Calls the host-only entry points of librlbm.so from plain C (no Python, no
 * torch): the quadratures, the stencil, and argument checks that fail before
 * any device work.  Prints one line per result for the test to check. */
#include <stdio.h>
#include <string.h>

#include "rlbm.h"
#include "rlbm_massive.h"

int main(void) {
  double w1[4], w2[4], p0[4];
  int rc = rlbm_quadrature(w1, w2, p0);
  printf("quadrature %d %.17g %.17g %.17g\n", rc, w1[0], w2[0], p0[1]);

  double v0, win[2], w[10], q0[10];
  rc = rlbm_massive_quadrature(&v0, win, w, q0);
  printf("massive_quadrature %d %.17g %.17g %.17g %.17g\n", rc, v0, win[0], win[1], w[0]);

  int vx[45], vy[45];
  rc = rlbm_massive_stencil(vx, vy);
  printf("stencil %d %d %d %d %d\n", rc, vx[0], vy[0], vx[43], vy[44]);

  /* bad configurations are rejected before any device call */
  rlbm_massive_config mc;
  memset(&mc, 0, sizeof mc);
  mc.nx = 4; mc.ny = 16; mc.tau = 1.0; mc.prec = RLBM_F32;
  rlbm_massive_ctx* m = (rlbm_massive_ctx*)&mc;
  rc = rlbm_massive_create(&mc, &m);
  printf("massive_create_bad %d %d %s\n", rc, m == NULL, rlbm_massive_last_error(NULL)[0] ? "msg" : "nomsg");

  rlbm_sample s;
  memset(&s, 0, sizeof s);
  s.nx = 64; s.ny = 32; s.tau = 0.5;          /* tau must exceed 1/2 */
  rlbm_config cfg;
  memset(&cfg, 0, sizeof cfg);
  cfg.prec = RLBM_F32; cfg.nsamples = 1; cfg.samples = &s;
  size_t bytes = 0;
  rc = rlbm_workspace_size(&cfg, &bytes);
  printf("workspace_bad %d %s\n", rc, rlbm_last_error(NULL)[0] ? "msg" : "nomsg");
  s.tau = 1.0;
  rc = rlbm_workspace_size(&cfg, &bytes);
  printf("workspace_ok %d %zu\n", rc, bytes);
  rlbm_destroy(NULL);
  rlbm_massive_destroy(NULL);
  printf("version %d\n", rlbm_version());
  return 0;
}
