/* A plain C99 caller of the library: the public headers compile as C (-std=c99 -pedantic) and the
 * argument checks answer without a GPU. Exit status 0 when every check holds. */
#include <stdio.h>
#include <string.h>

#include "ga.h"
#include "ga_ops.h"

static int failures = 0;

static void expect(int cond, const char* what) {
  if (!cond) {
    fprintf(stderr, "failed: %s\n", what);
    ++failures;
  }
}

int main(void) {
  ga_stats s;
  double out = 0.0;
  int tiles[6] = {0, 0, 0, 0, 0, 0};
  ga_ctx* ctx = NULL;
  ga_problem_desc d;
  ga_solver_opts o;
  double m[16 * 16];

  expect(ga_objective(NULL, NULL, GA_MEM_HOST, &out) == GA_ERR_ARG, "ga_objective(NULL)");
  expect(ga_get_stats(NULL, &s) == GA_ERR_ARG, "ga_get_stats(NULL)");
  expect(ga_op_get_tiles(NULL, tiles) == GA_ERR_ARG, "ga_op_get_tiles(NULL)");
  expect(ga_solve_batch(-1, NULL, NULL, GA_MEM_HOST, NULL) == GA_ERR_ARG, "ga_solve_batch(-1)");
  expect(strcmp(ga_status_str(GA_ERR_LINESEARCH), "GA_ERR_LINESEARCH") == 0, "ga_status_str");

  /* an invalid option set is refused before any device work */
  memset(&d, 0, sizeof d);
  memset(&o, 0, sizeof o);
  memset(m, 0, sizeof m);
  d.dim = 2;
  d.n[0] = 16;
  d.n[1] = 16;
  d.nt = 2;
  d.model = GA_MODEL_ADVECTION;
  d.reg_order = 1;
  d.alpha = 1e-2;
  d.prec = GA_PREC_FP64;
  o.window = 4;
  o.sigma = 2;
  o.tau = 1;
  o.max_iter = 5;
  o.rel_tol = 1e-2;
  o.armijo_c = 1e-4;
  o.max_backtracks = 10;
  o.variant = 1;
  o.method = GA_METHOD_GA_AA;
  o.graphs = 2; /* device-driven solves take GA-NGMRES and RPGD only */
  expect(ga_setup(&d, &o, m, m, GA_MEM_HOST, NULL, &ctx) == GA_ERR_ARG, "ga_setup(GA-AA, graphs = 2)");
  expect(ctx == NULL, "no context after a refused setup");

  if (failures == 0) printf("ok\n");
  return failures == 0 ? 0 : 1;
}
