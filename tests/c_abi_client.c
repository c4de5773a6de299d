/* A plain C99 client of the library: it includes only hifcn.h and links
 * libhifcn.so.  It runs the calls that need no GPU (defaults, messages and
 * the argument checks that every entry point makes before touching the
 * device) and exits 0 when every check holds, or with the number of the first
 * failed check. */
#include "hifcn.h"

#include <math.h>
#include <stdio.h>
#include <string.h>

static int g_check = 0;
#define CHECK(cond)                                              \
  do {                                                           \
    ++g_check;                                                   \
    if (!(cond)) {                                               \
      fprintf(stderr, "check %d failed: %s\n", g_check, #cond); \
      return g_check;                                            \
    }                                                            \
  } while (0)

static int setup_status(const hif_grid *g, const double *a, double dt, const hif_options *o) {
  hif_handle *h = (hif_handle *)&g_check; /* must be overwritten with NULL */
  int st = hif_setup(g, a, dt, o, NULL, &h);
  return (h == NULL) ? st : 1000;
}

int main(void) {
  hif_options o;
  hif_grid good = {2, 32, 8}, g;
  const double *a = (const double *)&o; /* never dereferenced: every call below fails first */
  double x = 0.0, y = 0.0;
  int it = 0, count = 0;
  size_t bytes = 0;
  hif_info info;
  const int codes[] = {HIF_OK, HIF_EINVAL, HIF_ENOMEM, HIF_ENOTSPD,
                       HIF_ENOCONV, HIF_ETIMEOUT, HIF_ECUDA, HIF_EFORMAT};
  static const char *const names[14] = {"eps", "eps", "theta", "theta", "precision", "x0_mode",
                                        "solver", "cg_maxit", "cg_tol", "cg_tol",
                                        "true_res_period", "skel_edges_3d", "bf16_top_levels",
                                        "eps"};
  int i, j;

  /* defaults */
  memset(&o, 0xff, sizeof(o));
  hif_default_options(&o);
  CHECK(o.eps == 1e-6 && o.precision == HIF_FP64 && o.skel_edges_3d == 1);
  CHECK(o.cg_tol == 1e-10 && o.cg_maxit == 1000 && o.true_res_period == 50);
  CHECK(o.theta == 0.5 && o.x0_mode == 0 && o.solver == 0 && o.bf16_top_levels == 0);
  hif_default_options(NULL);

  /* grid and argument checks of hif_setup */
  CHECK(hif_setup(&good, a, 1.0, NULL, NULL, NULL) == HIF_EINVAL);
  CHECK(setup_status(NULL, a, 1.0, NULL) == HIF_EINVAL);
  CHECK(setup_status(&good, NULL, 1.0, NULL) == HIF_EINVAL);
  g = good; g.n = 100; g.leaf = 16;                 /* not leaf * 2^L */
  CHECK(setup_status(&g, a, 1.0, NULL) == HIF_EINVAL);
  CHECK(strstr(hif_last_error(), "leaf * 2^L") != NULL);
  g = good; g.n = 8; g.leaf = 8;                    /* L = 0 */
  CHECK(setup_status(&g, a, 1.0, NULL) == HIF_EINVAL);
  g = good; g.dim = 4;
  CHECK(setup_status(&g, a, 1.0, NULL) == HIF_EINVAL);
  g = good; g.leaf = 1; g.n = 32;
  CHECK(setup_status(&g, a, 1.0, NULL) == HIF_EINVAL);
  g.dim = 3; g.n = 2048; g.leaf = 8;                /* N = 2047^3 > 2^31 - 1 */
  CHECK(setup_status(&g, a, 1.0, NULL) == HIF_EINVAL);
  CHECK(setup_status(&good, a, 0.0, NULL) == HIF_EINVAL);
  CHECK(setup_status(&good, a, -1.0, NULL) == HIF_EINVAL);
  CHECK(setup_status(&good, a, INFINITY, NULL) == HIF_EINVAL);
  CHECK(strstr(hif_last_error(), "dt") != NULL);

  /* options out of range */
  for (i = 0; i < 14; ++i) {
    hif_default_options(&o);
    switch (i) {
      case 0: o.eps = -1e-6; break;
      case 1: o.eps = NAN; break;
      case 2: o.theta = 0.0; break;
      case 3: o.theta = 1.5; break;
      case 4: o.precision = 7; break;
      case 5: o.x0_mode = 2; break;
      case 6: o.solver = -1; break;
      case 7: o.cg_maxit = -1; break;
      case 8: o.cg_tol = -1.0; break;
      case 9: o.cg_tol = INFINITY; break;
      case 10: o.true_res_period = -1; break;
      case 11: o.skel_edges_3d = 2; break;
      case 12: o.bf16_top_levels = -1; break;
      default: o.eps = INFINITY; break;
    }
    CHECK(setup_status(&good, a, 1.0, &o) == HIF_EINVAL);
    CHECK(strncmp(hif_last_error(), "option out of range: ", 21) == 0);
    CHECK(strcmp(hif_last_error() + 21, names[i]) == 0); /* names the option */
  }

  /* every handle call refuses a NULL handle without touching the device */
  CHECK(hif_apply(NULL, &x, &y, HIF_FP64, NULL) == HIF_EINVAL);
  CHECK(hif_apply_noalloc(NULL, &x, &y, NULL) == HIF_EINVAL);
  CHECK(strstr(hif_last_error(), "h is NULL") != NULL);
  CHECK(hif_inject_flow_stall(NULL, 0, 16) == HIF_EINVAL);
  CHECK(hif_release_fp64(NULL) == HIF_EINVAL);
  CHECK(hif_offload(NULL) == HIF_EINVAL);
  CHECK(hif_reload(NULL) == HIF_EINVAL);
  CHECK(hif_apply_multi(NULL, &x, &y, 1, NULL) == HIF_EINVAL);
  CHECK(cn_step_multi(NULL, &x, NULL, &y, 1, &it, NULL) == HIF_EINVAL);
  CHECK(hif_matvec(NULL, &x, &y, NULL) == HIF_EINVAL);
  CHECK(pcg_solve(NULL, &x, &y, &it, &x, NULL) == HIF_EINVAL);
  CHECK(cn_step(NULL, &x, NULL, &y, &it, NULL) == HIF_EINVAL);
  CHECK(cn_steps(NULL, &x, NULL, 1, &it, NULL) == HIF_EINVAL);
  CHECK(cn_step_batched(NULL, -1, NULL, NULL, NULL, NULL, NULL) == HIF_EINVAL);
  CHECK(cn_step_batched(NULL, 1, NULL, NULL, NULL, NULL, NULL) == HIF_EINVAL);
  CHECK(cn_step_batched(NULL, 0, NULL, NULL, NULL, NULL, NULL) == HIF_OK); /* empty batch */
  CHECK(hif_set_reaction(NULL, 1, 1.0, 1.0) == HIF_EINVAL);
  CHECK(hif_set_coefficient(NULL, a, NULL) == HIF_EINVAL);
  CHECK(hif_refactor(NULL, a, NULL) == HIF_EINVAL);
  CHECK(hif_autotune(NULL, NULL) == HIF_EINVAL);
  CHECK(hif_query(NULL, &info) == HIF_EINVAL);
  CHECK(hif_export_factor(NULL, NULL, &bytes) == HIF_EINVAL);
  CHECK(hif_stats_enable(NULL, 1) == HIF_EINVAL);
  CHECK(hif_stats_read(NULL, NULL, 0, &count) == HIF_EINVAL);
  CHECK(hif_destroy(NULL) == HIF_OK);
  {
    hif_handle *h = (hif_handle *)&g_check;
    CHECK(hif_import_factor(&good, NULL, 0, 1.0, a, NULL, NULL, &h) == HIF_EINVAL);
  }

  /* messages: one per status, all distinct, and one for an unknown code */
  for (i = 0; i < 8; ++i) {
    CHECK(hif_strerror(codes[i]) != NULL && hif_strerror(codes[i])[0] != '\0');
    for (j = 0; j < i; ++j) CHECK(strcmp(hif_strerror(codes[i]), hif_strerror(codes[j])) != 0);
  }
  CHECK(hif_strerror(-12345) != NULL);
  CHECK(hif_last_error() != NULL);
  CHECK(hif_launch_count() >= 0);

  printf("ok %d checks\n", g_check);
  return 0;
}
