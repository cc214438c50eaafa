/* Plain C client of include/tt.h: compiled with a C compiler and linked against
 * libttgb.so, it makes the host-only calls of the ABI (no device work) and prints
 * "ok" when each returns what the header documents. */
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "tt.h"

static int fail(const char *what) {
  printf("FAIL %s\n", what);
  return 1;
}

int main(void) {
  int64_t I[3] = {64, 32, 16};
  int64_t R[4] = {1, 8, 4, 1};
  void *cores[3] = {(void *)0x1000, (void *)0x2000, (void *)0x3000};
  tt_tensor x;
  size_t n = 0, m = 0, len = 0;
  char buf[4096];
  x.N = 3;
  x.dtype = TT_F64;
  x.I = I;
  x.R = R;
  x.cores = cores;

  if (tt_round_workspace_size(&x, TT_PREC_FP64, &n) != TT_OK || n == 0) return fail("workspace size");
  if (tt_round_workspace_size(&x, TT_PREC_FP32X2, &n) != TT_ERR_INVALID_ARG) return fail("precision vs dtype");
  if (tt_norm_workspace_size(&x, &m) != TT_OK || m == 0) return fail("norm workspace");
  if (tt_dot_workspace_size(&x, &x, &m) != TT_OK || m == 0) return fail("dot workspace");
  R[0] = 2;
  if (tt_round_workspace_size(&x, TT_PREC_FP64, &n) != TT_ERR_INVALID_ARG) return fail("R[0] != 1");
  R[0] = 1;
  R[1] = 300;
  if (tt_round_workspace_size(&x, TT_PREC_FP64, &n) != TT_ERR_UNSUPPORTED) return fail("rank above maximum");
  R[1] = 8;
  if (strlen(tt_status_string(TT_ERR_WORKSPACE)) == 0) return fail("status string");

  /* tile table: import, export, clear */
  if (tt_tune_clear() != TT_OK) return fail("clear");
  if (tt_tune_import("1 0 32 8 4 8 4 2 1\n") != TT_OK) return fail("import");
  if (tt_tune_export(NULL, 0, &len) != TT_OK || len < 2) return fail("export size");
  if (tt_tune_export(buf, sizeof buf, &len) != TT_OK || strstr(buf, "1 0 32 8 4 8 4 2 1") == NULL) return fail("export");
  if (tt_tune_import("1 0 32 8 4 8 4 2\n") != TT_ERR_INVALID_ARG) return fail("malformed import");
  if (tt_tune_clear() != TT_OK) return fail("clear again");
  printf("ok\n");
  return 0;
}
