/* A plain C99 client of include/trim.h: a 5-vertex chain v4 -> v3 -> v2 -> v1
 * -> v0 and a 2-cycle v5 <-> v6 feeding nothing. Exit status 0 when the levels
 * are (0, 1, 2, 3, 4, LIVE, LIVE) or, with expect_no_device, when trim_create
 * reports TRIM_ERR_NO_DEVICE; 1 otherwise. */
#include <stdio.h>
#include <string.h>

#include "trim.h"

int main(int argc, char** argv) {
  const int expect_no_device = argc > 1 && strcmp(argv[1], "--expect-no-device") == 0;
  const uint32_t offsets[8] = {0, 0, 1, 2, 3, 4, 5, 6};
  const uint32_t targets[6] = {0, 1, 2, 3, 6, 5};
  const uint32_t want[7] = {0, 1, 2, 3, 4, TRIM_LIVE, TRIM_LIVE};
  trim_params_t p;
  if (trim_default_params(&p) != TRIM_OK || p.block_threads == 0) return 1;
  trim_csr_t g;
  g.n = 7;
  g.m = 6;
  g.offsets = offsets;
  g.targets = targets;
  g.on_device = TRIM_MEM_HOST;
  trim_ctx* ctx = NULL;
  trim_err_t e = trim_create(&g, NULL, NULL, 0, &ctx);
  if (expect_no_device) {
    printf("trim_create: %d (%s)\n", (int)e, trim_last_error(NULL));
    return e == TRIM_ERR_NO_DEVICE ? 0 : 1;
  }
  if (e != TRIM_OK) {
    printf("trim_create failed: %s\n", trim_last_error(NULL));
    return 1;
  }
  int ok = 1;
  const trim_variant_t variants[4] = {TRIM_AC4_PUSH, TRIM_AC6_SUPPORT, TRIM_AC3_PULL,
                                      TRIM_SCHED_HEURISTIC};
  for (int k = 0; k < 4; ++k) {
    trim_run_stats_t s;
    uint32_t level[7];
    uint8_t status[7];
    if (trim_run(ctx, variants[k], &s) != TRIM_OK || trim_level(ctx, level, 0) != TRIM_OK ||
        trim_status(ctx, status, 0) != TRIM_OK) {
      printf("variant %d: %s\n", (int)variants[k], trim_last_error(ctx));
      ok = 0;
      continue;
    }
    for (int v = 0; v < 7; ++v)
      if (level[v] != want[v] || status[v] != (want[v] == TRIM_LIVE)) ok = 0;
    if (s.rounds != 5 || s.n_dead != 5) ok = 0;
  }
  trim_destroy(ctx);
  printf(ok ? "c client ok\n" : "c client: wrong result\n");
  return ok ? 0 : 1;
}
