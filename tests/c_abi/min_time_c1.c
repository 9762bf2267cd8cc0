/* A plain C99 caller of the C-ABI (include/mc.h, include/mc_pe.h): builds the
 * tiny model (global size 64, two compute units, WG in {1,2,4,8,16}, TS in
 * {1,2,4}, per-work-group cost ceil(WG/TS)*4 + WG + 2*TS), asks for the
 * minimal time and its configuration with a trace, and checks the property at
 * T_min - 1 (holds) and T_min (fails).
 *
 * Exit status: 0 when the answers are T_min = 80 at WG = 16, TS = 4 with a
 * trace of level + 1 states; 3 when the library reports MC_ERR_CUDA (no usable
 * device); 1 on any other outcome. */
#include <stdint.h>
#include <stdio.h>

#include "mc.h"
#include "mc_pe.h"

int main(void) {
  const uint32_t wg[5] = {1, 2, 4, 8, 16}, ts[3] = {1, 2, 4};
  uint32_t n[15], cost[15];
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 3; ++j) {
      n[i * 3 + j] = (64 + wg[i] - 1) / wg[i];
      cost[i * 3 + j] = (wg[i] + ts[j] - 1) / ts[j] * 4 + wg[i] + 2 * ts[j];
    }
  mc_model_desc d;
  d.n_wg = 5;
  d.n_ts = 3;
  d.P = 2;
  d.wg_values = wg;
  d.ts_values = ts;
  d.n_workgroups = n;
  d.cost = cost;
  d.speed = NULL;
  d.rule = MC_FREE;
  d.key_bits = 0;

  mc_model* m = NULL;
  int rc = mc_model_create(&d, NULL, &m);
  if (rc != MC_OK) {
    printf("mc_model_create: %s\n", mc_strerror(rc));
    return 1;
  }
  mc_min_result r;
  mc_trace* t = NULL;
  rc = mc_min_time(m, &r, &t);
  if (rc == MC_ERR_CUDA) {
    printf("mc_min_time: %s (%s)\n", mc_strerror(rc), mc_last_error(m));
    mc_model_destroy(m);
    return 3;
  }
  if (rc != MC_OK) {
    printf("mc_min_time: %s\n", mc_strerror(rc));
    mc_model_destroy(m);
    return 1;
  }
  const int len = mc_trace_length(t);
  printf("T_min %llu at WG %u TS %u, level %u, %d trace states, %llu states in %u checks\n",
         (unsigned long long)r.t_min, r.wg, r.ts, r.level, len, (unsigned long long)r.states, r.checks);
  int ok = r.t_min == 80 && r.wg == 16 && r.ts == 4 && len == (int)r.level + 1 &&
           mc_trace_states(t) != NULL && mc_trace_key_words(t) == 1;
  mc_trace_free(t);

  mc_check_result below, at;
  ok = ok && mc_check(m, r.t_min - 1, &below, NULL) == MC_OK && below.holds == 1;
  ok = ok && mc_check(m, r.t_min, &at, NULL) == MC_OK && at.holds == 0 && at.cex_time == r.t_min;
  mc_model_destroy(m);
  return ok ? 0 : 1;
}
