/* A C caller of the library: two robots (straight, no obstacles; one with an
 * actuator) grown to full length through the C ABI alone.  Prints
 * "ok <links> <tip x> <tip y>" per robot; then the largest tip move when a
 * second batch loaded with that state (vine_set_state) is relaxed with the
 * length held ("relax <m>"), the keep flags of a three-state pruning
 * ("prune a b c"), and a synthesised design ("synth <p index> <l0 index>");
 * or the library's error text. */
#include <stdint.h>
#include <stdio.h>

#include "vine.h"

int main(void) {
  int32_t n_links[2] = {12, 12};
  float l_seg[2] = {0.02f, 0.02f}, radius[2] = {0.025f, 0.025f}, pressure[2] = {5000.f, 5000.f};
  float base[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  int32_t act_ptr[3] = {0, 0, 1};
  float act_begin[1] = {2.f}, act_end[1] = {7.f}, act_pressure[1] = {8000.f}, act_l0[1] = {0.02f};
  int8_t act_side[1] = {1};
  int32_t obs_ptr[3] = {0, 0, 0};
  vine_batch_desc d = {0};
  d.n_inst = 2;
  d.mem_is_device = 0;
  d.n_links = n_links; d.l_seg = l_seg; d.radius = radius; d.pressure = pressure; d.base = base;
  d.act_ptr = act_ptr; d.act_begin = act_begin; d.act_end = act_end; d.act_side = act_side;
  d.act_pressure = act_pressure; d.act_l0 = act_l0; d.obs_ptr = obs_ptr;
  vine_params p;
  vine_batch* b = NULL;
  float tip[4];
  int32_t n_present[2], status[2];
  if (vine_params_default(&p) != VINE_OK || vine_batch_create(&d, &p, NULL, &b) != VINE_OK ||
      vine_simulate(b, NULL) != VINE_OK ||
      vine_get_state(b, NULL, NULL, NULL, tip, n_present, NULL, NULL, status, 0, NULL) != VINE_OK) {
    printf("error %s\n", vine_last_error());
    return 1;
  }
  for (int i = 0; i < 2; ++i) printf("%s %d %.6f %.6f\n", status[i] == VINE_INST_OK ? "ok" : "bad", n_present[i],
                                     tip[2 * i], tip[2 * i + 1]);
  /* continue from the read state in a second batch, relaxed with the length held */
  float theta[24], l_last[2], tip2[4];
  vine_batch* b2 = NULL;
  if (vine_get_state(b, theta, l_last, NULL, NULL, NULL, NULL, NULL, NULL, 0, NULL) != VINE_OK ||
      vine_batch_create(&d, &p, NULL, &b2) != VINE_OK ||
      vine_set_state(b2, n_present, theta, l_last, 0, NULL) != VINE_OK || vine_relax(b2, 1, NULL) != VINE_OK ||
      vine_get_state(b2, NULL, NULL, NULL, tip2, NULL, NULL, NULL, NULL, 0, NULL) != VINE_OK) {
    printf("error %s\n", vine_last_error());
    return 1;
  }
  float move = 0.f;
  for (int k = 0; k < 4; ++k) {
    const float dk = tip2[k] > tip[k] ? tip2[k] - tip[k] : tip[k] - tip2[k];
    if (dk > move) move = dk;
  }
  printf("relax %.3e\n", move);
  /* pruning: states 1 and 2 overlap (1 is cheaper), state 3 is far away */
  float pose[9] = {0.f, 0.f, 0.f, 3.f, 0.f, 0.f, 100.f, 0.f, 0.f};
  double cost[3] = {2.0, 1.0, 5.0};
  uint8_t keep[3];
  if (vine_sst_prune(0, NULL, NULL, NULL, 3, pose, cost, 10.f, 1.f, keep, NULL, 0, NULL) != VINE_OK) {
    printf("error %s\n", vine_last_error());
    return 1;
  }
  printf("prune %d %d %d\n", keep[0], keep[1], keep[2]);
  /* design synthesis for one target angle per joint */
  double pressures[3] = {10000.0, 20000.0, 40000.0}, target = 0.03, theta_eq;
  int32_t pi, li;
  vine_synth_spec spec = {0.03335, 10342.0, 0.025, pressures, 3, 0.020, 0.001, 61, 0.004};
  if (vine_synthesize(&spec, NULL, &target, 1, &pi, &li, &theta_eq, NULL, NULL) != VINE_OK) {
    printf("error %s\n", vine_last_error());
    return 1;
  }
  printf("synth %d %d %.6f\n", pi, li, theta_eq);
  vine_batch_destroy(b2);
  vine_batch_destroy(b);
  return 0;
}
