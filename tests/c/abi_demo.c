/* A C caller of the library: two robots (straight, no obstacles; one with an
 * actuator) grown to full length through the C ABI alone.  Prints
 * "ok <links> <tip x> <tip y>" per robot, or the library's error text. */
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
  vine_batch_destroy(b);
  return 0;
}
