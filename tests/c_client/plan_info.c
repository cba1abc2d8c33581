/* A plain C99 client of the QTAM C ABI (include/qtam.h): builds a host-only
 * plan of the 64 s workload (device = -1, no GPU needed), prints its plan
 * info as "key value" lines, checks an argument error, and destroys it.
 * Compiled and run by tests/test_c_client.py. */
#include <stdio.h>
#include <string.h>

#include "qtam.h"

int main(void) {
  static const double qs[] = {4.0, 8.0, 16.0, 32.0, 64.0};
  qtam_plan_desc d;
  qtam_plan_t plan = NULL;
  qtam_plan_info_t info;
  qtam_status s;

  qtam_plan_desc_init(&d);
  d.sample_rate = 4096.0;
  d.length = 262144;
  d.q = qs;
  d.n_q = 5;
  d.f_min = 20.0;
  d.f_max = 2048.0;
  d.rows_per_plane = 128;
  s = qtam_plan(&d, -1, &plan);
  if (s != QTAM_OK) {
    fprintf(stderr, "qtam_plan: %s: %s\n", qtam_status_string(s), qtam_last_error());
    return 1;
  }
  memset(&info, 0, sizeof info);
  s = qtam_plan_info(plan, &info);
  if (s != QTAM_OK) {
    fprintf(stderr, "qtam_plan_info: %s\n", qtam_status_string(s));
    return 1;
  }
  printf("length %lld\n", (long long)info.length);
  printf("n_bins %lld\n", (long long)info.n_bins);
  printf("n_planes %d\n", (int)info.n_planes);
  printf("rows_per_plane %d\n", (int)info.rows_per_plane);
  printf("n_out %d\n", (int)info.n_out);
  printf("h_max %d\n", (int)info.h_max);
  printf("max_window %d\n", (int)info.max_window);
  printf("envelope_bytes_per_segment %lld\n", (long long)info.envelope_bytes_per_segment);
  printf("band_bins %lld\n", (long long)info.band_bins);
  printf("kept_bins %lld\n", (long long)info.kept_bins);
  printf("p_floor_rel %.17g\n", info.p_floor_rel);
  printf("kappa %.17g\n", info.kappa);
  printf("row_variant %d\n", (int)info.row_variant);

  /* an odd length is rejected with QTAM_ERR_INVALID_ARG and a message */
  {
    qtam_plan_t bad = NULL;
    d.length = 262143;
    s = qtam_plan(&d, -1, &bad);
    printf("odd_length_status %d\n", (int)s);
    printf("odd_length_message %s\n", qtam_last_error()[0] ? "yes" : "no");
  }
  s = qtam_destroy(plan);
  printf("destroy %d\n", (int)s);
  return 0;
}
