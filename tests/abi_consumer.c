/* A plain C99 program that uses libsrp through include/libsrp.h alone, as a C caller
 * would: it fills a plan description for a 4-microphone square array, sizes the plan, and
 * checks the host-side argument checks of the entry points (status codes, cleared outputs,
 * the thread's last-error message).  None of the calls it makes needs a GPU.  Exit status 0
 * and "ok" on stdout when every check holds. */
#include <stdio.h>
#include <string.h>

#include "libsrp.h"

static int fails = 0;
#define CHECK(cond)                                                      \
  do {                                                                   \
    if (!(cond)) {                                                       \
      fprintf(stderr, "line %d: %s (%s)\n", __LINE__, #cond, srp_last_error()); \
      ++fails;                                                           \
    }                                                                    \
  } while (0)

int main(void) {
  double mics[4][3] = {{0, 0, 0}, {0.2, 0, 0}, {0, 0.2, 0}, {0.2, 0.2, 0}};
  double grid[100][3];
  srp_plan_desc d;
  size_t conv = 0, sspi = 0;
  srp_plan_t plan;
  srp_server_t server;
  srp_server_desc sd;
  int i;
  for (i = 0; i < 100; ++i) {
    grid[i][0] = 0.4 * (i % 10);
    grid[i][1] = 0.4 * (i / 10);
    grid[i][2] = 1.0;
  }
  memset(&d, 0, sizeof d);
  d.M = 4;
  d.mic_xyz = &mics[0][0];
  d.J = 100;
  d.grid_xyz = &grid[0][0];
  d.fs = 16000.0;
  d.N = 512;
  d.window = SRP_WIN_SQRT_HANN;
  d.c = 340.0;
  d.n_aux = 2;
  d.method = SRP_CONV;
  d.precision = SRP_BF16;
  d.max_frames = 64;

  /* sizing needs no device */
  CHECK(srp_plan_estimate_bytes(&d, &conv) == SRP_OK && conv > 0);
  CHECK(srp_last_error()[0] == '\0');
  d.method = SRP_SSPI;
  d.taps_per_loc_pair = 2.0;
  CHECK(srp_plan_estimate_bytes(&d, &sspi) == SRP_OK && sspi > 0);
  CHECK(srp_plan_estimate_bytes(&d, NULL) == SRP_EINVAL);
  CHECK(srp_plan_estimate_bytes(NULL, &sspi) == SRP_EINVAL);

  /* invalid descriptions are refused before any device work; *out is cleared */
  plan = (srp_plan_t)&d;
  d.N = 500; /* not a power of two */
  CHECK(srp_plan_create(&d, NULL, &plan) == SRP_EINVAL && plan == NULL);
  CHECK(strlen(srp_last_error()) > 0);
  d.N = 512;
  d.precision = 7;
  CHECK(srp_plan_create(&d, NULL, &plan) == SRP_EINVAL && plan == NULL);
  d.precision = SRP_BF16;
  d.taps_per_loc_pair = 0.0;
  CHECK(srp_plan_create(&d, NULL, &plan) == SRP_EINVAL && plan == NULL);
  d.taps_per_loc_pair = 2.0;
  CHECK(srp_plan_create(&d, NULL, NULL) == SRP_EINVAL);
  CHECK(srp_plan_create_from_file(&d, NULL, NULL, &plan) == SRP_EINVAL && plan == NULL);

  /* a NULL plan is an argument error, not a crash */
  CHECK(srp_map(NULL, NULL, 1, NULL, NULL, NULL) == SRP_EINVAL);
  CHECK(srp_plan_status(NULL, NULL) == SRP_EINVAL);
  CHECK(srp_plan_save(NULL, "x.plan") == SRP_EINVAL);
  srp_destroy(NULL);

  /* the server and the test hooks check their arguments on the host too */
  memset(&sd, 0, sizeof sd);
  sd.hbm_budget = (size_t)1 << 30;
  sd.max_sessions = 4;
  sd.max_batch = 3; /* not a power of two */
  sd.streams = 2;
  sd.slots_per_session = 2;
  sd.pending_frames = 64;
  server = (srp_server_t)&sd;
  CHECK(srp_server_create(&sd, &server) == SRP_EINVAL && server == NULL);
  CHECK(srp_debug_fail_allocations(-1, 1) == SRP_EINVAL);
  CHECK(srp_debug_fail_allocations(0, 0) == SRP_OK);
  CHECK(srp_server_now() >= 0.0);

  if (fails) return 1;
  printf("ok\n");
  return 0;
}
