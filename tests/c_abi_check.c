/* A plain C99 caller of the library (no C++, no Python): it includes the public header, links
 * libtbpm.so and uses the entry points that need no GPU, the way a C application would.
 * Prints one line per check; the test compares the numbers with the oracle and exits non-zero
 * on any mismatch of the status codes. */
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "tbpm.h"

int main(void) {
  int bad = 0;
  const double pi = 3.14159265358979323846;
  printf("truncation %lld %lld %lld\n", (long long)tbpm_truncation_order(pi),
         (long long)tbpm_truncation_order(4.0 * pi), (long long)tbpm_truncation_order(100.0 * pi));

  int64_t counts[3] = {0, 0, 0};
  if (tbpm_block_counts(2048, 40, pi, counts) != TBPM_OK) bad = 1;
  printf("counts %lld %lld %lld\n", (long long)counts[0], (long long)counts[1], (long long)counts[2]);
  printf("bopt %lld\n", (long long)tbpm_block_opt(2048, pi, 1.0, 0.05, 256));

  /* invalid arguments come back as status codes with a message, never as a crash */
  if (tbpm_block_counts(0, 1, pi, counts) != TBPM_EINVAL) bad = 1;
  if (strlen(tbpm_last_error()) == 0) bad = 1;
  tbpm_lattice* lat = NULL;
  if (tbpm_lattice_create(NULL, NULL, &lat) != TBPM_EINVAL || lat != NULL) bad = 1;
  if (tbpm_moments(NULL, NULL, NULL, NULL) != TBPM_EINVAL) bad = 1;
  if (tbpm_wait_probe(NULL, 0, 0.01) != TBPM_EINVAL) bad = 1;
  uint64_t words[3] = {1, 1, 1};
  if (tbpm_debug_status(NULL, words) != TBPM_EINVAL) bad = 1;
  printf("errors %s\n", bad ? "wrong" : "ok");
  return bad;
}
