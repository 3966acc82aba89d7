/*
 * The C ABI used from plain C, with no GPU: the host-only symbolic analysis
 * (Section 4.4) of a 2x2x1 grid's 3x3-block pattern, each cell joined to its
 * grid neighbours.  Prints the status text, the schedule, the set count and
 * the permutation for the level and colour schedules; exits non-zero on any
 * error status.
 */
#include <stdio.h>

#include "opm_bsr.h"

int main(void) {
  /* cells 0..3 at (x, y) = (0,0), (1,0), (0,1), (1,1); sorted columns, diagonal present */
  const int32_t rowptr[5] = {0, 3, 6, 9, 12};
  const int32_t colidx[12] = {0, 1, 2, 0, 1, 3, 0, 2, 3, 1, 2, 3};
  opm_options o;
  opm_options_default(&o);
  if (o.schedule != OPM_SCHED_AUTO || o.precision != OPM_PREC_FP64) return 2;
  const int32_t schedules[2] = {OPM_SCHED_LEVEL, OPM_SCHED_COLOUR};
  for (int q = 0; q < 2; ++q) {
    int32_t perm[4];
    opm_analysis_info info;
    opm_status st = opm_bsr_analyse(4, rowptr, colidx, NULL, schedules[q], perm, &info);
    printf("%s schedule=%d nsets=%d lower=%lld upper=%lld perm=%d,%d,%d,%d\n", opm_status_str(st), info.schedule,
           info.nsets, (long long)info.nnzb_lower, (long long)info.nnzb_upper, perm[0], perm[1], perm[2], perm[3]);
    if (st != OPM_OK) return 1;
  }
  /* a pattern error: row 1 without its diagonal block */
  const int32_t bad_col[12] = {0, 1, 2, 0, 2, 3, 0, 2, 3, 1, 2, 3};
  opm_status st = opm_bsr_analyse(4, rowptr, bad_col, NULL, OPM_SCHED_LEVEL, NULL, NULL);
  printf("%s row=%d\n", opm_status_str(st), opm_last_error_row(NULL));
  return st == OPM_ERR_NO_DIAG ? 0 : 3;
}
