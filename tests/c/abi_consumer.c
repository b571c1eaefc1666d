/* A plain C99 consumer of include/rid.h: it compiles against the header alone,
 * links librid.so and exercises the calls that need no GPU (status strings and
 * the host-side argument checks).  Exit status 0 and "ok" on success. */
#include <stdio.h>
#include <string.h>

#include "rid.h"

static int failures = 0;

static void expect(int cond, const char* what) {
  if (!cond) {
    fprintf(stderr, "FAILED: %s\n", what);
    ++failures;
  }
}

int main(void) {
  rid_plan_t plan = NULL;
  size_t bytes = 0;
  double out[2] = {0.0, 0.0};

  expect(strncmp(rid_status_string(RID_OK), "RID_OK", 6) == 0, "status string of RID_OK");
  expect(strncmp(rid_status_string(RID_ERANK), "RID_ERANK", 9) == 0, "status string of RID_ERANK");
  expect(strncmp(rid_status_string(RID_ETIMEOUT), "RID_ETIMEOUT", 12) == 0, "status string of RID_ETIMEOUT");

  /* sizes out of range: m = 0, k > n, l < k */
  expect(rid_plan_create(&plan, 0, 10, 1, 2, RID_C128, RID_FP64_NATIVE, 1, NULL) == RID_EINVAL, "m = 0");
  expect(plan == NULL, "no plan after a rejected create");
  expect(rid_plan_create(&plan, 10, 4, 5, 6, RID_C128, RID_FP64_NATIVE, 1, NULL) == RID_EINVAL, "k > n");
  expect(rid_plan_create(&plan, 10, 10, 3, 2, RID_C128, RID_FP64_NATIVE, 1, NULL) == RID_EINVAL, "l < k");
  expect(rid_plan_create(NULL, 10, 10, 3, 4, RID_C128, RID_FP64_NATIVE, 1, NULL) == RID_EINVAL, "null handle");
  /* unsupported combinations */
  expect(rid_plan_create(&plan, 100, 100, 5, 600, RID_C128, RID_FP64_NATIVE, 1, NULL) == RID_EUNSUPPORTED,
         "l > 512");
  expect(rid_plan_create(&plan, 100, 100, 5, 8, RID_C128, RID_MIXED_BF16, 1, NULL) == RID_EUNSUPPORTED,
         "mixed mode needs complex64");
  expect(rid_plan_footprint(100, 100, 5, 8, RID_C128, RID_FP64_NATIVE, NULL) == RID_EINVAL, "footprint out = NULL");

  /* every call rejects a null plan before touching the device */
  expect(rid_sketch(NULL, NULL, 1, NULL, 1) == RID_EINVAL, "rid_sketch(NULL)");
  expect(rid_select(NULL, NULL, 1, NULL) == RID_EINVAL, "rid_select(NULL)");
  expect(rid_solve(NULL, NULL, 1, NULL, 1) == RID_EINVAL, "rid_solve(NULL)");
  expect(rid_error(NULL, NULL, 1, NULL, NULL, 1, 8, 1, out) == RID_EINVAL, "rid_error(NULL)");
  expect(rid_sync_status(NULL) == RID_EINVAL, "rid_sync_status(NULL)");
  expect(rid_plan_set_select_grid(NULL, 0) == RID_EINVAL, "rid_plan_set_select_grid(NULL)");
  expect(rid_plan_destroy(NULL) == RID_OK, "rid_plan_destroy(NULL) is a no-op");
  (void)bytes;

  if (failures) return 1;
  printf("ok\n");
  return 0;
}
