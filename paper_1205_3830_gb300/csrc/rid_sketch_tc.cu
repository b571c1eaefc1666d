// Tensor-core sketch paths (FP64-emulated and mixed precision).
#include "rid_internal.cuh"

rid_status rid_tc_plan_init(rid_plan_s* p) {
  (void)p;
  return RID_EUNSUPPORTED;
}

void rid_tc_plan_free(rid_plan_s* p) { (void)p; }

cudaError_t rid_tc_sketch(const rid_plan_s* p, const void* A, int64_t lda, double2* Y, int64_t ldy) {
  (void)p; (void)A; (void)lda; (void)Y; (void)ldy;
  return cudaErrorNotSupported;
}
