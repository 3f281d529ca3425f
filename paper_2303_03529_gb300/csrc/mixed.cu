// Mixed-precision (fp16 / bf16 tensor-core) expansion chain.
#include "common.cuh"

int sxl_mixed_supported(sxl_ctx* c) {
  return sxl_fail(c, SXL_E_UNSUPPORTED, "mixed precision not built");
}
void sxl_mixed_free(sxl_ctx*) {}
