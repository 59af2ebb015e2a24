// Mixed-precision H_eff products (split-TF32 tensor-core path).
#include "common.h"

namespace vb {

size_t heff_mixed_work_bytes(const vb_mpo *mpo, int site, int two_site, int mL, int mR) {
  (void)mpo; (void)site; (void)two_site; (void)mL; (void)mR;
  return 0;
}

vb_status heff_mixed_apply(const vb_mpo *mpo, int site, int two_site, int mL, int mR, const cd *L,
                           const cd *R, const cd *x, cd *y, void *work, size_t work_bytes,
                           cudaStream_t st) {
  (void)mpo; (void)site; (void)two_site; (void)mL; (void)mR; (void)L; (void)R; (void)x; (void)y;
  (void)work; (void)work_bytes; (void)st;
  return fail(VB_EINVAL, "mixed-precision path not available in this build");
}

}  // namespace vb
