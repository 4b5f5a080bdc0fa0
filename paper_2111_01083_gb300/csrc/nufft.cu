// NUFFT far-field path (Sec. 6, Eqs. fastanterp, fastinterp).
#include "pfmm_impl.h"
namespace pfmm {
cudaError_t launch_far_nufft(const pfmm_plan*, char*, int64_t, int64_t, bool, double*, double*, cudaStream_t) {
  return cudaErrorNotSupported;
}
}  // namespace pfmm
