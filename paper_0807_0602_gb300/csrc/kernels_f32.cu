// FP32 and FP16-shifted-storage instantiations of the step and its
// reductions (FP32 arithmetic; FP64 only in the mass sums and the fronts).
#include "lbm_launch.cuh"

namespace sc {
template struct Launch<float>;
template struct Launch<__half>;
}  // namespace sc
