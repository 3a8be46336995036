// FP16-shifted-storage instantiation of the step (standard species) and of
// its reductions (FP32 arithmetic on decoded populations).
#include "lbm_launch.cuh"

namespace sc {
template struct Launch<__half>;
template struct Step<__half, false>;
}  // namespace sc
