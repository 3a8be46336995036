// FP32 instantiation of the step (standard species) and of its reductions
// (FP32 arithmetic; FP64 only in the mass sums and the fronts).
#include "lbm_launch.cuh"

namespace sc {
template struct Launch<float>;
template struct Step<float, false>;
}  // namespace sc
