// Step kernels for species with a free rest fraction alpha_k or a molecular
// mass m_k != 1 (Eqs. 3-5, 7, 8), FP32 storage; separate from the standard
// instantiation so that both compile in parallel.
#include "lbm_launch.cuh"

namespace sc {
template struct Step<float, true>;
}  // namespace sc
