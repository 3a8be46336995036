// FP64 step kernels for species with a free rest fraction alpha_k or a
// molecular mass m_k != 1 (Eqs. 3-5, 7, 8).  Built with --fmad=false like
// the standard FP64 instantiation: the canonical order, each operation
// rounded on its own.
#include "lbm_launch.cuh"

namespace sc {
template struct Step<double, true>;
}  // namespace sc
