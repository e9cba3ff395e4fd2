// float instantiation of the direct-sampling kernels (k_dl_env, k_direct).
#include "peps_direct.cuh"

namespace peps {
PEPS_INST_DIRECT(float)
}  // namespace peps
