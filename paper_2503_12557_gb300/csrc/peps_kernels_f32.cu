// FP32 instantiation of the contraction kernels.
#include "peps_kernels_impl.cuh"

namespace peps {
PEPS_INST(float)
}  // namespace peps
