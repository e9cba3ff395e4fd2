// FP64 instantiation of the contraction kernels (and the precision-independent combine step).
#define PEPS_DEFINE_COMMON
#include "peps_kernels_impl.cuh"

namespace peps {
PEPS_INST(double)
}  // namespace peps
