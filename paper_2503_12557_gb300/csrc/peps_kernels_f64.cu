// FP64 instantiation of the sandwich kernels (k_row, k_pair), the parameter padding and the
// precision-independent combine step.
#define PEPS_DEFINE_COMMON
#define PEPS_PART_ROW
#include "peps_kernels_impl.cuh"

namespace peps {
PEPS_INST_ROW(double)
}  // namespace peps
