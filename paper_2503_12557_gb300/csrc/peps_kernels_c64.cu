// complex128 (complex PEPS) instantiation of the sandwich kernels (k_row, k_pair) and the parameter padding.
#define PEPS_PART_ROW
#include "peps_kernels_impl.cuh"

namespace peps {
PEPS_INST_ROW(cplx<double>)
}  // namespace peps
