// cplx<float> instantiation of the variational-bound kernel k_bound.
#define PEPS_PART_BOUND
#include "peps_kernels_impl.cuh"

namespace peps {
PEPS_INST_BOUND(cplx<float>)
}  // namespace peps
