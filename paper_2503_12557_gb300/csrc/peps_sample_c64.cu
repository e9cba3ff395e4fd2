// complex128 (complex PEPS) instantiation of the Metropolis sampler kernel k_sample.
#define PEPS_PART_SAMPLE
#include "peps_kernels_impl.cuh"

namespace peps {
PEPS_INST_SAMPLE(cplx<double>)
}  // namespace peps
