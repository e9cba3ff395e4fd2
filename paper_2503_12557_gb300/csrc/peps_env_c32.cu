// complex64 (complex PEPS) instantiation of the environment kernel k_env.
#define PEPS_PART_ENV
#include "peps_kernels_impl.cuh"

namespace peps {
PEPS_INST_ENV(cplx<float>)
}  // namespace peps
