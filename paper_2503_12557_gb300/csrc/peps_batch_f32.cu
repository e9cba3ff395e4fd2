// F32 instantiation of the ragged multi-instance batch kernel k_batch.
#define PEPS_PART_BATCH
#include "peps_kernels_impl.cuh"

namespace peps {
PEPS_INST_BATCH(float)
}  // namespace peps
