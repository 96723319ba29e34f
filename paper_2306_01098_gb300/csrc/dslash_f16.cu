// dslash_f16.cu -- Dslash kernels with F16 links and vectors.
#include "dslash_kernel.cuh"

namespace hisq {
HISQ_DSLASH_INSTANTIATE(HISQ_F16, HISQ_F16)
}  // namespace hisq
