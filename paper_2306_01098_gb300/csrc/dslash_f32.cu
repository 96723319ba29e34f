// dslash_f32.cu -- Dslash kernels with F32 links and vectors.
#include "dslash_kernel.cuh"

namespace hisq {
HISQ_DSLASH_INSTANTIATE(HISQ_F32, HISQ_F32)
}  // namespace hisq
