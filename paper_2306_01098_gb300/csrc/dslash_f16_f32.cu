// dslash_f16_f32.cu -- Dslash kernels with F16 links, F32 vectors.
#include "dslash_kernel.cuh"

namespace hisq {
HISQ_DSLASH_INSTANTIATE(HISQ_F16, HISQ_F32)
}  // namespace hisq
