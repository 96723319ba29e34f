// dslash_bf16_f32.cu -- Dslash kernels with BF16 links, F32 vectors.
#include "dslash_kernel.cuh"

namespace hisq {
HISQ_DSLASH_INSTANTIATE(HISQ_BF16, HISQ_F32)
}  // namespace hisq
