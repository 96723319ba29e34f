// dslash_bf16.cu -- Dslash kernels with BF16 links and vectors.
#include "dslash_kernel.cuh"

namespace hisq {
HISQ_DSLASH_INSTANTIATE(HISQ_BF16, HISQ_BF16)
}  // namespace hisq
