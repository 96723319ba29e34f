// dslash_f64.cu -- Dslash kernels with F64 links and vectors.
#include "dslash_kernel.cuh"

namespace hisq {
HISQ_DSLASH_INSTANTIATE(HISQ_F64, HISQ_F64)
}  // namespace hisq
