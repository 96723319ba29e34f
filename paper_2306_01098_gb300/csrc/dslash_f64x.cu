// dslash_f64x.cu -- Dslash kernels with F64X links and vectors.
#include "dslash_kernel.cuh"

namespace hisq {
HISQ_DSLASH_INSTANTIATE(HISQ_F64X, HISQ_F64X)
}  // namespace hisq
