// cg_phase_bf16.cu -- persistent CG phase kernels with HISQ_BF16 sloppy links (cg_phase.cuh)
#include "cg_phase.cuh"

namespace hisq {
HISQ_PHASE_INSTANTIATE(HISQ_BF16)
}  // namespace hisq
