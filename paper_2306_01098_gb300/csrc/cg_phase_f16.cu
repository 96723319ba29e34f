// cg_phase_f16.cu -- persistent CG phase kernels with HISQ_F16 sloppy links (cg_phase.cuh)
#include "cg_phase.cuh"

namespace hisq {
HISQ_PHASE_INSTANTIATE(HISQ_F16)
}  // namespace hisq
