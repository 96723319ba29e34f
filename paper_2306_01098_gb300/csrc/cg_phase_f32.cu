// cg_phase_f32.cu -- persistent CG phase kernels with HISQ_F32 sloppy links (cg_phase.cuh)
#include "cg_phase.cuh"

namespace hisq {
HISQ_PHASE_INSTANTIATE(HISQ_F32)
}  // namespace hisq
