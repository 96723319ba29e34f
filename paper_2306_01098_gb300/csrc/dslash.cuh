// dslash.cuh -- arguments and launch entry of the Dslash kernels.
#pragma once

#include "internal.cuh"
#include "reduce.cuh"

namespace hisq {

constexpr int kDslashBlock = 128;

struct DslashArgs {
    Geom g;
    int p;                 // output parity
    const char *links;     // link store (16 slots)
    size_t slot_bytes;
    double scale[2];       // per link type multiplier (16-bit storage, 12-real c)
    const char *in;        // input field, parity 1-p, right-hand side 0
    char *out;             // output field, parity p
    size_t rhs_bytes;      // bytes between right-hand sides
    int nrhs;
    const Scalars *skip;   // if set: return at once when no right-hand side is active
    // normal-operator epilogue: out = m4 * pv - D in, <pv, out> reduced
    const char *pv;
    double m4;
    Reduce red;
};

DslashArgs make_dslash_args(hisq_ctx *ctx, int prec, int out_parity, const void *in, void *out, int nrhs,
                            size_t rhs_bytes);
cudaError_t dslash_launch(int prec, int epi, const DslashArgs &a, int nreal, int nr, cudaStream_t st);
int pick_inner(int prec, int nrhs);

cudaError_t dslash_launch_HISQ_F64(int epi, const DslashArgs &a, int nreal, int nr, cudaStream_t st);
cudaError_t dslash_launch_HISQ_F64X(int epi, const DslashArgs &a, int nreal, int nr, cudaStream_t st);
cudaError_t dslash_launch_HISQ_F32(int epi, const DslashArgs &a, int nreal, int nr, cudaStream_t st);
cudaError_t dslash_launch_HISQ_F16(int epi, const DslashArgs &a, int nreal, int nr, cudaStream_t st);
cudaError_t dslash_launch_HISQ_BF16(int epi, const DslashArgs &a, int nreal, int nr, cudaStream_t st);

}  // namespace hisq
