// dslash.cu -- precision dispatch and launch of the HISQ Dslash (kernel in dslash_kernel.cuh).
#include "dslash.cuh"

namespace hisq {

// largest N_inner in {8,4,2,1} dividing nrhs (N_inner <= 8; the paper finds spills beyond ~6
// on its hardware; registers on this GPU allow 8 for 32-bit storage)
int pick_inner(int prec, int nrhs)
{
    const int cap = (prec == HISQ_F64 || prec == HISQ_F64X) ? 4 : 8;
    for (int nr = cap; nr > 1; nr >>= 1)
        if (nrhs % nr == 0) return nr;
    return 1;
}

cudaError_t dslash_launch(int prec, int epi, const DslashArgs &a, int nreal, int nr, cudaStream_t st)
{
    switch (prec) {
    case HISQ_F64: return dslash_launch_HISQ_F64(epi, a, nreal, nr, st);
    case HISQ_F64X: return dslash_launch_HISQ_F64X(epi, a, nreal, nr, st);
    case HISQ_F32: return dslash_launch_HISQ_F32(epi, a, nreal, nr, st);
    case HISQ_F16: return dslash_launch_HISQ_F16(epi, a, nreal, nr, st);
    case HISQ_BF16: return dslash_launch_HISQ_BF16(epi, a, nreal, nr, st);
    }
    return cudaErrorInvalidValue;
}

DslashArgs make_dslash_args(hisq_ctx *ctx, int prec, int out_parity, const void *in, void *out, int nrhs,
                            size_t rhs_bytes)
{
    DslashArgs a{};
    const LinkStore &L = ctx->links[prec];
    a.g = ctx->g;
    a.p = out_parity;
    a.links = L.base;
    a.slot_bytes = L.slot_bytes;
    a.scale[0] = L.scale[0];
    a.scale[1] = L.scale[1];
    a.in = static_cast<const char *>(in);
    a.out = static_cast<char *>(out);
    a.rhs_bytes = rhs_bytes;
    a.nrhs = nrhs;
    return a;
}

int launch_dslash(hisq_ctx *ctx, int prec, int out_parity, const void *in, void *out, int nrhs, size_t rhs_bytes,
                  cudaStream_t st)
{
    const LinkStore &L = ctx->links[prec];
    DslashArgs a = make_dslash_args(ctx, prec, out_parity, in, out, nrhs, rhs_bytes);
    const int nr = pick_inner(prec, nrhs);
    cudaError_t e = dslash_launch(prec, 0, a, L.nreal, nr, st);
    if (e != cudaSuccess) return cuda_error(ctx, e, "dslash launch");
    return HISQ_OK;
}

}  // namespace hisq
