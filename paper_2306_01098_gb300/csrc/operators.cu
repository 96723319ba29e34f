// operators.cu -- C entry points that apply D and A = 4 m^2 - D_eo D_oe (Sec. 3.2, 5.1).
#include <cstring>

#include "dslash.cuh"

namespace hisq {

static bool overlap(const void *a, size_t na, const void *b, size_t nb)
{
    const char *x = static_cast<const char *>(a), *y = static_cast<const char *>(b);
    return x < y + nb && y < x + na;
}

static int check_prec(hisq_ctx *ctx, int prec)
{
    if (prec < 0 || prec >= HISQ_NPREC) return set_error(ctx, HISQ_EINVAL, "unknown precision");
    if (!ctx->links[prec].built) return set_error(ctx, HISQ_ENOTBUILT, "precision not built in this context");
    return HISQ_OK;
}

// t = D_oe in; out = m4 in - D_eo t (normal operator on even sites), internal layout.
// tune = false: use a shape already tuned for this key, else the default (no timing runs)
int apply_mdagm(hisq_ctx *ctx, int prec, double m, const void *in, void *tmp, void *out, int nrhs, size_t rhs_bytes,
                cudaStream_t st, const Reduce *red, bool tune)
{
    const LinkStore &L = ctx->links[prec];
    const int pv = vector_prec(prec);
    DslashShape sh;
    if (tune) {
        sh = dslash_shape(ctx, prec, pv, nrhs, in, tmp, rhs_bytes, st);
    } else {
        auto it = ctx->tune.find(tune_key(prec, pv, nrhs));
        sh.nr = it != ctx->tune.end() ? it->second.nr : pick_inner(pv, nrhs);
        sh.ds = it != ctx->tune.end() ? it->second.ds : (ctx->g.Vh < (1u << 20) ? 2 : 1);
        sh.order = it != ctx->tune.end() ? it->second.order : 0;
        sh.bs = it != ctx->tune.end() ? it->second.bs : kDslashBlock;
        sh.rg = it != ctx->tune.end() ? it->second.rg : 1;
    }
    DslashArgs a = make_dslash_args(ctx, prec, 1, in, tmp, nrhs, rhs_bytes);
    cudaError_t e = dslash_launch(prec, pv, 0, a, L.nreal, sh, st);
    if (e != cudaSuccess) return cuda_error(ctx, e, "dslash D_oe");
    DslashArgs b = make_dslash_args(ctx, prec, 0, tmp, out, nrhs, rhs_bytes);
    b.pv = static_cast<const char *>(in);
    b.m4 = 4.0 * m * m;
    if (red) b.red = *red;
    e = dslash_launch(prec, pv, 1, b, L.nreal, sh, st);
    if (e != cudaSuccess) return cuda_error(ctx, e, "dslash D_eo + epilogue");
    return HISQ_OK;
}

}  // namespace hisq

using namespace hisq;

extern "C" {

int hisq_dslash(hisq_ctx *ctx, int out_parity, const double *in, double *out, int nrhs, int prec, void *stream)
{
    if (!ctx) return HISQ_EINVAL;
    if (!in || !out || nrhs < 1 || (out_parity != 0 && out_parity != 1))
        return set_error(ctx, HISQ_EINVAL, "hisq_dslash: bad argument");
    HISQ_CUDA(ctx, cudaSetDevice(ctx->device));
    int rc = check_prec(ctx, prec);
    if (rc) return rc;
    const size_t bytes = (size_t)nrhs * ctx->g.Vh * 48;
    if (overlap(in, bytes, out, bytes)) return set_error(ctx, HISQ_EINVAL, "hisq_dslash: in and out overlap");
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == HISQ_F64) return launch_dslash(ctx, HISQ_F64, out_parity, in, out, nrhs, (size_t)ctx->g.Vh * 48, st);
    const int pv = vector_prec(prec);
    const size_t rb = (size_t)ctx->g.VhPad * spinor_bytes(pv);
    rc = ensure_workspace(ctx, 2 * rb * nrhs);
    if (rc) return rc;
    char *t_in = static_cast<char *>(ctx->ws), *t_out = t_in + rb * nrhs;
    if ((rc = launch_import(ctx, pv, in, t_in, nrhs, rb, st))) return rc;
    if ((rc = launch_dslash2(ctx, prec, pv, out_parity, t_in, t_out, nrhs, rb, st))) return rc;
    return launch_export(ctx, pv, t_out, out, nrhs, rb, st);
}

int hisq_dslash_field(hisq_ctx *ctx, int out_parity, const hisq_field *in, hisq_field *out, void *stream)
{
    if (!ctx) return HISQ_EINVAL;
    if (!in || !out || in->prec != out->prec || in->nrhs != out->nrhs || in == out || in->ctx != ctx ||
        out->ctx != ctx || (out_parity != 0 && out_parity != 1))
        return set_error(ctx, HISQ_EINVAL, "hisq_dslash_field: bad argument");
    HISQ_CUDA(ctx, cudaSetDevice(ctx->device));
    int rc = check_prec(ctx, in->prec);
    if (rc) return rc;
    return launch_dslash(ctx, in->prec, out_parity, in->data, out->data, in->nrhs, in->rhs_bytes, (cudaStream_t)stream);
}

int hisq_mdagm(hisq_ctx *ctx, double m, const double *in, double *out, int nrhs, int prec, void *stream)
{
    if (!ctx) return HISQ_EINVAL;
    if (!in || !out || nrhs < 1) return set_error(ctx, HISQ_EINVAL, "hisq_mdagm: bad argument");
    HISQ_CUDA(ctx, cudaSetDevice(ctx->device));
    int rc = check_prec(ctx, prec);
    if (rc) return rc;
    const size_t bytes = (size_t)nrhs * ctx->g.Vh * 48;
    if (overlap(in, bytes, out, bytes)) return set_error(ctx, HISQ_EINVAL, "hisq_mdagm: in and out overlap");
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == HISQ_F64) {
        const size_t rb = (size_t)ctx->g.Vh * 48;
        if ((rc = ensure_workspace(ctx, rb * nrhs))) return rc;
        return apply_mdagm(ctx, prec, m, in, ctx->ws, out, nrhs, rb, st, nullptr, true);
    }
    const int pv = vector_prec(prec);
    const size_t rb = (size_t)ctx->g.VhPad * spinor_bytes(pv);
    if ((rc = ensure_workspace(ctx, 3 * rb * nrhs))) return rc;
    char *t_in = static_cast<char *>(ctx->ws), *t_tmp = t_in + rb * nrhs, *t_out = t_tmp + rb * nrhs;
    if ((rc = launch_import(ctx, pv, in, t_in, nrhs, rb, st))) return rc;
    if ((rc = apply_mdagm(ctx, prec, m, t_in, t_tmp, t_out, nrhs, rb, st, nullptr, true))) return rc;
    return launch_export(ctx, pv, t_out, out, nrhs, rb, st);
}

}  // extern "C"
