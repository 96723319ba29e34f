// rational.cu -- a rational function of A applied to a vector from one multi-shift solve,
//   r(A) b = alpha0 b + sum_s alpha_s (A + sigma_s)^-1 b,
// the form in which RHMC's heat bath and force use the solver (Sec. 3.2 "Inverters": the
// multi-shift inverter for the rational approximation).  The coefficients are the caller's:
// the paper prints none.
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace hisq {

constexpr int kMaxTerms = 64; // the multi-shift solver's limit

// x = alpha0 b + sum_s alpha_s xs[s] in FP64, terms added in index order
__global__ void __launch_bounds__(256) k_rational_combine(const double2 *b, const double2 *const *xs, const double *alpha,
                                                          int n, double alpha0, double2 *x, size_t nc)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nc; i += (size_t)gridDim.x * blockDim.x) {
        const double2 bv = b[i];
        double re = alpha0 * bv.x, im = alpha0 * bv.y;
        for (int s = 0; s < n; s++) {
            const double2 v = xs[s][i];
            re = fma(alpha[s], v.x, re);
            im = fma(alpha[s], v.y, im);
        }
        x[i] = make_double2(re, im);
    }
}

}  // namespace hisq

using namespace hisq;

extern "C" int hisq_rational_apply(hisq_ctx *ctx, double m, int nterm, const double *alpha, const double *sigma,
                                   double alpha0, const double *b, double *x, const hisq_solve_opts *opts,
                                   hisq_stats *stats, double *residuals)
{
    if (!ctx) return HISQ_EINVAL;
    if (!alpha || !sigma || !b || !x || nterm < 1 || nterm > kMaxTerms || !(m >= 0.0) || !std::isfinite(alpha0))
        return set_error(ctx, HISQ_EINVAL, "hisq_rational_apply: bad argument");
    for (int s = 0; s < nterm; s++)
        if (!std::isfinite(alpha[s]) || !(sigma[s] >= 0.0) || !std::isfinite(sigma[s]))
            return set_error(ctx, HISQ_EINVAL, "hisq_rational_apply: bad coefficient or shift");
    const uint32_t Vh = ctx->g.Vh;
    const size_t nc = (size_t)Vh * 3, vb = nc * sizeof(double2);
    {
        const char *pb = reinterpret_cast<const char *>(b), *px = reinterpret_cast<const char *>(x);
        if (pb < px + vb && px < pb + vb) return set_error(ctx, HISQ_EINVAL, "hisq_rational_apply: b and x overlap");
    }
    hisq_solve_opts o;
    if (opts) o = *opts;
    else hisq_solve_opts_default(&o);
    if (o.host_buffers) return set_error(ctx, HISQ_EINVAL, "hisq_rational_apply: device buffers only");
    cudaSetDevice(ctx->device);
    // workspace for this call: the nterm solutions (zero initial guesses), their pointer
    // table and the coefficients on the device
    std::vector<double *> xs(nterm, nullptr);
    double2 **d_xs = nullptr;
    double *d_alpha = nullptr;
    auto release = [&]() {
        for (double *p : xs)
            if (p) cudaFree(p);
        if (d_xs) cudaFree(d_xs);
        if (d_alpha) cudaFree(d_alpha);
    };
    bool ok = cudaMalloc((void **)&d_xs, sizeof(double2 *) * nterm) == cudaSuccess &&
              cudaMalloc((void **)&d_alpha, sizeof(double) * nterm) == cudaSuccess;
    for (int s = 0; ok && s < nterm; s++)
        ok = cudaMalloc((void **)&xs[s], vb) == cudaSuccess && cudaMemset(xs[s], 0, vb) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        release();
        return set_error(ctx, HISQ_ENOMEM, "hisq_rational_apply: workspace");
    }
    // every shifted system to opts->tol (the multi-shift solve synchronises before returning)
    const int rc = hisq_multishift_cg(ctx, m, nterm, sigma, b, xs.data(), nullptr, &o, stats, residuals);
    if (rc != HISQ_OK && rc != HISQ_ENOTCONVERGED) {
        release();
        return rc;
    }
    cudaStream_t st = (cudaStream_t)o.stream;
    std::vector<double2 *> table(nterm);
    for (int s = 0; s < nterm; s++) table[s] = reinterpret_cast<double2 *>(xs[s]);
    cudaError_t e = cudaMemcpyAsync(d_xs, table.data(), sizeof(double2 *) * nterm, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_alpha, alpha, sizeof(double) * nterm, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        const unsigned grid = (unsigned)std::min<size_t>((nc + 255) / 256, 8ull * ctx->sm_count);
        k_rational_combine<<<grid, 256, 0, st>>>(reinterpret_cast<const double2 *>(b), d_xs, d_alpha, nterm, alpha0,
                                                 reinterpret_cast<double2 *>(x), nc);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st); // the workspace is released below
    release();
    if (e != cudaSuccess) return cuda_error(ctx, e, "hisq_rational_apply: combination");
    if (rc != HISQ_OK) return set_error(ctx, rc, "hisq_rational_apply: a shifted system missed the tolerance");
    return HISQ_OK;
}
