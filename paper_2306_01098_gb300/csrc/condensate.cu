// condensate.cu -- stochastic estimate of the chiral condensate (1/V) Tr M^-1 with the
// multi-RHS CG of Sec. 3.2, the measurement the paper runs on its ensembles (Sec. 3).
//
// For M = 2m + D, M^-1 = M^+ (M M^+)^-1 = (2m - D)(4m^2 - D^2)^-1; D only connects even and
// odd sites, so the diagonal blocks are 2m (4m^2 - D^2)^-1, and the odd block
// (4m^2 - D_oe D_eo)^-1 has the spectrum of the even block A^-1: Tr M^-1 = 4m Tr_e A^-1.
// Tr_e A^-1 is estimated by Re <eta_k, A^-1 eta_k> averaged over the caller's noise vectors
// eta_k on even sites (Z2 or Gaussian: unbiased when E[eta eta^+] = 1), solved by multi-RHS CG,
// up to 64 noise vectors per solve.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace hisq {

// per noise vector k and block: Re <eta_k, x_k> partial sums (FP64), grid (blocks, nnoise)
__global__ void __launch_bounds__(256) k_noise_dots(const double2 *eta, const double2 *x, size_t nc, double *partials)
{
    __shared__ double ws[8];
    const size_t off = (size_t)blockIdx.y * nc;
    double acc = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nc; i += (size_t)gridDim.x * blockDim.x) {
        const double2 a = eta[off + i], b = x[off + i];
        acc = fma(a.x, b.x, fma(a.y, b.y, acc));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) ws[w] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) s += ws[i];
        partials[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
    }
}

}  // namespace hisq

using namespace hisq;

extern "C" int hisq_condensate(hisq_ctx *ctx, double m, int nnoise, const double *eta, const hisq_solve_opts *opts,
                               double *samples, double *pbp, hisq_stats *stats)
{
    if (!ctx) return HISQ_EINVAL;
    if (!eta || nnoise < 1 || nnoise > 4096 || !(m > 0.0) || !std::isfinite(m))
        return set_error(ctx, HISQ_EINVAL, "hisq_condensate: bad argument");
    hisq_solve_opts o;
    if (opts) o = *opts;
    else hisq_solve_opts_default(&o);
    if (o.host_buffers) return set_error(ctx, HISQ_EINVAL, "hisq_condensate: device buffers only");
    o.zero_guess = 1;
    cudaSetDevice(ctx->device);
    const size_t nc = (size_t)ctx->g.Vh * 3, vb = nc * sizeof(double2);
    const int nblk = (int)std::min<size_t>((nc + 255) / 256, 2ull * ctx->sm_count);
    double *x = nullptr, *partials = nullptr;
    auto release = [&]() {
        if (x) cudaFree(x);
        if (partials) cudaFree(partials);
    };
    if (cudaMalloc((void **)&x, vb * nnoise) != cudaSuccess ||
        cudaMalloc((void **)&partials, sizeof(double) * nblk * nnoise) != cudaSuccess) {
        cudaGetLastError();
        release();
        return set_error(ctx, HISQ_ENOMEM, "hisq_condensate: workspace");
    }
    // A x_k = eta_k, up to 64 noise vectors per multi-RHS solve (each synchronises before
    // returning); the statistics add up over the solves (iterations: the largest)
    int rc = HISQ_OK;
    if (stats) std::memset(stats, 0, sizeof(*stats));
    for (int k0 = 0; k0 < nnoise; k0 += 64) {
        const int n = std::min(64, nnoise - k0);
        hisq_stats cs{};
        const int r = hisq_cg(ctx, m, eta + (size_t)k0 * nc * 2, x + (size_t)k0 * nc * 2, n, &o, &cs, nullptr);
        if (r != HISQ_OK && r != HISQ_ENOTCONVERGED) {
            release();
            return r;
        }
        if (r != HISQ_OK) rc = r;
        if (stats) {
            stats->iterations = std::max(stats->iterations, cs.iterations);
            stats->reliable_updates += cs.reliable_updates;
            stats->true_residual = std::max(stats->true_residual, cs.true_residual);
            stats->iterated_residual = std::max(stats->iterated_residual, cs.iterated_residual);
            stats->seconds += cs.seconds;
            stats->dslash_calls += cs.dslash_calls;
            stats->dslash_ms += cs.dslash_ms;
            stats->dslash_timed += cs.dslash_timed;
            stats->bytes_moved += cs.bytes_moved;
            stats->kernels += cs.kernels;
        }
    }
    cudaStream_t st = (cudaStream_t)o.stream;
    k_noise_dots<<<dim3(nblk, nnoise), 256, 0, st>>>(reinterpret_cast<const double2 *>(eta),
                                                     reinterpret_cast<const double2 *>(x), nc, partials);
    std::vector<double> h((size_t)nblk * nnoise);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), partials, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    release();
    if (e != cudaSuccess) return cuda_error(ctx, e, "hisq_condensate: noise dot products");
    double mean = 0.0;
    for (int k = 0; k < nnoise; k++) {
        double s = 0.0;
        for (int b = 0; b < nblk; b++) s += h[(size_t)k * nblk + b]; // fixed order
        if (samples) samples[k] = s;
        mean += s;
    }
    mean /= nnoise;
    const double V = 2.0 * (double)ctx->g.Vh;
    if (pbp) *pbp = 4.0 * m * mean / V;
    if (rc != HISQ_OK) return set_error(ctx, rc, "hisq_condensate: a noise solve missed the tolerance");
    return HISQ_OK;
}
