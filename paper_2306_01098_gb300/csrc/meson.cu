// meson.cu -- point-source staggered meson correlators along any direction (the hadronic
// correlation functions with point sources of Sec. 3.3), from one three-RHS CG solve.
//
// G = M^-1 on the three colour point sources at site y, M = 2m + D on the full lattice. The
// even-odd reduction of the solvers (Sec. 3.2): for M (x_e, x_o) = (b_e, b_o),
//   A x_e = 2m b_e - D_eo b_o,  A = 4m^2 - D_eo D_oe,   x_o = (b_o - D_oe x_e) / (2m).
// A point source lives on one parity, so the even right-hand side is 2m b_e (even source) or
// -D_eo b_o (odd source). The correlators
//   C[S][tau] = sum_{x: (x_d - y_d) mod N_d = tau} (-1)^(sum_{i in S} (x_{e_i} - y_{e_i}))
//               sum_{a,b} |G_ab(x, y)|^2,
// e_0 < e_1 < e_2 the directions other than d, are the eight local staggered channels
// (S = 0: the Goldstone pion). The slice sums are reduced per block in a fixed order and the
// blocks' partials summed on the host in a fixed order: the result does not depend on timing.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace hisq {

namespace meson {

constexpr int kBlock = 256;

// the three colour point sources at canonical half index s: b[c][s][c] = v
__global__ void k_point(double2 *b, uint32_t Vh, uint32_t s, double v)
{
    const int c = threadIdx.x;
    if (c < 3) b[((size_t)c * Vh + s) * 3 + c] = make_double2(v, 0.0);
}

// the propagator [3][V][3] (canonical, even half first) from the even solution and D_oe of it:
// G_e = sgn x_e, G_o = (b_o - sgn D_oe x_e) / (2m); sgn = -1 when the even system was solved
// for D_eo b_o (odd source), b_o the odd point source (none for an even source)
__global__ void k_assemble(const double2 *xe, const double2 *to, double2 *G, uint32_t Vh, double sgn, double m2,
                           int src_odd, uint32_t s0)
{
    const size_t n = (size_t)Vh * 3;
    const int c = blockIdx.y;
    const double2 *xc = xe + (size_t)c * n, *tc = to + (size_t)c * n;
    double2 *ge = G + (size_t)c * 2 * n, *go = ge + n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double2 a = xc[i], t = tc[i];
        ge[i] = make_double2(sgn * a.x, sgn * a.y);
        const double bo = (src_odd && i == (size_t)s0 * 3 + c) ? 1.0 : 0.0;
        go[i] = make_double2((bo - sgn * t.x) / m2, (-sgn * t.y) / m2);
    }
}

// w[lex] = sum over source and sink colours of |G|^2 at every site, in lexicographic order
__global__ void k_weights(Geom g, const double2 *G, double *w)
{
    const size_t n = (size_t)g.Vh * 3, V = 2 * (size_t)g.Vh;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < V; k += (size_t)gridDim.x * blockDim.x) {
        const int p = k >= g.Vh;
        const uint32_t s = (uint32_t)(k - (p ? g.Vh : 0));
        const Site c = site_coords(g, s, p);
        double acc = 0.0;
#pragma unroll
        for (int col = 0; col < 3; col++) {
            const double2 *gc = G + (size_t)col * 2 * n + k * 3;
#pragma unroll
            for (int a = 0; a < 3; a++) acc = fma(gc[a].x, gc[a].x, fma(gc[a].y, gc[a].y, acc));
        }
        const size_t lex = c.x + (size_t)g.n[0] * (c.y + (size_t)g.n[1] * (c.z + (size_t)g.n[2] * c.t));
        w[lex] = acc;
    }
}

struct SliceArgs {
    int n[4];   // Nx, Ny, Nz, Nt
    int src[4]; // source site
    int d;      // correlator direction
    int e[3];   // the other directions, increasing
};

// block (b, tau): the eight channel sums of the sites of slice tau that block b visits
__global__ void __launch_bounds__(kBlock) k_slices(SliceArgs a, const double *w, double *partials)
{
    __shared__ double red[kBlock / 32][8];
    const int tau = blockIdx.y;
    const int xd = (a.src[a.d] + tau) % a.n[a.d];
    const int n0 = a.n[a.e[0]], n1 = a.n[a.e[1]], n2 = a.n[a.e[2]];
    const size_t nslice = (size_t)n0 * n1 * n2;
    double acc[8];
#pragma unroll
    for (int S = 0; S < 8; S++) acc[S] = 0.0;
    for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < nslice; j += (size_t)gridDim.x * blockDim.x) {
        int X[4];
        const int c0 = (int)(j % n0);
        const size_t r = j / n0;
        const int c1 = (int)(r % n1), c2 = (int)(r / n1);
        X[a.d] = xd;
        X[a.e[0]] = c0;
        X[a.e[1]] = c1;
        X[a.e[2]] = c2;
        // the lattice extents are even, so (x - y) mod 2 = (x + y) mod 2
        const int bits = ((c0 + a.src[a.e[0]]) & 1) | (((c1 + a.src[a.e[1]]) & 1) << 1) |
                         (((c2 + a.src[a.e[2]]) & 1) << 2);
        const size_t lex = X[0] + (size_t)a.n[0] * (X[1] + (size_t)a.n[1] * (X[2] + (size_t)a.n[2] * X[3]));
        const double v = w[lex];
#pragma unroll
        for (int S = 0; S < 8; S++) acc[S] += (__popc(S & bits) & 1) ? -v : v;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int S = 0; S < 8; S++) {
        double v = acc[S];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[wid][S] = v;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        double s = 0.0;
        for (int i = 0; i < kBlock / 32; i++) s += red[i][threadIdx.x];
        partials[((size_t)tau * 8 + threadIdx.x) * gridDim.x + blockIdx.x] = s;
    }
}

}  // namespace meson

}  // namespace hisq

using namespace hisq;

extern "C" int hisq_meson_correlators(hisq_ctx *ctx, double m, const int src[4], int direction,
                                      const hisq_solve_opts *opts, double *corr, double *prop, hisq_stats *stats)
{
    using namespace hisq::meson;
    if (!ctx) return HISQ_EINVAL;
    if (ctx->batch) return set_error(ctx, HISQ_EINVAL, "hisq_meson_correlators: not a single-lattice context");
    if (!src || !corr || direction < 0 || direction > 3 || !(m > 0.0) || !std::isfinite(m))
        return set_error(ctx, HISQ_EINVAL, "hisq_meson_correlators: bad argument");
    for (int mu = 0; mu < 4; mu++)
        if (src[mu] < 0 || src[mu] >= ctx->dims[mu])
            return set_error(ctx, HISQ_EINVAL, "hisq_meson_correlators: source outside the lattice");
    hisq_solve_opts o;
    if (opts) o = *opts;
    else hisq_solve_opts_default(&o);
    if (o.host_buffers) return set_error(ctx, HISQ_EINVAL, "hisq_meson_correlators: device buffers only");
    o.zero_guess = 1;
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)o.stream;
    const uint32_t Vh = ctx->g.Vh;
    const size_t n = (size_t)Vh * 3, hb = n * sizeof(double2) * 3; // three half-lattice vectors
    const size_t V = 2 * (size_t)Vh;
    const int nd = ctx->dims[direction];
    const size_t nslice = V / nd;
    const int nblk = (int)std::max<size_t>(1, std::min<size_t>((nslice + kBlock - 1) / kBlock,
                                                                 (2 * (size_t)ctx->sm_count + nd - 1) / nd));
    const int nvec = (int)std::min<size_t>((n + kBlock - 1) / kBlock, 2 * (size_t)ctx->sm_count);

    // source parity and half index: lex / 2 within its parity (Sec. 4.3)
    const size_t lex0 = src[0] + (size_t)ctx->dims[0] * (src[1] + (size_t)ctx->dims[1] * (src[2] + (size_t)ctx->dims[2] * src[3]));
    const int odd = (src[0] + src[1] + src[2] + src[3]) & 1;
    const uint32_t s0 = (uint32_t)(lex0 / 2);

    char *wsp = nullptr;
    double2 *G = reinterpret_cast<double2 *>(prop);
    const size_t own_g = prop ? 0 : 2 * hb;
    const size_t bytes = own_g + 3 * hb + V * sizeof(double) + sizeof(double) * 8 * nd * nblk;
    if (cudaMalloc((void **)&wsp, bytes) != cudaSuccess) {
        cudaGetLastError();
        return set_error(ctx, HISQ_ENOMEM, "hisq_meson_correlators: workspace");
    }
    if (!G) G = reinterpret_cast<double2 *>(wsp);
    double2 *rhs = reinterpret_cast<double2 *>(wsp + own_g);
    double2 *xe = reinterpret_cast<double2 *>(wsp + own_g + hb);
    double2 *tmp = reinterpret_cast<double2 *>(wsp + own_g + 2 * hb);
    double *w = reinterpret_cast<double *>(wsp + own_g + 3 * hb);
    double *partials = w + V;
    auto fail = [&](int rc) {
        cudaStreamSynchronize(st);
        cudaFree(wsp);
        return rc;
    };

    // even right-hand side: 2m b_e, or D_eo b_o (solved for -x_e) for an odd source
    cudaError_t e = cudaMemsetAsync(rhs, 0, hb, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(tmp, 0, hb, st);
    if (e != cudaSuccess) return fail(cuda_error(ctx, e, "hisq_meson_correlators: clear"));
    if (!odd) {
        k_point<<<1, 32, 0, st>>>(rhs, Vh, s0, 2.0 * m);
    } else {
        k_point<<<1, 32, 0, st>>>(tmp, Vh, s0, 1.0);
        int rc = hisq_dslash(ctx, 0, reinterpret_cast<const double *>(tmp), reinterpret_cast<double *>(rhs), 3,
                             HISQ_F64, st);
        if (rc) return fail(rc);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(cuda_error(ctx, e, "hisq_meson_correlators: source"));

    hisq_stats cs{};
    const int rcg = hisq_cg(ctx, m, reinterpret_cast<const double *>(rhs), reinterpret_cast<double *>(xe), 3, &o, &cs,
                            nullptr);
    if (rcg != HISQ_OK && rcg != HISQ_ENOTCONVERGED) return fail(rcg);
    if (stats) *stats = cs;

    // odd half: D_oe x_e, then the propagator
    int rc = hisq_dslash(ctx, 1, reinterpret_cast<const double *>(xe), reinterpret_cast<double *>(tmp), 3, HISQ_F64, st);
    if (rc) return fail(rc);
    k_assemble<<<dim3(nvec, 3), kBlock, 0, st>>>(xe, tmp, G, Vh, odd ? -1.0 : 1.0, 2.0 * m, odd, s0);
    k_weights<<<2 * nvec, kBlock, 0, st>>>(ctx->g, G, w);
    SliceArgs a{};
    for (int mu = 0, k = 0; mu < 4; mu++) {
        a.n[mu] = ctx->dims[mu];
        a.src[mu] = src[mu];
        if (mu != direction) a.e[k++] = mu;
    }
    a.d = direction;
    k_slices<<<dim3(nblk, nd), kBlock, 0, st>>>(a, w, partials);
    std::vector<double> h((size_t)8 * nd * nblk);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), partials, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(wsp);
    if (e != cudaSuccess) return cuda_error(ctx, e, "hisq_meson_correlators: correlators");
    for (int tau = 0; tau < nd; tau++)
        for (int S = 0; S < 8; S++) {
            double s = 0.0;
            for (int b = 0; b < nblk; b++) s += h[((size_t)tau * 8 + S) * nblk + b]; // fixed order
            corr[(size_t)S * nd + tau] = s;
        }
    if (rcg != HISQ_OK) return set_error(ctx, rcg, "hisq_meson_correlators: the solve missed the tolerance");
    return HISQ_OK;
}
