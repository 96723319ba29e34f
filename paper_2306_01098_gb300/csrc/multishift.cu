// multishift.cu -- multi-shift CG (Sec. 3.2 and its reference to Jegerlehner): solves
// (A + sigma_s) x_s = b for all shifts with one operator application per iteration, on the
// smallest shift sigma_0; the other shifts follow from the shift invariance of the Krylov
// space at the cost of one fused vector update per iteration (for every shift):
//   q = (A + sigma_0) p_0,  alpha = |r|^2 / <p_0, q>                  (Dslash pair + epilogue)
//   r -= alpha q,  beta = |r_new|^2 / |r|^2                          (fused update + norm)
//   zeta_s' = zeta_s zeta_s^- alpha^- /
//             [alpha^- zeta_s^- (1 + alpha d_s) + alpha beta^- (zeta_s^- - zeta_s)]
//   alpha_s = alpha zeta_s' / zeta_s,  beta_s = beta (zeta_s' / zeta_s)^2     (one thread per shift)
//   x_s += alpha_s p_s,  p_s = zeta_s' r + beta_s p_s                (one pass, all shifts)
// with d_s = sigma_s - sigma_0; shift s stops once |zeta_s| |r| <= tol_s |b|.  Afterwards all
// shifts are finished together by one multi-right-hand-side CG of cg.cu with a per-right-hand-
// side shift (A + sigma_s) x_s = b started from the multi-shift iterates, so the links are read
// once per iteration for every shift; in a reduced sloppy precision this is a mixed-precision
// solve with FP64 reliable updates, in FP64 it only recomputes and confirms the residuals.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "blas.cuh"
#include "dslash.cuh"
#include "solver.cuh"

namespace hisq {

int run_cg(hisq_ctx *ctx, double m, const double *b, double *x, int nrhs, const hisq_solve_opts &o, hisq_stats *stats,
           double *residuals, const double *shifts);

constexpr int kMaxShift = 64;

struct ShiftState {
    double zeta[kMaxShift], zeta_old[kMaxShift];
    double alpha_s[kMaxShift], beta_s[kMaxShift], zeta_new[kMaxShift];
    double delta[kMaxShift], tol2[kMaxShift];
    int active[kMaxShift];
    double alpha_prev, beta_prev;
};

struct MsWork {
    int nshift = 0, ps = -1, pv = -1, px = -1; // sloppy links, sloppy vectors, accumulator
    DslashShape shape;
    uint32_t Vh = 0;
    size_t rbS = 0, rbX = 0, rb64 = 0;
    char *r = nullptr, *q = nullptr, *t = nullptr, *p = nullptr, *x = nullptr, *b64 = nullptr;
    char *ball = nullptr, *xall = nullptr; // [nshift][Vh] FP64: b repeated, iterates (refinement)
    Scalars *sc = nullptr, *h_sc = nullptr;
    ShiftState *ss = nullptr, *h_ss = nullptr;
    double *partials = nullptr;
    unsigned *counter = nullptr;
    int nblk_vec = 0, nblk_dslash = 0;
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    std::vector<void *> allocs;
    void release()
    {
        for (void *a : allocs) cudaFree(a);
        allocs.clear();
        if (h_sc) cudaFreeHost(h_sc);
        if (h_ss) cudaFreeHost(h_ss);
        h_sc = nullptr;
        h_ss = nullptr;
        if (st) cudaStreamDestroy(st);
        if (ev) cudaEventDestroy(ev);
        st = nullptr;
        ev = nullptr;
    }
    Reduce red(int op, int nb, int ntotal) const
    {
        Reduce R;
        R.partials = partials;
        R.counter = counter;
        R.sc = sc;
        R.op = op;
        R.nblocks = nb;
        R.ntotal = ntotal;
        return R;
    }
};

// ---------------------------------------------------------------- kernels
__global__ void k_shift_init(ShiftState *ss, const Scalars *sc, int n)
{
    const int s = threadIdx.x;
    if (s == 0) {
        ss->alpha_prev = 1.0;
        ss->beta_prev = 0.0;
    }
    if (s < n) {
        ss->zeta[s] = ss->zeta_old[s] = 1.0;
        ss->alpha_s[s] = ss->beta_s[s] = 0.0;
        ss->zeta_new[s] = 1.0;
        ss->active[s] = sc->rr > ss->tol2[s] * sc->bb;
    }
}

// zeta recurrences for every shift after the base iteration produced alpha and beta
__global__ void k_shift_scalars(ShiftState *ss, const Scalars *sc, int n)
{
    const int s = threadIdx.x;
    // alpha and beta of this iteration, or nothing when the base launch was skipped
    const double alpha = (sc->astamp == sc->it_all - 1) ? sc->alpha : 0.0, beta = sc->beta;
    __syncthreads();
    if (s < n) {
        if (alpha == 0.0 || !ss->active[s]) {
            ss->alpha_s[s] = 0.0;
            ss->beta_s[s] = 0.0;
        } else {
            const double z = ss->zeta[s], zo = ss->zeta_old[s], ap = ss->alpha_prev, bp = ss->beta_prev;
            const double den = ap * zo * (1.0 + alpha * ss->delta[s]) + alpha * bp * (zo - z);
            const double zn = z * zo * ap / den;
            const double ratio = zn / z;
            ss->alpha_s[s] = alpha * ratio;
            ss->beta_s[s] = beta * ratio * ratio;
            ss->zeta_new[s] = zn;
            ss->zeta_old[s] = z;
            ss->zeta[s] = zn;
            // |r_new|^2 = sc->rr after the base update
            if (zn * zn * sc->rr <= ss->tol2[s] * sc->bb || !isfinite(zn)) ss->active[s] = 0;
        }
    }
    __syncthreads();
    if (s == 0 && alpha != 0.0) {
        ss->alpha_prev = alpha;
        ss->beta_prev = beta;
    }
}

// x_s += alpha_s p_s ; p_s = zeta_s' r + beta_s p_s  for every shift with alpha_s != 0
template <int PS, int PX>
__global__ void __launch_bounds__(kVecBlock) k_shift_update(VecRef x, VecRef p, VecRef r, uint32_t Vh, const ShiftState *ss,
                                                            int n)
{
    using BS = Blas<PS>;
    using BX = Blas<PX>;
    static_assert(std::is_same<typename BS::Vec, typename BX::Vec>::value, "accumulator shares the sloppy vector type");
    // The shifts' coefficients once per block: read from global memory, compared and
    // converted per site and shift, they kept this GPU's FP64 pipe (1/64 of the FP32 rate)
    // busy for about four operations per site and shift.  FP32 vectors use float copies.
    constexpr bool FL = std::is_same<typename BS::Vec, FloatArith::Vec>::value;
    __shared__ double cd[3][kMaxShift];
    __shared__ float cf[3][kMaxShift];
    __shared__ int on[kMaxShift], act[kMaxShift];
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        cd[0][k] = ss->alpha_s[k];
        cd[1][k] = ss->zeta_new[k];
        cd[2][k] = ss->beta_s[k];
        for (int i = 0; i < 3; i++) cf[i][k] = (float)cd[i][k];
        on[k] = cd[0][k] != 0.0;
        act[k] = ss->active[k];
    }
    __syncthreads();
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < Vh; s += gridDim.x * blockDim.x) {
        typename BS::Vec rv;
        bool have_r = false;
        for (int k = 0; k < n; k++) {
            if (!on[k]) continue;
            typename BS::Vec pv;
            vload<PS>(p.rhs(k), s, pv);
            typename BX::Vec xv;
            vload<PX>(x.rhs(k), s, xv);
            if constexpr (FL) {
                const float a = cf[0][k];
#pragma unroll
                for (int i = 0; i < 6; i++) xv.v[i] = fmaf(a, pv.v[i], xv.v[i]);
            } else {
                BX::axpy(xv, cd[0][k], pv);
            }
            BX::store(x.rhs(k), s, xv);
            if (act[k]) {
                if (!have_r) {
                    vload<PS>(r.rhs(0), s, rv);
                    have_r = true;
                }
                if constexpr (FL) {
                    const float z = cf[1][k], b = cf[2][k];
#pragma unroll
                    for (int i = 0; i < 6; i++) pv.v[i] = fmaf(z, rv.v[i], b * pv.v[i]);
                } else {
                    BS::axpby(pv, cd[1][k], rv, cd[2][k]);
                }
                BS::store(p.rhs(k), s, pv);
            }
        }
    }
}

template <int PS, int PX>
struct MsTyped {
    static void update_r(MsWork &w, cudaStream_t st)
    {
        k_update_r<PS><<<dim3(w.nblk_vec, 1), kVecBlock, 0, st>>>(VecRef{w.r, w.rbS}, VecRef{w.q, w.rbS}, w.Vh,
                                                                  w.red(FIN_RR, w.nblk_vec, w.nblk_vec));
    }
    static void shift_update(MsWork &w, cudaStream_t st)
    {
        k_shift_update<PS, PX><<<w.nblk_vec, kVecBlock, 0, st>>>(VecRef{w.x, w.rbX}, VecRef{w.p, w.rbS},
                                                                  VecRef{w.r, w.rbS}, w.Vh, w.ss, w.nshift);
    }
    static void start(MsWork &w, cudaStream_t st)
    {
        // r = sloppy(b); p_s = r; x_s = 0
        k_convert<HISQ_F64, PS><<<dim3(w.nblk_vec, 1), kVecBlock, 0, st>>>(VecRef{w.b64, w.rb64}, VecRef{w.r, w.rbS}, w.Vh);
        k_convert<PS, PS><<<dim3(w.nblk_vec, w.nshift), kVecBlock, 0, st>>>(VecRef{w.r, 0}, VecRef{w.p, w.rbS}, w.Vh);
    }
    static void finish(MsWork &w, double *const *xout, cudaStream_t st)
    {
        for (int k = 0; k < w.nshift; k++)
            k_convert<PX, HISQ_F64><<<dim3(w.nblk_vec, 1), kVecBlock, 0, st>>>(VecRef{w.x + k * w.rbX, w.rbX},
                                                                             VecRef{reinterpret_cast<char *>(xout[k]), w.rb64}, w.Vh);
    }
};

template <class F>
static void ms_dispatch(int ps, F &&f)
{
    switch (ps) {
    case HISQ_F64: f(MsTyped<HISQ_F64, HISQ_F64>{}); break;
    case HISQ_F64X: f(MsTyped<HISQ_F64X, HISQ_F64X>{}); break;
    case HISQ_F32: f(MsTyped<HISQ_F32, HISQ_F32>{}); break;
    case HISQ_F16: f(MsTyped<HISQ_F16, HISQ_F32>{}); break;
    default: f(MsTyped<HISQ_BF16, HISQ_F32>{}); break;
    }
}

static int ms_alloc(hisq_ctx *ctx, MsWork &w, char **p, size_t bytes)
{
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
    if (e != cudaSuccess) return cuda_error(ctx, e, "multishift workspace");
    cudaMemset(q, 0, bytes ? bytes : 16);
    w.allocs.push_back(q);
    *p = static_cast<char *>(q);
    return HISQ_OK;
}

void release_ms_work(hisq_ctx *ctx)
{
    if (ctx->msolver) {
        ctx->msolver->release();
        delete ctx->msolver;
        ctx->msolver = nullptr;
    }
}

static int get_ms_work(hisq_ctx *ctx, int nshift, int ps, MsWork **out)
{
    MsWork *&w = ctx->msolver;
    if (w && w->nshift == nshift && w->ps == ps) {
        *out = w;
        return HISQ_OK;
    }
    if (w) {
        cudaDeviceSynchronize();
        release_ms_work(ctx);
    }
    w = new MsWork();
    MsWork &W = *w;
    W.nshift = nshift;
    W.ps = ps;
    W.pv = vector_prec(ps);
    W.px = (W.pv == HISQ_F64 || W.pv == HISQ_F64X) ? W.pv : HISQ_F32;
    W.Vh = ctx->g.Vh;
    W.rbS = (size_t)ctx->g.VhPad * spinor_bytes(W.pv);
    W.rbX = (size_t)ctx->g.VhPad * spinor_bytes(W.px);
    W.rb64 = (size_t)ctx->g.Vh * 48;
    W.nblk_vec = (int)std::min<long>((W.Vh + kVecBlock - 1) / kVecBlock, 4L * ctx->sm_count);
    W.nblk_dslash = (int)((4ull * W.Vh + 63) / 64); // blocks at 4 threads per site and 64 threads per block (upper bound)
    int rc = HISQ_OK;
    auto A = [&](char **p, size_t b) { if (rc == HISQ_OK) rc = ms_alloc(ctx, W, p, b); };
    A(&W.r, W.rbS);
    A(&W.q, W.rbS);
    A(&W.t, W.rbS);
    A(&W.p, W.rbS * nshift);
    A(&W.x, W.rbX * nshift);
    A(&W.b64, W.rb64);
    A(&W.ball, W.rb64 * nshift);
    A(&W.xall, W.rb64 * nshift);
    char *tmp = nullptr;
    A(&tmp, sizeof(Scalars) * 4);
    W.sc = reinterpret_cast<Scalars *>(tmp);
    A(&tmp, sizeof(ShiftState));
    W.ss = reinterpret_cast<ShiftState *>(tmp);
    A(&tmp, sizeof(double) * 4 * (size_t)std::max(W.nblk_vec, W.nblk_dslash));
    W.partials = reinterpret_cast<double *>(tmp);
    A(&tmp, 64);
    W.counter = reinterpret_cast<unsigned *>(tmp);
    if (rc) return rc;
    if (cudaMallocHost(&W.h_sc, sizeof(Scalars) * 4) != cudaSuccess ||
        cudaMallocHost(&W.h_ss, sizeof(ShiftState)) != cudaSuccess)
        return set_error(ctx, HISQ_ENOMEM, "pinned scalars");
    if (cudaStreamCreateWithFlags(&W.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&W.ev, cudaEventDisableTiming) != cudaSuccess)
        return set_error(ctx, HISQ_ECUDA, "multishift stream");
    *out = w;
    return HISQ_OK;
}

// one multi-shift iteration on the base system
static int ms_iteration(hisq_ctx *ctx, MsWork &w, double m4s, cudaStream_t st)
{
    const LinkStore &L = ctx->links[w.ps];
    DslashArgs a = make_dslash_args(ctx, w.ps, 1, w.p, w.t, 1, w.rbS); // p_0 is shift 0
    a.skip = w.sc;
    cudaError_t e = dslash_launch(w.ps, w.pv, 0, a, L.nreal, w.shape, st);
    if (e != cudaSuccess) return cuda_error(ctx, e, "multishift dslash");
    DslashArgs b = make_dslash_args(ctx, w.ps, 0, w.t, w.q, 1, w.rbS);
    b.skip = w.sc;
    b.pv = w.p;
    b.m4 = m4s;
    b.red = w.red(FIN_ALPHA, 0, 0); // block counts filled in by the launcher
    e = dslash_launch(w.ps, w.pv, 1, b, L.nreal, w.shape, st);
    if (e != cudaSuccess) return cuda_error(ctx, e, "multishift dslash + epilogue");
    ms_dispatch(w.pv, [&](auto T) { decltype(T)::update_r(w, st); });
    k_shift_scalars<<<1, kMaxShift, 0, st>>>(w.ss, w.sc, w.nshift);
    ms_dispatch(w.pv, [&](auto T) { decltype(T)::shift_update(w, st); });
    return HISQ_OK;
}

__global__ void k_ms_init_scalars(Scalars *sc, double tol2)
{
    Scalars &S = sc[0];
    S.bb = S.last;
    S.rr = S.last;
    S.rr_ref = S.last;
    S.stop = tol2 * S.last;
    S.delta2 = 0.0;
    S.alpha = S.beta = 0.0;
    S.flag = 0;
    S.iters = 0;
    S.it_all = 0;
    S.astamp = -2;
    S.bad = !isfinite(S.last);
    S.active = isfinite(S.last) && S.last > S.stop;
}

}  // namespace hisq

using namespace hisq;

extern "C" int hisq_multishift_cg(hisq_ctx *ctx, double m, int nshift, const double *sigma, const double *b,
                                  double *const *x, const double *tol, const hisq_solve_opts *opts, hisq_stats *stats,
                                  double *residuals)
{
    if (!ctx) return HISQ_EINVAL;
    if (!sigma || !b || !x || nshift < 1 || nshift > kMaxShift || !(m >= 0.0))
        return set_error(ctx, HISQ_EINVAL, "hisq_multishift_cg: bad argument");
    hisq_solve_opts o;
    if (opts) o = *opts;
    else hisq_solve_opts_default(&o);
    if (o.host_buffers) return set_error(ctx, HISQ_EINVAL, "hisq_multishift_cg: device buffers only");
    if (!(o.tol > 0.0) || o.maxiter < 1) return set_error(ctx, HISQ_EINVAL, "hisq_multishift_cg: bad tolerance");
    for (int s = 0; s < nshift; s++) {
        if (!(sigma[s] >= 0.0) || !x[s]) return set_error(ctx, HISQ_EINVAL, "hisq_multishift_cg: bad shift");
        if (tol && !(tol[s] > 0.0)) return set_error(ctx, HISQ_EINVAL, "hisq_multishift_cg: bad shift tolerance");
    }
    const int ps = o.prec_sloppy;
    if (ps < 0 || ps >= HISQ_NPREC || !ctx->links[ps].built) return set_error(ctx, HISQ_ENOTBUILT, "sloppy precision not built");
    if (stats) std::memset(stats, 0, sizeof(*stats));
    cudaSetDevice(ctx->device);
    auto t0 = std::chrono::steady_clock::now();

    // base shift = smallest sigma; the solver's shift k is the caller's shift order[k]
    std::vector<int> order(nshift);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return sigma[a] < sigma[c]; });
    MsWork *wp = nullptr;
    int rc = get_ms_work(ctx, nshift, ps, &wp);
    if (rc) return rc;
    MsWork &w = *wp;
    cudaStream_t st = w.st;
    HISQ_CUDA(ctx, cudaEventRecord(w.ev, (cudaStream_t)o.stream));
    HISQ_CUDA(ctx, cudaStreamWaitEvent(st, w.ev, 0));

    // sloppy stage target: the requested tolerance in FP64, otherwise a level the sloppy
    // recurrences still resolve; the per-shift CG below finishes the job
    const double floor_tol = ps == HISQ_F64 ? 0.0 : ps == HISQ_F64X ? 1e-12 : ps == HISQ_F32 ? 1e-6 : 1e-4;
    std::vector<double> tgt(nshift);
    double tmin = 1.0;
    for (int k = 0; k < nshift; k++) {
        const int s = order[k];
        tgt[k] = std::max(tol ? tol[s] : o.tol, floor_tol);
        tmin = std::min(tmin, tgt[k]);
    }
    ShiftState init{};
    for (int k = 0; k < nshift; k++) {
        init.delta[k] = sigma[order[k]] - sigma[order[0]];
        init.tol2[k] = tgt[k] * tgt[k];
    }
    HISQ_CUDA(ctx, cudaMemcpyAsync(w.b64, b, w.rb64, cudaMemcpyDeviceToDevice, st));
    std::memcpy(w.h_ss, &init, sizeof(ShiftState));
    HISQ_CUDA(ctx, cudaMemcpyAsync(w.ss, w.h_ss, sizeof(ShiftState), cudaMemcpyHostToDevice, st));
    HISQ_CUDA(ctx, cudaMemsetAsync(w.x, 0, w.rbX * nshift, st));
    k_norm_f64<<<dim3(w.nblk_vec, 1), kVecBlock, 0, st>>>(VecRef{w.b64, w.rb64}, w.Vh, w.red(FIN_STORE, w.nblk_vec, w.nblk_vec));
    k_ms_init_scalars<<<1, 1, 0, st>>>(w.sc, tmin * tmin);
    k_shift_init<<<1, kMaxShift, 0, st>>>(w.ss, w.sc, nshift);
    ms_dispatch(w.pv, [&](auto T) { decltype(T)::start(w, st); });
    HISQ_CUDA(ctx, cudaGetLastError());
    w.shape = dslash_shape(ctx, ps, w.pv, 1, w.p, w.t, w.rbS, st);

    const double m4s = 4.0 * m * m + sigma[order[0]];
    const int ci = std::max(1, o.check_interval);
    int total = 0;
    for (;;) {
        HISQ_CUDA(ctx, cudaMemcpyAsync(w.h_sc, w.sc, sizeof(Scalars), cudaMemcpyDeviceToHost, st));
        HISQ_CUDA(ctx, cudaStreamSynchronize(st));
        if (!w.h_sc[0].active || w.h_sc[0].bad || total >= o.maxiter) break;
        const int n = std::min(ci, o.maxiter - total);
        for (int i = 0; i < n; i++)
            if ((rc = ms_iteration(ctx, w, m4s, st))) return rc;
        HISQ_CUDA(ctx, cudaGetLastError());
        total += n;
    }
    const int ms_iters = w.h_sc[0].iters;
    const bool bad = w.h_sc[0].bad != 0;
    std::vector<double *> xs(nshift);
    for (int k = 0; k < nshift; k++) xs[k] = x[order[k]];
    ms_dispatch(w.pv, [&](auto T) { decltype(T)::finish(w, xs.data(), st); });
    HISQ_CUDA(ctx, cudaStreamSynchronize(st));
    if (bad) return set_error(ctx, HISQ_ENOTCONVERGED, "hisq_multishift_cg: non-finite residual");

    // finish every shift together: multi-RHS CG on (A + sigma_s) x_s = b from the iterates
    hisq_solve_opts co = o;
    co.zero_guess = 0;
    co.host_buffers = 0;
    co.stream = nullptr;
    if (ps == HISQ_F64 || ps == HISQ_F64X) co.prec_precise = ps;
    double tmin_all = o.tol;
    std::vector<double> shifts(nshift);
    for (int k = 0; k < nshift; k++) {
        const int s = order[k];
        if (tol) tmin_all = std::min(tmin_all, tol[s]);
        shifts[k] = sigma[s];
        HISQ_CUDA(ctx, cudaMemcpyAsync(w.ball + k * w.rb64, b, w.rb64, cudaMemcpyDeviceToDevice, st));
        HISQ_CUDA(ctx, cudaMemcpyAsync(w.xall + k * w.rb64, x[s], w.rb64, cudaMemcpyDeviceToDevice, st));
    }
    co.tol = tmin_all;
    HISQ_CUDA(ctx, cudaStreamSynchronize(st));
    hisq_stats cs{};
    std::vector<double> res(nshift, 0.0);
    const int r2 = run_cg(ctx, m, (const double *)w.ball, (double *)w.xall, nshift, co, &cs, res.data(), shifts.data());
    if (r2 != HISQ_OK && r2 != HISQ_ENOTCONVERGED) return r2;
    int worst_rc = r2;
    for (int k = 0; k < nshift; k++)
        HISQ_CUDA(ctx, cudaMemcpyAsync(x[order[k]], w.xall + k * w.rb64, w.rb64, cudaMemcpyDeviceToDevice, st));
    HISQ_CUDA(ctx, cudaStreamSynchronize(st));
    double worst = 0.0;
    for (int k = 0; k < nshift; k++) {
        if (residuals) residuals[order[k]] = res[k];
        worst = std::max(worst, res[k]);
    }
    const int extra = cs.iterations, nru = cs.reliable_updates;
    if (stats) {
        stats->iterations = ms_iters + extra;
        stats->reliable_updates = nru;
        stats->true_residual = worst;
        stats->iterated_residual = worst;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        stats->dslash_calls = 2L * (ms_iters + extra);
    }
    if (worst_rc != HISQ_OK) return set_error(ctx, worst_rc, "hisq_multishift_cg: tolerance not reached");
    return HISQ_OK;
}
