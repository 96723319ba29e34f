// fcg.cu -- flexible CG (inexact-preconditioner CG) with the learned preconditioner; the
// paper's CG (Sec. 3.2) with z = K(r) in place of r.  Not in the paper.
//
// With <a, b> = sum conj(a) b, q = A p and z = K r:
//   alpha = conj(<r, z>) / <p, q>     (the A-norm-minimising step along p: <p, r> = <z, r>)
//   x += alpha p ;  r' = r - alpha q ;  z' = K r'
//   beta = <r' - r, z'> / <r, z> = -conj(alpha) <q, z'> / <r, z>   (Polak-Ribiere)
//   p = z' + beta p
// Vectors are FP64; A is applied with the FP64 or the float-pair (F64X) operator, and a
// converged solve is confirmed with the FP64 operator.  The iterations run inside a CUDA
// graph with one WHILE node; every scalar stays on the device, and the finishing block of
// the last reduction of an iteration decides whether the loop goes on, so the host waits
// once per loop (normally once per solve).  The loop stops when the iterated residual
// reaches the target, the network output is not finite, the residual has not decreased
// for 50 iterations with the network, the curvature <p, A p> is not positive, or the
// iteration cap is reached; the host then confirms, drops the network (the solve goes on
// as plain CG from the current iterate), or reports.
#include <chrono>
#include <cmath>
#include <cstring>

#include "blas.cuh"
#include "dslash.cuh"
#include "net.cuh"

namespace hisq {

int apply_mdagm(hisq_ctx *ctx, int prec, double m, const void *in, void *tmp, void *out, int nrhs, size_t rhs_bytes,
                cudaStream_t st, const Reduce *red, bool tune);

enum FcgState {
    FCG_RUN = 0,
    FCG_CONVERGED = 1,  // iterated |r|^2 <= tol^2 |b|^2
    FCG_NONFINITE = 2,  // a dot product of the step is not finite (network output)
    FCG_STAGNATED = 3,  // no new smallest residual for kStagnation iterations
    FCG_CURVATURE = 4,  // <p, A p> not positive or not finite
    FCG_CAP = 5         // iteration cap of this loop reached
};
constexpr int kStagnation = 50;
constexpr int kMaxRestarts = 20; // FP64 confirmations that may fail before the solve gives up

struct FcgScalars {
    double2 rz;    // <r, z>
    double2 alpha; // conj(<r, z>) / <p, A p>
    double2 beta;
    double pq;     // <p, A p>
    double rr;     // |r|^2
    double stop;   // tol^2 |b|^2
    double best;   // smallest |r|^2 seen
    int since_best;
    int iters;     // iterations performed in this solve
    int cap;       // last iteration allowed in the current loop
    int state;     // FcgState
    int stagnation_check; // 1 while the network preconditions (plain CG has no stagnation stop)
    int pad;
};

}  // namespace hisq

struct hisq::FcgWork {
    int device = 0;
    uint32_t Vh = 0;
    size_t vb = 0, pb = 0; // bytes of one canonical FP64 vector, of one padded F64X vector
    double2 *b = nullptr, *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *t = nullptr;
    char *xx = nullptr, *tx = nullptr, *Ax = nullptr; // float-pair operator buffers
    double *partials = nullptr;
    unsigned *counter = nullptr;
    FcgScalars *sc = nullptr, *h_sc = nullptr;
    int nblk = 0;
    cudaStream_t st = nullptr;
    cudaGraphExec_t graph = nullptr;
    // the graph bakes in the operator, the mass and the network
    int g_pa = -1, g_net_on = -1;
    double g_m = -1.0;
    unsigned long long g_uid = 0;
};

namespace hisq {

// ---------------------------------------------------------------- reductions
// Each block supplies NV block sums (thread 0); the last block to arrive adds the partials
// of each value in a fixed order and calls fin(totals) on thread 0, then resets the counter.
template <int NV, class Fin>
__device__ __forceinline__ void fcg_reduce(double (&v)[NV], double *partials, unsigned *counter, Fin fin)
{
    block_sum_multi<NV>(v);
    __shared__ bool last;
    const int nb = gridDim.x;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) partials[k * nb + blockIdx.x] = v[k];
        // acquire-release arrival (publishes the partials; the last block sees all of them)
        unsigned prev;
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(prev) : "l"(counter) : "memory");
        last = prev == (unsigned)nb - 1;
    }
    __syncthreads();
    if (!last) return;
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    double tot[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) {
        double s = 0.0;
        for (int i = threadIdx.x; i < nb; i += blockDim.x) s += __ldcg(partials + k * nb + i);
        tot[k] = s;
    }
    block_sum_multi<NV>(tot);
    if (threadIdx.x == 0) {
        fin(tot);
        __threadfence();
        *counter = 0u;
    }
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cdiv(double2 a, double2 b)
{
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

// ---------------------------------------------------------------- kernels
// set-up scalars after r and z: rz = <r, z>, rr = |r|^2 (values 0, 1 + 2i of the partials)
__global__ void __launch_bounds__(kVecBlock) k_fcg_start(const double2 *r, const double2 *z, size_t n,
                                                          double *partials, unsigned *counter, FcgScalars *sc,
                                                          int stagnation_check)
{
    double v[3] = {0.0, 0.0, 0.0};
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double2 a = r[i], c = z[i];
        v[0] += a.x * a.x + a.y * a.y;
        v[1] += a.x * c.x + a.y * c.y;
        v[2] += a.x * c.y - a.y * c.x;
    }
    fcg_reduce<3>(v, partials, counter, [&](const double (&t)[3]) {
        FcgScalars &S = *sc;
        S.rr = t[0];
        S.rz = make_double2(t[1], t[2]);
        S.best = t[0];
        S.since_best = 0;
        S.stagnation_check = stagnation_check;
        S.state = (isfinite(t[0]) && isfinite(t[1]) && isfinite(t[2])) ? FCG_RUN : FCG_NONFINITE;
        if (S.state == FCG_RUN && t[0] <= S.stop) S.state = FCG_CONVERGED;
    });
}

// |b|^2 -> stop = tol^2 |b|^2 ; iteration counter reset
__global__ void __launch_bounds__(kVecBlock) k_fcg_norm_b(const double2 *b, size_t n, double *partials,
                                                           unsigned *counter, FcgScalars *sc, double tol2)
{
    double v[1] = {0.0};
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double2 a = b[i];
        v[0] += a.x * a.x + a.y * a.y;
    }
    fcg_reduce<1>(v, partials, counter, [&](const double (&t)[1]) {
        sc->stop = tol2 * t[0];
        sc->iters = 0;
    });
}

// q (FP64) from the operator output (F64X float pairs, or already FP64), and <p, q> -> alpha
template <int PA>
__global__ void __launch_bounds__(kVecBlock) k_fcg_pq(const char *Ax, double2 *q, const double2 *p, uint32_t Vh,
                                                       double *partials, unsigned *counter, FcgScalars *sc)
{
    if (sc->state != FCG_RUN) return; // uniform: set before this launch
    double v[1] = {0.0};
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < Vh; s += gridDim.x * blockDim.x) {
        double2 a[3];
        if constexpr (PA == HISQ_F64X) {
            typename Prec<HISQ_F64X>::Vec w;
            Prec<HISQ_F64X>::load(Ax, s, w);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                a[k] = make_double2(Blas<HISQ_F64X>::get(w, 2 * k), Blas<HISQ_F64X>::get(w, 2 * k + 1));
                q[(size_t)s * 3 + k] = a[k];
            }
        } else {
#pragma unroll
            for (int k = 0; k < 3; k++) a[k] = q[(size_t)s * 3 + k];
        }
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const double2 c = p[(size_t)s * 3 + k];
            v[0] += c.x * a[k].x + c.y * a[k].y; // Re <p, q>; A is Hermitian
        }
    }
    fcg_reduce<1>(v, partials, counter, [&](const double (&t)[1]) {
        FcgScalars &S = *sc;
        S.pq = t[0];
        if (!(t[0] > 0.0 && isfinite(t[0]))) {
            S.state = FCG_CURVATURE;
            S.alpha = make_double2(0.0, 0.0);
        } else {
            S.alpha = make_double2(S.rz.x / t[0], -S.rz.y / t[0]);
        }
    });
}

// x += alpha p ; r -= alpha q
__global__ void __launch_bounds__(256) k_fcg_update(double2 *x, const double2 *p, const double2 *q, double2 *r,
                                                     size_t n, const FcgScalars *sc)
{
    if (sc->state != FCG_RUN) return;
    const double2 al = sc->alpha;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double2 pv = p[i], qv = q[i];
        double2 xv = x[i], rv = r[i];
        xv.x += al.x * pv.x - al.y * pv.y;
        xv.y += al.x * pv.y + al.y * pv.x;
        rv.x -= al.x * qv.x - al.y * qv.y;
        rv.y -= al.x * qv.y + al.y * qv.x;
        x[i] = xv;
        r[i] = rv;
    }
}

// z = r (no network)
__global__ void __launch_bounds__(256) k_fcg_copy(const double2 *r, double2 *z, size_t n, const FcgScalars *sc)
{
    if (sc->state != FCG_RUN) return;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) z[i] = r[i];
}

// |r'|^2, <q, z'>, <r', z'>: beta, the new <r, z>, and the loop decision
__global__ void __launch_bounds__(kVecBlock) k_fcg_dots(const double2 *r, const double2 *q, const double2 *z, size_t n,
                                                         double *partials, unsigned *counter, FcgScalars *sc,
                                                         unsigned long long cond)
{
    if (sc->state != FCG_RUN) { // uniform; the loop is ending (curvature): still release it
        if (blockIdx.x == 0 && threadIdx.x == 0 && cond)
            cudaGraphSetConditional((cudaGraphConditionalHandle)cond, 0u);
        return;
    }
    double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double2 a = r[i], c = z[i], d = q[i];
        v[0] += a.x * a.x + a.y * a.y;
        v[1] += d.x * c.x + d.y * c.y;
        v[2] += d.x * c.y - d.y * c.x;
        v[3] += a.x * c.x + a.y * c.y;
        v[4] += a.x * c.y - a.y * c.x;
    }
    fcg_reduce<5>(v, partials, counter, [&](const double (&t)[5]) {
        FcgScalars &S = *sc;
        S.iters++;
        bool finite = true;
#pragma unroll
        for (int k = 0; k < 5; k++) finite &= (bool)isfinite(t[k]);
        if (!finite) {
            S.state = FCG_NONFINITE;
        } else {
            const double2 qz = make_double2(t[1], t[2]);
            const double2 rz_new = make_double2(t[3], t[4]);
            const double2 num = cmul(cconj(S.alpha), qz);
            S.beta = cdiv(make_double2(-num.x, -num.y), S.rz);
            S.rz = rz_new;
            S.rr = t[0];
            if (t[0] < S.best) {
                S.best = t[0];
                S.since_best = 0;
            } else if (++S.since_best >= kStagnation && S.stagnation_check) {
                S.state = FCG_STAGNATED;
            }
            if (t[0] <= S.stop) S.state = FCG_CONVERGED;
            else if (S.state == FCG_RUN && S.iters >= S.cap) S.state = FCG_CAP;
        }
        if (cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, S.state == FCG_RUN ? 1u : 0u);
    });
}

// p = z + beta p
__global__ void __launch_bounds__(256) k_fcg_p(double2 *p, const double2 *z, size_t n, const FcgScalars *sc)
{
    if (sc->state != FCG_RUN) return;
    const double2 be = sc->beta;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double2 pv = p[i], zv = z[i];
        p[i] = make_double2(zv.x + be.x * pv.x - be.y * pv.y, zv.y + be.x * pv.y + be.y * pv.x);
    }
}

__global__ void k_fcg_loop_begin(FcgScalars *sc, int cap)
{
    sc->cap = sc->iters + cap;
    if (sc->state == FCG_CAP) sc->state = FCG_RUN;
}

// r = b - q ; |r|^2 -> rr (FP64 confirmation of a converged solve)
__global__ void __launch_bounds__(kVecBlock) k_fcg_residual(const double2 *b, const double2 *q, double2 *r, size_t n,
                                                             double *partials, unsigned *counter, FcgScalars *sc)
{
    double v[1] = {0.0};
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double2 a = make_double2(b[i].x - q[i].x, b[i].y - q[i].y);
        r[i] = a;
        v[0] += a.x * a.x + a.y * a.y;
    }
    fcg_reduce<1>(v, partials, counter, [&](const double (&t)[1]) { sc->rr = t[0]; });
}

// ---------------------------------------------------------------- workspace
void release_fcg_work(hisq_ctx *ctx)
{
    FcgWork *w = ctx ? ctx->fcg : nullptr;
    if (!w) return;
    cudaSetDevice(w->device);
    if (w->st) cudaStreamSynchronize(w->st);
    if (w->graph) cudaGraphExecDestroy(w->graph);
    void *bufs[] = {w->b, w->x, w->r, w->z, w->p, w->q, w->t, w->xx, w->tx, w->Ax, w->partials, w->counter, w->sc};
    for (void *p : bufs)
        if (p) cudaFree(p);
    if (w->h_sc) cudaFreeHost(w->h_sc);
    if (w->st) cudaStreamDestroy(w->st);
    delete w;
    ctx->fcg = nullptr;
}

static int get_fcg_work(hisq_ctx *ctx, FcgWork **out)
{
    if (ctx->fcg) {
        *out = ctx->fcg;
        return HISQ_OK;
    }
    FcgWork *w = new FcgWork();
    ctx->fcg = w;
    w->device = ctx->device;
    w->Vh = ctx->g.Vh;
    w->vb = (size_t)ctx->g.Vh * 48;
    w->pb = (size_t)ctx->g.VhPad * 48;
    w->nblk = (int)std::min<size_t>((ctx->g.Vh + kVecBlock - 1) / kVecBlock, 4ull * ctx->sm_count);
    auto A = [&](size_t bytes, void **p) { return cudaMalloc(p, bytes) == cudaSuccess; };
    bool ok = A(w->vb, (void **)&w->b) && A(w->vb, (void **)&w->x) && A(w->vb, (void **)&w->r) &&
              A(w->vb, (void **)&w->z) && A(w->vb, (void **)&w->p) && A(w->vb, (void **)&w->q) &&
              A(w->vb, (void **)&w->t) && A(w->pb, (void **)&w->xx) && A(w->pb, (void **)&w->tx) &&
              A(w->pb, (void **)&w->Ax) && A(sizeof(double) * 8 * (size_t)w->nblk, (void **)&w->partials) &&
              A(64, (void **)&w->counter) && A(sizeof(FcgScalars), (void **)&w->sc);
    ok = ok && cudaMallocHost((void **)&w->h_sc, sizeof(FcgScalars)) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&w->st, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaMemset(w->counter, 0, 64) == cudaSuccess && cudaMemset(w->sc, 0, sizeof(FcgScalars)) == cudaSuccess;
    // padding sites of the float-pair buffers stay zero
    ok = ok && cudaMemset(w->xx, 0, w->pb) == cudaSuccess && cudaMemset(w->tx, 0, w->pb) == cudaSuccess &&
         cudaMemset(w->Ax, 0, w->pb) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        release_fcg_work(ctx);
        return set_error(ctx, HISQ_ENOMEM, "hisq_fcg: workspace");
    }
    *out = w;
    return HISQ_OK;
}

// q = A in (FP64 canonical in, FP64 canonical q) with the operator pa; tune: allowed to time shapes
static int fcg_apply(hisq_ctx *ctx, FcgWork &w, int pa, double m, const double2 *in, bool tune)
{
    const dim3 g(w.nblk, 1);
    if (pa == HISQ_F64) return apply_mdagm(ctx, HISQ_F64, m, in, w.t, w.q, 1, w.vb, w.st, nullptr, tune);
    k_convert<HISQ_F64, HISQ_F64X><<<g, kVecBlock, 0, w.st>>>(VecRef{(char *)in, 0}, VecRef{w.xx, 0}, w.Vh);
    return apply_mdagm(ctx, HISQ_F64X, m, w.xx, w.tx, w.Ax, 1, w.pb, w.st, nullptr, tune);
}

// z = K(r) with the network, or z = r
static int fcg_precond(hisq_net *net, FcgWork &w, bool use_net)
{
    if (use_net) return net_forward(net, (const double *)w.r, (double *)w.z, w.st);
    const size_t n = (size_t)w.Vh * 3;
    k_fcg_copy<<<(unsigned)std::min<size_t>((n + 255) / 256, 1024), 256, 0, w.st>>>(w.r, w.z, n, w.sc);
    return HISQ_OK;
}

// one iteration (captured into the loop body); cond: the WHILE node's handle
static int fcg_iteration(hisq_ctx *ctx, FcgWork &w, hisq_net *net, bool use_net, int pa, double m,
                         unsigned long long cond)
{
    const size_t n = (size_t)w.Vh * 3;
    const unsigned gb = (unsigned)std::min<size_t>((n + 255) / 256, 8ull * ctx->sm_count);
    int rc = fcg_apply(ctx, w, pa, m, w.p, false);
    if (rc) return rc;
    if (pa == HISQ_F64X)
        k_fcg_pq<HISQ_F64X><<<w.nblk, kVecBlock, 0, w.st>>>(w.Ax, w.q, w.p, w.Vh, w.partials, w.counter, w.sc);
    else
        k_fcg_pq<HISQ_F64><<<w.nblk, kVecBlock, 0, w.st>>>(nullptr, w.q, w.p, w.Vh, w.partials, w.counter, w.sc);
    k_fcg_update<<<gb, 256, 0, w.st>>>(w.x, w.p, w.q, w.r, n, w.sc);
    if ((rc = fcg_precond(net, w, use_net))) return rc;
    k_fcg_dots<<<w.nblk, kVecBlock, 0, w.st>>>(w.r, w.q, w.z, n, w.partials, w.counter, w.sc, cond);
    k_fcg_p<<<gb, 256, 0, w.st>>>(w.p, w.z, n, w.sc);
    HISQ_CUDA(ctx, cudaGetLastError());
    return HISQ_OK;
}

static int build_fcg_graph(hisq_ctx *ctx, FcgWork &w, hisq_net *net, bool use_net, int pa, double m)
{
    if (w.graph) {
        cudaGraphExecDestroy(w.graph);
        w.graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    HISQ_CUDA(ctx, cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_error(ctx, e, "hisq_fcg: conditional node");
    }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(w.st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_error(ctx, e, "hisq_fcg: capture");
    }
    int rc = fcg_iteration(ctx, w, net, use_net, pa, m, (unsigned long long)h);
    e = cudaStreamEndCapture(w.st, &body);
    if (rc || e != cudaSuccess) {
        cudaGraphDestroy(g);
        cudaGetLastError();
        return rc ? rc : cuda_error(ctx, e, "hisq_fcg: capture");
    }
    e = cudaGraphInstantiate(&w.graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_error(ctx, e, "hisq_fcg: graph instantiate");
    w.g_pa = pa;
    w.g_m = m;
    w.g_net_on = use_net ? 1 : 0;
    w.g_uid = use_net ? net->uid : 0;
    return HISQ_OK;
}

static int read_fcg(hisq_ctx *ctx, FcgWork &w)
{
    HISQ_CUDA(ctx, cudaMemcpyAsync(w.h_sc, w.sc, sizeof(FcgScalars), cudaMemcpyDeviceToHost, w.st));
    HISQ_CUDA(ctx, cudaStreamSynchronize(w.st));
    return HISQ_OK;
}

// r = b - A x (operator pa), z = K r, p = z, rz, rr: the start of a solve or a restart
static int fcg_restart(hisq_ctx *ctx, FcgWork &w, hisq_net *net, bool use_net, int pa, double m)
{
    const size_t n = (size_t)w.Vh * 3;
    int rc = fcg_apply(ctx, w, pa, m, w.x, true);
    if (rc) return rc;
    if (pa == HISQ_F64X)
        k_convert<HISQ_F64X, HISQ_F64><<<w.nblk, kVecBlock, 0, w.st>>>(VecRef{w.Ax, 0}, VecRef{(char *)w.q, 0}, w.Vh);
    k_fcg_residual<<<w.nblk, kVecBlock, 0, w.st>>>(w.b, w.q, w.r, n, w.partials, w.counter, w.sc);
    // z = K r: the copy kernel reads the state, so mark the solve running first
    HISQ_CUDA(ctx, cudaMemsetAsync(&w.sc->state, 0, sizeof(int), w.st));
    if ((rc = fcg_precond(net, w, use_net))) return rc;
    k_fcg_start<<<w.nblk, kVecBlock, 0, w.st>>>(w.r, w.z, n, w.partials, w.counter, w.sc, use_net ? 1 : 0);
    HISQ_CUDA(ctx, cudaMemcpyAsync(w.p, w.z, w.vb, cudaMemcpyDeviceToDevice, w.st));
    HISQ_CUDA(ctx, cudaGetLastError());
    return HISQ_OK;
}

}  // namespace hisq

using namespace hisq;

extern "C" int hisq_fcg(hisq_ctx *ctx, double m, hisq_net *net, const double *b, double *x,
                        const hisq_solve_opts *opts, hisq_stats *stats)
{
    if (!ctx) return HISQ_EINVAL;
    if (!b || !x || !(m >= 0.0) || (net && net->ctx != ctx)) return set_error(ctx, HISQ_EINVAL, "hisq_fcg: bad argument");
    hisq_solve_opts o;
    if (opts) o = *opts;
    else hisq_solve_opts_default(&o);
    const int pa = o.prec_precise == HISQ_F64X ? HISQ_F64X : HISQ_F64;
    if (!ctx->links[pa].built || !ctx->links[HISQ_F64].built) return set_error(ctx, HISQ_ENOTBUILT, "hisq_fcg: precision");
    if (o.host_buffers) return set_error(ctx, HISQ_EINVAL, "hisq_fcg: device buffers only");
    if (!(o.tol > 0.0) || o.maxiter < 1) return set_error(ctx, HISQ_EINVAL, "hisq_fcg: tol and maxiter must be positive");
    if (stats) std::memset(stats, 0, sizeof(*stats));
    cudaSetDevice(ctx->device);
    const auto t0 = std::chrono::steady_clock::now();
    FcgWork *wp = nullptr;
    int rc = get_fcg_work(ctx, &wp);
    if (rc) return rc;
    FcgWork &w = *wp;
    const size_t n = (size_t)w.Vh * 3;
    const double tol2 = o.tol * o.tol;
    // the caller's stream is ordered before and after the solve
    cudaStream_t ust = (cudaStream_t)o.stream;
    cudaEvent_t ev;
    HISQ_CUDA(ctx, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaEventRecord(ev, ust);
    cudaStreamWaitEvent(w.st, ev, 0);
    HISQ_CUDA(ctx, cudaMemcpyAsync(w.b, b, w.vb, cudaMemcpyDeviceToDevice, w.st));
    if (o.zero_guess) HISQ_CUDA(ctx, cudaMemsetAsync(w.x, 0, w.vb, w.st));
    else HISQ_CUDA(ctx, cudaMemcpyAsync(w.x, x, w.vb, cudaMemcpyDeviceToDevice, w.st));
    k_fcg_norm_b<<<w.nblk, kVecBlock, 0, w.st>>>(w.b, n, w.partials, w.counter, w.sc, tol2);
    bool use_net = net != nullptr;
    int fallbacks = 0, loops = 0, restarts = 0;
    long kernels = 0;
    if ((rc = fcg_restart(ctx, w, net, use_net, pa, m))) goto done;
    if ((rc = read_fcg(ctx, w))) goto done;
    if (w.h_sc->state == FCG_NONFINITE && use_net) { // network output not finite: plain CG
        use_net = false;
        fallbacks++;
        if ((rc = fcg_restart(ctx, w, net, false, pa, m)) || (rc = read_fcg(ctx, w))) goto done;
    }
    for (;;) {
        const FcgScalars &S = *w.h_sc;
        if (S.state == FCG_CONVERGED) {
            // confirm with the FP64 operator
            if ((rc = fcg_apply(ctx, w, HISQ_F64, m, w.x, true))) break;
            k_fcg_residual<<<w.nblk, kVecBlock, 0, w.st>>>(w.b, w.q, w.t, n, w.partials, w.counter, w.sc);
            if ((rc = read_fcg(ctx, w))) break;
            if (w.h_sc->rr <= w.h_sc->stop) break; // done
            // the iterated residual ran ahead of the true one: restart from the iterate with
            // the FP64 residual (so a restart cannot report convergence the FP64 check denies)
            if (++restarts > kMaxRestarts) { rc = HISQ_ENOTCONVERGED; break; }
            if ((rc = fcg_restart(ctx, w, net, use_net, HISQ_F64, m)) || (rc = read_fcg(ctx, w))) break;
            continue;
        }
        if (S.state == FCG_NONFINITE || S.state == FCG_STAGNATED) {
            if (!use_net) { rc = HISQ_ENOTCONVERGED; break; }
            use_net = false; // drop the network; continue as CG from the current iterate
            fallbacks++;
            if ((rc = fcg_restart(ctx, w, net, false, pa, m)) || (rc = read_fcg(ctx, w))) break;
            continue;
        }
        if (S.state == FCG_CURVATURE) { rc = HISQ_ENOTCONVERGED; break; }
        const int left = o.maxiter - S.iters;
        if (left <= 0) { rc = HISQ_ENOTCONVERGED; break; }
        if (!w.graph || w.g_pa != pa || w.g_m != m || w.g_net_on != (use_net ? 1 : 0) ||
            (use_net && w.g_uid != net->uid)) {
            // tune the operator's launch shapes before capturing
            if ((rc = fcg_apply(ctx, w, pa, m, w.p, true))) break;
            if ((rc = build_fcg_graph(ctx, w, net, use_net, pa, m))) break;
        }
        k_fcg_loop_begin<<<1, 1, 0, w.st>>>(w.sc, left);
        if (cudaGraphLaunch(w.graph, w.st) != cudaSuccess) { rc = cuda_error(ctx, cudaGetLastError(), "hisq_fcg: graph"); break; }
        loops++;
        if ((rc = read_fcg(ctx, w))) break;
    }
done:
    {
        const int iters = w.h_sc->iters;
        const double rr = w.h_sc->rr, bb = w.h_sc->stop / tol2;
        cudaMemcpyAsync(x, w.x, w.vb, cudaMemcpyDeviceToDevice, w.st);
        cudaEventRecord(ev, w.st);
        cudaStreamWaitEvent(ust, ev, 0);
        cudaStreamSynchronize(w.st);
        cudaEventDestroy(ev);
        const int per_it = (pa == HISQ_F64X ? 3 : 2) + 4 + (use_net ? 2 + net->nlayer : 1);
        kernels = (long)iters * per_it + 8L * (loops + fallbacks + 1);
        if (stats) {
            stats->iterations = iters;
            stats->reliable_updates = fallbacks;
            stats->true_residual = std::sqrt(rr / bb);
            stats->iterated_residual = std::sqrt(rr / bb);
            stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            stats->dslash_calls = 2L * (iters + 2);
            stats->kernels = kernels;
        }
        if (rc && rc != HISQ_ENOTCONVERGED) return rc;
        if (net || fallbacks) {
            const int ds = check_device_status(ctx, w.st);
            if (ds) return ds;
        }
        if (rc == HISQ_ENOTCONVERGED || !(rr <= w.h_sc->stop))
            return set_error(ctx, HISQ_ENOTCONVERGED, "hisq_fcg: tolerance not reached");
    }
    return HISQ_OK;
}
