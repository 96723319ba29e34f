// cg.cu -- conjugate gradient on A = 4m^2 - D_eo D_oe (Sec. 3.2), single and multi-RHS,
// plain FP64 or mixed precision with reliable updates.
//
// Iteration (all scalars stay on the device; one grid reduction per inner product):
//   t  = D_oe p                          sloppy Dslash
//   Ap = m4 p - D_eo t, <p,Ap> -> alpha  sloppy Dslash + fused epilogue/reduction
//   r -= alpha Ap, |r|^2 -> beta         fused update/reduction
//   x_lo += alpha p, p = r + beta p      fused update
// The host launches blocks of `check_interval` iterations (optionally one captured CUDA
// graph per block) and reads the scalars only between blocks.  Reliable update (mixed
// precision; the scheme the paper's mixed-precision citation describes):
//   x_hi += x_lo, x_lo = 0, r_hi = b - A_precise x_hi (FP64 or float-pair operator),
//   r = sloppy(r_hi), beta = |r_hi|^2 / |r_old|^2, p = r + beta p;
// triggered every `reliable_interval` iterations, when the sloppy residual fell below
// delta times the last true one, or when it reached the target.  The solve ends when
// every recomputed residual |b - A x| / |b| <= tol.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "blas.cuh"
#include "cg_phase.cuh"
#include "dslash.cuh"
#include "solver.cuh"

namespace hisq {

int apply_mdagm(hisq_ctx *ctx, int prec, double m, const void *in, void *tmp, void *out, int nrhs, size_t rhs_bytes,
                cudaStream_t st, const Reduce *red, bool tune);

// ---------------------------------------------------------------- scalar bookkeeping
enum { SC_INIT_BB = 0, SC_INIT_R = 1, SC_RU = 2 };

__global__ void k_scalars(Scalars *sc, int n, int mode, double tol2, double delta2)
{
    const int r = threadIdx.x;
    if (r >= n) return;
    Scalars &S = sc[r];
    switch (mode) {
    case SC_INIT_BB:
        S.bb = S.last;
        S.stop = tol2 * S.last;
        S.delta2 = delta2;
        S.iters = 0;
        S.it_all = 0;
        S.astamp = -2;
        S.bad = 0;
        break;
    case SC_INIT_R:
        S.rr = S.last;
        S.rr_ref = S.last;
        S.alpha = S.beta = 0.0;
        S.flag = 0;
        S.paused = 0;
        S.active = (S.last > S.stop) && isfinite(S.last);
        if (!isfinite(S.last)) S.bad = 1;
        break;
    default: { // reliable update: S.last = |b - A x_hi|^2
        const double rt = S.last;
        if (!isfinite(rt)) {
            S.bad = 1;
            S.active = 0;
            S.beta = 0.0;
        } else if (rt <= S.stop) {
            S.active = 0;
            S.beta = 0.0;
        } else {
            // continuing: beta = |r_true|^2 / |r_old|^2 with |r_old|^2 = rr / beta; a right-hand
            // side that had met the sloppy target restarts from p = r
            const bool going = S.active || S.paused;
            S.beta = (going && S.rr > 0.0) ? S.beta * rt / S.rr : 0.0;
            S.active = 1;
        }
        S.rr = rt;
        S.rr_ref = rt;
        S.flag = 0;
        S.paused = 0;
        break;
    }
    }
}

static double wall()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

static int accum_prec(int ps) { return (ps == HISQ_F64 || ps == HISQ_F64X) ? ps : HISQ_F32; }

// ---------------------------------------------------------------- typed launches
template <int PS, int PX>
struct Typed {
    static void update_r(SolverWork &w, cudaStream_t st, LoopCtl *ctl = nullptr, unsigned long long cond = 0)
    {
        Reduce R = w.red(FIN_RR, w.nblk_vec);
        R.ctl = ctl;
        R.cond = cond;
        k_update_r<PS><<<dim3(w.nblk_vec, w.nrhs), kVecBlock, 0, st>>>(VecRef{w.r, w.rbS}, VecRef{w.Ap, w.rbS}, w.len(), R);
    }
    static void update_xrp(SolverWork &w, cudaStream_t st, const LoopCtl *ctl)
    {
        k_update_xrp<PS, PX><<<dim3(w.nblk_vec, w.nrhs), kVecBlock, 0, st>>>(
            VecRef{w.xlo, w.rbX}, VecRef{w.p, w.rbS}, VecRef{w.r, w.rbS}, VecRef{w.Ap, w.rbS}, w.len(), w.sc, 0, ctl);
    }
    static void update_xp(SolverWork &w, int mode, cudaStream_t st, const LoopCtl *ctl = nullptr)
    {
        k_update_xp<PS, PX><<<dim3(w.nblk_vec, w.nrhs), kVecBlock, 0, st>>>(
            VecRef{w.xlo, w.rbX}, VecRef{w.p, w.rbS}, VecRef{w.r, w.rbS}, w.len(), w.sc, mode, ctl);
    }
    static void accum_hi(SolverWork &w, cudaStream_t st)
    {
        k_accum_hi<PX><<<dim3(w.nblk_vec, w.nrhs), kVecBlock, 0, st>>>(VecRef{w.x64, w.rb64}, VecRef{w.xlo, w.rbX}, w.len());
    }
    // re-orthogonalise p against the replaced residual, then p = r + beta p
    static void reortho(SolverWork &w, cudaStream_t st)
    {
        const dim3 g(w.nblk_vec, w.nrhs);
        k_cdot<PS><<<g, kVecBlock, 0, st>>>(VecRef{w.r, w.rbS}, VecRef{w.p, w.rbS}, w.len(),
                                            w.red(FIN_CDOT, w.nblk_vec, w.nblk_vec * w.nrhs));
        k_p_reortho<PS><<<g, kVecBlock, 0, st>>>(VecRef{w.p, w.rbS}, VecRef{w.r, w.rbS}, w.len(), w.sc);
    }
    static void from_hi(SolverWork &w, char *dst, cudaStream_t st)
    {
        k_convert<HISQ_F64, PS><<<dim3(w.nblk_vec, w.nrhs), kVecBlock, 0, st>>>(VecRef{w.rhi, w.rb64}, VecRef{dst, w.rbS},
                                                                               w.len());
    }
};

template <class F>
static void dispatch(int ps, F &&f)
{
    switch (ps) {
    case HISQ_F64: f(Typed<HISQ_F64, HISQ_F64>{}); break;
    case HISQ_F64X: f(Typed<HISQ_F64X, HISQ_F64X>{}); break;
    case HISQ_F32: f(Typed<HISQ_F32, HISQ_F32>{}); break;
    case HISQ_F16: f(Typed<HISQ_F16, HISQ_F32>{}); break;
    default: f(Typed<HISQ_BF16, HISQ_F32>{}); break;
    }
}

// ---------------------------------------------------------------- workspace
void SolverWork::release()
{
    for (void *q : allocs) cudaFree(q);
    allocs.clear();
    if (graph) cudaGraphExecDestroy(graph);
    graph = nullptr;
    for (auto e : prof) cudaEventDestroy(e);
    prof.clear();
    if (h_sc) cudaFreeHost(h_sc);
    h_sc = nullptr;
    if (h_shift) cudaFreeHost(h_shift);
    h_shift = nullptr;
    if (h_status) cudaFreeHost(h_status);
    h_status = nullptr;
    if (st) cudaStreamDestroy(st);
    st = nullptr;
    if (ev) cudaEventDestroy(ev);
    ev = nullptr;
    if (ev_sc) cudaEventDestroy(ev_sc);
    ev_sc = nullptr;
}

int SolverWork::alloc(hisq_ctx *ctx, char **ptr, size_t bytes)
{
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
    if (e != cudaSuccess) return cuda_error(ctx, e, "solver workspace");
    cudaMemset(q, 0, bytes ? bytes : 16);
    allocs.push_back(q);
    *ptr = static_cast<char *>(q);
    return HISQ_OK;
}

Reduce SolverWork::red(int op, int nblocks_per_value, int ntotal) const
{
    Reduce R;
    R.partials = partials;
    R.counter = counter;
    R.sc = sc;
    R.op = op;
    R.nblocks = nblocks_per_value;
    R.ntotal = ntotal ? ntotal : nblocks_per_value * nrhs;
    return R;
}

int get_work(hisq_ctx *ctx, int nrhs, int ps, int pp, SolverWork **out)
{
    SolverWork *&w = ctx->solver;
    if (w && w->nrhs == nrhs && w->ps == ps && w->pp == pp) {
        *out = w;
        return HISQ_OK;
    }
    if (w) {
        cudaDeviceSynchronize();
        w->release();
        delete w;
        w = nullptr;
    }
    w = new SolverWork();
    SolverWork &W = *w;
    W.nrhs = nrhs;
    W.ps = ps;
    W.pv = vector_prec(ps);
    W.px = accum_prec(W.pv);
    W.pp = pp;
    W.Vh = ctx->g.Vh;
    if (ctx->batch)
        W.vh_rhs = reinterpret_cast<const uint32_t *>(reinterpret_cast<const char *>(ctx->batch) + offsetof(BatchDesc, vh));
    W.rbS = (size_t)ctx->g.VhPad * spinor_bytes(W.pv);
    W.rbX = (size_t)ctx->g.VhPad * spinor_bytes(W.px);
    W.rb64 = (size_t)ctx->g.Vh * 48;
    W.rbP = (size_t)ctx->g.VhPad * 48;
    // blocks per right-hand side of the vector passes: at most one block per 256 sites and
    // about one resident wave (eight 256-thread blocks per SM) over all right-hand sides; a
    // block costs a few memory round trips (scalars, arrival) whatever its share of sites,
    // so with many right-hand sides (a batch of small lattices) extra waves of nearly empty
    // blocks took longer than the vector traffic
    W.nblk_vec = (int)std::min<long>({(W.Vh + kVecBlock - 1) / kVecBlock, 4L * ctx->sm_count,
                                      std::max(1L, 8L * ctx->sm_count / nrhs)});
    W.nblk_dslash = (int)((4ull * W.Vh + 63) / 64); // blocks at 4 threads per site and 64 threads per block (upper bound)
    int rc = HISQ_OK;
    auto A = [&](char **p, size_t b) { if (rc == HISQ_OK) rc = W.alloc(ctx, p, b); };
    A(&W.r, W.rbS * nrhs);
    A(&W.p, W.rbS * nrhs);
    A(&W.Ap, W.rbS * nrhs);
    A(&W.t, W.rbS * nrhs);
    A(&W.xlo, W.rbX * nrhs);
    A(&W.b64, W.rb64 * nrhs);
    A(&W.x64, W.rb64 * nrhs);
    A(&W.rhi, W.rb64 * nrhs);
    A(&W.Axhi, W.rb64 * nrhs);
    A(&W.thi, W.rb64 * nrhs);
    if (pp == HISQ_F64X) {
        A(&W.xx, W.rbP * nrhs);
        A(&W.tx, W.rbP * nrhs);
        A(&W.Axx, W.rbP * nrhs);
    }
    char *tmp = nullptr;
    A(&tmp, sizeof(Scalars) * (nrhs + 64));
    W.sc = reinterpret_cast<Scalars *>(tmp);
    A(&tmp, sizeof(double) * (size_t)(4 * nrhs + 64) * std::max(W.nblk_vec, W.nblk_dslash));
    W.partials = reinterpret_cast<double *>(tmp);
    A(&tmp, 64);
    W.counter = reinterpret_cast<unsigned *>(tmp);
    A(&tmp, sizeof(LoopCtl));
    W.ctl = reinterpret_cast<LoopCtl *>(tmp);
    A(&tmp, sizeof(PhaseSlot) * kPhaseMaxBlocks);
    W.phase_slots = tmp;
    A(&tmp, sizeof(double) * (nrhs + 64));
    W.shift_buf = reinterpret_cast<double *>(tmp);
    if (rc) return rc;
    if (cudaMallocHost(&W.h_sc, sizeof(Scalars) * (nrhs + 64)) != cudaSuccess ||
        cudaMallocHost(&W.h_shift, sizeof(double) * (nrhs + 64)) != cudaSuccess ||
        cudaMallocHost(&W.h_status, sizeof(DevStatus)) != cudaSuccess)
        return set_error(ctx, HISQ_ENOMEM, "pinned scalars");
    if (cudaStreamCreateWithFlags(&W.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&W.ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&W.ev_sc, cudaEventDisableTiming) != cudaSuccess)
        return set_error(ctx, HISQ_ECUDA, "solver stream");
    *out = w;
    return HISQ_OK;
}

void release_work(hisq_ctx *ctx)
{
    if (ctx->solver) {
        ctx->solver->release();
        delete ctx->solver;
        ctx->solver = nullptr;
    }
}

// ---------------------------------------------------------------- L2 residency of the links
// A persisting access-policy window over the sloppy link store keeps it in L2 across the
// iterations when it fits (16-bit links of a 32^3 x 8 lattice: 75 MB of the 129 MB L2).
// Everything the window changes is undone when the solve returns, on every return path:
// the stream's window is cleared, the persisting lines are released and the device's
// persisting-L2 limit is put back to the caller's value.
static void set_stream_window(cudaStream_t st, const cudaAccessPolicyWindow &w)
{
    cudaStreamAttrValue v{};
    v.accessPolicyWindow = w;
    cudaStreamSetAttribute(st, cudaStreamAttributeAccessPolicyWindow, &v);
}

struct L2Residency {
    cudaStream_t st = nullptr;
    bool window = false;  // the stream carries the window
    bool raised = false;  // the persisting limit was raised from old_limit
    size_t old_limit = 0;
    ~L2Residency()
    {
        if (window) {
            set_stream_window(st, cudaAccessPolicyWindow{});
            cudaCtxResetPersistingL2Cache();
        }
        if (raised) cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, old_limit);
        cudaGetLastError();
    }
};

// mode: 0 off, 1 on, -1 automatic (on when the whole store fits in the persisting L2 limit)
static cudaAccessPolicyWindow link_window(hisq_ctx *ctx, int ps, int mode, L2Residency &res)
{
    cudaAccessPolicyWindow w{};
    if (mode == 0) return w;
    const LinkStore &L = ctx->links[ps];
    int maxw = 0, maxp = 0;
    cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxAccessPolicyWindowSize, ctx->device);
    cudaDeviceGetAttribute(&maxp, cudaDevAttrMaxPersistingL2CacheSize, ctx->device);
    const size_t store = L.slot_bytes * kSlots;
    const size_t bytes = std::min(store, (size_t)maxw);
    if (maxp <= 0 || bytes == 0) return w;
    if (mode < 0 && (store > (size_t)maxp || store > (size_t)maxw)) return w;
    size_t lim = 0;
    cudaDeviceGetLimit(&lim, cudaLimitPersistingL2CacheSize);
    const size_t want = std::min(bytes, (size_t)maxp);
    if (lim < want && cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want) == cudaSuccess) {
        res.raised = true;
        res.old_limit = lim;
    }
    cudaGetLastError();
    cudaDeviceGetLimit(&lim, cudaLimitPersistingL2CacheSize);
    w.base_ptr = L.base;
    w.num_bytes = bytes;
    w.hitRatio = (float)std::min(1.0, (double)lim / (double)bytes);
    w.hitProp = cudaAccessPropertyPersisting;
    w.missProp = cudaAccessPropertyStreaming;
    return w;
}

// give every kernel node of a captured graph the window (explicitly, not relying on capture)
static void set_graph_window(cudaGraph_t g, const cudaAccessPolicyWindow &w)
{
    size_t n = 0;
    if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess || n == 0) return;
    std::vector<cudaGraphNode_t> nodes(n);
    if (cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return;
    cudaKernelNodeAttrValue v{};
    v.accessPolicyWindow = w;
    for (auto nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel)
            cudaGraphKernelNodeSetAttribute(nd, cudaKernelNodeAttributeAccessPolicyWindow, &v);
    }
    cudaGetLastError();
}

// ---------------------------------------------------------------- pieces of the iteration
// fused: the D_eo launch carries the single-reduction CG epilogue, whose finishing block
// also runs the loop control (ctl, cond)
static int sloppy_dslash_pair(hisq_ctx *ctx, SolverWork &w, double m, cudaStream_t st, cudaEvent_t *evs,
                              bool fused = false, unsigned long long cond = 0)
{
    const LinkStore &L = ctx->links[w.ps];
    DslashArgs a = make_dslash_args(ctx, w.ps, 1, w.p, w.t, w.nrhs, w.rbS);
    a.skip = w.sc;
    if (evs) cudaEventRecord(evs[0], st);
    cudaError_t e = dslash_launch(w.ps, w.pv, 0, a, L.nreal, w.shape, st);
    if (evs) cudaEventRecord(evs[1], st);
    if (e != cudaSuccess) return cuda_error(ctx, e, "sloppy dslash");
    DslashArgs b = make_dslash_args(ctx, w.ps, 0, w.t, w.Ap, w.nrhs, w.rbS);
    b.skip = w.sc;
    b.pv = w.p;
    b.m4 = 4.0 * m * m;
    b.shift = w.shift;
    b.red = w.red(fused ? FIN_AB : FIN_ALPHA, 0, 0); // block counts filled in by the launcher
    if (fused) {
        b.rv = w.r;
        b.red.ctl = w.ctl;
        b.red.cond = cond;
    }
    if (evs) cudaEventRecord(evs[2], st);
    e = dslash_launch(w.ps, w.pv, fused ? 2 : 1, b, L.nreal, w.shape, st);
    if (evs) cudaEventRecord(evs[3], st);
    if (e != cudaSuccess) return cuda_error(ctx, e, "sloppy dslash + epilogue");
    return HISQ_OK;
}

// one iteration: Dslash pair, r update (whose last block also runs the loop control), x/p
// update (its mode comes from the loop control: p is left alone in a phase's last iteration).
// Single-reduction form (w.fused): the D_eo epilogue reduces <p,Ap>, |r|^2, <r,Ap> and
// <Ap,Ap>; its finishing block produces alpha = |r|^2/<p,Ap>, the next
// |r - alpha Ap|^2 = |r|^2 - 2 alpha <r,Ap> + alpha^2 <Ap,Ap>, beta and the loop decision, and
// one pass updates x, r and p: three launches and one grid reduction per iteration instead
// of four and two.  |r|^2 is taken from the stored r every iteration: carried over from the
// previous expansion instead, its rounding error (about eps |b|^2) would never decay and the
// iterated residual could not fall below it.
static int launch_iteration(hisq_ctx *ctx, SolverWork &w, double m, cudaStream_t st, cudaEvent_t *evs,
                            unsigned long long cond)
{
    if (w.fused) {
        int rc = sloppy_dslash_pair(ctx, w, m, st, evs, true, cond);
        if (rc) return rc;
        dispatch(w.pv, [&](auto T) { decltype(T)::update_xrp(w, st, w.ctl); });
        HISQ_CUDA(ctx, cudaGetLastError());
        return HISQ_OK;
    }
    int rc = sloppy_dslash_pair(ctx, w, m, st, evs);
    if (rc) return rc;
    dispatch(w.pv, [&](auto T) {
        decltype(T)::update_r(w, st, w.ctl, cond);
        decltype(T)::update_xp(w, 0, st, w.ctl);
    });
    HISQ_CUDA(ctx, cudaGetLastError());
    return HISQ_OK;
}

__global__ void k_phase_begin(LoopCtl *ctl, const Scalars *sc, int cap)
{
    ctl->start = sc[0].it_all;
    ctl->cap = cap;
    ctl->mode = 0;
}

// The iteration loop as a CUDA graph: one WHILE node whose body is one iteration; the
// r update's finishing block clears the condition when no right-hand side is active or the
// phase's iteration cap is reached, so the device runs exactly the iterations needed
static int build_loop_graph(hisq_ctx *ctx, SolverWork &w, double m, const cudaAccessPolicyWindow &win, cudaStream_t st)
{
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
        return cuda_error(ctx, e, "conditional graph node");
    }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_error(ctx, e, "capture into loop body");
    }
    int rc = launch_iteration(ctx, w, m, st, nullptr, (unsigned long long)h);
    e = cudaStreamEndCapture(st, &body);
    if (rc || e != cudaSuccess) {
        cudaGraphDestroy(g);
        return rc ? rc : cuda_error(ctx, e, "capture into loop body");
    }
    set_graph_window(body, win);
    e = cudaGraphInstantiate(&w.graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_error(ctx, e, "loop graph instantiate");
    return HISQ_OK;
}

// ---------------------------------------------------------------- persistent phases
cudaError_t phase_launch_HISQ_F32(const PhaseArgs &a, int nreal, int ds, int sms, cudaStream_t st);
cudaError_t phase_launch_HISQ_F16(const PhaseArgs &a, int nreal, int ds, int sms, cudaStream_t st);
cudaError_t phase_launch_HISQ_BF16(const PhaseArgs &a, int nreal, int ds, int sms, cudaStream_t st);

// launch shape of the persistent kernel for o.persistent (0: the multi-kernel loop)
static int persistent_ds(hisq_ctx *ctx, const SolverWork &w, const hisq_solve_opts &o, bool shifted)
{
    if (o.persistent == 0 || w.nrhs != 1 || shifted || w.pv != HISQ_F32 || ctx->batch) return 0;
    int coop = 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device) != cudaSuccess || !coop) {
        cudaGetLastError();
        return 0;
    }
    // the block's x, r, p and Ap must fit in shared memory
    if (phase_chunk(w.Vh, ctx->sm_count) == 0) return 0;
    if (o.persistent >= 1 && o.persistent <= 5) return o.persistent;
    return 2;
}

// the sloppy iterations of one phase (at most cap, and none once Scalars.it_all reaches
// it_end) in one cooperative launch; reortho: the launch first re-orthogonalises p against
// the r of the reliable update before it
static int launch_persistent_phase(hisq_ctx *ctx, SolverWork &w, double m, int cap, int it_end, int ds, int reortho,
                                   int selftest, cudaStream_t st)
{
    PhaseArgs a{};
    a.doe = make_dslash_args(ctx, w.ps, 1, w.p, w.t, 1, w.rbS);
    a.doe.zt = 0;
    a.deo = make_dslash_args(ctx, w.ps, 0, w.t, w.Ap, 1, w.rbS);
    a.deo.zt = 0;
    a.deo.m4 = 4.0 * m * m;
    for (DslashArgs *d : {&a.doe, &a.deo}) {
        d->m4f = (float)d->m4;
        d->scale_f[0] = (float)d->scale[0];
        d->scale_f[1] = (float)d->scale[1];
    }
    a.x = w.xlo;
    a.p = w.p;
    a.r = w.r;
    a.Vh = w.Vh;
    a.sc = w.sc;
    a.slots = static_cast<PhaseSlot *>(w.phase_slots);
    a.status = ctx->status;
    a.cap = cap;
    a.it_end = it_end;
    a.reortho = reortho;
    a.selftest = selftest;
    a.wait_ns = selftest ? 1000000ull : 1000000000ull;
    HISQ_CUDA(ctx, cudaMemsetAsync(w.phase_slots, 0, sizeof(PhaseSlot) * kPhaseMaxBlocks, st));
    const int nreal = ctx->links[w.ps].nreal;
    cudaError_t e = cudaErrorInvalidValue;
    switch (w.ps) {
    case HISQ_F32: e = phase_launch_HISQ_F32(a, nreal, ds, ctx->sm_count, st); break;
    case HISQ_F16: e = phase_launch_HISQ_F16(a, nreal, ds, ctx->sm_count, st); break;
    case HISQ_BF16: e = phase_launch_HISQ_BF16(a, nreal, ds, ctx->sm_count, st); break;
    }
    if (e != cudaSuccess) return cuda_error(ctx, e, "persistent CG phase launch");
    return HISQ_OK;
}

// r_hi = b - A_precise x_hi ; |r_hi|^2 -> Scalars.last
int precise_residual(hisq_ctx *ctx, SolverWork &w, double m, cudaStream_t st, int prec)
{
    int rc;
    const dim3 g(w.nblk_vec, w.nrhs);
    if (prec == HISQ_F64) {
        if ((rc = apply_mdagm(ctx, HISQ_F64, m, w.x64, w.thi, w.Axhi, w.nrhs, w.rb64, st, nullptr, true))) return rc;
        k_residual<HISQ_F64><<<g, kVecBlock, 0, st>>>(VecRef{w.b64, w.rb64}, VecRef{w.Axhi, w.rb64}, VecRef{w.rhi, w.rb64},
                                                     w.len(), w.red(FIN_STORE, w.nblk_vec), w.shift,
                                                     VecRef{w.x64, w.rb64});
    } else {
        k_convert<HISQ_F64, HISQ_F64X><<<g, kVecBlock, 0, st>>>(VecRef{w.x64, w.rb64}, VecRef{w.xx, w.rbP}, w.len());
        if ((rc = apply_mdagm(ctx, HISQ_F64X, m, w.xx, w.tx, w.Axx, w.nrhs, w.rbP, st, nullptr, true))) return rc;
        k_residual<HISQ_F64X><<<g, kVecBlock, 0, st>>>(VecRef{w.b64, w.rb64}, VecRef{w.Axx, w.rbP}, VecRef{w.rhi, w.rb64},
                                                      w.len(), w.red(FIN_STORE, w.nblk_vec), w.shift,
                                                      VecRef{w.x64, w.rb64});
    }
    HISQ_CUDA(ctx, cudaGetLastError());
    return HISQ_OK;
}

static int read_scalars(hisq_ctx *ctx, SolverWork &w, cudaStream_t st)
{
    HISQ_CUDA(ctx, cudaMemcpyAsync(w.h_sc, w.sc, sizeof(Scalars) * w.nrhs, cudaMemcpyDeviceToHost, st));
    HISQ_CUDA(ctx, cudaStreamSynchronize(st));
    return HISQ_OK;
}

// ---------------------------------------------------------------- the solve
// shifts (host, may be NULL): per right-hand side sigma, solving (A + sigma_k) x_k = b_k
int run_cg(hisq_ctx *ctx, double m, const double *b, double *x, int nrhs, const hisq_solve_opts &o, hisq_stats *stats,
           double *residuals, const double *shifts)
{
    const double t0 = wall();
    int ps = o.prec_sloppy, pp = o.prec_precise;
    if (ps < 0 || ps >= HISQ_NPREC || (pp != HISQ_F64 && pp != HISQ_F64X))
        return set_error(ctx, HISQ_EINVAL, "hisq_cg: bad precision");
    if (!ctx->links[ps].built || !ctx->links[pp].built)
        return set_error(ctx, HISQ_ENOTBUILT, "hisq_cg: precision not built");
    SolverWork *wp = nullptr;
    int rc = get_work(ctx, nrhs, ps, pp, &wp);
    if (rc) return rc;
    SolverWork &w = *wp;
    cudaStream_t ust = (cudaStream_t)o.stream, st = w.st;
    HISQ_CUDA(ctx, cudaEventRecord(w.ev, ust));
    HISQ_CUDA(ctx, cudaStreamWaitEvent(st, w.ev, 0));
    const size_t vb = (size_t)nrhs * w.rb64;
    const cudaMemcpyKind k_in = o.host_buffers ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    HISQ_CUDA(ctx, cudaMemcpyAsync(w.b64, b, vb, k_in, st));
    if (o.zero_guess) HISQ_CUDA(ctx, cudaMemsetAsync(w.x64, 0, vb, st));
    else HISQ_CUDA(ctx, cudaMemcpyAsync(w.x64, x, vb, k_in, st));
    HISQ_CUDA(ctx, cudaMemsetAsync(w.xlo, 0, w.rbX * nrhs, st));
    // per right-hand side shifts (the operator's m4 + sigma_k in the epilogue and residuals)
    if (shifts) {
        std::memcpy(w.h_shift, shifts, sizeof(double) * nrhs);
        HISQ_CUDA(ctx, cudaMemcpyAsync(w.shift_buf, w.h_shift, sizeof(double) * nrhs, cudaMemcpyHostToDevice, st));
        w.shift = w.shift_buf;
        w.shift_key = std::vector<double>(shifts, shifts + nrhs);
    } else {
        w.shift = nullptr;
        w.shift_key.clear();
    }
    const dim3 g(w.nblk_vec, nrhs);
    const double tol2 = o.tol * o.tol;
    const double delta2 = o.reliable_delta * o.reliable_delta;
    // |b|^2
    k_norm_f64<<<g, kVecBlock, 0, st>>>(VecRef{w.b64, w.rb64}, w.len(), w.red(FIN_STORE, w.nblk_vec));
    k_scalars<<<1, 64, 0, st>>>(w.sc, nrhs, SC_INIT_BB, tol2, ps == HISQ_F64 ? 0.0 : delta2);
    // r_hi = b - A x0
    if (o.zero_guess) {
        HISQ_CUDA(ctx, cudaMemcpyAsync(w.rhi, w.b64, vb, cudaMemcpyDeviceToDevice, st));
        k_norm_f64<<<g, kVecBlock, 0, st>>>(VecRef{w.rhi, w.rb64}, w.len(), w.red(FIN_STORE, w.nblk_vec));
    } else if ((rc = precise_residual(ctx, w, m, st, w.pp))) {
        return rc;
    }
    k_scalars<<<1, 64, 0, st>>>(w.sc, nrhs, SC_INIT_R, tol2, delta2);
    dispatch(w.pv, [&](auto T) {
        decltype(T)::from_hi(w, w.r, st);
        decltype(T)::from_hi(w, w.p, st);
    });
    HISQ_CUDA(ctx, cudaGetLastError());

    // before any capture: the shape (timed on the solver's buffers the first time)
    w.shape = dslash_shape(ctx, ps, w.pv, nrhs, w.p, w.t, w.rbS, st);
    w.fused = o.single_reduction != 0;
    const int pds = persistent_ds(ctx, w, o, shifts != nullptr);
    const long per_it = w.fused ? 3 : 4; // launches per iteration
    L2Residency l2res;
    const cudaAccessPolicyWindow win = link_window(ctx, ps, o.l2_persist, l2res);
    set_stream_window(st, win);
    l2res.st = st;
    l2res.window = win.num_bytes > 0;
    const int ci = std::max(1, o.check_interval);
    const int interval = ps == HISQ_F64 ? (1 << 30) : std::max(1, o.reliable_interval);
    const bool prof = o.profile != 0;
    if (prof && (int)w.prof.size() < 4) {
        for (int i = (int)w.prof.size(); i < 4; i++) {
            cudaEvent_t e;
            HISQ_CUDA(ctx, cudaEventCreate(&e));
            w.prof.push_back(e);
        }
        if (w.graph) { cudaGraphExecDestroy(w.graph); w.graph = nullptr; }
    }
    int since_ru = 0, nru = 0, prev_iters = 0, it_all = 0;
    long kernels = 6 + (o.zero_guess ? 0 : 3); // setup: norms, scalars, conversions (+ residual)
    long dcalls = 0;
    double dms = 0.0, pms = 0.0;
    long dtimed = 0, piters = 0, plaunch = 0;
    bool done = false;
    rc = read_scalars(ctx, w, st);
    if (rc) return rc;
    {
        bool any = false;
        for (int r = 0; r < nrhs; r++) any |= w.h_sc[r].active != 0;
        done = !any;
        it_all = w.h_sc[0].it_all;
    }
    const int it_start = it_all;
    // reliable update: x_hi += x_lo, r_hi = b - A_precise x_hi, scalars, r = sloppy(r_hi)
    auto queue_ru = [&]() -> int {
        dispatch(w.pv, [&](auto T) { decltype(T)::accum_hi(w, st); });
        int e = precise_residual(ctx, w, m, st, w.pp);
        if (e) return e;
        k_scalars<<<1, 64, 0, st>>>(w.sc, nrhs, SC_RU, tol2, delta2);
        dispatch(w.pv, [&](auto T) { decltype(T)::from_hi(w, w.r, st); });
        kernels += 5 + (w.pp == HISQ_F64X ? 1 : 0);
        return HISQ_OK;
    };
    // certify a solve the float-pair operator found converged with the FP64 operator
    auto certify = [&](bool &any) -> int {
        int e = precise_residual(ctx, w, m, st, HISQ_F64);
        if (e) return e;
        k_scalars<<<1, 64, 0, st>>>(w.sc, nrhs, SC_RU, tol2, delta2);
        dispatch(w.pv, [&](auto T) { decltype(T)::from_hi(w, w.r, st); });
        kernels += 5;
        if ((e = read_scalars(ctx, w, st))) return e;
        for (int r = 0; r < nrhs; r++) any |= w.h_sc[r].active != 0;
        return HISQ_OK;
    };
    if (pds && !done && o.maxiter > 0) {
        // Persistent phases, pipelined: every phase ends in a reliable update, and the next
        // phase (which starts with the re-orthogonalisation of p) is queued behind that
        // update's read-back of the scalars before the host looks at them, so the GPU does
        // not wait for the host between phases.  The device bounds each phase itself (the reliable
        // interval, the iteration budget it_end, convergence), so the phase queued after the
        // last update runs no iteration; only the next reliable update waits for the host.
        const int it_end = it_start + o.maxiter;
        int slot = 0;           // pair of timing events of the phase being queued
        bool need_phase = true; // no phase is queued behind the last update
        bool first = true;
        auto queue_phase = [&](bool reortho) -> int {
            if (prof) HISQ_CUDA(ctx, cudaEventRecord(w.prof[2 * slot], st));
            int e = launch_persistent_phase(ctx, w, m, interval, it_end, pds, reortho ? 1 : 0,
                                            first ? o.selftest_wait : 0, st);
            if (e) return e;
            if (prof) HISQ_CUDA(ctx, cudaEventRecord(w.prof[2 * slot + 1], st));
            kernels++;
            first = false;
            return HISQ_OK;
        };
        for (;;) {
            if (need_phase && (rc = queue_phase(!first))) return rc;
            const int done_slot = slot;
            if ((rc = queue_ru())) return rc;
            HISQ_CUDA(ctx, cudaMemcpyAsync(w.h_sc, w.sc, sizeof(Scalars) * w.nrhs, cudaMemcpyDeviceToHost, st));
            HISQ_CUDA(ctx, cudaMemcpyAsync(w.h_status, ctx->status, sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
            HISQ_CUDA(ctx, cudaEventRecord(w.ev_sc, st));
            slot ^= 1;
            if ((rc = queue_phase(true))) return rc; // the next phase, before the host decides
            HISQ_CUDA(ctx, cudaEventSynchronize(w.ev_sc));
            if (w.h_status->error) {
                cudaStreamSynchronize(st);
                cudaMemsetAsync(ctx->status, 0, sizeof(DevStatus), st);
                cudaStreamSynchronize(st);
                return set_error(ctx, HISQ_EDEVICE, "a grid-barrier wait of the persistent CG kernel ran out");
            }
            const int executed = w.h_sc[0].it_all - it_all;
            it_all = w.h_sc[0].it_all;
            if (prof) {
                float ms = 0.f;
                if (cudaEventElapsedTime(&ms, w.prof[2 * done_slot], w.prof[2 * done_slot + 1]) == cudaSuccess) {
                    pms += ms;
                    piters += executed;
                    plaunch++;
                }
            }
            const int it = w.h_sc[0].iters;
            dcalls += 2L * (it - prev_iters);
            prev_iters = it;
            nru++;
            bool any = w.h_sc[0].active != 0;
            const bool last = it_all - it_start >= o.maxiter;
            need_phase = false;
            if (!any && w.pp != HISQ_F64 && ctx->links[HISQ_F64].built) {
                // the queued phase has run no iteration (nothing was active); if the FP64
                // residual is above the tolerance the solve goes on with a fresh phase
                if ((rc = certify(any))) return rc;
                need_phase = true;
            }
            if (!any || last) break;
        }
        done = true;
    }
    // Phases of the multi-kernel loop: a phase runs iterations until every right-hand side
    // pauses or converges, or until its cap (the next scheduled reliable update, maxiter, or
    // check_interval for direct launches); then the host looks at the scalars once.
    while (!done) {
        const int budget = o.maxiter - (it_all - it_start);
        if (budget <= 0) break;
        int cap = std::min(interval - since_ru, budget);
        if (!o.use_graph) cap = std::min(cap, ci);
        // Sampled timing (multi-kernel loop): the phase's first two iterations run as direct
        // launches and the second one's Dslash pair is timed; queued behind the first, its
        // launches start back to back on the GPU, so the events hold no host launch gaps.
        // Taken only when the phase may run three or more iterations; kept only if both did
        // work.
        const bool sample = prof && cap >= 3;
        if (o.use_graph) {
            k_phase_begin<<<1, 1, 0, st>>>(w.ctl, w.sc, cap);
            kernels++;
            if (sample) {
                if ((rc = launch_iteration(ctx, w, m, st, nullptr, 0))) return rc;
                if ((rc = launch_iteration(ctx, w, m, st, &w.prof[0], 0))) return rc;
                kernels += 2 * per_it;
            }
            if (!w.graph || w.graph_m != m || w.graph_l2 != (win.num_bytes > 0) || w.graph_shift != w.shift_key ||
                w.graph_fused != w.fused) {
                if (w.graph) { cudaGraphExecDestroy(w.graph); w.graph = nullptr; }
                if ((rc = build_loop_graph(ctx, w, m, win, st))) return rc;
                w.graph_m = m;
                w.graph_shift = w.shift_key;
                w.graph_l2 = win.num_bytes > 0;
                w.graph_fused = w.fused;
            }
            HISQ_CUDA(ctx, cudaGraphLaunch(w.graph, st));
        } else {
            k_phase_begin<<<1, 1, 0, st>>>(w.ctl, w.sc, cap);
            kernels++;
            for (int i = 0; i < cap; i++)
                if ((rc = launch_iteration(ctx, w, m, st, (sample && i == 1) ? &w.prof[0] : nullptr, 0))) return rc;
        }
        if ((rc = read_scalars(ctx, w, st))) return rc;
        const int executed = w.h_sc[0].it_all - it_all; // iterations the device ran in this phase
        it_all = w.h_sc[0].it_all;
        since_ru += executed;
        kernels += per_it * executed - (o.use_graph && sample ? 2 * per_it : 0);
        int it = 0;
        bool any_active = false, any_flag = false;
        for (int r = 0; r < nrhs; r++) {
            it = std::max(it, w.h_sc[r].iters);
            any_active |= w.h_sc[r].active != 0;
            any_flag |= w.h_sc[r].flag != 0;
        }
        const int ran = it - prev_iters; // iterations that did work
        prev_iters = it;
        dcalls += 2L * ran;
        if (sample && ran >= 2) {
            for (int j = 0; j < 2; j++) {
                float ms = 0.f;
                if (cudaEventElapsedTime(&ms, w.prof[2 * j], w.prof[2 * j + 1]) == cudaSuccess) {
                    dms += ms;
                    dtimed++;
                }
            }
        }
        const bool last = it_all - it_start >= o.maxiter;
        if (any_flag || since_ru >= interval || !any_active || last) {
            if ((rc = queue_ru())) return rc;
            if ((rc = read_scalars(ctx, w, st))) return rc;
            nru++;
            since_ru = 0;
            bool any = false;
            for (int r = 0; r < nrhs; r++) any |= w.h_sc[r].active != 0;
            // converged by the float-pair operator: certify with the FP64 operator
            if (!any && w.pp != HISQ_F64 && ctx->links[HISQ_F64].built && (rc = certify(any))) return rc;
            if (!any || last) break;
            dispatch(w.pv, [&](auto T) { decltype(T)::reortho(w, st); });
            kernels += 2;
            continue;
        }
        // the phase ended at its cap with p not yet updated
        dispatch(w.pv, [&](auto T) { decltype(T)::update_xp(w, 2, st); });
        kernels++;
    }
    // every exit from the loop follows a reliable update (or no iteration at all), so
    // x_hi holds the whole solution and Scalars.rr its recomputed residual
    HISQ_CUDA(ctx, cudaGetLastError());
    const cudaMemcpyKind k_out = o.host_buffers ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    HISQ_CUDA(ctx, cudaMemcpyAsync(x, w.x64, vb, k_out, st));
    if ((rc = read_scalars(ctx, w, st))) return rc;
    // later work on the caller's stream is ordered after the solve
    HISQ_CUDA(ctx, cudaEventRecord(w.ev, st));
    HISQ_CUDA(ctx, cudaStreamWaitEvent(ust, w.ev, 0));
    double worst = 0.0, worst_it = 0.0;
    bool ok = true;
    int iters = 0;
    for (int r = 0; r < nrhs; r++) {
        const Scalars &S = w.h_sc[r];
        const double res = S.bb > 0 ? std::sqrt(S.rr / S.bb) : 0.0;
        if (residuals) residuals[r] = res;
        worst = std::max(worst, res);
        worst_it = std::max(worst_it, res);
        iters = std::max(iters, S.iters);
        if (S.bad || !(res <= o.tol)) ok = false;
    }
    if (stats) {
        stats->iterations = iters;
        stats->reliable_updates = nru;
        stats->true_residual = worst;
        stats->iterated_residual = worst_it;
        stats->seconds = wall() - t0;
        stats->dslash_calls = dcalls + 2L * (nru + (o.zero_guess ? 0 : 1));
        stats->dslash_ms = dms;
        stats->dslash_timed = dtimed;
        const LinkStore &L = ctx->links[ps];
        const double dsl = (double)w.Vh * (16.0 * link_bytes(ps, L.nreal) + 2.0 * nrhs * spinor_bytes(w.pv));
        stats->bytes_moved = 2.0 * iters * dsl;
        stats->kernels = kernels;
        stats->phase_ms = pms;
        stats->phase_iterations = piters;
        stats->phase_launches = plaunch;
        stats->persistent_ds = pds;
    }
    if (!ok) return set_error(ctx, HISQ_ENOTCONVERGED, "hisq_cg: tolerance not reached");
    return HISQ_OK;
}

}  // namespace hisq

using namespace hisq;

extern "C" {

void hisq_solve_opts_default(hisq_solve_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->tol = 1e-10;
    o->maxiter = 100000;
    o->prec_sloppy = HISQ_F64;
    o->prec_precise = HISQ_F64;
    o->reliable_interval = 100;
    o->reliable_delta = 0.1;
    o->zero_guess = 1;
    o->check_interval = 50;
    o->single_reduction = 0;
    o->use_graph = 1;
    o->l2_persist = -1;
    o->persistent = -1;
}

int hisq_cg(hisq_ctx *ctx, double m, const double *b, double *x, int nrhs, const hisq_solve_opts *opts,
            hisq_stats *stats, double *residuals)
{
    if (!ctx) return HISQ_EINVAL;
    if (!b || !x || nrhs < 1 || nrhs > 64 || !(m >= 0.0)) return set_error(ctx, HISQ_EINVAL, "hisq_cg: bad argument");
    hisq_solve_opts o;
    if (opts) o = *opts;
    else hisq_solve_opts_default(&o);
    if (!(o.tol > 0.0) || o.maxiter < 1) return set_error(ctx, HISQ_EINVAL, "hisq_cg: bad tolerance or maxiter");
    if (stats) std::memset(stats, 0, sizeof(*stats));
    cudaSetDevice(ctx->device);
    return run_cg(ctx, m, b, x, nrhs, o, stats, residuals, nullptr);
}

}  // extern "C"
